"""Host logic of the launch-shape autotuner (no GPU): which tiling keys it
times for which context, and how it keys its cache."""
from types import SimpleNamespace

from paper_1109_1027_gb300 import autotune
from paper_1109_1027_gb300 import nlse


def _solver(shape, prec="fp32", bc="dirichlet", lap="2shoc", flags=0, stack=1):
    n = list(shape[::-1]) + [1] * (3 - len(shape))
    if stack > 1:
        n[2] = stack
    params = SimpleNamespace(dim=len(shape), prec=0 if prec == "fp32" else 1, bc=nlse.BC[bc],
                             lap=nlse.LAP[lap], flags=flags, n=n)
    return SimpleNamespace(shape=shape, prec=prec, params=params)


def test_2d_fp32_dirichlet_times_rows_then_two_stages_per_launch():
    for lap in ("2shoc", "cd"):
        assert autotune._keys_for(_solver((512, 512), lap=lap)) == [nlse.TILE_ROWS, nlse.TILE_2D_FUSE]
    stack = _solver((64, 128), flags=nlse.FLAG_STACK, stack=8)
    assert autotune._keys_for(stack) == [nlse.TILE_ROWS, nlse.TILE_2D_FUSE]


def test_contexts_without_the_fused_kernels_time_rows_only():
    for kw in ({"prec": "fp64"}, {"lap": "2shoc_ms"}, {"bc": "msd"}, {"bc": "periodic"},
               {"flags": nlse.FLAG_PLAIN_SCHEDULE}):
        assert autotune._keys_for(_solver((512, 512), **kw)) == [nlse.TILE_ROWS], kw


def test_other_dimensions():
    assert autotune._keys_for(_solver((2048,))) == [nlse.TILE_1D_RESIDENT]
    assert autotune._keys_for(_solver((8192,))) == []
    assert autotune._keys_for(_solver((64, 64, 64))) == [nlse.TILE_PLANES]
    assert autotune._keys_for(_solver((64, 64, 64), prec="fp64")) == []


def test_every_key_has_candidates_and_the_defaults_among_them():
    assert set(autotune.CANDIDATES) == {nlse.TILE_ROWS, nlse.TILE_PLANES, nlse.TILE_BATCH_NARROW,
                                        nlse.TILE_1D_RESIDENT, nlse.TILE_2D_FUSE}
    assert 16 in autotune.CANDIDATES[nlse.TILE_ROWS]
    assert 32 in autotune.CANDIDATES[nlse.TILE_PLANES]
    assert 0 in autotune.CANDIDATES[nlse.TILE_2D_FUSE] and 1 in autotune.CANDIDATES[nlse.TILE_2D_FUSE]
