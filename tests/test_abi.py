"""The C ABI without a GPU: the library builds for sm_103a, loads, exports
every entry point that include/nlse.h declares, and rejects invalid
parameters on the host before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_1109_1027_gb300 import build as nbuild
from paper_1109_1027_gb300 import nlse

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = []
    for fname in sorted(os.listdir(HEADER_DIR)):
        if not fname.endswith(".h"):
            continue
        with open(os.path.join(HEADER_DIR, fname)) as f:
            text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(nlse_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return nlse.load_library()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("nlse_create", "nlse_lap2shoc", "nlse_rk4_step", "nlse_run",
                     "nlse_invariants", "nlse_destroy", "nlse_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def _params(**kw):
    base = dict(shape=(16, 16), h=0.1, dt=1e-3, a=1.0, s=1.0)
    base.update(kw)
    shape = base.pop("shape")
    stack = base.pop("stack", 0)
    p = nlse.make_params(shape, **base)
    if stack:
        p.n[2] = stack
        p.flags |= nlse.FLAG_STACK
    return p


@pytest.mark.parametrize("kw,code", [
    (dict(shape=(2, 16)), nlse.EINVAL),               # n < 3
    (dict(h=0.0), nlse.EINVAL),
    (dict(h=float("nan")), nlse.EINVAL),
    (dict(dt=-1.0), nlse.EINVAL),
    (dict(a=0.0), nlse.EINVAL),                       # a > 0 (Eq. NLSE)
    (dict(s=float("inf")), nlse.EINVAL),
    (dict(bc=5), nlse.EINVAL),
    (dict(prec=7), nlse.EINVAL),
    (dict(lap=3), nlse.EINVAL),
    (dict(bc="msd", lap="2shoc_ms"), nlse.EUNSUPPORTED),     # no MSD rule for the multi-storage form
    (dict(bc="periodic", lap="2shoc_ms"), nlse.EUNSUPPORTED),
    (dict(bc="lapzero", lap="2shoc_ms"), nlse.EUNSUPPORTED),
    (dict(shape=(8, 8, 8), stack=2), nlse.EINVAL),          # stacks are of 2D grids
    (dict(bc="msd", stack=2), nlse.EUNSUPPORTED),
    (dict(plain=True, stack=2), nlse.EUNSUPPORTED),
    (dict(lap="2shoc_ms", plain=True), nlse.EUNSUPPORTED),   # unfused schedule: single storage only
])
def test_invalid_parameters_are_rejected_on_the_host(lib, kw, code):
    ctx = ctypes.c_void_p()
    rc = lib.nlse_create(ctypes.byref(_params(**kw)), ctypes.c_void_p(4096), ctypes.byref(ctx))
    assert rc == code
    assert ctx.value is None
    assert lib.nlse_last_error().decode()


def test_dimension_out_of_range(lib):
    p = _params()
    p.dim = 4
    ctx = ctypes.c_void_p()
    assert lib.nlse_create(ctypes.byref(p), ctypes.c_void_p(4096), ctypes.byref(ctx)) == nlse.EINVAL


def test_null_arguments(lib):
    ctx = ctypes.c_void_p()
    assert lib.nlse_create(None, ctypes.c_void_p(4096), ctypes.byref(ctx)) == nlse.EINVAL
    assert lib.nlse_create(ctypes.byref(_params()), None, ctypes.byref(ctx)) == nlse.EINVAL
    assert lib.nlse_rk4_step(None, ctypes.c_void_p(4096), None) == nlse.EINVAL
    assert lib.nlse_run(None, ctypes.c_void_p(4096), 1, None) == nlse.EINVAL
    assert lib.nlse_lap2shoc(None, None, None, None) == nlse.EINVAL


def test_misaligned_potential_is_rejected(lib):
    ctx = ctypes.c_void_p()
    rc = lib.nlse_create(ctypes.byref(_params()), ctypes.c_void_p(4100), ctypes.byref(ctx))
    assert rc == nlse.EINVAL


def test_batch_validation_on_the_host(lib):
    ctx = ctypes.c_void_p()
    bad = [_params(shape=(16, 16)), _params(shape=(8, 10))]        # width not a multiple of 4
    arr = (nlse.Params * 2)(*bad)
    assert lib.nlse_create_batch(2, arr, ctypes.c_void_p(4096), ctypes.byref(ctx)) == nlse.EUNSUPPORTED
    mixed = [_params(shape=(16, 16)), _params(shape=(8, 12), prec="fp64")]
    arr = (nlse.Params * 2)(*mixed)
    assert lib.nlse_create_batch(2, arr, ctypes.c_void_p(4096), ctypes.byref(ctx)) == nlse.EINVAL
    three_d = [_params(shape=(4, 16, 16))]
    arr = (nlse.Params * 1)(*three_d)
    assert lib.nlse_create_batch(1, arr, ctypes.c_void_p(4096), ctypes.byref(ctx)) == nlse.EUNSUPPORTED
    assert lib.nlse_create_batch(0, arr, ctypes.c_void_p(4096), ctypes.byref(ctx)) == nlse.EINVAL
    assert ctx.value is None


def _header_constants():
    """#define values and enum members of include/nlse.h, by name."""
    with open(os.path.join(HEADER_DIR, "nlse.h")) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    consts = {m[0]: int(m[1]) for m in re.findall(r"#define\s+(NLSE_\w+)\s+(\d+)u?\b", text)}
    consts.update({m[0]: int(m[1]) for m in re.findall(r"\b(NLSE_\w+)\s*=\s*(\d+)", text)})
    return consts


def test_binding_constants_match_the_header():
    """The Python binding's status codes, enums, flags and tiling keys are the
    header's values (marshalling only: a mismatch would pass the wrong
    boundary, precision or schedule to the library)."""
    h = _header_constants()
    statuses = ["NLSE_OK", "NLSE_EINVAL", "NLSE_ENOMEM", "NLSE_ECUDA", "NLSE_EUNSTABLE", "NLSE_ENONFINITE",
                "NLSE_ETIMEOUT", "NLSE_EUNSUPPORTED", "NLSE_EBOUNDS"]
    assert [h[n] for n in statuses] == [nlse.OK, nlse.EINVAL, nlse.ENOMEM, nlse.ECUDA, nlse.EUNSTABLE,
                                        nlse.ENONFINITE, nlse.ETIMEOUT, nlse.EUNSUPPORTED, nlse.EBOUNDS]
    assert {k: h["NLSE_BC_" + {"lapzero": "LAPZERO"}.get(k, k.upper())] for k in nlse.BC} == nlse.BC
    assert {k: h["NLSE_" + k.upper()] for k in nlse.PREC} == nlse.PREC
    assert {k: h["NLSE_LAP_" + k.upper()] for k in nlse.LAP} == nlse.LAP
    assert h["NLSE_FLAG_NO_STABILITY_CHECK"] == nlse.FLAG_NO_STABILITY_CHECK
    assert h["NLSE_FLAG_PLAIN_SCHEDULE"] == nlse.FLAG_PLAIN_SCHEDULE
    assert h["NLSE_FLAG_STACK"] == nlse.FLAG_STACK
    for key in ("ROWS", "PLANES", "BATCH_NARROW", "1D_RESIDENT", "2D_FUSE", "ADJ_ROWS"):
        assert h["NLSE_TILE_" + key] == getattr(nlse, "TILE_" + key), key


def test_every_entry_point_cites_its_passage():
    """Each declaration in include/nlse.h is preceded by a comment that cites
    the passage of the paper defining the operation (Sec., Eq., Table) or says
    that the paper has no counterpart, and states its errors or result."""
    with open(os.path.join(HEADER_DIR, "nlse.h")) as f:
        text = f.read()
    decls = list(re.finditer(r"(/\*(?:[^*]|\*(?!/))*\*/)\s*((?:int|void|const char\*)\s+(nlse_\w+)\s*\([^;]*\);)",
                             text))
    found = {m.group(3) for m in decls}
    assert set(declared_functions()) <= found, set(declared_functions()) - found
    for m in decls:
        comment, name = re.sub(r"\s*\n\s*\*?\s*", " ", m.group(1)), m.group(3)   # one line of prose
        assert re.search(r"Sec\.|Eqs?\.|Table|no counterpart", comment, flags=re.I), name
