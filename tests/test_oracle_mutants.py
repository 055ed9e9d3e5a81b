"""The pins earn their place: a copy of the oracle's C source with one planted
mistake (built on the CPU, in a temporary directory) fails the pins named
beside the mistake, while an unmodified copy passes the same pins.  Each
mistake is a plausible slip in the passage it touches: a wrong weight, a
dropped factor, a reversed sign, an off-by-one index."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what, original line of oracle/nlse_oracle.c, planted mistake, pins that must fail (pytest -k))
MUTANTS = [
    ("1D step 2: centre weight 7/6 -> 8/6",
     "return c_sub(c_scale(7.0 / 6.0, get(D, p)), c_scale(1.0 / 12.0, nb));",
     "return c_sub(c_scale(8.0 / 6.0, get(D, p)), c_scale(1.0 / 12.0, nb));",
     "noncompact"),
    ("2D step 2: centre weight 12 -> 11",
     "cplx dpart = c_scale(-1.0 / 12.0, c_sub(dsum, c_scale(12.0, get(D, p))));",
     "cplx dpart = c_scale(-1.0 / 12.0, c_sub(dsum, c_scale(11.0, get(D, p))));",
     "noncompact"),
    ("3D step 2: centre weight 10 -> 9",
     "cplx dpart = c_scale(-1.0 / 12.0, c_sub(dsum, c_scale(10.0, get(D, p))));",
     "cplx dpart = c_scale(-1.0 / 12.0, c_sub(dsum, c_scale(9.0, get(D, p))));",
     "noncompact"),
    ("3D step 2: edge term weight 1/(6h^2) -> 1/(4h^2)",
     "cplx ppart = c_scale(1.0 / (6.0 * P->h * P->h), c_sub(edges, c_scale(12.0, get(psi, p))));",
     "cplx ppart = c_scale(1.0 / (4.0 * P->h * P->h), c_sub(edges, c_scale(12.0, get(psi, p))));",
     "noncompact"),
    ("Dirichlet D_b without its 1/a",
     "if (P->bc == 0) return c_scale(-Nb / P->a, pb);",
     "if (P->bc == 0) return c_scale(-Nb, pb);",
     "general_a"),
    ("N with the sign of V reversed",
     "return P->s * c_abs2(psi) - V;",
     "return P->s * c_abs2(psi) + V;",
     "general_a"),
    ("RK4: K_2 weighted 1 instead of 2",
     "for (p = 0; p < N; ++p) put(Ktot, p, c_add(get(Ktot, p), c_scale(2.0, get(Ktmp, p))));    /* 4 */",
     "for (p = 0; p < N; ++p) put(Ktot, p, c_add(get(Ktot, p), c_scale(1.0, get(Ktmp, p))));    /* 4 */",
     "stability_polynomial"),
    ("MSD inward point one too far on the upper side",
     "if (v > n - 2) return n - 2;",
     "if (v > n - 3) return n - 3;",
     "symmetries"),
    ("Laplacian-zero F_b without the nonlinearity",
     "put(F, b, c_times_i(c_scale(nonlin(P, pb, V[b]), pb)));",
     "put(F, b, c_make(0.0, 0.0));",
     "laplacian_zero"),
    ("periodic wrap with period n - 1",
     "x = (x % P->n[0] + P->n[0]) % P->n[0];",
     "x = (x % (P->n[0] - 1) + P->n[0] - 1) % (P->n[0] - 1);",
     "periodic"),
    ("stability bound: G entries in units of 1/6",
     "double d = fabs(L - G[g] / 12.0);",
     "double d = fabs(L - G[g] / 6.0);",
     "linear_stability_bound"),
    ("energy: quartic term without its 1/2",
     "- 0.5 * P.s * rho * rho",
     "- P.s * rho * rho",
     "mass_and_energy"),
]


def _copy_tree(dst):
    """The oracle and what the pins import, under dst."""
    ign = shutil.ignore_patterns("_build", "__pycache__")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    os.makedirs(os.path.join(dst, "paper_1109_1027_gb300"))
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_1109_1027_gb300", f), os.path.join(dst, "paper_1109_1027_gb300", f))
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("conftest.py", "test_oracle_pins.py", "paper_experiments.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"), ignore=ign)


def _run_pins(root, kexpr):
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-k", kexpr,
                        os.path.join("tests", "test_oracle_pins.py")],
                       cwd=root, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout + r.stderr


@pytest.mark.parametrize("what,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pins(what, old, new, pins, tmp_path):
    _copy_tree(str(tmp_path))
    src = os.path.join(str(tmp_path), "oracle", "nlse_oracle.c")
    with open(src) as f:
        text = f.read()
    assert text.count(old) == 1, what
    with open(src, "w") as f:
        f.write(text.replace(old, new))
    rc, out = _run_pins(str(tmp_path), pins)
    assert rc == 1, (what, out[-3000:])          # 1: tests ran and failed (5 would be: none selected)


def test_unmodified_copy_passes_the_same_pins(tmp_path):
    _copy_tree(str(tmp_path))
    kexpr = " or ".join(sorted({m[3] for m in MUTANTS}))
    rc, out = _run_pins(str(tmp_path), kexpr)
    assert rc == 0, out[-3000:]
