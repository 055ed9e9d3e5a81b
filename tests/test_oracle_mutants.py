"""The pins earn their place: a copy of the oracle (its C source or the
reference adjoint) with one planted mistake, built on the CPU in a temporary
directory, fails the pins named beside the mistake, while an unmodified copy
passes the same pins.  Each mistake is a plausible slip in the passage it
touches: a wrong weight, a dropped factor, a reversed sign, an off-by-one
index, a wrong part of a complex number."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C, PINS = "nlse_oracle.c", "test_oracle_pins.py"
ADJ, ADJ_PINS = "adjoint.py", "test_oracle_adjoint.py"

# (what, oracle file, original text, planted mistake, pin file, pins that must fail (pytest -k))
MUTANTS = [
    ("1D step 2: centre weight 7/6 -> 8/6",
     C, "return c_sub(c_scale(7.0 / 6.0, get(D, p)), c_scale(1.0 / 12.0, nb));",
     "return c_sub(c_scale(8.0 / 6.0, get(D, p)), c_scale(1.0 / 12.0, nb));",
     PINS, "noncompact"),
    ("2D step 2: centre weight 12 -> 11",
     C, "cplx dpart = c_scale(-1.0 / 12.0, c_sub(dsum, c_scale(12.0, get(D, p))));",
     "cplx dpart = c_scale(-1.0 / 12.0, c_sub(dsum, c_scale(11.0, get(D, p))));",
     PINS, "noncompact"),
    ("3D step 2: centre weight 10 -> 9",
     C, "cplx dpart = c_scale(-1.0 / 12.0, c_sub(dsum, c_scale(10.0, get(D, p))));",
     "cplx dpart = c_scale(-1.0 / 12.0, c_sub(dsum, c_scale(9.0, get(D, p))));",
     PINS, "noncompact"),
    ("3D step 2: edge term weight 1/(6h^2) -> 1/(4h^2)",
     C, "cplx ppart = c_scale(1.0 / (6.0 * P->h * P->h), c_sub(edges, c_scale(12.0, get(psi, p))));",
     "cplx ppart = c_scale(1.0 / (4.0 * P->h * P->h), c_sub(edges, c_scale(12.0, get(psi, p))));",
     PINS, "noncompact"),
    ("Dirichlet D_b without its 1/a",
     C, "if (P->bc == 0) return c_scale(-Nb / P->a, pb);",
     "if (P->bc == 0) return c_scale(-Nb, pb);",
     PINS, "general_a"),
    ("N with the sign of V reversed",
     C, "return P->s * c_abs2(psi) - V;",
     "return P->s * c_abs2(psi) + V;",
     PINS, "general_a"),
    ("RK4: K_2 weighted 1 instead of 2",
     C, "    rhs(P, ptmp, V, Ktmp, work);                                              /* K_tmp = F(psi_tmp) */\n"
        "#pragma omp parallel for schedule(static)\n"
        "    for (p = 0; p < N; ++p) put(Ktot, p, c_add(get(Ktot, p), c_scale(2.0, get(Ktmp, p))));    /* K_tot += 2 K_tmp */\n"
        "#pragma omp parallel for schedule(static)\n"
        "    for (p = 0; p < N; ++p) put(ptmp, p, c_add(get(psi, p), c_scale(k / 2.0, get(Ktmp, p))));",
     "    rhs(P, ptmp, V, Ktmp, work);                                              /* K_tmp = F(psi_tmp) */\n"
        "#pragma omp parallel for schedule(static)\n"
        "    for (p = 0; p < N; ++p) put(Ktot, p, c_add(get(Ktot, p), c_scale(1.0, get(Ktmp, p))));    /* K_tot += 2 K_tmp */\n"
        "#pragma omp parallel for schedule(static)\n"
        "    for (p = 0; p < N; ++p) put(ptmp, p, c_add(get(psi, p), c_scale(k / 2.0, get(Ktmp, p))));",
     PINS, "stability_polynomial"),
    ("MSD inward point one too far on the upper side",
     C, "if (v > n - 2) return n - 2;",
     "if (v > n - 3) return n - 3;",
     PINS, "symmetries"),
    ("Laplacian-zero F_b without the nonlinearity",
     C, "put(F, b, c_times_i(c_scale(nonlin(P, pb, V[b]), pb)));",
     "put(F, b, c_make(0.0, 0.0));",
     PINS, "laplacian_zero"),
    ("periodic wrap with period n - 1",
     C, "x = (x % P->n[0] + P->n[0]) % P->n[0];",
     "x = (x % (P->n[0] - 1) + P->n[0] - 1) % (P->n[0] - 1);",
     PINS, "periodic"),
    ("stability bound: G entries in units of 1/6",
     C, "double d = fabs(L - G[g] / 12.0);",
     "double d = fabs(L - G[g] / 6.0);",
     PINS, "linear_stability_bound"),
    ("energy: quartic term without its 1/2",
     C, "- 0.5 * P.s * rho * rho",
     "- P.s * rho * rho",
     PINS, "mass_and_energy"),
    ("multi storage: boundary split adds the other axes instead of subtracting them",
     C, "rest = c_sub(rest, d);",
     "rest = c_add(rest, d);",
     PINS, "multi_storage_boundary_split"),
    ("RK4: second stage input at k instead of k/2",
     C, "put(ptmp, p, c_add(get(psi, p), c_scale(k / 2.0, get(Ktot, p))));  /* psi_tmp */",
     "put(ptmp, p, c_add(get(psi, p), c_scale(k, get(Ktot, p))));  /* psi_tmp */",
     PINS, "stability_polynomial"),
    ("RK4: final weight k/6 -> k/3",
     C, "put(psi, p, c_add(get(psi, p), c_scale(k / 6.0, c_add(get(Ktot, p), get(Ktmp, p)))));",
     "put(psi, p, c_add(get(psi, p), c_scale(k / 3.0, c_add(get(Ktot, p), get(Ktmp, p)))));",
     PINS, "stability_polynomial"),
    ("MSD F_b from the real part of F/psi",
     C, "double w = c_div(get(F, q), get(psi, q)).im;",
     "double w = c_div(get(F, q), get(psi, q)).re;",
     PINS, "msd_plane_wave"),
    ("MSD D_b from Re(i z) instead of Im(i z)",
     C, "double factor = c_times_i(ratio).im + (Nq - Nb) / P->a;",
     "double factor = c_times_i(ratio).re + (Nq - Nb) / P->a;",
     PINS, "plane_wave_symbol_and_msd"),
    ("CD computed with the 2SHOC step 2",
     C, "if (is_boundary(P, x, y, z) || P->lap == 1)",
     "if (is_boundary(P, x, y, z))",
     PINS, "cd_laplacian"),
    ("mass without the cell volume h^d",
     C, "*mass = hd * m;",
     "*mass = m;",
     PINS, "mass_and_energy"),
    ("adjoint: transposed step 2 with the neighbour sign reversed",
     ADJ, "E = (16 - 2 * d) / 12 * u - _axial_sum(u) / 12",
     "E = (16 - 2 * d) / 12 * u + _axial_sum(u) / 12",
     ADJ_PINS, "rhs_vjp"),
    ("adjoint: conjugate term of the boundary derivative with the wrong sign",
     ADJ, "beta = -s * Y * Y / a",
     "beta = s * Y * Y / a",
     ADJ_PINS, "rhs_vjp"),
    ("adjoint: stage-3 cotangent weighted k/2 instead of k",
     ADJ, "Kb[2] = Kb[2] + k * Yb4",
     "Kb[2] = Kb[2] + k / 2 * Yb4",
     ADJ_PINS, "loss_gradient"),
]


def _copy_tree(dst):
    """The oracle and what the pins import, under dst."""
    ign = shutil.ignore_patterns("_build", "__pycache__")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    os.makedirs(os.path.join(dst, "paper_1109_1027_gb300"))
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_1109_1027_gb300", f), os.path.join(dst, "paper_1109_1027_gb300", f))
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("conftest.py", PINS, ADJ_PINS, "paper_experiments.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"), ignore=ign)


def _run_pins(root, pin_file, kexpr):
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-k", kexpr,
                        os.path.join("tests", pin_file)],
                       cwd=root, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout + r.stderr


@pytest.mark.parametrize("what,fname,old,new,pin_file,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pins(what, fname, old, new, pin_file, pins, tmp_path):
    _copy_tree(str(tmp_path))
    src = os.path.join(str(tmp_path), "oracle", fname)
    with open(src) as f:
        text = f.read()
    assert text.count(old) == 1, what
    with open(src, "w") as f:
        f.write(text.replace(old, new))
    rc, out = _run_pins(str(tmp_path), pin_file, pins)
    assert rc == 1, (what, out[-3000:])          # 1: tests ran and failed (5 would be: none selected)


@pytest.mark.parametrize("pin_file", [PINS, ADJ_PINS])
def test_unmodified_copy_passes_the_same_pins(pin_file, tmp_path):
    _copy_tree(str(tmp_path))
    kexpr = " or ".join(sorted({m[5] for m in MUTANTS if m[4] == pin_file}))
    rc, out = _run_pins(str(tmp_path), pin_file, kexpr)
    assert rc == 0, out[-3000:]
