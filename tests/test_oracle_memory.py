"""The oracle's C code under AddressSanitizer: every entry point, each
boundary rule and Laplacian, 1D to 3D, on grids down to three points.  An
out-of-bounds access in the oracle would corrupt the test process's heap and
surface far from its cause, so it is checked here directly."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r'''
import sys
sys.path.insert(0, {root!r})
import oracle
oracle._libs.clear()
oracle.build = lambda threaded=False: {lib!r}
from paper_1109_1027_gb300 import workloads as wl
for shape in [(3,), (4,), (37,), (3, 3), (17, 12), (3, 3, 3), (6, 7, 8)]:
    psi = wl.random_field(shape, seed=1) + 2.5
    V = wl.random_potential(shape, seed=2)
    for bc in (oracle.BC_DIRICHLET, oracle.BC_MSD, oracle.BC_PERIODIC, oracle.BC_LAPZERO):
        for lap in (oracle.LAP_2SHOC, oracle.LAP_CD, oracle.LAP_2SHOC_MS):
            if bc in (oracle.BC_MSD, oracle.BC_LAPZERO) and lap == oracle.LAP_2SHOC_MS and len(shape) > 1:
                continue
            prob = oracle.Problem(shape, 0.3, 0.8, -1.0, bc=bc, lap=lap)
            oracle.laplacian(prob, psi, V, return_D=True)
            oracle.rhs(prob, psi, V)
            oracle.run(prob, psi, V, 1e-3, 2)
            oracle.invariants(prob, psi, V)
print("clean")
'''


def test_oracle_is_clean_under_address_sanitizer(tmp_path):
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not asan or not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("libasan not available")
    lib = str(tmp_path / "oracle_asan.so")
    subprocess.check_call(["gcc", "-std=c11", "-O1", "-g", "-fsanitize=address", "-fno-omit-frame-pointer",
                           "-ffp-contract=off", "-fPIC", "-shared", "-o", lib,
                           os.path.join(ROOT, "oracle", "nlse_oracle.c"), "-lm"])
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0")
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, lib=lib)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "clean" in r.stdout, r.stderr[-3000:]
