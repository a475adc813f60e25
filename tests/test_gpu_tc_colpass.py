"""The column pass on the tensor cores (csrc/tc_colpass.cu, switched on by
BEM_TC_COLUMN_PASS=1): the length-4096 column transform of Eq. 13 as four
64-point DFT products in split BF16 (six products per term) on tcgen05.  Its
transform must meet the FP32 transform's parity bar against the oracle's
direct sum of Eq. 7: 2e-6 of the maximum on a whole 64 x 1100 field (a 128 x
4096 torus, square elements), and 5e-6 on 64 sampled outputs of a 2048^2
field, as the FFT column pass does in test_gpu_parity.py.  Run in a child process because the
switch is read once per process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASE = r"""
import json, sys
import numpy as np
sys.path.insert(0, %r)
from paper_1612_08395_gb300 import build, bem
build.build()
nx, ny, dx, k, p_path, out_path = %r
p = np.load(p_path)
with bem.Handle(nx, ny, dx, dx, k, 0.3) as h:
    assert h.info().Py == 4096
    u = h.convolve(p, "fp32")
np.save(out_path, u)
"""


def run_tc(nx, ny, dx, k, p, tmp_path):
    np.save(tmp_path / "p.npy", p)
    out = tmp_path / "u.npy"
    env = dict(os.environ, BEM_TC_COLUMN_PASS="1")
    r = subprocess.run([sys.executable, "-c", CASE % (ROOT, (nx, ny, dx, k, str(tmp_path / "p.npy"), str(out)))],
                       capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


@pytest.mark.parametrize("k", [0.4, -0.5])
def test_tc_column_pass_whole_field(oracle_mod, cuda_ok, tmp_path, k):
    nx, ny = 64, 1100
    dx = 1.0 / ny  # square elements
    p = I.random_pressure(nx, ny, seed=21, density=0.7)
    u = run_tc(nx, ny, dx, k, p, tmp_path)
    Kq = oracle_mod.influence_quarter(k, dx, dx, nx, ny)
    uo = oracle_mod.compliance(k, 0.3) * oracle_mod.convolve_direct(Kq, p)
    assert np.abs(u - uo).max() <= 2e-6 * np.abs(uo).max()


def test_tc_column_pass_2048_sampled(oracle_mod, cuda_ok, tmp_path):
    n, k = 2048, 0.3
    dx = 1.0 / n
    p = np.maximum(0.0, 1.0 - (I.radius_grid(n, n, dx) / 0.3) ** 2) \
        + 0.1 * I.random_pressure(n, n, seed=7, density=0.01)
    u = run_tc(n, n, dx, k, p, tmp_path).ravel()
    rng = np.random.Generator(np.random.PCG64(3))
    idx = np.concatenate([rng.integers(0, n * n, 60), [0, n - 1, n * n - 1, n * (n // 2) + n // 2]])
    Kq = oracle_mod.influence_quarter(k, dx, dx, n, n)
    uo = oracle_mod.compliance(k, 0.3) * oracle_mod.convolve_direct_at(Kq, p, idx)
    assert np.abs(u[idx] - uo).max() <= 5e-6 * np.abs(uo).max()
