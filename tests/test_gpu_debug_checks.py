"""The bounds-checked debug build (BEM_DEBUG_CHECKS=1): solves that exercise
every pass and launch shape -- FP64 and FP32 row/column passes, the contact
band of the fixed-set loop, box sub-tori, a rectangular grid and a ragged
row count -- run with every check passing (a failed one is reported as an
error by the solver) and give the release build's results."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r"""
import json, sys
import numpy as np
sys.path.insert(0, %r)
from paper_1612_08395_gb300 import build
build.build(debug_checks=%r)
import paper_1612_08395_gb300.bem as bem
import paper_1612_08395_gb300.inputs as I
out = {}
# adhesive sweep, FP32: band and box sub-tori while unloading
n = 256
with bem.Handle(n, n, 1.0 / n, 1.0 / n, 0.3, 0.3) as h:
    res, rc = h.sweep(I.paraboloid(n), np.linspace(0.01, -0.02, 61), dgamma=1e-3, precision="fp32")
out["sweep32"] = [rc, [r.force for r in res], [r.contact_count for r in res]]
# rectangular grid with an odd row count, FP64 and FP32 with refinement
nx, ny = 96, 75
x = I.centres(nx, 1.0 / nx); y = I.centres(ny, 1.0 / nx)
X, Y = np.meshgrid(x, y)
prof = np.ascontiguousarray((X ** 2 + Y ** 2) / 2.0)
for prec in ("fp64", "fp32_refine"):
    p = np.empty((ny, nx))
    with bem.Handle(nx, ny, 1.0 / nx, 1.0 / nx, -0.3, 0.3) as h:
        res, rc = h.sweep(prof, np.linspace(0.006, -0.02, 25), dgamma=2e-3, final_pressure=p, precision=prec)
    out["rect_" + prec] = [rc, [r.force for r in res], [r.contact_count for r in res], p.tolist()]
# rough surface on the whole torus
n = 512
prof, zrms = I.rough_self_affine(n, q1_over_q0=64.0, seed=3)
p = np.empty((n, n))
with bem.Handle(n, n, 1.0 / n, 1.0 / n, 0.5, 0.3) as h:
    r, rc = h.solve(prof, zrms, pressure_out=p, precision="fp32")
out["rough32"] = [rc, [r.force], [r.contact_count], float(np.linalg.norm(p))]
print(json.dumps(out))
"""


def run(debug, tmp_path):
    env = dict(os.environ, BEM_DEBUG_CHECKS="1" if debug else "0")
    r = subprocess.run([sys.executable, "-c", CASES % (ROOT, debug)], capture_output=True, text=True,
                       env=env, timeout=900, cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_checks_pass_and_match_release(cuda_ok, tmp_path):
    dbg = run(True, tmp_path)
    rel = run(False, tmp_path)
    for key in rel:
        rc_d, F_d, cnt_d = dbg[key][:3]
        rc_r, F_r, cnt_r = rel[key][:3]
        assert rc_d == 0 and rc_r == 0, key
        assert cnt_d == cnt_r, key
        np.testing.assert_allclose(F_d, F_r, rtol=1e-6, atol=1e-12, err_msg=key)
    for prec in ("fp64", "fp32_refine"):
        a, b = np.array(dbg["rect_" + prec][3]), np.array(rel["rect_" + prec][3])
        assert np.linalg.norm(a - b) <= 1e-9 * max(np.linalg.norm(b), 1e-300)


TIMEOUT_CASE = r"""
import json, os, sys, time
sys.path.insert(0, %r)
from paper_1612_08395_gb300 import build
build.build(debug_checks=True)
import paper_1612_08395_gb300.bem as bem
import paper_1612_08395_gb300.inputs as I
n = 64
prof = I.paraboloid(n)
out = {}
with bem.Handle(n, n, 1.0 / n, 1.0 / n, 0.5, 0.3) as h:
    r0, rc0 = h.solve(prof, 0.01, precision="fp32")
    os.environ["BEM_INJECT_WAIT_TIMEOUT"] = "1"
    t0 = time.time()
    r1, rc1 = h.solve(prof, 0.01, precision="fp32", check=False)
    out["wait_s"] = time.time() - t0
    out["msg"] = bem.load_library().bem_last_error().decode()
    del os.environ["BEM_INJECT_WAIT_TIMEOUT"]
    r2, rc2 = h.solve(prof, 0.01, precision="fp32")
out["rc"] = [rc0, rc1, rc2]
out["force"] = [r0.force, r2.force]
out["count"] = [r0.contact_count, r2.contact_count]
print(json.dumps(out))
"""


def test_bounded_wait_runs_out_and_handle_recovers(cuda_ok, tmp_path):
    """A persistent pass waits (bounded) on a barrier that nothing completes --
    a debug-build test hook, after every copy the pass issued has landed.  The
    wait runs out, the kernel gives up and the solve returns BEM_ETIMEOUT; the
    next solve on the same handle gives the clean solve's result."""
    env = dict(os.environ, BEM_DEBUG_CHECKS="1")
    env.pop("BEM_INJECT_WAIT_TIMEOUT", None)
    r = subprocess.run([sys.executable, "-c", TIMEOUT_CASE % ROOT], capture_output=True, text=True,
                       env=env, timeout=600, cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["rc"] == [0, -5, 0], out
    assert "gave up waiting" in out["msg"]
    assert out["wait_s"] < 30.0
    assert out["force"][0] == out["force"][1] and out["count"][0] == out["count"][1]
