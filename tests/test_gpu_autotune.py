"""Launch-shape autotuner of the FP32 passes: every handle of a grid size in a
process gets the shapes the first one chose, the shapes are launchable (the
radix-16 column pass only where it exists), and a solve with tuned shapes
agrees with one at the default shapes (a process with BEM_AUTOTUNE=0) within
the FP32 path's tolerance."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SOLVE = r"""
import json, sys
import numpy as np
sys.path.insert(0, %r)
import paper_1612_08395_gb300.bem as bem
import paper_1612_08395_gb300.inputs as I
n = %d
p = np.empty((n, n))
with bem.Handle(n, n, 1.0 / n, 1.0 / n, 0.3, 0.3) as h:
    inf = h.info()
    res, rc = h.solve(I.paraboloid(n), 0.02, pressure_out=p, precision="fp32", tol=1e-7)
np.save(sys.argv[1], p)
print(json.dumps({"rows": inf.rows_per_cta, "cols": inf.cols_per_cta, "rc": rc, "F": res.force}))
"""


def test_same_size_same_shapes(bem_mod, cuda_ok):
    for n in (96, 256):
        with bem_mod.Handle(n, n, 1.0 / n, 1.0 / n, 0.3, 0.3) as a, \
                bem_mod.Handle(n, n, 1.0 / n, 1.0 / n, -0.4, 0.2) as b:
            ia, ib = a.info(), b.info()
        assert (ia.rows_per_cta, ia.cols_per_cta, ia.col_radix) == (ib.rows_per_cta, ib.cols_per_cta,
                                                                    ib.col_radix)
        for v in (ia.rows_per_cta, ia.cols_per_cta):
            assert v >= 1 and v & (v - 1) == 0
        # the radix-16 column pass exists for 512- to 8192-point columns only
        assert ia.col_radix in ((8, 16) if n >= 256 else (8,))


@pytest.mark.parametrize("n", [256, 1024])
def test_tuned_and_default_shapes_agree(tmp_path, cuda_ok, n):
    out = {}
    for tune in ("1", "0"):
        f = str(tmp_path / f"p{tune}.npy")
        env = dict(os.environ, BEM_AUTOTUNE=tune)
        r = subprocess.run([sys.executable, "-c", SOLVE % (ROOT, n), f], capture_output=True, text=True,
                           env=env, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        out[tune] = (json.loads(r.stdout.strip().splitlines()[-1]), np.load(f))
    assert out["1"][0]["rc"] == 0 and out["0"][0]["rc"] == 0
    pa, pb = out["1"][1], out["0"][1]
    assert np.linalg.norm(pa - pb) <= 1e-5 * np.linalg.norm(pb)
    assert out["1"][0]["F"] == pytest.approx(out["0"][0]["F"], rel=1e-5)
