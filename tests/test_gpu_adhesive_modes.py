"""The adhesive pull-off sweep (Sec. 3.1: hold the contact set, solve, detach
every element with -p > p_crit of Eq. 24, repeat) in the precision modes the
benchmark times: plain FP32 and FP32 with FP64 refinement, at their default
tolerances.

- 64^2 and 128^2: step by step against the FP64 oracle (the path is the same
  only if every detach decision is): exact contact counts at every step, force
  within the mode's pressure tolerance times the largest |F| of the sweep
  (FP32 1e-4, the rounding floor of its transform times the conditioning;
  FP32 + refinement 1e-9), final pressure by relative L2.
- 2048^2, the benchmark's workload (k = 0.3, nu = 0.3, R = 1, dgamma = 1e-3,
  preload 0.02, 400 unloading steps of 1.1e-4): both modes against the FP64
  GPU sweep, which the oracle pins at the small sizes above and in
  test_gpu_parity.py.  Contact counts at every step and the held contact sets
  at four checkpoints must agree exactly; forces and checkpoint pressures are
  compared by relative error.  The sweep runs as four resumed segments
  (bem_sweep_from, bitwise equal to one call) so the pressures at the
  checkpoints can be read.
"""
import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu

K, NU, GAM, D0 = 0.3, 0.3, 1e-3, 0.02


def relL2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def oracle_sweeps(oracle_mod):
    out = {}
    for n in (64, 128):
        dx = 1.0 / n
        A = oracle_mod.compliance(K, NU)
        conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(K, dx, dx, n + 1, n + 1), n, n)
        steps = np.linspace(D0, -0.03, 101)
        res, p, S = oracle_mod.adhesive_unload(A, conv, I.paraboloid(n), D0, steps[1:],
                                               oracle_mod.p_crit(K, NU, GAM, dx), dx * dx,
                                               tol_pk=1e-12, tol_cg=1e-13)
        pre = oracle_mod.pk_solve(A, conv, I.paraboloid(n), D0, tol=1e-12)
        out[n] = dict(steps=steps, res=res, p=p, S=S, pre_count=int((pre.p > 0).sum()),
                      pre_force=dx * dx * float(pre.p.sum()))
    return out


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("prec,ftol,ptol", [("fp32", 1e-4, 1e-4), ("fp32_refine", 1e-9, 1e-9)])
def test_adhesive_sweep_mode_vs_oracle(bem_mod, cuda_ok, oracle_sweeps, n, prec, ftol, ptol):
    o = oracle_sweeps[n]
    dx = 1.0 / n
    p = np.empty((n, n))
    with bem_mod.Handle(n, n, dx, dx, K, NU) as h:
        res, rc = h.sweep(I.paraboloid(n), o["steps"], dgamma=GAM, final_pressure=p, precision=prec)
        S = h.contact_set()
    assert rc == bem_mod.BEM_OK
    fmax = max(abs(r["force"]) for r in o["res"])
    assert res[0].contact_count == o["pre_count"]
    assert abs(res[0].force - o["pre_force"]) <= ftol * fmax
    detached = False
    for ro, r in zip(o["res"], res[1:]):
        assert r.contact_count == ro["count"], (ro["d"], r.contact_count, ro["count"])
        assert abs(r.force - ro["force"]) <= ftol * fmax, (ro["d"], r.force, ro["force"])
        detached |= ro["rounds"] > 0
    assert detached  # the sweep reaches the detaching part of the path
    np.testing.assert_array_equal(S.astype(bool), o["S"])
    if np.linalg.norm(o["p"]) > 0:
        assert relL2(p, o["p"]) <= ptol


def test_sweep_2048_modes_vs_fp64(bem_mod, cuda_ok):
    n = 2048
    dx = 1.0 / n
    steps = np.array([D0] + [D0 - 1.1e-4 * j for j in range(1, 401)])
    cuts = [0, 101, 201, 301, 351]   # segments [cut_i, cut_{i+1}); checkpoints at their last steps
    import torch
    prof = torch.from_numpy(I.paraboloid(n, 1.0)).cuda()
    runs = {}
    with bem_mod.Handle(n, n, dx, dx, K, NU) as h:
        for prec in ("fp64", "fp32", "fp32_refine"):
            res_all, chk = [], []
            p = torch.empty((n, n), dtype=torch.float64, device="cuda")
            for i in range(len(cuts) - 1):
                seg = steps[cuts[i]:cuts[i + 1]]
                if i == 0:
                    res, rc = h.sweep(prof, seg, dgamma=GAM, final_pressure=p, precision=prec)
                else:
                    res, rc = h.sweep_from(prof, seg, p_state=p.clone(), S_state=S, dgamma=GAM,
                                           final_pressure=p, precision=prec)
                assert rc == bem_mod.BEM_OK, (prec, i)
                S = h.contact_set()
                torch.cuda.synchronize()
                chk.append((p.cpu().numpy().copy(), S.copy()))
                res_all += res
            runs[prec] = (res_all, chk)
    ref_res, ref_chk = runs["fp64"]
    fmax = max(abs(r.force) for r in ref_res)
    assert min(r.force for r in ref_res) < 0  # the path goes through pull-off tension
    assert sum(r.detach_rounds for r in ref_res) > 0
    for prec, ftol, ptol in (("fp32", 2e-5, 1e-4), ("fp32_refine", 1e-9, 1e-9)):
        res, chk = runs[prec]
        counts = [r.contact_count for r in res]
        assert counts == [r.contact_count for r in ref_res], prec
        df = max(abs(a.force - b.force) for a, b in zip(res, ref_res))
        assert df <= ftol * fmax, (prec, df / fmax)
        for (pc, Sc), (pr, Sr) in zip(chk, ref_chk):
            np.testing.assert_array_equal(Sc, Sr)
            assert relL2(pc, pr) <= ptol, (prec, relL2(pc, pr))
