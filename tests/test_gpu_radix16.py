"""The radix-16 column pass (FP32 pass B with radix-16 stages, 512 to 8192
points) against the oracle, with the radix fixed by BEM_RADIX_B=16 (the
autotuner otherwise picks the radix per grid size):

- the transform u = A K*p (Eq. 7 via Eq. 13) for every column length the pass
  supports, against the oracle's direct sum, at the FP32 transform bar of
  2e-6 of the field's maximum (ragged grids; square elements);
- the adhesive pull-off sweep (Sec. 3.1, Eq. 24) at 256^2 in plain FP32 and
  FP32 + refinement, step by step against the oracle (exact contact counts);
- the 2048^2 benchmark sweep in plain FP32 against the same sweep with the
  radix-8 pass (its box tori have 2048-point columns): equal contact counts at
  every step, forces within 2e-5 of the largest |F|;
- batched loops of concurrent server jobs (the several-instance kernel) at
  256^2 against each job alone and, for a non-adhesive one, the oracle.
"""
import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu

K, NU, GAM, D0 = 0.3, 0.3, 1e-3, 0.02


def relL2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture
def radix16(monkeypatch):
    monkeypatch.setenv("BEM_RADIX_B", "16")
    yield


# columns of 512, 1024, 2048, 4096 and 8192 points (Py = 2 Ny rounded up)
@pytest.mark.parametrize("nx,ny,k", [(40, 200, 0.4), (33, 300, -0.6), (16, 700, 0.4), (24, 1500, -0.6),
                                     (8, 4096, 0.4)])
def test_radix16_transform_vs_oracle(bem_mod, oracle_mod, cuda_ok, radix16, nx, ny, k):
    d = 1.0 / max(nx, ny)
    p = I.random_pressure(nx, ny, seed=nx * 1000 + ny, density=0.7)
    Ko = oracle_mod.influence_quarter(k, d, d, nx, ny)
    uo = oracle_mod.compliance(k, NU) * oracle_mod.convolve_direct(Ko, p)
    with bem_mod.Handle(nx, ny, d, d, k, NU) as h:
        assert h.info().col_radix == 16
        u32 = h.convolve(p, "fp32")
        u64 = h.convolve(p, "fp64")
    scale = np.abs(uo).max()
    assert np.abs(u32 - uo).max() <= 2e-6 * scale
    assert np.abs(u64 - uo).max() <= 1e-12 * scale


@pytest.fixture(scope="module")
def oracle_sweep_256(oracle_mod):
    n = 256
    dx = 1.0 / n
    A = oracle_mod.compliance(K, NU)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(K, dx, dx, n + 1, n + 1), n, n)
    steps = np.linspace(D0, -0.03, 61)
    res, p, S = oracle_mod.adhesive_unload(A, conv, I.paraboloid(n), D0, steps[1:],
                                           oracle_mod.p_crit(K, NU, GAM, dx), dx * dx,
                                           tol_pk=1e-12, tol_cg=1e-13)
    pre = oracle_mod.pk_solve(A, conv, I.paraboloid(n), D0, tol=1e-12)
    return dict(steps=steps, res=res, p=p, S=S, pre_count=int((pre.p > 0).sum()),
                pre_force=dx * dx * float(pre.p.sum()))


@pytest.mark.parametrize("prec,ftol,ptol", [("fp32", 1e-4, 1e-4), ("fp32_refine", 1e-9, 1e-9)])
def test_radix16_adhesive_sweep_vs_oracle(bem_mod, cuda_ok, radix16, oracle_sweep_256, prec, ftol, ptol):
    o = oracle_sweep_256
    n = 256
    dx = 1.0 / n
    p = np.empty((n, n))
    with bem_mod.Handle(n, n, dx, dx, K, NU) as h:
        assert h.info().col_radix == 16
        res, rc = h.sweep(I.paraboloid(n), o["steps"], dgamma=GAM, final_pressure=p, precision=prec)
        S = h.contact_set()
    assert rc == bem_mod.BEM_OK
    fmax = max(abs(r["force"]) for r in o["res"])
    assert res[0].contact_count == o["pre_count"]
    assert abs(res[0].force - o["pre_force"]) <= ftol * fmax
    for ro, r in zip(o["res"], res[1:]):
        assert r.contact_count == ro["count"], (ro["d"], r.contact_count, ro["count"])
        assert abs(r.force - ro["force"]) <= ftol * fmax, (ro["d"], r.force, ro["force"])
    assert sum(ro["rounds"] for ro in o["res"]) > 0
    np.testing.assert_array_equal(S.astype(bool), o["S"])
    if np.linalg.norm(o["p"]) > 0:
        assert relL2(p, o["p"]) <= ptol


def test_radix16_sweep_2048_matches_radix8(bem_mod, cuda_ok, monkeypatch):
    n = 2048
    dx = 1.0 / n
    steps = np.array([D0] + [D0 - 1.1e-4 * j for j in range(1, 401)])
    prof = I.paraboloid(n, 1.0)
    runs = {}
    for radix in ("8", "16"):
        monkeypatch.setenv("BEM_RADIX_B", radix)
        with bem_mod.Handle(n, n, dx, dx, K, NU) as h:
            res, rc = h.sweep(prof, steps, dgamma=GAM, precision="fp32")
        assert rc == bem_mod.BEM_OK
        runs[radix] = res
    fmax = max(abs(r.force) for r in runs["8"])
    assert [r.contact_count for r in runs["16"]] == [r.contact_count for r in runs["8"]]
    assert max(abs(a.force - b.force) for a, b in zip(runs["16"], runs["8"])) <= 2e-5 * fmax
    assert min(r.force for r in runs["16"]) < 0


def test_radix16_batched_loops(bem_mod, oracle_mod, cuda_ok, radix16):
    """Six rough-surface jobs of one size class (256^2 at d = rms height: the
    contact spots spread over the grid, so the loops run on the 512^2 torus
    with the radix-16 column pass), four adhesive (9 unloading depths, many
    fixed-set solves each) and two not, on six workers: their loops run
    batched, every result matches the job alone, and a non-adhesive one
    matches the oracle."""
    from test_gpu_server import assert_close, assert_matches_oracle, run_alone, submit
    jobs = [{"n": 256, "k": -0.6 + 0.2 * i, "nu": 0.3, "dgamma": 1e-3 if i < 4 else 0.0, "adhesive": i < 4,
             "profile": "rough", "seed": 300 + i, "precision": "fp32_refine"} for i in range(6)]
    alone = [run_alone(bem_mod, j) for j in jobs]
    with bem_mod.Server(nworkers=6, hbm_budget_bytes=8 << 30) as srv:
        tags = [submit(srv, j) for j in jobs]
        comps = {c["tag"]: c for c in srv.drain()}
        launches, loops = srv.loop_stats()
    for t, a in zip(tags, alone):
        assert_close(a, comps[t], "fp32_refine")
    assert launches > 0 and loops >= 1.5 * launches, (launches, loops)
    assert_matches_oracle(oracle_mod, jobs[4], comps[tags[4]]["results"], comps[tags[4]]["final_pressure"])
