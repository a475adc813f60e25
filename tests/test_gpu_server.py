"""The request server (bem_server_*): each job's result is the same alone and
in a mix of concurrent jobs (within its precision's tolerance: jobs whose CG
loops share a batched launch run the several-instance kernels, whose rounding
may differ from the single-instance ones in the last bits; a job that runs
alone in the server is bitwise its alone result), cached spectra are reused
across materials, admission keeps the device bytes within the budget, and a
failing job reports its status without stopping the others."""
import numpy as np
import pytest

import paper_1612_08395_gb300.inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("force", "area", "contact_radius", "final_eps", "max_gap_violation", "depth",
          "iterations", "detach_rounds", "contact_count", "status", "stalled")

# pressure tolerance of each precision mode against the FP64 oracle at the
# default solver tolerances (plain FP32: the rounding floor of its transform
# times the conditioning; the others: the FP64 stopping rules)
MODE_TOL = {"fp64": 1e-8, "fp32_refine": 1e-8, "fp32": 5e-4}


def oracle_job(oracle_mod, job):
    """The oracle's result for a job: per-step contact counts and the final pressure
    (non-adhesive: Polonsky-Keer at the depth; adhesive: preload, then the held-set
    solve and detach loop at each unloading depth, Sec. 3.1)."""
    n = job["n"]
    dx = 1.0 / n
    h, ds = I.job_profile(job)
    A = oracle_mod.compliance(job["k"], job["nu"])
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(job["k"], dx, dx, n + 1, n + 1), n, n)
    if job["dgamma"] > 0:
        out, p, S = oracle_mod.adhesive_unload(A, conv, h, ds[0], ds[1:],
                                               oracle_mod.p_crit(job["k"], job["nu"], job["dgamma"], dx),
                                               dx * dx, tol_pk=1e-12, tol_cg=1e-13)
        pre = oracle_mod.pk_solve(A, conv, h, ds[0], tol=1e-12)
        return [int((pre.p > 0).sum())] + [o["count"] for o in out], p
    res = oracle_mod.pk_solve(A, conv, h, ds[0], tol=1e-12)
    return [int((res.p > 0).sum())], res.p


def assert_matches_oracle(oracle_mod, job, results, p):
    counts, p_ref = oracle_job(oracle_mod, job)
    tol = MODE_TOL[job["precision"]]
    got = [r["contact_count"] if isinstance(r, dict) else r.contact_count for r in results]
    if job["precision"] == "fp32":
        # plain FP32 may round an element at the contact edge to the other side
        assert all(abs(a - b) <= max(2, 0.002 * b) for a, b in zip(got, counts)), (got, counts)
    else:
        assert got == counts, (job, got, counts)
    nrm = np.linalg.norm(p_ref)
    if nrm > 0:
        assert np.linalg.norm(p - p_ref) <= tol * nrm, (job, np.linalg.norm(p - p_ref) / nrm)
    else:
        assert np.abs(p).max() == 0


def small_jobs():
    """A mix of grids, k, materials, precisions and adhesion (paraboloid R=1 and rough)."""
    jobs = []
    for i, (n, k, nu, dg, prec, rough) in enumerate([
            (64, 0.5, 0.3, 0.0, "fp64", False),
            (64, 0.5, 0.45, 0.0, "fp64", False),        # same key as the first, other nu
            (96, -0.4, 0.3, 1e-3, "fp32_refine", False),
            (128, 0.3, 0.3, 0.0, "fp32_refine", True),
            (80, 0.0, 0.25, 2e-3, "fp64", False),
            (128, 0.3, 0.3, 1e-4, "fp32", True),
            (48, -0.7, 0.3, 0.0, "fp32_refine", False),
            (96, -0.4, 0.3, 1e-3, "fp32_refine", False)]):  # repeat of job 2
        job = {"n": n, "k": k, "nu": nu, "dgamma": dg, "adhesive": dg > 0,
               "profile": "rough" if rough else "paraboloid", "seed": 77 + i, "precision": prec}
        jobs.append(job)
    return jobs


def run_alone(bem_mod, job):
    n = job["n"]
    h, ds = I.job_profile(job)
    p = np.empty((n, n))
    with bem_mod.Handle(n, n, 1.0 / n, 1.0 / n, job["k"], job["nu"]) as hd:
        res, rc = hd.sweep(h, ds, dgamma=job["dgamma"], final_pressure=p, precision=job["precision"])
        held = hd.info().device_bytes
    return [r.as_dict() for r in res], p, rc, held


def submit(srv, job):
    n = job["n"]
    h, ds = I.job_profile(job)
    p = np.empty((n, n))
    return srv.submit(n, n, 1.0 / n, 1.0 / n, job["k"], job["nu"], h, ds, dgamma=job["dgamma"],
                      final_pressure=p, precision=job["precision"])


def assert_same(alone, comp):
    """Bitwise the alone result."""
    res_a, p_a, rc_a, _ = alone
    assert comp["status"] == rc_a
    for ra, rb in zip(res_a, comp["results"]):
        rb = rb.as_dict()
        for f in FIELDS:
            assert ra[f] == rb[f] or (np.isnan(ra[f]) and np.isnan(rb[f])), f
    assert np.array_equal(p_a, comp["final_pressure"])


# a result alone and in a batched mix: pressure and force within these of the
# alone result (relative), contact counts exact
MIX_TOL = {"fp64": 1e-10, "fp32_refine": 1e-9, "fp32": 1e-5}


def assert_close(alone, comp, prec):
    res_a, p_a, rc_a, _ = alone
    tol = MIX_TOL[prec]
    assert comp["status"] == rc_a
    fmax = max(max(abs(r["force"]) for r in res_a), 1e-300)
    for ra, rb in zip(res_a, comp["results"]):
        assert ra["contact_count"] == rb.contact_count
        assert abs(ra["force"] - rb.force) <= tol * fmax
    nrm = np.linalg.norm(p_a)
    assert np.linalg.norm(p_a - comp["final_pressure"]) <= tol * max(nrm, 1e-300)


def test_alone_equals_mix(bem_mod, oracle_mod):
    jobs = small_jobs()
    alone = [run_alone(bem_mod, j) for j in jobs]
    with bem_mod.Server(nworkers=4, hbm_budget_bytes=4 << 30) as srv:
        tags = [submit(srv, j) for j in jobs]
        comps = {c["tag"]: c for c in srv.drain()}
        assert srv.pending() == 0
    assert sorted(comps) == sorted(tags)
    for t, a, j in zip(tags, alone, jobs):
        assert_close(a, comps[t], j["precision"])
        assert comps[t]["device"] >= 0
        # and each served result is the oracle's, within its precision's tolerance
        assert_matches_oracle(oracle_mod, j, comps[t]["results"], comps[t]["final_pressure"])
    # several jobs overlapped on the device
    iv = sorted((c["t_start"], c["t_end"]) for c in comps.values())
    assert any(iv[i + 1][0] < iv[i][1] for i in range(len(iv) - 1))


def test_cached_spectrum_reused_with_new_material(bem_mod):
    """One worker: the second job has the first one's key (grid, element size, k)
    and another nu, so it runs on the cached handle after bem_set_material."""
    jobs = small_jobs()[:2]
    alone = [run_alone(bem_mod, j) for j in jobs]
    with bem_mod.Server(nworkers=1, hbm_budget_bytes=1 << 30) as srv:
        tags = [submit(srv, j) for j in jobs]
        comps = {c["tag"]: c for c in srv.drain()}
        held = srv.device_bytes()
    for t, a in zip(tags, alone):
        assert_same(a, comps[t])
    assert held == alone[0][3]  # a single cached handle, reused


def test_admission_within_budget(bem_mod):
    n = 1024
    budget = int(1.5 * bem_mod.Server.footprint(n, n))
    job = {"n": n, "nu": 0.3, "dgamma": 0.0, "adhesive": False, "profile": "paraboloid",
           "seed": 0, "precision": "fp32_refine"}
    with bem_mod.Server(nworkers=4, hbm_budget_bytes=budget) as srv:
        for i in range(4):  # distinct k: no handle can be shared
            submit(srv, dict(job, k=-0.6 + 0.4 * i))
        comps = srv.drain()
        assert srv.device_bytes() <= budget
        big = 2048
        h = np.zeros((big, big))
        with pytest.raises(bem_mod.BemError) as e:
            srv.submit(big, big, 1 / big, 1 / big, 0.3, 0.3, h, [0.01])
        assert e.value.code == bem_mod.BEM_ENOMEM
    assert all(c["status"] == bem_mod.BEM_OK for c in comps)
    iv = sorted((c["t_start"], c["t_end"]) for c in comps)
    # only one 1024^2 job fits: the jobs ran one after another
    assert all(iv[i + 1][0] >= iv[i][1] for i in range(len(iv) - 1))


def test_failing_job_reports_status(bem_mod):
    good = small_jobs()[0]
    with bem_mod.Server(nworkers=2, hbm_budget_bytes=1 << 30) as srv:
        t_bad = submit(srv, dict(good, nu=0.7))  # nu > 0.5: rejected by bem_create
        t_good = submit(srv, good)
        comps = {c["tag"]: c for c in srv.drain()}
    assert comps[t_bad]["status"] == bem_mod.BEM_EINVAL
    assert comps[t_good]["status"] == bem_mod.BEM_OK


def test_batch_fp32_refine_matches_fp64(bem_mod, oracle_mod):
    """Jobs of the batched mix (grid sides 128 and 256 here) at FP32 + refinement
    agree with the FP64 path: pressure relative L2 <= 1e-5 and equal contact counts;
    the 128^2 jobs also match the oracle (contact counts at every step exact,
    final pressure within 1e-8 relative L2)."""
    jobs = [j for j in I.batch_jobs(48, seed=4, sides=(128, 256))][:12]
    with bem_mod.Server(nworkers=4, hbm_budget_bytes=8 << 30) as srv:
        t32 = [submit(srv, dict(j, precision="fp32_refine")) for j in jobs]
        t64 = [submit(srv, dict(j, precision="fp64")) for j in jobs]
        comps = {c["tag"]: c for c in srv.drain()}
    for a, b in zip(t32, t64):
        ca, cb = comps[a], comps[b]
        assert ca["status"] == bem_mod.BEM_OK and cb["status"] == bem_mod.BEM_OK
        pa, pb = ca["final_pressure"], cb["final_pressure"]
        nrm = np.linalg.norm(pb)
        if nrm > 0:
            assert np.linalg.norm(pa - pb) <= 1e-5 * nrm
        assert ca["results"][-1].contact_count == cb["results"][-1].contact_count
    checked = 0
    for j, a in zip(jobs, t32):
        if j["n"] == 128:
            assert_matches_oracle(oracle_mod, dict(j, precision="fp32_refine"), comps[a]["results"],
                                  comps[a]["final_pressure"])
            checked += 1
    assert checked >= 3


def test_cancel_a_queued_job(bem_mod):
    """One worker busy with a 1024^2 adhesive sweep: the job queued behind it can
    be cancelled (its completion carries BEM_ECANCELED, its arrays are untouched);
    the running job cannot, and finishes normally."""
    n = 1024
    h = I.paraboloid(n)
    steps = np.linspace(0.02, -0.02, 81)
    with bem_mod.Server(nworkers=1, hbm_budget_bytes=8 << 30) as srv:
        t_run = srv.submit(n, n, 1.0 / n, 1.0 / n, 0.3, 0.3, h, steps, dgamma=1e-3, precision="fp32")
        p = np.full((64, 64), -7.0)
        t_q = srv.submit(64, 64, 1 / 64, 1 / 64, 0.3, 0.3, I.paraboloid(64), [0.01], final_pressure=p)
        assert srv.cancel(t_q)
        assert not srv.cancel(t_q)  # no longer queued
        comps = {c["tag"]: c for c in srv.drain()}
    assert comps[t_q]["status"] == bem_mod.BEM_ECANCELED
    assert (p == -7.0).all()
    assert comps[t_run]["status"] == bem_mod.BEM_OK


def test_concurrent_loops_share_launches(bem_mod, oracle_mod):
    """Eight jobs of one size class (128^2 paraboloids, each with its own k, so
    each has its own handle) on eight workers: their CG loops run batched, one
    launch per pass carrying several solves, every result equals the job's
    alone result within its precision's tolerance, and one of them is also
    checked against the oracle."""
    jobs = [{"n": 128, "k": -0.7 + 0.2 * i, "nu": 0.3, "dgamma": 0.0, "adhesive": False,
             "profile": "paraboloid", "seed": 0, "precision": "fp32_refine"} for i in range(8)]
    alone = [run_alone(bem_mod, j) for j in jobs]
    with bem_mod.Server(nworkers=8, hbm_budget_bytes=8 << 30) as srv:
        tags = [submit(srv, j) for j in jobs]
        comps = {c["tag"]: c for c in srv.drain()}
        launches, loops = srv.loop_stats()
    for t, a in zip(tags, alone):
        assert_close(a, comps[t], "fp32_refine")
    assert launches > 0 and loops >= 1.5 * launches, (launches, loops)
    assert_matches_oracle(oracle_mod, jobs[3], comps[tags[3]]["results"], comps[tags[3]]["final_pressure"])
