"""Continuous-batching server on the GPU: a job's result does not depend on the
other jobs in the batch (bitwise), matches the single-system MD path and the
FP64 oracle, and admission, back-pressure, timeouts and errors behave as the
header states."""
import time

import numpy as np
import pytest

from oracle import oracle
from paper_1710_00882_gb300 import workloads as wl

from gpu_common import MIX_E_REL, SGL_E_REL, oracle_table, product_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available()
    from paper_1710_00882_gb300 import tersoff
    return tersoff


@pytest.fixture(scope="module")
def ctx(T):
    return T.Context(0)


@pytest.fixture(scope="module")
def P(T, ctx):
    # one table for all jobs: Si-only jobs use type 0 of the Si-C table
    return product_params(ctx, ("Si", "C"))


def jobs_mix():
    """Three systems of different sizes, boxes, species and step counts."""
    a = wl.si_box(4, 4, 4, seed=31, T=1200.0)
    b = wl.sic_box(3, seed=32, T=1500.0)
    c = wl.si_box(5, 4, 3, seed=33, T=800.0)
    return [(a, 1e-3, 37), (b, 0.5e-3, 23), (c, 1e-3, 61)]


def run_jobs(T, ctx, P, jobs, prec, chunk=7, budget=1 << 28, slots=16, stagger=False):
    srv = T.Server(ctx, P, prec=prec, skin=0.3, budget_bytes=budget, max_slots=slots, chunk_steps=chunk)
    ids = []
    for k, (s, dt, n) in enumerate(jobs):
        ids.append(srv.submit(s.pos, s.vel, s.types, s.box, dt, n))
        if stagger and k == 0:
            time.sleep(0.05)
    out = []
    for jid in ids:
        assert srv.wait(jid, timeout=120.0)
        out.append(srv.result(jid))
    st = srv.stats()
    srv.close()
    return out, st


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED", "SINGLE"])
def test_job_result_independent_of_batch(T, ctx, P, prec_name):
    prec = getattr(T, prec_name)
    jobs = jobs_mix()
    mixed, st = run_jobs(T, ctx, P, jobs, prec, stagger=True)
    assert st["completed"] == 3 and st["failed"] == 0
    for k, job in enumerate(jobs):
        alone, _ = run_jobs(T, ctx, P, [job], prec, chunk=11)
        pa, va, ea, _ = alone[0]
        pm, vm, em, _ = mixed[k]
        assert np.array_equal(pa, pm), f"job {k} positions differ alone vs in the batch"
        assert np.array_equal(va, vm), f"job {k} velocities differ alone vs in the batch"
        assert ea == em


def test_fp64_job_matches_oracle(T, ctx, P):
    jobs = jobs_mix()
    res, _ = run_jobs(T, ctx, P, jobs, T.FP64)
    tab, m = oracle_table(("Si", "C"))
    for (s, dt, n), (p, v, (epot, ekin), _) in zip(jobs, res):
        po, vo, tro = oracle.md_run(s.pos, s.vel, s.types, s.box, tab, m, dt, n)
        assert np.abs(p - po).max() < 1e-9 * 50
        assert np.abs(v - vo).max() < 1e-9 * 20
        assert abs(epot - tro[-1, 0]) <= 1e-9 * abs(tro[-1, 0])
        assert abs(ekin - tro[-1, 1]) <= 1e-9 * abs(tro[-1, 1])


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED", "SINGLE"])
def test_job_matches_single_system_md(T, ctx, P, prec_name):
    prec = getattr(T, prec_name)
    jobs = jobs_mix()
    res, _ = run_jobs(T, ctx, P, jobs, prec)
    tol = {T.FP64: 1e-9, T.MIXED: 1e-6, T.SINGLE: 1e-5}[prec]
    for (s, dt, n), (p, v, (epot, ekin), _) in zip(jobs, res):
        pr, vr, tr = T.md_run(ctx, P, s.pos, s.vel, s.types, s.box, dt, n, 0.3, prec=prec)
        assert np.abs(p - pr).max() < tol
        assert np.abs(v - vr).max() < 20 * tol
        assert abs(epot - tr[-1, 0]) <= {T.FP64: 1e-10, T.MIXED: MIX_E_REL, T.SINGLE: SGL_E_REL}[prec] * abs(tr[-1, 0])


def test_admission_limited_by_budget_and_slots(T, ctx, P):
    base = jobs_mix()
    jobs = [base[k % 3] for k in range(7)]
    # room for about two of these systems at a time, at most two slots
    res, st = run_jobs(T, ctx, P, jobs, T.MIXED, chunk=5, budget=1200 * 900, slots=2)
    assert st["completed"] == 7 and st["admitted"] == 7 and st["failed"] == 0
    assert st["queued"] == 0 and st["running"] == 0
    assert st["repacks"] >= 4
    assert st["atom_steps"] == sum(s.n * n for s, _, n in jobs)
    ref, _ = run_jobs(T, ctx, P, base, T.MIXED)
    for k, (p, v, e, t) in enumerate(res):
        assert np.array_equal(p, ref[k % 3][0])
        assert t[0] >= 0 and t[1] > 0 and abs(t[2] - t[0] - t[1]) < 1e-9


def test_freed_ranges_and_compaction_keep_results(T, ctx, P, monkeypatch):
    """Jobs keep their atom ranges: a retired job leaves a freed range that a later
    job may fill, and a job that fits no free range compacts the layout (resident
    jobs move, every list and force is rebuilt).  Results stay bitwise those of the
    jobs run alone, with and without compaction at every admission."""
    a, b, c = jobs_mix()
    # about 1050 atoms of capacity, three slots: b (205 atoms) leaves a hole below a
    # (512) that c (480) does not fit, so c's admission compacts the layout
    jobs = [b, a, c, b, a]
    ref = {id(j): run_jobs(T, ctx, P, [j], T.MIXED, chunk=9)[0][0] for j in (a, b, c)}
    for env in (None, "0"):
        if env is not None:
            monkeypatch.setenv("TERSOFF_COMPACT_FREED", env)
        res, st = run_jobs(T, ctx, P, jobs, T.MIXED, chunk=5, budget=1200 * 900, slots=3)
        assert st["completed"] == len(jobs) and st["failed"] == 0
        assert st["compactions"] >= 1
        for job, (p, v, e, _) in zip(jobs, res):
            pr, vr, er, _ = ref[id(job)]
            assert np.array_equal(p, pr) and np.array_equal(v, vr) and e == er


def test_tiny_jobs_in_a_mix(T, ctx, P):
    """Jobs of one, two and three atoms (a lone atom drifts, a dimer and an Si-C pair
    vibrate) next to a bulk job: each route segment is a fraction of a warp, and every
    result matches the same job run alone (bitwise) and the FP64 oracle."""
    box = np.array([12.0, 12.0, 12.0])
    def job(pos, types, vel, n=40):
        s = wl.System(pos=np.array(pos, float), types=np.array(types, np.int32), box=box, species=("Si", "C"),
                      vel=np.array(vel, float))
        return (s, 0.5e-3, n)
    tiny = [job([[1.0, 2.0, 3.0]], [0], [[0.5, -0.2, 0.1]]),
            job([[5.0, 5.0, 5.0], [7.3, 5.0, 5.0]], [0, 0], [[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]),
            job([[5.0, 5.0, 5.0], [6.8, 5.3, 5.0]], [0, 1], [[0.1, 0.0, 0.0], [-0.2, 0.0, 0.0]]),
            job([[5.0, 5.0, 5.0], [7.3, 5.0, 5.0], [4.2, 7.2, 5.0]], [0, 1, 0], [[0.0] * 3] * 3)]
    jobs = tiny + [jobs_mix()[1]]
    mixed, st = run_jobs(T, ctx, P, jobs, T.FP64, chunk=7)
    assert st["completed"] == len(jobs) and st["failed"] == 0
    tab, m = oracle_table(("Si", "C"))
    for k, (s, dt, n) in enumerate(tiny):
        alone, _ = run_jobs(T, ctx, P, [(s, dt, n)], T.FP64, chunk=11)
        assert np.array_equal(alone[0][0], mixed[k][0]) and np.array_equal(alone[0][1], mixed[k][1])
        po, vo, tro = oracle.md_run(s.pos, s.vel, s.types, s.box, tab, m, dt, n)
        assert np.abs(mixed[k][0] - po).max() < 1e-9
        assert np.abs(mixed[k][1] - vo).max() < 1e-8


def test_wait_timeout_poll_and_errors(T, ctx, P):
    srv = T.Server(ctx, P, prec=T.MIXED, skin=0.3, budget_bytes=1 << 26, max_slots=4, chunk_steps=50)
    s = wl.si_box(4, 4, 4, seed=41, T=1000.0)
    jid = srv.submit(s.pos, s.vel, s.types, s.box, 1e-3, 4000)
    assert srv.wait(jid, timeout=0.0) is False
    assert srv.stats()["capacity_atoms"] < 110592
    assert srv.poll(jid) is False
    with pytest.raises(T.TersoffError) as e:
        srv.result(jid)
    assert e.value.code == T.ERR_BUSY
    assert srv.wait(jid, timeout=120.0) is True
    assert srv.poll(jid) is True
    p, v, (epot, ekin), _ = srv.result(jid)
    assert np.isfinite(p).all() and epot < 0 and ekin > 0
    with pytest.raises(T.TersoffError) as e:
        srv.poll(jid)
    assert e.value.code == T.ERR_NOT_FOUND
    # rejected submissions
    with pytest.raises(T.TersoffError) as e:
        srv.submit(s.pos, s.vel, s.types, [5.0, 5.0, 5.0], 1e-3, 10)
    assert e.value.code == T.ERR_BOX_TOO_SMALL
    with pytest.raises(T.TersoffError) as e:
        srv.submit(s.pos, s.vel, np.full(s.n, 7), s.box, 1e-3, 10)
    assert e.value.code == T.ERR_ARG
    big = wl.si_box(24, 24, 24, seed=42)   # 110,592 atoms, above the ~66k the 64 MB budget holds
    with pytest.raises(T.TersoffError) as e:
        srv.submit(big.pos, big.vel, big.types, big.box, 1e-3, 10)
    assert e.value.code == T.ERR_NOMEM
    # zero steps: the input comes back
    jid = srv.submit(s.pos, s.vel, s.types, s.box, 1e-3, 0)
    assert srv.wait(jid, timeout=60.0)
    p, v, _, _ = srv.result(jid)
    assert np.array_equal(p, s.pos) and np.array_equal(v, s.vel)
    srv.close()


def test_close_with_jobs_in_flight(T, ctx, P):
    srv = T.Server(ctx, P, prec=T.MIXED, skin=0.3, budget_bytes=1 << 26, max_slots=2, chunk_steps=20)
    s = wl.si_box(4, 4, 4, seed=43, T=1000.0)
    for _ in range(4):
        srv.submit(s.pos, s.vel, s.types, s.box, 1e-3, 100000)
    time.sleep(0.2)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 30.0


def test_many_jobs_admitted_together(T, ctx, P):
    """A stream of jobs queued at once: many new systems enter one admission, jobs
    leave at different chunks, and a sample of them matches its run alone bitwise."""
    stream = wl.serving_stream(48, seed=7, max_atoms=3000)
    jobs = [(j.system, j.dt, j.steps) for j in stream]
    res, st = run_jobs(T, ctx, P, jobs, T.MIXED, chunk=10, slots=32, budget=1 << 27)
    assert st["completed"] == len(jobs) and st["failed"] == 0
    for k in (0, 17, 47):
        alone, _ = run_jobs(T, ctx, P, [jobs[k]], T.MIXED, chunk=13)
        assert np.array_equal(alone[0][0], res[k][0]) and np.array_equal(alone[0][1], res[k][1])
