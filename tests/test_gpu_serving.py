"""GPU: continuous-batching serving.  Jobs of mixed kinds, sizes and precisions arrive while
others run, wait for a batch slot and for device memory (admission by gbr_workspace_bytes in a
pool that holds only a few of them), run in the mix, and leave; each result must equal -- bitwise --
the same job run alone through gbr_rk_step, and the server reports time-to-N-steps percentiles."""
import numpy as np
import pytest

from paper_2303_10785_b300 import gbr, serving
from paper_2303_10785_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def small_stream(n=14, seed=3, rate=400.0):
    specs = I.serving_stream(n, seed=seed, rate=rate, edge2d=(24, 72), edge3d=(12, 24), steps=(3, 14))
    jobs = []
    for sp in specs:
        case, nodes, q, cfl = I.serving_job_inputs(sp)
        jobs.append(serving.Job(sp["id"], case, nodes, q, sp["steps"], cfl, sp["arrival"]))
    return jobs


def test_serving_results_equal_alone_and_in_the_mix():
    jobs = small_stream()
    alone = serving.run_serial([serving.Job(j.id, j.case, j.nodes, j.q, j.steps, j.cfl, 0.0) for j in jobs])
    pool = int(2.5 * max(j.footprint() for j in jobs))
    srv = serving.Server(pool, max_active=4, chunk_steps=3)
    srv.run(jobs)
    assert len(srv.done) == len(jobs) and not srv.queue and not srv.active
    assert 1 < srv.peak_active <= 4 and srv.peak_pool <= pool
    for j, a in zip(sorted(jobs, key=lambda x: x.id), sorted(alone, key=lambda x: x.id)):
        assert j.error is None
        assert np.array_equal(j.result, a.result), j.id
        assert j.time == a.time
    st = serving.latency_stats(jobs)
    assert st["jobs"] == len(jobs) and 0 < st["p50_s"] <= st["p99_s"]
    assert all(j.admitted >= j.arrival - 1e-9 and j.finished >= j.admitted for j in jobs)
    srv.close()


def test_serving_rejects_a_job_larger_than_the_pool():
    jobs = small_stream(3)
    big = max(jobs, key=lambda j: j.footprint())
    srv = serving.Server(big.footprint() - 4096, max_active=2)
    srv.run(jobs)
    assert big.error and "larger than the device pool" in big.error
    assert all(j.result is not None for j in jobs if j is not big)
    srv.close()


def test_a_job_whose_state_goes_bad_fails_alone():
    # one job starts from a state with a NaN (as an unstable job would end): the batch reports it,
    # the server retires it with the error and frees its memory, and the other jobs finish with the
    # states they reach alone; the plain per-job form isolates it the same way
    jobs = small_stream(5, seed=11)
    bad = jobs[2]
    q = bad.q.copy()
    q[0].flat[q[0].size // 2] = np.nan
    bad.q = q
    alone = serving.run_serial([serving.Job(j.id, j.case, j.nodes, j.q, j.steps, j.cfl, 0.0) for j in jobs])
    assert [a.error is not None for a in alone] == [j is bad for j in jobs]
    pool = int(4 * max(j.footprint() for j in jobs))
    srv = serving.Server(pool, max_active=4, chunk_steps=2)
    srv.run(jobs)
    assert len(srv.done) == len(jobs) and not srv.active and srv.arena.stats()["used"] == 0
    assert bad.error and "ENONFINITE" in bad.error and bad.result is None
    for j, a in zip(jobs, alone):
        if j is not bad:
            assert j.error is None and np.array_equal(j.result, a.result), j.id
    st = serving.latency_stats(jobs)
    assert st["jobs"] == len(jobs) - 1 and st["failed"] == 1
    srv.close()


def test_served_jobs_match_the_oracle():
    """Served jobs of each precision and kind against the FP64 oracle after their steps: FP64 jobs
    within L1 1e-8 (the Sod slabs' limiter is active at the waves) and, when smooth, 1e-10 of max |Q|;
    mixed-precision jobs within 1e-5 (L-infinity)."""
    import oracle as O
    from test_gpu_parity import rel_state

    jobs = small_stream(12, seed=5)
    pool = int(3 * max(j.footprint() for j in jobs))
    srv = serving.Server(pool, max_active=4, chunk_steps=3)
    srv.run(jobs)
    specs = {sp["id"]: sp for sp in I.serving_stream(12, seed=5, rate=400.0, edge2d=(24, 72), edge3d=(12, 24),
                                                         steps=(3, 14))}
    seen = set()
    for j in jobs:
        sp = specs[j.id]
        key = (sp["kind"], sp["precision"])
        if key in seen:
            continue
        seen.add(key)
        assert j.error is None
        orc = O.Oracle(dict(j.case, precision="fp64"), j.nodes)
        qo = j.q.copy()
        for _ in range(j.steps):
            qo = orc.rk3(qo, orc.dt(qo, j.cfl))
        nv = qo.shape[0]
        if sp["precision"] == "mixed":
            assert rel_state(j.result, qo) < 1e-5, key
        else:
            _, det = orc.cell_metrics()
            l1 = (np.abs(j.result - qo) * det).reshape(nv, -1).sum(axis=1) / (np.abs(qo) * det).reshape(nv, -1).sum(axis=1)
            assert l1.max() < 1e-8, key
            if sp["kind"] != "sod":
                assert rel_state(j.result, qo) < 1e-10, key
    assert {k[1] for k in seen} == {"fp64", "mixed"}
    srv.close()
