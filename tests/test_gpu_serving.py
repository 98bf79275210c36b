"""Serving loop (continuous batching of cooling runs): each request gives the same result
alone and in a mix of concurrent requests, admission respects the memory budget, and the
loop reports per-step latency percentiles."""
import numpy as np
import pytest

from paper_2409_05285_gb300 import binding

pytestmark = pytest.mark.gpu

REQS = [  # (L1, L2, D, chi, n_chains, J2, t_end, seed)
    (3, 3, 2, 4, 64, 0.0, 0.06, 1),
    (4, 4, 2, 4, 48, 0.3, 0.04, 2),
    (3, 4, 3, 6, 32, 0.5, 0.06, 3),
    (4, 3, 2, 3, 40, 0.2, 0.02, 4),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


def _run(reqs, max_active, budget=0):
    srv = binding.Server(hbm_budget=budget, max_active=max_active, blocks_per_request=8)
    ids = [srv.submit(L1, L2, D, chi, n, t_end=te, J2=J2, seed=sd, init_noise=1e-2)
           for (L1, L2, D, chi, n, J2, te, sd) in reqs]
    srv.drain()
    out = []
    for rid in ids:
        state, steps = srv.poll(rid)
        assert state == binding.PEPS_REQ_DONE
        out.append((srv.theta(rid), steps))
    m = srv.metrics()
    srv.close()
    return out, m


def test_results_identical_alone_and_in_the_mix():
    alone = [_run([r], 1)[0][0] for r in REQS]
    mix, m = _run(REQS, max_active=4)
    for (th_a, st_a), (th_m, st_m), r in zip(alone, mix, REQS):
        assert np.array_equal(th_a, th_m), r
        assert len(st_a) == len(st_m) == int(round(r[6] / 0.02))
        for a, b in zip(st_a, st_m):
            assert a["E_site"] == b["E_site"] and a["cg_iters"] == b["cg_iters"]
    assert m["steps"] == sum(int(round(r[6] / 0.02)) for r in REQS)
    assert 0 < m["p50_ms"] <= m["p99_ms"] and m["samples_per_s"] > 0


def test_admission_by_memory_budget():
    # a budget that holds one request at a time still serves every request, in order
    lib = binding.load()
    fps = []
    for (L1, L2, D, chi, n, J2, te, sd) in REQS:
        P = binding.Params(L1=L1, L2=L2, model=0, J1=1.0, J2=J2, D=D, chi=chi, n_chains=n,
                           precision=0, init_noise=1e-2, seed=sd, n_blocks=8, block_mode=0)
        fps.append(lib.peps_footprint(P))
    assert min(fps) > 0
    tight, _ = _run(REQS, max_active=4, budget=max(fps) + 1)
    free, _ = _run(REQS, max_active=4)
    for (a, _), (b, _) in zip(tight, free):
        assert np.array_equal(a, b)


def test_submit_rejects_invalid_and_oversized_requests():
    srv = binding.Server(hbm_budget=1 << 20, max_active=2)
    with pytest.raises(binding.PepsError):
        srv.submit(1, 4, 2, 4, 8, t_end=0.02)          # invalid lattice
    with pytest.raises(binding.PepsError):
        srv.submit(8, 8, 4, 16, 4096, t_end=0.02)      # footprint above the budget
    srv.close()


def test_stop_cancels_queued_and_ends_running_requests():
    # a request that would run for many steps and a queue behind it (one slot): stop ends
    # the running one after a finished step and cancels the queued ones; the finished steps
    # stay in the statistics, and later submissions are refused
    import time
    srv = binding.Server(max_active=1, blocks_per_request=8)
    long_id = srv.submit(4, 4, 2, 4, 64, t_end=50.0, seed=7)
    queued = [srv.submit(3, 3, 2, 4, 32, t_end=0.04, seed=8 + k) for k in range(3)]
    t0 = time.time()
    while srv.poll(long_id)[0] == binding.PEPS_REQ_RUNNING and len(srv.poll(long_id)[1]) < 2:
        assert time.time() - t0 < 60
        time.sleep(0.05)
    srv.stop()
    srv.drain()
    st, steps = srv.poll(long_id)
    assert st == binding.PEPS_REQ_CANCELLED and 2 <= len(steps) < 2500
    for rid in queued:
        assert srv.poll(rid)[0] == binding.PEPS_REQ_CANCELLED
    m = srv.metrics()
    assert m["steps"] == len(steps) and m["p50_ms"] > 0
    with pytest.raises(binding.PepsError):
        srv.submit(3, 3, 2, 4, 32, t_end=0.04, seed=1)
    srv.close()
