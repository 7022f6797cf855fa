"""Serving loop: continuous batching of independent simulations.  Every
result must equal the same simulation run alone, requests that arrive while
others run must be admitted as slots and memory free up, and the memory
budget must be respected."""
import numpy as np
import pytest

from paper_1611_08536_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_08536_gb300 import build, drts
    build.build()
    drts.load()
    return drts


def rel_l1(a, b):
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


def small_stream(n, seed=11):
    return [I.served_request(seed, i, sides=(8, 12, 16), steps=(20, 60), max_sources=4)
            for i in range(n)]


def run_alone(gpu, req):
    with gpu.Context(req.problem, max_steps=req.n_steps) as ctx:
        prof = req.sources[0]
        for r, s in enumerate(req.sources):
            ctx.inject_source(r, s.state, s.weight, prof.t0, prof.profile)
        ctx.step_n(req.n_steps)
        out = [ctx.read_detectors(r) for r in range(len(req.sources))]
    return out


def test_server_results_equal_alone_and_admit_while_running(gpu):
    reqs = small_stream(7)
    with gpu.Server(max_resident=3, steps_per_tick=7, n_streams=3) as srv:
        ids = [srv.submit(reqs[0].problem, reqs[0].sources, reqs[0].n_steps),
               srv.submit(reqs[1].problem, reqs[1].sources, reqs[1].n_steps)]
        srv.tick()                                  # admits the first two
        assert srv.stats()["failed"] == 0
        assert srv.stats()["resident"] == 2
        for r in reqs[2:]:                          # arrive while those run
            ids.append(srv.submit(r.problem, r.sources, r.n_steps))
        seen_mixed = False
        for _ in range(500):
            srv.tick()
            st = srv.stats()
            states = [srv.poll(i).state for i in ids]
            if gpu.REQ_DONE in states and gpu.REQ_RUNNING in states:
                seen_mixed = True
            assert st["resident"] <= 3
            if st["completed"] + st["failed"] == len(ids):
                break
        st = srv.stats()
        assert st["completed"] == len(ids) and st["failed"] == 0
        assert seen_mixed                           # continuous batching, not one batch
        # every tick launched one graph; ticks with the same resident set
        # updated the kept executable graph instead of instantiating one
        assert st["graph_updates"] + st["graph_instantiations"] == st["graph_launches"]
        assert st["graph_updates"] >= 1 and st["host_graph_s"] > 0.0
        for rid, req in zip(ids, reqs):
            alone = run_alone(gpu, req)
            for r in range(len(req.sources)):
                det, led = srv.result(rid, r)
                d0, l0 = alone[r]
                assert rel_l1(det, d0) < 1e-6, (rid, r)
                assert np.allclose(led, l0, rtol=1e-6, atol=1e-12), (rid, r, led, l0)
            info = srv.poll(rid)
            assert info.latency_s >= info.queue_s >= 0.0
            srv.release(rid)


def test_server_memory_budget_limits_residency(gpu):
    reqs = small_stream(4, seed=3)
    probe = gpu.Server(max_resident=8, steps_per_tick=5, n_streams=2)
    rid = probe.submit(reqs[0].problem, reqs[0].sources, reqs[0].n_steps)
    fp = max(probe.poll(rid).footprint_bytes, 1)
    probe.close()
    biggest = 0
    with gpu.Server(mem_budget_bytes=int(fp * 1.5), max_resident=8, steps_per_tick=5, n_streams=2) as srv:
        ids = []
        for r in reqs:
            try:
                ids.append(srv.submit(r.problem, r.sources, r.n_steps))
            except gpu.DrtsError as e:
                assert e.status == gpu.ENOMEM          # larger than the whole budget
        for _ in range(500):
            srv.tick()
            st = srv.stats()
            assert st["used_bytes"] <= st["budget_bytes"]
            biggest = max(biggest, st["resident"])
            if st["completed"] + st["failed"] == len(ids):
                break
        assert srv.stats()["completed"] == len(ids)
    assert biggest >= 1


def test_server_stats_count_submissions_before_a_tick(gpu):
    """A request is counted as queued as soon as it is submitted (a serving
    loop that waits for queued work must see it before the next tick)."""
    reqs = small_stream(2, seed=5)
    with gpu.Server(max_resident=1, steps_per_tick=10, n_streams=2) as srv:
        assert srv.stats()["queued"] == 0
        ids = [srv.submit(r.problem, r.sources, r.n_steps) for r in reqs]
        st = srv.stats()
        assert st["queued"] == 2 and st["resident"] == 0 and st["submitted"] == 2
        srv.tick()                                     # admits one (one slot)
        st = srv.stats()
        assert st["resident"] == 1 and st["queued"] == 1 and st["used_bytes"] > 0
        while srv.stats()["completed"] < 2:
            srv.tick()
        st = srv.stats()
        assert st["resident"] == 0 and st["queued"] == 0 and st["used_bytes"] == 0
        for i in ids:
            assert srv.poll(i).state == gpu.REQ_DONE


@pytest.mark.parametrize("policy,order", [(0, [0, 1, 2]), (1, [1, 2, 0])])
def test_server_admission_policy(gpu, policy, order):
    """One slot, three requests queued together (steps 60, 20, 40): arrival
    order is kept by DRTS_SERVE_FIFO; DRTS_SERVE_SHORTEST_FIRST runs the least
    work first.  Results are the same either way."""
    base = small_stream(1, seed=3)[0]
    steps = [60, 20, 40]
    with gpu.Server(max_resident=1, steps_per_tick=10, n_streams=1, policy=policy) as srv:
        ids = [srv.submit(base.problem, base.sources, n) for n in steps]
        done = []
        while len(done) < 3:
            srv.tick()
            for k, i in enumerate(ids):
                if k not in done and srv.poll(i).state == gpu.REQ_DONE:
                    done.append(k)
        assert done == order
        det = srv.result(ids[1])[0]
    alone = run_alone(gpu, type(base)(base.arrival_s, base.problem, base.sources, 20))
    assert rel_l1(det, alone[0][0]) < 1e-6


def test_server_rejects_unknown_policy(gpu):
    with pytest.raises(gpu.DrtsError):
        gpu.Server(policy=7)


def test_server_results_match_oracle(gpu, oracle_mod):
    """Every source of every served request stays within relative L1 1e-4 of
    the FP64 oracle (Eq. 26 stepped on the same problem, Eq. 27 detectors and
    the energy ledger), with the requests overlapping on the device: three
    resident slots, requests submitted while others run, the tick graph
    fanned over three streams, and the batched step for the requests with
    several sources."""
    reqs = [I.served_request(17, i, sides=(8, 12, 16), steps=(100, 300), max_sources=6)
            for i in range(6)]
    assert any(len(r.sources) > 1 for r in reqs)
    with gpu.Server(max_resident=3, steps_per_tick=25, n_streams=3, keep_state=True) as srv:
        ids = [srv.submit(reqs[0].problem, reqs[0].sources, reqs[0].n_steps)]
        srv.tick()
        ids += [srv.submit(r.problem, r.sources, r.n_steps) for r in reqs[1:]]
        for _ in range(1000):
            srv.tick()
            st = srv.stats()
            if st["completed"] + st["failed"] == len(ids):
                break
        assert srv.stats()["completed"] == len(ids)
        worst = 0.0
        for rid, req in zip(ids, reqs):
            prob = req.problem
            csr = oracle_mod.assemble(prob)
            colinfo = oracle_mod.column_info(prob)
            prof = req.sources[0]
            for r, s in enumerate(req.sources):
                xo, deto, ledo = oracle_mod.run(prob, csr, req.n_steps,
                                                (s.state, s.weight, prof.t0, prof.profile),
                                                colinfo=colinfo)
                x = srv.result_state(rid, r, n_states=prob.n_states)
                det, led = srv.result(rid, r)
                ex = rel_l1(x, xo)
                ed = rel_l1(det, deto[:, :det.shape[1]])
                worst = max(worst, ex, ed)
                assert ex <= 1e-4, (rid, r, ex)
                assert ed <= 1e-4, (rid, r, ed)
                assert np.allclose(led, ledo, rtol=1e-4, atol=1e-12), (rid, r, led, ledo)
        with pytest.raises(gpu.DrtsError):
            srv.result_state(ids[0], len(reqs[0].sources), n_states=reqs[0].problem.n_states)
    print(f"served vs oracle: worst relative L1 {worst:.2e}")


def test_server_result_state_needs_keep_state(gpu):
    req = small_stream(1, seed=9)[0]
    with gpu.Server(max_resident=1, steps_per_tick=50, n_streams=1) as srv:
        rid = srv.submit(req.problem, req.sources, req.n_steps)
        while srv.stats()["completed"] < 1:
            srv.tick()
        with pytest.raises(gpu.DrtsError) as e:
            srv.result_state(rid, 0, n_states=req.problem.n_states)
        assert e.value.status == gpu.ESTATE


def test_server_cancel_queued_and_running(gpu):
    """A queued request cancelled leaves the queue; a running one is stopped
    between ticks and its footprint returns to the budget; the others finish
    with the results they have alone.  Neither cancelled request has
    results, a finished one cannot be cancelled, and cancelled ones can be
    released."""
    reqs = small_stream(3, seed=5)
    for r in reqs:
        r.n_steps = 60
    with gpu.Server(max_resident=2, steps_per_tick=5, n_streams=2) as srv:
        ids = [srv.submit(r.problem, r.sources, r.n_steps) for r in reqs]
        srv.tick()                                   # admits the first two
        srv.tick()                                   # they step
        assert srv.poll(ids[0]).state == gpu.REQ_RUNNING
        assert srv.poll(ids[1]).state == gpu.REQ_RUNNING
        assert srv.poll(ids[2]).state == gpu.REQ_QUEUED
        used = srv.stats()["used_bytes"]
        srv.cancel(ids[2])                           # queued
        assert srv.poll(ids[2]).state == gpu.REQ_CANCELLED
        assert srv.stats()["queued"] == 0
        srv.cancel(ids[0])                           # running
        assert srv.poll(ids[0]).state == gpu.REQ_CANCELLED
        st = srv.stats()
        assert st["resident"] == 1 and st["cancelled"] == 2
        assert st["used_bytes"] == used - srv.poll(ids[0]).footprint_bytes
        for _ in range(100):
            srv.tick()
            if srv.poll(ids[1]).state == gpu.REQ_DONE:
                break
        assert srv.poll(ids[1]).state == gpu.REQ_DONE
        alone = run_alone(gpu, reqs[1])
        for r in range(len(reqs[1].sources)):
            det, led = srv.result(ids[1], r)
            assert rel_l1(det, alone[r][0]) < 1e-12
            assert np.allclose(led, alone[r][1], rtol=1e-12)
        for i in (ids[0], ids[2]):
            with pytest.raises(gpu.DrtsError) as e:
                srv.result(i)
            assert e.value.status == gpu.ESTATE
        with pytest.raises(gpu.DrtsError) as e:
            srv.cancel(ids[1])                       # already finished
        assert e.value.status == gpu.ESTATE
        srv.release(ids[0])
        srv.release(ids[2])
        st = srv.stats()
        assert st["completed"] == 1 and st["failed"] == 0 and st["used_bytes"] == 0
