"""Continuous-batching server: each request's result is the same alone and in a
mix where requests arrive while others run and wait for pool memory, and it is
the same as a plain context run for the same number of sweeps (tolerance zero).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pt():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2506_14781_gb300 import build as b

    b.build()
    import paper_2506_14781_gb300 as m

    return m


INTERVAL, EVENTS_PER_STEP, MAX_SWEEPS = 5, 4, 600


def _requests(pt):
    out = []
    for k, (N, alpha) in enumerate([(14, 0.5), (30, 0.25), (22, 0.75), (40, 0.5), (18, 0.25), (55, 0.5)]):
        inst = synth.wishart_planted(N, alpha, 300 + k)
        phys = pt.sparsify(inst.Jq, "max_edges", 3)
        beta = synth.beta_ladder(8, 0.2, 3.0, inst.scale)
        P = synth.penalty_ladder(4, 0.5, 4.0, 32767)
        out.append(dict(phys=phys, beta=beta, P=P, seed=9000 + k, target=inst.E_planted, inst=inst))
    return out


def _drain(server, ids):
    for _ in range(10000):
        server.step()
        if all(server.status(i)["state"] == "done" for i in ids):
            return
    raise AssertionError("requests did not finish")


RESULT_KEYS = ("best_f", "best_event", "solved_event", "sweeps_done")


def test_result_alone_equals_result_in_mix(pt):
    reqs = _requests(pt)
    alone = []
    for r in reqs:
        srv = pt.Server(1 << 26, 3, 8, INTERVAL, EVENTS_PER_STEP)
        rid = srv.submit(r["phys"], r["beta"], r["P"], r["seed"], r["target"], MAX_SWEEPS)
        _drain(srv, [rid])
        alone.append(srv.status(rid, with_state=True))
        srv.close()
    # mixed: a pool that holds about three requests, arrivals while others run
    probe = pt.Batch(1 << 24, 3, 8, trace_capacity=0)
    sizes = [probe.instance_bytes(r["phys"], 8, 4, 1) for r in reqs]
    probe.close()
    srv = pt.Server(sum(sorted(sizes)[-3:]) + 4096, 3, 8, INTERVAL, EVENTS_PER_STEP)
    ids = [srv.submit(r["phys"], r["beta"], r["P"], r["seed"], r["target"], MAX_SWEEPS)
           for r in reqs[:3]]
    a, q, _ = srv.step()
    srv.step()
    ids += [srv.submit(r["phys"], r["beta"], r["P"], r["seed"], r["target"], MAX_SWEEPS)
            for r in reqs[3:]]
    _drain(srv, ids)
    for i, rid in enumerate(ids):
        got = srv.status(rid, with_state=True)
        for k in RESULT_KEYS:
            assert got[k] == alone[i][k], (i, k)
        assert np.array_equal(got["best_state"], alone[i]["best_state"]), i
        assert got["sweeps_done"] % (INTERVAL * EVENTS_PER_STEP) == 0
        stopped_early = got["solved_event"] >= 0
        assert stopped_early or got["sweeps_done"] >= MAX_SWEEPS
    # and each equals a plain context run for the same number of sweeps
    for i, rid in enumerate(ids):
        r = reqs[i]
        got = srv.status(rid, with_state=True)
        ctx = pt.PT2D(r["phys"], r["beta"], r["P"], 1, trace_capacity=0)
        ctx.write(pt.TARGET, [r["target"]])
        ctx.run(got["sweeps_done"], INTERVAL, r["seed"])
        assert ctx.read(pt.BEST_F)[0] == got["best_f"]
        assert ctx.read(pt.BEST_EVENT)[0] == got["best_event"]
        assert ctx.read(pt.SOLVED_EVENT)[0] == got["solved_event"]
        if got["best_event"] >= 0:
            assert np.array_equal(ctx.read(pt.BEST_STATE)[0], got["best_state"])
        ctx.close()


def test_fifo_admission_by_memory_and_cancel(pt):
    reqs = _requests(pt)
    probe = pt.Batch(1 << 24, 3, 8, trace_capacity=0)
    need = probe.instance_bytes(reqs[5]["phys"], 8, 4, 1)
    probe.close()
    srv = pt.Server(need + 1024, 3, 8, INTERVAL, EVENTS_PER_STEP)
    free0 = srv.free_bytes
    r1 = srv.submit(reqs[5]["phys"], reqs[5]["beta"], reqs[5]["P"], 1, reqs[5]["target"], 10**6)
    r2 = srv.submit(reqs[0]["phys"], reqs[0]["beta"], reqs[0]["P"], 2, reqs[0]["target"], 10**6)
    active, queued, _ = srv.step()
    assert (active, queued) == (1, 1)
    assert srv.status(r1)["state"] == "running" and srv.status(r2)["state"] == "queued"
    srv.cancel(r1)
    assert srv.status(r1)["state"] == "cancelled"
    assert srv.free_bytes == free0
    active, queued, _ = srv.step()
    assert (active, queued) == (1, 0) and srv.status(r2)["state"] == "running"
    srv.cancel(r2)
    srv.forget(r1)
    with pytest.raises(pt.Pt2dError):
        srv.status(r1)


def test_submit_rejects_what_can_never_run(pt):
    """A request larger than the whole pool is refused at submission (it would
    block the FIFO head for ever), and so is one a batch cannot hold."""
    reqs = _requests(pt)
    probe = pt.Batch(1 << 24, 3, 8, trace_capacity=0)
    need = probe.instance_bytes(reqs[5]["phys"], 8, 4, 1)
    probe.close()
    srv = pt.Server(need // 2, 3, 8, INTERVAL, EVENTS_PER_STEP)
    with pytest.raises(pt.Pt2dError) as e:
        srv.submit(reqs[5]["phys"], reqs[5]["beta"], reqs[5]["P"], 1, reqs[5]["target"], 100)
    assert "OOM" in str(e.value)
    small = reqs[0]
    rid = srv.submit(small["phys"], small["beta"], small["P"], 1, small["target"], 40)
    _drain(srv, [rid])
    lk_ptr, lk_col, lk_w, hk, g0 = pt.onehot_penalty(6, [[0, 1, 2], [3, 4, 5]])
    pen = pt.PhysicalInstance(6, np.zeros(7, np.int32), [], [], lk_ptr, lk_col, lk_w=lk_w, hk=hk, g0=g0)
    with pytest.raises(pt.Pt2dError):
        srv.submit(pen, small["beta"], small["P"], 1, 0, 40)
    srv.close()


def test_malformed_problem_fails_at_admission(pt):
    """Submission checks only the degrees and the size; a CSR that is not
    symmetric is caught when the request is admitted: it ends FAILED with
    INVALID_ARG, and the requests around it run to completion."""
    reqs = _requests(pt)
    srv = pt.Server(1 << 28, 3, 8, INTERVAL, EVENTS_PER_STEP)
    bad = pt.PhysicalInstance(4, np.array([0, 1, 1, 1, 1], np.int32), np.array([1], np.int32),
                              np.array([5], np.int16), np.zeros(5, np.int32), np.zeros(0, np.int32))
    before = srv.submit(reqs[0]["phys"], reqs[0]["beta"], reqs[0]["P"], 1, reqs[0]["target"], 40)
    rid = srv.submit(bad, reqs[0]["beta"], reqs[0]["P"], 2, 0, 40)
    after = srv.submit(reqs[1]["phys"], reqs[1]["beta"], reqs[1]["P"], 3, reqs[1]["target"], 40)
    assert srv.status(rid)["state"] == "queued"
    _drain(srv, [before, after])
    st = srv.status(rid)
    assert st["state"] == "failed" and st["error"] == -1  # PT2D_ERR_INVALID_ARG
    srv.close()


def test_requests_in_a_mix_match_the_oracle(pt):
    """Requests served in a mix (arrivals while others run, a pool that holds
    only some of them) give the oracle's result for the same instance, ladders
    and seed, run for the sweeps the server reports: best feasible f, the event
    it was found at, the solving event and the best state."""
    import oracle

    reqs = _requests(pt)
    probe = pt.Batch(1 << 24, 3, 8, trace_capacity=0)
    sizes = [probe.instance_bytes(r["phys"], 8, 4, 1) for r in reqs]
    probe.close()
    srv = pt.Server(sum(sorted(sizes)[-3:]) + 4096, 3, 8, INTERVAL, EVENTS_PER_STEP)
    ids = [srv.submit(r["phys"], r["beta"], r["P"], r["seed"], r["target"], MAX_SWEEPS) for r in reqs[:4]]
    srv.step()
    ids += [srv.submit(r["phys"], r["beta"], r["P"], r["seed"], r["target"], MAX_SWEEPS) for r in reqs[4:]]
    _drain(srv, ids)
    for k in (0, 3, 5):
        r, got = reqs[k], srv.status(ids[k], with_state=True)
        orc = oracle.OracleRun(oracle.OracleInstance(oracle.sparsify(r["inst"].Jq, "max_edges", 3)), r["beta"],
                               r["P"], [0], r["seed"], target=r["target"])
        orc.run(got["sweeps_done"], INTERVAL)
        assert got["best_f"] == orc.best_f[0], k
        assert got["best_event"] == orc.best_event[0], k
        assert got["solved_event"] == orc.solved_event[0], k
        if got["best_event"] >= 0:
            assert np.array_equal(got["best_state"], orc.best_state[0]), k
    srv.close()
