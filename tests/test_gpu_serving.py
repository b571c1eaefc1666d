"""Serving with continuous batching: requests admitted by slot and HBM
footprint run concurrently on per-slot streams; each result must be the same
alone and in the mix (bit for bit: every kernel sums in a fixed order), the
budget must hold, and the requests must really overlap on the device."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import to_dev_colmajor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    from paper_1205_3830_gb300 import build
    build.build()
    from paper_1205_3830_gb300 import serve
    return serve


def make_requests(count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        m, n = (int(x) for x in rng.integers(256, 1400, size=2))
        k = int(rng.integers(8, 40))
        A = synth.lowrank_plus_noise(m, n, k, 1e-10, seed=seed * 100 + i)
        reqs.append((i, A, k, k + 10, 500 + i))
    return reqs


@pytest.mark.parametrize("mode,select_ctas", [("fp64_emulated", None), ("fp64", None), ("fp64_emulated", 0)])
def test_served_results_equal_solo_results(serve, mode, select_ctas):
    # select_ctas = 0: the served selects run one launch per step; the solo
    # runs keep the default cooperative launch, and the bits must not change
    reqs = make_requests(10, seed=1)
    dev = {i: to_dev_colmajor(A) for (i, A, k, l, s) in reqs}
    solo = {i: serve.run_one(dev[i], k, l, s, mode=mode) for (i, A, k, l, s) in reqs}
    torch.cuda.synchronize()
    budget = 3 * max(serve.footprint(*A.shape, k, l, mode=mode) for (i, A, k, l, s) in reqs)
    srv = serve.Server(slots=4, hbm_budget=budget, mode=mode, select_ctas=select_ctas)
    try:
        handles = [srv.submit(i, dev[i], k, l, s) for (i, A, k, l, s) in reqs]
        done = srv.drain(timeout=300)
    finally:
        srv.close()
    assert len(done) == len(reqs)
    assert srv.peak_used <= budget
    assert srv.peak_running >= 2                    # the requests overlapped
    for h in handles:
        assert h.error is None, h.error
        a, b = h.result, solo[h.rid]
        assert torch.equal(a["perm"], b["perm"]) and torch.equal(a["T"], b["T"])
        assert a["est"] == b["est"] and a["upper"] == b["upper"]
    # and the served IDs are the oracle's
    for (i, A, k, l, s) in reqs[:3]:
        out = oracle.rid(A, k, l, seed=s)
        h = next(x for x in handles if x.rid == i)
        assert np.array_equal(h.result["perm"].numpy()[:k], out["J"])
        T = h.result["T"].numpy()
        assert np.abs(T - out["T"]).max() <= 1e-10 * np.abs(out["T"]).max()


def test_admission_waits_for_memory(serve):
    # five requests of one shape and a budget of one footprint: no two may overlap
    reqs = [(i, synth.lowrank_plus_noise(700, 500, 16, 1e-10, seed=300 + i), 16, 26, 700 + i) for i in range(5)]
    dev = {i: to_dev_colmajor(A) for (i, A, k, l, s) in reqs}
    biggest = max(serve.footprint(*A.shape, k, l) for (i, A, k, l, s) in reqs)
    srv = serve.Server(slots=4, hbm_budget=biggest)         # room for one request at a time
    try:
        for (i, A, k, l, s) in reqs:
            srv.submit(i, dev[i], k, l, s)
        done = srv.drain(timeout=300)
    finally:
        srv.close()
    assert len(done) == 5 and all(r.error is None for r in done)
    assert srv.peak_running == 1 and srv.peak_used <= biggest
    lat = serve.latency_stats(done)
    assert lat["p99_ms"] >= lat["p50_ms"] > 0


def test_reused_plans_give_the_bits_of_new_plans(serve):
    """Requests of repeated shapes take finished requests' plans from the pool
    (rid_plan_reseed, rid_plan_set_stream); every result is still bit for bit
    the solo result of a new plan with its own seed."""
    shapes = [(900, 700, 12), (600, 1100, 20)]
    reqs = []
    for i in range(12):
        m, n, k = shapes[i % 2]
        reqs.append((i, synth.lowrank_plus_noise(m, n, k, 1e-10, seed=900 + i), k, k + 10, 3000 + i))
    dev = {i: to_dev_colmajor(A) for (i, A, k, l, s) in reqs}
    solo = {i: serve.run_one(dev[i], k, l, s) for (i, A, k, l, s) in reqs}
    torch.cuda.synchronize()
    srv = serve.Server(slots=2)
    try:
        handles = [srv.submit(i, dev[i], k, l, s) for (i, A, k, l, s) in reqs]
        done = srv.drain(timeout=300)
    finally:
        srv.close()
    assert len(done) == len(reqs) and srv.reused >= len(reqs) - 4     # at most one new plan per slot and shape
    assert srv.used == 0 and not srv.idle                                # close() released the pool
    for h in handles:
        assert h.error is None, h.error
        a, b = h.result, solo[h.rid]
        assert torch.equal(a["perm"], b["perm"]) and torch.equal(a["T"], b["T"])
        assert a["est"] == b["est"] and a["upper"] == b["upper"]


def test_reseeded_plan_matches_new_plan(serve):
    import paper_1205_3830_gb300 as rid
    A = synth.lowrank_plus_noise(1500, 2300, 24, 1e-10, seed=77)
    Ad = to_dev_colmajor(A)
    for mode in ("fp64_emulated", "fp64"):
        outs = []
        with rid.Plan(1500, 2300, 24, 34, seed=1, mode=mode, nprobe=8, probe_seed=2) as plan:
            plan.reseed(5, 6)
            side = torch.cuda.Stream()
            plan.set_stream(side)
            with torch.cuda.stream(side):
                Y = plan.sketch(Ad)
                perm = plan.select(Y)
                T = plan.solve(Y)
                outs.append((perm.cpu(), T.cpu(), plan.error_sketched(perm, T)))
        with rid.Plan(1500, 2300, 24, 34, seed=5, mode=mode, nprobe=8, probe_seed=6) as plan:
            Y = plan.sketch(Ad)
            perm = plan.select(Y)
            T = plan.solve(Y)
            outs.append((perm.cpu(), T.cpu(), plan.error_sketched(perm, T)))
        (pa, Ta, ea), (pb, Tb, eb) = outs
        assert torch.equal(pa, pb) and torch.equal(Ta, Tb) and ea == eb, mode
