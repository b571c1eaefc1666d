"""Batched IDs (one persistent launch for many uneven problems) against the
CPU oracle and against the single-problem plan path.

Same tolerances as the plan path: J exactly, T within 1e-10 max|T| of the
oracle; against the plan path (same Omega, same FP64 algorithm, different
summation blocking in the sketch) T within 1e-12, and the plan path's error
pass on the batch's own (perm, T) gives its estimates within the FP64
rounding bound of E w~ (the estimate is a cancellation).  Results do not depend on the sketch tile or on which other
problems share the batch (bit for bit).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U64, to_dev_colmajor, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rid():
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    return rid


def make_problems(count, seed, m_range=(64, 420), n_range=(64, 420), k_range=(4, 24)):
    shapes = synth.batched_shapes(count, seed, m_range=m_range, n_range=n_range, k_range=k_range)
    probs = []
    for i, (m, n, k, l) in enumerate(shapes):
        A = synth.lowrank_plus_noise(m, n, k, 1e-10, seed=seed * 1000 + i)
        probs.append((A, k, l, 7000 + i))
    return probs


def test_batch_matches_oracle_and_plan_path(rid):
    probs = make_problems(24, seed=3)
    dev = [(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs]
    res = rid.batch_decompose(dev, nprobe=8, probe_seed=5)
    for (A, k, l, s), (Ad, _, _, _), r in zip(probs, dev, res):
        assert r["status"] == 0
        out = oracle.rid(A, k, l, seed=s)
        perm, T = to_host(r["perm"]), to_host(r["T"])
        assert np.array_equal(perm[:k], out["J"])
        if T.size:
            assert np.abs(T - out["T"]).max() <= 1e-10 * np.abs(out["T"]).max()
        one = rid.decompose(Ad, k, l, seed=s, mode="fp64", nprobe=8, probe_seed=5)
        assert torch.equal(one["perm"], r["perm"])
        if T.size:
            T1 = to_host(one["T"])
            assert np.abs(T - T1).max() <= 1e-12 * np.abs(T1).max()
        # the estimate cancels terms of size |A| |T| |w| down to ~1e-10: compare
        # the batch's estimate with the plan path's error pass on the same (perm, T)
        with rid.Plan(A.shape[0], A.shape[1], k, l, seed=s) as plan:
            est, up = plan.error(Ad, r["perm"], r["T"] if T.size else torch.empty((k, 0), dtype=torch.complex128).cuda(),
                                 8, 5)
        # rounding bound of two FP64 evaluations of E w~ (the estimate cancels
        # terms of size |A| |w~| down to ~1e-8 of that)
        n = A.shape[1]
        omega = oracle.probe_matrix(n, 8, 5)
        w_abs = np.abs(omega)
        if T.size:
            w_abs[perm[:k]] = np.abs(T) @ np.abs(omega[perm[k:]])
        bound_q = 2 * 4 * (n + k) * U64 * np.linalg.norm(np.abs(A) @ w_abs, axis=0)
        assert abs(r["est"] - est) <= np.max(bound_q / np.linalg.norm(omega, axis=0)) + 1e-14 * est
        assert abs(r["upper"] - up) <= 10 * np.sqrt(2 / np.pi) * np.max(bound_q) + 1e-14 * up


def test_batch_is_independent_of_tile_and_company(rid):
    probs = make_problems(12, seed=4)
    dev = [(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs]
    b = rid.Batch(dev, nprobe=4, probe_seed=1)
    r16 = [dict(x, T=x["T"].clone(), perm=x["perm"].clone()) for x in b.run(tile=16).results()]
    r32 = b.run(tile=32).results()
    for a, c in zip(r16, r32):
        assert torch.equal(a["perm"], c["perm"]) and torch.equal(a["T"], c["T"]) and a["est"] == c["est"]
    alone = rid.batch_decompose([dev[5]], nprobe=4, probe_seed=1)[0]
    assert torch.equal(alone["perm"], r32[5]["perm"]) and torch.equal(alone["T"], r32[5]["T"])
    assert alone["est"] == r32[5]["est"]


def test_batch_reports_rank_deficiency_per_problem(rid):
    probs = make_problems(5, seed=6)
    A0 = np.zeros((100, 80), dtype=np.complex128)
    A0[:, 3] = 1.0                       # rank 1
    dev = [(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs] + [(to_dev_colmajor(A0), 4, 8, 1)]
    res = rid.batch_decompose(dev)
    assert [r["status"] for r in res[:5]] == [0] * 5
    assert res[5]["status"] == 4 and res[5]["est"] == -1.0


def test_batch_autotune_picks_a_tile(rid):
    probs = make_problems(16, seed=8)
    b = rid.Batch([(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs])
    tile, ms = b.autotune()
    assert tile in (16, 32) and ms > 0


def test_batch_graph_replay_equals_direct_launch(rid):
    """The prepared batch captured in a CUDA graph: replays give the direct
    launch's results bit for bit, and a replay after the outputs were wiped
    writes them again."""
    probs = make_problems(10, seed=9)
    dev = [(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs]
    b = rid.Batch(dev, nprobe=6, probe_seed=2)
    ref = [dict(x, T=x["T"].clone(), perm=x["perm"].clone()) for x in b.run(tile=32).results()]
    b.capture(tile=32)
    for rep in range(2):
        for t in b.T:
            t.zero_()
        b.err.zero_()
        b.replay()
        got = b.results()
        for a, c in zip(ref, got):
            assert torch.equal(a["perm"], c["perm"]) and torch.equal(a["T"], c["T"])
            assert a["est"] == c["est"] and a["upper"] == c["upper"] and c["status"] == 0


# ---- the tensor-core batch (rid_batch_tc_*) ---------------------------------------------
def test_batch_tc_matches_oracle_and_plan_path(rid):
    """Every problem's sketch on its own FP64-emulated plan, select / solve /
    row-probe error in one launch: J as the oracle's, T within 1e-10, the
    estimate within the row-probe rounding bound of the oracle's, and J, T as
    the problem's own plan gives them."""
    from gpu_util import row_probe_tolerances
    probs = make_problems(20, seed=11)
    dev = [(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs]
    b = rid.BatchTC(dev, nprobe=8, probe_seed=1)
    res = b.run().results()
    for (A, k, l, s), r, (Ad, _, _, _) in zip(probs, res, dev):
        assert r["status"] == 0
        out = oracle.rid(A, k, l, seed=s)
        perm, T = to_host(r["perm"]), to_host(r["T"])
        assert np.array_equal(perm[:k], out["J"])
        if T.size:
            assert np.abs(T - out["T"]).max() <= 1e-10 * np.abs(out["T"]).max()
        G = oracle.left_probe_matrix(8, A.shape[0], 1)
        est_o, up_o, _ = oracle.error_estimate_left(A, perm, T, G)
        tol_est, tol_up = row_probe_tolerances(A, perm, T, G, "fp64_emulated")
        assert abs(r["est"] - est_o) <= tol_est + 1e-14 * est_o
        assert abs(r["upper"] - up_o) <= tol_up + 1e-14 * up_o
        with rid.Plan(A.shape[0], A.shape[1], k, l, seed=s, mode="fp64_emulated") as plan:
            plan.set_probes(8, 1)
            Y = plan.sketch(Ad)
            pp = plan.select(Y)
            Tp = plan.solve(Y)
            assert torch.equal(pp, r["perm"])
            if T.size:
                assert (Tp - r["T"]).abs().max().item() <= 1e-12 * Tp.abs().max().item()
    b.close()


def test_batch_tc_replays_and_reports_rank_deficiency(rid):
    probs = make_problems(6, seed=12)
    A0 = np.zeros((100, 80), dtype=np.complex128)
    A0[:, 3] = 1.0                       # rank 1
    dev = [(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs] + [(to_dev_colmajor(A0), 4, 8, 1)]
    b = rid.BatchTC(dev, nprobe=4, probe_seed=2)
    first = [dict(x, T=x["T"].clone(), perm=x["perm"].clone()) for x in b.run().results()]
    second = b.run().results()
    for a, c in zip(first[:6], second[:6]):
        assert torch.equal(a["perm"], c["perm"]) and torch.equal(a["T"], c["T"])
        assert a["est"] == c["est"] and a["status"] == c["status"] == 0
    assert second[6]["status"] == 4 and second[6]["est"] == -1.0
    b.close()


def test_batch_tc_is_independent_of_tiles_waves_and_company(rid):
    """The persistent tensor-core sketch: the N-tile width, the number of
    waves (a small digit buffer forces one problem or two per wave) and the
    other problems of the batch change nothing, bit for bit; a K-split moves
    T by rounding only."""
    probs = make_problems(14, seed=21, m_range=(64, 700), n_range=(64, 420), k_range=(4, 40))
    dev = [(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs]

    def run(**kw):
        b = rid.BatchTC(dev if "sub" not in kw else kw.pop("sub"), nprobe=8, probe_seed=3, **kw)
        res = [dict(x, T=x["T"].clone(), perm=x["perm"].clone()) for x in b.run().results()]
        info = b.info()
        b.close()
        return res, info

    ref, info0 = run()
    assert info0["waves"] == 1
    narrow, _ = run(tile_n=64)
    waves, info_w = run(wave_bytes=1 << 20)
    assert info_w["waves"] >= 4 and info_w["bytes"] < info0["bytes"]
    for a, b2, c in zip(ref, narrow, waves):
        assert a["status"] == b2["status"] == c["status"] == 0
        for x in (b2, c):
            assert torch.equal(a["perm"], x["perm"]) and torch.equal(a["T"], x["T"])
            assert a["est"] == x["est"] and a["upper"] == x["upper"]
    alone, _ = run(sub=[dev[4]])
    assert torch.equal(alone[0]["perm"], ref[4]["perm"]) and torch.equal(alone[0]["T"], ref[4]["T"])
    assert alone[0]["est"] == ref[4]["est"]
    split, _ = run(ksplit=2)
    from gpu_util import row_probe_tolerances
    for (A, k, l, s), a, x in zip(probs, ref, split):
        assert torch.equal(a["perm"], x["perm"])
        if a["T"].numel():
            assert (a["T"] - x["T"]).abs().max().item() <= 1e-12 * a["T"].abs().max().item()
        # the estimate cancels down to ~1e-8 of |G| |A|: two sketches' rounding
        # moves it by up to twice the row-probe bound
        perm, T = to_host(a["perm"]), to_host(a["T"])
        G = oracle.left_probe_matrix(8, A.shape[0], 3)
        tol_est, _ = row_probe_tolerances(A, perm, T, G, "fp64_emulated")
        assert abs(a["est"] - x["est"]) <= 2 * tol_est + 1e-14 * a["est"]


def test_batch_tc_tall_problems_with_k_splits_match_oracle(rid):
    """Tall problems (many 256-real chunks per column) split over K: J as the
    oracle's, T within 1e-10, est within the row-probe bound."""
    from gpu_util import row_probe_tolerances
    shapes = [(5000, 130, 6, 14), (3000, 64, 10, 18), (4100, 200, 20, 28)]
    probs = [(synth.lowrank_plus_noise(m, n, k, 1e-10, seed=40 + i), k, l, 900 + i) for i, (m, n, k, l) in enumerate(shapes)]
    dev = [(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs]
    b = rid.BatchTC(dev, nprobe=6, probe_seed=2, ksplit=[4, 8, 3], tile_n=[0, 64, 96])
    res = b.run().results()
    for (A, k, l, s), r in zip(probs, res):
        assert r["status"] == 0
        out = oracle.rid(A, k, l, seed=s)
        perm, T = to_host(r["perm"]), to_host(r["T"])
        assert np.array_equal(perm[:k], out["J"])
        assert np.abs(T - out["T"]).max() <= 1e-10 * np.abs(out["T"]).max()
        G = oracle.left_probe_matrix(6, A.shape[0], 2)
        est_o, up_o, _ = oracle.error_estimate_left(A, perm, T, G)
        tol_est, tol_up = row_probe_tolerances(A, perm, T, G, "fp64_emulated")
        assert abs(r["est"] - est_o) <= tol_est + 1e-14 * est_o
        assert abs(r["upper"] - up_o) <= tol_up + 1e-14 * up_o
    b.close()


def test_batch_tc_argument_checks(rid):
    from paper_1205_3830_gb300._native import RIDError
    probs = make_problems(2, seed=22)
    dev = [(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs]
    for bad in (8, 130, 100):
        with pytest.raises(RIDError, match="EINVAL"):
            rid.BatchTC(dev, nprobe=4, tile_n=bad)
    with pytest.raises(RIDError, match="EINVAL"):
        rid.BatchTC(dev, nprobe=4, ksplit=-1)


def test_tc_tuning_picks_and_caches_a_choice_per_class(rid, tmp_path):
    probs = make_problems(24, seed=23, m_range=(64, 700), n_range=(64, 300), k_range=(4, 30))
    dev = [(to_dev_colmajor(A), k, l, s) for (A, k, l, s) in probs]
    path = str(tmp_path / "tc_tiles.json")
    tun = rid.TcTuning(path)
    report = tun.tune(dev, nprobe=8, probe_seed=1, per_class=8, reps=1)
    classes = {rid.TcTuning.size_class(int(A.shape[0]), int(A.shape[1]), l + 8) for (A, k, l, s) in dev}
    assert set(report) == classes
    for key, (t, s, ms) in report.items():
        assert (t, s) in rid.TcTuning.candidates(key) and ms > 0
    again = rid.TcTuning(path)                    # read back from the cache file
    assert again.table == tun.table
    b = rid.BatchTC(dev, nprobe=8, probe_seed=1, tuning=again)
    for r, (A, k, l, s) in zip(b.run().results(), probs):
        assert r["status"] == 0
        assert np.array_equal(to_host(r["perm"])[:k], oracle.rid(A, k, l, seed=s)["J"])
    b.close()


@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (1, 50, 1, 5), (50, 1, 1, 3), (777, 129, 64, 64),
                                   (300, 4096, 64, 128), (20000, 200, 10, 20)], ids=str)
def test_batch_tc_edge_shapes_match_oracle(rid, shape):
    """Degenerate and extreme problems in one batch with ordinary ones: one
    row, one column, k = l, the largest n, k and l the batch takes (3 N-tiles
    of Omega' rows), and a tall problem of 157 chunks."""
    from gpu_util import row_probe_tolerances
    m, n, k, l = shape
    probs = [(synth.lowrank_plus_noise(m, n, k, 1e-10, seed=60 + m + n), k, l, 4242)] + \
        make_problems(3, seed=24)
    dev = [(to_dev_colmajor(A), kk, ll, s) for (A, kk, ll, s) in probs]
    b = rid.BatchTC(dev, nprobe=8, probe_seed=3)
    res = b.run().results()
    for (A, kk, ll, s), r in zip(probs, res):
        assert r["status"] == 0
        out = oracle.rid(A, kk, ll, seed=s)
        perm, T = to_host(r["perm"]), to_host(r["T"])
        assert np.array_equal(perm[:kk], out["J"])
        assert sorted(perm.tolist()) == list(range(A.shape[1]))
        if T.size:
            # two FP64 evaluations differ in rounding by ~u per entry of Y; the
            # triangular solve amplifies that by kappa(R11) (large for k = l,
            # where R11 comes from a square sketch): first-order bound
            # 8 l sqrt(n) u kappa(R11), at least the 1e-10 of the other tests
            kappa = np.linalg.cond(np.triu(out["R"][:kk, :kk]))
            tol_T = max(1e-10, 8 * ll * np.sqrt(A.shape[1]) * 2.0 ** -53 * kappa)
            assert np.abs(T - out["T"]).max() <= tol_T * np.abs(out["T"]).max()
            G = oracle.left_probe_matrix(8, A.shape[0], 3)
            est_o, up_o, _ = oracle.error_estimate_left(A, perm, T, G)
            tol_est, tol_up = row_probe_tolerances(A, perm, T, G, "fp64_emulated")
            assert abs(r["est"] - est_o) <= tol_est + 1e-14 * est_o
        else:
            assert r["est"] == 0.0 and r["upper"] == 0.0
    b.close()
