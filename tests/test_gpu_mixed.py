"""Mixed-precision sketch (complex64 A, BF16x3 splits, FP32 accumulation on the
tensor cores) against the FP64 oracle run on the same A (upcast exactly).

Stated accuracy: the sketch is FP32-grade, |Y - Y_FP64| <= 2^-16 ||Omega_i|| ||A_j||
per entry (three BF16 terms carry about 24 bits of every value; the FP32 sums
over the K range add the rest); the ID keeps the FP64 oracle's J whenever the
spectral gap exceeds that noise, and T within 1e-3 of the oracle.  The QR,
solve and error estimate after the sketch are FP64.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U64, row_probe_tolerances, to_dev_colmajor, to_host

pytestmark = pytest.mark.gpu

SHAPES = [(2048, 1024, 32, 42), (1000, 777, 17, 27), (4096, 333, 5, 15), (300, 200, 100, 110)]


@pytest.fixture(scope="module")
def rid():
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    return rid


def c64_lowrank(m, n, k, eps=1e-5, seed=0):
    return np.asfortranarray(synth.lowrank_plus_noise(m, n, k, eps, seed=seed + m + n).astype(np.complex64))


@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_mixed_sketch_accuracy(rid, shape):
    m, n, k, l = shape
    A = c64_lowrank(m, n, k)
    Oo = oracle.gaussian_test_matrix(l, m, 3)
    with rid.Plan(m, n, k, l, seed=3, dtype=torch.complex64, mode="bf16") as plan:
        plan.set_omega(torch.from_numpy(Oo).cuda())
        Y = to_host(plan.sketch(to_dev_colmajor(A, torch.complex64)))
        plan.sync_status()
    Yo = oracle.randomize(Oo, A.astype(np.complex128))
    scale = np.outer(np.linalg.norm(Oo, axis=1), np.linalg.norm(A.astype(np.complex128), axis=0))
    rel = np.abs(Y - Yo) / scale
    print(f"mixed sketch {shape}: max |dY| / (||Omega_i|| ||A_j||) = {rel.max():.2e}")
    assert rel.max() <= 2.0 ** -16


@pytest.mark.parametrize("shape", SHAPES[:3], ids=str)
def test_mixed_whole_id_against_fp64_oracle(rid, shape):
    m, n, k, l = shape
    A = c64_lowrank(m, n, k)
    out = oracle.rid(A.astype(np.complex128), k, l, seed=11)
    res = rid.decompose(to_dev_colmajor(A, torch.complex64), k, l, seed=11, mode="bf16", nprobe=8, probe_seed=2)
    perm, T = to_host(res["perm"]), to_host(res["T"])
    assert np.array_equal(perm[:k], out["J"])
    dT = np.abs(T - out["T"]).max() / np.abs(out["T"]).max()
    print(f"mixed ID {shape}: max |dT| / max |T| = {dT:.2e}")
    assert dT <= 1e-3


def test_mixed_error_estimate_is_fp64(rid):
    """The error pass on complex64 A computes in FP64: same as the oracle on the
    upcast A within the FP64 rounding bound."""
    m, n, k, l = 1500, 600, 12, 20
    A = c64_lowrank(m, n, k, eps=1e-4)
    A128 = A.astype(np.complex128)
    out = oracle.rid(A128, k, l, seed=4)
    omega = oracle.probe_matrix(n, 8, 9)
    est_o, up_o, _ = oracle.error_estimate(A128, out["perm"], out["T"], omega)
    with rid.Plan(m, n, k, l, seed=4, dtype=torch.complex64, mode="bf16") as plan:
        est, up = plan.error(to_dev_colmajor(A, torch.complex64), torch.from_numpy(out["perm"].astype(np.int32)).cuda(),
                             to_dev_colmajor(out["T"]), 8, 9)
    w_abs = np.abs(omega)
    w_abs[out["perm"][:k]] = np.abs(out["T"]) @ np.abs(omega[out["perm"][k:]])
    bound = 4 * (n + k) * U64 * np.linalg.norm(np.abs(A128) @ w_abs, axis=0)
    assert abs(est - est_o) <= np.max(bound / np.linalg.norm(omega, axis=0)) + 1e-13 * est_o


@pytest.mark.parametrize("shape", [(4096, 600, 20, 30), (1000, 777, 17, 27)], ids=str)
def test_mixed_row_probe_estimate_is_fp64(rid, shape):
    """Row probes on a mixed plan: Y takes the BF16x3 product, X = G A the
    FP64-emulated one on the complex64 A (exact in FP64), so the estimate
    meets the FP64 row-probe bound against the oracle on the upcast A."""
    m, n, k, l = shape
    A = c64_lowrank(m, n, k)
    with rid.Plan(m, n, k, l, seed=4, dtype=torch.complex64, mode="bf16") as plan:
        plan.set_probes(8, 6)
        Y = plan.sketch(to_dev_colmajor(A, torch.complex64))
        perm = plan.select(Y)
        T = plan.solve(Y)
        est, up = plan.error_sketched(perm, T)
    A128 = A.astype(np.complex128)
    perm_h, T_h = to_host(perm), to_host(T)
    G = oracle.left_probe_matrix(8, m, 6)
    est_o, up_o, _ = oracle.error_estimate_left(A128, perm_h, T_h, G)
    tol_est, tol_up = row_probe_tolerances(A128, perm_h, T_h, G, "fp64_emulated")
    assert abs(est - est_o) <= tol_est + 1e-14 * est_o
    assert abs(up - up_o) <= tol_up + 1e-14 * up_o
    assert est_o > 100 * tol_est


@pytest.mark.parametrize("shape", [(2048, 1000, 20, 30), (700, 2100, 10, 16)], ids=str)
def test_mixed_panels_equal_one_sketch(rid, shape):
    """Column panels of a mixed plan (BF16x3 Y and the FP64-emulated row
    probes), sketched out of order, give the one-call Y and estimate bit for
    bit."""
    m, n, k, l = shape
    A = to_dev_colmajor(c64_lowrank(m, n, k), torch.complex64)
    with rid.Plan(m, n, k, l, seed=9, dtype=torch.complex64, mode="bf16") as plan:
        plan.set_probes(8, 2)
        Y0 = plan.sketch(A).clone()
        R = Y0.clone()
        perm = plan.select(R)
        T = plan.solve(R)
        e0 = plan.error_sketched(perm, T)
        Y1 = torch.full_like(Y0, float("nan"))
        starts = list(range(0, n, 384))
        for c0 in reversed(starts):
            plan.sketch_cols(A, Y1, c0, min(384, n - c0))
        e1 = plan.error_sketched(perm, T)
    assert torch.equal(Y0, Y1)
    assert e0 == e1


# ---- the accuracy floor of the mixed mode ---------------------------------------
# A sweep of the spectral gap sigma_{k+1} / sigma_1 from 1e-2 to 1e-9 on a
# complex64 A with a prescribed spectrum.  At every point the mixed ID is
# compared with the FP64 oracle on the same (upcast) A: J, T and the exact
# error ||A - A(:, J) P||_2 of both.  The plan's own accuracy check
# (rid_plan_accuracy) must accept exactly where the mixed result is as good as
# the FP64 path's: J equal and an ID error within twice the FP64 path's.
FLOOR_RATIOS = [1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9]


def gap_matrix_c64(m, n, k, ratio, seed):
    r = min(m, n)
    sigma = np.concatenate([np.ones(k), ratio * 0.95 ** np.arange(r - k)])
    return np.asfortranarray(synth.prescribed_spectrum(m, n, sigma, seed).astype(np.complex64))


@pytest.mark.parametrize("ratio", FLOOR_RATIOS, ids=lambda r: f"{r:.0e}")
def test_mixed_accuracy_floor_sweep(rid, ratio):
    m, n, k, l = 4096, 1024, 20, 30
    A = gap_matrix_c64(m, n, k, ratio, seed=17)
    A64 = A.astype(np.complex128)
    want = oracle.rid(A64, k, l, seed=23)
    err_fp64 = oracle.exact_error(A64, want["perm"], want["T"])
    with rid.Plan(m, n, k, l, seed=23, dtype=torch.complex64, mode="bf16") as plan:
        Y = plan.sketch(to_dev_colmajor(A, torch.complex64))
        perm_d = plan.select(Y)
        T_d = plan.solve(Y)
        rho, floor, accepted = plan.accuracy(Y)
        plan.sync_status()
    perm, T = to_host(perm_d), to_host(T_d)
    j_equal = bool(np.array_equal(perm[:k], want["J"]))
    err_mixed = oracle.exact_error(A64, perm, T)
    dT = np.abs(T - want["T"]).max() / np.abs(want["T"]).max() if j_equal else float("inf")
    print(f"mixed floor sweep: sigma_k+1/sigma_1 = {ratio:.0e}  rho = {rho:.2e}  J equal = {j_equal}  "
          f"max|dT|/max|T| = {dT:.2e}  error mixed / FP64 = {err_mixed:.2e} / {err_fp64:.2e}  "
          f"floor = {floor:.0e}  accepted = {accepted}")
    # rho estimates the gap of the sketch: within a factor 30 of sigma_{k+1} / sigma_1
    assert ratio / 30 <= rho <= ratio * 30 or (ratio < 1e-7 and rho <= 1e-5)
    if accepted:
        assert j_equal, "accepted above the floor, but J differs from the FP64 path's"
        assert err_mixed <= 2.0 * err_fp64 + 1e-12, (err_mixed, err_fp64)
    if ratio <= 1e-8:
        # far below the floor the mixed sketch's own noise sets the error: the
        # plan must not accept it
        assert not accepted
