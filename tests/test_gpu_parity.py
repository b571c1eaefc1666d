"""CUDA path vs the CPU oracle, element by element, on the same seeded inputs
(every call goes through the C ABI of include/rid.h via the ctypes binding).

Tolerances:
  * Omega: each side evaluates log, cos, sin of the same 53-bit uniforms; the
    results differ only by the last bits of those functions: |dOmega| <=
    1e-14 (1 + |Omega|).
  * sketch: same Omega, different summation order: the textbook dot-product
    bound 2 gamma_m |Omega| |A| per entry (gpu_util.dot_bound); integer
    inputs must agree bit for bit.
  * select: J and the whole permutation exactly; R (and the reflectors)
    within 1e-12 max|R| (rounding of k Householder steps on O(1) data).
  * solve: same R1, R2 -> T within 1e-11 max|T| (back substitution).
  * whole ID: J exactly wherever sigma_k / sigma_{k+1} >= 1e3, and
    max|T_gpu - T_oracle| <= 1e-10 max|T_oracle| (P within 1e-10 relative).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U64, dot_bound, to_dev_colmajor, to_dev_colmajor_ld, to_host

pytestmark = pytest.mark.gpu

# (m, n, k, l): several tiles with ragged tails, l > m, k = 1, k = n, l = k
SHAPES = [
    (2048, 1024, 32, 40),
    (1000, 777, 17, 25),
    (50, 300, 40, 60),
    (4096, 333, 1, 3),
    (300, 64, 64, 70),
    (513, 129, 9, 9),
    (3000, 2000, 100, 110),
]


@pytest.fixture(scope="module")
def rid():
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    return rid


def lowrank(m, n, k, eps=1e-10, seed=0):
    return synth.lowrank_plus_noise(m, n, k, eps, seed=seed + 7 * m + 13 * n + k)


@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_omega_matches_oracle(rid, shape):
    m, n, k, l = shape
    seed = 1000 + m
    with rid.Plan(m, n, k, l, seed=seed) as plan:
        Om = to_host(plan.omega())
    Oo = oracle.gaussian_test_matrix(l, m, seed)
    assert np.all(np.abs(Om - Oo) <= 1e-14 * (1 + np.abs(Oo)))


MODES = ["fp64", "fp64_emulated"]


def emulation_bound(Om, A):
    """Extra error of the tensor-core emulation: 56-bit digits of every value
    (relative to its row / chunk maximum), the dropped slice pairs and the
    double-FP32 running sums stay below 2^-46 (2m) max|Omega_i| max|A_j|."""
    m = A.shape[0]
    return 2.0 ** -46 * (2 * m) * np.outer(np.abs(Om).max(axis=1), np.abs(A).max(axis=0))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_sketch_matches_oracle(rid, shape, mode):
    m, n, k, l = shape
    A = lowrank(m, n, k)
    Oo = oracle.gaussian_test_matrix(l, m, 5)
    with rid.Plan(m, n, k, l, seed=5, mode=mode) as plan:
        plan.set_omega(torch.from_numpy(Oo).cuda())
        Y = to_host(plan.sketch(to_dev_colmajor(A)))
        plan.sync_status()
    Yo = oracle.randomize(Oo, A)
    tol = dot_bound(Oo, A) + (emulation_bound(Oo, A) if mode != "fp64" else 0.0)
    assert np.all(np.abs(Y - Yo) <= tol)


@pytest.mark.parametrize("mode", MODES)
def test_sketch_wide_dynamic_range(rid, mode):
    """Rows of A scaled by 2^-40 .. 2^40, zero columns and a zero row block:
    the per-chunk exponents keep every chunk at full relative precision."""
    m, n, k, l = 1200, 300, 10, 16
    A = lowrank(m, n, k, eps=1e-3)
    A *= (2.0 ** np.linspace(-40, 40, m))[:, None]
    A[:, [0, 7, 299]] = 0.0
    A[256:512, :] = 0.0
    Oo = oracle.gaussian_test_matrix(l, m, 8)
    with rid.Plan(m, n, k, l, seed=8, mode=mode) as plan:
        plan.set_omega(torch.from_numpy(Oo).cuda())
        Y = to_host(plan.sketch(to_dev_colmajor(A)))
        plan.sync_status()
    Yo = oracle.randomize(Oo, A)
    assert np.all(Y[:, [0, 7, 299]] == 0)
    # chunk-relative bound: each 128-row chunk contributes at its own scale
    chunk_max = np.zeros_like(np.abs(A))
    for c0 in range(0, m, 128):
        chunk_max[c0:c0 + 128] = np.abs(A[c0:c0 + 128]).max(axis=0, keepdims=True)
    tol = dot_bound(Oo, A) + 2.0 ** -46 * 256 * np.abs(Oo).max(axis=1)[:, None] * chunk_max.sum(axis=0)[None, :]
    assert np.all(np.abs(Y - Yo) <= tol)


@pytest.mark.parametrize("mode", MODES)
def test_sketch_integer_inputs_bit_exact(rid, mode):
    m, n, k, l = 1500, 700, 20, 37
    A = synth.integer_valued(m, n, 64, seed=1)
    Oi = np.ascontiguousarray(synth.integer_valued(m, l, 64, seed=2).T)
    with rid.Plan(m, n, k, l, seed=1, mode=mode) as plan:
        plan.set_omega(torch.from_numpy(Oi).cuda())
        Y = to_host(plan.sketch(to_dev_colmajor(A)))
    assert np.array_equal(Y, oracle.randomize(Oi, A))


def test_sketch_leading_dimension(rid):
    m, n, k, l = 600, 400, 20, 28
    A = lowrank(m, n, k)
    with rid.Plan(m, n, k, l, seed=9) as plan:
        Y1 = to_host(plan.sketch(to_dev_colmajor(A)))
        Y2 = to_host(plan.sketch(to_dev_colmajor_ld(A, 640)))
    assert np.array_equal(Y1, Y2)


@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_select_matches_oracle(rid, shape):
    m, n, k, l = shape
    A = lowrank(m, n, k)
    Yo = oracle.randomize(oracle.gaussian_test_matrix(l, m, 3), A)
    Ro, tau_o, perm_o = oracle.qr_select(Yo, k)
    with rid.Plan(m, n, k, l, seed=3) as plan:
        Yd = to_dev_colmajor(Yo)
        perm = to_host(plan.select(Yd))
        plan.sync_status()
        R = to_host(Yd)
    assert np.array_equal(perm, perm_o)
    scale = np.abs(Ro[:k]).max()
    upper = np.triu(np.ones((k, n), dtype=bool))
    assert np.abs(R[:k][upper] - Ro[:k][upper]).max() <= 1e-12 * scale
    lower = np.tril(np.ones((l, k), dtype=bool), -1)           # reflectors v below the diagonal
    assert np.abs(R[:, :k][lower] - Ro[:, :k][lower]).max(initial=0) <= 1e-12 * max(1.0, np.abs(Ro[:, :k][lower]).max(initial=0))


@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_solve_matches_oracle(rid, shape):
    m, n, k, l = shape
    A = lowrank(m, n, k)
    Yo = oracle.randomize(oracle.gaussian_test_matrix(l, m, 4), A)
    Ro, _, _ = oracle.qr_select(Yo, k)
    To = oracle.factor_r(Ro[:k, :k], Ro[:k, k:])
    with rid.Plan(m, n, k, l, seed=4) as plan:
        T = to_host(plan.solve(to_dev_colmajor(Ro)))
    assert T.shape == To.shape
    if To.size:
        assert np.abs(T - To).max() <= 1e-11 * np.abs(To).max()


@pytest.mark.parametrize("shape", SHAPES, ids=str)
@pytest.mark.parametrize("nprobe", [1, 8, 16])
def test_error_estimate_matches_oracle(rid, shape, nprobe):
    m, n, k, l = shape
    A = lowrank(m, n, k, eps=1e-6)
    out = oracle.rid(A, k, l, seed=6)
    perm, T = out["perm"], out["T"]
    omega = oracle.probe_matrix(n, nprobe, 77)
    est_o, up_o, Ew = oracle.error_estimate(A, perm, T, omega)
    with rid.Plan(m, n, k, l, seed=6) as plan:
        est, up = plan.error(to_dev_colmajor(A), torch.from_numpy(perm.astype(np.int32)).cuda(),
                             to_dev_colmajor(T) if T.size else torch.empty((k, 0), dtype=torch.complex128).cuda(),
                             nprobe=nprobe, probe_seed=77)
    # rounding bound on E w: |A| (|w~| + |T| |w_Jc| on J) times gamma_(n+k)
    w_abs = np.abs(omega)
    w_abs[perm[:k]] = np.abs(T) @ np.abs(omega[perm[k:]]) if T.size else 0.0
    bound_q = 4 * (n + k) * U64 * np.linalg.norm(np.abs(A) @ w_abs, axis=0)
    wn = np.linalg.norm(omega, axis=0)
    tol_est = np.max(bound_q / wn) + 1e-14 * est_o
    assert abs(est - est_o) <= tol_est
    assert abs(up - up_o) <= 10 * math.sqrt(2 / math.pi) * np.max(bound_q) + 1e-14 * up_o


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_whole_id_matches_oracle(rid, shape, mode):
    m, n, k, l = shape
    seed = 20 + m
    A = lowrank(m, n, k)
    out = oracle.rid(A, k, l, seed=seed)
    Ad = to_dev_colmajor(A)
    res = rid.decompose(Ad, k, l, seed=seed, nprobe=8, probe_seed=3, mode=mode)
    perm, T = to_host(res["perm"]), to_host(res["T"])
    assert np.array_equal(perm[:k], out["J"])
    if T.size:
        assert np.abs(T - out["T"]).max() <= 1e-10 * np.abs(out["T"]).max()
    # B is A(:, J) exactly and P(:, J) = I exactly, by construction
    P = oracle.interpolation_matrix(perm, T, n)
    assert np.array_equal(P[:, perm[:k]], np.eye(k))
    # the estimate lies below the true error, which obeys the sigma_{k+1} bound
    err = np.linalg.norm(A - A[:, perm[:k]] @ P, 2) if m * n <= 2048 * 1024 else None
    if err is not None:
        assert res["est"] <= err * (1 + 1e-6) + 1e-13 * np.abs(A).max()
        s = np.linalg.svd(A, compute_uv=False)
        sk1 = s[k] if k < min(m, n) else 0.0
        assert err <= 10 * math.sqrt(1 + k * (n - k)) * sk1 + 1e-12 * s[0]


def test_rank_deficient_sketch_reports_erank(rid):
    m, n, k, l = 64, 40, 5, 8
    A = np.zeros((m, n), dtype=np.complex128)
    A[:, 3] = synth.cgauss(np.random.default_rng(1), m)
    A[:, 17] = synth.cgauss(np.random.default_rng(2), m)
    with rid.Plan(m, n, k, l, seed=1) as plan:
        Y = plan.sketch(to_dev_colmajor(A))
        plan.select(Y)
        with pytest.raises(rid.RIDError) as info:
            plan.sync_status()
        assert info.value.status == 4
        # the plan stays usable: a rank-2 problem on the same shape succeeds
        A2 = lowrank(m, n, k)
        res = rid.decompose(to_dev_colmajor(A2), k, l, seed=1, plan=plan)
        assert res["perm"].shape == (n,)


@pytest.mark.parametrize("mode", MODES)
def test_results_are_deterministic(rid, mode):
    m, n, k, l = 2048, 1024, 32, 40
    A = to_dev_colmajor(lowrank(m, n, k))
    r1 = rid.decompose(A, k, l, seed=2, mode=mode)
    r2 = rid.decompose(A, k, l, seed=2, mode=mode)
    assert torch.equal(r1["perm"], r2["perm"]) and torch.equal(r1["T"], r2["T"])
    assert r1["est"] == r2["est"]


# --- the paper's randomization: Omega = S F D (Sec. 2) ---------------------------
def srft_matrix(l, m, seed):
    """Rows s_q of F D built from the oracle's SRFT parameters (definition)."""
    phi, s = oracle.srft_parameters(l, m, seed)
    jk = np.outer(s, np.arange(m)) % m
    return np.exp(-2j * np.pi * (jk / m)) * np.exp(2j * np.pi * phi)[None, :]


@pytest.mark.parametrize("shape", [(2048, 1024, 32, 40), (1000, 777, 17, 25), (4096, 333, 1, 3)], ids=str)
def test_srft_omega_matches_oracle(rid, shape):
    m, n, k, l = shape
    with rid.Plan(m, n, k, l, seed=1) as plan:
        plan.use_srft(99)
        Om = to_host(plan.omega())
    Oo = srft_matrix(l, m, 99)
    assert np.abs(np.abs(Om) - 1).max() < 1e-14
    assert np.abs(Om - Oo).max() <= 1e-13


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", [(2048, 1024, 32, 40), (1000, 777, 17, 25)], ids=str)
def test_srft_sketch_matches_oracle(rid, shape, mode):
    m, n, k, l = shape
    A = lowrank(m, n, k)
    with rid.Plan(m, n, k, l, seed=1, mode=mode) as plan:
        plan.use_srft(7)
        Y = to_host(plan.sketch(to_dev_colmajor(A)))
        plan.sync_status()
    Yo = oracle.srft_randomize(A, l, 7)
    Oo = srft_matrix(l, m, 7)
    tol = dot_bound(Oo, A) + 1e-13 * (np.abs(Oo) @ np.abs(A))
    if mode != "fp64":
        tol = tol + emulation_bound(Oo, A)
    assert np.all(np.abs(Y - Yo) <= tol)


@pytest.mark.parametrize("mode", MODES)
def test_srft_whole_id_matches_oracle(rid, mode):
    m, n, k, l = 2048, 1024, 32, 64
    A = lowrank(m, n, k)
    Oo = srft_matrix(l, m, 5)
    out = oracle.rid(A, k, l, seed=0, Omega=Oo)
    with rid.Plan(m, n, k, l, seed=0, mode=mode) as plan:
        plan.use_srft(5)
        res = rid.decompose(to_dev_colmajor(A), k, l, plan=plan)
    perm, T = to_host(res["perm"]), to_host(res["T"])
    assert np.array_equal(perm[:k], out["J"])
    assert np.abs(T - out["T"]).max() <= 1e-10 * np.abs(out["T"]).max()
