"""Row probes fused into the sketch (rid_plan_set_probes / rid_error_sketched)
against the oracle's row-probe estimate (oracle.error_estimate_left), which
forms E = A - A(:, J) P densely from its definition.

Tolerance: the CUDA path computes Z_q = X_q(Jc) - X_q(J) T from X = G A, the
oracle Z_q = G_q (A - A_J P).  With dX the sketch bound on X (the dot-product
bound, plus 2^-46 (2m) max|g_q| max|A_j| for the emulated product) the two
differ by at most
  dZ = dX(Jc) + dX(J) |T| + 4 gamma_k |X_J| |T|            (CUDA path)
     + 4 (gamma_m + gamma_k) |G| (|A| + |A_J| |P|)(Jc)      (oracle)
per entry, so |est - est_o| <= max_q ||dZ_q|| / ||g_q||; the two generators
of G agree to 1e-14 relative, which moves the estimate by 1e-13 ||E||_F at
most.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dot_bound, row_probe_tolerances, to_dev_colmajor, to_host

pytestmark = pytest.mark.gpu

SHAPES = [
    (2048, 1024, 32, 40),
    (1000, 777, 17, 25),
    (50, 300, 40, 60),
    (4096, 333, 1, 3),
    (300, 64, 64, 70),
    (513, 129, 9, 9),
]
MODES = ["fp64", "fp64_emulated"]


@pytest.fixture(scope="module")
def rid():
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    return rid


def lowrank(m, n, k, eps=1e-6, seed=0):
    return synth.lowrank_plus_noise(m, n, k, eps, seed=seed + 3 * m + 5 * n + k)


def run_with_probes(rid, A, k, l, seed, mode, nprobe, probe_seed, perm=None, T=None):
    m, n = A.shape
    with rid.Plan(m, n, k, l, seed=seed, mode=mode) as plan:
        plan.set_probes(nprobe, probe_seed)
        Ad = to_dev_colmajor(A)
        Y = plan.sketch(Ad)
        if perm is None:
            perm_d = plan.select(Y)
            T_d = plan.solve(Y)
        else:
            perm_d = torch.from_numpy(perm.astype(np.int32)).cuda()
            T_d = to_dev_colmajor(T) if T.size else torch.empty((k, 0), dtype=torch.complex128).cuda()
        est, up = plan.error_sketched(perm_d, T_d)
        return est, up, to_host(perm_d), to_host(T_d)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nprobe", [1, 8, 16])
@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_row_probe_estimate_matches_oracle(rid, shape, nprobe, mode):
    m, n, k, l = shape
    A = lowrank(m, n, k)
    out = oracle.rid(A, k, l, seed=9)
    perm, T = out["perm"], out["T"]
    est, up, _, _ = run_with_probes(rid, A, k, l, 9, mode, nprobe, 41, perm, T)
    G = oracle.left_probe_matrix(nprobe, m, 41)
    est_o, up_o, _ = oracle.error_estimate_left(A, perm, T, G)
    tol_est, tol_up = row_probe_tolerances(A, perm, T, G, mode)
    assert abs(est - est_o) <= tol_est + 1e-14 * est_o
    assert abs(up - up_o) <= tol_up + 1e-14 * up_o
    if n > k:
        assert est_o > 100 * tol_est          # the comparison has teeth
    else:
        assert est == 0.0 and up == 0.0       # A = B P exactly when every column is in J


@pytest.mark.parametrize("mode", MODES)
def test_row_probes_leave_the_sketch_unchanged(rid, mode):
    m, n, k, l = 3000, 700, 20, 30
    A = to_dev_colmajor(lowrank(m, n, k))
    with rid.Plan(m, n, k, l, seed=4, mode=mode) as plan:
        Y0 = plan.sketch(A).clone()
        plan.set_probes(8, 2)
        Y1 = plan.sketch(A).clone()
        plan.set_probes(0)
        Y2 = plan.sketch(A).clone()
    assert torch.equal(Y0, Y1) and torch.equal(Y0, Y2)


@pytest.mark.parametrize("mode", MODES)
def test_row_probe_estimate_brackets_the_true_error(rid, mode):
    m, n, k, l = 1500, 600, 25, 35
    A = lowrank(m, n, k, eps=1e-8)
    est, up, perm, T = run_with_probes(rid, A, k, l, 3, mode, 8, 5)
    err = oracle.exact_error(A, perm, T)
    # est <= ||E||_2 always.  From below: ||g E|| >= sigma_1 |<g, u_1>| with
    # |<g, u_1>|^2 ~ Exp(1), so the best of 8 probes has ||g E|| >= 0.1 ||E||_2
    # except with probability (1 - e^-0.01)^8 < 1e-15, and ||g||^2 <= 2m (a
    # chi-square tail far smaller still): est >= 0.1 ||E||_2 / sqrt(2m).
    # (Row probes are normalised by ||g|| ~ sqrt(m), so for tall A with a flat
    # residual spectrum est sits near ||E||_F / sqrt(m).)
    assert 0.1 * err / math.sqrt(2 * m) <= est <= err * (1 + 1e-6)
    assert err <= up


def test_row_probes_with_srft(rid):
    m, n, k, l = 1024, 300, 12, 24
    A = lowrank(m, n, k)
    Ad = to_dev_colmajor(A)
    with rid.Plan(m, n, k, l, seed=1, mode="fp64_emulated") as plan:
        plan.set_probes(6, 8)
        plan.use_srft(4)                      # replaces the l test rows, keeps the probes
        Y = plan.sketch(Ad)
        perm = plan.select(Y)
        T = plan.solve(Y)
        est, up = plan.error_sketched(perm, T)
    perm_h, T_h = to_host(perm), to_host(T)
    G = oracle.left_probe_matrix(6, m, 8)
    est_o, up_o, _ = oracle.error_estimate_left(A, perm_h, T_h, G)
    tol_est, tol_up = row_probe_tolerances(A, perm_h, T_h, G, "fp64_emulated")
    assert abs(est - est_o) <= tol_est + 1e-14 * est_o
    assert abs(up - up_o) <= tol_up + 1e-14 * up_o


def test_row_probe_argument_errors(rid):
    from paper_1205_3830_gb300._native import RIDError
    m, n, k, l = 256, 100, 5, 10
    A = to_dev_colmajor(lowrank(m, n, k))
    with rid.Plan(m, n, k, l, seed=1, mode="fp64_emulated") as plan:
        Y = plan.sketch(A)
        perm = plan.select(Y)
        T = plan.solve(Y)
        with pytest.raises(RIDError, match="EINVAL"):
            plan.error_sketched(perm, T)              # no probes set
        plan.set_probes(4, 1)
        with pytest.raises(RIDError, match="EINVAL"):
            plan.error_sketched(perm, T)              # set, but no sketch since
        with pytest.raises(RIDError, match="EINVAL"):
            plan.set_probes(17, 1)
        plan.sketch(A)
        plan.error_sketched(perm, T)
        plan.set_probes(0)
        with pytest.raises(RIDError, match="EINVAL"):
            plan.error_sketched(perm, T)
    with rid.Plan(m, n, k, 500, seed=1, mode="fp64") as plan:
        with pytest.raises(RIDError, match="EUNSUPPORTED"):
            plan.set_probes(13, 1)                   # l + nprobe > 512
    with rid.Plan(m, n, k, l, seed=1, dtype=torch.complex64, mode="bf16") as plan:
        plan.set_probes(4, 1)                        # mixed plans take FP64-grade row probes too
        with pytest.raises(RIDError, match="EINVAL"):
            plan.sketch_cols(torch.zeros((n, m), dtype=torch.complex64, device="cuda").t(),
                             rid.colmajor_empty(l, n), 64, 36)           # col0 not a multiple of 128


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", [(2048, 1000, 20, 30), (700, 384, 10, 16), (3000, 129, 5, 9)], ids=str)
def test_sketch_by_column_panels_equals_one_sketch(rid, shape, mode):
    """Panels of columns, sketched in any order, give rid_sketch's Y and the
    same row-probe estimate, bit for bit."""
    m, n, k, l = shape
    A = to_dev_colmajor(lowrank(m, n, k))
    with rid.Plan(m, n, k, l, seed=21, mode=mode) as plan:
        plan.set_probes(8, 3)
        Y0 = plan.sketch(A).clone()
        R = Y0.clone()
        perm = plan.select(R)
        T = plan.solve(R)
        e0 = plan.error_sketched(perm, T)
        Y1 = torch.full_like(Y0, float("nan"))
        starts = list(range(0, n, 256))
        for c0 in reversed(starts):                       # out of order on purpose
            plan.sketch_cols(A, Y1, c0, min(256, n - c0))
        e1 = plan.error_sketched(perm, T)
    assert torch.equal(Y0, Y1)
    assert e0 == e1



def test_sketch_cols_argument_errors(rid):
    from paper_1205_3830_gb300._native import RIDError
    m, n, k, l = 300, 400, 5, 10
    A = to_dev_colmajor(lowrank(m, n, k))
    with rid.Plan(m, n, k, l, seed=1, mode="fp64_emulated") as plan:
        Y = plan.sketch(A)
        for c0, nc in ((64, 128), (0, 100), (256, 256), (-128, 128)):
            with pytest.raises(RIDError, match="EINVAL"):
                plan.sketch_cols(A, Y, c0, nc)
        plan.sketch_cols(A, Y, 256, 144)                  # the last, ragged panel


@pytest.mark.parametrize("mode", MODES + ["bf16"])
def test_plan_created_with_probes_matches_set_probes(rid, mode):
    """rid_plan_create_probes gives the bits of rid_plan_create + rid_plan_set_probes:
    the sketch Y (and the probe products behind the estimate), J, T and the estimate."""
    m, n, k, l = 3000, 2200, 24, 34            # 18 column blocks: the CTA-pair product in the emulated mode
    A = lowrank(m, n, k, seed=8)
    dtype = torch.complex64 if mode == "bf16" else torch.complex128
    Ad = to_dev_colmajor(A.astype(np.complex64) if mode == "bf16" else A, dtype)
    outs = []
    for built_in in (False, True):
        kw = {"nprobe": 8, "probe_seed": 4} if built_in else {}
        with rid.Plan(m, n, k, l, seed=6, dtype=dtype, mode=mode, **kw) as plan:
            if not built_in:
                plan.set_probes(8, 4)
            assert plan.nrow == 8
            Y = plan.sketch(Ad)
            Y0 = Y.clone()
            perm = plan.select(Y)
            T = plan.solve(Y)
            est = plan.error_sketched(perm, T)
            plan.sync_status()
            outs.append((to_host(Y0), to_host(perm), to_host(T), est))
    (Ya, pa, Ta, ea), (Yb, pb, Tb, eb) = outs
    assert np.array_equal(Ya, Yb) and np.array_equal(pa, pb) and np.array_equal(Ta, Tb)
    assert ea == eb


# ---- the probe products X = G A themselves -------------------------------------
# X is read back through rid_plan_probe_products and compared entry by entry
# with the oracle's G A (one library product on the upcast A).  Bound: the
# FP64 dot-product bound, 2^-46 (2m) max|g_q| max|A_j| for the emulated
# products (56-bit digits, double-FP32 sums), and 1e-14 |G| |A| for the two
# generators of G.
def probe_products_bound(G, A):
    m = A.shape[0]
    return (dot_bound(G, A) + 2.0 ** -46 * (2 * m) * np.outer(np.abs(G).max(axis=1), np.abs(A).max(axis=0))
            + 1e-14 * (np.abs(G) @ np.abs(A)))


def probe_products(rid, A, mode, nprobe, probe_seed, panel=None):
    m, n = A.shape
    dtype = torch.complex64 if mode == "bf16" else torch.complex128
    k = min(3, m, n)
    with rid.Plan(m, n, k, k + 2, seed=1, dtype=dtype, mode=mode, nprobe=nprobe, probe_seed=probe_seed) as plan:
        Ad = to_dev_colmajor(A, dtype)
        if panel is None:
            plan.sketch(Ad)
        else:                                       # column panels, last first
            Y = rid.colmajor_empty(k + 2, n)
            for c0 in reversed(range(0, n, panel)):
                plan.sketch_cols(Ad, Y, c0, min(panel, n - c0))
        X = to_host(plan.probe_products())
        plan.sync_status()
    return X


@pytest.mark.parametrize("mode", MODES + ["bf16"])
@pytest.mark.parametrize("shape,nprobe", [((1000, 777), 8), ((8192, 300), 13), ((333, 129), 1), ((5, 1), 16),
                                          ((4096, 1030), 16), ((2048, 256), 7)], ids=str)
def test_probe_products_match_oracle(rid, mode, shape, nprobe):
    """X = G A of every mode (the mixed mode's from the complex64 A) against
    the oracle: several column blocks with a ragged last one, K ranges of one
    and of several chunks with a ragged tail, K-splits (m = 8192), and both
    widths of the mixed mode's probe kernel (2 nprobe <= 16 and <= 32)."""
    m, n = shape
    A = lowrank(m, n, min(5, m, n), eps=1e-3, seed=nprobe)
    if mode == "bf16":
        A = A.astype(np.complex64).astype(np.complex128)
    X = probe_products(rid, A, mode, nprobe, 5)
    G = oracle.left_probe_matrix(nprobe, m, 5)
    assert X.shape == (nprobe, n)
    d = np.abs(X - G @ A)
    bound = probe_products_bound(G, A)
    print(f"{mode} {shape} r={nprobe}: max |dX| / bound = {np.max(d / bound):.2e}")
    assert np.all(d <= bound)


def scaled_c64(m, n, direction, seed):
    """Complex64 A whose chunk exponents change along K (rising or falling by
    2^12 over the column), with a zero chunk, one column of subnormal floats
    and one column whose first half is zero."""
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))).astype(np.complex128)
    t = np.arange(m) / m
    s = 2.0 ** (12 * t if direction == "rising" else 12 * (1 - t))
    A *= s[:, None]
    A[1024:1152, :] = 0                      # a whole chunk of zeros
    A[:, 5] = (1e-40 * (rng.integers(-40, 40, m) + 1j * rng.integers(-40, 40, m)))   # subnormal floats
    A[: m // 2, 9] = 0
    return np.asfortranarray(A.astype(np.complex64).astype(np.complex128))


@pytest.mark.parametrize("direction", ["rising", "falling"])
def test_mixed_probe_products_chunk_exponents(rid, direction):
    """The mixed mode's probe kernel keeps a running exponent per column and
    K-split: chunk exponents that grow along K (the sums are rescaled), that
    shrink, zero chunks and subnormal floats, against the oracle."""
    m, n = 8192, 260
    A = scaled_c64(m, n, direction, 3)
    X = probe_products(rid, A, "bf16", 8, 4)
    G = oracle.left_probe_matrix(8, m, 4)
    Xo = G @ A
    d = np.abs(X - Xo)
    bound = probe_products_bound(G, A)
    print(f"{direction}: max |dX| / bound = {np.max(d / bound):.2e}")
    assert np.all(d <= bound)
    assert np.all(np.abs(Xo[:, 5]) < 1e-36) and np.all(np.abs(X[:, 5] - Xo[:, 5]) <= bound[:, 5])


def test_mixed_probe_products_panels(rid):
    """Column panels of a mixed plan give the one-call X bit for bit."""
    m, n = 4096, 1000
    A = lowrank(m, n, 5, eps=1e-3, seed=2).astype(np.complex64).astype(np.complex128)
    X0 = probe_products(rid, A, "bf16", 8, 3)
    X1 = probe_products(rid, A, "bf16", 8, 3, panel=384)
    assert np.array_equal(X0, X1)
