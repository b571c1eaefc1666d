"""Pins for the CPU oracle: each check ties one oracle function to something
other than itself (published known-answer vectors, exact integer arithmetic,
LAPACK's pivoted QR, least squares, the SVD, brute force, distribution tests).

Every check takes the oracle module as an argument, so tests can also run it
against a deliberately broken copy (tests/test_oracle_mutations.py) and
confirm that the pin catches the mistake.
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np
import scipy.linalg
import scipy.stats

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_philox_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


# --- random numbers ---------------------------------------------------------
def pin_philox_kat(o):
    for ctr, key, out in load_philox_kat():
        got = o.philox4x32_10(np.array(ctr, dtype=np.uint64), key)
        assert [int(x) for x in got] == out, (ctr, key, [hex(int(x)) for x in got])


def pin_uniform53(o):
    u1, u2 = o.uniform53_pair(np.array([0, 0, 0, 0], dtype=np.uint64))
    assert u1 == 2.0 ** -53 and u2 == 0.0
    u1, u2 = o.uniform53_pair(np.array([0xFFFFFFFF] * 4, dtype=np.uint64))
    assert u1 == 1.0 and u2 == 1.0 - 2.0 ** -53
    # the top word carries the high bits
    u1, u2 = o.uniform53_pair(np.array([1 << 31, 0, 1 << 31, 0], dtype=np.uint64))
    assert u1 == 0.5 + 2.0 ** -53 and u2 == 0.5


def pin_gaussian_distribution(o):
    z = o.complex_gaussian(64, 1024, seed=7, stream=o.STREAM_OMEGA).ravel()
    for part in (z.real, z.imag):
        p = scipy.stats.kstest(part * math.sqrt(2.0), "norm").pvalue
        assert p > 1e-4, p
    p = scipy.stats.kstest(np.abs(z) ** 2, "expon").pvalue
    assert p > 1e-4, p
    # re and im uncorrelated, streams and seeds independent
    assert abs(np.corrcoef(z.real, z.imag)[0, 1]) < 0.02
    z2 = o.complex_gaussian(64, 1024, seed=7, stream=o.STREAM_PROBES).ravel()
    z3 = o.complex_gaussian(64, 1024, seed=8, stream=o.STREAM_OMEGA).ravel()
    assert abs(np.vdot(z, z2)) / z.size < 0.02 and abs(np.vdot(z, z3)) / z.size < 0.02
    # a sub-block drawn with offsets equals the block of the full matrix
    sub = o.complex_gaussian(5, 7, seed=7, stream=o.STREAM_OMEGA, row0=10, col0=100)
    full = o.complex_gaussian(64, 1024, seed=7, stream=o.STREAM_OMEGA)
    assert np.array_equal(sub, full[10:15, 100:107])


# --- step 1: Y = Omega A --------------------------------------------------
def pin_randomize_exact(o):
    """Gaussian integers: every product and sum is exact in FP64, so the sketch
    must equal exact integer arithmetic bit for bit."""
    Om = np.ascontiguousarray(synth.integer_valued(57, 13, 100, seed=1).T)
    A = synth.integer_valued(57, 21, 100, seed=2)
    Y = o.randomize(Om, A)
    orr, oi = Om.real.astype(np.int64), Om.imag.astype(np.int64)
    ar, ai = A.real.astype(np.int64), A.imag.astype(np.int64)
    yr = orr @ ar - oi @ ai
    yi = orr @ ai + oi @ ar
    assert Y.shape == (13, 21)
    assert np.array_equal(Y.real, yr.astype(np.float64)) and np.array_equal(Y.imag, yi.astype(np.float64))


# --- step 2: pivoted QR -----------------------------------------------------
def householder_q(R, tau, k):
    """Q = H_0 H_1 ... H_{k-1} (l x k) from the stored reflectors."""
    l = R.shape[0]
    Q = np.eye(l, k, dtype=np.complex128)
    for j in range(k - 1, -1, -1):
        v = np.zeros(l, dtype=np.complex128)
        v[j] = 1.0
        v[j + 1:] = R[j + 1:, j]
        Q -= tau[j] * np.outer(v, v.conj() @ Q)
    return Q


def pin_qr_lapack(o):
    """Same J and R as LAPACK's zgeqp3 (scipy.linalg.qr(pivoting=True)) on a
    Gaussian Y (no near ties); Q orthonormal; Y(:, perm) = Q R on the first k."""
    rng = np.random.default_rng(3)
    for (l, n, k) in [(12, 40, 8), (30, 30, 30), (9, 200, 9), (40, 17, 5)]:
        Y = synth.cgauss(rng, (l, n))
        R, tau, perm = o.qr_select(Y, k)
        Rl, Pl = scipy.linalg.qr(Y, pivoting=True, mode="r")
        assert np.array_equal(perm[:k], Pl[:k]), (perm[:k], Pl[:k])
        Rk = np.triu(R[:k, :])
        scale = np.abs(Rl).max()
        assert np.abs(Rk[:, :k] - Rl[:k, :k]).max() <= 1e-12 * scale
        # LAPACK keeps pivoting after step k: match trailing columns by original index
        pos_l = np.empty(n, dtype=np.int64)
        pos_l[Pl] = np.arange(n)
        if k < n:
            assert np.abs(Rk[:, k:] - Rl[:k, pos_l[perm[k:]]]).max() <= 1e-12 * scale
        Q = householder_q(R, tau, k)
        assert np.abs(Q.conj().T @ Q - np.eye(k)).max() < 1e-13
        assert np.abs(Y[:, perm[:k]] - Q @ Rk[:, :k]).max() <= 1e-12 * scale
        # the trailing columns: Q^H Y(:, perm[k:]) = R2
        if k < n:
            assert np.abs(Q.conj().T @ Y[:, perm[k:]] - Rk[:, k:]).max() <= 1e-12 * scale


def pin_qr_pivot_rule(o):
    """Each pivot is the largest remaining column (recomputed exactly), and
    ties go to the lowest index: a Y with duplicated columns."""
    rng = np.random.default_rng(4)
    Y = synth.cgauss(rng, (6, 5))
    Y[:, 2] *= 10.0                                  # column 2 is the largest ...
    Y = np.concatenate([Y, Y[:, [2]]], axis=1)      # ... and column 5 duplicates it
    R, tau, perm = o.qr_select(Y, 2)
    assert perm[0] == 2                              # tie -> lowest index
    assert perm[1] != 5                              # the duplicate is annihilated
    # k = 1 closed form: J = argmax column norm, T = y_J^H Y_Jc / ||y_J||^2
    Y = synth.cgauss(rng, (7, 11))
    out = o.rid(Y, 1, 7, seed=0, Omega=np.eye(7))
    j = int(np.argmax(np.sum(np.abs(Y) ** 2, axis=0)))
    assert out["J"][0] == j
    y = Y[:, j]
    Tcf = (y.conj() @ Y[:, out["perm"][1:]]) / np.vdot(y, y).real
    assert np.allclose(out["T"][0], Tcf, rtol=1e-13, atol=1e-14)


def pin_rank_deficient(o):
    """A with only two nonzero columns cannot give k = 3 pivots."""
    A = np.zeros((10, 6), dtype=np.complex128)
    rng = np.random.default_rng(5)
    A[:, 1] = synth.cgauss(rng, 10)
    A[:, 4] = synth.cgauss(rng, 10)
    Om = synth.cgauss(rng, (5, 10))
    raised = False
    try:
        o.rid(A, 3, 5, seed=0, Omega=Om)
    except o.RankDeficient:
        raised = True
    assert raised
    out = o.rid(A, 2, 5, seed=0, Omega=Om)
    assert sorted(out["J"].tolist()) == [1, 4]


# --- step 3: factor R -------------------------------------------------------
def pin_factor_r(o):
    """T = R1^-1 R2 equals the least-squares solution Y_J^+ Y_Jc and LAPACK's
    triangular solve; P(:, J) = I exactly and B = A(:, J)."""
    rng = np.random.default_rng(6)
    for (m, n, k, l) in [(60, 50, 6, 10), (40, 80, 12, 12), (33, 20, 1, 4)]:
        A = synth.lowrank_plus_noise(m, n, k, 1e-9, seed=int(rng.integers(1 << 30)))
        out = o.rid(A, k, l, seed=11)
        Y, R, perm, T = out["Y"], out["R"], out["perm"], out["T"]
        J, Jc = perm[:k], perm[k:]
        Tl = np.linalg.lstsq(Y[:, J], Y[:, Jc], rcond=None)[0]
        assert np.abs(T - Tl).max() <= 1e-9 * max(1.0, np.abs(Tl).max())
        Ts = scipy.linalg.solve_triangular(R[:k, :k], R[:k, k:])
        assert np.abs(T - Ts).max() <= 1e-12 * max(1.0, np.abs(Ts).max())
        P = out["P"]
        assert np.array_equal(P[:, J], np.eye(k))
        assert np.array_equal(P[:, Jc], T)


# --- the whole ID -----------------------------------------------------------
def pin_exact_rank(o):
    for (m, n, k) in [(120, 90, 7), (64, 200, 16)]:
        A = synth.lowrank_plus_noise(m, n, k, 0.0, seed=m * n)
        out = o.rid(A, k, k + 8, seed=3)
        E = A - A[:, out["J"]] @ out["P"]
        assert np.linalg.norm(E) <= 1e-12 * np.linalg.norm(A)


def pin_spectrum_bound(o):
    """||A - BP||_2 between sigma_{k+1} (Eckart-Young) and
    10 sqrt(1 + k(n-k)) sigma_{k+1}; eq. (1) of Sec. 2 with eps = 1e-10."""
    m, n, k = 160, 120, 10
    sigma = np.concatenate([np.ones(k), 1e-8 * np.ones(min(m, n) - k)])
    A = synth.prescribed_spectrum(m, n, sigma, seed=9)
    for seed in (1, 2, 3):
        out = o.rid(A, k, k + 8, seed=seed)
        err = o.exact_error(A, out["perm"], out["T"])
        s1 = sigma[k]
        assert err >= s1 * (1 - 1e-6)
        assert err <= 10 * math.sqrt(1 + k * (n - k)) * s1
        assert err <= 50 * math.sqrt(m * n) * (1e10) ** (1.0 / k) * s1


def pin_brute_force(o):
    """Tiny inputs: the best k columns e* = min_J ||A - A_J A_J^+ A||_2 obeys
    sigma_{k+1} <= e* <= sqrt(1 + k(n-k)) sigma_{k+1}; the ID is no better
    than e* and within 10 sqrt(1 + k(n-k)) sigma_{k+1}.  With Omega = I the
    ID is LAPACK's pivoted QR of A itself."""
    rng = np.random.default_rng(12)
    for (m, n, k) in [(12, 9, 2), (10, 8, 3), (7, 10, 1)]:
        sigma = np.concatenate([[3.0, 2.0, 1.5][:k], 1e-3 * rng.uniform(0.5, 1.0, min(m, n) - k)])
        A = synth.prescribed_spectrum(m, n, sigma, seed=int(rng.integers(1 << 30)))
        s = np.linalg.svd(A, compute_uv=False)
        best = min(np.linalg.norm(A - A[:, list(J)] @ np.linalg.pinv(A[:, list(J)]) @ A, 2)
                   for J in itertools.combinations(range(n), k))
        bound = math.sqrt(1 + k * (n - k))
        assert s[k] * (1 - 1e-9) <= best <= bound * s[k]
        out = o.rid(A, k, k + 4, seed=5)
        err = o.exact_error(A, out["perm"], out["T"])
        assert best <= err * (1 + 1e-9)
        assert err <= 10 * bound * s[k]
        ident = o.rid(A, k, m, seed=0, Omega=np.eye(m))
        _, _, Pl = scipy.linalg.qr(A, pivoting=True)
        assert np.array_equal(ident["J"], Pl[:k])


# --- step 4: error estimate -----------------------------------------------
def pin_error_estimate(o):
    """est <= ||E||_2 always; ||E||_2 <= upper (w.p. >= 1 - 10^-r); E w equals
    A w - A_J (P w) formed directly."""
    m, n, k = 90, 70, 5
    A = synth.lowrank_plus_noise(m, n, k, 1e-6, seed=21)
    out = o.rid(A, k, k + 6, seed=4)
    exact = o.exact_error(A, out["perm"], out["T"])
    for ps in (1, 2, 3):
        omega = o.probe_matrix(n, 6, ps)
        est, upper, Ew = o.error_estimate(A, out["perm"], out["T"], omega)
        assert est <= exact * (1 + 1e-9)
        assert exact <= upper
        assert est >= 0.05 * exact
        direct = A @ omega - A[:, out["J"]] @ (out["P"] @ omega)
        # both sides cancel terms of size |A| |P| |omega| down to ~1e-6 of that
        scale = np.abs(A).max() * np.abs(out["P"]).max() * np.abs(omega).max() * n
        assert np.abs(Ew - direct).max() <= 1e-13 * scale
        assert np.abs(direct).max() > 1e3 * 1e-13 * scale     # the check has teeth


def pin_error_estimate_left(o):
    """Row probes.  A residual built to be sigma u v^H on the columns Jc (and 0
    on J) gives ||g E|| = sigma |sum_i g_i u_i| for every row probe g, a closed
    form that fixes the probe orientation, the conjugation and the norms; on an
    ID of a noisy low-rank matrix, est <= ||E||_2 <= upper."""
    rng = np.random.default_rng(41)
    m, n, k, r = 60, 25, 4, 5
    perm = rng.permutation(n)
    J, Jc = perm[:k], perm[k:]
    AJ = synth.cgauss(rng, (m, k))
    T = synth.cgauss(rng, (k, n - k))
    u = synth.cgauss(rng, (m,))
    u /= np.linalg.norm(u)
    v = synth.cgauss(rng, (n - k,))
    v /= np.linalg.norm(v)
    sigma = 3e-7
    A = np.zeros((m, n), dtype=np.complex128)
    A[:, J] = AJ
    A[:, Jc] = AJ @ T + sigma * np.outer(u, v.conj())
    G = o.left_probe_matrix(r, m, 7)
    assert G.shape == (r, m)
    est, upper, Z = o.error_estimate_left(A, perm, T, G)
    gu = np.array([abs(sum(G[q, i] * u[i] for i in range(m))) for q in range(r)])
    gn = np.array([math.sqrt(sum(abs(G[q, i]) ** 2 for i in range(m))) for q in range(r)])
    # rounding of A_Jc - A_J T (entries O(k)) leaves ~1e-15 k on a residual of 3e-7
    assert abs(est - sigma * np.max(gu / gn)) <= 1e-6 * sigma * np.max(gu / gn)
    assert abs(upper - 10.0 * math.sqrt(2.0 / math.pi) * sigma * np.max(gu)) <= 1e-6 * upper
    assert np.all(Z[:, J] == 0)
    # bounds on a real ID
    m, n, k = 90, 70, 5
    A = synth.lowrank_plus_noise(m, n, k, 1e-6, seed=22)
    out = o.rid(A, k, k + 6, seed=5)
    exact = o.exact_error(A, out["perm"], out["T"])
    for ps in (1, 2, 3):
        est, upper, _ = o.error_estimate_left(A, out["perm"], out["T"], o.left_probe_matrix(6, m, ps))
        assert 0.05 * exact <= est <= exact * (1 + 1e-9)
        assert exact <= upper


def pin_round_test_matrix(o):
    """Rounded rows: multiples of 2^(E - bits) with E the row's exponent, within
    half a step of the input, ties to even, idempotent; an entry that is already
    on the grid is unchanged (the row maximum keeps its value at any bits >= 1
    when it is a power of two)."""
    Om = o.gaussian_test_matrix(6, 300, 5)
    for bits in (8, 16, 24):
        R = o.round_test_matrix(Om, bits)
        for r in range(Om.shape[0]):
            parts = np.concatenate([Om[r].real, Om[r].imag])
            E = max(math.frexp(float(x))[1] for x in parts if x != 0.0)
            step = 2.0 ** (E - bits)
            for x, y in ((Om[r].real, R[r].real), (Om[r].imag, R[r].imag)):
                assert np.all(np.abs(y - x) <= step / 2)
                assert np.all(np.mod(y, step) == 0.0)
        assert np.array_equal(o.round_test_matrix(R, bits), R)
    # exact halves go to the even multiple: row maximum 0.75 (E = 0), step 2^-2
    row = np.array([[0.75 + 0.375j, 0.625 - 0.125j, 0.5 + 0.0j]])
    R = o.round_test_matrix(row, 2)
    assert np.array_equal(R, np.array([[0.75 + 0.5j, 0.5 - 0.0j, 0.5 + 0.0j]]))
    assert np.array_equal(o.round_test_matrix(np.zeros((1, 3), complex), 8), np.zeros((1, 3), complex))
    # a value that would round up to 2^E keeps the exponent: 1 - 2^-30 (E = 0) -> 255/256 at 8 bits
    row = np.array([[1.0 - 2.0 ** -30 - 1j * (1.0 - 2.0 ** -30), 0.25 + 0.0j]])
    assert np.array_equal(o.round_test_matrix(row, 8), np.array([[255 / 256 - 255j / 256, 0.25 + 0.0j]]))


# --- the paper's SRFT ---------------------------------------------------------
def pin_srft(o):
    """S F D A equals rows s of numpy's FFT (along columns) of D A."""
    m, n, l = 64, 9, 12
    A = synth.cgauss(np.random.default_rng(31), (m, n))
    phi, s = o.srft_parameters(l, m, seed=2)
    assert phi.shape == (m,) and s.shape == (l,) and s.min() >= 0 and s.max() < m
    Y = o.srft_randomize(A, l, seed=2)
    D = np.exp(2j * np.pi * phi)
    Yf = np.fft.fft(D[:, None] * A, axis=0)[s, :]
    assert np.abs(Y - Yf).max() <= 1e-12 * np.abs(Yf).max()


def pin_srft_distribution(o):
    """The SRFT's random parts (Sec. 2): phases phi uniform on [0, 1), row
    samples s uniform on {0..m-1}, drawn independently of Omega's stream and of
    each other."""
    m = 20000
    phi, _ = o.srft_parameters(4, m, seed=9)
    assert phi.min() >= 0.0 and phi.max() < 1.0
    assert scipy.stats.kstest(phi, "uniform").pvalue > 1e-4
    assert abs(np.corrcoef(phi[:-1], phi[1:])[0, 1]) < 0.03        # no serial dependence
    # independent of the Gaussian test matrix drawn under the same seed: the
    # angle of Omega's row-0 entries is that stream's uniform at the same counter
    om = o.gaussian_test_matrix(1, m, seed=9)[0]
    u_om = np.mod(np.angle(om) / (2.0 * np.pi), 1.0)
    assert abs(np.corrcoef(phi, u_om)[0, 1]) < 0.03
    assert np.mean(np.abs(phi - u_om) < 1e-12) < 0.01
    for m_s, l_s in ((16, 16000), (1000, 50000)):
        _, s = o.srft_parameters(l_s, m_s, seed=4)
        assert s.dtype.kind == "i" and s.min() >= 0 and s.max() < m_s
        counts = np.bincount(s, minlength=m_s)
        assert scipy.stats.chisquare(counts).pvalue > 1e-4, m_s
    phi2, s2 = o.srft_parameters(20000, 20000, seed=4)
    assert abs(np.corrcoef(phi2, s2 / 20000.0)[0, 1]) < 0.03       # phases and samples independent


ALL_PINS = [
    pin_philox_kat, pin_uniform53, pin_gaussian_distribution, pin_randomize_exact,
    pin_qr_lapack, pin_qr_pivot_rule, pin_rank_deficient, pin_factor_r, pin_exact_rank,
    pin_spectrum_bound, pin_brute_force, pin_error_estimate, pin_error_estimate_left, pin_round_test_matrix, pin_srft,
    pin_srft_distribution,
]
