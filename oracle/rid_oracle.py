"""Plain FP64 CPU oracle for the randomized interpolative decomposition (ID).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product path (``paper_1205_3830_gb300``) never imports it, and this
module imports nothing from the product path: the two share no code.

What it computes (Lucas, Stalzer & Feo, "Parallel implementation of fast
randomized algorithms for the decomposition of low rank matrices", Sec. 2):
an m x n complex matrix A of approximate rank k is written A ~= B P with
B = A(:, J) (k chosen columns of A) and P = [I | T] Pi^T.  The steps, in the
paper's order and notation:

1. randomization  Y = Omega A                     (Sec. 2, "Y = S F D A"; the
   paper allows any faster randomization in place of the SRFT, end of Sec. 2;
   here Omega is an l x m complex Gaussian test matrix, l = k + p)
2. truncated QR   Y Pi ~= Q [R1 | R2]             (Sec. 2, "Y ~= Q R", with the
   column permutation the paper asks for chosen by column pivoting)
3. factor R       R2 = R1 T,  P = [I | T] Pi^T     (Sec. 2, "R2 = R1 T", "P = (I T)")
4. error          ||A - B P||_2                    (Sec. 3.3, Table 5; measured
   here with Gaussian probes, since the paper does not say how)
plus the paper's own SRFT randomization Y = S F D A (Sec. 2, the three
definitions of S, F and D) for comparison.

Everything is complex128 and written for a reader to check against the
paper by eye: loops run in the paper's order, and numpy is used only for
single library primitives (a matrix product, a dot product, an FFT).

Parity status: every function below is pinned by tests/test_oracle_pins.py
(known-answer vectors, closed forms, LAPACK special cases, brute force and
invariants).  No function here is "parity unpinned".
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "RankDeficient",
    "philox4x32_10",
    "uniform53_pair",
    "complex_gaussian",
    "gaussian_test_matrix",
    "round_test_matrix",
    "probe_matrix",
    "randomize",
    "householder_reflector",
    "qr_select",
    "factor_r",
    "interpolation_matrix",
    "error_estimate",
    "exact_error",
    "rid",
    "srft_randomize",
    "srft_parameters",
    "STREAM_OMEGA",
    "STREAM_PROBES",
    "STREAM_SRFT",
    "STREAM_LPROBES",
    "left_probe_matrix",
    "error_estimate_left",
]

# Philox counter "stream" word for each random object of the method.
STREAM_OMEGA = 3   # the l x m Gaussian test matrix Omega
STREAM_PROBES = 4  # the n x r Gaussian probes of the error estimate
STREAM_SRFT = 5    # the SRFT's random phases D and row samples S
STREAM_LPROBES = 6 # the r x m Gaussian row probes of the row-probe error estimate


class RankDeficient(ArithmeticError):
    """Raised when the sketch Y has rank < k: every remaining column norm is
    exactly zero before k pivots were chosen.  Sec. 2: the remedy is to repeat
    with a different instance of the random matrices (a new seed)."""


# ---------------------------------------------------------------------------
# Counter-based random numbers: Philox4x32-10
# (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3",
#  SC 2011, Sec. 3.2).  Each round multiplies words 0 and 2 by fixed 32-bit
#  constants, swaps the high/low halves into a new word order and XORs in the
#  round key; the key is bumped by two Weyl constants between rounds.
# ---------------------------------------------------------------------------
_PHILOX_M0 = 0xD2511F53
_PHILOX_M1 = 0xCD9E8D57
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds.

    counter: integer array of shape (..., 4), each entry in [0, 2^32).
    key:     pair (k0, k1) of integers in [0, 2^32).
    Returns a uint32 array of shape (..., 4).
    """
    c = np.asarray(counter, dtype=np.uint64)
    x0, x1, x2, x3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = int(key[0]) & _MASK32, int(key[1]) & _MASK32
    m0, m1, mask = np.uint64(_PHILOX_M0), np.uint64(_PHILOX_M1), np.uint64(_MASK32)
    s32 = np.uint64(32)
    for _ in range(10):
        p0 = x0 * m0            # < 2^64: exact in uint64
        p1 = x2 * m1
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        x0, x1, x2, x3 = hi1 ^ x1 ^ np.uint64(k0), lo1, hi0 ^ x3 ^ np.uint64(k1), lo0
        k0 = (k0 + _PHILOX_W0) & _MASK32
        k1 = (k1 + _PHILOX_W1) & _MASK32
    return np.stack([x0, x1, x2, x3], axis=-1).astype(np.uint32)


def uniform53_pair(words):
    """Two 53-bit uniforms from one Philox output block (..., 4).

    u1 = ((w0 >> 5) * 2^26 + (w1 >> 6) + 1) * 2^-53 lies in (0, 1] (safe for log);
    u2 = ((w2 >> 5) * 2^26 + (w3 >> 6)) * 2^-53 lies in [0, 1).
    Both are exact in double precision.
    """
    w = np.asarray(words, dtype=np.uint64)
    a = (w[..., 0] >> np.uint64(5)) * np.uint64(1 << 26) + (w[..., 1] >> np.uint64(6))
    b = (w[..., 2] >> np.uint64(5)) * np.uint64(1 << 26) + (w[..., 3] >> np.uint64(6))
    scale = 2.0 ** -53
    u1 = (a.astype(np.float64) + 1.0) * scale
    u2 = b.astype(np.float64) * scale
    return u1, u2


def complex_gaussian(rows, cols, seed, stream, row0=0, col0=0):
    """rows x cols complex normal matrix, re and im iid N(0, 1/2).

    Entry (i, j) (global indices i + row0, j + col0) takes the Philox block at
    counter (j mod 2^32, j div 2^32, i, stream) under key (seed mod 2^32,
    seed div 2^32), and Box-Muller: rho = sqrt(-log u1), z = rho * exp(2 pi i u2).
    Then |z|^2 ~ Exp(1), so E|z|^2 = 1.
    """
    i = np.arange(row0, row0 + rows, dtype=np.uint64)[:, None]
    j = np.arange(col0, col0 + cols, dtype=np.uint64)[None, :]
    ctr = np.empty((rows, cols, 4), dtype=np.uint64)
    ctr[..., 0] = j & np.uint64(_MASK32)
    ctr[..., 1] = j >> np.uint64(32)
    ctr[..., 2] = i
    ctr[..., 3] = np.uint64(stream)
    seed = int(seed)
    words = philox4x32_10(ctr, (seed & _MASK32, (seed >> 32) & _MASK32))
    u1, u2 = uniform53_pair(words)
    rho = np.sqrt(-np.log(u1))
    theta = 2.0 * np.pi * u2
    return rho * np.cos(theta) + 1j * (rho * np.sin(theta))


def gaussian_test_matrix(l, m, seed):
    """The l x m complex Gaussian test matrix Omega of the randomization step."""
    return complex_gaussian(l, m, seed, STREAM_OMEGA)


def round_test_matrix(Omega, bits):
    """Omega with every entry rounded to `bits` bits below its row's largest entry.

    Row r gets the exponent E_r with |Re w|, |Im w| < 2^E_r for all its entries
    (E_r = the largest binary exponent e of x = f 2^e, 1/2 <= |f| < 1), and each
    real part is rounded to the nearest multiple of 2^(E_r - bits), ties to even;
    a value that would reach +-2^E_r takes the multiple just below it, so the
    row keeps its exponent.  Any random matrix serves as the test matrix of the
    randomization (Sec. 2 uses the SRFT); a rounded one holds bits / 8 base-256
    digits exactly.
    """
    Omega = np.array(Omega, dtype=np.complex128)
    for r in range(Omega.shape[0]):
        row = Omega[r]
        parts = np.concatenate([row.real, row.imag])
        nz = parts[parts != 0.0]
        if nz.size == 0:
            continue
        E = int(np.max(np.frexp(nz)[1]))
        top = 2.0 ** bits - 1.0
        re = np.ldexp(np.clip(np.rint(np.ldexp(row.real, bits - E)), -top, top), E - bits)
        im = np.ldexp(np.clip(np.rint(np.ldexp(row.imag, bits - E)), -top, top), E - bits)
        Omega[r] = re + 1j * im
    return Omega


def probe_matrix(n, r, seed):
    """The n x r complex Gaussian probes of the error estimate (row = column of A)."""
    return complex_gaussian(n, r, seed, STREAM_PROBES)


def left_probe_matrix(r, m, seed):
    """The r x m complex Gaussian row probes of the row-probe error estimate."""
    return complex_gaussian(r, m, seed, STREAM_LPROBES)


# ---------------------------------------------------------------------------
# Step 1: randomization  Y = Omega A   (Sec. 2)
# ---------------------------------------------------------------------------
def randomize(Omega, A):
    """Y = Omega A, the l x n sketch.  One library matrix product in FP64."""
    Omega = np.asarray(Omega, dtype=np.complex128)
    A = np.asarray(A, dtype=np.complex128)
    return Omega @ A


# ---------------------------------------------------------------------------
# Step 2: truncated QR with column pivoting on Y   (Sec. 2, "Y ~= Q R")
# ---------------------------------------------------------------------------
def householder_reflector(alpha, x):
    """Elementary reflector H = I - tau v v^H with H^H (alpha, x) = (beta, 0).

    Convention of LAPACK's zlarfg: beta is real, beta = -sign(Re alpha) *
    ||(alpha, x)||_2 (sign(0) = +), tau = (beta - alpha) / beta,
    v = (1, x / (alpha - beta)).  When x = 0 and alpha is real, H = I (tau = 0).
    Returns (beta, tau, v_tail).
    """
    x = np.asarray(x, dtype=np.complex128)
    alphr, alphi = float(np.real(alpha)), float(np.imag(alpha))
    xnorm2 = float(np.sum(x.real * x.real + x.imag * x.imag))
    if xnorm2 == 0.0 and alphi == 0.0:
        return complex(alphr, 0.0), 0j, np.zeros_like(x)
    nrm = math.sqrt(alphr * alphr + alphi * alphi + xnorm2)
    beta = -nrm if alphr >= 0.0 else nrm
    tau = complex((beta - alphr) / beta, -alphi / beta)
    scale = 1.0 / (complex(alphr, alphi) - beta)
    return complex(beta, 0.0), tau, x * scale


def qr_select(Y, k):
    """k steps of Householder QR with column pivoting (Businger-Golub) on Y.

    At step j: recompute nu_c = sum_{i >= j} |Y_ic|^2 for every column c >= j,
    pick p = the first column of largest nu (ties -> lowest current index),
    stop with RankDeficient if nu_p == 0, swap columns j and p (and perm),
    form the reflector of column j below row j-1, apply H^H = I - conj(tau) v v^H
    to the columns right of j.

    Returns (R, tau, perm): R is Y overwritten (rows 0..k-1 hold [R1 | R2] in
    pivoted column order, Householder vectors below the diagonal), perm[c] is
    the original index of pivoted column c, so J = perm[:k].
    """
    R = np.array(Y, dtype=np.complex128, copy=True)
    l, n = R.shape
    if not (1 <= k <= min(l, n)):
        raise ValueError("need 1 <= k <= min(l, n)")
    perm = np.arange(n, dtype=np.int64)
    tau = np.zeros(k, dtype=np.complex128)
    for j in range(k):
        tail = R[j:, j:]
        nu = np.sum(tail.real * tail.real + tail.imag * tail.imag, axis=0)
        p = j + int(np.argmax(nu))          # argmax returns the first maximum
        if nu[p - j] == 0.0:
            raise RankDeficient(f"sketch has rank {j} < k = {k}")
        if p != j:
            R[:, [j, p]] = R[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        beta, tau_j, v_tail = householder_reflector(R[j, j], R[j + 1:, j])
        R[j, j] = beta
        R[j + 1:, j] = v_tail
        tau[j] = tau_j
        if j + 1 < n and tau_j != 0:
            v = np.concatenate(([1.0 + 0j], v_tail))
            C = R[j:, j + 1:]
            w = v.conj() @ C                 # w = v^H C
            C -= np.conj(tau_j) * np.outer(v, w)
    return R, tau, perm


# ---------------------------------------------------------------------------
# Step 3: factor R   (Sec. 2, "R2 = R1 T" and "P = (I T)")
# ---------------------------------------------------------------------------
def factor_r(R1, R2):
    """T with R1 T = R2 by back substitution (R1 k x k upper triangular).

    Row i of T, from the last row up:  T_i = (R2_i - sum_{t > i} R1_it T_t) / R1_ii.
    Every right-hand side column is independent (Sec. 3.2).
    """
    R1 = np.asarray(R1, dtype=np.complex128)
    R2 = np.asarray(R2, dtype=np.complex128)
    k = R1.shape[0]
    T = np.zeros_like(R2)
    for i in range(k - 1, -1, -1):
        T[i, :] = (R2[i, :] - R1[i, i + 1:] @ T[i + 1:, :]) / R1[i, i]
    return T


def interpolation_matrix(perm, T, n):
    """Dense k x n P with P(:, perm[j]) = e_j (j < k) and P(:, perm[k + i]) = T(:, i)."""
    k = T.shape[0]
    P = np.zeros((k, n), dtype=np.complex128)
    perm = np.asarray(perm)
    P[np.arange(k), perm[:k]] = 1.0
    P[:, perm[k:]] = T
    return P


# ---------------------------------------------------------------------------
# Step 4: error of the ID   (Sec. 3.3, Table 5 reports ||A - B P||_2)
# ---------------------------------------------------------------------------
def error_estimate(A, perm, T, omega):
    """Probe estimate of ||A - B P||_2 with B = A(:, J).

    For each probe column w of omega (n x r), E w = A w~ where w~(Jc) = w(Jc)
    and w~(J) = -T w(Jc), since (A - A_J P) w = A_Jc w_Jc - A_J T w_Jc.
    Returns (est, upper, Ew): est = max_q ||E w_q|| / ||w_q|| (never above
    ||E||_2) and upper = 10 sqrt(2/pi) max_q ||E w_q|| (Halko, Martinsson &
    Tropp, SIAM Review 2011, Lemma 4.1: holds with probability >= 1 - 10^-r).
    """
    A = np.asarray(A, dtype=np.complex128)
    omega = np.asarray(omega, dtype=np.complex128)
    perm = np.asarray(perm)
    k = T.shape[0]
    J, Jc = perm[:k], perm[k:]
    w = omega.copy()
    w[J, :] = -(T @ omega[Jc, :])
    Ew = A @ w
    e_norm = np.sqrt(np.sum(Ew.real ** 2 + Ew.imag ** 2, axis=0))
    w_norm = np.sqrt(np.sum(omega.real ** 2 + omega.imag ** 2, axis=0))
    est = float(np.max(e_norm / w_norm))
    upper = float(10.0 * math.sqrt(2.0 / math.pi) * np.max(e_norm))
    return est, upper, Ew


def error_estimate_left(A, perm, T, G):
    """Row-probe estimate of ||A - B P||_2 with B = A(:, J).

    E = A - A(:, J) P is formed densely from its definition and Z = G E for the
    r x m row probes G.  Returns (est, upper, Z): est = max_q ||Z_q|| / ||G_q||
    (never above ||E||_2) and upper = 10 sqrt(2/pi) max_q ||Z_q||.  This is the
    probe bound of Halko, Martinsson & Tropp (SIAM Review 2011, Lemma 4.1)
    applied to E^T, whose 2-norm is that of E; it needs G independent of E,
    which holds because E depends on A and Omega only.
    """
    A = np.asarray(A, dtype=np.complex128)
    G = np.asarray(G, dtype=np.complex128)
    n = A.shape[1]
    k = T.shape[0]
    P = interpolation_matrix(perm, T, n)
    E = A - A[:, np.asarray(perm)[:k]] @ P
    Z = G @ E
    z_norm = np.sqrt(np.sum(Z.real ** 2 + Z.imag ** 2, axis=1))
    g_norm = np.sqrt(np.sum(G.real ** 2 + G.imag ** 2, axis=1))
    est = float(np.max(z_norm / g_norm))
    upper = float(10.0 * math.sqrt(2.0 / math.pi) * np.max(z_norm))
    return est, upper, Z


def exact_error(A, perm, T):
    """||A - A(:, J) P||_2 by a library SVD (small inputs only)."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[1]
    k = T.shape[0]
    P = interpolation_matrix(perm, T, n)
    return float(np.linalg.norm(A - A[:, np.asarray(perm)[:k]] @ P, 2))


# ---------------------------------------------------------------------------
# The whole ID
# ---------------------------------------------------------------------------
def rid(A, k, l, seed, Omega=None):
    """Randomized ID of A: returns dict with Omega, Y, R, tau, perm, J, T, P.

    Omega defaults to the seeded Gaussian test matrix gaussian_test_matrix(l, m, seed).
    """
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    if Omega is None:
        Omega = gaussian_test_matrix(l, m, seed)
    Y = randomize(Omega, A)
    R, tau, perm = qr_select(Y, k)
    T = factor_r(R[:k, :k], R[:k, k:])
    return {
        "Omega": Omega, "Y": Y, "R": R, "tau": tau, "perm": perm,
        "J": perm[:k].copy(), "T": T, "P": interpolation_matrix(perm, T, n),
    }


# ---------------------------------------------------------------------------
# The paper's own randomization: Y = S F D A   (Sec. 2)
# ---------------------------------------------------------------------------
def srft_parameters(l, m, seed):
    """Random phases phi (m,) uniform on [0, 1) and row samples s (l,) uniform
    on {0..m-1}, both from Philox stream STREAM_SRFT.

    phi_j uses the first uniform (u2 word pair) of block (j, 0); s_q uses the
    block (q, 1): s_q = floor(u2 * m).
    """
    seed = int(seed)
    key = (seed & _MASK32, (seed >> 32) & _MASK32)
    ctr = np.zeros((m, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(m, dtype=np.uint64) & np.uint64(_MASK32)
    ctr[:, 1] = np.arange(m, dtype=np.uint64) >> np.uint64(32)
    ctr[:, 2] = 0
    ctr[:, 3] = STREAM_SRFT
    _, phi = uniform53_pair(philox4x32_10(ctr, key))
    ctr = np.zeros((l, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(l, dtype=np.uint64)
    ctr[:, 2] = 1
    ctr[:, 3] = STREAM_SRFT
    _, u = uniform53_pair(philox4x32_10(ctr, key))
    s = np.minimum(np.floor(u * m).astype(np.int64), m - 1)
    return phi, s


def srft_randomize(A, l, seed):
    """Y = S F D A with D = diag(exp(2 pi i phi_j)), F_jk = exp(-2 pi i j k / m)
    (0-based), and S selecting rows s_1..s_l of F D A.

    Written as the definition: row q of Y is sum_j F[s_q, j] D_jj A[j, :].
    """
    A = np.asarray(A, dtype=np.complex128)
    m = A.shape[0]
    phi, s = srft_parameters(l, m, seed)
    DA = np.exp(2j * np.pi * phi)[:, None] * A
    j = np.arange(m)
    jk = np.outer(s, j) % m                        # exact integer phase index
    F_rows = np.exp(-2j * np.pi * (jk / m))         # the l sampled rows of F
    return F_rows @ DA
