"""Seeded synthetic inputs for the randomized ID (shared by tests and bench).

This module only draws input matrices and workload descriptions; it contains
none of the ID's own arithmetic (no sketch, no QR, no solve), so both the CPU
oracle and the CUDA path can be fed from it.  The random numbers the method
itself draws (the test matrix Omega, the error probes) are NOT made here: each
side generates them from the published Philox4x32-10 definition.

Workload recipe (the paper benchmarks dense low-rank complex Gaussian matrices,
A = B P with Gaussian factors, Sec. 3.3):
  * low rank plus noise: A = X Y + eps N with X (m x r), Y (r x n), N (m x n),
    all entries complex with re, im iid N(0, 1/2);
  * prescribed spectrum: A = U diag(sigma) V^H with U, V orthonormalised
    complex Gaussian (flat top spectrum, tiny tail);
  * integer valued: small Gaussian integers, for bit-exact sums.
All host draws use numpy's PCG64 generator seeded with the given seed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASTER_SEED = 12053830


def cgauss(rng, shape, dtype=np.complex128):
    """Complex normal array with re, im iid N(0, 1/2)."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return ((re + 1j * im) * math.sqrt(0.5)).astype(dtype)


def lowrank_plus_noise(m, n, rank, eps, seed, dtype=np.complex128):
    """A = X Y + eps N (column-major friendly: returned Fortran-ordered)."""
    rng = np.random.default_rng(seed)
    X = cgauss(rng, (m, rank))
    Y = cgauss(rng, (rank, n))
    A = X @ Y
    if eps:
        A = A + eps * cgauss(rng, (m, n))
    return np.asfortranarray(A.astype(dtype))


def orthonormal_columns(rng, rows, cols):
    """Q of the thin QR of a complex Gaussian rows x cols matrix."""
    G = cgauss(rng, (rows, cols))
    Q, _ = np.linalg.qr(G)
    return Q


def prescribed_spectrum(m, n, sigma, seed):
    """A = U diag(sigma) V^H with orthonormalised complex Gaussian U (m x r), V (n x r),
    r = len(sigma) <= min(m, n)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.size
    rng = np.random.default_rng(seed)
    U = orthonormal_columns(rng, m, r)
    V = orthonormal_columns(rng, n, r)
    return np.asfortranarray((U * sigma[None, :]) @ V.conj().T)


def integer_valued(m, n, bound, seed):
    """Gaussian integers with |re|, |im| <= bound (exact in every sum we form)."""
    rng = np.random.default_rng(seed)
    re = rng.integers(-bound, bound + 1, size=(m, n))
    im = rng.integers(-bound, bound + 1, size=(m, n))
    return np.asfortranarray((re + 1j * im).astype(np.complex128))


# ---------------------------------------------------------------------------
# The benchmark configurations (sizes of the paper's workloads, Sec. 3.3)
# ---------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class IDConfig:
    name: str
    m: int
    n: int
    k: int
    l: int
    kind: str            # "lowrank" or "spectrum"
    eps: float           # noise level (lowrank) or tail singular value (spectrum)
    rank: int            # rank of X Y, or number of unit singular values
    dtype: str = "c128"
    seed: int = MASTER_SEED

    @property
    def a_bytes(self):
        return self.m * self.n * (16 if self.dtype == "c128" else 8)


CONFIGS = {
    # plain FP64 ID: A = X Y + 1e-10 N, X 2048x32, Y 32x1024; k = 32, l = 40
    "plain_fp64": IDConfig("plain_fp64", 2048, 1024, 32, 40, "lowrank", 1e-10, 32,
                           seed=MASTER_SEED + 0),
    # large FP64 ID, square: m = n = 32768 (16 GiB), sigma = 1 (200x) then 1e-12
    "large_square": IDConfig("large_square", 32768, 32768, 200, 208, "spectrum", 1e-12, 200,
                             seed=MASTER_SEED + 1),
    # large FP64 ID, non-square: m = 262144, n = 8192 (32 GiB), same spectrum
    "large_tall": IDConfig("large_tall", 262144, 8192, 200, 208, "spectrum", 1e-12, 200,
                           seed=MASTER_SEED + 2),
    # mixed-precision sketch: A = X Y + 1e-5 N stored complex64, 65536 x 16384, k = 100, l = 110
    "mixed_c64": IDConfig("mixed_c64", 65536, 16384, 100, 110, "lowrank", 1e-5, 100,
                          dtype="c64", seed=MASTER_SEED + 3),
}


def host_matrix(cfg: IDConfig):
    """The config's A on the host (small configs only)."""
    if cfg.kind == "lowrank":
        A = lowrank_plus_noise(cfg.m, cfg.n, cfg.rank, cfg.eps, cfg.seed)
    else:
        rng = np.random.default_rng(cfg.seed)
        U = orthonormal_columns(rng, cfg.m, cfg.rank)
        V = orthonormal_columns(rng, cfg.n, cfg.rank)
        tail = cgauss(rng, (cfg.m, cfg.n)) * (cfg.eps / (math.sqrt(cfg.m) + math.sqrt(cfg.n)))
        A = np.asfortranarray(U @ V.conj().T + tail)
    if cfg.dtype == "c64":
        A = np.asfortranarray(A.astype(np.complex64))
    return A


def scaled_config(cfg: IDConfig, m, n, k=None, l=None):
    """The same recipe at other sizes (for oracle-sized parity cases)."""
    k = cfg.k if k is None else k
    l = cfg.l if l is None else l
    return dataclasses.replace(cfg, m=m, n=n, k=k, l=l, rank=min(k, m, n))


# ---------------------------------------------------------------------------
# Batched and serving workloads
# ---------------------------------------------------------------------------
def batched_shapes(count, seed, m_range=(64, 1024), n_range=(64, 1024), k_range=(4, 64), p=8):
    """count independent ID problems: m, n, k uniform integers, l = k + p."""
    rng = np.random.default_rng(seed)
    m = rng.integers(m_range[0], m_range[1] + 1, size=count)
    n = rng.integers(n_range[0], n_range[1] + 1, size=count)
    k = rng.integers(k_range[0], k_range[1] + 1, size=count)
    k = np.minimum(k, np.minimum(m, n))
    return [(int(a), int(b), int(c), int(c) + p) for a, b, c in zip(m, n, k)]


def serving_requests(count, rate_per_s, seed, mn_range=(256, 16384), k_range=(8, 256), p=10):
    """Poisson arrivals; m, n, k log-uniform; l = k + p.  Returns list of
    (arrival_time_s, m, n, k, l)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)

    def logu(lo, hi, size):
        return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size)).astype(np.int64)

    m = logu(*mn_range, count)
    n = logu(*mn_range, count)
    k = np.minimum(logu(*k_range, count), np.minimum(m, n))
    return [(float(a), int(b), int(c), int(d), int(d) + p) for a, b, c, d in zip(t, m, n, k)]
