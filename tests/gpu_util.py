"""Helpers for the GPU parity tests: move numpy arrays to column-major device
tensors and back, and error bounds derived from the arithmetic."""
import math

import numpy as np
import torch

import oracle

U64 = 2.0 ** -53     # unit roundoff of FP64


def to_dev_colmajor(a, dtype=torch.complex128):
    a = np.asfortranarray(a)
    t = torch.from_numpy(np.ascontiguousarray(a.T)).to(dtype)
    return t.cuda().t()


def to_dev_colmajor_ld(a, ld):
    """Column-major device copy with leading dimension ld > rows (padding rows are NaN)."""
    rows, cols = a.shape
    buf = torch.full((cols, ld), complex(float("nan"), float("nan")), dtype=torch.complex128)
    buf[:, :rows] = torch.from_numpy(np.ascontiguousarray(np.asarray(a).T))
    return buf.cuda().t()[:rows, :]


def to_host(t):
    return t.detach().cpu().numpy()


def dot_bound(Om, A):
    """Entrywise bound on |fl(Omega A) - Omega A| for two summation orders:
    2 * gamma_m * (|Omega| |A|) with gamma_m = m u / (1 - m u), complex
    products adding a factor sqrt(2) * 2 (textbook dot-product error bound)."""
    m = A.shape[0]
    gamma = 2 * m * U64 / (1 - 2 * m * U64)
    return 4.0 * gamma * (np.abs(Om) @ np.abs(A))


def row_probe_tolerances(A, perm, T, G, mode):
    """(tol_est, tol_upper) between the CUDA row-probe estimate, formed as
    Z_q = X_q(Jc) - X_q(J) T from X = G A, and the oracle's G_q (A - A_J P):
      dZ = dX(Jc) + dX(J) |T| + 4 gamma_k |X_J| |T|          (CUDA path)
         + 4 (gamma_m + gamma_k) |G| (|A| + |A_J| |P|)(Jc)    (oracle)
    with dX the sketch bound on X (plus the emulation bound for the emulated
    product); the two generators of G agree to 1e-14 relative, which moves the
    estimate by at most 1e-13 ||E||_F."""
    m, n = A.shape
    k = T.shape[0]
    J, Jc = perm[:k], perm[k:]
    gk = 2 * k * U64 / (1 - 2 * k * U64)
    gm = 2 * m * U64 / (1 - 2 * m * U64)
    X = G @ A
    dX = dot_bound(G, A)
    if mode == "fp64_emulated":
        dX = dX + 2.0 ** -46 * (2 * m) * np.outer(np.abs(G).max(axis=1), np.abs(A).max(axis=0))
    P = oracle.interpolation_matrix(perm, T, n)
    absT = np.abs(T)
    dZ = dX[:, Jc] + dX[:, J] @ absT + 4 * gk * (np.abs(X[:, J]) @ absT)
    dZ = dZ + 4 * (gm + gk) * (np.abs(G) @ (np.abs(A) + np.abs(A[:, J]) @ np.abs(P)))[:, Jc]
    B = np.linalg.norm(dZ, axis=1)
    gn = np.linalg.norm(G, axis=1)
    EF = np.linalg.norm(A - A[:, J] @ P)
    tol_est = np.max(B / gn) + 1e-13 * EF
    tol_up = 10 * math.sqrt(2 / math.pi) * (np.max(B) + 1e-13 * EF * np.max(gn))
    return tol_est, tol_up
