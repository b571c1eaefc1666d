"""Helpers for the GPU parity tests: move numpy arrays to column-major device
tensors and back, and error bounds derived from the arithmetic."""
import numpy as np
import torch

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
