"""Seeded synthetic inputs generated directly on the GPU with torch (input
tooling for the multi-GB configurations; none of the ID's arithmetic).

Same recipes as synth.host_matrix, drawn with torch's seeded CUDA generator
(re, im iid N(0, 1/2) for complex randn).  A is returned column-major
(stride(0) == 1).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import IDConfig, orthonormal_columns


def _colmajor_randn(rows, cols, gen, device, dtype=torch.complex128):
    return torch.randn((cols, rows), generator=gen, dtype=dtype, device=device).t()


def device_matrix(cfg: IDConfig, device="cuda"):
    gen = torch.Generator(device=device)
    gen.manual_seed(int(cfg.seed))
    m, n, r = cfg.m, cfg.n, cfg.rank
    c128 = torch.complex128
    if cfg.kind == "lowrank":
        X = torch.randn((m, r), generator=gen, dtype=c128, device=device)
        Y = torch.randn((r, n), generator=gen, dtype=c128, device=device)
        if cfg.eps:
            A = _colmajor_randn(m, n, gen, device).mul_(cfg.eps)
        else:
            A = torch.zeros((n, m), dtype=c128, device=device).t()
        A.addmm_(X, Y)
        del X, Y
    else:
        # A = U V^H + tail: U, V orthonormalised complex Gaussian (m x r, n x r),
        # tail = eps / (sqrt(m) + sqrt(n)) * G, whose largest singular value is
        # about eps (edge of the Marchenko-Pastur law), so sigma_j = 1 for j <= r
        # and sigma_j <~ eps after.
        # (the thin QRs run in numpy on the host: tall-skinny, a second or two)
        rng = np.random.default_rng(int(cfg.seed))
        U = torch.from_numpy(orthonormal_columns(rng, m, r)).to(device)
        V = torch.from_numpy(orthonormal_columns(rng, n, r)).to(device)
        A = _colmajor_randn(m, n, gen, device).mul_(cfg.eps / (math.sqrt(m) + math.sqrt(n)))
        A.addmm_(U, V.conj().t())
        del U, V
    if cfg.dtype == "c64":
        A = A.t().to(torch.complex64).t()
    return A
