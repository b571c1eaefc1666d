"""Full-size parity: the two large FP64 configurations, in the launch
configuration bench.py times, against the CPU oracle run on the same A
(copied to the host) with its own Omega.  The oracle's sketch is one library
product (minutes of host BLAS at most); its QR and solve run on the l x n sketch.

Tolerances: J exactly (sigma_200 / sigma_201 = 1e12 here); T within 1e-10
max|T|; Y within the dot-product bound 4 gamma_m ||Omega_i|| ||A_j||
(Cauchy-Schwarz form of the entrywise bound, since |Omega| |A| would cost a
second full product); the error estimate on the oracle's own (perm, T) within
the rounding bound of E w.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U64, to_dev_colmajor

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def rid():
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    return rid


def run_case(rid, cfg, mode):
    import synth.device
    m, n, k, l = cfg.m, cfg.n, cfg.k, cfg.l
    A = synth.device.device_matrix(cfg)
    with rid.Plan(m, n, k, l, seed=cfg.seed, mode=mode) as plan:
        plan.set_probes(8, 7)                 # row probes ride along in the sketch
        Y = plan.sketch(A)
        Y_h = Y.cpu().numpy()
        perm = plan.select(Y)
        T = plan.solve(Y)
        plan.sync_status()
        perm_h, T_h = perm.cpu().numpy(), T.cpu().numpy()
        A_h = np.asfortranarray(A.cpu().numpy())
        # oracle, step by step, on the same A with its own Omega
        Om = oracle.gaussian_test_matrix(l, m, cfg.seed)
        Yo = oracle.randomize(Om, A_h)
        bound = 4 * (2 * m * U64) * np.outer(np.linalg.norm(Om, axis=1), np.linalg.norm(A_h, axis=0))
        if mode != "fp64":    # emulation: 2^-46 (2m) max|Omega_i| max|A_j|
            bound = bound + 2.0 ** -46 * (2 * m) * np.outer(np.abs(Om).max(axis=1), np.abs(A_h).max(axis=0))
        assert np.all(np.abs(Y_h - Yo) <= bound)
        Ro, _, perm_o = oracle.qr_select(Yo, k)
        To = oracle.factor_r(Ro[:k, :k], Ro[:k, k:])
        assert np.array_equal(perm_h[:k], perm_o[:k])
        assert np.abs(T_h - To).max() <= 1e-10 * np.abs(To).max()
        # the error estimate on the oracle's (perm, T): the CUDA path and the oracle agree
        r = 8
        est, up = plan.error(A, torch.from_numpy(perm_o.astype(np.int32)).cuda(), to_dev_colmajor(To), r, 5)
        omega = oracle.probe_matrix(n, r, 5)
        est_o, up_o, _ = oracle.error_estimate(A_h, perm_o, To, omega)
        w_abs = np.abs(omega)
        w_abs[perm_o[:k]] = np.abs(To) @ np.abs(omega[perm_o[k:]])
        bound_q = 4 * (n + k) * U64 * np.linalg.norm(np.abs(A_h) @ w_abs, axis=0)
        assert abs(est - est_o) <= np.max(bound_q / np.linalg.norm(omega, axis=0)) + 1e-12 * est_o
        assert abs(up - up_o) <= 10 * math.sqrt(2 / math.pi) * np.max(bound_q) + 1e-12 * up_o
        # sigma_{k+1} <~ 1e-12: the ID error obeys 10 sqrt(1 + k (n - k)) sigma_{k+1}
        assert est <= 10 * math.sqrt(1 + k * (n - k)) * 1.1 * cfg.eps
        # the row-probe estimate on the same (perm, T).  A dense E does not fit
        # on the host at this size; E(:, J) = 0 exactly, so the host forms
        # Z = X(Jc) - X(J) T from X = G A in FP64 (library products).
        est_s, up_s = plan.error_sketched(torch.from_numpy(perm_o.astype(np.int32)).cuda(), to_dev_colmajor(To))
        G = oracle.left_probe_matrix(8, m, 7)
        X = G @ A_h
        J, Jc = perm_o[:k], perm_o[k:]
        Z = X[:, Jc] - X[:, J] @ To
        gn = np.linalg.norm(G, axis=1)
        zn = np.linalg.norm(Z, axis=1)
        est_h, up_h = np.max(zn / gn), 10 * math.sqrt(2 / math.pi) * np.max(zn)
        absG = np.abs(G)
        dX = 2 * 4 * (2 * m * U64) * (absG @ np.abs(A_h))          # both sides' products
        if mode != "fp64":
            dX = dX + 2.0 ** -46 * (2 * m) * np.outer(absG.max(axis=1), np.abs(A_h).max(axis=0))
        absT = np.abs(To)
        dZ = dX[:, Jc] + dX[:, J] @ absT + 2 * 4 * (2 * k * U64) * (np.abs(X[:, J]) @ absT)
        B = np.linalg.norm(dZ, axis=1)
        assert abs(est_s - est_h) <= np.max(B / gn) + 1e-12 * est_h
        assert abs(up_s - up_h) <= 10 * math.sqrt(2 / math.pi) * np.max(B) + 1e-12 * up_h
        # both estimators bound the same ||E||_2 from below and above
        assert est_s <= up * (1 + 1e-9) and est <= up_s * (1 + 1e-9)


@pytest.mark.parametrize("mode", ["fp64", "fp64_emulated"])
def test_large_tall_32gib(rid, mode):
    run_case(rid, synth.CONFIGS["large_tall"], mode)


def test_large_square_16gib(rid):
    run_case(rid, synth.CONFIGS["large_square"], "fp64")
