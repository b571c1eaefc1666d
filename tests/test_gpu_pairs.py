"""The CTA-pair form of the tensor-core product (16 or more column blocks of
128, tiles of 32 or more rows of Omega') against the oracle.

Shapes: an odd number of column blocks (the last pair multiplies a block of
zeros), a ragged last block of one column, an exact multiple, and a last
N-tile narrower than the others.  Tolerances are those of the single-CTA
parity tests: the dot-product bound plus the emulation bound
2^-46 (2m) max|Omega_i| max|A_j|; integer inputs bit for bit; J exactly and
T within 1e-10 of the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dot_bound, row_probe_tolerances, to_dev_colmajor, to_host

pytestmark = pytest.mark.gpu

# (m, n, k, l): 17 blocks (odd, ragged); 17 blocks with a 1-column last block
# and 32 rows of Omega'; 32 blocks exactly; 18 blocks with three N-tiles of
# 96, 96 and 68 rows (2l = 260)
SHAPES = [
    (1000, 2100, 20, 30),
    (513, 2049, 9, 16),
    (700, 4096, 60, 64),
    (600, 2304, 120, 130),
]


@pytest.fixture(scope="module")
def rid():
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    return rid


def emulation_bound(Om, A):
    m = A.shape[0]
    return 2.0 ** -46 * (2 * m) * np.outer(np.abs(Om).max(axis=1), np.abs(A).max(axis=0))


def lowrank(m, n, k, eps=1e-10, seed=0):
    return synth.lowrank_plus_noise(m, n, k, eps, seed=seed + 3 * m + 11 * n + k)


@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_pair_sketch_matches_oracle(rid, shape):
    m, n, k, l = shape
    A = lowrank(m, n, k)
    with rid.Plan(m, n, k, l, seed=31, mode="fp64_emulated") as plan:
        Om = to_host(plan.omega())
        Y = to_host(plan.sketch(to_dev_colmajor(A)))
    Yo = oracle.randomize(Om, A)
    assert np.all(np.abs(Y - Yo) <= dot_bound(Om, A) + emulation_bound(Om, A))


@pytest.mark.parametrize("shape", SHAPES[:2], ids=str)
def test_pair_sketch_integer_inputs_bit_exact(rid, shape):
    # Omega rounded to 8 bits below each row's maximum, |a| <= 2^7: every
    # product and every partial sum is exact
    m, n, k, l = shape
    A = synth.integer_valued(m, n, 7, seed=8)
    with rid.Plan(m, n, k, l, seed=32, mode="fp64_emulated") as plan:
        plan.round_omega(8)
        Om = to_host(plan.omega())
        Y = to_host(plan.sketch(to_dev_colmajor(A)))
    assert np.array_equal(Y, oracle.randomize(Om, A))


@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_pair_whole_id_matches_oracle(rid, shape):
    m, n, k, l = shape
    A = lowrank(m, n, k)
    with rid.Plan(m, n, k, l, seed=33, mode="fp64_emulated") as plan:
        res = rid.decompose(to_dev_colmajor(A), k, l, plan=plan)
    out = oracle.rid(A, k, l, seed=33)
    perm, T = to_host(res["perm"]), to_host(res["T"])
    assert np.array_equal(perm[:k], out["J"])
    assert np.abs(T - out["T"]).max() <= 1e-10 * np.abs(out["T"]).max()


@pytest.mark.parametrize("shape", SHAPES[:3], ids=str)
def test_pair_row_probes_match_oracle(rid, shape):
    m, n, k, l = shape
    A = lowrank(m, n, k, eps=1e-7)
    out = oracle.rid(A, k, l, seed=34)
    perm, T = out["perm"], out["T"]
    with rid.Plan(m, n, k, l, seed=34, mode="fp64_emulated") as plan:
        plan.set_probes(8, 12)
        plan.sketch(to_dev_colmajor(A))
        est, up = plan.error_sketched(torch.from_numpy(perm.astype(np.int32)).cuda(), to_dev_colmajor(T))
    G = oracle.left_probe_matrix(8, m, 12)
    est_o, up_o, _ = oracle.error_estimate_left(A, perm, T, G)
    tol_est, tol_up = row_probe_tolerances(A, perm, T, G, "fp64_emulated")
    assert abs(est - est_o) <= tol_est + 1e-14 * est_o
    assert abs(up - up_o) <= tol_up + 1e-14 * up_o
    assert est_o > 100 * tol_est


@pytest.mark.parametrize("width", [384, 640, 2048])
def test_pair_panels_equal_one_sketch(rid, width):
    """Column panels of an odd number of blocks: a launch's last pair takes
    the next panel's first block (or the spare block past the last) as its
    partner and must not write results for it."""
    m, n, k, l = 1000, 2100, 20, 30
    A = to_dev_colmajor(lowrank(m, n, k))
    with rid.Plan(m, n, k, l, seed=35, mode="fp64_emulated") as plan:
        plan.set_probes(8, 3)
        Y0 = plan.sketch(A).clone()
        R = Y0.clone()
        perm = plan.select(R)
        T = plan.solve(R)
        e0 = plan.error_sketched(perm, T)
        Y1 = torch.full_like(Y0, float("nan"))
        starts = list(range(0, n, width))
        for c0 in starts[1::2] + starts[0::2]:           # out of order
            plan.sketch_cols(A, Y1, c0, min(width, n - c0))
        e1 = plan.error_sketched(perm, T)
    assert torch.equal(Y0, Y1)
    assert e0 == e1


def test_pair_rounded_omega_matches_oracle(rid):
    m, n, k, l = 1000, 2100, 20, 30
    A = lowrank(m, n, k)
    with rid.Plan(m, n, k, l, seed=36, mode="fp64_emulated") as plan:
        plan.round_omega(24)
        Om = to_host(plan.omega())
        Y = to_host(plan.sketch(to_dev_colmajor(A)))
    Yo = oracle.randomize(Om, A)
    assert np.all(np.abs(Y - Yo) <= dot_bound(Om, A) + emulation_bound(Om, A))
