"""A rounded test matrix (rid_plan_round_omega) against the oracle's
round_test_matrix.

  * the rounding itself: bit for bit against oracle.round_test_matrix applied to
    the same plan's unrounded Omega;
  * the sketch: a rounded Omega holds bits / 8 digits, and the emulated product
    multiplies only those, so the tolerances are the same as for a full Omega
    (the dot-product bound plus the emulation bound of A's digits); integer
    inputs stay bit-exact;
  * the whole ID on the plan's own (rounded) Omega: J exactly, T within 1e-10;
  * probes set before or after the rounding are rounded as well.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dot_bound, row_probe_tolerances, to_dev_colmajor, to_host

pytestmark = pytest.mark.gpu

SHAPES = [(2048, 1024, 32, 40), (1000, 777, 17, 25), (4096, 333, 1, 3), (513, 129, 9, 9)]
MODES = ["fp64", "fp64_emulated"]


@pytest.fixture(scope="module")
def rid():
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    return rid


def emulation_bound(Om, A):
    m = A.shape[0]
    return 2.0 ** -46 * (2 * m) * np.outer(np.abs(Om).max(axis=1), np.abs(A).max(axis=0))


@pytest.mark.parametrize("bits", [8, 16, 24, 48])
@pytest.mark.parametrize("shape", SHAPES[:2], ids=str)
def test_rounding_matches_oracle_bit_for_bit(rid, shape, bits):
    m, n, k, l = shape
    with rid.Plan(m, n, k, l, seed=11) as plan:
        Om0 = to_host(plan.omega())
        plan.round_omega(bits)
        Om = to_host(plan.omega())
    R = oracle.round_test_matrix(Om0, bits)
    assert np.array_equal(Om.view(np.float64), R.view(np.float64))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("bits", [16, 24])
@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_rounded_sketch_matches_oracle(rid, shape, bits, mode):
    m, n, k, l = shape
    A = synth.lowrank_plus_noise(m, n, k, 1e-10, seed=m + n)
    with rid.Plan(m, n, k, l, seed=12, mode=mode) as plan:
        plan.round_omega(bits)
        Om = to_host(plan.omega())
        Y = to_host(plan.sketch(to_dev_colmajor(A)))
    Yo = oracle.randomize(Om, A)
    bound = dot_bound(Om, A)
    if mode == "fp64_emulated":
        bound = bound + emulation_bound(Om, A)
    assert np.all(np.abs(Y - Yo) <= bound)


@pytest.mark.parametrize("mode", MODES)
def test_rounded_sketch_integer_inputs_bit_exact(rid, mode):
    # 8-bit rows times integers |a| <= 2^7: every product and partial sum is exact
    m, n, k, l = 3000, 200, 5, 12
    A = synth.integer_valued(m, n, 7, seed=3)
    with rid.Plan(m, n, k, l, seed=13, mode=mode) as plan:
        plan.round_omega(8)
        Om = to_host(plan.omega())
        Y = to_host(plan.sketch(to_dev_colmajor(A)))
    assert np.array_equal(Y, oracle.randomize(Om, A))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_rounded_whole_id_matches_oracle(rid, shape, mode):
    m, n, k, l = shape
    A = synth.lowrank_plus_noise(m, n, k, 1e-10, seed=2 * m + n)
    with rid.Plan(m, n, k, l, seed=14, mode=mode) as plan:
        plan.round_omega(16)
        Om = to_host(plan.omega())
        res = rid.decompose(to_dev_colmajor(A), k, l, plan=plan)
    out = oracle.rid(A, k, l, seed=14, Omega=Om)
    perm, T = to_host(res["perm"]), to_host(res["T"])
    assert np.array_equal(perm[:k], out["J"])
    if T.size:
        assert np.abs(T - out["T"]).max() <= 1e-10 * np.abs(out["T"]).max()


def test_probes_are_rounded_in_either_order(rid):
    m, n, k, l = 1500, 400, 10, 20
    A = synth.lowrank_plus_noise(m, n, k, 1e-8, seed=5)
    Ad = to_dev_colmajor(A)
    results = []
    for first in ("probes", "round"):
        with rid.Plan(m, n, k, l, seed=15, mode="fp64_emulated") as plan:
            if first == "probes":
                plan.set_probes(6, 3)
                plan.round_omega(24)
            else:
                plan.round_omega(24)
                plan.set_probes(6, 3)
            Y = plan.sketch(Ad)
            perm = plan.select(Y)
            T = plan.solve(Y)
            results.append((plan.error_sketched(perm, T), to_host(perm), to_host(T)))
    (e0, p0, t0), (e1, p1, t1) = results
    assert e0 == e1 and np.array_equal(p0, p1) and np.array_equal(t0, t1)
    G = oracle.round_test_matrix(oracle.left_probe_matrix(6, m, 3), 24)
    est_o, up_o, _ = oracle.error_estimate_left(A, p0, t0, G)
    tol_est, tol_up = row_probe_tolerances(A, p0, t0, G, "fp64_emulated")
    # a probe entry that sits on a rounding boundary may round the other way on
    # the two sides (their generators agree to 1e-14): 2^-24 of that entry
    tol_est += 2.0 ** -24 * est_o
    tol_up += 2.0 ** -24 * up_o
    assert abs(e0[0] - est_o) <= tol_est and abs(e0[1] - up_o) <= tol_up


def test_round_omega_argument_errors(rid):
    from paper_1205_3830_gb300._native import RIDError
    with rid.Plan(256, 100, 5, 10, seed=1) as plan:
        for bits in (0, 7, 12, 56, 64):
            with pytest.raises(RIDError, match="EINVAL"):
                plan.round_omega(bits)
