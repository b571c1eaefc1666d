"""The launch shapes of select give bitwise the same Y and permutation.

rid_plan_set_select_grid switches select between one cooperative launch of
the default grid, one of fewer CTAs, and one launch per step.  A column's
arithmetic, the pivot rule (largest remaining norm, ties to the lowest index)
and the reflector do not depend on which CTA or warp handles a column, so
every shape must return the same bits; the default shape is held to the
oracle as in the parity tests (J and the whole permutation exactly, R within
1e-12 max|R|).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_dev_colmajor, to_host

pytestmark = pytest.mark.gpu

# (m, n, k, l): l <= 256 and l > 256 (the two register budgets of the column
# update), a ragged n, k = l, and n smaller than two columns per warp
SHAPES = [
    (3000, 2000, 100, 110),
    (1000, 777, 17, 25),
    (2000, 1500, 280, 300),
    (300, 64, 64, 64),
    (600, 40, 8, 12),
]
GRIDS = [0, 1, 3, 7, 64]


@pytest.fixture(scope="module")
def rid():
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    return rid


def sketch(m, n, k, l, seed):
    A = synth.lowrank_plus_noise(m, n, k, 1e-10, seed=seed + 5 * m + 3 * n + k)
    return oracle.randomize(oracle.gaussian_test_matrix(l, m, seed), A)


@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_select_shapes_agree_bit_for_bit(rid, shape):
    m, n, k, l = shape
    Yo = sketch(m, n, k, l, 41)
    out = {}
    with rid.Plan(m, n, k, l, seed=41) as plan:
        default_launches = plan.stats()["select_launches"]
        for g in [-1] + GRIDS:
            plan.set_select_grid(g)
            assert plan.stats()["select_launches"] == (1 + k if g == 0 else default_launches if g < 0 else 1)
            Yd = to_dev_colmajor(Yo)
            perm = to_host(plan.select(Yd))
            plan.sync_status()
            out[g] = (perm, to_host(Yd))
    perm0, Y0 = out[-1]
    for g in GRIDS:
        assert np.array_equal(out[g][0], perm0), g
        assert np.ascontiguousarray(out[g][1]).tobytes() == np.ascontiguousarray(Y0).tobytes(), g
    Ro, _, perm_o = oracle.qr_select(Yo, k)
    assert np.array_equal(perm0, perm_o)
    upper = np.triu(np.ones((k, n), dtype=bool))
    assert np.abs(Y0[:k][upper] - Ro[:k][upper]).max() <= 1e-12 * np.abs(Ro[:k]).max()


def test_select_shape_reports_rank_deficiency(rid):
    """A sketch of rank 2 asked for k = 3: every shape reports RID_ERANK."""
    m, n, k, l = 200, 300, 3, 6
    rng = np.random.default_rng(7)
    Yo = np.zeros((l, n), dtype=np.complex128)
    Yo[:, 10] = synth.cgauss(rng, l)
    Yo[:, 200] = synth.cgauss(rng, l)
    with rid.Plan(m, n, k, l, seed=1) as plan:
        for g in [-1, 0, 2]:
            plan.set_select_grid(g)
            Yd = to_dev_colmajor(Yo)
            plan.select(Yd)
            with pytest.raises(rid.RIDError) as info:
                plan.sync_status()
            assert info.value.status == 4                # RID_ERANK
