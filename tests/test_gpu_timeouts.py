"""The bounded waits fail as designed, without a GPU fault: an mbarrier that
nothing completes and a grid barrier that one CTA more than the grid must
reach both give up after their clock budgets and report RID_ETIMEOUT, and the
context keeps working afterwards (a sketch right after matches the oracle)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dot_bound, to_dev_colmajor, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rid():
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    return rid


def test_waits_time_out_and_the_context_survives(rid):
    assert rid.selftest_timeouts() == ("RID_ETIMEOUT", "RID_ETIMEOUT")
    m, n, k, l = 700, 300, 10, 16
    A = synth.lowrank_plus_noise(m, n, k, 1e-10, seed=3)
    with rid.Plan(m, n, k, l, seed=2, mode="fp64_emulated") as plan:
        Om = to_host(plan.omega())
        Y = to_host(plan.sketch(to_dev_colmajor(A)))
        plan.sync_status()
    Yo = oracle.randomize(Om, A)
    emul = 2.0 ** -46 * (2 * m) * np.outer(np.abs(Om).max(axis=1), np.abs(A).max(axis=0))
    assert np.all(np.abs(Y - Yo) <= dot_bound(Om, A) + emul)
