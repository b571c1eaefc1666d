"""The allocation-free select (rid_select_noalloc) against the plan-based
rid_select, through the C ABI.

rid_select_noalloc serves callers that cannot call cudaMalloc (code under
another allocator's lock, loops that forbid allocation after start-up): it
keeps its scratch in a fixed array inside the library.  This file is named to
be collected last, so that a stop-at-first-failure run has already run every
other test; it builds and loads the library itself, so it also passes alone.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1205_3830_gb300 import _native, build
    build.build()
    return _native.load()


def colmajor(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).cuda().t()


def sketch_of(m, n, k, l, seed):
    A = synth.lowrank_plus_noise(m, n, k, 1e-10, seed=seed)
    return oracle.randomize(oracle.gaussian_test_matrix(l, m, seed), A)


def select_noalloc(lib, Y, l, n, k):
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.rid_select_noalloc(ctypes.c_void_p(Y.data_ptr()), Y.stride(1), l, n, k,
                                ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                                ctypes.c_void_p(stream))
    return st, perm, status


def test_select_noalloc_matches_plan_select_twice(lib):
    import paper_1205_3830_gb300 as rid
    # two calls in a row on different problems: the shared scratch must not leak between them
    for (m, n, k, l, seed) in [(2048, 1024, 32, 40, 1), (1000, 777, 17, 25, 2)]:
        Yo = sketch_of(m, n, k, l, seed)
        with rid.Plan(m, n, k, l, seed=seed) as plan:
            Y_ref = colmajor(Yo)
            perm_ref = plan.select(Y_ref)
            plan.sync_status()
        Y = colmajor(Yo)
        st, perm, status = select_noalloc(lib, Y, l, n, k)
        assert st == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(perm, perm_ref)
        R, R_ref = Y.cpu().numpy(), Y_ref.cpu().numpy()
        assert np.abs(R[:k] - R_ref[:k]).max() <= 1e-12 * np.abs(R_ref[:k]).max()


@pytest.mark.parametrize("shape", [(2048, 8192, 200, 208), (300, 64, 64, 70), (4096, 333, 1, 3),
                                   (700, 2500, 40, 512), (513, 129, 9, 9)], ids=str)
def test_select_noalloc_and_plan_select_agree_bit_for_bit(lib, shape):
    """The plan runs all k steps in one cooperative launch, the allocation-free
    entry one launch per step; both take the same arithmetic in the same order."""
    import paper_1205_3830_gb300 as rid
    m, n, k, l = shape
    Yo = oracle.randomize(oracle.gaussian_test_matrix(l, m, 3), synth.lowrank_plus_noise(m, n, min(k, 60), 1e-10, seed=4))
    with rid.Plan(m, n, k, l, seed=3) as plan:
        Y_ref = colmajor(Yo)
        perm_ref = plan.select(Y_ref)
        plan.sync_status()
    Y = colmajor(Yo)
    st, perm, status = select_noalloc(lib, Y, l, n, k)
    assert st == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(perm, perm_ref)
    assert torch.equal(Y, Y_ref)          # R, the reflectors below it and the trailing rows


def test_select_noalloc_reports_rank_deficiency(lib):
    m, n, k, l = 64, 40, 5, 8
    A = np.zeros((m, n), dtype=np.complex128)
    A[:, 3] = synth.cgauss(np.random.default_rng(1), m)
    A[:, 17] = synth.cgauss(np.random.default_rng(2), m)
    Y = colmajor(oracle.randomize(oracle.gaussian_test_matrix(l, m, 1), A))
    st, perm, status = select_noalloc(lib, Y, l, n, k)
    assert st == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 4          # RID_ERANK


def test_select_noalloc_rejects_sizes_beyond_its_scratch(lib):
    Y = torch.zeros((10, 600), dtype=torch.complex128, device="cuda").t()      # 600 x 10 column-major
    st, _, _ = select_noalloc(lib, Y, 600, 10, 5)
    assert st == 1                          # RID_EINVAL: l > 512, beyond the static scratch
