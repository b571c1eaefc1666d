"""GB300-native randomized interpolative decomposition (ID).

Lucas, Stalzer & Feo, "Parallel implementation of fast randomized algorithms
for the decomposition of low rank matrices", Sec. 2: A (m x n, complex) ~= B P
with B = A(:, J) and P = [I | T] Pi^T, computed in four steps that each run as
hand-written sm_103a CUDA kernels behind the C ABI of include/rid.h:

    plan = Plan(m, n, k, l, seed)          # draws Omega on the device
    Y    = plan.sketch(A)                  # Y = Omega A
    perm = plan.select(Y)                  # pivoted QR, J = perm[:k]
    T    = plan.solve(Y)                   # R1 T = R2
    est, upper = plan.error(A, perm, T)    # ||A - B P||_2 by probes

This module only marshals arguments: torch supplies device memory and streams.
Matrices are column-major torch views (stride(0) == 1), e.g. colmajor_empty().
"""
from __future__ import annotations

import ctypes

import torch

from . import _native
from ._native import RIDError, check

__all__ = ["Plan", "RIDError", "colmajor_empty", "as_colmajor", "decompose", "MODES", "Batch", "batch_decompose"]

MODES = {
    "fp64": _native.RID_FP64_NATIVE,
    "fp64_emulated": _native.RID_FP64_EMULATED,
    "bf16": _native.RID_MIXED_BF16,
    "3xtf32": _native.RID_MIXED_3XTF32,
}
_DTYPES = {torch.complex128: _native.RID_C128, torch.complex64: _native.RID_C64}


def colmajor_empty(rows, cols, dtype=torch.complex128, device="cuda"):
    """Uninitialised rows x cols column-major tensor (a transposed contiguous one)."""
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def as_colmajor(x):
    """x itself if it is column-major with stride(1) >= rows, else a column-major copy."""
    if x.dim() == 2 and x.stride(0) == 1 and x.stride(1) >= max(1, x.shape[0]):
        return x
    return x.t().contiguous().t()


def _need(cond, msg):
    """Argument check that survives python -O: the kernels trust these shapes."""
    if not cond:
        raise ValueError(msg)


def _check_matrix(x, name, rows, cols, dtype, exact=False):
    """x: a column-major CUDA tensor of `dtype` with at least (exactly, if
    `exact`) rows x cols entries; the kernels read and write rows x cols."""
    _need(isinstance(x, torch.Tensor) and x.is_cuda, f"{name} must be a CUDA tensor")
    _check_layout(x, name, rows, cols, dtype, exact)


def _check_layout(x, name, rows, cols, dtype, exact=False):
    """The device-independent part of _check_matrix: dtype, shape and a
    column-major layout whose columns do not overlap."""
    _need(isinstance(x, torch.Tensor), f"{name} must be a tensor")
    _need(x.dtype == dtype, f"{name} must be {dtype}, got {x.dtype}")
    _need(x.dim() == 2, f"{name} must be a matrix")
    if exact:
        _need(tuple(x.shape) == (rows, cols), f"{name} must be {rows} x {cols}, got {tuple(x.shape)}")
    else:
        _need(x.shape[0] >= rows and x.shape[1] >= cols,
              f"{name} must hold at least {rows} x {cols}, got {tuple(x.shape)}")
    # the row stride of a one-row matrix and the column stride of a
    # one-column matrix are never used; every other column must start at
    # least `rows` entries after the previous one (no overlapping views)
    _need(x.numel() == 0 or x.shape[0] <= 1 or x.stride(0) == 1,
          f"{name} must be column-major (use as_colmajor)")
    _need(x.numel() == 0 or x.shape[1] <= 1 or x.stride(1) >= max(1, x.shape[0]),
          f"{name} has overlapping columns (stride(1) = {x.stride(1)} < {x.shape[0]} rows)")


def _check_perm(perm, n):
    _need(isinstance(perm, torch.Tensor) and perm.is_cuda and perm.dtype == torch.int32,
          "perm must be an int32 CUDA tensor")
    _need(perm.numel() >= n and (perm.dim() == 1 and perm.stride(0) == 1),
          f"perm must be a contiguous vector of at least {n} entries")


def _ld(x):
    """Leading dimension of a column-major matrix view: its column stride, at
    least its row count (a one-column view's stride(1) is arbitrary)."""
    if x.dim() < 2:
        return max(int(x.shape[0]) if x.dim() else 1, 1)
    if x.shape[1] <= 1:
        return max(int(x.shape[0]), 1)
    return max(int(x.stride(1)), int(x.shape[0]), 1)


class _CudaView:
    """Minimal __cuda_array_interface__ holder for a device pointer owned elsewhere."""

    def __init__(self, ptr, shape, strides_bytes, typestr):
        self.__cuda_array_interface__ = {
            "data": (int(ptr), False), "shape": tuple(shape), "strides": tuple(strides_bytes),
            "typestr": typestr, "version": 3,
        }


class Plan:
    """One ID shape (m, n, k, l) with its seeded Gaussian test matrix Omega."""

    def __init__(self, m, n, k, l, seed=0, dtype=torch.complex128, mode="fp64", stream=None,
                 device=None, nprobe=0, probe_seed=1):
        """nprobe > 0 builds the plan with row probes from the start (as
        set_probes(nprobe, probe_seed) after it, without its synchronization)."""
        self._lib = _native.load()
        self.m, self.n, self.k, self.l = int(m), int(n), int(k), int(l)
        self.seed = int(seed)
        self.dtype = dtype
        self.mode = mode
        self.nrow = 0
        self.omega_bits = 0
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if nprobe:
                st = self._lib.rid_plan_create_probes(ctypes.byref(handle), self.m, self.n, self.k, self.l,
                                                      _DTYPES[dtype], MODES[mode], self.seed & (2 ** 64 - 1),
                                                      ctypes.c_void_p(stream.cuda_stream), int(nprobe),
                                                      int(probe_seed) & (2 ** 64 - 1))
            else:
                st = self._lib.rid_plan_create(ctypes.byref(handle), self.m, self.n, self.k, self.l,
                                               _DTYPES[dtype], MODES[mode], self.seed & (2 ** 64 - 1),
                                               ctypes.c_void_p(stream.cuda_stream))
        check(st, "rid_plan_create_probes" if nprobe else "rid_plan_create")
        self._h = handle
        self.nrow = int(nprobe)

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.rid_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- Omega -------------------------------------------------------------
    def omega(self):
        """A copy of the plan's Omega as an l x m complex128 tensor."""
        ptr, ldo = ctypes.c_void_p(), ctypes.c_int64()
        check(self._lib.rid_plan_omega(self._h, ctypes.byref(ptr), ctypes.byref(ldo)), "rid_plan_omega")
        view = _CudaView(ptr.value, (self.l, self.m), (16 * ldo.value, 16), "<c16")
        self.stream.synchronize()
        return torch.as_tensor(view, device=self.device).clone()

    def probe_products(self):
        """A copy of the row probes' products X = G A of the last sketch
        (nprobe x n complex128)."""
        ptr, ldx = ctypes.c_void_p(), ctypes.c_int64()
        check(self._lib.rid_plan_probe_products(self._h, ctypes.byref(ptr), ctypes.byref(ldx)),
              "rid_plan_probe_products")
        view = _CudaView(ptr.value, (ldx.value, self.n), (16, 16 * ldx.value), "<c16")
        self.stream.synchronize()
        return torch.as_tensor(view, device=self.device).clone()

    def set_omega(self, omega):
        """Use a caller-supplied l x m complex128 Omega (row-major, on the device)."""
        omega = omega.to(device=self.device, dtype=torch.complex128)
        if omega.stride(1) != 1:
            omega = omega.contiguous()
        _need(tuple(omega.shape) == (self.l, self.m), f"omega must be {self.l} x {self.m}")
        check(self._lib.rid_plan_set_omega(self._h, ctypes.c_void_p(omega.data_ptr()), omega.stride(0)),
              "rid_plan_set_omega")
        self._keep = omega

    def reseed(self, seed, probe_seed=1):
        """Redraw Omega (and the row probes) in place for new seeds: the plan
        then gives the bits of a new plan with these seeds (no allocation)."""
        check(self._lib.rid_plan_reseed(self._h, int(seed) & (2 ** 64 - 1), int(probe_seed) & (2 ** 64 - 1)),
              "rid_plan_reseed")
        self.seed = int(seed)

    def set_stream(self, stream):
        """Run the plan's later work on `stream` (after its queued work)."""
        check(self._lib.rid_plan_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)), "rid_plan_set_stream")
        self.stream = stream

    def use_srft(self, srft_seed):
        """Use the paper's randomization Omega = S F D (subsampled DFT with random phases)."""
        check(self._lib.rid_plan_use_srft(self._h, int(srft_seed) & (2 ** 64 - 1)), "rid_plan_use_srft")

    # -- the four steps --------------------------------------------------------
    def sketch(self, A, Y=None):
        """Y = Omega A (l x n complex128, column-major)."""
        _check_matrix(A, "A", self.m, self.n, self.dtype, exact=True)
        if Y is None:
            Y = colmajor_empty(self.l, self.n, torch.complex128, self.device)
        _check_matrix(Y, "Y", self.l, self.n, torch.complex128)
        check(self._lib.rid_sketch(self._h, ctypes.c_void_p(A.data_ptr()), _ld(A),
                                   ctypes.c_void_p(Y.data_ptr()), _ld(Y)), "rid_sketch")
        return Y

    def sketch_cols(self, A, Y, col0, ncols):
        """Columns col0 .. col0 + ncols - 1 of Y = Omega A (A, Y: the whole
        matrices); panels covering every column give sketch()'s Y bit for bit."""
        _check_matrix(A, "A", self.m, self.n, self.dtype, exact=True)
        _check_matrix(Y, "Y", self.l, self.n, torch.complex128)
        check(self._lib.rid_sketch_cols(self._h, ctypes.c_void_p(A.data_ptr()), _ld(A),
                                        ctypes.c_void_p(Y.data_ptr()), _ld(Y), int(col0), int(ncols)),
              "rid_sketch_cols")
        return Y

    def select(self, Y, perm=None):
        """Pivoted QR of Y in place; returns perm (int32[n], J = perm[:k])."""
        _check_matrix(Y, "Y", self.l, self.n, torch.complex128)
        if perm is None:
            perm = torch.empty(self.n, dtype=torch.int32, device=self.device)
        _check_perm(perm, self.n)
        check(self._lib.rid_select(self._h, ctypes.c_void_p(Y.data_ptr()), _ld(Y),
                                   ctypes.c_void_p(perm.data_ptr())), "rid_select")
        return perm

    def solve(self, Y, T=None):
        """T = R1^-1 R2 (k x (n-k) complex128, column-major)."""
        _check_matrix(Y, "Y", self.k, self.n, torch.complex128)
        if T is None:
            T = colmajor_empty(self.k, self.n - self.k, torch.complex128, self.device)
        _check_matrix(T, "T", self.k, self.n - self.k, torch.complex128)
        ptr = T.data_ptr() if T.numel() else 0
        check(self._lib.rid_solve(self._h, ctypes.c_void_p(Y.data_ptr()), _ld(Y), ctypes.c_void_p(ptr),
                                  max(_ld(T), self.k)), "rid_solve")
        return T

    def error(self, A, perm, T, nprobe=8, probe_seed=1):
        """(est, upper) of ||A - A(:, J) P||_2 by nprobe Gaussian probes (synchronizes)."""
        _check_matrix(A, "A", self.m, self.n, self.dtype, exact=True)
        _check_perm(perm, self.n)
        _check_matrix(T, "T", self.k, self.n - self.k, torch.complex128)
        out = (ctypes.c_double * 2)()
        ptr = T.data_ptr() if T.numel() else 0
        check(self._lib.rid_error(self._h, ctypes.c_void_p(A.data_ptr()), _ld(A),
                                  ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(ptr),
                                  max(_ld(T), self.k), int(nprobe), int(probe_seed) & (2 ** 64 - 1),
                                  out), "rid_error")
        return float(out[0]), float(out[1])

    def round_omega(self, bits=24):
        """Round every row of Omega (and of the row probes) to `bits` bits below
        the row's largest entry; the emulated sketch then multiplies bits / 8
        digits of it (synchronizes)."""
        check(self._lib.rid_plan_round_omega(self._h, int(bits)), "rid_plan_round_omega")
        self.omega_bits = int(bits)

    def set_probes(self, nprobe=8, probe_seed=1):
        """Row probes G (nprobe x m) multiplied by every later sketch in its pass
        over A, for error_sketched(); nprobe = 0 removes them (synchronizes)."""
        check(self._lib.rid_plan_set_probes(self._h, int(nprobe), int(probe_seed) & (2 ** 64 - 1)),
              "rid_plan_set_probes")
        self.nrow = int(nprobe)

    def error_sketched(self, perm, T):
        """(est, upper) of ||A - A(:, J) P||_2 from the row probes of the last
        sketch: no pass over A (synchronizes)."""
        _check_perm(perm, self.n)
        _check_matrix(T, "T", self.k, self.n - self.k, torch.complex128)
        out = (ctypes.c_double * 2)()
        ptr = T.data_ptr() if T.numel() else 0
        check(self._lib.rid_error_sketched(self._h, ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(ptr),
                                           max(_ld(T), self.k), out), "rid_error_sketched")
        return float(out[0]), float(out[1])

    def set_select_grid(self, ctas):
        """Launch shape of select (same results for every shape): ctas > 0
        one cooperative launch of at most that many CTAs, 0 one launch per
        step (no CTA waits on another), < 0 the plan's default."""
        check(self._lib.rid_plan_set_select_grid(self._h, int(ctas)), "rid_plan_set_select_grid")

    def accuracy(self, Y):
        """After select(Y): (rho, floor, accepted) with rho the pivoted QR's
        estimate of sigma_{k+1} / sigma_1 of the sketch and floor the smallest
        rho at which this plan's mode was measured to match the FP64 path
        (0 for FP64 modes); accepted is rho >= floor (synchronizes)."""
        _check_matrix(Y, "Y", self.l, self.n, torch.complex128)
        out = (ctypes.c_double * 3)()
        check(self._lib.rid_plan_accuracy(self._h, ctypes.c_void_p(Y.data_ptr()), _ld(Y), out), "rid_plan_accuracy")
        return float(out[0]), float(out[1]), bool(out[2] != 0.0)

    def stats(self):
        """Launch counts per call, K-splits and device bytes of the plan."""
        out = (ctypes.c_int64 * 8)()
        check(self._lib.rid_plan_stats(self._h, out), "rid_plan_stats")
        keys = ("sketch_launches", "select_launches", "solve_launches", "error_launches", "split_k",
                "device_bytes", "mode", "dtype")
        return dict(zip(keys, [int(x) for x in out]))

    def enable_timing(self):
        """Record CUDA events around the sketch's kernels from now on."""
        check(self._lib.rid_plan_timing(self._h, 1, None), "rid_plan_timing")

    def sketch_times(self):
        """(slicing, product, reduction) ms of the last sketch (waits for it)."""
        out = (ctypes.c_double * 3)()
        check(self._lib.rid_plan_timing(self._h, 0, out), "rid_plan_timing")
        return tuple(float(x) for x in out)

    def sync_status(self):
        """Synchronize the plan's stream and raise RIDError on a device-side error."""
        check(self._lib.rid_sync_status(self._h), "rid_sync_status")


class Batch:
    """Many independent complex128 IDs run together in one persistent launch.

    problems: list of (A, k, l, seed) with A a column-major complex128 device
    tensor.  Outputs (Y holding R, perm, T) are allocated here and the batch is
    prepared once (rid_batch_prepare: checks, cost order, descriptors on the
    device); run() launches it (rid_batch_launch) on the current stream, and
    capture() records that launch in a CUDA graph for replay().
    """

    _tile_cache = {}

    def __init__(self, problems, nprobe=8, probe_seed=1, device=None):
        self._lib = _native.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.nprobe, self.probe_seed = int(nprobe), int(probe_seed)
        self.Y, self.perm, self.T, self.A = [], [], [], []
        items = (_native.BatchItem * len(problems))()
        for i, (A, k, l, seed) in enumerate(problems):
            _check_matrix(A, f"problem {i}: A", 1, 1, torch.complex128)
            m, n = A.shape
            Y = colmajor_empty(l, n, device=self.device)
            perm = torch.empty(n, dtype=torch.int32, device=self.device)
            T = colmajor_empty(k, n - k, device=self.device)
            self.A.append(A), self.Y.append(Y), self.perm.append(perm), self.T.append(T)
            it = items[i]
            it.m, it.n, it.k, it.l = m, n, int(k), int(l)
            it.A, it.lda = A.data_ptr(), _ld(A)
            it.Y, it.ldy = Y.data_ptr(), _ld(Y)
            it.perm = perm.data_ptr()
            it.T, it.ldt = (T.data_ptr() if T.numel() else 0), max(_ld(T), int(k))
            it.seed = int(seed) & (2 ** 64 - 1)
        self.items = items
        self.count = len(problems)
        need = ctypes.c_size_t()
        check(self._lib.rid_batch_workspace(self.count, ctypes.byref(need)), "rid_batch_workspace")
        self.ws = torch.empty(max(1, need.value), dtype=torch.uint8, device=self.device)
        self.err = torch.empty(2 * max(1, self.count), dtype=torch.float64, device=self.device)
        self.status = torch.empty(max(1, self.count), dtype=torch.int32, device=self.device)
        self.signature = (self.count, sum(int(p[0].shape[0]) * int(p[0].shape[1]) for p in problems) // max(1, self.count))
        self.graph = None
        stream = torch.cuda.current_stream(self.device)
        check(self._lib.rid_batch_prepare(ctypes.byref(self.items), self.count, self.nprobe,
                                          ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                          ctypes.c_void_p(stream.cuda_stream)), "rid_batch_prepare")

    def _launch(self, tile, stream):
        check(self._lib.rid_batch_launch(self.count, self.nprobe, self.probe_seed & (2 ** 64 - 1), int(tile),
                                         ctypes.c_void_p(self.err.data_ptr()), ctypes.c_void_p(self.status.data_ptr()),
                                         ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_void_p(stream.cuda_stream)),
              "rid_batch_launch")

    def run(self, tile=None, stream=None):
        """Launch the prepared batch (one memset, one persistent kernel)."""
        tile = tile or self._tile_cache.get(self.signature, 32)
        self._launch(tile, stream or torch.cuda.current_stream(self.device))
        return self

    def capture(self, tile=None):
        """Record the batch's launch in a CUDA graph; replay() then runs it."""
        tile = tile or self._tile_cache.get(self.signature, 32)
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=side):
            self._launch(tile, side)
        torch.cuda.current_stream(self.device).wait_stream(side)
        return self

    def replay(self):
        self.graph.replay()
        return self

    def autotune(self, tiles=(16, 32), reps=2):
        """Time each sketch tile on this batch and remember the fastest for
        batches of the same signature (results do not depend on the tile)."""
        best, best_ms = None, float("inf")
        for t in tiles:
            self.run(tile=t)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                self.run(tile=t)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            if ms < best_ms:
                best, best_ms = t, ms
        self._tile_cache[self.signature] = best
        return best, best_ms

    def results(self):
        """List of dicts (J, perm, T, est, upper, status) after run()."""
        torch.cuda.synchronize()
        err = self.err.cpu().numpy()
        status = self.status.cpu().numpy()
        out = []
        for i in range(self.count):
            k = int(self.items[i].k)
            out.append({"perm": self.perm[i], "J": self.perm[i][:k], "T": self.T[i], "Y": self.Y[i],
                        "est": float(err[2 * i]), "upper": float(err[2 * i + 1]), "status": int(status[i])})
        return out


class BatchTC:
    """Many complex128 IDs on the tensor cores (rid_batch_tc_*): every
    problem's sketch Y = Omega A and row-probe products X = G A in one
    persistent tensor-core launch, then one persistent launch of select, solve
    and the row-probe error for all problems, replayed as one CUDA graph.

    problems: list of (A, k, l, seed) as for Batch.  tile_n / ksplit: per
    problem (lists, or one value for all) the widest N-tile in rows of the real
    test matrix and the K-splits; tuning: a TcTuning whose per-size-class
    choice fills in what tile_n / ksplit leave open.  wave_bytes: the size of
    each of the two digit buffers (0: 2 GiB).  run() replays the graph on the
    current stream; results() as for Batch; info() the device bytes, waves,
    work items and CTAs of the sketch launch.
    """

    def __init__(self, problems, nprobe=8, probe_seed=1, device=None, tile_n=None, ksplit=None, wave_bytes=0,
                 tuning=None):
        self._lib = _native.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.nprobe, self.probe_seed = int(nprobe), int(probe_seed)
        self.Y, self.perm, self.T, self.A = [], [], [], []
        count = len(problems)
        items = (_native.BatchItem * count)()
        tn = (ctypes.c_int32 * max(1, count))()
        ksp = (ctypes.c_int32 * max(1, count))()
        for i, (A, k, l, seed) in enumerate(problems):
            _check_matrix(A, f"problem {i}: A", 1, 1, torch.complex128)
            m, n = A.shape
            Y = colmajor_empty(l, n, device=self.device)
            perm = torch.empty(n, dtype=torch.int32, device=self.device)
            T = colmajor_empty(k, n - k, device=self.device)
            self.A.append(A), self.Y.append(Y), self.perm.append(perm), self.T.append(T)
            it = items[i]
            it.m, it.n, it.k, it.l = m, n, int(k), int(l)
            it.A, it.lda = A.data_ptr(), _ld(A)
            it.Y, it.ldy = Y.data_ptr(), _ld(Y)
            it.perm = perm.data_ptr()
            it.T, it.ldt = (T.data_ptr() if T.numel() else 0), max(_ld(T), int(k))
            it.seed = int(seed) & (2 ** 64 - 1)
            choice = tuning.choice(m, n, int(l) + self.nprobe) if tuning is not None else (0, 0)
            tn[i] = int(_per_problem(tile_n, i, choice[0]))
            ksp[i] = int(_per_problem(ksplit, i, choice[1]))
        self.items = items
        self.count = count
        self.tile_n, self.ksplit = list(tn)[:count], list(ksp)[:count]
        self.err = torch.empty(2 * max(1, self.count), dtype=torch.float64, device=self.device)
        self.status = torch.empty(max(1, self.count), dtype=torch.int32, device=self.device)
        self._h = ctypes.c_void_p()
        stream = torch.cuda.current_stream(self.device)
        check(self._lib.rid_batch_tc_create_tuned(ctypes.byref(self._h), ctypes.byref(self.items), self.count,
                                                  self.nprobe, self.probe_seed & (2 ** 64 - 1),
                                                  ctypes.c_void_p(self.err.data_ptr()),
                                                  ctypes.c_void_p(self.status.data_ptr()),
                                                  ctypes.cast(tn, ctypes.c_void_p), ctypes.cast(ksp, ctypes.c_void_p),
                                                  int(wave_bytes), ctypes.c_void_p(stream.cuda_stream)),
              "rid_batch_tc_create_tuned")

    def info(self):
        """dict: device bytes the handle holds, waves, work items and CTAs of the sketch launch."""
        out = (ctypes.c_double * 4)()
        check(self._lib.rid_batch_tc_info(self._h, out), "rid_batch_tc_info")
        return {"bytes": int(out[0]), "waves": int(out[1]), "items": int(out[2]), "ctas": int(out[3])}

    def run(self, stream=None):
        stream = stream or torch.cuda.current_stream(self.device)
        check(self._lib.rid_batch_tc_run(self._h, ctypes.c_void_p(stream.cuda_stream)), "rid_batch_tc_run")
        return self

    results = Batch.results

    def times(self):
        """(sketch ms, finishing ms) of the last run (waits for it)."""
        out = (ctypes.c_double * 2)()
        check(self._lib.rid_batch_tc_times(self._h, out), "rid_batch_tc_times")
        return float(out[0]), float(out[1])

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rid_batch_tc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _per_problem(v, i, default):
    if v is None:
        return default
    if isinstance(v, (list, tuple)):
        return v[i] if v[i] is not None else default
    return v


class TcTuning:
    """Tile shapes of the tensor-core batch per size class, chosen by timing.

    A size class is (m class, n class, rows class): the power of two at or
    above m (at least 256), the column-block count class of n (1, 2, 4 or 8+
    blocks of 128) and the N-tile count the default 128-row tiles give for
    2 (l + nprobe) rows.  For each class the candidates are the widest N-tile
    (128, 96 or 64 rows) and the K-splits (1, 2, 4; only where the problem has
    at least twice as many 256-real chunks), timed on the sketch launch of a
    batch of that class's problems; the fastest is kept.  Choices are cached
    per device name in a JSON file when `path` is given (read at creation,
    written after tuning).  Results do not depend on the N-tile; a K-split
    changes a problem's Y in the last bits only (partial sums in split order).
    """

    TILES = (128, 96, 64)
    SPLITS = (1, 2, 4)

    def __init__(self, path=None):
        import json
        import os
        self.path = path
        self.device = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
        self.table = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = {tuple(json.loads(k)): tuple(v) for k, v in json.load(f).get(self.device, {}).items()}

    @staticmethod
    def size_class(m, n, rows):
        mc = 256
        while mc < m:
            mc *= 2
        blocks = (n + 127) // 128
        nc = 1 if blocks <= 1 else 2 if blocks <= 2 else 4 if blocks <= 4 else 8
        return (mc, nc, (2 * rows + 127) // 128)

    def choice(self, m, n, rows):
        """(tile_n, ksplit) for a problem; (0, 0), the defaults, for an untuned class."""
        return self.table.get(self.size_class(m, n, rows), (0, 0))

    @classmethod
    def candidates(cls, cls_key):
        mc, _, _ = cls_key
        chunks = (2 * mc + 255) // 256
        return [(t, s) for t in cls.TILES for s in cls.SPLITS if s == 1 or chunks >= 2 * s]

    def tune(self, problems, nprobe=8, probe_seed=1, per_class=256, reps=3, force=True):
        """Time every candidate on up to per_class problems of each class present
        in `problems` ((A, k, l, seed) tuples) and keep the fastest; returns
        {class: (tile_n, ksplit, ms)} for the classes timed.  force=False skips
        the classes the table (or its cache file) already holds."""
        groups = {}
        for p in problems:
            A, k, l, seed = p
            key = self.size_class(int(A.shape[0]), int(A.shape[1]), int(l) + int(nprobe))
            groups.setdefault(key, []).append(p)
        report = {}
        for key, probs in sorted(groups.items()):
            if not force and key in self.table:
                continue
            sample = probs[:per_class]
            best = None
            for t, s in self.candidates(key):
                b = BatchTC(sample, nprobe, probe_seed, tile_n=t, ksplit=s)
                b.run()
                ms = []
                for _ in range(reps):
                    b.run()
                    ms.append(b.times()[0])
                b.close()
                cand = (t, s, min(ms))
                if best is None or cand[2] < best[2]:
                    best = cand
            self.table[key] = (best[0], best[1])
            report[key] = best
        self.save()
        return report

    def save(self):
        import json
        import os
        if not self.path:
            return
        data = {}
        if os.path.exists(self.path):
            with open(self.path) as f:
                data = json.load(f)
        data[self.device] = {json.dumps(list(k)): list(v) for k, v in sorted(self.table.items())}
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        with open(self.path, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


def selftest_timeouts(stream=None):
    """Run the bounded-wait self-test (rid_selftest_timeouts); returns the two
    status names, ("RID_ETIMEOUT", "RID_ETIMEOUT") when both waits give up as
    designed."""
    lib = _native.load()
    out = (ctypes.c_int32 * 2)()
    s = stream if stream is not None else torch.cuda.current_stream()
    check(lib.rid_selftest_timeouts(ctypes.c_void_p(s.cuda_stream), out), "rid_selftest_timeouts")
    return tuple(lib.rid_status_string(int(x)).decode().split(":")[0] for x in out)


def batch_decompose(problems, nprobe=8, probe_seed=1, tile=None):
    """Run a list of (A, k, l, seed) problems as one batch; returns Batch.results()."""
    return Batch(problems, nprobe, probe_seed).run(tile).results()


def decompose(A, k, l, seed=0, mode="fp64", nprobe=8, probe_seed=1, plan=None):
    """The whole ID of a column-major device matrix A; returns a dict with
    J, perm, T, Y (holding R) and the error estimate (est, upper)."""
    m, n = A.shape
    own = plan is None
    if own:
        plan = Plan(m, n, k, l, seed=seed, dtype=A.dtype, mode=mode)
    try:
        Y = plan.sketch(A)
        perm = plan.select(Y)
        T = plan.solve(Y)
        est, upper = plan.error(A, perm, T, nprobe, probe_seed)
        plan.sync_status()
        return {"J": perm[:k], "perm": perm, "T": T, "Y": Y, "est": est, "upper": upper}
    finally:
        if own:
            plan.close()
