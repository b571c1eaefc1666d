// Truncated QR with column pivoting of the sketch Y (Sec. 2, "Y ~= Q R", with
// the column permutation chosen by Businger-Golub pivoting).
//
// One launch per Householder step j.  Every CTA applies H_j^H to a set of
// trailing columns (one warp per column, the column kept in registers between
// the dot product and the update), recomputes the column's remaining norm
// sum_{i>j} |Y_ic|^2 exactly, and posts its best (norm, column) pair.  The
// last CTA to finish (found with a fence + atomic counter; no CTA ever waits
// on another) reduces the pairs, swaps the pivot column into place and forms
// the next reflector in LAPACK zlarfg convention, so the following launch can
// start at once.  Ties go to the lowest column index.
#include <climits>

#include "rid_internal.cuh"

namespace {

constexpr int QR_THREADS = 256;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr int QR_PER_LANE = 16;            // rows per lane kept in registers: l <= 512

struct ArgMax {
  double v;
  int i;
};

__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
  return (b.v > a.v || (b.v == a.v && b.i < a.i)) ? b : a;
}

__device__ __forceinline__ ArgMax warp_argmax(ArgMax a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ArgMax o;
    o.v = __shfl_xor_sync(0xffffffffu, a.v, off);
    o.i = __shfl_xor_sync(0xffffffffu, a.i, off);
    a = better(a, o);
  }
  return a;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// Block-wide argmax; result valid in every thread.
__device__ ArgMax block_argmax(ArgMax a) {
  __shared__ ArgMax red[QR_WARPS];
  __shared__ ArgMax result;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = warp_argmax(a);
  if (lane == 0) red[warp] = a;
  __syncthreads();
  if (warp == 0) {
    ArgMax b = lane < QR_WARPS ? red[lane] : ArgMax{-1.0, INT_MAX};
    b = warp_argmax(b);
    if (lane == 0) result = b;
  }
  __syncthreads();
  return result;
}

// Block-wide sum in a fixed order; result valid in every thread.
__device__ double block_sum(double x) {
  __shared__ double red[QR_WARPS];
  __shared__ double result;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  x = warp_sum(x);
  if (lane == 0) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    double y = lane < QR_WARPS ? red[lane] : 0.0;
    y = warp_sum(y);
    if (lane == 0) result = y;
  }
  __syncthreads();
  return result;
}

struct SelectArgs {
  double2* Y;
  int64_t ldy;
  int l, k;
  int64_t n;
  int32_t* perm;
  double* part_val;
  int* part_idx;
  unsigned* counter;
  double2* tau;
  int* status;
};

// Post this CTA's best pair; returns true in every thread of the CTA that
// finished last (all other CTAs' writes are then visible to it).
__device__ bool post_and_check_last(const SelectArgs& a, ArgMax best) {
  __shared__ bool am_last;
  __threadfence();
  best = block_argmax(best);
  if (threadIdx.x == 0) {
    a.part_val[blockIdx.x] = best.v;
    a.part_idx[blockIdx.x] = best.i;
    __threadfence();
    const unsigned ticket = atomicAdd(a.counter, 1u);
    am_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Run by the last CTA: pick pivot j, swap it into column j, form reflector j.
__device__ void pivot_and_reflect(const SelectArgs& a, int j) {
  __shared__ double2 s_scale;
  ArgMax best{-1.0, INT_MAX};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
    best = better(best, ArgMax{__ldcg(a.part_val + b), __ldcg(a.part_idx + b)});
  best = block_argmax(best);
  if (threadIdx.x == 0) *a.counter = 0u;          // ready for the next launch
  if (!(best.v > 0.0)) {                          // rank(Y) = j < k (Sec. 2)
    if (threadIdx.x == 0) *a.status = RID_ERANK;
    return;
  }
  const int p = best.i;
  double2* colj = a.Y + (int64_t)j * a.ldy;
  if (p != j) {
    double2* colp = a.Y + (int64_t)p * a.ldy;
    for (int i = threadIdx.x; i < a.l; i += blockDim.x) {
      const double2 t = __ldcg(colj + i);
      colj[i] = __ldcg(colp + i);
      colp[i] = t;
    }
    if (threadIdx.x == 0) {
      const int32_t t = a.perm[j];
      a.perm[j] = a.perm[p];
      a.perm[p] = t;
    }
  }
  __syncthreads();
  double part = 0.0;
  for (int i = j + 1 + threadIdx.x; i < a.l; i += blockDim.x) part += cabs2(__ldcg(colj + i));
  const double xnorm2 = block_sum(part);
  if (threadIdx.x == 0) {
    const double2 alpha = __ldcg(colj + j);
    double2 tau = make_double2(0.0, 0.0);
    double2 scale = make_double2(0.0, 0.0);
    if (!(xnorm2 == 0.0 && alpha.y == 0.0)) {
      const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xnorm2);
      const double beta = alpha.x >= 0.0 ? -nrm : nrm;
      tau = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
      scale = cdiv(make_double2(1.0, 0.0), make_double2(alpha.x - beta, alpha.y));
      colj[j] = make_double2(beta, 0.0);
    }
    a.tau[j] = tau;
    s_scale = scale;
  }
  __syncthreads();
  const double2 scale = s_scale;
  if (scale.x != 0.0 || scale.y != 0.0)
    for (int i = j + 1 + threadIdx.x; i < a.l; i += blockDim.x) colj[i] = cmul(__ldcg(colj + i), scale);
}

// Step 0 preparation: perm = identity, full column norms, pivot 0.
__global__ void __launch_bounds__(QR_THREADS) select_init_kernel(SelectArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * QR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * QR_WARPS;
  for (int64_t c = (int64_t)blockIdx.x * QR_THREADS + threadIdx.x; c < a.n;
       c += (int64_t)gridDim.x * QR_THREADS)
    a.perm[c] = (int32_t)c;
  ArgMax best{-1.0, INT_MAX};
  for (int64_t c = gwarp; c < a.n; c += nwarps) {
    const double2* col = a.Y + c * a.ldy;
    double s = 0.0;
    for (int i = lane; i < a.l; i += 32) s += cabs2(col[i]);
    s = warp_sum(s);
    best = better(best, ArgMax{s, (int)c});
  }
  if (post_and_check_last(a, best)) pivot_and_reflect(a, 0);
}

// Step j: apply H_j^H to columns j+1..n-1, new norms, then pivot j+1.
__global__ void __launch_bounds__(QR_THREADS) select_step_kernel(SelectArgs a, int j) {
  __shared__ double2 v[32 * QR_PER_LANE];
  if (*(volatile int*)a.status != RID_OK) return;
  const int lane = threadIdx.x & 31;
  const int rows = a.l - j;                         // rows j..l-1 of the reflector
  for (int i = threadIdx.x; i < rows; i += blockDim.x)
    v[i] = (i == 0) ? make_double2(1.0, 0.0) : a.Y[(int64_t)j * a.ldy + j + i];
  const double2 t = a.tau[j];
  const double2 ctau = make_double2(t.x, -t.y);
  __syncthreads();

  const int64_t gwarp = ((int64_t)blockIdx.x * QR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * QR_WARPS;
  ArgMax best{-1.0, INT_MAX};
  for (int64_t c = j + 1 + gwarp; c < a.n; c += nwarps) {
    double2* col = a.Y + c * a.ldy + j;
    double2 x[QR_PER_LANE];
    double2 w = make_double2(0.0, 0.0);
#pragma unroll
    for (int u = 0; u < QR_PER_LANE; ++u) {
      const int i = lane + 32 * u;
      x[u] = (i < rows) ? col[i] : make_double2(0.0, 0.0);
      if (i < rows) w = cfma_conj(v[i], x[u], w);
    }
    w.x = warp_sum(w.x);
    w.y = warp_sum(w.y);
    const double2 s = cmul(ctau, w);                // conj(tau) (v^H y)
    double nu = 0.0;
#pragma unroll
    for (int u = 0; u < QR_PER_LANE; ++u) {
      const int i = lane + 32 * u;
      if (i < rows) {
        const double2 vs = cmul(v[i], s);
        x[u].x -= vs.x;
        x[u].y -= vs.y;
        col[i] = x[u];
        if (i > 0) nu += cabs2(x[u]);
      }
    }
    nu = warp_sum(nu);
    best = better(best, ArgMax{nu, (int)c});
  }
  if (j + 1 >= a.k) return;                         // last step: no further pivot
  if (post_and_check_last(a, best)) pivot_and_reflect(a, j + 1);
}

}  // namespace

cudaError_t rid_launch_select(const rid_plan_s* p, double2* Y, int64_t ldy, int32_t* perm) {
  if (p->l > 32 * QR_PER_LANE) return cudaErrorInvalidValue;
  SelectArgs a{Y, ldy, p->l, p->k, p->n, perm, p->qr_val, p->qr_idx, p->qr_counter, p->tau,
               p->status};
  cudaError_t e = cudaMemsetAsync(p->status, 0, sizeof(int), p->stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(p->qr_counter, 0, sizeof(unsigned), p->stream);
  if (e != cudaSuccess) return e;
  select_init_kernel<<<p->qr_grid, QR_THREADS, 0, p->stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int j = 0; j < p->k; ++j) {
    select_step_kernel<<<p->qr_grid, QR_THREADS, 0, p->stream>>>(a, j);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Allocation-free pivoted QR.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// allocator's critical section, real-time loops that forbid allocation after
// start-up, or hosts whose device memory is fully owned by a pool they do not
// control.  rid_select_noalloc gives them the select step without a plan:
// its scratch (per-CTA argmax pairs, the last-CTA counter and the reflector
// scalars tau) lives in the fixed-size array below, which every GPU that
// loads this library holds until the process exits.  Every call shares that
// array, so calls whose work overlaps on the GPU (different streams, or
// different host threads on one device) race; calls on one stream are
// ordered and safe.  The array keeps the last call's contents; each call
// clears the counter it relies on before its first launch.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int NOALLOC_MAX_GRID = 1024;                 // CTAs of one select launch
constexpr int NOALLOC_MAX_STEPS = 32 * QR_PER_LANE;    // reflectors: k <= l <= 512
constexpr size_t NOALLOC_OFF_VAL = 0;
constexpr size_t NOALLOC_OFF_IDX = NOALLOC_OFF_VAL + NOALLOC_MAX_GRID * sizeof(double);
constexpr size_t NOALLOC_OFF_TAU = NOALLOC_OFF_IDX + NOALLOC_MAX_GRID * sizeof(int);
constexpr size_t NOALLOC_OFF_CNT = NOALLOC_OFF_TAU + NOALLOC_MAX_STEPS * sizeof(double2);
constexpr size_t NOALLOC_SCRATCH_BYTES = (NOALLOC_OFF_CNT + sizeof(unsigned) + 255) / 256 * 256;
static_assert(NOALLOC_SCRATCH_BYTES == 20736, "scratch layout changed: update include/rid.h");

static __device__ __align__(256) unsigned char g_select_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_scratch_mutex;
unsigned char* g_scratch_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_select_scratch on the current device (looked up once per device).
cudaError_t scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_select_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = (unsigned char*)ptr;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" RID_API rid_status rid_select_noalloc(void* Y, int64_t ldy, int32_t l, int64_t n, int32_t k,
                                                 int32_t* perm, int32_t* status, void* stream) {
  if (!Y || !perm || !status) return RID_EINVAL;
  if (l < 1 || n < 1 || k < 1 || k > l || k > n || ldy < l || n > 0x7fffffffLL) return RID_EINVAL;
  if (l > NOALLOC_MAX_STEPS) return RID_EINVAL;        // beyond the static scratch / register tile
  if (((uintptr_t)Y & 15u) || ((uintptr_t)perm & 3u) || ((uintptr_t)status & 3u)) return RID_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return RID_ECUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RID_ECUDA;
  int64_t grid = (n + 7) / 8;
  if (grid > 4 * (int64_t)sms) grid = 4 * (int64_t)sms;
  if (grid > NOALLOC_MAX_GRID) grid = NOALLOC_MAX_GRID;
  SelectArgs a{(double2*)Y, ldy, l, k, n, perm,
               (double*)(scratch + NOALLOC_OFF_VAL), (int*)(scratch + NOALLOC_OFF_IDX),
               (unsigned*)(scratch + NOALLOC_OFF_CNT), (double2*)(scratch + NOALLOC_OFF_TAU),
               (int*)status};
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return RID_ECUDA;
  select_init_kernel<<<(unsigned)grid, QR_THREADS, 0, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return RID_ECUDA;
  for (int j = 0; j < k; ++j) {
    select_step_kernel<<<(unsigned)grid, QR_THREADS, 0, s>>>(a, j);
    if (cudaGetLastError() != cudaSuccess) return RID_ECUDA;
  }
  return RID_OK;
}
