// Error of the ID, ||A - B P||_2 (Sec. 3.3, Table 5), estimated with r
// Gaussian probes in one pass over A.
//
// For a probe w, (A - A_J P) w = A_Jc w_Jc - A_J T w_Jc = A w~, where
// w~(Jc) = w(Jc) and w~(J) = -T w(Jc).  So the probes are first modified with
// one small product T w(Jc) (k x (n-k) times (n-k) x r), then A is streamed
// once: one thread per row of A, 16-byte coalesced loads down each column,
// the r modified probe entries of the column broadcast from shared memory.
// All sums use a fixed order (no floating-point atomics).
#include "rid_internal.cuh"

namespace {

constexpr int EW_THREADS = 256;
constexpr int EW_COLS = 32;          // columns of A staged per shared-memory round
constexpr int RM = RID_MAX_PROBES;

__global__ void probes_kernel(double2* __restrict__ probes, double2* __restrict__ wtilde,
                              int64_t n, int r, uint64_t seed) {
  const int64_t total = n * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / r;
    const int q = (int)(e - c * r);
    const double2 v = philox_complex_normal((uint64_t)c, (uint64_t)q, seed, RID_STREAM_PROBES);
    probes[c * RM + q] = v;
    wtilde[c * RM + q] = v;
  }
}

// Partial sums of T w(Jc) over a chunk of T's columns: part[g][i][q].
__global__ void __launch_bounds__(EW_THREADS)
wj_kernel(const double2* __restrict__ T, int64_t ldt, const int32_t* __restrict__ perm,
          const double2* __restrict__ probes, int k, int64_t ncols, int r, int64_t chunk,
          double2* __restrict__ part) {
  __shared__ double2 s_w[EW_COLS][RM];
  const int64_t t_begin = (int64_t)blockIdx.x * chunk;
  int64_t t_end = t_begin + chunk;
  if (t_end > ncols) t_end = ncols;
  for (int i0 = 0; i0 < k; i0 += EW_THREADS) {
    const int i = i0 + threadIdx.x;
    double2 acc[RM];
#pragma unroll
    for (int q = 0; q < RM; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int64_t t0 = t_begin; t0 < t_end; t0 += EW_COLS) {
      __syncthreads();
      for (int e = threadIdx.x; e < EW_COLS * r; e += EW_THREADS) {
        const int tt = e / r, q = e - tt * r;
        const int64_t t = t0 + tt;
        s_w[tt][q] = (t < t_end) ? probes[(int64_t)perm[k + t] * RM + q] : make_double2(0.0, 0.0);
      }
      __syncthreads();
      if (i < k) {
        const int64_t tn = (t_end - t0) < EW_COLS ? (t_end - t0) : EW_COLS;
        for (int tt = 0; tt < tn; ++tt) {
          const double2 a = T[i + (t0 + tt) * ldt];
#pragma unroll
          for (int q = 0; q < RM; ++q)
            if (q < r) acc[q] = cfma(a, s_w[tt][q], acc[q]);
        }
      }
    }
    if (i < k) {
#pragma unroll
      for (int q = 0; q < RM; ++q)
        if (q < r) part[((int64_t)blockIdx.x * k + i) * RM + q] = acc[q];
    }
  }
}

// w~(perm[i], q) = -sum_g part[g][i][q] for the k skeleton columns.
__global__ void wj_finalize_kernel(const double2* __restrict__ part, int groups,
                                   const int32_t* __restrict__ perm, int k, int r,
                                   double2* __restrict__ wtilde) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * r) return;
  const int i = e / r, q = e - i * r;
  double2 s = make_double2(0.0, 0.0);
  for (int g = 0; g < groups; ++g) {
    const double2 v = part[((int64_t)g * k + i) * RM + q];
    s.x += v.x;
    s.y += v.y;
  }
  wtilde[(int64_t)perm[i] * RM + q] = make_double2(-s.x, -s.y);
}

__device__ __forceinline__ double2 load_a(const double2* p) { return __ldg(p); }
__device__ __forceinline__ double2 load_a(const float2* p) {
  const float2 v = __ldg(p);
  return make_double2((double)v.x, (double)v.y);
}

// E w~ for a block of rows and a range of columns: part[s][q][row].  A is
// complex128 or complex64; the arithmetic is FP64 either way.
template <typename TA>
__global__ void __launch_bounds__(EW_THREADS)
ew_kernel(const TA* __restrict__ A, int64_t lda, int64_t m, int64_t n,
          const double2* __restrict__ wtilde, int r, int64_t chunk, double2* __restrict__ part) {
  __shared__ double2 s_w[EW_COLS][RM];
  const int64_t i = (int64_t)blockIdx.x * EW_THREADS + threadIdx.x;
  const int64_t c_begin = (int64_t)blockIdx.y * chunk;
  int64_t c_end = c_begin + chunk;
  if (c_end > n) c_end = n;
  double2 acc[RM];
#pragma unroll
  for (int q = 0; q < RM; ++q) acc[q] = make_double2(0.0, 0.0);
  for (int64_t c0 = c_begin; c0 < c_end; c0 += EW_COLS) {
    __syncthreads();
    for (int e = threadIdx.x; e < EW_COLS * RM; e += EW_THREADS) {
      const int cc = e / RM, q = e - cc * RM;
      const int64_t c = c0 + cc;
      s_w[cc][q] = (c < c_end && q < r) ? wtilde[c * RM + q] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (i < m) {
      const int cn = (int)((c_end - c0) < EW_COLS ? (c_end - c0) : EW_COLS);
      const TA* a_ptr = A + i + c0 * lda;
      for (int cc = 0; cc < cn; ++cc) {
        const double2 a = load_a(a_ptr + cc * lda);
#pragma unroll
        for (int q = 0; q < RM; ++q)
          if (q < r) acc[q] = cfma(a, s_w[cc][q], acc[q]);
      }
    }
  }
  if (i < m) {
    double2* dst = part + (int64_t)blockIdx.y * RM * m;
#pragma unroll
    for (int q = 0; q < RM; ++q)
      if (q < r) dst[q * m + i] = acc[q];
  }
}

__device__ double block_sum_256(double x, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;   // valid in thread 0
}

// Per row block: sum over column splits, then |E w_q|^2 summed over the rows.
__global__ void __launch_bounds__(EW_THREADS)
ew_norm_kernel(const double2* __restrict__ part, int splits, int64_t m, int r,
               double* __restrict__ norm_part) {
  __shared__ double red[EW_THREADS / 32];
  const int64_t i = (int64_t)blockIdx.x * EW_THREADS + threadIdx.x;
  for (int q = 0; q < r; ++q) {
    double v = 0.0;
    if (i < m) {
      double2 s = make_double2(0.0, 0.0);
      for (int t = 0; t < splits; ++t) {
        const double2 x = part[(int64_t)t * RM * m + (int64_t)q * m + i];
        s.x += x.x;
        s.y += x.y;
      }
      v = cabs2(s);
    }
    const double tot = block_sum_256(v, red);
    if (threadIdx.x == 0) norm_part[(int64_t)blockIdx.x * RM + q] = tot;
  }
}

// One CTA: the estimate and the probabilistic upper bound.
__global__ void __launch_bounds__(EW_THREADS)
error_finalize_kernel(const double* __restrict__ norm_part, int blocks,
                      const double2* __restrict__ probes, int64_t n, int r,
                      double* __restrict__ out) {
  __shared__ double red[EW_THREADS / 32];
  __shared__ double e2[RM], w2[RM];
  for (int q = 0; q < r; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < blocks; b += blockDim.x) s += norm_part[(int64_t)b * RM + q];
    s = block_sum_256(s, red);
    if (threadIdx.x == 0) e2[q] = s;
    double t = 0.0;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) t += cabs2(probes[c * RM + q]);
    t = block_sum_256(t, red);
    if (threadIdx.x == 0) w2[q] = t;
  }
  if (threadIdx.x == 0) {
    double est = 0.0, emax = 0.0;
    for (int q = 0; q < r; ++q) {
      const double en = sqrt(e2[q]);
      const double ratio = en / sqrt(w2[q]);
      if (ratio > est) est = ratio;
      if (en > emax) emax = en;
    }
    out[0] = est;
    out[1] = 10.0 * sqrt(0.63661977236758134308 /* 2 / pi */) * emax;
  }
}

}  // namespace

cudaError_t rid_launch_error(const rid_plan_s* p, const void* A, int64_t lda,
                             const int32_t* perm, const double2* T, int64_t ldt, int nprobe,
                             uint64_t probe_seed) {
  const int r = nprobe;
  const int k = p->k;
  const int64_t n = p->n, m = p->m, ncols = n - k;
  {
    int64_t blocks = (n * r + 255) / 256;
    if (blocks > (int64_t)p->num_sms * 32) blocks = (int64_t)p->num_sms * 32;
    probes_kernel<<<(unsigned)blocks, 256, 0, p->stream>>>(p->probes, p->wtilde, n, r, probe_seed);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ncols > 0) {
    const int groups = p->err_wj_grid;
    const int64_t chunk = (ncols + groups - 1) / groups;
    const int used = (int)((ncols + chunk - 1) / chunk);
    wj_kernel<<<used, EW_THREADS, 0, p->stream>>>(T, ldt, perm, p->probes, k, ncols, r, chunk,
                                                 p->wj_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    wj_finalize_kernel<<<(k * r + 255) / 256, 256, 0, p->stream>>>(p->wj_part, used, perm, k, r,
                                                                   p->wtilde);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    // n == k: A = B P exactly, w~(J) = 0
    wj_finalize_kernel<<<(k * r + 255) / 256, 256, 0, p->stream>>>(p->wj_part, 0, perm, k, r,
                                                                   p->wtilde);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int row_blocks = p->err_row_blocks;
  const int splits = p->err_col_split;
  const int64_t chunk = (n + splits - 1) / splits;
  if (p->dtype == RID_C64)
    ew_kernel<float2><<<dim3(row_blocks, splits), EW_THREADS, 0, p->stream>>>((const float2*)A, lda, m, n,
                                                                             p->wtilde, r, chunk, p->ew_part);
  else
    ew_kernel<double2><<<dim3(row_blocks, splits), EW_THREADS, 0, p->stream>>>((const double2*)A, lda, m, n,
                                                                              p->wtilde, r, chunk, p->ew_part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ew_norm_kernel<<<row_blocks, EW_THREADS, 0, p->stream>>>(p->ew_part, splits, m, r, p->norm_part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  error_finalize_kernel<<<1, EW_THREADS, 0, p->stream>>>(p->norm_part, row_blocks, p->probes, n, r,
                                                         p->err_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row probes fused into the sketch.  G (rows l..ls-1 of Omega) is drawn
// independently of Omega, so Lemma 4.1 of Halko, Martinsson & Tropp (2011)
// holds for E^T and the row probes g_q:  ||E||_2 <= 10 sqrt(2/pi) max ||g_q E||
// with probability >= 1 - 10^-r.  The sketch wrote X = G A next to Y; since
// E(:, J) = 0 and E(:, perm[k+i]) = A(:, perm[k+i]) - A_J T(:, i),
//   (g_q E)(perm[k+i]) = X(q, perm[k+i]) - sum_a X(q, perm[a]) T(a, i),
// which needs k (n-k) products per probe and no access to A.
// ---------------------------------------------------------------------------
namespace {

constexpr int LP_THREADS = 256;
constexpr int LP_WARPS = LP_THREADS / 32;

// ||g_q||^2 over the m entries of row l + q of Omega, one CTA per probe.
__global__ void __launch_bounds__(EW_THREADS)
row_probe_norm_kernel(const double2* __restrict__ G, int64_t ldo, int64_t m, double* __restrict__ out) {
  __shared__ double red[EW_THREADS / 32];
  const double2* g = G + (int64_t)blockIdx.x * ldo;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += EW_THREADS) s += cabs2(g[i]);
  s = block_sum_256(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// One warp per column i of T: lanes split the k-long dot products X_q(J) T(:, i)
// (X_q(J) staged q-major in shared memory), a fixed-order shuffle tree sums
// them, lane 0 forms |Z_q(i)|^2.  part[b][q] = the CTA's sum over its columns.
__global__ void __launch_bounds__(LP_THREADS)
row_probe_resid_kernel(const double2* __restrict__ X, int r, const int32_t* __restrict__ perm,
                       const double2* __restrict__ T, int64_t ldt, int k, int64_t ncols,
                       double* __restrict__ part) {
  extern __shared__ double2 xj[];                 // xj[q * k + a] = X(q, perm[a])
  __shared__ double wsum[LP_WARPS][RM];
  for (int e = threadIdx.x; e < k * r; e += LP_THREADS) {
    const int q = e / k, a = e - q * k;
    xj[e] = X[q + (int64_t)perm[a] * r];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double sq[RM];
#pragma unroll
  for (int q = 0; q < RM; ++q) sq[q] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * LP_WARPS + warp; i < ncols; i += (int64_t)gridDim.x * LP_WARPS) {
    double2 acc[RM];
#pragma unroll
    for (int q = 0; q < RM; ++q) acc[q] = make_double2(0.0, 0.0);
    const double2* Ti = T + i * ldt;
    for (int a = lane; a < k; a += 32) {
      const double2 t = Ti[a];
#pragma unroll
      for (int q = 0; q < RM; ++q)
        if (q < r) acc[q] = cfma(xj[q * k + a], t, acc[q]);
    }
    const int64_t col = perm[k + i];
#pragma unroll
    for (int q = 0; q < RM; ++q) {
      if (q < r) {
        double2 v = acc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          v.x += __shfl_down_sync(0xffffffffu, v.x, off);
          v.y += __shfl_down_sync(0xffffffffu, v.y, off);
        }
        if (lane == 0) {
          const double2 x = X[q + col * r];
          sq[q] += cabs2(make_double2(x.x - v.x, x.y - v.y));
        }
      }
    }
  }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < RM; ++q) wsum[warp][q] = sq[q];
  __syncthreads();
  if (threadIdx.x < r) {
    double s = 0.0;
    for (int w = 0; w < LP_WARPS; ++w) s += wsum[w][threadIdx.x];
    part[(int64_t)blockIdx.x * RM + threadIdx.x] = s;
  }
}

__global__ void row_probe_finalize_kernel(const double* __restrict__ part, int blocks, int r,
                                          const double* __restrict__ g_norm2, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double est = 0.0, zmax = 0.0;
  for (int q = 0; q < r; ++q) {
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += part[(int64_t)b * RM + q];
    const double zn = sqrt(s);
    const double ratio = zn / sqrt(g_norm2[q]);
    if (ratio > est) est = ratio;
    if (zn > zmax) zmax = zn;
  }
  out[0] = est;
  out[1] = 10.0 * sqrt(0.63661977236758134308 /* 2 / pi */) * zmax;
}

}  // namespace

cudaError_t rid_launch_row_probe_norms(const rid_plan_s* p) {
  row_probe_norm_kernel<<<p->nrow, EW_THREADS, 0, p->stream>>>(p->omega + (int64_t)p->l * p->ldo, p->ldo, p->m,
                                                              p->grow_norm2);
  return cudaGetLastError();
}

cudaError_t rid_launch_error_sketched(const rid_plan_s* p, const int32_t* perm, const double2* T, int64_t ldt) {
  const int64_t ncols = p->n - p->k;
  const size_t smem = (size_t)p->k * p->nrow * sizeof(double2);   // <= 512 * 16 * 16 = 128 KiB
  // one fixed limit (k <= 512, r <= 16): the attribute is process-wide and
  // plans on other host threads launch this kernel concurrently
  cudaError_t e = cudaFuncSetAttribute(row_probe_resid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(512 * RID_MAX_PROBES * sizeof(double2)));
  if (e != cudaSuccess) return e;
  row_probe_resid_kernel<<<p->lp_grid, LP_THREADS, smem, p->stream>>>(p->xrow, p->nrow, perm, T, ldt, p->k, ncols,
                                                                      p->lp_part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  row_probe_finalize_kernel<<<1, 32, 0, p->stream>>>(p->lp_part, p->lp_grid, p->nrow, p->grow_norm2, p->err_out);
  return cudaGetLastError();
}
