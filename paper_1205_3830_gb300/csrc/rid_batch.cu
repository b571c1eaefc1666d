// Batched randomized IDs: many independent problems of uneven sizes.
//
// The FP64 persistent batch (rid_batch_prepare / rid_batch_launch) runs all
// problems in one launch.  A CTA takes whole problems from a work queue (one
// atomic counter; problems are queued largest first) and runs every step of
// the ID for its problem with CTA-wide synchronisation only, so no CTA ever
// waits on another:
//   sketch   Y = Omega A        (Sec. 2; Omega drawn once per problem from its
//                                seed, the same Philox counters as a plan with
//                                that seed, into the CTA's workspace slice)
//   select   k Householder steps with column pivoting on Y (Sec. 2)
//   solve    R1 T = R2 by back substitution (Sec. 2)
//   error    probe estimate of ||A - A(:, J) P||_2 (Sec. 3.3)
// The tensor-core batch (rid_batch_tc_*, at the end of this file) sketches
// every problem in one persistent tensor-core launch (rid_batch_tc.cu) and
// finishes every problem (select, solve, row-probe error) in one persistent
// launch of the same per-CTA QR and solve.
//
// All arithmetic is FP64; sums run in a fixed order, so a problem's result
// does not depend on which CTA ran it or what ran beside it.
#include <climits>

#include "rid_internal.cuh"

namespace {

constexpr int BT_THREADS = 256;
constexpr int BT_WARPS = BT_THREADS / 32;
constexpr int BT_KC = 32;                  // rows of A per sketch chunk
constexpr int BT_MAX_L = 128;
constexpr int BT_MAX_K = 64;
constexpr int BT_MAX_N = 4096;
constexpr int BT_NR = 32;                  // right-hand sides per solve block
// Omega drawn once per problem into the CTA's slice of the workspace when
// l m is at most this many entries (2 MiB); larger problems draw each K chunk
// where it is used.  The draw is a Philox block plus an FP64 log and sincospi
// per entry, so drawing it once per column tile multiplied the FP64 work.
constexpr int64_t BT_OMEGA_CAP = 131072;

struct BatchItemDev {
  int64_t m, n;
  int32_t k, l;
  const double2* A;
  int64_t lda;
  double2* Y;
  int64_t ldy;
  int32_t* perm;
  double2* T;
  int64_t ldt;
  uint64_t seed;
};

struct BatchArgs {
  const BatchItemDev* items;
  const int32_t* order;       // queue order (largest first)
  int count;
  unsigned* next;             // work-queue counter
  int nprobe;
  uint64_t probe_seed;
  double* err_out;            // 2 per problem
  int32_t* status_out;        // per problem
  int ct;                     // sketch column tile: 16 or 32 (tuned)
  double2* omega_ws;          // BT_OMEGA_CAP entries per CTA
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// Block sum in a fixed order; valid in all threads.
__device__ double block_sum(double x, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  x = warp_sum(x);
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < BT_WARPS; ++w) s += red[w];
  return s;
}

// ---- step 1: Y = Omega A, column tiles of ct, K chunks of BT_KC rows ------------------
template <int CT>
__device__ void batch_sketch(const BatchItemDev& it, double2* smem, double2* __restrict__ om) {
  const int l = it.l;
  const int64_t m = it.m, n = it.n;
  double2* As = smem;                                  // CT x (BT_KC + 1)
  double2* Os = smem + CT * (BT_KC + 1);               // l x (BT_KC + 1)
  // Omega once, row-major l x m, into this CTA's workspace (when it fits)
  const bool cached = (int64_t)l * m <= BT_OMEGA_CAP;
  if (cached) {
    for (int64_t e = threadIdx.x; e < (int64_t)l * m; e += BT_THREADS) {
      const int64_t i = e / m, r = e - i * m;
      om[e] = philox_complex_normal((uint64_t)i, (uint64_t)r, it.seed, RID_STREAM_OMEGA);
    }
    __syncthreads();
  }
  constexpr int MAXE = (BT_MAX_L * CT + BT_THREADS - 1) / BT_THREADS;
  for (int64_t c0 = 0; c0 < n; c0 += CT) {
    double2 acc[MAXE];
#pragma unroll
    for (int u = 0; u < MAXE; ++u) acc[u] = make_double2(0.0, 0.0);
    for (int64_t r0 = 0; r0 < m; r0 += BT_KC) {
      __syncthreads();
      for (int e = threadIdx.x; e < CT * BT_KC; e += BT_THREADS) {
        const int c = e / BT_KC, rr = e % BT_KC;
        const int64_t gc = c0 + c, gr = r0 + rr;
        As[c * (BT_KC + 1) + rr] = (gc < n && gr < m) ? it.A[gc * it.lda + gr] : make_double2(0.0, 0.0);
      }
      for (int e = threadIdx.x; e < l * BT_KC; e += BT_THREADS) {
        const int i = e / BT_KC, rr = e % BT_KC;
        const int64_t gr = r0 + rr;
        Os[i * (BT_KC + 1) + rr] =
            gr >= m ? make_double2(0.0, 0.0)
                    : (cached ? om[i * m + gr]
                              : philox_complex_normal((uint64_t)i, (uint64_t)gr, it.seed, RID_STREAM_OMEGA));
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < MAXE; ++u) {
        const int e = threadIdx.x + u * BT_THREADS;
        if (e < l * CT) {
          const int i = e / CT, c = e % CT;
          const double2* o = Os + i * (BT_KC + 1);
          const double2* a = As + c * (BT_KC + 1);
          double2 s = acc[u];
#pragma unroll 8
          for (int rr = 0; rr < BT_KC; ++rr) s = cfma(o[rr], a[rr], s);
          acc[u] = s;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < MAXE; ++u) {
      const int e = threadIdx.x + u * BT_THREADS;
      if (e < l * CT) {
        const int i = e / CT, c = e % CT;
        if (c0 + c < n) it.Y[i + (c0 + c) * it.ldy] = acc[u];
      }
    }
  }
  __syncthreads();
}

// ---- step 2: pivoted Householder QR on Y (k steps) ---------------------------------
// Returns RID_OK or RID_ERANK.
__device__ int batch_select(const BatchItemDev& it, double2* tau, double* nu, double* red, double2* v) {
  const int l = it.l, k = it.k;
  const int64_t n = it.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double s_best_v;
  __shared__ int s_best_i;
  __shared__ double2 s_scale;
  for (int64_t c = threadIdx.x; c < n; c += BT_THREADS) it.perm[c] = (int32_t)c;
  // nu_c = |Y(j:, c)|^2 for the current step j, recomputed after every update
  for (int64_t c = warp; c < n; c += BT_WARPS) {
    double s = 0.0;
    for (int i = lane; i < l; i += 32) s += cabs2(it.Y[i + c * it.ldy]);
    s = warp_sum(s);
    if (lane == 0) nu[c] = s;
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    // pivot: first maximum of nu over columns j..n-1
    if (warp == 0) {
      double bv = -1.0;
      int bi = INT_MAX;
      for (int64_t c = j + lane; c < n; c += 32) {
        const double x = nu[c];
        if (x > bv) {
          bv = x;
          bi = (int)c;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_best_v = bv;
        s_best_i = bi;
      }
    }
    __syncthreads();
    if (!(s_best_v > 0.0)) return RID_ERANK;
    const int p = s_best_i;
    double2* colj = it.Y + (int64_t)j * it.ldy;
    if (p != j) {
      double2* colp = it.Y + (int64_t)p * it.ldy;
      for (int i = threadIdx.x; i < l; i += BT_THREADS) {
        const double2 t = colj[i];
        colj[i] = colp[i];
        colp[i] = t;
      }
      if (threadIdx.x == 0) {
        const int32_t t = it.perm[j];
        it.perm[j] = it.perm[p];
        it.perm[p] = t;
        nu[p] = nu[j];
      }
    }
    __syncthreads();
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < l; i += BT_THREADS) part += cabs2(colj[i]);
    const double xnorm2 = block_sum(part, red);
    if (warp == 0) {          // the reflector's divisions spread over the lanes
      double2 t, scale;
      double beta;
      const bool h = zlarfg_scalars_warp(colj[j], xnorm2, lane, t, scale, beta);
      if (lane == 0) {
        if (h) colj[j] = make_double2(beta, 0.0);
        tau[j] = t;
        s_scale = scale;
      }
    }
    __syncthreads();
    const double2 scale = s_scale;
    for (int i = j + 1 + threadIdx.x; i < l; i += BT_THREADS)
      if (scale.x != 0.0 || scale.y != 0.0) colj[i] = cmul(colj[i], scale);
    __syncthreads();
    // v = (1, Y(j+1:, j)); apply H^H to columns j+1..n-1, then their new norms.
    // One thread per column: the columns are short (l <= 128), so warp-wide
    // sums would cost more FP64 additions than the products themselves.
    for (int i = threadIdx.x; i < l - j; i += BT_THREADS) v[i] = i == 0 ? make_double2(1.0, 0.0) : colj[j + i];
    __syncthreads();
    const double2 ctau = make_double2(tau[j].x, -tau[j].y);
    const int rows = l - j;
    for (int64_t c = j + 1 + threadIdx.x; c < n; c += BT_THREADS) {
      double2* col = it.Y + c * it.ldy + j;
      double2 w0 = make_double2(0.0, 0.0), w1 = make_double2(0.0, 0.0);
      int i = 0;
      for (; i + 1 < rows; i += 2) {
        w0 = cfma_conj(v[i], col[i], w0);
        w1 = cfma_conj(v[i + 1], col[i + 1], w1);
      }
      if (i < rows) w0 = cfma_conj(v[i], col[i], w0);
      const double2 s = cmul(ctau, make_double2(w0.x + w1.x, w0.y + w1.y));
      double nr = 0.0, ni = 0.0;
      for (i = 0; i < rows; ++i) {
        const double2 vi = v[i];
        double2 x = col[i];
        x.x = fma(-vi.x, s.x, x.x);
        x.x = fma(vi.y, s.y, x.x);
        x.y = fma(-vi.x, s.y, x.y);
        x.y = fma(-vi.y, s.x, x.y);
        col[i] = x;
        if (i > 0) {
          nr = fma(x.x, x.x, nr);
          ni = fma(x.y, x.y, ni);
        }
      }
      nu[c] = nr + ni;
    }
    __syncthreads();
  }
  return RID_OK;
}

// ---- step 3: T = R1^-1 R2 -------------------------------------------------------------
__device__ void batch_solve(const BatchItemDev& it, double2* rhs, double2* rcol) {
  const int k = it.k;
  const int64_t ncols = it.n - k;
  for (int64_t c0 = 0; c0 < ncols; c0 += BT_NR) {
    const int nvalid = (int)min((int64_t)BT_NR, ncols - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < k * BT_NR; e += BT_THREADS) {
      const int c = e / k, i = e % k;
      rhs[i * BT_NR + c] = c < nvalid ? it.Y[i + (k + c0 + c) * it.ldy] : make_double2(0.0, 0.0);
    }
    for (int j = k - 1; j >= 0; --j) {
      __syncthreads();
      if (threadIdx.x < BT_NR) rhs[j * BT_NR + threadIdx.x] = cdiv(rhs[j * BT_NR + threadIdx.x], it.Y[j + (int64_t)j * it.ldy]);
      for (int i = threadIdx.x; i < j; i += BT_THREADS) rcol[i] = it.Y[i + (int64_t)j * it.ldy];
      __syncthreads();
      for (int e = threadIdx.x; e < j * BT_NR; e += BT_THREADS) {
        const int i = e / BT_NR, c = e % BT_NR;
        const double2 r = rcol[i], t = rhs[j * BT_NR + c];
        double2 x = rhs[e];
        x.x = fma(-r.x, t.x, x.x);
        x.x = fma(r.y, t.y, x.x);
        x.y = fma(-r.x, t.y, x.y);
        x.y = fma(-r.y, t.x, x.y);
        rhs[e] = x;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * BT_NR; e += BT_THREADS) {
      const int c = e / k, i = e % k;
      if (c < nvalid) it.T[i + (c0 + c) * it.ldt] = rhs[i * BT_NR + c];
    }
  }
  __syncthreads();
}

// ---- step 4: error estimate ------------------------------------------------------------
__device__ void batch_error(const BatchItemDev& it, int r, uint64_t probe_seed, double2* wj, int* inv, double2* wc,
                            double* red, double* out) {
  const int k = it.k;
  const int64_t m = it.m, n = it.n, ncols = n - k;
  // inverse permutation: position of each column of A, and w~(J) = -T w(Jc)
  for (int64_t c = threadIdx.x; c < n; c += BT_THREADS) inv[it.perm[c]] = (int)c;
  for (int e = threadIdx.x; e < k * RID_MAX_PROBES; e += BT_THREADS) wj[e] = make_double2(0.0, 0.0);
  __syncthreads();
  {
    // each thread owns up to 4 (i, q) pairs of the k x r product; the probes of
    // 32 columns of Jc at a time are drawn once into shared memory
    constexpr int OWN = (BT_MAX_K * RID_MAX_PROBES + BT_THREADS - 1) / BT_THREADS;
    double2 s[OWN];
#pragma unroll
    for (int u = 0; u < OWN; ++u) s[u] = make_double2(0.0, 0.0);
    for (int64_t t0 = 0; t0 < ncols; t0 += 32) {
      __syncthreads();
      for (int e = threadIdx.x; e < 32 * r; e += BT_THREADS) {
        const int tt = e / r, q = e % r;
        const int64_t t = t0 + tt;
        wc[tt * RID_MAX_PROBES + q] =
            t < ncols ? philox_complex_normal((uint64_t)it.perm[k + t], (uint64_t)q, probe_seed, RID_STREAM_PROBES)
                      : make_double2(0.0, 0.0);
      }
      __syncthreads();
      const int tn = (int)min((int64_t)32, ncols - t0);
#pragma unroll
      for (int u = 0; u < OWN; ++u) {
        const int e = threadIdx.x + u * BT_THREADS;
        if (e < k * r) {
          const int i = e / r, q = e % r;
          for (int tt = 0; tt < tn; ++tt) s[u] = cfma(it.T[i + (t0 + tt) * it.ldt], wc[tt * RID_MAX_PROBES + q], s[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < OWN; ++u) {
      const int e = threadIdx.x + u * BT_THREADS;
      if (e < k * r) wj[(e / r) * RID_MAX_PROBES + (e % r)] = make_double2(-s[u].x, -s[u].y);
    }
  }
  __syncthreads();
  double e2[RID_MAX_PROBES];
#pragma unroll
  for (int q = 0; q < RID_MAX_PROBES; ++q) e2[q] = 0.0;
  for (int64_t r0 = 0; r0 < m; r0 += BT_THREADS) {
    const int64_t row = r0 + threadIdx.x;
    double2 acc[RID_MAX_PROBES];
#pragma unroll
    for (int q = 0; q < RID_MAX_PROBES; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int64_t c0 = 0; c0 < n; c0 += 32) {
      __syncthreads();
      for (int e = threadIdx.x; e < 32 * r; e += BT_THREADS) {
        const int cc = e / r, q = e % r;
        const int64_t c = c0 + cc;
        double2 w = make_double2(0.0, 0.0);
        if (c < n) {
          const int pos = inv[c];
          w = pos < k ? wj[pos * RID_MAX_PROBES + q]
                      : philox_complex_normal((uint64_t)c, (uint64_t)q, probe_seed, RID_STREAM_PROBES);
        }
        wc[cc * RID_MAX_PROBES + q] = w;
      }
      __syncthreads();
      if (row < m) {
        const int cn = (int)min((int64_t)32, n - c0);
        for (int cc = 0; cc < cn; ++cc) {
          const double2 a = it.A[row + (c0 + cc) * it.lda];
#pragma unroll
          for (int q = 0; q < RID_MAX_PROBES; ++q)
            if (q < r) acc[q] = cfma(a, wc[cc * RID_MAX_PROBES + q], acc[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RID_MAX_PROBES; ++q) e2[q] += cabs2(acc[q]);
  }
  double est = 0.0, emax = 0.0;
  for (int q = 0; q < r; ++q) {
    const double en2 = block_sum(e2[q], red);
    double w2 = 0.0;
    for (int64_t c = threadIdx.x; c < n; c += BT_THREADS)
      w2 += cabs2(philox_complex_normal((uint64_t)c, (uint64_t)q, probe_seed, RID_STREAM_PROBES));
    w2 = block_sum(w2, red);
    const double en = sqrt(en2);
    est = fmax(est, en / sqrt(w2));
    emax = fmax(emax, en);
  }
  if (threadIdx.x == 0) {
    out[0] = est;
    out[1] = 10.0 * sqrt(0.63661977236758134308 /* 2 / pi */) * emax;
  }
  __syncthreads();
}

template <int CT>
__global__ void __launch_bounds__(BT_THREADS) batch_kernel(BatchArgs a) {
  extern __shared__ double2 smem[];
  __shared__ double red[BT_WARPS];
  __shared__ int s_task;
  __shared__ double2 tau[BT_MAX_K];
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_task = (int)atomicAdd(a.next, 1u);
    __syncthreads();
    const int t = s_task;
    if (t >= a.count) break;
    const BatchItemDev it = a.items[a.order[t]];
    const int pid = a.order[t];
    batch_sketch<CT>(it, smem, a.omega_ws + (int64_t)blockIdx.x * BT_OMEGA_CAP);
    // scratch of the later steps shares the sketch's shared memory
    double* nu = (double*)smem;                                   // n doubles
    double2* v = (double2*)(nu + BT_MAX_N);                        // l entries
    const int st = batch_select(it, tau, nu, red, v);
    if (st != RID_OK) {
      if (threadIdx.x == 0) {
        a.status_out[pid] = st;
        a.err_out[2 * pid] = -1.0;
        a.err_out[2 * pid + 1] = -1.0;
      }
      continue;
    }
    batch_solve(it, smem, smem + BT_MAX_K * BT_NR);
    double2* wj = smem;                                            // k x 16
    int* inv = (int*)(smem + BT_MAX_K * RID_MAX_PROBES);           // n ints
    double2* wc = (double2*)(inv + BT_MAX_N);                      // 32 x 16
    batch_error(it, a.nprobe, a.probe_seed, wj, inv, wc, red, a.err_out + 2 * pid);
    if (threadIdx.x == 0) a.status_out[pid] = RID_OK;
  }
}

// ---- the tensor-core batch: select, solve and the row-probe error after the sketches ----
// Each problem's Y and X = G A come from the persistent batched sketch
// (rid_batch_tc.cu); this persistent kernel finishes every problem.
struct PostItemDev {
  const double2* X;            // r x n, column-major, ld r: the row probes' products
  const double* g_norm2;       // r: ||g_q||^2
};

struct PostArgs {
  const BatchItemDev* items;
  const PostItemDev* post;
  const int32_t* order;
  int count;
  unsigned* next;
  int r;
  double* err_out;
  int32_t* status_out;
  const int* sketch_err;       // non-zero: a wait of the sketch launch gave up
};

// (g_q E)(perm[k+i]) = X(q, perm[k+i]) - sum_a X(q, perm[a]) T(a, i): one warp
// per column of T, lanes over a, fixed-order sums; est / upper as rid_error_sketched.
__device__ void batch_error_rows(const BatchItemDev& it, const PostItemDev& pi, int r, double2* xj, double* red,
                                 double* out) {
  __shared__ double wsum[BT_WARPS][RID_MAX_PROBES];
  const int k = it.k;
  const int64_t ncols = it.n - k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < k * r; e += BT_THREADS) {
    const int q = e / k, a = e - q * k;
    xj[e] = pi.X[q + (int64_t)it.perm[a] * r];          // xj[q * k + a] = X(q, perm[a])
  }
  __syncthreads();
  // one thread per column of T (k <= 64: the sums stay in the thread), the
  // probes four at a time (few registers, so more CTAs fit on an SM); each
  // probe's sum runs in the same order whatever the grouping
  constexpr int QG = 4;
  for (int q0 = 0; q0 < r; q0 += QG) {
    double sq[QG];
#pragma unroll
    for (int g = 0; g < QG; ++g) sq[g] = 0.0;
    for (int64_t i = threadIdx.x; i < ncols; i += BT_THREADS) {
      double2 acc[QG];
#pragma unroll
      for (int g = 0; g < QG; ++g) acc[g] = make_double2(0.0, 0.0);
      const double2* Ti = it.T + i * it.ldt;
      for (int a = 0; a < k; ++a) {
        const double2 t = Ti[a];
#pragma unroll
        for (int g = 0; g < QG; ++g)
          if (q0 + g < r) acc[g] = cfma(xj[(q0 + g) * k + a], t, acc[g]);
      }
      const int64_t col = it.perm[k + i];
#pragma unroll
      for (int g = 0; g < QG; ++g) {
        if (q0 + g < r) {
          const double2 x = pi.X[q0 + g + col * r];
          sq[g] += cabs2(make_double2(x.x - acc[g].x, x.y - acc[g].y));
        }
      }
    }
    // fixed-order sums: over the warp, then (below) over the warps
#pragma unroll
    for (int g = 0; g < QG; ++g) {
      double v = sq[g];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0 && q0 + g < r) wsum[warp][q0 + g] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double est = 0.0, zmax = 0.0;
    for (int q = 0; q < r; ++q) {
      double s2 = 0.0;
      for (int w = 0; w < BT_WARPS; ++w) s2 += wsum[w][q];
      const double zn = sqrt(s2);
      const double ratio = zn / sqrt(pi.g_norm2[q]);
      if (ratio > est) est = ratio;
      if (zn > zmax) zmax = zn;
    }
    out[0] = est;
    out[1] = 10.0 * sqrt(0.63661977236758134308 /* 2 / pi */) * zmax;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(BT_THREADS, 4) batch_post_kernel(PostArgs a) {
  extern __shared__ double2 smem[];
  __shared__ double red[BT_WARPS];
  __shared__ int s_task;
  __shared__ double2 tau[BT_MAX_K];
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_task = (int)atomicAdd(a.next, 1u);
    __syncthreads();
    const int t = s_task;
    if (t >= a.count) break;
    const int pid = a.order[t];
    const BatchItemDev it = a.items[pid];
    double* nu = (double*)smem;                                   // n doubles
    double2* v = (double2*)(nu + BT_MAX_N);                        // l entries
    const int st = *a.sketch_err ? (int)RID_ETIMEOUT : batch_select(it, tau, nu, red, v);
    if (st != RID_OK) {
      if (threadIdx.x == 0) {
        a.status_out[pid] = st;
        a.err_out[2 * pid] = -1.0;
        a.err_out[2 * pid + 1] = -1.0;
      }
      continue;
    }
    batch_solve(it, smem, smem + BT_MAX_K * BT_NR);
    batch_error_rows(it, a.post[pid], a.r, smem, red, a.err_out + 2 * pid);
    if (threadIdx.x == 0) a.status_out[pid] = RID_OK;
  }
}

size_t batch_post_smem_bytes() {
  const size_t select = BT_MAX_N * sizeof(double) + BT_MAX_L * sizeof(double2);
  const size_t solve = (size_t)(BT_MAX_K * BT_NR + BT_MAX_K) * sizeof(double2);
  const size_t error = (size_t)BT_MAX_K * RID_MAX_PROBES * sizeof(double2);
  size_t s = select;
  if (solve > s) s = solve;
  if (error > s) s = error;
  return s;
}

size_t batch_smem_bytes(int ct) {
  const size_t sketch = (size_t)(ct + BT_MAX_L) * (BT_KC + 1) * sizeof(double2);
  const size_t select = BT_MAX_N * sizeof(double) + BT_MAX_L * sizeof(double2);
  const size_t solve = (size_t)(BT_MAX_K * BT_NR + BT_MAX_K) * sizeof(double2);
  const size_t error = BT_MAX_K * RID_MAX_PROBES * sizeof(double2) + BT_MAX_N * sizeof(int) +
                       32 * RID_MAX_PROBES * sizeof(double2);
  size_t s = sketch;
  if (select > s) s = select;
  if (solve > s) s = solve;
  if (error > s) s = error;
  return s;
}

// Resident CTAs of the persistent kernel for `tile`, at most `count`.  The
// shared-memory attributes are fixed per tile, so setting them here before
// the occupancy query never races and always gives the launch's answer.
int batch_grid(int tile, int32_t count) {
  cudaFuncSetAttribute(batch_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes(16));
  cudaFuncSetAttribute(batch_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes(32));
  int dev_id = 0, sms = 0;
  if (cudaGetDevice(&dev_id) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  const size_t smem = batch_smem_bytes(tile);
  int per_sm = 1;
  if (tile == 16)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<16>, BT_THREADS, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<32>, BT_THREADS, smem);
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm < count ? sms * per_sm : count;
}

int batch_grid_max(int32_t count) {
  if (count == 0) return 0;
  const int a = batch_grid(16, count), b = batch_grid(32, count);
  if (a < 0 || b < 0) return -1;
  return a > b ? a : b;
}

// The per-CTA Omega slices start after the descriptors, the order and the queue counter.
size_t omega_offset(int32_t count) {
  return ((size_t)count * (sizeof(BatchItemDev) + sizeof(int32_t)) + sizeof(unsigned) + 255) / 256 * 256;
}

}  // namespace

extern "C" {

rid_status rid_batch_workspace(int32_t count, size_t* bytes) {
  if (count < 0 || !bytes) return RID_EINVAL;
  const int grid = batch_grid_max(count);
  if (grid < 0) return RID_ECUDA;
  *bytes = omega_offset(count) + (size_t)grid * BT_OMEGA_CAP * sizeof(double2);
  return RID_OK;
}

rid_status rid_batch_prepare(const rid_batch_item* items, int32_t count, int32_t nprobe, void* workspace,
                             size_t ws_bytes, void* stream) {
  if (count < 0 || (count > 0 && (!items || !workspace))) return RID_EINVAL;
  if (nprobe < 1 || nprobe > RID_MAX_PROBES) return RID_EINVAL;
  size_t need = 0;
  rid_batch_workspace(count, &need);
  if (ws_bytes < need) return RID_EINVAL;
  if (count == 0) return RID_OK;
  // host-side checks, the queue order (largest first) and the device descriptors
  BatchItemDev* dev = (BatchItemDev*)malloc(sizeof(BatchItemDev) * (size_t)count);
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)count);
  double* cost = (double*)malloc(sizeof(double) * (size_t)count);
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)count);
  if (!dev || !order || !cost || !tmp) {
    free(dev);
    free(order);
    free(cost);
    free(tmp);
    return RID_ENOMEM;
  }
  rid_status st = RID_OK;
  for (int32_t i = 0; i < count && st == RID_OK; ++i) {
    const rid_batch_item& x = items[i];
    if (x.m < 1 || x.n < 1 || x.k < 1 || x.l < x.k || x.k > x.m || x.k > x.n || x.lda < x.m || x.ldy < x.l ||
        x.ldt < x.k || !x.A || !x.Y || !x.perm || (x.n > x.k && !x.T))
      st = RID_EINVAL;
    else if (x.l > BT_MAX_L || x.k > BT_MAX_K || x.n > BT_MAX_N)
      st = RID_EUNSUPPORTED;
    dev[i] = BatchItemDev{x.m, x.n, x.k, x.l, (const double2*)x.A, x.lda, (double2*)x.Y, x.ldy, x.perm,
                          (double2*)x.T, x.ldt, x.seed};
    order[i] = i;
    cost[i] = 8.0 * x.l * (double)x.m * (double)x.n + 8.0 * nprobe * (double)x.m * (double)x.n;
  }
  if (st == RID_OK) {
    // largest first: bottom-up merge sort of order[] by descending cost (stable)
    for (int32_t w = 1; w < count; w *= 2) {
      for (int32_t lo = 0; lo < count; lo += 2 * w) {
        int32_t mid = lo + w < count ? lo + w : count, hi = lo + 2 * w < count ? lo + 2 * w : count;
        int32_t a = lo, b = mid, o = lo;
        while (a < mid && b < hi) tmp[o++] = cost[order[a]] >= cost[order[b]] ? order[a++] : order[b++];
        while (a < mid) tmp[o++] = order[a++];
        while (b < hi) tmp[o++] = order[b++];
      }
      for (int32_t i = 0; i < count; ++i) order[i] = tmp[i];
    }
  }
  cudaError_t e = cudaSuccess;
  if (st == RID_OK) {
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    e = cudaMemcpyAsync(ws, dev, sizeof(BatchItemDev) * (size_t)count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ws + (size_t)count * sizeof(BatchItemDev), order, sizeof(int32_t) * (size_t)count,
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);      // the host arrays are pageable
    // the per-tile shared memory is fixed, so setting it here never races
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(batch_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes(16));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(batch_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes(32));
  }
  free(dev);
  free(order);
  free(cost);
  free(tmp);
  if (st != RID_OK) return st;
  return e == cudaSuccess ? RID_OK : RID_ECUDA;
}

rid_status rid_batch_launch(int32_t count, int32_t nprobe, uint64_t probe_seed, int32_t tile, double* err_out,
                            int32_t* status_out, void* workspace, void* stream) {
  if (count < 0 || (count > 0 && (!err_out || !status_out || !workspace))) return RID_EINVAL;
  if (nprobe < 1 || nprobe > RID_MAX_PROBES) return RID_EINVAL;
  if (tile != 16 && tile != 32) return RID_EINVAL;
  if (count == 0) return RID_OK;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  BatchItemDev* d_items = (BatchItemDev*)ws;
  int32_t* d_order = (int32_t*)(ws + (size_t)count * sizeof(BatchItemDev));
  unsigned* d_next = (unsigned*)(ws + (size_t)count * (sizeof(BatchItemDev) + sizeof(int32_t)));
  if (cudaMemsetAsync(d_next, 0, sizeof(unsigned), s) != cudaSuccess) return RID_ECUDA;
  const size_t smem = batch_smem_bytes(tile);
  BatchArgs args{d_items, d_order, count, d_next, nprobe, probe_seed, err_out, status_out, tile,
                 (double2*)(ws + omega_offset(count))};
  // persistent grid: as many CTAs as can be resident at once (the workspace
  // holds an Omega slice for each)
  const int grid = batch_grid(tile, count);
  if (grid < 1) return RID_ECUDA;
  if (tile == 16)
    batch_kernel<16><<<grid, BT_THREADS, smem, s>>>(args);
  else
    batch_kernel<32><<<grid, BT_THREADS, smem, s>>>(args);
  return cudaGetLastError() == cudaSuccess ? RID_OK : RID_ECUDA;
}

rid_status rid_batch_run(const rid_batch_item* items, int32_t count, int32_t nprobe, uint64_t probe_seed,
                         int32_t tile, double* err_out, int32_t* status_out, void* workspace, size_t ws_bytes,
                         void* stream) {
  if (count < 0 || (count > 0 && (!items || !err_out || !status_out || !workspace))) return RID_EINVAL;
  if (tile != 16 && tile != 32) return RID_EINVAL;
  const rid_status st = rid_batch_prepare(items, count, nprobe, workspace, ws_bytes, stream);
  if (st != RID_OK) return st;
  return rid_batch_launch(count, nprobe, probe_seed, tile, err_out, status_out, workspace, stream);
}

// ---------------------------------------------------------------------------
// The tensor-core batch: every problem's sketch (Y and the row probes' X) in
// one persistent cooperative launch (rid_batch_tc.cu), then one persistent
// launch of select, solve and the row-probe error for all problems, both
// recorded once in a CUDA graph.
// ---------------------------------------------------------------------------
struct rid_batch_plan_s {
  int device;
  int32_t count;
  int nprobe;
  rid_btc_s* sketch;
  cudaStream_t home;
  cudaEvent_t times[3];      // start, before the finishing launch, end (event-record nodes of the graph)
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  char* dev;                 // items, post items, order, queue counter
  size_t dev_bytes;
};

static void batch_plan_release(rid_batch_plan_s* bp) {
  if (!bp) return;
  if (bp->home) cudaStreamSynchronize(bp->home);
  if (bp->exec) cudaGraphExecDestroy(bp->exec);
  if (bp->graph) cudaGraphDestroy(bp->graph);
  if (bp->sketch) rid_btc_destroy(bp->sketch, bp->home);
  if (bp->dev) rid_dev_free(bp->dev, bp->home);
  if (bp->home) cudaStreamSynchronize(bp->home);
  for (int i = 0; i < 3; ++i)
    if (bp->times[i]) cudaEventDestroy(bp->times[i]);
  free(bp);
}

rid_status rid_batch_tc_create_tuned(rid_batch_plan_t* out, const rid_batch_item* items, int32_t count,
                                     int32_t nprobe, uint64_t probe_seed, double* err_out, int32_t* status_out,
                                     const int32_t* tile_n, const int32_t* ksplit, size_t wave_bytes, void* stream) {
  if (!out) return RID_EINVAL;
  *out = nullptr;
  if (count < 1 || !items || !err_out || !status_out) return RID_EINVAL;
  if (nprobe < 1 || nprobe > RID_MAX_PROBES) return RID_EINVAL;
  for (int32_t i = 0; i < count; ++i) {
    const rid_batch_item& x = items[i];
    if (x.m < 1 || x.n < 1 || x.k < 1 || x.l < x.k || x.k > x.m || x.k > x.n || x.lda < x.m || x.ldy < x.l ||
        x.ldt < x.k || !x.A || !x.Y || !x.perm || (x.n > x.k && !x.T))
      return RID_EINVAL;
    if (x.l > BT_MAX_L || x.k > BT_MAX_K || x.n > BT_MAX_N) return RID_EUNSUPPORTED;
    if (((uintptr_t)x.A & 15u) || ((uintptr_t)x.Y & 15u) || (x.T && ((uintptr_t)x.T & 15u))) return RID_EINVAL;
    if (tile_n && tile_n[i] != 0 && (tile_n[i] < 16 || tile_n[i] > 128 || tile_n[i] % 16)) return RID_EINVAL;
    if (ksplit && ksplit[i] < 0) return RID_EINVAL;
  }
  rid_batch_plan_s* bp = (rid_batch_plan_s*)calloc(1, sizeof(rid_batch_plan_s));
  if (!bp) return RID_ENOMEM;
  bp->count = count;
  bp->nprobe = nprobe;
  bp->home = (cudaStream_t)stream;
  cudaGetDevice(&bp->device);
  rid_status st = RID_OK;
  {
    rid_btc_problem* probs = (rid_btc_problem*)malloc(sizeof(rid_btc_problem) * (size_t)count);
    if (!probs) st = RID_ENOMEM;
    for (int32_t i = 0; st == RID_OK && i < count; ++i) {
      const rid_batch_item& x = items[i];
      probs[i] = rid_btc_problem{(const double2*)x.A, x.lda, x.m, x.n, (double2*)x.Y, x.ldy, x.l, x.seed,
                                 tile_n ? tile_n[i] : 0, ksplit ? ksplit[i] : 0};
    }
    if (st == RID_OK) st = rid_btc_create(&bp->sketch, probs, count, nprobe, probe_seed, wave_bytes, bp->home);
    free(probs);
  }
  // the finishing launch's queue order (largest first) and descriptors
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)count);
  double* cost = (double*)malloc(sizeof(double) * (size_t)count);
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)count);
  BatchItemDev* hitems = (BatchItemDev*)malloc(sizeof(BatchItemDev) * (size_t)count);
  PostItemDev* hpost = (PostItemDev*)malloc(sizeof(PostItemDev) * (size_t)count);
  if (st == RID_OK && (!order || !cost || !tmp || !hitems || !hpost)) st = RID_ENOMEM;
  if (st == RID_OK) {
    for (int32_t i = 0; i < count; ++i) {
      const rid_batch_item& x = items[i];
      hitems[i] = BatchItemDev{x.m, x.n, x.k, x.l, (const double2*)x.A, x.lda, (double2*)x.Y, x.ldy, x.perm,
                               (double2*)x.T, x.ldt, x.seed};
      hpost[i] = PostItemDev{rid_btc_x(bp->sketch, i), rid_btc_gnorm2(bp->sketch, i)};
      order[i] = i;
      cost[i] = 16.0 * (double)x.n * x.l * x.k + 8.0 * (double)x.n * x.k * nprobe;   // QR, solve and error flops
    }
    for (int32_t w = 1; w < count; w *= 2) {
      for (int32_t lo = 0; lo < count; lo += 2 * w) {
        int32_t mid = lo + w < count ? lo + w : count, hi = lo + 2 * w < count ? lo + 2 * w : count;
        int32_t a = lo, b = mid, o = lo;
        while (a < mid && b < hi) tmp[o++] = cost[order[a]] >= cost[order[b]] ? order[a++] : order[b++];
        while (a < mid) tmp[o++] = order[a++];
        while (b < hi) tmp[o++] = order[b++];
      }
      for (int32_t i = 0; i < count; ++i) order[i] = tmp[i];
    }
  }
  const size_t off_post = (size_t)count * sizeof(BatchItemDev);
  const size_t off_order = off_post + (size_t)count * sizeof(PostItemDev);
  const size_t off_next = off_order + (size_t)count * sizeof(int32_t);
  bp->dev_bytes = off_next + 256;
  cudaError_t e = cudaSuccess;
  if (st == RID_OK) {
    if (rid_dev_alloc((void**)&bp->dev, bp->dev_bytes, bp->home, bp->device) != cudaSuccess) st = RID_ENOMEM;
  }
  if (st == RID_OK) {
    e = cudaMemcpyAsync(bp->dev, hitems, off_post, cudaMemcpyHostToDevice, bp->home);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bp->dev + off_post, hpost, off_order - off_post, cudaMemcpyHostToDevice, bp->home);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bp->dev + off_order, order, off_next - off_order, cudaMemcpyHostToDevice, bp->home);
    if (e == cudaSuccess) e = cudaStreamSynchronize(bp->home);     // the host arrays are pageable
    if (e != cudaSuccess) st = RID_ECUDA;
  }
  for (int i = 0; st == RID_OK && i < 3; ++i)
    if (cudaEventCreate(&bp->times[i]) != cudaSuccess) st = RID_ECUDA;
  // the persistent finishing launch
  int per_sm = 1, sms = 0;
  if (st == RID_OK) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, bp->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_post_kernel, BT_THREADS, batch_post_smem_bytes());
    if (per_sm < 1) per_sm = 1;
  }
  // capture: the sketch launch, then the finishing launch
  cudaStream_t cap = nullptr;
  if (st == RID_OK && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) st = RID_ECUDA;
  if (st == RID_OK) {
    bool capturing = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (!capturing) st = RID_ECUDA;
    if (st == RID_OK && cudaEventRecordWithFlags(bp->times[0], cap, cudaEventRecordExternal) != cudaSuccess) st = RID_ECUDA;
    if (st == RID_OK && rid_btc_launch(bp->sketch, cap) != cudaSuccess) st = RID_ECUDA;
    if (st == RID_OK && cudaEventRecordWithFlags(bp->times[1], cap, cudaEventRecordExternal) != cudaSuccess) st = RID_ECUDA;
    if (st == RID_OK && cudaMemsetAsync(bp->dev + off_next, 0, sizeof(unsigned), cap) != cudaSuccess) st = RID_ECUDA;
    if (st == RID_OK) {
      PostArgs args{(const BatchItemDev*)bp->dev, (const PostItemDev*)(bp->dev + off_post),
                    (const int32_t*)(bp->dev + off_order), count, (unsigned*)(bp->dev + off_next), nprobe, err_out,
                    status_out, rid_btc_error_word(bp->sketch)};
      const int grid = sms * per_sm < count ? sms * per_sm : count;
      batch_post_kernel<<<grid, BT_THREADS, batch_post_smem_bytes(), cap>>>(args);
      if (cudaGetLastError() != cudaSuccess) st = RID_ECUDA;
    }
    if (st == RID_OK && cudaEventRecordWithFlags(bp->times[2], cap, cudaEventRecordExternal) != cudaSuccess) st = RID_ECUDA;
    if (capturing) {
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(cap, &g);
      if (st == RID_OK && ce != cudaSuccess) st = RID_ECUDA;
      if (st == RID_OK) {
        bp->graph = g;
        if (cudaGraphInstantiate(&bp->exec, g, 0) != cudaSuccess) st = RID_ECUDA;
      } else if (g) {
        cudaGraphDestroy(g);
      }
      cudaGetLastError();
    }
  }
  if (cap) cudaStreamDestroy(cap);
  free(order);
  free(cost);
  free(tmp);
  free(hitems);
  free(hpost);
  if (st != RID_OK) {
    batch_plan_release(bp);
    return st;
  }
  *out = bp;
  return RID_OK;
}

rid_status rid_batch_tc_create(rid_batch_plan_t* out, const rid_batch_item* items, int32_t count, int32_t nprobe,
                               uint64_t probe_seed, double* err_out, int32_t* status_out, void* stream) {
  return rid_batch_tc_create_tuned(out, items, count, nprobe, probe_seed, err_out, status_out, nullptr, nullptr, 0,
                                   stream);
}

rid_status rid_batch_tc_run(rid_batch_plan_t bp, void* stream) {
  if (!bp || !bp->exec) return RID_EINVAL;
  return cudaGraphLaunch(bp->exec, (cudaStream_t)stream) == cudaSuccess ? RID_OK : RID_ECUDA;
}

rid_status rid_batch_tc_times(rid_batch_plan_t bp, double out[2]) {
  if (!bp || !out || !bp->exec) return RID_EINVAL;
  float a = 0.f, b = 0.f;
  if (cudaEventSynchronize(bp->times[2]) != cudaSuccess ||
      cudaEventElapsedTime(&a, bp->times[0], bp->times[1]) != cudaSuccess ||
      cudaEventElapsedTime(&b, bp->times[1], bp->times[2]) != cudaSuccess)
    return RID_ECUDA;
  out[0] = a;
  out[1] = b;
  return RID_OK;
}

rid_status rid_batch_tc_info(rid_batch_plan_t bp, double out[4]) {
  if (!bp || !out || !bp->sketch) return RID_EINVAL;
  rid_btc_info(bp->sketch, out);
  out[0] += (double)bp->dev_bytes;
  return RID_OK;
}

rid_status rid_batch_tc_destroy(rid_batch_plan_t bp) {
  batch_plan_release(bp);
  return RID_OK;
}

}  // extern "C"
