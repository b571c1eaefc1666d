// Internal declarations of the GB300 randomized-ID library (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rid.h"

// ---------------------------------------------------------------------------
// Plan: sizes, the test matrix Omega and all device workspace of one ID shape.
// ---------------------------------------------------------------------------
// Column panels of the emulated sketch a plan times at most (rid_plan_timing).
#define RID_MAX_PANELS 8
#define RID_TIMING_EVENTS (2 + 2 * RID_MAX_PANELS)

struct rid_plan_s {
  int64_t m, n;
  int32_t k, l;
  rid_dtype dtype;
  rid_mode mode;
  uint64_t seed;
  cudaStream_t stream;
  int device;
  int num_sms;

  double2* omega;          // ls x m complex128, row-major, row stride ldo: the l rows of
                           // the test matrix, then the row probes G (rows l..ls-1)
  int64_t ldo;
  int32_t ls;              // rows the sketch computes: l + nrow
  int32_t omega_bits;      // 0, or the bits every row of Omega is rounded to (rid_plan_round_omega)
  int32_t omega_kind;      // 0: the Gaussian of seed; 1: a caller's (rid_plan_set_omega); 2: the SRFT
  int* status;             // device status word (RID_OK / RID_ERANK)

  // sketch (native FP64): split-K partial sums, split_k x ls x n (ld = ls)
  int split_k;
  int64_t k_per_split;
  double2* sk_partial;

  // select: per-CTA argmax partials, last-CTA counter, reflector scalars
  int qr_grid;
  double* qr_val;
  int* qr_idx;
  unsigned* qr_counter;
  double2* tau;            // k
  // select in one cooperative launch (sel_grid CTAs; 0: one launch per step)
  int sel_grid;
  int sel_grid_max;        // the default sel_grid; the posted buffers are sized for it
  double2* sel_cand;       // 2 x sel_grid_max x l posted columns
  double* sel_val;         // 2 x sel_grid_max
  int* sel_idx;            // 2 x sel_grid_max
  unsigned* sel_bar;       // grid barrier: arrivals, generation
  // select with Y resident in shared memory (res_grid CTAs of res_cpc columns; 0: not possible)
  int res_grid;
  int res_cpc;
  size_t res_smem;         // dynamic shared memory of one CTA
  double2* res_cand;       // 2 x res_grid x l posted columns
  double* res_val;         // 2 x res_grid
  int* res_pos;            // 2 x res_grid
  int* res_col;            // 2 x res_grid
  unsigned* res_flag;      // res_grid

  // error: probes, modified probes, partial sums, result
  int err_wj_grid;         // CTAs over the columns of T
  int err_row_blocks;      // CTAs over the rows of A
  int err_col_split;       // CTAs over the columns of A
  double2* probes;         // n x RID_MAX_PROBES (row c holds the probes of column c)
  double2* wtilde;         // n x RID_MAX_PROBES
  double2* wj_part;        // err_wj_grid x k x RID_MAX_PROBES
  double2* ew_part;        // err_col_split x RID_MAX_PROBES x m
  double* norm_part;       // err_row_blocks x RID_MAX_PROBES
  double* err_out;         // 2 doubles (device)

  size_t ws_bytes;         // bytes of the plan's workspace allocation
  void* ws_base;           // that allocation (Omega starts it until row probes are set)

  // row probes fused into the sketch (rid_plan_set_probes)
  int32_t nrow;            // row probes (0: none)
  int x_valid;             // a rid_sketch has written X since the probes were set
  double2* xrow;           // X = G A: nrow x n, column-major, ld nrow
  double* grow_norm2;      // ||g_q||^2, nrow
  double* lp_part;         // lp_grid x RID_MAX_PROBES partial sums of |g_q E|^2
  int lp_grid;
  void* probe_base;        // allocation of Omega + G, X, norms, partials (null: none)
  size_t probe_bytes;

  // optional per-kernel timing of rid_sketch (CUDA events on the plan's stream):
  // ev[0] before the sketch; per panel i (ev_panels of them) ev[1 + 2i] after
  // its first pass (slicing) and ev[2 + 2i] after its product; ev[1 + 2 ev_panels]
  // after the reduction
  int timing;
  cudaEvent_t ev[RID_TIMING_EVENTS];
  mutable int ev_panels;

  // emulated / mixed sketch state (owned by the tensor-core path)
  void* tc_state;
  size_t tc_bytes;
  // mixed-precision plans with row probes: the FP64-emulated state of the probe rows
  void* tc_probe_state;
  size_t tc_probe_bytes;
  int tc_sketch_launches;
};

#define RID_MAX_PROBES 16
#define RID_STREAM_OMEGA 3u
#define RID_STREAM_PROBES 4u
#define RID_STREAM_SRFT 5u
#define RID_STREAM_LPROBES 6u

// ---------------------------------------------------------------------------
// Device memory of plans: a library-private stream-ordered pool per device
// (allocation and release are ordered on the plan's stream; nothing
// synchronizes the device, and freed memory stays in the pool for the next
// plan).
// ---------------------------------------------------------------------------
cudaError_t rid_dev_alloc(void** ptr, size_t bytes, cudaStream_t stream, int device);
void rid_dev_free(void* ptr, cudaStream_t stream);

// ---------------------------------------------------------------------------
// Launchers (each returns cudaGetLastError() of its launches).
// ---------------------------------------------------------------------------
// Gaussian matrix: entry (i, j) at out[i * row_stride + j * col_stride].
cudaError_t rid_launch_gaussian(double2* out, int64_t rows, int64_t cols, int64_t row_stride,
                                int64_t col_stride, uint64_t seed, uint32_t stream_id,
                                cudaStream_t stream);

// Rows of Omega rounded to `bits` bits below each row's largest entry (ties to even).
cudaError_t rid_launch_round_rows(double2* om, int64_t rows, int64_t m, int64_t ldo, int bits, cudaStream_t stream);

// Omega = rows s_1..s_l of F D (the paper's subsampled randomized Fourier transform).
cudaError_t rid_launch_srft(double2* out, int64_t l, int64_t m, int64_t ldo, uint64_t seed, cudaStream_t stream);

cudaError_t rid_launch_sketch_fp64(const rid_plan_s* p, const double2* A, int64_t lda, double2* Y,
                                   int64_t ldy, int64_t col0, int64_t ncols);

cudaError_t rid_launch_select(const rid_plan_s* p, double2* Y, int64_t ldy, int32_t* perm);
// CTAs of the cooperative select for n columns on this device (0: not available).
int rid_select_coop_grid(int device, int num_sms, int64_t n, int l);
// Shape of the select with Y resident in shared memory: CTAs (0 when the
// columns do not fit, l > 256 or no cooperative launch), columns per CTA and
// the dynamic shared memory of a CTA.
int rid_select_resident_grid(int device, int num_sms, int64_t n, int l, int* cpc, size_t* smem);

cudaError_t rid_launch_solve(const rid_plan_s* p, const double2* Y, int64_t ldy, double2* T,
                             int64_t ldt);
size_t rid_solve_smem_bytes(int k, int* nr_out);

cudaError_t rid_launch_error(const rid_plan_s* p, const void* A, int64_t lda,
                             const int32_t* perm, const double2* T, int64_t ldt, int nprobe,
                             uint64_t probe_seed);

// ||g_q||^2 of the row probes (rows l..ls-1 of Omega), once per rid_plan_set_probes.
cudaError_t rid_launch_row_probe_norms(const rid_plan_s* p);

// Re-cut the FP64-emulated state's digit tiles of Omega after Omega's values
// changed in place (same shape and row count).
cudaError_t rid_tc_refresh_omega_fp64(const rid_plan_s* p);

// Digit tiles of nrows rows of Omega' (rows 2i, 2i + 1 of each complex row),
// as the exact-slice products read them: [N-tile][K stage][digit] tiles of
// tile_w rows x 32 bf16 in the 64-byte swizzle (pairs: [half] before
// [digit]), and the row exponents om_exp[2 nrows].  Rows past 2 nrows are
// left as the caller set them.
cudaError_t rid_tc_cut_omega(const double2* om, int64_t ldo, int64_t m, int nrows, int64_t KP, int tile_w, bool pair,
                             int* om_exp, uint16_t* tiles, int num_sms, cudaStream_t stream);
// The chunk exponents of a mixed plan's row-probe state, [*nc][n] (set by
// the BF16x3 slicer, read by the probe product); null without row probes.
int* rid_tc_probe_chunk_exp(const rid_plan_s* p, int* nc);
// K-splits of NC chunks so that `units` CTAs (or clusters) per split fill whole
// waves of `slots` resident ones.
int rid_tc_choose_ksplit(int units, int NC, int slots);

// out[0] = |R(0,0)|, out[1] = max_{c >= k} ||Y(k:l-1, c)|| of a selected Y (device doubles).
cudaError_t rid_launch_tail_ratio(const rid_plan_s* p, const double2* Y, int64_t ldy, double* out);
// est / upper from X of the last sketch, perm and T, into p->err_out.
cudaError_t rid_launch_error_sketched(const rid_plan_s* p, const int32_t* perm, const double2* T, int64_t ldt);

// The batched tensor-core sketch (rid_batch_tc.cu): Y = Omega A and the row
// probes' X = G A of every problem in one persistent cooperative launch.
struct rid_btc_problem {
  const double2* A;
  int64_t lda, m, n;
  double2* Y;
  int64_t ldy;
  int32_t l;
  uint64_t seed;
  int32_t tile_n;          // widest N-tile (rows of Omega', 16 .. 128); 0: 128
  int32_t ksplit;          // K-splits; 0: 1
};
struct rid_btc_s;
// Draws every problem's Omega' (seed; the probe rows from probe_seed) and
// lays out the waves and work lists; synchronizes `stream`.
rid_status rid_btc_create(rid_btc_s** out, const rid_btc_problem* probs, int32_t count, int32_t nprobe,
                          uint64_t probe_seed, size_t wave_bytes, cudaStream_t stream);
// Clears the work counters and launches the persistent kernel (capturable).
cudaError_t rid_btc_launch(const rid_btc_s* h, cudaStream_t stream);
const double2* rid_btc_x(const rid_btc_s* h, int32_t i);       // r x n, ld r, of problem i (input order)
const double* rid_btc_gnorm2(const rid_btc_s* h, int32_t i);   // ||g_q||^2 of problem i
const int* rid_btc_error_word(const rid_btc_s* h);             // non-zero after a wait gave up
// out: device bytes, waves, work items, CTAs
void rid_btc_info(const rid_btc_s* h, double out[4]);
void rid_btc_destroy(rid_btc_s* h, cudaStream_t stream);

// ---------------------------------------------------------------------------
// Device helpers shared by the kernels.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc += a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc += conj(a) * b
__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }

// Complex division a / d by Smith's algorithm (R. L. Smith, "Algorithm 116:
// Complex division", CACM 5(8), 1962): scale by the larger component of d.
__device__ __forceinline__ double2 cdiv(double2 a, double2 d) {
  if (fabs(d.x) >= fabs(d.y)) {
    double r = d.y / d.x;
    double den = fma(d.y, r, d.x);
    return make_double2(fma(a.y, r, a.x) / den, fma(-a.x, r, a.y) / den);
  } else {
    double r = d.x / d.y;
    double den = fma(d.x, r, d.y);
    return make_double2(fma(a.x, r, a.y) / den, fma(a.y, r, -a.x) / den);
  }
}

// Reflector scalars in LAPACK zlarfg convention from alpha = Y(j, j) and
// xnorm2 = sum_{i>j} |Y(i, j)|^2: beta = -sign(Re alpha) ||(alpha, x)||,
// tau = (beta - alpha) / beta, scale = 1 / (alpha - beta) for v = x * scale.
// The norm is formed with explicit fma so that every kernel rounds it alike.
// Returns false when H = I (x = 0 and alpha real): tau = 0, nothing scaled.
__device__ __forceinline__ bool zlarfg_scalars(double2 alpha, double xnorm2, double2& tau, double2& scale,
                                               double& beta) {
  tau = make_double2(0.0, 0.0);
  scale = make_double2(0.0, 0.0);
  beta = alpha.x;
  if (xnorm2 == 0.0 && alpha.y == 0.0) return false;
  const double nrm = sqrt(fma(alpha.x, alpha.x, fma(alpha.y, alpha.y, xnorm2)));
  beta = alpha.x >= 0.0 ? -nrm : nrm;
  tau = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
  scale = cdiv(make_double2(1.0, 0.0), make_double2(alpha.x - beta, alpha.y));
  return true;
}

// zlarfg_scalars by a whole warp, bit for bit the same: the divisions that do
// not depend on one another run in different lanes (one SIMT division per
// pass), so the chain is sqrt, division, division instead of sqrt and five
// divisions in a row.  Every lane returns the results.
__device__ __forceinline__ bool zlarfg_scalars_warp(double2 alpha, double xnorm2, int lane, double2& tau,
                                                    double2& scale, double& beta) {
  tau = make_double2(0.0, 0.0);
  scale = make_double2(0.0, 0.0);
  beta = alpha.x;
  if (xnorm2 == 0.0 && alpha.y == 0.0) return false;
  const double nrm = sqrt(fma(alpha.x, alpha.x, fma(alpha.y, alpha.y, xnorm2)));
  beta = alpha.x >= 0.0 ? -nrm : nrm;
  // scale = cdiv((1, 0), d) with d = alpha - beta, the same steps as cdiv
  const double2 d = make_double2(alpha.x - beta, alpha.y);
  const bool xbig = fabs(d.x) >= fabs(d.y);
  // first division: lane 0 tau.x, lane 1 tau.y, lane 2 the ratio r of cdiv
  const double num1 = lane == 0 ? beta - alpha.x : lane == 1 ? -alpha.y : (xbig ? d.y : d.x);
  const double den1 = lane <= 1 ? beta : (xbig ? d.x : d.y);
  const double q1 = num1 / den1;
  tau.x = __shfl_sync(0xffffffffu, q1, 0);
  tau.y = __shfl_sync(0xffffffffu, q1, 1);
  const double r = __shfl_sync(0xffffffffu, q1, 2);
  // second division: lane 0 and lane 1 the two components of cdiv
  const double den = xbig ? fma(d.y, r, d.x) : fma(d.x, r, d.y);
  const double num2 = xbig ? (lane == 0 ? fma(0.0, r, 1.0) : fma(-1.0, r, 0.0))
                           : (lane == 0 ? fma(1.0, r, 0.0) : fma(0.0, r, -1.0));
  const double q2 = num2 / den;
  scale.x = __shfl_sync(0xffffffffu, q2, 0);
  scale.y = __shfl_sync(0xffffffffu, q2, 1);
  return true;
}

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC 2011, Sec. 3.2).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 key) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ key.x, lo1, hi0 ^ c.w ^ key.y, lo0);
    key.x += 0x9E3779B9u;
    key.y += 0xBB67AE85u;
  }
  return c;
}

// Complex normal (re, im iid N(0, 1/2)) from one Philox block: two 53-bit
// uniforms u1 in (0, 1], u2 in [0, 1), Box-Muller rho = sqrt(-log u1),
// angle 2 pi u2.
__device__ __forceinline__ double2 philox_complex_normal(uint64_t row, uint64_t col,
                                                         uint64_t seed, uint32_t stream_id) {
  const uint4 ctr = make_uint4((uint32_t)col, (uint32_t)(col >> 32), (uint32_t)row, stream_id);
  const uint4 w = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const uint64_t a = ((uint64_t)(w.x >> 5) << 26) + (uint64_t)(w.y >> 6);
  const uint64_t b = ((uint64_t)(w.z >> 5) << 26) + (uint64_t)(w.w >> 6);
  const double u1 = ((double)a + 1.0) * 0x1p-53;
  const double u2 = (double)b * 0x1p-53;
  const double rho = sqrt(-log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  return make_double2(rho * c, rho * s);
}
#endif
