// Randomization Y = Omega A (Sec. 2) with FP64 FMA on the CUDA cores.
//
// Tiled complex GEMM: a CTA of 256 threads owns a 32 x 32 tile of Y (rows of
// Omega x columns of A) and one K-range of the m-long reduction.  Both
// operands are K-contiguous (Omega row-major, A column-major), so each
// 16-element K-chunk of a row/column is one 256-byte coalesced load staged in
// shared memory.  The FP64 pipe of GB300 (about 2 DFMA per clock per SM)
// bounds this kernel; every other resource is far from its limit.
// Split-K partials are summed by a second kernel in a fixed order, so the
// result does not depend on scheduling.  With row probes set, Omega has
// ls = l + r rows: rows below l go to Y, the r probe rows to X = G A.
#include "rid_internal.cuh"

namespace {

constexpr int BL = 32;   // rows of Y per CTA
constexpr int BN = 32;   // columns of Y per CTA
constexpr int BK = 16;   // reduction chunk (complex elements)

__global__ void __launch_bounds__(256)
sketch_fp64_kernel(const double2* __restrict__ Om, int64_t ldo, const double2* __restrict__ A,
                   int64_t lda, double2* __restrict__ out, int64_t ldout, int64_t out_split_stride,
                   int64_t l, int64_t m, int64_t n, int64_t k_per_split, int64_t ly,
                   double2* __restrict__ X, int64_t ldx) {
  __shared__ double2 Os[BL][BK + 1];
  __shared__ double2 As[BN][BK + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * BL;
  const int64_t j0 = (int64_t)blockIdx.y * BN;
  const int64_t r_begin = (int64_t)blockIdx.z * k_per_split;
  int64_t r_end = r_begin + k_per_split;
  if (r_end > m) r_end = m;

  double2 acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0.0, 0.0);

  for (int64_t r0 = r_begin; r0 < r_end; r0 += BK) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + h * 256;
      const int row = e / BK, rr = e % BK;
      const int64_t gi = i0 + row, gr = r0 + rr, gj = j0 + row;
      Os[row][rr] = (gi < l && gr < r_end) ? Om[gi * ldo + gr] : make_double2(0.0, 0.0);
      As[row][rr] = (gj < n && gr < r_end) ? A[gj * lda + gr] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < BK; ++rr) {
      const double2 o0 = Os[ty][rr], o1 = Os[ty + 16][rr];
      const double2 a0 = As[tx][rr], a1 = As[tx + 16][rr];
      acc[0][0] = cfma(o0, a0, acc[0][0]);
      acc[0][1] = cfma(o0, a1, acc[0][1]);
      acc[1][0] = cfma(o1, a0, acc[1][0]);
      acc[1][1] = cfma(o1, a1, acc[1][1]);
    }
    __syncthreads();
  }

  double2* dst = out + (int64_t)blockIdx.z * out_split_stride;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int64_t gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * b;
      if (gi < l && gj < n) {
        if (gi < ly) dst[gi + gj * ldout] = acc[a][b];
        else X[(gi - ly) + gj * ldx] = acc[a][b];
      }
    }
}

// Y(i, j) = sum_{s = 0..S-1} partial_s(i, j), in that order (rows i >= ly: X).
__global__ void splitk_reduce_kernel(const double2* __restrict__ part, int64_t split_stride,
                                     int splits, double2* __restrict__ Y, int64_t ldy, int64_t l,
                                     int64_t n, int64_t ly, double2* __restrict__ X, int64_t ldx) {
  const int64_t total = l * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / l, i = e - j * l;
    double2 s = part[e];
    for (int t = 1; t < splits; ++t) {
      const double2 v = part[(int64_t)t * split_stride + e];
      s.x += v.x;
      s.y += v.y;
    }
    if (i < ly) Y[i + j * ldy] = s;
    else X[(i - ly) + j * ldx] = s;
  }
}

}  // namespace

cudaError_t rid_launch_sketch_fp64(const rid_plan_s* p, const double2* A, int64_t lda, double2* Y,
                                   int64_t ldy, int64_t col0, int64_t ncols) {
  // columns col0 .. col0 + ncols - 1: every column is independent
  if (ncols <= 0) return cudaSuccess;
  const int64_t ls = p->ls, ly = p->l, ldx = p->nrow > 0 ? p->nrow : 1;
  A += col0 * lda;
  Y += col0 * ldy;
  double2* X = p->xrow ? p->xrow + col0 * ldx : nullptr;
  const int64_t n = ncols;
  const dim3 grid((unsigned)((ls + BL - 1) / BL), (unsigned)((n + BN - 1) / BN),
                  (unsigned)p->split_k);
  if (p->timing) {
    p->ev_panels = 1;
    cudaEventRecord(p->ev[0], p->stream);
    cudaEventRecord(p->ev[1], p->stream);
  }
  if (p->split_k == 1) {
    sketch_fp64_kernel<<<grid, 256, 0, p->stream>>>(p->omega, p->ldo, A, lda, Y, ldy, 0, ls,
                                                    p->m, n, p->k_per_split, ly, X, ldx);
    if (p->timing) {
      cudaEventRecord(p->ev[2], p->stream);
      cudaEventRecord(p->ev[3], p->stream);
    }
    return cudaGetLastError();
  }
  const int64_t stride = ls * n;
  sketch_fp64_kernel<<<grid, 256, 0, p->stream>>>(p->omega, p->ldo, A, lda, p->sk_partial, ls,
                                                  stride, ls, p->m, n, p->k_per_split, ls, nullptr, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t blocks = (stride + 255) / 256;
  if (blocks > (int64_t)p->num_sms * 16) blocks = (int64_t)p->num_sms * 16;
  if (p->timing) cudaEventRecord(p->ev[2], p->stream);
  splitk_reduce_kernel<<<(unsigned)blocks, 256, 0, p->stream>>>(p->sk_partial, stride,
                                                                p->split_k, Y, ldy, ls, n, ly, X, ldx);
  if (p->timing) cudaEventRecord(p->ev[3], p->stream);
  return cudaGetLastError();
}
