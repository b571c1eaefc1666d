// Seeded Gaussian matrices on the device: the test matrix Omega of the
// randomization step (Sec. 2) and the probes of the error estimate.
#include "rid_internal.cuh"

namespace {

__global__ void gaussian_kernel(double2* __restrict__ out, int64_t rows, int64_t cols,
                                int64_t row_stride, int64_t col_stride, uint64_t seed,
                                uint32_t stream_id) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    // consecutive threads take consecutive columns of one row
    const int64_t i = e / cols, j = e - i * cols;
    out[i * row_stride + j * col_stride] = philox_complex_normal(i, j, seed, stream_id);
  }
}

}  // namespace

cudaError_t rid_launch_gaussian(double2* out, int64_t rows, int64_t cols, int64_t row_stride,
                                int64_t col_stride, uint64_t seed, uint32_t stream_id,
                                cudaStream_t stream) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  gaussian_kernel<<<(unsigned)blocks, 256, 0, stream>>>(out, rows, cols, row_stride, col_stride,
                                                        seed, stream_id);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The paper's randomization (Sec. 2): Y = S F D A, with D = diag(exp(2 pi i
// phi_j)) (random phases), F the m x m DFT F_jk = exp(-2 pi i j k / m) (0-based)
// and S the l x m row sampler picking rows s_1..s_l.  As a test matrix,
// row q of S F D is  Omega_srft(q, j) = exp(-2 pi i s_q j / m) exp(2 pi i phi_j).
// phi_j is the second uniform of the Philox block at counter (j lo, j hi, 0, 5);
// s_q = floor(u2 m) of the block at counter (q, 0, 1, 5).
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ double philox_u2(uint64_t c01, uint32_t c2, uint64_t seed) {
  const uint4 ctr = make_uint4((uint32_t)c01, (uint32_t)(c01 >> 32), c2, RID_STREAM_SRFT);
  const uint4 w = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const uint64_t b = ((uint64_t)(w.z >> 5) << 26) + (uint64_t)(w.w >> 6);
  return (double)b * 0x1p-53;
}

__global__ void srft_kernel(double2* __restrict__ out, int64_t l, int64_t m, int64_t ldo, uint64_t seed) {
  const int64_t total = l * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / m, j = e - q * m;
    int64_t s = (int64_t)floor(philox_u2((uint64_t)q, 1u, seed) * (double)m);
    if (s > m - 1) s = m - 1;
    const double phi = philox_u2((uint64_t)j, 0u, seed);
    // exact phase index (s j mod m), then the angle in turns
    const unsigned __int128 sj = (unsigned __int128)(uint64_t)s * (uint64_t)j;
    const int64_t r = (int64_t)(sj % (unsigned __int128)(uint64_t)m);
    double turns = phi - (double)r / (double)m;       // in (-1, 1)
    double sn, cs;
    sincospi(2.0 * turns, &sn, &cs);
    out[q * ldo + j] = make_double2(cs, sn);
  }
}

}  // namespace

cudaError_t rid_launch_srft(double2* out, int64_t l, int64_t m, int64_t ldo, uint64_t seed, cudaStream_t stream) {
  const int64_t total = l * m;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  srft_kernel<<<(unsigned)blocks, 256, 0, stream>>>(out, l, m, ldo, seed);
  return cudaGetLastError();
}
