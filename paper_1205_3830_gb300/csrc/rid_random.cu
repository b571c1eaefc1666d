// Seeded Gaussian matrices on the device: the test matrix Omega of the
// randomization step (Sec. 2) and the probes of the error estimate.
#include <climits>

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

// ---------------------------------------------------------------------------
// Rounded test matrix: every entry of a row rounded to `bits` bits below the
// row's largest entry.  Row r gets E_r with |Re w|, |Im w| < 2^E_r (E = the
// exponent of x = f 2^E, 1/2 <= |f| < 1; zeros ignored), and each real part
// becomes the nearest multiple of 2^(E_r - bits), ties to even, except that a
// value which would reach +-2^E_r takes the multiple below (the row keeps
// E_r).  The rounded row then holds ceil(bits / 8) base-256 digits exactly.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ int frexp_exp(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  return ex == 0 ? INT_MIN : ex - 1022;      // subnormals and zero carry no exponent here
}

__global__ void __launch_bounds__(256) round_rows_kernel(double2* __restrict__ om, int64_t ldo, int64_t m,
                                                         int bits) {
  __shared__ int red[8];
  double2* row = om + (int64_t)blockIdx.x * ldo;
  int e = INT_MIN;
  for (int64_t j = threadIdx.x; j < m; j += 256) {
    const double2 w = row[j];
    e = max(e, max(frexp_exp(w.x), frexp_exp(w.y)));
  }
  e = __reduce_max_sync(0xffffffffu, e);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  int E = red[0];
  for (int w = 1; w < 8; ++w) E = max(E, red[w]);
  if (E == INT_MIN) return;                   // an all-zero row stays zero
  // a value that would round up to +-2^E takes the multiple below: the row keeps E
  const double top = scalbn(1.0, bits) - 1.0;
  for (int64_t j = threadIdx.x; j < m; j += 256) {
    const double2 w = row[j];
    row[j] = make_double2(scalbn(fmin(fmax(rint(scalbn(w.x, bits - E)), -top), top), E - bits),
                          scalbn(fmin(fmax(rint(scalbn(w.y, bits - E)), -top), top), E - bits));
  }
}

}  // namespace

cudaError_t rid_launch_round_rows(double2* om, int64_t rows, int64_t m, int64_t ldo, int bits, cudaStream_t stream) {
  if (rows <= 0) return cudaSuccess;
  round_rows_kernel<<<(unsigned)rows, 256, 0, stream>>>(om, ldo, m, bits);
  return cudaGetLastError();
}
