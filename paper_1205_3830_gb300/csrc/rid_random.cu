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
