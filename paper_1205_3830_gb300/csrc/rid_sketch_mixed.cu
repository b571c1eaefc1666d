// Mixed-precision randomization for complex64 A: Y = Omega A with BF16x3
// splits on the tcgen05 tensor cores and FP32 accumulation; the pivoted QR,
// the solve and the error estimate that follow stay FP64 (the sketch Y is
// complex128).
//
// Every real value x (FP32 entries of A, FP64 entries of Omega) is split into
// three BF16 terms, hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid),
// which carry about 24 bits of x.  The product keeps the six term pairs with
// s + t <= 2 (the others are below 2^-24 of the leading term) and sums them,
// over the CTA's K range of at most 2048 reals, in one FP32 TMEM accumulator.
// The same real view as the FP64-emulated path is used (Omega' of 2l x 2m
// real rows, A' = A's floats read as 2m x n), N-tiles of up to 256 rows of
// Omega', 64-byte rows of K = 32 per stage.  K-split partials are summed in
// FP64.
#include <cudaTypedefs.h>

#include "rid_internal.cuh"
#include "rid_tc.cuh"
#include "rid_tc_digits.cuh"

using namespace rid_tc;

namespace {

constexpr int MX_S = 3;                    // BF16 terms per value
constexpr int MX_PAIRS = 6;                // (s, t) with s + t <= 2
constexpr int MX_KS = 32;                  // K per stage (64-byte rows)
constexpr int MX_STAGES = 3;
constexpr int MX_THREADS = 192;            // warp 0 TMA, 1 MMA + TMEM, 2-5 epilogue
// K stages one FP32 accumulator sums at most (2048 reals): the rounding of the
// FP32 sums grows with the square root of their length, so the K-split is
// raised until every split is this short; the splits are summed in
// double-FP32 pairs (mx_reduce_kernel).
constexpr int MX_MAX_STAGES_PER_SPLIT = 64;
constexpr long long MX_WAIT_BUDGET = 4000000000ll;
constexpr int MX_SMEM_MAX = MX_STAGES * MX_S * (128 + 256) * MX_KS * 2 + 1024;   // 222208 bytes
static_assert(MX_SMEM_MAX <= 232448 - 1024, "mixed stages exceed shared memory");

struct MxState {
  int64_t KP;              // padded 2m (multiple of MX_KS)
  int nchunk;              // K stages in total
  int l2, ntiles, tile_w, l2p, nblocks, ksplit, stages_per_split;
  uint16_t* om_slices;     // [3][l2][KP]
  uint16_t* a_slices;      // [3][n][KP]
  float* partial;          // [ksplit][n][l2p]
  int* err;
  CUtensorMap map_a, map_om;
};

__device__ __forceinline__ uint16_t bf16_rn(float x) {
  const uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);   // inf / nan: keep
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);          // round to nearest even
}
__device__ __forceinline__ float bf16_to_f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// hi / mid / lo BF16 terms of x.
__device__ __forceinline__ void split3(double x, uint16_t (&t)[MX_S]) {
  const uint16_t h = bf16_rn((float)x);
  const double r1 = x - (double)bf16_to_f(h);
  const uint16_t m = bf16_rn((float)r1);
  const double r2 = r1 - (double)bf16_to_f(m);
  t[0] = h;
  t[1] = m;
  t[2] = bf16_rn((float)r2);
}

// Omega' rows 2i = (Re w, -Im w), 2i+1 = (Im w, Re w), split into 3 terms.
__global__ void mx_omega_slice_kernel(const double2* __restrict__ om, int64_t ldo, int64_t m, int l, int64_t KP,
                                      uint16_t* __restrict__ slices) {
  const int64_t per_row = KP / 2;
  const int64_t total = (int64_t)l * per_row;
  const int64_t slice_stride = (int64_t)2 * l * KP;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / per_row);
    const int64_t r = e - (int64_t)i * per_row;
    const double2 w = r < m ? om[i * ldo + r] : make_double2(0.0, 0.0);
    uint16_t re[MX_S], nim[MX_S], im[MX_S];
    split3(w.x, re);
    split3(-w.y, nim);
    split3(w.y, im);
    for (int s = 0; s < MX_S; ++s) {
      uint16_t* row0 = slices + s * slice_stride + (int64_t)(2 * i) * KP + 2 * r;
      *(uint32_t*)row0 = (uint32_t)re[s] | ((uint32_t)nim[s] << 16);
      *(uint32_t*)(row0 + KP) = (uint32_t)im[s] | ((uint32_t)re[s] << 16);
    }
  }
}

// hi / mid / lo BF16 terms of an FP32 value: every step is exact in FP32
// (x - hi keeps the 16 bits below hi, minus mid the last 8), so this equals
// split3((double)x) bit for bit at FP32 speed.
__device__ __forceinline__ void split3f(float x, uint16_t (&t)[MX_S]) {
  const uint16_t h = bf16_rn(x);
  const float r1 = x - __uint_as_float((uint32_t)h << 16);
  const uint16_t m = bf16_rn(r1);
  const float r2 = r1 - __uint_as_float((uint32_t)m << 16);
  t[0] = h;
  t[1] = m;
  t[2] = bf16_rn(r2);
}

// A' columns (complex64 A read as 2m floats), split into 3 terms; zero padding
// to KP.  A warp takes one chunk of 128 complex rows of one column, lane l
// the rows 4l .. 4l + 3: 8-byte or (every column 16-byte aligned: vec) 16-byte
// loads and one 16-byte store per term.  With cexp (plans with row probes),
// the warp also stores the chunk's exponent (the largest entry's, exp_of_f)
// at cexp[chunk * ldce + column]: the row probes' product cuts A's digits
// relative to it (rid_probe_tc.cu).  Every chunk of every column of the range
// is written.
__global__ void __launch_bounds__(256) mx_a_slice_kernel(const float2* __restrict__ A, int64_t lda, int64_t m,
                                                         int64_t n, int64_t KP, int64_t slice_stride, bool vec,
                                                         uint16_t* __restrict__ slices, int* __restrict__ cexp,
                                                         int64_t ldce) {
  // A, slices and cexp start at the first of the n columns of the range; the
  // term planes of the whole matrix are slice_stride apart
  const int64_t rows_p = KP / 2;                      // complex rows with the padding (a multiple of 16)
  const int64_t cpc = (rows_p + 127) / 128;           // chunks per column
  const int64_t units = n * cpc;
  const int lane = threadIdx.x & 31;
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < units; u += wstride) {
    const int64_t j = u / cpc;
    const int c = (int)(u - j * cpc);
    const int64_t r0 = (int64_t)c * 128 + 4 * lane;
    const float2* col = A + j * lda + r0;
    float2 x[4];
    if (vec && r0 + 4 <= m) {
      const float4 f0 = __ldcs((const float4*)col), f1 = __ldcs((const float4*)col + 1);
      x[0] = make_float2(f0.x, f0.y);
      x[1] = make_float2(f0.z, f0.w);
      x[2] = make_float2(f1.x, f1.y);
      x[3] = make_float2(f1.z, f1.w);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = r0 + q < m ? __ldcs(col + q) : make_float2(0.f, 0.f);
    }
    if (r0 < rows_p) {                                 // rows_p is a multiple of 4: all four or none
      uint32_t w[MX_S][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint16_t re[MX_S], im[MX_S];
        split3f(x[q].x, re);
        split3f(x[q].y, im);
#pragma unroll
        for (int s = 0; s < MX_S; ++s) w[s][q] = (uint32_t)re[s] | ((uint32_t)im[s] << 16);
      }
#pragma unroll
      for (int s = 0; s < MX_S; ++s)
        *(uint4*)(slices + s * slice_stride + j * KP + 2 * r0) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
    if (cexp) {
      // |x| orders as the bit pattern of |x| does
      uint32_t mx = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        mx = max(mx, max(__float_as_uint(x[q].x) & 0x7FFFFFFFu, __float_as_uint(x[q].y) & 0x7FFFFFFFu));
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) cexp[c * ldce + j] = exp_of_f(__uint_as_float(mx));
    }
  }
}

struct MxArgs {
  int n, l2, l2p, tile_w, stages_per_split, nchunk;
  int jb0;                // first column block of the launch
  int64_t j_end;          // columns below this have results in the launch
  uint32_t stage_bytes;
  float* partial;
  int* err;
};

__global__ void __launch_bounds__(MX_THREADS, 1)
sketch_mixed_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_om, MxArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[MX_STAGES], empty_bar[MX_STAGES], acc_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = blockIdx.x, jb = a.jb0 + (int)blockIdx.y, ks = blockIdx.z;
  const int row0 = nb * a.tile_w;
  const int n_tile = min(a.tile_w, a.l2 - row0);
  const int n_mma = (n_tile + 15) & ~15;
  const int st_begin = ks * a.stages_per_split;
  const int nst = max(0, min(a.nchunk, st_begin + a.stages_per_split) - st_begin);
  const int a_tile_bytes = 128 * MX_KS * 2;
  const int o_tile_bytes = a.tile_w * MX_KS * 2;
  const int stage_stride = MX_S * (a_tile_bytes + o_tile_bytes);

  if (warp == 1) tmem_alloc(&tmem_slot, 256);
  if (threadIdx.x == 0) {
    for (int i = 0; i < MX_STAGES; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    mbar_init(&acc_done, 1);
    fence_barrier_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  auto a_tile = [&](int slot, int s) { return smem + slot * stage_stride + s * a_tile_bytes; };
  auto o_tile = [&](int slot, int s) { return smem + slot * stage_stride + MX_S * a_tile_bytes + s * o_tile_bytes; };
  auto fail = [&](int code) {
    s_abort = 1;
    atomicCAS(a.err, 0, code);
  };

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tensormap(&map_a);
      prefetch_tensormap(&map_om);
      int it = 0;
      for (; it < nst && !s_abort; ++it) {
        const int slot = it % MX_STAGES, round = it / MX_STAGES;
        if (round > 0 && !mbar_wait(&empty_bar[slot], (round - 1) & 1, MX_WAIT_BUDGET)) {
          fail(41);
          break;
        }
        const int x = (st_begin + it) * MX_KS;
        mbar_arrive_expect_tx(&full_bar[slot], a.stage_bytes);
        for (int s = 0; s < MX_S; ++s) {
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
              ::"r"(smem_u32(a_tile(slot, s))), "l"((uint64_t)&map_a), "r"(smem_u32(&full_bar[slot])), "r"(x),
              "r"(jb * 128), "r"(s)
              : "memory");
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
              ::"r"(smem_u32(o_tile(slot, s))), "l"((uint64_t)&map_om), "r"(smem_u32(&full_bar[slot])), "r"(x),
              "r"(row0), "r"(s)
              : "memory");
        }
      }
      for (int k = max(0, it - MX_STAGES); k < it; ++k)
        if (!mbar_wait(&full_bar[k % MX_STAGES], (k / MX_STAGES) & 1, MX_WAIT_BUDGET)) fail(42);
    }
  } else if (warp == 1) {
    // the whole warp runs the issue loop; elect.sync picks the lane that issues
    const uint32_t idesc = idesc_bf16_f32(128, n_mma);
    bool first = true;
    for (int it = 0; it < nst && !s_abort; ++it) {
      const int slot = it % MX_STAGES, round = it / MX_STAGES;
      if (!__all_sync(0xffffffffu, mbar_wait(&full_bar[slot], round & 1, MX_WAIT_BUDGET))) {
        if (lane == 0) fail(43);
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int d = 2; d >= 0; --d) {           // smallest terms first
#pragma unroll
        for (int s = 0; s <= d; ++s) {
          const int t = d - s;
          const uint64_t da = desc_sw64(a_tile(slot, t)), db = desc_sw64(o_tile(slot, s));
#pragma unroll
          for (int kk = 0; kk < MX_KS / 16; ++kk) {
            mma_bf16_w(tmem, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc, first ? 0u : 1u);
            first = false;
          }
        }
      }
      mma_commit_w(&empty_bar[slot]);
    }
    mma_commit_w(&acc_done);
  } else {
    // epilogue (warps 2-5): the accumulator rows of this warp's lane quarter
    const int quarter = warp & 3;
    const int64_t j = (int64_t)jb * 128 + quarter * 32 + lane;
    const bool waited = mbar_wait(&acc_done, 0, MX_WAIT_BUDGET * 4);
    const bool ok = __all_sync(0xffffffffu, waited);      // one decision for the whole warp
    if (!ok && lane == 0) fail(44);
    tc_fence_after();
    const bool go = __all_sync(0xffffffffu, ok && !s_abort && nst > 0);
    if (go) {
      for (int c0 = 0; c0 < n_mma; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, r);
        tmem_ld_wait();
        if (j < a.j_end) {
          float* dst = a.partial + ((int64_t)ks * a.n + j) * a.l2p + row0 + c0;
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (c0 + q < n_tile) dst[q] = __uint_as_float(r[q]);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    if (!mbar_wait(&acc_done, 0, MX_WAIT_BUDGET)) fail(45);
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

// columns j0 .. j0 + ncols - 1 of the n-column partial sums
__global__ void mx_reduce_kernel(const float* __restrict__ partial, int ksplit, int64_t n, int l, int l2p,
                                 double2* __restrict__ Y, int64_t ldy, int64_t j0, int64_t ncols) {
  const int64_t total = ncols * l;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = j0 + e / l;
    const int i = (int)(e - (j - j0) * l);
    // The splits in order, their loads batched ahead of the additions, summed
    // as double-FP32 pairs (hi + lo; TwoSum keeps each addition's rounding
    // error): about 48 bits, far below the FP32 grade of the partials, on
    // the FP32 pipe rather than GB300's narrow FP64 one.
    float re_h = 0.f, re_l = 0.f, im_h = 0.f, im_l = 0.f;
    auto two_sum = [](float& h, float& lo, float v) {
      const float s = __fadd_rn(h, v);
      const float bp = __fsub_rn(s, h);
      lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(v, bp)));
      h = s;
    };
    const float2* p = (const float2*)(partial + j * l2p) + i;
    const int64_t split_stride = n * l2p / 2;                     // float2 units
    for (int s0 = 0; s0 < ksplit; s0 += 8) {
      float2 q[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (s0 + u < ksplit) q[u] = __ldcs(p + (int64_t)(s0 + u) * split_stride);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (s0 + u < ksplit) {
          two_sum(re_h, re_l, q[u].x);
          two_sum(im_h, im_l, q[u].y);
        }
    }
    Y[i + j * ldy] = make_double2((double)re_h + (double)re_l, (double)im_h + (double)im_l);
  }
}

int make_map(CUtensorMap* map, const void* base, int64_t KP, int64_t rows, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return -1;
    enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  cuuint64_t gdim[3] = {(cuuint64_t)KP, (cuuint64_t)rows, (cuuint64_t)MX_S};
  cuuint64_t gstride[2] = {(cuuint64_t)KP * 2, (cuuint64_t)(KP * 2 * rows)};
  cuuint32_t box[3] = {MX_KS, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, gdim, gstride, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

}  // namespace

void rid_mx_plan_free(rid_plan_s* p) {
  MxState* st = (MxState*)p->tc_state;
  if (!st) return;
  rid_dev_free(st->om_slices, p->stream);   // released in stream order
  free(st);
  p->tc_state = nullptr;
  p->tc_bytes = 0;
}

rid_status rid_mx_plan_setup(rid_plan_s* p, int dry_run) {
  if (p->mode != RID_MIXED_BF16 || p->dtype != RID_C64) return RID_EUNSUPPORTED;
  MxState* st = (MxState*)calloc(1, sizeof(MxState));
  if (!st) return RID_ENOMEM;
  st->KP = (2 * p->m + MX_KS - 1) / MX_KS * MX_KS;
  st->nchunk = (int)(st->KP / MX_KS);
  st->l2 = 2 * p->l;
  st->ntiles = (st->l2 + 255) / 256;
  st->tile_w = ((st->l2 + st->ntiles - 1) / st->ntiles + 15) / 16 * 16;
  st->l2p = st->ntiles * st->tile_w;
  st->nblocks = (int)((p->n + 127) / 128);
  {
    const int units = st->ntiles * st->nblocks;
    int ks = (2 * p->num_sms + units - 1) / units;
    const int max_ks = st->nchunk / 16 > 0 ? st->nchunk / 16 : 1;   // at least 16 stages per split
    if (ks > max_ks) ks = max_ks;
    const int min_ks = (st->nchunk + MX_MAX_STAGES_PER_SPLIT - 1) / MX_MAX_STAGES_PER_SPLIT;
    if (ks < min_ks) ks = min_ks;
    if (ks < 1) ks = 1;
    st->stages_per_split = (st->nchunk + ks - 1) / ks;
    st->ksplit = (st->nchunk + st->stages_per_split - 1) / st->stages_per_split;
  }
  const size_t om_bytes = (size_t)MX_S * st->l2 * st->KP * 2;
  const size_t a_bytes = (size_t)MX_S * p->n * st->KP * 2;
  const size_t part_bytes = (size_t)st->ksplit * p->n * st->l2p * 4;
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  const size_t total = al(om_bytes) + al(a_bytes) + al(part_bytes) + al(4);
  if (dry_run) {
    p->tc_bytes = total;
    free(st);
    return RID_OK;
  }
  char* base = nullptr;
  if (rid_dev_alloc((void**)&base, total, p->stream, p->device) != cudaSuccess) {
    free(st);
    return RID_ENOMEM;
  }
  st->om_slices = (uint16_t*)base;
  st->a_slices = (uint16_t*)(base + al(om_bytes));
  st->partial = (float*)(base + al(om_bytes) + al(a_bytes));
  st->err = (int*)(base + al(om_bytes) + al(a_bytes) + al(part_bytes));
  p->tc_state = st;
  p->tc_bytes = total;
  p->tc_sketch_launches = 3;
  if (make_map(&st->map_a, st->a_slices, st->KP, p->n, 128) ||
      make_map(&st->map_om, st->om_slices, st->KP, st->l2, st->tile_w)) {
    rid_mx_plan_free(p);
    return RID_ECUDA;
  }
  cudaError_t e = cudaMemsetAsync(st->err, 0, 4, p->stream);
  if (e == cudaSuccess) {
    int64_t blocks = ((int64_t)p->l * (st->KP / 2) + 255) / 256;
    if (blocks > (int64_t)p->num_sms * 32) blocks = (int64_t)p->num_sms * 32;
    mx_omega_slice_kernel<<<(unsigned)blocks, 256, 0, p->stream>>>(p->omega, p->ldo, p->m, p->l, st->KP,
                                                                    st->om_slices);
    e = cudaGetLastError();
  }
  const int smem = MX_STAGES * MX_S * (128 * MX_KS * 2 + st->tile_w * MX_KS * 2) + 1024;
  // the attribute is process-wide and plans of other shapes launch the kernel
  // from other host threads: always the bound for the widest tile (256 rows)
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sketch_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MX_SMEM_MAX);
  if (e != cudaSuccess) {
    rid_mx_plan_free(p);
    return RID_ECUDA;
  }
  return RID_OK;
}

// Columns col0 .. col0 + ncols - 1 (col0 a multiple of 128) of Y; the
// K-split is the plan's, so column ranges give the same Y as one call.
cudaError_t rid_mx_sketch_cols(const rid_plan_s* p, const void* A_, int64_t lda, double2* Y, int64_t ldy,
                               int64_t col0, int64_t ncols) {
  const MxState* st = (const MxState*)p->tc_state;
  if (!st) return cudaErrorNotSupported;
  if (ncols <= 0) return cudaSuccess;
  const float2* A = (const float2*)A_ + col0 * lda;
  if (p->timing) {
    p->ev_panels = 1;
    cudaEventRecord(p->ev[0], p->stream);
  }
  cudaError_t e;
  {
    const int64_t units = ncols * ((st->KP / 2 + 127) / 128);   // a warp per chunk of a column
    int64_t blocks = (units + 7) / 8;
    if (blocks > (int64_t)p->num_sms * 32) blocks = (int64_t)p->num_sms * 32;
    // with row probes, also the chunk exponents of these columns
    int nc = 0;
    int* cexp = p->nrow > 0 ? rid_tc_probe_chunk_exp(p, &nc) : nullptr;
    const bool vec = ((uintptr_t)A_ & 15u) == 0 && lda % 2 == 0;
    mx_a_slice_kernel<<<(unsigned)blocks, 256, 0, p->stream>>>(A, lda, p->m, ncols, st->KP, p->n * st->KP, vec,
                                                              st->a_slices + col0 * st->KP,
                                                              cexp ? cexp + col0 : nullptr, p->n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (p->timing) cudaEventRecord(p->ev[1], p->stream);
  MxArgs args{(int)p->n, st->l2, st->l2p, st->tile_w, st->stages_per_split, st->nchunk, (int)(col0 / 128),
              col0 + ncols, (uint32_t)(MX_S * (128 + st->tile_w) * MX_KS * 2), st->partial, st->err};
  const int smem = MX_STAGES * MX_S * (128 * MX_KS * 2 + st->tile_w * MX_KS * 2) + 1024;
  const dim3 grid((unsigned)st->ntiles, (unsigned)((ncols + 127) / 128), (unsigned)st->ksplit);
  sketch_mixed_kernel<<<grid, MX_THREADS, smem, p->stream>>>(st->map_a, st->map_om, args);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (p->timing) cudaEventRecord(p->ev[2], p->stream);
  {
    const int64_t total = ncols * (int64_t)p->l;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)p->num_sms * 32) blocks = (int64_t)p->num_sms * 32;
    mx_reduce_kernel<<<(unsigned)blocks, 256, 0, p->stream>>>(st->partial, st->ksplit, p->n, p->l, st->l2p, Y, ldy,
                                                             col0, ncols);
    e = cudaGetLastError();
  }
  if (p->timing) cudaEventRecord(p->ev[3], p->stream);
  return e;
}

cudaError_t rid_mx_sketch(const rid_plan_s* p, const void* A, int64_t lda, double2* Y, int64_t ldy) {
  return rid_mx_sketch_cols(p, A, lda, Y, ldy, 0, p->n);
}

int rid_mx_error_word(const rid_plan_s* p) {
  const MxState* st = (const MxState*)p->tc_state;
  if (!st) return 0;
  int h = 0;
  cudaMemcpyAsync(&h, st->err, 4, cudaMemcpyDeviceToHost, p->stream);
  cudaStreamSynchronize(p->stream);
  return h;
}

rid_status rid_mx_plan_init(rid_plan_s* p) { return rid_mx_plan_setup(p, 0); }
