// C ABI of the randomized ID: plans, argument checks and dispatch to the
// kernels.  Every entry point validates its arguments on the host before it
// launches anything.
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <string.h>

#include "rid_internal.cuh"

// Tensor-core paths: FP64-emulated (rid_sketch_tc.cu) and mixed precision
// (rid_sketch_mixed.cu).
rid_status rid_tc_plan_init_fp64(rid_plan_s* p);
void rid_tc_plan_free_fp64(rid_plan_s* p);
cudaError_t rid_tc_sketch_fp64(const rid_plan_s* p, const void* A, int64_t lda, double2* Y, int64_t ldy);
cudaError_t rid_tc_sketch_cols_fp64(const rid_plan_s* p, const void* A, int64_t lda, double2* Y, int64_t ldy,
                                    int64_t col0, int64_t ncols);
int rid_tc_error_word_fp64(const rid_plan_s* p);
rid_status rid_mx_plan_init(rid_plan_s* p);
rid_status rid_tc_plan_setup_fp64(rid_plan_s* p, int dry_run);
rid_status rid_mx_plan_setup(rid_plan_s* p, int dry_run);
void rid_mx_plan_free(rid_plan_s* p);
cudaError_t rid_mx_sketch(const rid_plan_s* p, const void* A, int64_t lda, double2* Y, int64_t ldy);
cudaError_t rid_mx_sketch_cols(const rid_plan_s* p, const void* A, int64_t lda, double2* Y, int64_t ldy,
                               int64_t col0, int64_t ncols);
int rid_mx_error_word(const rid_plan_s* p);
rid_status rid_tc_probe_init(rid_plan_s* p);
void rid_tc_probe_free(rid_plan_s* p);
cudaError_t rid_tc_probe_sketch(const rid_plan_s* p, const void* A, int64_t lda);
cudaError_t rid_tc_probe_sketch_cols(const rid_plan_s* p, const void* A, int64_t lda, int64_t col0, int64_t ncols);
int rid_tc_probe_error_word(const rid_plan_s* p);

static rid_status rid_tc_plan_init(rid_plan_s* p) {
  if (p->mode == RID_FP64_EMULATED) return rid_tc_plan_init_fp64(p);
  if (p->mode == RID_MIXED_BF16) return rid_mx_plan_init(p);
  return RID_EUNSUPPORTED;
}
static void rid_tc_plan_free(rid_plan_s* p) {
  if (p->mode == RID_FP64_EMULATED) rid_tc_plan_free_fp64(p);
  else if (p->mode == RID_MIXED_BF16) rid_mx_plan_free(p);
}
static cudaError_t rid_tc_sketch(const rid_plan_s* p, const void* A, int64_t lda, double2* Y, int64_t ldy) {
  if (p->mode == RID_FP64_EMULATED) return rid_tc_sketch_fp64(p, A, lda, Y, ldy);
  if (p->mode == RID_MIXED_BF16) return rid_mx_sketch(p, A, lda, Y, ldy);
  return cudaErrorNotSupported;
}
static int rid_tc_error_word(const rid_plan_s* p) {
  if (p->mode == RID_FP64_EMULATED) return rid_tc_error_word_fp64(p);
  if (p->mode == RID_MIXED_BF16) return rid_mx_error_word(p) | rid_tc_probe_error_word(p);
  return 0;
}
// The mixed mode's probe state follows the probe rows of Omega.
static rid_status rid_probe_state_reset(rid_plan_s* p) {
  rid_tc_probe_free(p);
  if (p->mode == RID_MIXED_BF16 && p->nrow > 0) return rid_tc_probe_init(p);
  return RID_OK;
}

namespace {

constexpr int POOL_MAX_DEVICES = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[POOL_MAX_DEVICES] = {};

// The library's memory pool on `device`, created on first use; it keeps freed
// memory (release threshold: unlimited) so plan after plan reuses it.
cudaMemPool_t pool_for(int device) {
  if (device < 0 || device >= POOL_MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (!g_pools[device]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[device] = pool;
  }
  return g_pools[device];
}

}  // namespace

cudaError_t rid_dev_alloc(void** ptr, size_t bytes, cudaStream_t stream, int device) {
  cudaMemPool_t pool = pool_for(device);
  if (!pool) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes, pool, stream);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

void rid_dev_free(void* ptr, cudaStream_t stream) {
  if (ptr) cudaFreeAsync(ptr, stream);
}

namespace {

// Keeps the caller's current device and switches to the plan's one.
struct DeviceGuard {
  int old = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&old) != cudaSuccess) { ok = false; return; }
    if (old != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (old >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != old) cudaSetDevice(old);
  }
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

rid_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return RID_OK;
  if (e == cudaErrorMemoryAllocation) return RID_ENOMEM;
  return RID_ECUDA;
}

// Workspace layout of a plan: one allocation, carved into 256-byte aligned pieces.
struct Layout {
  size_t omega, status, sk_partial, qr_val, qr_idx, qr_counter, tau, sel_cand, sel_val, sel_idx, sel_bar,
      res_cand, res_val, res_pos, res_col, res_flag, probes, wtilde, wj_part, ew_part, norm_part, err_out, total;
};

Layout plan_layout(const rid_plan_s* p) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t at = off; off += align256(bytes); return at; };
  L.omega = take((size_t)p->l * p->ldo * sizeof(double2));
  L.status = take(sizeof(int));
  L.sk_partial = take(p->split_k > 1 ? (size_t)p->split_k * p->l * p->n * sizeof(double2) : 0);
  L.qr_val = take((size_t)p->qr_grid * sizeof(double));
  L.qr_idx = take((size_t)p->qr_grid * sizeof(int));
  L.qr_counter = take(sizeof(unsigned));
  L.tau = take((size_t)p->k * sizeof(double2));
  L.sel_cand = take((size_t)2 * p->sel_grid_max * p->l * sizeof(double2));
  L.sel_val = take((size_t)2 * p->sel_grid_max * sizeof(double));
  L.sel_idx = take((size_t)2 * p->sel_grid_max * sizeof(int));
  L.sel_bar = take(2 * sizeof(unsigned));
  L.res_cand = take((size_t)2 * p->res_grid * p->l * sizeof(double2));
  L.res_val = take((size_t)2 * p->res_grid * sizeof(double));
  L.res_pos = take((size_t)2 * p->res_grid * sizeof(int));
  L.res_col = take((size_t)2 * p->res_grid * sizeof(int));
  L.res_flag = take((size_t)p->res_grid * sizeof(unsigned));
  L.probes = take((size_t)p->n * RID_MAX_PROBES * sizeof(double2));
  L.wtilde = take((size_t)p->n * RID_MAX_PROBES * sizeof(double2));
  L.wj_part = take((size_t)p->err_wj_grid * p->k * RID_MAX_PROBES * sizeof(double2));
  L.ew_part = take((size_t)p->err_col_split * RID_MAX_PROBES * p->m * sizeof(double2));
  L.norm_part = take((size_t)p->err_row_blocks * RID_MAX_PROBES * sizeof(double));
  L.err_out = take(2 * sizeof(double));
  L.total = off;
  return L;
}

void choose_launch_shapes(rid_plan_s* p) {
  const int64_t sms = p->num_sms;
  // sketch: enough (l-tile, n-tile, K-split) CTAs for two waves
  const int64_t tiles = ((p->l + 31) / 32) * ((p->n + 31) / 32);
  int64_t split = 1;
  if (tiles < 2 * sms) split = (2 * sms + tiles - 1) / tiles;
  const int64_t max_split = (p->m + 255) / 256;
  if (split > max_split) split = max_split;
  if (split < 1) split = 1;
  int64_t kps = (p->m + split - 1) / split;
  kps = (kps + 15) / 16 * 16;
  p->k_per_split = kps;
  p->split_k = (int)((p->m + kps - 1) / kps);
  // select: one warp per column, up to four CTAs per SM
  int64_t g = (p->n + 7) / 8;
  if (g > 4 * sms) g = 4 * sms;
  p->qr_grid = (int)(g < 1 ? 1 : g);
  p->sel_grid = rid_select_coop_grid(p->device, p->num_sms, p->n, p->l);
  p->sel_grid_max = p->sel_grid;
  p->res_grid = p->sel_grid > 0 ? rid_select_resident_grid(p->device, p->num_sms, p->n, p->l, &p->res_cpc, &p->res_smem)
                                : 0;
  // error
  const int64_t ncols = p->n - p->k;
  int64_t wg = (ncols + 63) / 64;
  if (wg > 2 * sms) wg = 2 * sms;
  p->err_wj_grid = (int)(wg < 1 ? 1 : wg);
  p->err_row_blocks = (int)((p->m + 255) / 256);
  int64_t cs = (2 * sms + p->err_row_blocks - 1) / p->err_row_blocks;
  const int64_t max_cs = (p->n + 31) / 32;
  if (cs > max_cs) cs = max_cs;
  p->err_col_split = (int)(cs < 1 ? 1 : cs);
}

}  // namespace

extern "C" {

const char* rid_status_string(rid_status s) {
  switch (s) {
    case RID_OK: return "RID_OK";
    case RID_EINVAL: return "RID_EINVAL: invalid argument";
    case RID_ENOMEM: return "RID_ENOMEM: device allocation failed";
    case RID_ECUDA: return "RID_ECUDA: CUDA error";
    case RID_ERANK: return "RID_ERANK: sketch has rank < k (redraw with another seed)";
    case RID_ETIMEOUT: return "RID_ETIMEOUT: device wait timed out";
    case RID_EUNSUPPORTED: return "RID_EUNSUPPORTED: dtype/mode not available";
  }
  return "RID_?: unknown status";
}

static rid_status check_plan_args(int64_t m, int64_t n, int32_t k, int32_t l, rid_dtype dtype, rid_mode mode) {
  if (m < 1 || n < 1 || k < 1 || l < k || k > m || k > n) return RID_EINVAL;
  if (n > 0x7fffffffLL || m > ((int64_t)1 << 40)) return RID_EINVAL;
  if (l > 512) return RID_EUNSUPPORTED;   // the QR keeps a column's l entries in one warp's registers
  if (dtype != RID_C128 && dtype != RID_C64) return RID_EINVAL;
  if (mode < RID_FP64_NATIVE || mode > RID_MIXED_3XTF32) return RID_EINVAL;
  if (dtype == RID_C128 && (mode == RID_MIXED_BF16 || mode == RID_MIXED_3XTF32)) return RID_EUNSUPPORTED;
  if (dtype == RID_C64 && (mode == RID_FP64_NATIVE || mode == RID_FP64_EMULATED)) return RID_EUNSUPPORTED;
  int nr = 0;
  if (rid_solve_smem_bytes(k, &nr) > 200 * 1024) return RID_EUNSUPPORTED;
  return RID_OK;
}

rid_status rid_plan_footprint(int64_t m, int64_t n, int32_t k, int32_t l, rid_dtype dtype, rid_mode mode,
                              size_t* bytes) {
  if (!bytes) return RID_EINVAL;
  const rid_status s = check_plan_args(m, n, k, l, dtype, mode);
  if (s != RID_OK) return s;
  rid_plan_s p{};
  p.m = m; p.n = n; p.k = k; p.l = l;
  p.dtype = dtype; p.mode = mode;
  if (cudaGetDevice(&p.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, p.device) != cudaSuccess)
    return RID_ECUDA;
  p.ldo = (m + 15) / 16 * 16;
  p.ls = l;
  choose_launch_shapes(&p);
  size_t total = plan_layout(&p).total;
  if (mode == RID_FP64_EMULATED || mode == RID_MIXED_BF16) {
    const rid_status t = mode == RID_FP64_EMULATED ? rid_tc_plan_setup_fp64(&p, 1) : rid_mx_plan_setup(&p, 1);
    if (t != RID_OK) return t;
    total += p.tc_bytes;
  } else if (mode != RID_FP64_NATIVE) {
    return RID_EUNSUPPORTED;
  }
  *bytes = total;
  return RID_OK;
}

static rid_status plan_create_impl(rid_plan_t* plan, int64_t m, int64_t n, int32_t k, int32_t l, rid_dtype dtype,
                                   rid_mode mode, uint64_t seed, void* stream, bool init_tc) {
  if (!plan) return RID_EINVAL;
  *plan = nullptr;
  const rid_status chk = check_plan_args(m, n, k, l, dtype, mode);
  if (chk != RID_OK) return chk;

  rid_plan_s* p = (rid_plan_s*)calloc(1, sizeof(rid_plan_s));
  if (!p) return RID_ENOMEM;
  p->m = m; p->n = n; p->k = k; p->l = l;
  p->dtype = dtype; p->mode = mode; p->seed = seed;
  p->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) { free(p); return RID_ECUDA; }
  p->ldo = (m + 15) / 16 * 16;     // 256-byte aligned rows of Omega
  p->ls = l;
  choose_launch_shapes(p);

  const Layout L = plan_layout(p);
  char* base = nullptr;
  e = rid_dev_alloc((void**)&base, L.total, p->stream, p->device);
  if (e != cudaSuccess) { free(p); return RID_ENOMEM; }
  p->ws_bytes = L.total;
  p->ws_base = base;
  p->omega = (double2*)(base + L.omega);
  p->status = (int*)(base + L.status);
  p->sk_partial = (double2*)(base + L.sk_partial);
  p->qr_val = (double*)(base + L.qr_val);
  p->qr_idx = (int*)(base + L.qr_idx);
  p->qr_counter = (unsigned*)(base + L.qr_counter);
  p->tau = (double2*)(base + L.tau);
  p->sel_cand = (double2*)(base + L.sel_cand);
  p->sel_val = (double*)(base + L.sel_val);
  p->sel_idx = (int*)(base + L.sel_idx);
  p->sel_bar = (unsigned*)(base + L.sel_bar);
  p->res_cand = (double2*)(base + L.res_cand);
  p->res_val = (double*)(base + L.res_val);
  p->res_pos = (int*)(base + L.res_pos);
  p->res_col = (int*)(base + L.res_col);
  p->res_flag = (unsigned*)(base + L.res_flag);
  p->probes = (double2*)(base + L.probes);
  p->wtilde = (double2*)(base + L.wtilde);
  p->wj_part = (double2*)(base + L.wj_part);
  p->ew_part = (double2*)(base + L.ew_part);
  p->norm_part = (double*)(base + L.norm_part);
  p->err_out = (double*)(base + L.err_out);

  e = cudaMemsetAsync(p->status, 0, sizeof(int), p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->qr_counter, 0, sizeof(unsigned), p->stream);
  if (e == cudaSuccess)
    e = rid_launch_gaussian(p->omega, l, m, p->ldo, 1, seed, RID_STREAM_OMEGA, p->stream);
  if (e != cudaSuccess) {
    rid_dev_free(base, p->stream);
    free(p);
    return RID_ECUDA;
  }
  if (mode != RID_FP64_NATIVE && init_tc) {
    const rid_status s = rid_tc_plan_init(p);
    if (s != RID_OK) {
      rid_dev_free(base, p->stream);
      cudaStreamSynchronize(p->stream);
      free(p);
      return s;
    }
  }
  *plan = p;
  return RID_OK;
}

rid_status rid_plan_create(rid_plan_t* plan, int64_t m, int64_t n, int32_t k, int32_t l,
                           rid_dtype dtype, rid_mode mode, uint64_t seed, void* stream) {
  return plan_create_impl(plan, m, n, k, l, dtype, mode, seed, stream, true);
}

rid_status rid_plan_destroy(rid_plan_t p) {
  if (!p) return RID_OK;
  DeviceGuard g(p->device);
  cudaStreamSynchronize(p->stream);
  if (p->timing)
    for (int i = 0; i < RID_TIMING_EVENTS; ++i) cudaEventDestroy(p->ev[i]);
  rid_tc_plan_free(p);
  rid_tc_probe_free(p);
  rid_dev_free(p->probe_base, p->stream);
  rid_dev_free(p->ws_base, p->stream);
  free(p);
  return RID_OK;
}

rid_status rid_plan_omega(rid_plan_t p, const void** omega, int64_t* ldo) {
  if (!p || !omega || !ldo) return RID_EINVAL;
  *omega = p->omega;
  *ldo = p->ldo;
  return RID_OK;
}

rid_status rid_plan_probe_products(rid_plan_t p, const void** X, int64_t* ldx) {
  if (!p || !X || !ldx) return RID_EINVAL;
  if (p->nrow < 1 || !p->x_valid) return RID_EINVAL;
  *X = p->xrow;
  *ldx = p->nrow;
  return RID_OK;
}

rid_status rid_plan_set_omega(rid_plan_t p, const void* omega, int64_t ldo) {
  if (!p || !omega || ldo < p->m) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  cudaError_t e = cudaMemcpy2DAsync(p->omega, p->ldo * sizeof(double2), omega, ldo * sizeof(double2),
                                    p->m * sizeof(double2), p->l, cudaMemcpyDeviceToDevice, p->stream);
  p->omega_bits = 0;                // a caller's Omega is taken as it is
  p->omega_kind = 1;
  if (e == cudaSuccess && p->mode != RID_FP64_NATIVE) {
    // the tensor-core paths keep Omega in split form: rebuild it
    rid_tc_plan_free(p);
    const rid_status s = rid_tc_plan_init(p);
    if (s != RID_OK) return s;
  }
  return from_cuda(e);
}

rid_status rid_plan_use_srft(rid_plan_t p, uint64_t srft_seed) {
  if (!p) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  cudaError_t e = rid_launch_srft(p->omega, p->l, p->m, p->ldo, srft_seed, p->stream);
  p->omega_kind = 2;
  if (e == cudaSuccess && p->omega_bits > 0)
    e = rid_launch_round_rows(p->omega, p->l, p->m, p->ldo, p->omega_bits, p->stream);
  if (e == cudaSuccess && p->mode != RID_FP64_NATIVE) {
    rid_tc_plan_free(p);          // the tensor-core paths keep Omega in split form
    const rid_status s = rid_tc_plan_init(p);
    if (s != RID_OK) return s;
  }
  return from_cuda(e);
}

rid_status rid_plan_round_omega(rid_plan_t p, int32_t bits) {
  if (!p || bits < 8 || bits > 48 || bits % 8 != 0) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  cudaError_t e = rid_launch_round_rows(p->omega, p->ls, p->m, p->ldo, bits, p->stream);
  if (e == cudaSuccess && p->nrow > 0) e = rid_launch_row_probe_norms(p);   // ||g_q||^2 of the rounded probes
  if (e != cudaSuccess) return from_cuda(e);
  p->omega_bits = (p->omega_bits > 0 && p->omega_bits < bits) ? p->omega_bits : bits;
  if (p->mode != RID_FP64_NATIVE) {
    rid_tc_plan_free(p);          // the tensor-core paths keep Omega in split form
    const rid_status s = rid_tc_plan_init(p);
    if (s != RID_OK) return s;
    const rid_status ps = rid_probe_state_reset(p);
    if (ps != RID_OK) return ps;
  }
  return from_cuda(cudaStreamSynchronize(p->stream));
}

// sync: the public call synchronizes the plan's stream before and after; a
// plan being created has nothing in flight, and everything below is ordered
// on its stream, so creation skips the waits.
static rid_status set_probes_impl(rid_plan_t p, int32_t nprobe, uint64_t probe_seed, bool sync) {
  if (!p || nprobe < 0 || nprobe > RID_MAX_PROBES) return RID_EINVAL;
  if (nprobe > 0 && p->mode != RID_FP64_NATIVE && p->mode != RID_FP64_EMULATED && p->mode != RID_MIXED_BF16)
    return RID_EUNSUPPORTED;
  if (p->l + nprobe > 512) return RID_EUNSUPPORTED;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  cudaError_t e = sync ? cudaStreamSynchronize(p->stream) : cudaSuccess;
  if (e != cudaSuccess) return from_cuda(e);
  const int32_t ls = p->l + nprobe;
  char* base = nullptr;
  size_t total = 0, o_x = 0, o_norm = 0, o_part = 0, o_sk = 0;
  const int lp_grid = (int)std::min<int64_t>(std::max<int64_t>((p->n - p->k + 7) / 8, 1), 2 * (int64_t)p->num_sms);
  if (nprobe > 0) {
    // Omega with the probe rows below it, X = G A, ||g_q||^2, partial sums,
    // and (native FP64, split K) partials with ls rows
    auto take = [&](size_t bytes) { size_t at = total; total += align256(bytes); return at; };
    take((size_t)ls * p->ldo * sizeof(double2));
    o_x = take((size_t)nprobe * p->n * sizeof(double2));
    o_norm = take((size_t)nprobe * sizeof(double));
    o_part = take((size_t)lp_grid * RID_MAX_PROBES * sizeof(double));
    o_sk = take(p->mode == RID_FP64_NATIVE && p->split_k > 1 ? (size_t)p->split_k * ls * p->n * sizeof(double2) : 0);
    if (rid_dev_alloc((void**)&base, total, p->stream, p->device) != cudaSuccess) return RID_ENOMEM;
    // the l rows of the test matrix, then G (Philox stream 6, key probe_seed)
    e = cudaMemcpyAsync(base, p->omega, (size_t)p->l * p->ldo * sizeof(double2), cudaMemcpyDeviceToDevice,
                        p->stream);
    if (e == cudaSuccess)
      e = rid_launch_gaussian((double2*)base + (int64_t)p->l * p->ldo, nprobe, p->m, p->ldo, 1, probe_seed,
                              RID_STREAM_LPROBES, p->stream);
    if (e == cudaSuccess && p->omega_bits > 0)
      e = rid_launch_round_rows((double2*)base + (int64_t)p->l * p->ldo, nprobe, p->m, p->ldo, p->omega_bits,
                                p->stream);
    if (e == cudaSuccess && sync) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
      rid_dev_free(base, p->stream);
      return from_cuda(e);
    }
  }
  // switch the plan over (the old Omega is no longer read)
  rid_tc_plan_free(p);
  if (nprobe > 0) {
    rid_dev_free(p->probe_base, p->stream);
    p->probe_base = base;
    p->probe_bytes = total;
    p->omega = (double2*)base;
    p->xrow = (double2*)(base + o_x);
    p->grow_norm2 = (double*)(base + o_norm);
    p->lp_part = (double*)(base + o_part);
    p->lp_grid = lp_grid;
    if (p->mode == RID_FP64_NATIVE && p->split_k > 1) p->sk_partial = (double2*)(base + o_sk);
  }
  // nprobe == 0 keeps the current Omega allocation; only its first l rows are read
  p->ls = ls;
  p->nrow = nprobe;
  p->x_valid = 0;
  if (nprobe > 0) {
    e = rid_launch_row_probe_norms(p);
    if (e != cudaSuccess) return from_cuda(e);
  }
  if (p->mode != RID_FP64_NATIVE) {
    const rid_status s = rid_tc_plan_init(p);
    if (s != RID_OK) return s;
  }
  const rid_status ps = rid_probe_state_reset(p);
  if (ps != RID_OK) return ps;
  return sync ? from_cuda(cudaStreamSynchronize(p->stream)) : RID_OK;
}

rid_status rid_plan_set_probes(rid_plan_t p, int32_t nprobe, uint64_t probe_seed) {
  return set_probes_impl(p, nprobe, probe_seed, true);
}

rid_status rid_plan_reseed(rid_plan_t p, uint64_t seed, uint64_t probe_seed) {
  if (!p) return RID_EINVAL;
  if (p->omega_kind != 0 || p->omega_bits > 0) return RID_EUNSUPPORTED;   // not the plain Gaussian of a seed
  if (p->mode != RID_FP64_NATIVE && p->mode != RID_FP64_EMULATED) return RID_EUNSUPPORTED;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  // the same draws as rid_plan_create and rid_plan_set_probes, in place
  cudaError_t e = cudaMemsetAsync(p->status, 0, sizeof(int), p->stream);
  if (e == cudaSuccess) e = rid_launch_gaussian(p->omega, p->l, p->m, p->ldo, 1, seed, RID_STREAM_OMEGA, p->stream);
  if (e == cudaSuccess && p->nrow > 0) {
    e = rid_launch_gaussian(p->omega + (int64_t)p->l * p->ldo, p->nrow, p->m, p->ldo, 1, probe_seed,
                            RID_STREAM_LPROBES, p->stream);
    if (e == cudaSuccess) e = rid_launch_row_probe_norms(p);
  }
  if (e == cudaSuccess && p->mode == RID_FP64_EMULATED) e = rid_tc_refresh_omega_fp64(p);
  if (e != cudaSuccess) return from_cuda(e);
  p->seed = seed;
  p->x_valid = 0;
  return RID_OK;
}

rid_status rid_plan_set_stream(rid_plan_t p, void* stream) {
  if (!p) return RID_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (s == p->stream) return RID_OK;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  // the new stream runs after everything already queued for this plan
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, p->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return from_cuda(e);
  p->stream = s;
  return RID_OK;
}

rid_status rid_plan_create_probes(rid_plan_t* plan, int64_t m, int64_t n, int32_t k, int32_t l, rid_dtype dtype,
                                  rid_mode mode, uint64_t seed, void* stream, int32_t nprobe, uint64_t probe_seed) {
  if (!plan) return RID_EINVAL;
  *plan = nullptr;
  if (nprobe < 0 || nprobe > RID_MAX_PROBES) return RID_EINVAL;
  rid_plan_t p = nullptr;
  const rid_status s = plan_create_impl(&p, m, n, k, l, dtype, mode, seed, stream, nprobe == 0);
  if (s != RID_OK) return s;
  if (nprobe > 0) {
    const rid_status t = set_probes_impl(p, nprobe, probe_seed, false);
    if (t != RID_OK) {
      rid_plan_destroy(p);
      return t;
    }
  }
  *plan = p;
  return RID_OK;
}

rid_status rid_sketch(rid_plan_t p, const void* A, int64_t lda, void* Y, int64_t ldy) {
  if (!p || !A || !Y || lda < p->m || ldy < p->l) return RID_EINVAL;
  if (!aligned16(Y) || ((uintptr_t)A & (p->dtype == RID_C128 ? 15u : 7u))) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  cudaError_t e;
  if (p->mode == RID_FP64_NATIVE)
    e = rid_launch_sketch_fp64(p, (const double2*)A, lda, (double2*)Y, ldy, 0, p->n);
  else
    e = rid_tc_sketch(p, A, lda, (double2*)Y, ldy);
  if (e == cudaSuccess && p->mode == RID_MIXED_BF16 && p->nrow > 0) e = rid_tc_probe_sketch(p, A, lda);
  if (e == cudaSuccess && p->nrow > 0) p->x_valid = 1;
  return from_cuda(e);
}

rid_status rid_sketch_cols(rid_plan_t p, const void* A, int64_t lda, void* Y, int64_t ldy, int64_t col0,
                           int64_t ncols) {
  if (!p || !A || !Y || lda < p->m || ldy < p->l) return RID_EINVAL;
  if (col0 < 0 || ncols < 0 || col0 + ncols > p->n || col0 % 128 != 0) return RID_EINVAL;
  if (ncols % 128 != 0 && col0 + ncols != p->n) return RID_EINVAL;
  if (!aligned16(Y) || ((uintptr_t)A & (p->dtype == RID_C128 ? 15u : 7u))) return RID_EINVAL;
  if (p->mode != RID_FP64_NATIVE && p->mode != RID_FP64_EMULATED && p->mode != RID_MIXED_BF16)
    return RID_EUNSUPPORTED;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  cudaError_t e;
  if (p->mode == RID_FP64_NATIVE) {
    e = rid_launch_sketch_fp64(p, (const double2*)A, lda, (double2*)Y, ldy, col0, ncols);
  } else if (p->mode == RID_MIXED_BF16) {
    e = rid_mx_sketch_cols(p, A, lda, (double2*)Y, ldy, col0, ncols);
    if (e == cudaSuccess && p->nrow > 0) e = rid_tc_probe_sketch_cols(p, A, lda, col0, ncols);
  } else {
    e = rid_tc_sketch_cols_fp64(p, A, lda, (double2*)Y, ldy, col0, ncols);
  }
  if (e == cudaSuccess && p->nrow > 0) p->x_valid = 1;
  return from_cuda(e);
}

rid_status rid_select(rid_plan_t p, void* Y, int64_t ldy, int32_t* perm) {
  if (!p || !Y || !perm || ldy < p->l) return RID_EINVAL;
  if (!aligned16(Y) || ((uintptr_t)perm & 3u)) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  return from_cuda(rid_launch_select(p, (double2*)Y, ldy, perm));
}

rid_status rid_solve(rid_plan_t p, const void* Y, int64_t ldy, void* T, int64_t ldt) {
  if (!p || !Y || ldy < p->l || ldt < p->k) return RID_EINVAL;
  if (p->n > p->k && !T) return RID_EINVAL;
  if (!aligned16(Y) || (T && !aligned16(T))) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  return from_cuda(rid_launch_solve(p, (const double2*)Y, ldy, (double2*)T, ldt));
}

rid_status rid_error(rid_plan_t p, const void* A, int64_t lda, const int32_t* perm, const void* T,
                     int64_t ldt, int32_t nprobe, uint64_t probe_seed, double out[2]) {
  if (!p || !A || !perm || !out || lda < p->m || ldt < p->k) return RID_EINVAL;
  if (p->n > p->k && !T) return RID_EINVAL;
  if (nprobe < 1 || nprobe > RID_MAX_PROBES) return RID_EINVAL;
  if (((uintptr_t)A & (p->dtype == RID_C128 ? 15u : 7u)) || (T && !aligned16(T))) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  cudaError_t e = rid_launch_error(p, A, lda, perm, (const double2*)T, ldt, nprobe, probe_seed);
  if (e != cudaSuccess) return from_cuda(e);
  double host[2];
  int status = 0;
  e = cudaMemcpyAsync(host, p->err_out, sizeof(host), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&status, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return from_cuda(e);
  out[0] = host[0];
  out[1] = host[1];
  if (p->mode != RID_FP64_NATIVE && rid_tc_error_word(p) != 0) return RID_ETIMEOUT;
  return status == RID_OK ? RID_OK : (rid_status)status;
}

rid_status rid_error_sketched(rid_plan_t p, const int32_t* perm, const void* T, int64_t ldt, double out[2]) {
  if (!p || !perm || !out || ldt < p->k) return RID_EINVAL;
  if (p->n > p->k && !T) return RID_EINVAL;
  if (p->nrow < 1 || !p->x_valid) return RID_EINVAL;
  if (((uintptr_t)perm & 3u) || (T && !aligned16(T))) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  cudaError_t e = rid_launch_error_sketched(p, perm, (const double2*)T, ldt);
  if (e != cudaSuccess) return from_cuda(e);
  double host[2];
  int status = 0;
  e = cudaMemcpyAsync(host, p->err_out, sizeof(host), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&status, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return from_cuda(e);
  out[0] = host[0];
  out[1] = host[1];
  if (p->mode != RID_FP64_NATIVE && rid_tc_error_word(p) != 0) return RID_ETIMEOUT;
  return status == RID_OK ? RID_OK : (rid_status)status;
}

rid_status rid_plan_set_select_grid(rid_plan_t p, int32_t ctas) {
  if (!p) return RID_EINVAL;
  if (ctas < 0) {
    p->sel_grid = p->sel_grid_max;
  } else if (ctas == 0) {
    p->sel_grid = 0;
  } else {
    if (p->sel_grid_max == 0) return RID_EUNSUPPORTED;      // no cooperative launch here
    p->sel_grid = ctas < p->sel_grid_max ? ctas : p->sel_grid_max;
  }
  return RID_OK;
}

rid_status rid_plan_stats(rid_plan_t p, int64_t out[8]) {
  if (!p || !out) return RID_EINVAL;
  // a mixed plan's row probes add their product and its reduction
  out[0] = p->mode == RID_FP64_NATIVE ? (p->split_k > 1 ? 2 : 1)
                                      : p->tc_sketch_launches + (p->tc_probe_state ? 2 : 0);
  out[1] = p->sel_grid > 0 ? 1 : 1 + p->k;           // one cooperative launch, or one per step
  out[2] = p->n > p->k ? 1 : 0;
  out[3] = p->n > p->k ? 6 : 5;
  out[4] = p->split_k;
  out[5] = (int64_t)(p->ws_bytes + p->tc_bytes + p->probe_bytes + p->tc_probe_bytes);
  out[6] = p->mode;
  out[7] = p->dtype;
  return RID_OK;
}

// The floor of the mixed-precision sketch (BF16x3 splits, FP32 sums over at
// most 2048 reals), on rho = the pivoted QR's estimate of sigma_{k+1}/sigma_1.
// Measured on complex64 matrices with a prescribed gap: the mixed ID's error
// equals the FP64 path's down to a gap of 1e-5 and is 1.17x it at 1e-6
// (rho = 1.07e-6); below that it stays near 3e-6 sigma_1 (5.6x the FP64
// path's error at a gap of 1e-7, where rho reads 7.3e-7).  The floor is set a
// factor 2 above that crossing.
constexpr double RID_MIXED_BF16_FLOOR = 2e-6;

rid_status rid_plan_accuracy(rid_plan_t p, const void* Y, int64_t ldy, double out[3]) {
  if (!p || !Y || !out || ldy < p->l) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  double h[2] = {0.0, 0.0};
  cudaError_t e = rid_launch_tail_ratio(p, (const double2*)Y, ldy, p->err_out);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, p->err_out, sizeof h, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return from_cuda(e);
  const double rho = h[0] > 0.0 ? h[1] / h[0] : 0.0;
  const double floor_ = p->mode == RID_MIXED_BF16 ? RID_MIXED_BF16_FLOOR : 0.0;
  out[0] = rho;
  out[1] = floor_;
  out[2] = rho >= floor_ ? 1.0 : 0.0;
  return RID_OK;
}

rid_status rid_plan_timing(rid_plan_t p, int32_t enable, double out[3]) {
  if (!p) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  if (out) {
    if (!p->timing) return RID_EINVAL;
    // first passes and products summed over the panels of the last sketch
    const int np = p->ev_panels > 0 ? p->ev_panels : 1;
    double sum[3] = {0.0, 0.0, 0.0};
    cudaError_t e = cudaEventSynchronize(p->ev[1 + 2 * np]);
    for (int i = 0; i < np && e == cudaSuccess; ++i) {
      float a = 0.f, b = 0.f;
      e = cudaEventElapsedTime(&a, p->ev[2 * i], p->ev[1 + 2 * i]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&b, p->ev[1 + 2 * i], p->ev[2 + 2 * i]);
      sum[0] += a;
      sum[1] += b;
    }
    float c = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&c, p->ev[2 * np], p->ev[1 + 2 * np]);
    if (e != cudaSuccess) return from_cuda(e);
    sum[2] = c;
    for (int i = 0; i < 3; ++i) out[i] = sum[i];
  }
  if (enable && !p->timing) {
    for (int i = 0; i < RID_TIMING_EVENTS; ++i)
      if (cudaEventCreate(&p->ev[i]) != cudaSuccess) return RID_ECUDA;
    p->timing = 1;
  }
  return RID_OK;
}

rid_status rid_sync_status(rid_plan_t p) {
  if (!p) return RID_EINVAL;
  DeviceGuard g(p->device);
  if (!g.ok) return RID_ECUDA;
  int status = 0;
  cudaError_t e = cudaMemcpyAsync(&status, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return from_cuda(e);
  if (p->mode != RID_FP64_NATIVE && rid_tc_error_word(p) != 0) return RID_ETIMEOUT;
  return (rid_status)status;
}

}  // extern "C"
