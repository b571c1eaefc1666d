/*
 * rid.h -- C ABI of the GB300 randomized interpolative decomposition (ID).
 *
 * Method (Lucas, Stalzer & Feo, "Parallel implementation of fast randomized
 * algorithms for the decomposition of low rank matrices", Sec. 2): an m x n
 * complex matrix A of approximate rank k is factored as A ~= B P, where
 * B = A(:, J) holds k columns of A and P = [I | T] Pi^T is k x n.  Four calls
 * make one ID, in the paper's order:
 *
 *   rid_sketch  Y = Omega A           randomization (Sec. 2; Gaussian Omega,
 *                                     the paper's "faster randomization")
 *   rid_select  Y Pi ~= Q [R1 | R2]   truncated QR with column pivoting (Sec. 2)
 *   rid_solve   R1 T = R2             the factorization of R (Sec. 2, Sec. 3.2)
 *   rid_error   ||A - B P||_2         error of the ID (Sec. 3.3, Table 5); or
 *               rid_error_sketched    the same from row probes that rid_sketch
 *                                     multiplied in its pass over A
 *
 * Conventions shared by every call:
 *   - Matrices are complex, interleaved (re, im), COLUMN-MAJOR with a leading
 *     dimension ld >= rows, except Omega, which is ROW-MAJOR (l x m, each row
 *     contiguous along m).  complex128 = two doubles, complex64 = two floats.
 *   - Unless a parameter says "host", pointers are DEVICE pointers owned by
 *     the caller, and must stay valid until the plan's stream has run the work.
 *   - Every call is asynchronous on the plan's stream, except rid_error and
 *     rid_sync_status, which synchronize it.
 *   - Argument errors are detected on the host before anything is launched
 *     and return RID_EINVAL (bad size, null pointer, ld too small) or
 *     RID_EUNSUPPORTED (dtype/mode combination not built); nothing is
 *     written then.  CUDA launch or allocation errors return RID_ECUDA /
 *     RID_ENOMEM.  Conditions found on the device (rank deficiency) are
 *     recorded in the plan's device status word and reported by
 *     rid_sync_status / rid_error.
 *   - A plan is not thread-safe; different plans are independent.
 */
#ifndef RID_H
#define RID_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RID_API __attribute__((visibility("default")))
#else
#define RID_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rid_plan_s* rid_plan_t;

typedef enum {
  RID_OK = 0,
  RID_EINVAL = 1,        /* bad argument (size, pointer, leading dimension) */
  RID_ENOMEM = 2,        /* device allocation failed */
  RID_ECUDA = 3,         /* a CUDA call or kernel launch failed */
  RID_ERANK = 4,         /* the sketch has rank < k (Sec. 2: redraw Omega, i.e. new seed) */
  RID_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
  RID_EUNSUPPORTED = 6   /* dtype / mode combination not available */
} rid_status;

typedef enum {
  RID_C128 = 0,          /* A is complex128 */
  RID_C64 = 1            /* A is complex64 (mixed-precision sketch) */
} rid_dtype;

typedef enum {
  RID_FP64_NATIVE = 0,   /* sketch with FP64 FMA on the CUDA cores */
  RID_FP64_EMULATED = 1, /* sketch on tcgen05 tensor cores with exact BF16 slices, FP64-grade result */
  RID_MIXED_BF16 = 2,    /* complex64 A: sketch from 3 BF16 slices, FP32 accumulation */
  RID_MIXED_3XTF32 = 3   /* complex64 A: sketch from 3xTF32 splits, FP32 accumulation */
} rid_mode;

/* Create a plan for IDs of m x n matrices of rank k with an l x m test matrix.
 *   Requires 1 <= k <= min(m, n, l); l >= k (Sec. 2: "l >= k"; the paper
 *   uses l = 2k, the configurations here use l = k + p).
 *   seed selects the Gaussian test matrix Omega: entry (i, j) is drawn from
 *   Philox4x32-10 (Salmon et al., SC 2011) at counter (j mod 2^32, j div 2^32,
 *   i, 3) under key (seed mod 2^32, seed div 2^32), then Box-Muller,
 *   rho = sqrt(-log u1), Omega_ij = rho exp(2 pi i u2), so re and im are
 *   iid N(0, 1/2).  u1, u2 are 53-bit uniforms built from the four words.
 *   stream is a cudaStream_t (NULL = legacy default stream) on which every
 *   call of this plan runs.
 *   The plan allocates and owns Omega (l x m, row-major) and its workspace on
 *   the current device; Omega is generated on the stream before return. */
RID_API rid_status rid_plan_create(rid_plan_t* plan, int64_t m, int64_t n, int32_t k, int32_t l,
                           rid_dtype dtype, rid_mode mode, uint64_t seed, void* stream);

/* Device bytes rid_plan_create would allocate for these arguments (Omega, its
 * split forms and every workspace), computed without allocating anything:
 * what a server admitting requests by HBM footprint needs.  Same argument
 * checks and return codes as rid_plan_create. */
RID_API rid_status rid_plan_footprint(int64_t m, int64_t n, int32_t k, int32_t l, rid_dtype dtype, rid_mode mode,
                                      size_t* bytes);

/* Free the plan's device memory (synchronizes its stream first).  NULL is a no-op. */
RID_API rid_status rid_plan_destroy(rid_plan_t plan);

/* Device pointer to the plan's Omega (complex128, l x m row-major) and its
 * row stride ldo (elements).  Read-only for the caller. */
RID_API rid_status rid_plan_omega(rid_plan_t plan, const void** omega, int64_t* ldo);

/* Replace the plan's Omega by a caller-supplied l x m complex128 row-major
 * device matrix with row stride ldo >= m (copied on the stream). */
RID_API rid_status rid_plan_set_omega(rid_plan_t plan, const void* omega, int64_t ldo);

/* Replace the plan's Omega by the paper's own randomization (Sec. 2, "Y = S F D A"):
 * row q of S F D, Omega(q, j) = exp(-2 pi i s_q j / m) exp(2 pi i phi_j), with
 * D = diag(exp(2 pi i phi_j)) random phases (phi_j uniform on [0, 1)), F the
 * m x m DFT (0-based, F_jk = exp(-2 pi i j k / m)) and S sampling rows
 * s_q uniform on {0..m-1}.  phi_j = u2 of the Philox4x32-10 block at counter
 * (j mod 2^32, j div 2^32, 0, 5), s_q = floor(m u2) of the block at counter
 * (q, 0, 1, 5), key = srft_seed.  Generated on the plan's stream.  The
 * subsampled DFT is applied as this dense l x m matrix by rid_sketch. */
RID_API rid_status rid_plan_use_srft(rid_plan_t plan, uint64_t srft_seed);

/* Randomization, Sec. 2:  Y = Omega A.
 *   A: m x n, column-major, leading dimension lda >= m, dtype of the plan.
 *   Y: l x n complex128 output, column-major, ldy >= l.  Fully overwritten.
 *   A is read once per l-tile; the result is deterministic (fixed reduction order). */
RID_API rid_status rid_sketch(rid_plan_t plan, const void* A, int64_t lda, void* Y, int64_t ldy);

/* Truncated QR with column pivoting of Y (Sec. 2, "Y ~= Q R"; the permutation
 * the paper asks for is chosen by Businger-Golub pivoting):
 *   k steps; at step j the pivot is the column of largest remaining norm
 *   sum_{i>=j} |Y_ic|^2 (recomputed exactly, ties to the lowest index); the
 *   reflector follows LAPACK zlarfg (real beta, H = I - tau v v^H).
 *   Y (in/out, l x n complex128, ldy >= l): on return rows 0..k-1 hold
 *   [R1 | R2] in pivoted column order, Householder vectors below the diagonal.
 *   perm (out, int32[n]): perm[c] = original column of pivoted column c,
 *   so J = perm[0..k-1] and B = A(:, J).
 *   If the sketch has rank < k (a pivot norm is exactly zero) the status word
 *   becomes RID_ERANK and later steps of this call are skipped. */
RID_API rid_status rid_select(rid_plan_t plan, void* Y, int64_t ldy, int32_t* perm);

/* Launch shape of rid_select.  The results are bitwise the same for every
 * shape: each column's arithmetic, the pivot rule and the reflector do not
 * depend on which CTA or warp handles a column.
 *   ctas > 0: all k steps in one cooperative launch of min(ctas, the plan's
 *   default) CTAs, each step ending in a grid barrier;
 *   ctas == 0: one launch per step, and no CTA ever waits on another, so
 *   kernels of other streams can share the GPU with it;
 *   ctas < 0: back to the plan's default, chosen at rid_plan_create, where
 *   the device supports cooperative launch: for l <= 256, when Y's columns
 *   fit in the shared memory of one CTA per SM, one cooperative launch that
 *   keeps them there for all k steps (no column crosses L2 between steps);
 *   otherwise one cooperative launch of as many CTAs as the GPU holds at
 *   once, but no more than one per 16 columns.  Without cooperative launch:
 *   one launch per step.
 * RID_EINVAL for a null plan; RID_EUNSUPPORTED for ctas > 0 when the device
 * has no cooperative launch.  No device work; takes effect at the next
 * rid_select. */
RID_API rid_status rid_plan_set_select_grid(rid_plan_t plan, int32_t ctas);

/* Factorization of R, Sec. 2 "R2 = R1 T":  T = R1^-1 R2 by back substitution,
 * every right-hand side column independent (Sec. 3.2).
 *   Y: the output of rid_select (R1 = Y[0:k, 0:k] upper triangular,
 *   R2 = Y[0:k, k:n]).  T: k x (n-k) complex128 output, column-major,
 *   ldt >= k; column i of T belongs to original column perm[k+i], so
 *   P(:, perm[j]) = e_j (j < k) and P(:, perm[k+i]) = T(:, i).  n == k is
 *   allowed (T is empty). */
RID_API rid_status rid_solve(rid_plan_t plan, const void* Y, int64_t ldy, void* T, int64_t ldt);

/* Error of the ID (Sec. 3.3, Table 5 reports ||A - B P||_2), by Gaussian probes:
 * for r = nprobe columns w_q of an n x r complex Gaussian matrix (Philox
 * counter (q, 0, c, 4) for row c, key = probe_seed, Box-Muller as for Omega),
 * E w = A w~ with w~(Jc) = w(Jc), w~(J) = -T w(Jc), in one pass over A.
 *   out (HOST, double[2]): out[0] = max_q ||E w_q|| / ||w_q|| (never above
 *   ||E||_2); out[1] = 10 sqrt(2/pi) max_q ||E w_q||, an upper bound on
 *   ||E||_2 with probability >= 1 - 10^-r (Halko, Martinsson & Tropp 2011,
 *   Lemma 4.1).  1 <= nprobe <= 16.  Synchronizes the stream; returns
 *   RID_ERANK if the last rid_select found a rank-deficient sketch. */
RID_API rid_status rid_error(rid_plan_t plan, const void* A, int64_t lda, const int32_t* perm,
                     const void* T, int64_t ldt, int32_t nprobe, uint64_t probe_seed,
                     double out[2]);

/* Round the test matrix: every entry of each row of Omega (and of the row
 * probes, if set) is rounded to `bits` bits below the row's largest entry:
 * with E_r the exponent of the row (|Re w|, |Im w| < 2^E_r, E_r the exponent
 * of x = f 2^E_r, 1/2 <= |f| < 1), each real part becomes the nearest
 * multiple of 2^(E_r - bits), ties to even (a value that would reach
 * +-2^E_r takes the multiple below it).  Omega stays a seeded random test
 * matrix (Sec. 2 only needs one; the paper's own is the SRFT); rounded, it
 * holds bits / 8 base-256 digits, and RID_FP64_EMULATED multiplies only
 * those: 28 digit-pair products become 18 at bits = 24 and 13 at 16, with the
 * product still exact for that Omega.  bits in {8, 16, ..., 48}
 * (RID_EINVAL otherwise).  Later rid_plan_use_srft / rid_plan_set_probes
 * round the rows they draw the same way; rid_plan_set_omega takes the
 * caller's Omega unrounded and ends the rounding.  Synchronizes the stream. */
RID_API rid_status rid_plan_round_omega(rid_plan_t plan, int32_t bits);

/* The sketch of a column range: Y(:, c) = Omega A(:, c) (and X(:, c) = G A(:, c)
 * for the row probes) for c = col0 .. col0 + ncols - 1, so that a caller can
 * sketch A panel by panel as its columns reach the device (a host->device
 * copy of the next panel overlaps the sketch of this one).  A and Y point to
 * column 0 of the whole matrices as for rid_sketch; col0 a multiple of 128,
 * ncols a multiple of 128 unless the range ends at column n (RID_EINVAL
 * otherwise).  Each column's arithmetic is the same as in rid_sketch, so
 * covering all columns once, in any ranges, gives rid_sketch's Y and X bit for
 * bit.  Modes RID_FP64_NATIVE, RID_FP64_EMULATED and RID_MIXED_BF16
 * (RID_EUNSUPPORTED otherwise).  Ranges of one plan are sketched in stream
 * order; the row-probe error may follow once every column has been sketched. */
RID_API rid_status rid_sketch_cols(rid_plan_t plan, const void* A, int64_t lda, void* Y, int64_t ldy,
                                   int64_t col0, int64_t ncols);

/* Row probes for the error of the ID (Sec. 3.3), computed in the sketch's
 * own pass over A.  Appends nprobe rows g_q to Omega: an nprobe x m complex
 * Gaussian G, entry (q, i) from the Philox block at counter (i lo, i hi, q, 6)
 * with key = probe_seed and Box-Muller as for Omega, independent of Omega.
 * Every later rid_sketch also computes X = G A (nprobe x n, plan memory) in
 * the same pass as Y = Omega A; Y is unchanged.  nprobe = 0 removes them.
 *   1 <= nprobe <= 16 and l + nprobe <= 512 (RID_EINVAL / RID_EUNSUPPORTED).
 *   X is FP64-grade in every mode: RID_MIXED_BF16 plans multiply the probe
 *   rows by the complex64 A with the exact-slice emulation of the
 *   FP64-emulated mode (in a kernel of their own that cuts A's digits in
 *   shared memory) while Y takes the BF16x3 product, so their error estimate
 *   stays FP64.
 *   Allocates (l + nprobe) x m complex128 for Omega and G plus small buffers
 *   (RID_ENOMEM if that fails; the plan is then unchanged) and synchronizes
 *   the stream.  rid_plan_omega still returns the l rows of the test matrix. */
RID_API rid_status rid_plan_set_probes(rid_plan_t plan, int32_t nprobe, uint64_t probe_seed);

/* Device pointer to the row probes' products X = G A of the last sketch
 * (Sec. 3.3: the estimate is formed from them): nprobe x n complex128,
 * column-major with leading dimension *ldx = nprobe, in plan memory and
 * overwritten by the next sketch.  Read-only for the caller; read it in the
 * plan's stream order.  RID_EINVAL without probes or before a sketch since
 * they were set. */
RID_API rid_status rid_plan_probe_products(rid_plan_t plan, const void** X, int64_t* ldx);

/* rid_plan_create and rid_plan_set_probes(plan, nprobe, probe_seed) in one
 * call: the plan is built with its nprobe row probes (0 <= nprobe <= 16) from
 * the start, so the tensor-core modes cut the digits of the test matrix and
 * the probe rows once, and nothing synchronizes (all work is ordered on
 * stream).  The results are those of the two calls.  Errors as for
 * rid_plan_create and rid_plan_set_probes; *plan is NULL on failure. */
RID_API rid_status rid_plan_create_probes(rid_plan_t* plan, int64_t m, int64_t n, int32_t k, int32_t l,
                                          rid_dtype dtype, rid_mode mode, uint64_t seed, void* stream,
                                          int32_t nprobe, uint64_t probe_seed);

/* Reuse a plan for another ID of the same shape: redraw its test matrix for
 * seed (and, if it has row probes, the probes for probe_seed) in place and
 * re-cut their digits, as rid_plan_create_probes with these seeds would;
 * nothing is allocated.  Later calls give the bits of a new plan with these
 * seeds.  Asynchronous on the plan's stream.  RID_EUNSUPPORTED for a plan
 * whose Omega was replaced or rounded (rid_plan_set_omega, rid_plan_use_srft,
 * rid_plan_round_omega) and for the mixed-precision modes. */
RID_API rid_status rid_plan_reseed(rid_plan_t plan, uint64_t seed, uint64_t probe_seed);

/* Move a plan's later work to stream (a cudaStream_t of the plan's device):
 * the new stream first waits for everything already queued for the plan on
 * its old stream.  No device work of its own. */
RID_API rid_status rid_plan_set_stream(rid_plan_t plan, void* stream);

/* Error of the ID from the row probes of the last rid_sketch, without reading
 * A.  E = A - A(:, J) P has E(:, J) = 0 and E(:, perm[k+i]) =
 * A(:, perm[k+i]) - A(:, J) T(:, i), so
 *   (g_q E)(perm[k+i]) = X(q, perm[k+i]) - sum_a X(q, perm[a]) T(a, i).
 *   out (HOST, double[2]): out[0] = max_q ||g_q E|| / ||g_q|| (never above
 *   ||E||_2); out[1] = 10 sqrt(2/pi) max_q ||g_q E||, an upper bound on
 *   ||E||_2 with probability >= 1 - 10^-r (Halko, Martinsson & Tropp 2011,
 *   Lemma 4.1, applied to E^T, whose 2-norm is that of E).
 *   perm, T: the outputs of rid_select and rid_solve for the Y of that
 *   rid_sketch (T may be null when n == k).  RID_EINVAL if no row probes are
 *   set or no rid_sketch ran since they were set.  Synchronizes the stream;
 *   returns RID_ERANK if the last rid_select found a rank-deficient sketch. */
RID_API rid_status rid_error_sketched(rid_plan_t plan, const int32_t* perm, const void* T, int64_t ldt,
                                      double out[2]);

/* Synchronize the plan's stream and return the device status word
 * (RID_OK or RID_ERANK), or RID_ECUDA if the stream reported an error. */
RID_API rid_status rid_sync_status(rid_plan_t plan);

/* Plan facts for callers that account for work (no device work, no sync):
 *   out[0] = kernel launches of one rid_sketch     out[1] = of one rid_select
 *   out[2] = of one rid_solve                      out[3] = of one rid_error
 *   out[4] = K-splits of the sketch                out[5] = device bytes the plan owns
 *   out[6] = mode (rid_mode)                       out[7] = dtype (rid_dtype) */
RID_API rid_status rid_plan_stats(rid_plan_t plan, int64_t out[8]);

/* Per-kernel device time of this plan's rid_sketch, for performance accounting.
 *   enable != 0 creates CUDA events (once) and from then on every rid_sketch
 *   records them on the plan's stream around its kernels.  If out (HOST,
 *   double[3]) is not NULL, waits for the last rid_sketch and returns its
 *   times in ms: out[0] = digit slicing of A (0 in the native mode),
 *   out[1] = the product kernel, out[2] = the split-K reduction.  In the
 *   FP64-emulated mode a wide A is sliced and multiplied in up to four
 *   column panels (the plan's digit tiles hold one panel); out[0] and out[1]
 *   are then the sums over the panels.
 *   RID_EINVAL if out is given before timing was enabled. */
RID_API rid_status rid_plan_timing(rid_plan_t plan, int32_t enable, double out[3]);

/* The sketch's accuracy against the plan's mode, read after rid_select.  The
 * ID's error is governed by sigma_{k+1} (Sec. 2, Eq. 1); a sketch computed in
 * low precision resolves only a spectrum that decays less than its own noise.
 *   Y: the rid_select output of this plan (DEVICE, l x n, ldy >= l): R in rows
 *   0..k-1, and in rows k..l-1 of columns k..n-1 what the k reflectors left.
 *   out (HOST, double[3]):
 *     out[0] = rho = max_{c >= k} ||Y(k:l-1, c)|| / |R(0, 0)|, the largest
 *              remaining column norm of the pivoted QR relative to the first
 *              pivot (the pivoted QR's estimate of sigma_{k+1} / sigma_1 of
 *              the sketch; 0 when k = n or k = l);
 *     out[1] = the floor of the plan's mode: rho above which that mode was
 *              measured to return the FP64 path's J and an ID error within
 *              twice the FP64 path's (0 for the FP64 modes; 2e-6 for
 *              RID_MIXED_BF16);
 *     out[2] = 1.0 if rho >= out[1] (the result is accepted), else 0.0: the
 *              spectrum decays below what the mode resolves, and the ID should
 *              be recomputed in an FP64 mode.
 *   Synchronizes the stream.  RID_EINVAL for a null plan, Y or out, or
 *   ldy < l. */
RID_API rid_status rid_plan_accuracy(rid_plan_t plan, const void* Y, int64_t ldy, double out[3]);

/* Allocation-free pivoted QR (the paper has no counterpart: this is a service
 * for callers that cannot call cudaMalloc, e.g. code running under another
 * allocator's lock, or real-time loops that forbid allocation after start-up).
 * Same computation and results as rid_select, without a plan:
 *   Y (in/out, l x n complex128, column-major, ldy >= l), perm (out, int32[n]),
 *   status (out, DEVICE int32: RID_OK, or RID_ERANK if the sketch has rank < k),
 *   stream: cudaStream_t (NULL = legacy default stream).  Asynchronous.
 *   Scratch: a fixed 20736-byte array inside this library (per device, held
 *   until the process exits); nothing is allocated.  Limits: 1 <= k <= l <= 512,
 *   k <= n; larger sizes return RID_EINVAL before any work.
 *   All calls share the scratch array: calls whose work overlaps on the GPU
 *   (other streams, other host threads) race; calls on one stream are safe.
 *   The first call on a device looks up the array's device address; make that
 *   first call before any stream capture. */
RID_API rid_status rid_select_noalloc(void* Y, int64_t ldy, int32_t l, int64_t n, int32_t k,
                                      int32_t* perm, int32_t* status, void* stream);

/* Self-test of the bounded waits every kernel relies on (a failure detector
 * that needs no GPU fault): on `stream`, one launch waits on an mbarrier that
 * nothing completes (budget about 1 ms) and on a grid barrier that one CTA
 * more than the grid must reach (budget about 10 ms).  Each gives up and
 * records its status: out[0] (the mbarrier) and out[1] (the grid barrier)
 * are RID_ETIMEOUT when the waits end as designed.  Synchronizes the stream;
 * the context stays usable.  RID_EINVAL for a null out. */
RID_API rid_status rid_selftest_timeouts(void* stream, int32_t out[2]);

/* ---- Batched IDs -------------------------------------------------------------------
 * Many independent complex128 IDs of uneven sizes (e.g. the blocks of a
 * hierarchical-matrix compressor) in one persistent launch.  Each problem is
 * the whole four-step ID of Sec. 2 / Sec. 3.3 with the plan's conventions:
 * Omega from `seed` exactly as rid_plan_create draws it, Householder QR with
 * column pivoting, back substitution, probe error estimate; FP64 arithmetic. */
typedef struct {
  int64_t m, n;          /* A is m x n */
  int32_t k, l;          /* 1 <= k <= min(m, n), k <= l <= 128, k <= 64, n <= 4096 */
  const void* A;         /* device, complex128, column-major, lda >= m */
  int64_t lda;
  void* Y;               /* device, l x n complex128 (ldy >= l): the sketch, then R (like rid_select) */
  int64_t ldy;
  int32_t* perm;         /* device, int32[n]: J = perm[0..k-1] */
  void* T;               /* device, k x (n-k) complex128 (ldt >= k); NULL allowed when n == k */
  int64_t ldt;
  uint64_t seed;         /* Omega of this problem */
} rid_batch_item;

/* Device workspace bytes rid_batch_run needs for `count` problems. */
RID_API rid_status rid_batch_workspace(int32_t count, size_t* bytes);

/* Run `count` IDs (items: HOST array) on `stream`.  err_out (device,
 * double[2 count]) receives each problem's (est, upper) as rid_error returns
 * them; status_out (device, int32[count]) RID_OK or RID_ERANK per problem
 * (est = upper = -1 then).  tile = 16 or 32: the sketch's column tile (pick
 * with an autotuner; results do not depend on it).  workspace: device,
 * >= rid_batch_workspace bytes.  Returns RID_EINVAL / RID_EUNSUPPORTED for
 * sizes beyond the limits above before anything is launched; synchronizes the
 * stream once to stage the descriptors, then runs asynchronously. */
RID_API rid_status rid_batch_run(const rid_batch_item* items, int32_t count, int32_t nprobe, uint64_t probe_seed,
                                 int32_t tile, double* err_out, int32_t* status_out, void* workspace,
                                 size_t ws_bytes, void* stream);

/* The two halves of rid_batch_run, for callers that run one batch many
 * times or capture it in a CUDA graph:
 *   rid_batch_prepare checks the items (RID_EINVAL / RID_EUNSUPPORTED as
 *   rid_batch_run), orders them by cost (largest first) and stages their
 *   descriptors in `workspace`; it synchronizes the stream once.
 *   rid_batch_launch then runs the prepared batch: one memset of the work
 *   queue and one persistent kernel launch on `stream`, nothing else (no host
 *   copies, no synchronization), so it can be captured in a CUDA graph and
 *   replayed.  count and nprobe must match the prepare call; the pointers of
 *   the items (A, Y, perm, T) must stay valid while launches may run. */
RID_API rid_status rid_batch_prepare(const rid_batch_item* items, int32_t count, int32_t nprobe, void* workspace,
                                     size_t ws_bytes, void* stream);
RID_API rid_status rid_batch_launch(int32_t count, int32_t nprobe, uint64_t probe_seed, int32_t tile,
                                    double* err_out, int32_t* status_out, void* workspace, void* stream);

/* Batches on the tensor cores (Sec. 2 sketch, Sec. 3.3 row-probe error, for
 * many problems at once).  rid_batch_tc_create draws every problem's Omega
 * (from its seed, exactly as rid_plan_create does) and nprobe row probes
 * (probe_seed, as rid_plan_set_probes), then records, once, a CUDA graph of
 * two persistent launches:
 *   1. one cooperative tensor-core launch computes every problem's sketch
 *      Y = Omega A and X = G A with the FP64-emulated product (the problems,
 *      largest first, in waves whose digit tiles fit a workspace buffer; per
 *      wave all CTAs cut the digits, meet at a grid barrier, then multiply
 *      their longest-first work lists of (problem, N-tile, column block,
 *      K-split) items);
 *   2. one launch runs the pivoted QR, the solve and the row-probe error (as
 *      rid_error_sketched) of every problem, writing err_out (device,
 *      double[2 count]) and status_out (device, int32[count]) as
 *      rid_batch_run does; a problem whose sketch launch gave up a bounded
 *      wait gets RID_ETIMEOUT and est = upper = -1.
 * Items and their limits as for rid_batch_run; A, Y and T 16-byte aligned.
 * The items' pointers and err_out / status_out must stay valid for the
 * handle's life.  Device memory: each problem's Omega and probe rows (16 (l +
 * nprobe) m bytes), X, and two digit buffers of at most 2 GiB each (or of
 * the largest problem's digit tiles, about 14 (2 (l + nprobe) + n) 2m bytes,
 * if larger); rid_batch_tc_info reports the total.  Creating synchronizes `stream`; rid_batch_tc_run
 * launches the graph on `stream` (asynchronous).  With one K-split (the
 * default) a problem's Y has the bits of its own FP64-emulated plan's sketch,
 * so J and T equal that plan's up to the rounding order of the QR. */
typedef struct rid_batch_plan_s* rid_batch_plan_t;
RID_API rid_status rid_batch_tc_create(rid_batch_plan_t* plan, const rid_batch_item* items, int32_t count,
                                       int32_t nprobe, uint64_t probe_seed, double* err_out, int32_t* status_out,
                                       void* stream);
/* The same with the tile shapes chosen per problem (an autotuner's choice):
 * tile_n[i] (HOST, may be NULL) the widest N-tile of problem i in rows of the
 * real test matrix (16 .. 128, a multiple of 16; 0: 128), ksplit[i] (HOST,
 * may be NULL) its K-splits (0 or 1: none; larger values are capped at the
 * number of 256-real chunks; partial sums are then added in split order, so
 * Y differs from a plan's in the last bits), wave_bytes the digit buffer
 * size (0: 2 GiB).  RID_EINVAL for a tile_n outside those values. */
RID_API rid_status rid_batch_tc_create_tuned(rid_batch_plan_t* plan, const rid_batch_item* items, int32_t count,
                                             int32_t nprobe, uint64_t probe_seed, double* err_out,
                                             int32_t* status_out, const int32_t* tile_n, const int32_t* ksplit,
                                             size_t wave_bytes, void* stream);
RID_API rid_status rid_batch_tc_run(rid_batch_plan_t plan, void* stream);
/* Milliseconds of the last run: out[0] the sketch launch, out[1] the
 * finishing launch (HOST double[2]); waits for that run to end. */
RID_API rid_status rid_batch_tc_times(rid_batch_plan_t plan, double out[2]);
/* out (HOST double[4]): device bytes the handle holds, waves, work items of
 * the sketch launch, its CTAs. */
RID_API rid_status rid_batch_tc_info(rid_batch_plan_t plan, double out[4]);
RID_API rid_status rid_batch_tc_destroy(rid_batch_plan_t plan);

/* Static, human-readable name of a status code. */
RID_API const char* rid_status_string(rid_status status);

#ifdef __cplusplus
}
#endif

#endif /* RID_H */
