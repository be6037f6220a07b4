/*
 * libpcwave — wavelet-domain matrix of a product-convolution operator on one GB300.
 *
 * Escande & Weiss, "Fast wavelet decomposition of linear operators through
 * product-convolution expansions".  The operator (Eq. (2), Section 1) is
 *     H f = sum_{k=1..m} u_k * (v_k . f)          (PC_ORDER_MULT_THEN_CONV, the paper's)
 * or  H f = sum_{k=1..m} v_k . (u_k * f)          (PC_ORDER_CONV_THEN_MULT)
 * on periodic 1-D signals or 2-D images of side n, and the library assembles
 *     Theta = Psi^* H Psi,   Theta[mu, lambda] = <psi_mu, H psi_lambda>      (Section 3.2)
 * in an orthonormal periodic Daubechies or Symmlet basis (Section 2), keeping only the entries of a
 * prescribed pattern: | |mu| - |lambda| | <= gap (the band rule (i) of Remark 5.3) and, on
 * each axis, supp psi_lambda within distance r (the kernel radius) of supp psi_mu on the
 * torus (the support test of Section 5.2; entries failing it are exactly zero).
 *
 * Conventions.
 *   - Pixels are row-major (axis 0 slow).  Levels j = 1 (finest) .. L (coarsest).
 *   - Coefficient order ("canonical"): approximation band (level L) first, then levels
 *     L..1, within a level bands e = (0,1), (1,0), (1,1) (e0 on axis 0), translates
 *     row-major.  mu indexes rows (output), lambda columns (input): y = Theta x maps the
 *     input's coefficients to the output's.
 *   - Kernels u_k are (2r+1)^d stencils, row-major, centre index = offset 0:
 *     (u * f)(y) = sum_t u(t) f(y - t).  Windows v_k are n^d pixels.
 *   - Filters: low-pass h with 2*delta taps on [0, 2 delta - 1], sum sqrt(2) -- Daubechies'
 *     minimum-phase factor or the least-asymmetric (Symmlet) one, see pc_filter_taps;
 *     g[i] = (-1)^(1-i) h[1-i] (Section 2.1).
 *
 * Storage of Theta ("stencil-ELL").  Rows of the stored matrix S are the filtered-side
 * elements: S = Theta in the paper's order, S = Theta^T in the convolution-first order.
 * Row s holds one block per kept column band, bands in canonical order; a block is the
 * W0 x W1 run of kept translates (row-major), so column indices are implicit.
 *
 * Threading and streams.  Every call that takes a `stream` (a cudaStream_t, NULL = legacy
 * default stream) is stream-ordered and asynchronous unless stated otherwise.  A handle
 * must not be used from two host threads at once.  Errors are returned as pc_status codes,
 * never thrown; pc_last_error() gives a message.  Faults detected inside kernels (an index
 * outside a buffer, a work queue that overran) set a device flag read by pc_sync().
 *
 * Ownership.  The handle owns the device buffers it allocates (Theta, filtered wavelets,
 * plans, scratch, and the solver's transposed copy and vectors once a solver call ran).  The
 * caller owns every pointer it passes (inputs, x, y, dtheta, du, dv, z0, w, sigma, z).
 */
#ifndef PCWAVE_H
#define PCWAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pc_op* pc_handle;

typedef enum {
    PC_OK = 0,
    PC_ERR_INVALID_ARG = 1,   /* a size, pointer or flag is outside what the call accepts */
    PC_ERR_UNSUPPORTED = 2,   /* valid but not handled (e.g. m > 256 terms) */
    PC_ERR_OOM = 3,           /* a device allocation failed */
    PC_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    PC_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    PC_ERR_NOT_ASSEMBLED = 6, /* Theta is needed but pc_assemble has not run */
    PC_ERR_DEVICE = 7         /* a kernel flagged an internal fault (see pc_last_error) */
} pc_status;

typedef enum { PC_ORDER_MULT_THEN_CONV = 0, PC_ORDER_CONV_THEN_MULT = 1 } pc_order;
typedef enum { PC_FP32 = 0, PC_FP64 = 1 } pc_precision;
/* Wavelet family (Section 2.1 filter banks; the experiments of Section 4.3 use Symmlets):
 * both have 2*delta taps on [0, 2 delta - 1] and delta vanishing moments. */
typedef enum { PC_DAUBECHIES = 0, PC_SYMMLET = 1 } pc_family;

typedef struct {
    int dim;       /* 1 or 2 */
    int n;         /* side of the periodic grid, a power of two >= 2 */
    int levels;    /* L >= 1 with n >> L >= 1 (the paper's J when L = log2 n) */
    int delta;     /* filter order (vanishing moments), 1..10; 2*delta taps (db2 = 2, db4 = 4, sym6 = 6) */
    int m;         /* number of product-convolution terms, 1..256 */
    int radius;    /* kernel radius r >= 0: kernels are (2r+1)^dim */
    int gap;       /* band rule: keep | |mu| - |lambda| | <= gap; -1 keeps every entry (dense) */
    int order;     /* pc_order */
    int precision; /* PC_FP32: FP32 arithmetic, compensated (Kahan) sum over k, FP32 Theta;
                      PC_FP64: FP64 arithmetic and FP64 Theta (the plain baseline) */
    int store_bf16;/* PC_FP32 only: also keep a BF16 copy of Theta, used by pc_apply */
    int family;    /* pc_family: PC_DAUBECHIES (minimum phase; a zeroed descriptor) or
                      PC_SYMMLET (least-asymmetric factor of the same |m0|^2) */
} pc_desc;

/* ---------------------------------------------------------------------------------------
 * Host-only planning (no GPU needed).  Validate a descriptor and size the pattern.
 * --------------------------------------------------------------------------------------- */

/* Validates desc.  Returns PC_OK or PC_ERR_INVALID_ARG / PC_ERR_UNSUPPORTED. */
pc_status pc_plan_check(const pc_desc* desc);

/* Total number of stored entries (nnz of the pattern).  Host only. */
pc_status pc_plan_nnz(const pc_desc* desc, int64_t* nnz);

/* Column indices (canonical, of the STORED matrix S) of stored row `row`, in storage order.
 * cols may be NULL to query the count only; otherwise it must hold *count entries
 * (query first).  Host only. */
pc_status pc_plan_row(const pc_desc* desc, int64_t row, int64_t* cols, int64_t* count);

/* Host only: the low-pass taps h[0 .. 2 delta - 1] (FP64, sum sqrt 2) the library uses for a
 * family and order.  Daubechies: the minimum-phase spectral factor of |m0(w)|^2 =
 * cos^(2 delta)(w/2) P(sin^2(w/2)) (Section 2.1).  Symmlet: of the real spectral factors (z_i
 * or 1/z_i per root of P, conjugate roots alike), the one whose phase of prod (e^{-iw} - z_i)
 * has the smallest mean squared residual from its least-squares line on w_k = (k + 1/2) pi /
 * 512, k < 512; a tie with the mirror filter goes to the smaller energy centre sum n h[n]^2.
 * h: caller-owned, 2 delta doubles.  PC_ERR_INVALID_ARG for NULL h, delta outside 1..10 or an
 * unknown family. */
pc_status pc_filter_taps(int family, int delta, double* h);

/* ---------------------------------------------------------------------------------------
 * Operator lifetime.
 * --------------------------------------------------------------------------------------- */

/* Creates an operator.  u: m x (2r+1)^dim kernels, v: m x n^dim windows, both of the
 * precision's type (float for PC_FP32, double for PC_FP64), host or device memory (detected);
 * both are copied.  Computes the FP64 filter taps, plans the pattern (row offsets) and
 * allocates Theta and, for 2-D operators, the s scratch (one value per region pixel of every
 * stored row: step 3 below writes it, pc_backward reuses it).  Synchronous with respect to the
 * host for planning and allocation; the copies of u and v are ordered on `stream`. */
pc_status pc_create(const pc_desc* desc, const void* u, const void* v, void* stream,
                    pc_handle* out);

/* Replaces the kernels and windows (same shapes and type as pc_create); either may be NULL
 * to keep the current one.  Theta is stale until the next pc_assemble.  When v is given the
 * call rebuilds the per-pixel lists of nonzero windows and synchronises `stream` (it reads
 * back the largest number of nonzero windows at one pixel). */
pc_status pc_set_params(pc_handle h, const void* u, const void* v, void* stream);

/* Frees everything the handle owns.  Synchronises the device first. */
void pc_destroy(pc_handle h);

/* ---------------------------------------------------------------------------------------
 * The hot path.
 * --------------------------------------------------------------------------------------- */

/* Assembles Theta restricted to the pattern (Section 3.2, Algorithm 1 without thresholding:
 * the exact sum_k A_k B_k on the pattern):
 *   1. base wavelets phi_{j,0}, psi_{j,0} by the FP64 cascade of the taps (Section 2.1);
 *   2. filtered base wavelets F_{k,beta} = kappa_k * rho_beta (kappa_k = u_k flipped in the
 *      paper's order, u_k otherwise): the circulant generators of A_k (Lemma 5.1);
 *   3. for every stored row s: the window-weighted sum sum_k v_k . F_{k,beta}(. - shift)
 *      over the row's support (compensated over k in FP32), then a localized forward wavelet
 *      transform of it (Lemma 5.5) whose kept coefficients are the row's entries.
 * Asynchronous on `stream`. */
pc_status pc_assemble(pc_handle h, void* stream);

/* y = Theta x for nrhs right-hand sides (Section 4.3 uses two such products per FISTA
 * iteration).  x: N x nrhs, element (i, c) at x[i*ldx + c] (ldx >= nrhs), FP32, device;
 * y likewise (ldy >= nrhs), overwritten.  Reads the BF16 copy when store_bf16 is set, else
 * the FP32 (or FP64) values; accumulates in FP32 (FP64 for PC_FP64 handles, where x and y
 * are double).  1 <= nrhs <= 64.  Returns PC_ERR_NOT_ASSEMBLED before the first assembly. */
pc_status pc_apply(pc_handle h, const void* x, void* y, int nrhs, int ldx, int ldy,
                   void* stream);

/* y = Theta^T x: the adjoint product, same arguments, layout, value copy and errors as
 * pc_apply.  The product that is not the stored direction scatters with atomic adds, so its
 * FP32 rounding order (not its value) varies between runs. */
pc_status pc_apply_adjoint(pc_handle h, const void* x, void* y, int nrhs, int ldx, int ldy,
                           void* stream);

/* Wavelet-domain deblurring (Section 4.3, min_z 1/2 ||Theta z - z0||^2 + ||z||_{1,w}; the
 * FISTA-W and FISTA-WP iterations of the appendix on deblurring algorithms).  These three
 * calls use the FP32 (or FP64) stored values, never the BF16 copy; vectors are N elements of
 * the handle's type, device, in the canonical coefficient order.  They share handle-owned
 * scratch of 3 N elements (allocated on first use), so a handle runs one of them at a time.
 *
 * pc_jacobi: diag[lambda] = sum_mu Theta[mu, lambda]^2, the diagonal of Theta^T Theta (the
 * Jacobi preconditioner of FISTA-WP).  diag is overwritten.  Asynchronous.
 *
 * pc_power_norm: *norm2 = estimate of the largest eigenvalue of S^(1/2) Theta^T Theta S^(1/2),
 * S = diag(sigma) (sigma NULL: S = I, so *norm2 estimates ||Theta||_2^2), by `iters` >= 1
 * power iterations from u = (1, ..., 1)/sqrt(N): g = M u, estimate ||g||, u = g/||g||.  The
 * estimate never exceeds the eigenvalue; a FISTA step tau <= 1 / *norm2 needs a margin.
 * Synchronises `stream` (it returns a host value).
 *
 * pc_fista: `iters` >= 0 iterations of
 *     z^(i)   = soft(y^(i) - tau S Theta^T (Theta y^(i) - z0), tau S w),
 *     y^(i+1) = z^(i) + (i - 1)/(i + 2) (z^(i) - z^(i-1)),
 * with soft() entrywise soft thresholding and S = diag(sigma) (NULL: FISTA-W; a Jacobi
 * sigma = 1/pc_jacobi(): FISTA-WP).  z holds z^(0) = y^(1) on entry and z^(iters) on return;
 * z0 (the observed image's wavelet coefficients) and the weights w (>= 0) are inputs.
 * tau > 0 (convergence needs tau <= 1 / pc_power_norm(sigma)).  Asynchronous; three kernel
 * launches per iteration (r = Theta y - z0, g = Theta^T r, the update), both products
 * gathering over stored rows: the one against the stored direction reads a transposed copy
 * of the values (the pattern is symmetric).  The first solver call on a handle builds per-row
 * column-block descriptors (12 bytes per row and kept block), and the first after each
 * assembly rebuilds the transposed copy (4 bytes per entry in FP32, 8 in FP64; pc_jacobi and
 * pc_power_norm build them too).  PC_ERR_INVALID_ARG for NULL z0/w/z, iters < 0 or tau <= 0. */
pc_status pc_jacobi(pc_handle h, void* diag, void* stream);
pc_status pc_power_norm(pc_handle h, const void* sigma, int iters, double* norm2, void* stream);
pc_status pc_fista(pc_handle h, const void* z0, const void* w, const void* sigma, void* z, int iters,
                   double tau, void* stream);

/* The two stages of pc_assemble, for callers that time or overlap them separately:
 * stage 0 = base wavelets, filtered wavelets and window tile masks (steps 1-2 above);
 * stage 1 = step 3 (for 2-D operators the window-weighted sums of all rows in one launch into
 * the s scratch, then the per-row localized transforms), which needs a stage 0 for the current
 * parameters before it.  pc_assemble(h, s) equals stage 0 then 1. */
pc_status pc_assemble_stage(pc_handle h, int stage, void* stream);

/* Gradient of a loss of Theta.  dtheta: dL/dTheta on the stored entries, same layout and
 * type as the stored values (nnz elements), device.  du: m x (2r+1)^dim and dv: m x n^dim,
 * device, overwritten with dL/du_k and dL/dv_k.  The filtered wavelets are recomputed, not
 * kept from the forward pass.  Uses handle-owned scratch (allocated on first call). */
pc_status pc_backward(pc_handle h, const void* dtheta, void* du, void* dv, void* stream);

/* Allocation-free pc_backward.  The paper has no counterpart; this is a library concern.
 *
 * Same arguments, results and stream semantics as pc_backward, but the call never allocates
 * device memory: its scratch (dL/dF and dL/dG, the adjoints of the filtered wavelets) lives in
 * one file-scope device array of PC_NOALLOC_SCRATCH_BYTES, which every GPU that loads this
 * library holds until the process exits.  It is meant for callers that cannot call
 * cudaMalloc: a framework that has reserved the whole device for its own pool allocator, or a
 * loop where the implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
 * (pc_backward instead allocates its scratch on the handle at its first call.)
 *
 * Limit: the operator must need at most PC_NOALLOC_SCRATCH_BYTES of scratch (bytes of one
 * element times the sizes of its filtered wavelets and their first-pass products);
 * otherwise PC_ERR_UNSUPPORTED with the required size in pc_last_error().
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of the process;
 * make that first call before any stream capture.  The kept address does not survive
 * cudaDeviceReset (which unloads the library's device code): do not call this entry point
 * after resetting a device it has already run on.  Sharing: all calls on a device use the same array and it keeps the last call's
 * contents (the call clears what must start at zero).  Calls that overlap on the GPU (two
 * streams, two host threads, two handles) race on it: order them. */
#define PC_NOALLOC_SCRATCH_BYTES (8u << 20)
pc_status pc_backward_noalloc(pc_handle h, const void* dtheta, void* du, void* dv, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batches: many operators (any mix of 1-D / 2-D, sizes, terms, kernel radii, db orders and
 * levels; PC_FP32 only) assembled by one persistent launch per kernel kind (1-D rows, and
 * each 2-D filter template), the kinds running side by side.  A launch takes work items
 * (operator, row band, run of rows) from its own global counter, longest first, each with its
 * own thread-group shape (the operator's plan, see pc_autotune).  The batch object captures
 * the whole sequence (every operator's base and filtered wavelets and stage-1 sums, the queue
 * resets and the persistent kernels) in a CUDA graph once; pc_batch_run replays it.
 * --------------------------------------------------------------------------------------- */
typedef struct pc_batch* pc_batch_handle;

/* Plans and captures a batch over `count` handles, which must stay alive (and keep their
 * plans) until pc_batch_destroy.  Runs the sequence once eagerly on `stream` (which also
 * assembles every operator), then captures it on a private stream.  Synchronous. */
pc_status pc_batch_create(pc_handle* ops, int count, void* stream, pc_batch_handle* out);

/* Replays the captured graph on `stream`: re-assembles every operator of the batch from
 * its current parameters.  Asynchronous. */
pc_status pc_batch_run(pc_batch_handle b, void* stream);

/* Work items and graph launches of one run (for counting launches). */
pc_status pc_batch_info(pc_batch_handle b, int* items, int* kernels_per_run);

void pc_batch_destroy(pc_batch_handle b);

/* Convenience: pc_batch_create, one run, pc_batch_destroy (synchronous). */
pc_status pc_batch_assemble(pc_handle* ops, int count, void* stream);

/* Autotuner: for every row band of h, times the row-assembly kernel with each thread-group
 * size (32, 64, 128, 256 threads per row, groups per CTA and s batch following) on the
 * operator's current parameters and keeps the fastest in the handle's plan, which
 * pc_assemble, pc_backward and batches then use.  Synchronous; overwrites Theta (which is
 * left assembled). */
pc_status pc_autotune(pc_handle h, void* stream);

/* ---------------------------------------------------------------------------------------
 * Building an expansion.
 * --------------------------------------------------------------------------------------- */

/* Product-convolution expansion of a space-varying operator from its space-varying impulse
 * response (SVIR), by randomized SVD (Section 2.4: the best rank-m approximation of the SVIR in
 * Frobenius norm gives the expansion; Halko, Martinsson and Tropp's randomized range finder).
 *   S: N x K, FP32, device, row-major: S[x * K + t] is the response at stencil offset t (a
 *      (2r+1)^d stencil, row-major, centre = offset 0) to a unit source at pixel x, so that
 *      (H f)(x + t) = sum_x f(x) S[x, t] on the torus.
 *   omega: K x l test matrix (FP32, device, row-major; the caller draws it, e.g. N(0,1)),
 *      l = m + oversampling, 1 <= m <= l <= min(64, K); power_iters >= 0 refinements
 *      Q <- orth(S orth(S^T Q)).
 * Computes Q = orth(S omega) (refined), B = Q^T S, B = U diag(s) W^T (FP64 on the host) and
 * writes u_k = W[:, k] (u: m x K) and v_k = s_k (Q U)[:, k] (v: m x N), both FP32 device,
 * caller-owned: S ~ sum_k v_k u_k^T, and (u, v) are the kernels and windows of pc_create in
 * the paper's order.  Directions of the sketch below 1e-12 of its largest are dropped, and
 * terms past the sketch's numerical rank come out zero.  sing (host, l doubles, may be NULL)
 * receives s.  The tall products run as cuBLAS FP32 GEMMs on `stream`; the call allocates
 * device scratch (about (N + 2K) l floats) and a cuBLAS handle, and synchronises `stream`.
 * PC_ERR_INVALID_ARG for NULL pointers or sizes out of range. */
pc_status pc_svir_expansion(const float* S, int64_t N, int K, int m, int l, int power_iters, const float* omega,
                            float* u, float* v, double* sing, void* stream);

/* ---------------------------------------------------------------------------------------
 * Inspection.
 * --------------------------------------------------------------------------------------- */

/* nnz and the device bytes owned by the handle. */
pc_status pc_info(pc_handle h, int64_t* nnz, int64_t* device_bytes);

/* Device pointers of the stored values (FP32 or FP64 per precision; BF16 copy or NULL)
 * and of the row offsets (int64, N+1).  Valid until pc_destroy. */
pc_status pc_theta(pc_handle h, void** values, void** values_bf16, int64_t** row_ptr);

/* Host copy of Theta (Section 3.2: Theta[mu, lambda] = <psi_mu, H psi_lambda>, rows = outputs)
 * in CSR form with ascending columns in every row, in either operator order: row_ptr (N + 1),
 * cols (nnz) and vals (nnz, double; the FP32 or FP64 stored values, not the BF16 copy), all
 * caller-owned host arrays.  Copies the values to the host (synchronises `stream`) and sorts
 * on one host thread: meant for inspection and for operators of modest size.
 * PC_ERR_NOT_ASSEMBLED before the first assembly; PC_ERR_INVALID_ARG for NULL arrays. */
pc_status pc_export(pc_handle h, int64_t* row_ptr, int64_t* cols, double* vals, void* stream);

/* Storage position of Theta[mu, lambda] for n pairs (host arrays), -1 when outside the
 * pattern.  Host only; no device work. */
pc_status pc_lookup(pc_handle h, int64_t n, const int64_t* mu, const int64_t* lambda,
                    int64_t* pos);

/* Number of kernel launches this library has issued in the process so far (all handles),
 * for counting the launches inside a timed region. */
int64_t pc_launch_counter(void);

/* ---------------------------------------------------------------------------------------
 * Thresholded Algorithm 1 (Section 3.2): a sparse eta-approximation of Theta.
 *
 * For k = 1..m: A_k = Psi^* U_k Psi (U_k: convolution with u_k), thresholded at tau_k to
 * A~_k, times B_k = Psi^* V_k Psi (V_k = diag(v_k)), accumulated: Theta~ = sum_k A~_k B_k.
 * Threshold: tau_k is the largest value whose discarded part D = A_k restricted to the entries
 * |a| < tau_k has Schur bound sqrt(||D||_1 ||D||_inf) <= eps_k = eta / (m ||v_k||_inf), found
 * by 80 bisection steps on [0, top] with top = max|A_k| (1 + 1e-15) + 1e-300 (taken outright when
 * top itself satisfies the bound, i.e. everything is discarded; eps_k is 1e300 for v_k = 0).
 * Since ||B_k||_2 = ||v_k||_inf (Section 5.5), ||Theta - Theta~||_2 <= eta.
 * Theta~ is stored on the support the products can reach (Section 5.3): row mu holds the
 * coefficients lambda whose wavelet meets the union of the supports of the wavelets kept in
 * row mu of any A~_k (entries there may be zero).  The rows of A_k fall into 2^(levels dim)
 * classes whose rows are translates (sub-band circulant structure), and every stage works per
 * class: no N x N matrix is formed.
 * --------------------------------------------------------------------------------------- */
typedef struct pc_alg1* pc_alg1_handle;

/* Threshold rules for A_k: PC_ALG1_SCHUR is the certified rule above; PC_ALG1_HARD drops the
 * entries below eps_k itself (tau_k = eps_k, the threshold step read literally), which keeps far
 * fewer entries but certifies only max|A_k - A~_k| < eps_k, not the 2-norm bound. */
typedef enum { PC_ALG1_SCHUR = 0, PC_ALG1_HARD = 1 } pc_alg1_rule;

/* Flags.  PC_ALG1_DISCARD: every row of Theta~ is formed, into one device buffer of at most 8 GB
 * (or the largest class's rows) that the groups of row classes overwrite in turn, and the matrix
 * is not kept: the thresholds, counts and stage times remain, pc_alg1_export and pc_alg1_row
 * return PC_ERR_UNSUPPORTED.  For timing sizes whose Theta~ exceeds the device. */
enum { PC_ALG1_DISCARD = 1 };

/* Runs Algorithm 1 on the device and keeps Theta~ in the handle.  desc: dim, n, levels,
 * delta, family, m, radius as for pc_create; order must be PC_ORDER_MULT_THEN_CONV (the other
 * order's matrix is the transpose of this one's for the flipped kernels u_k(-t)); rule is a
 * pc_alg1_rule, flags 0 or PC_ALG1_DISCARD; gap and
 * store_bf16 are ignored.  The generator rows, thresholds and the synthesis of the kept rows run
 * in FP64 in either precision (so both precisions keep the same entries); PC_FP64 forms the
 * products s~ = sum_k v_k F~_k and their transforms in FP64 and stores Theta~ in FP64, PC_FP32
 * in FP32 with the sum over k compensated (Kahan), Theta~ in FP32.  u: m x (2r+1)^dim,
 * v: m x n^dim, FP64, host or device (copied).  eta >= 0.  Synchronous on `stream`.
 * PC_ERR_INVALID_ARG for NULL pointers, eta < 0, an unknown rule or flag or a descriptor out of range,
 * PC_ERR_UNSUPPORTED for the other order or more than 2^16 row classes (dim * levels > 16),
 * PC_ERR_OOM when the generator, product or Theta~ storage does not fit. */
pc_status pc_alg1_create(const pc_desc* desc, const double* u, const double* v, double eta, int rule, int flags,
                         void* stream, pc_alg1_handle* out);

/* nnz: stored entries of Theta~; tau[m]: the thresholds; kept[m]: nonzero entries of A~_k
 * (over the whole N x N matrix); stage_ms[4]: device time of the generator rows, the thresholds,
 * the synthesis of the kept rows and the products.  Any pointer may be NULL. */
pc_status pc_alg1_info(pc_alg1_handle h, int64_t* nnz, double* tau, int64_t* kept, double* stage_ms);

/* Host CSR copy of Theta~ in canonical order: row_ptr (N + 1), cols and vals (nnz each; columns
 * of a row in storage order, unsorted), caller-owned host memory.  Synchronous. */
pc_status pc_alg1_export(pc_alg1_handle h, int64_t* row_ptr, int64_t* cols, double* vals);

/* One row of Theta~ (canonical index `row`): with cols and vals NULL, *count receives its length;
 * otherwise cols and vals (host, *count entries at least) receive the columns (storage order) and
 * values and *count the length.  Synchronous.  PC_ERR_INVALID_ARG for a row outside [0, N) or
 * buffers shorter than the row. */
pc_status pc_alg1_row(pc_alg1_handle h, int64_t row, int64_t* cols, double* vals, int64_t* count);

void pc_alg1_destroy(pc_alg1_handle h);

/* Waits for `stream`, then reports any device-side fault flagged since the last call
 * (PC_ERR_DEVICE) and clears it. */
pc_status pc_sync(pc_handle h, void* stream);

/* Message of the last failing call on h (or of the last failing call without a handle
 * when h is NULL).  Never NULL. */
const char* pc_last_error(pc_handle h);

#ifdef __cplusplus
}
#endif
#endif /* PCWAVE_H */
