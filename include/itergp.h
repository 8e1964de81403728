/*
 * itergp.h -- C ABI of the IterNCGP hot path for NVIDIA GB300 (sm_103a).
 *
 * IterNCGP (Tatzel, Wenger, Schneider, Hennig, arXiv 2310.20285) fits a multi-class GP
 * classifier with a softmax likelihood by Newton steps (Alg. 1).  Each step is a GP
 * regression problem with pseudo targets y_hat = f + W^+ grad log p(y|f) and noise
 * W^+ (Eqs. 6-7, footnote on the pseudo-inverse, Lemma A.6), solved approximately by
 * IterGP (Alg. 2) with actions recycled between steps and compressed to rank R (Alg. 3).
 * All of its cost sits in products with the kernel matrix K (Sec. 3.5, App. B.3.1),
 * which this library evaluates on the fly and never stores.
 *
 * Conventions shared by every entry point
 *  - Matrices are row-major and contiguous.  Vectors over the training set are N x C
 *    arrays in the paper's CN ordering (class index fastest, App. B.1).  The multi-output
 *    prior is K = k(X, X) kron I_C, one kernel shared by the C independent latent GPs
 *    (App. C.3), so K w is k(X, X) @ w for w viewed as N x C.
 *  - Pointers named "device" must point to memory of the current CUDA device.  The
 *    caller owns every pointer argument; the library never frees caller memory.
 *  - Every call is stream-ordered on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and returns without waiting for the GPU, except where stated.
 *  - Errors: functions return ITERGP_OK (0) or a negative itergp_status.  Arguments are
 *    validated on the host before any launch; nothing is launched when validation
 *    fails.  Faults detected on the device (a bounded wait that expired, a non-finite
 *    value) are recorded in a per-device status word that itergp_sync_status() reads.
 *    No function aborts the process or throws across the ABI.
 *  - Thread safety: calls may come from several host threads on different streams.
 *    Scratch memory is drawn stream-ordered from a library-owned pool per device.
 */
#ifndef ITERGP_H_
#define ITERGP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ITERGP_OK = 0,
  ITERGP_EINVAL = -1,       /* invalid argument (host-side check, nothing launched)      */
  ITERGP_ENOMEM = -2,       /* device allocation failed                                   */
  ITERGP_ECUDA = -3,        /* a CUDA runtime call failed                                 */
  ITERGP_ENUMERIC = -4,     /* a non-finite value was produced on the device              */
  ITERGP_ETIMEOUT = -5,     /* a device-side wait exceeded its bound; the kernel returned */
  ITERGP_EUNSUPPORTED = -6, /* the current device is not sm_103a / sm_100 family          */
  ITERGP_ESCRATCH = -7,     /* itergp_kmatvec_noalloc: sizes need more than its fixed scratch */
  ITERGP_EGONE = -8         /* server: the model is not resident (evicted, released, failed) */
} itergp_status;

/* Kernel functions (App. C.1 / C.3 use GPyTorch's RBF and Matern-3/2 kernels):
 *   RBF        k(r) = s exp(-r^2 / (2 l^2))
 *   Matern-3/2 k(r) = s (1 + sqrt(3) r / l) exp(-sqrt(3) r / l)
 * with r^2 = max(0, |a|^2 + |b|^2 - 2 a.b), lengthscale l > 0, outputscale s > 0. */
typedef enum { ITERGP_RBF = 0, ITERGP_MATERN32 = 1 } itergp_kernel_kind;

typedef struct {
  int32_t kind;         /* itergp_kernel_kind */
  float lengthscale;    /* l */
  float outputscale;    /* s */
} itergp_kernel;

/* Arithmetic of the two contractions inside the kernel product (distance over D and the
 * kernel-weighted sum over the data points).  Accumulation is FP32 in every mode.
 *   ITERGP_FP32      plain FP32 SIMT (FFMA) for both contractions.
 *   ITERGP_BF16X3    tensor cores; each operand split into 16-bit hi + lo parts (FP16 with
 *                    a power-of-two scale per 128-row tile of the rows, per weight column,
 *                    and for the kernel values; 22 significant bits) and each contraction
 *                    formed from the three products hi*hi + hi*lo + lo*hi.  FP32-level
 *                    accuracy (normwise relative error ~1e-6 on products).  The name
 *                    keeps the first version's (BF16 parts).
 *   ITERGP_BF16      tensor cores; one BF16 product per contraction; the squared distance
 *                    uses the norms of the BF16-rounded rows.
 *   ITERGP_BF16_COMP tensor cores; split-precision (3-product) distance with FP32 norms,
 *                    one-product BF16 kernel-weighted sum.
 *   ITERGP_TF32      tensor cores; the distance from TF32 operands (rows rounded once to
 *                    10 mantissa bits, nearest-even; norms of the rounded rows; one
 *                    product, K = 8 per instruction), the kernel-weighted sum as in
 *                    BF16X3. */
typedef enum {
  ITERGP_FP32 = 0,
  ITERGP_BF16X3 = 1,
  ITERGP_BF16 = 2,
  ITERGP_BF16_COMP = 3,
  ITERGP_TF32 = 4
} itergp_precision;

typedef void* itergp_stream; /* cudaStream_t */

/* ----------------------------------------------------------------------------------
 * Kernel matrix times block of vectors (App. B.3.1 "Products with K"; Alg. 2 t_j = K s_j;
 * Eq. 9 predictive mean).
 *
 *   Y[i, :] = sum_j k(A[i, :], B[j, :]) S[j, :]        i < m, j < n
 *
 * A: device, m x d FP32.  B: device, n x d FP32.  S: device, n x p FP32.
 * Y: device, m x p FP32, overwritten (Y = 0 when n == 0).  k is never stored: each CTA
 * evaluates tiles of it on the fly and contracts them with S.  m, n, p >= 0, d >= 1,
 * d <= 4096, p <= 65536.  Y must not alias A, B or S.  Scratch (BF16 copies, norms,
 * split partial sums) comes from the library's stream-ordered pool.
 * Returns ITERGP_EINVAL for bad sizes/pointers, ITERGP_EUNSUPPORTED if a tensor-core
 * precision is requested on a device without tcgen05. */
int itergp_kmatvec(const itergp_kernel* kernel, int32_t precision, const float* A, int64_t m,
                   const float* B, int64_t n, int64_t d, const float* S, int64_t p, float* Y,
                   itergp_stream stream);

/* Kernel product with one kernel per class (the multi-output prior of independent GPs,
 * Sec. 5 / App. C.3, each with its own hyperparameters):
 *
 *   Y[i, j] = sum_l k_{j mod c}(A[i, :], B[l, :]) S[l, j]        i < m, l < n, j < p
 *
 * i.e. the columns of S are NC-vectors viewed as n x c blocks side by side (CN ordering)
 * and column j belongs to class j mod c.  kernels: host, c entries (1 <= c <= 64).  Runs c
 * grouped products over each class's columns (the distance contraction is repeated per
 * class).  Sizes, pointers, layouts and errors as itergp_kmatvec. */
int itergp_kmatvec_classes(const itergp_kernel* kernels, int32_t c, int32_t precision, const float* A,
                           int64_t m, const float* B, int64_t n, int64_t d, const float* S, int64_t p,
                           float* Y, itergp_stream stream);

/* ----------------------------------------------------------------------------------
 * Kernel product for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of itergp_kmatvec.
 *
 * Some callers must not call cudaMalloc or any allocating routine while they run: code
 * inside a CUDA-graph-building or real-time serving loop that has reserved all device
 * memory up front, plug-in hosts whose allocator is not the CUDA one, or processes that
 * forbid allocation after start-up.  For them this entry point computes exactly what
 * itergp_kmatvec computes (same kernels, same arguments, same result) but takes every
 * byte of scratch (BF16 copies, row norms, transposed S, split partial sums) from one
 * file-scope static device array of ITERGP_NOALLOC_SCRATCH_BYTES (64 MiB) that each GPU
 * loading the library holds until the process exits.  It calls no cudaMalloc, cudaFree
 * or allocating library routine.
 *
 *  - The caller passes inputs and outputs exactly as for itergp_kmatvec; `device_status`
 *    (device int, may be NULL) receives ITERGP_ETIMEOUT if a device-side wait gives up;
 *    the caller zeroes it.
 *  - Sizes whose scratch would exceed the array are rejected with ITERGP_ESCRATCH before
 *    any launch (for the tensor precisions roughly rows x round_up(d, 64) x 4 bytes per
 *    operand, so e.g. m = n = 8192, d = 784 fits; the FP32 precision needs far less).
 *  - The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress (device set-up, once per device); make that first call before
 *    any stream capture.  Under CUDA's default lazy module loading the 64 MiB array is
 *    created on the device at that lookup (under eager loading, when the library loads),
 *    so the first call needs 64 MiB of free device memory: make it before reserving the
 *    rest of the device.  A call with m = 0 (or p = 0) performs only this set-up.
 *  - Every call shares the one array, which keeps the previous call's contents; all of it
 *    that is read is written first within the call.  Calls whose work overlaps on the GPU
 *    (different streams, or host threads without ordering) race on the array: serialise
 *    them, e.g. on one stream. */
#define ITERGP_NOALLOC_SCRATCH_BYTES (64ull << 20)
int itergp_kmatvec_noalloc(const itergp_kernel* kernel, int32_t precision, const float* A,
                           int64_t m, const float* B, int64_t n, int64_t d, const float* S,
                           int64_t p, float* Y, int* device_status, itergp_stream stream);

/* ----------------------------------------------------------------------------------
 * Softmax-likelihood building blocks (Alg. 1 lines "W(f)^-1" and "y_hat"; Lemma A.6).
 * f, x, out: device, n x c FP32; y: device, n int32 labels in [0, c); c >= 2.
 *
 * itergp_winv_apply:     out_n = P diag(1/pi_n) P x_n,  pi_n = softmax(f_n),
 *                        P = I - 11^T / c  (the pseudo-inverse W(f)^+ of Lemma A.6);
 *                        1/pi is formed as exp(logsumexp(f_n) - f_n).
 * itergp_pseudo_targets: out = f + W(f)^+ (onehot(y) - softmax(f))   (Alg. 1 / Eq. 6).
 * Labels outside [0, c) set ITERGP_EINVAL in the device status word. */
int itergp_winv_apply(const float* f, int64_t n, int32_t c, const float* x, float* out,
                      itergp_stream stream);
int itergp_pseudo_targets(const float* f, const int32_t* y, int64_t n, int32_t c, float* out,
                          itergp_stream stream);

/* ----------------------------------------------------------------------------------
 * Symmetric eigendecomposition of the projected Gram matrix of Alg. 3 in FP64 on the
 * device (cyclic Jacobi, one CTA).  M: device, b x b FP64 (only its symmetric part is
 * used); lam: device, b FP64, eigenvalues in descending order (ties by index);
 * U: device, b x b FP64 row-major, column k = eigenvector of lam[k].  1 <= b <= 512.
 * M is not modified. */
int itergp_sym_eig(const double* M, int32_t b, double* lam, double* U, itergp_stream stream);

/* ----------------------------------------------------------------------------------
 * IterNCGP fit (Alg. 1 with Alg. 2 inner solves and Alg. 3 recycling/compression).
 * Prior mean m = 0 and f_0 = m (App. C.3); buffers start empty. */

typedef enum { ITERGP_POLICY_CG = 0, ITERGP_POLICY_UNIT = 1 } itergp_policy;

typedef enum {
  ITERGP_STOP_MAXITER = 0,  /* inner solver ran max_iters iterations            */
  ITERGP_STOP_TOL = 1,      /* |r| < max(tol_abs, tol_rel |y_hat - m|)  (App. B.2) */
  ITERGP_STOP_ETA = 2       /* eta_j <= 0: action not kept                        */
} itergp_stop_reason;

/* Likelihoods p(y | f).  Softmax is the paper's multi-class model; the others are its
 * one-latent specialisations and the conjugate case, all solved by the same Alg. 1-3
 * (only W^-1 and the pointwise terms change).  Objectives drop terms constant in f. */
typedef enum {
  ITERGP_LIK_SOFTMAX = 0,    /* c >= 2 classes, y labels in [0, c): W^+ of Lemma A.6     */
  ITERGP_LIK_BERNOULLI = 1,  /* c = 1, y in {0, 1}, logistic link: W^-1 = 1/(pi (1-pi)) (App. C) */
  ITERGP_LIK_POISSON = 2,    /* c = 1, counts y >= 0, log link: W^-1 = e^-f (App. A)     */
  ITERGP_LIK_GAUSSIAN = 3    /* c >= 1 outputs, real targets y_real, W^-1 = noise I (Thm. A.2) */
} itergp_likelihood;

typedef struct {
  int64_t n;              /* number of training points, >= 1                       */
  int64_t d;              /* input dimension, 1 .. 4096                            */
  int32_t c;              /* classes (softmax: 2 .. 64), outputs (Gaussian: 1 .. 64),
                             1 for Bernoulli and Poisson                            */
  const float* X;         /* device, n x d FP32 (copied into the model)           */
  const int32_t* y;       /* device, n labels in [0, c) / {0,1} / counts (not Gaussian) */
  itergp_kernel kernel;
  int32_t precision;      /* itergp_precision of every kernel product             */
  int32_t policy;         /* itergp_policy: residual actions (CG) or unit vectors */
  int32_t max_newton;     /* Newton steps (outer iterations), >= 1                */
  int32_t max_iters;      /* solver iterations per Newton step (j_max), >= 0       */
  int32_t rank;           /* compression limit R (Alg. 3); < 0 means no limit      */
  int32_t recycle;        /* 1: virtual solver run (Alg. 3); 0: fresh buffers       */
  int32_t literal_kv;     /* 0: K v_{j-1} is carried from the T buffer (one K product
                             per iteration); 1: recomputed by a K product as printed
                             in Alg. 2 (two per iteration, plus f_{i+1} = K v + m)  */
  double tol_newton;      /* outer stop on |g_i - g_{i-1}| / |g_i| <= tol (<= 0: off)*/
  double tol_abs;         /* inner stop, absolute (paper default 1e-5)             */
  double tol_rel;         /* inner stop, relative to |y_hat - m| (default 1e-5); the
                             BF16 and BF16_COMP precisions also stop at 2^-8 |y_hat - m|,
                             the rounding level of their products                   */
  int32_t graph;          /* 1: capture the whole fit into one CUDA graph and launch
                             it (fewer launch overheads); 0: launch kernels directly */
  const float* f0;        /* device, n x c starting iterate, or NULL for f_0 = m = 0
                             (Alg. 1); with a start, Psi(f_0) is reported with v = 0  */
  int32_t likelihood;     /* itergp_likelihood (0 = softmax)                        */
  float noise;            /* Gaussian likelihood: noise variance sigma^2 > 0          */
  const float* y_real;    /* Gaussian likelihood: device, n x c real targets (y unused) */
  /* One kernel per output GP (the c latent GPs are independent, Sec. 5 / App. C.3): host,
   * c entries, NULL for one shared `kernel`.  K is then block-diagonal over the classes in
   * CN ordering and every product runs as c grouped products (one per class, each over
   * its own columns).  Under the softmax likelihood the W^+ substitution (footnote to
   * Eq. 6) is Newton's step only while all classes share a kernel; with distinct kernels
   * Alg. 1 as printed converges to a point off the posterior mode.  Copied by the fit;
   * batched fits with per-class kernels run their problems one after another. */
  const itergp_kernel* class_kernels;
  uint64_t wait_limit_ns; /* bound of every device-side wait of the fit's kernel products,
                             1e6 .. 6e10 ns, or 0 for the default 4 s; a wait that runs
                             out ends the product with ITERGP_ETIMEOUT (the fit returns
                             it) instead of hanging                                 */
} itergp_fit_params;

#define ITERGP_MAX_REPORT_STEPS 64

typedef struct {
  int32_t newton_steps;   /* Newton steps taken                                   */
  int32_t total_iters;    /* solver iterations over all steps                     */
  int32_t buffer_cols;    /* columns of S, T, Q at the end                        */
  int32_t stop_reason;    /* of the last inner solve (itergp_stop_reason)         */
  int32_t iters[ITERGP_MAX_REPORT_STEPS];       /* per Newton step                 */
  int32_t stops[ITERGP_MAX_REPORT_STEPS];       /* per Newton step                 */
  int32_t kept[ITERGP_MAX_REPORT_STEPS];        /* buffer columns after Alg. 3     */
  double objective[ITERGP_MAX_REPORT_STEPS];    /* Psi(f_i), Eq. 2, per step       */
  double rel_change[ITERGP_MAX_REPORT_STEPS];   /* |g_i - g_{i-1}|/|g_i| (i >= 1)  */
  double resid_norm;      /* |r| at the last residual evaluation                   */
  int64_t device_bytes;   /* bytes held by the model and its buffers              */
  int32_t status;         /* this problem's outcome: ITERGP_OK, ITERGP_EINVAL (a    */
                          /* label out of range) or ITERGP_ENUMERIC (1/pi overflow)  */
  int32_t reserved;
  int64_t peak_bytes;     /* library-pool bytes the call held at its peak: models,
                             fit workspace and product scratch (all problems of a
                             batched call together)                                  */
} itergp_fit_report;

typedef struct itergp_model itergp_model;

/* Runs the whole fit on `stream` and waits for it (the report needs the device's
 * counters).  On success *out owns device memory until itergp_model_free.
 * Returns ITERGP_ENUMERIC if a non-finite value appeared during the fit. */
int itergp_fit(const itergp_fit_params* params, itergp_model** out, itergp_fit_report* report,
               itergp_stream stream);

/* Batched fit of `count` independent problems (different n, d, c, X, y, lengthscale and
 * outputscale) with one schedule: every phase of Alg. 1-3 runs as one launch over all
 * problems (per-problem flags mask finished solves) and the kernel products run as one
 * persistent launch over the row tiles of all problems.  Fields that must agree across
 * params[0 .. count-1]: kernel.kind, precision, policy, max_newton, max_iters, rank,
 * recycle, tol_newton, tol_abs, tol_rel, graph; literal_kv must be 0.  models[i] and
 * reports[i] (reports may be NULL) receive each problem's result.  A problem that fails
 * on the device (a label out of range, a non-finite value) stops alone: models[i] is
 * NULL, reports[i].status holds its code and the call still returns ITERGP_OK for the
 * others.  Errors of the call itself (arguments, memory, CUDA, a wait limit) return
 * their code and no model.  Waits for the stream like itergp_fit. */
int itergp_fit_batch(const itergp_fit_params* params, int32_t count, itergp_model** models,
                     itergp_fit_report* reports, itergp_stream stream);

/* Posterior predictive of the fitted model (Eqs. 9-10 with C_j = Q Q^T) and the probit
 * approximation of App. C.3:
 *   mean[i, c]  = sum_n k(x*_i, x_n) v[n, c]
 *   var[i, c]   = s - sum_b (sum_n k(x*_i, x_n) Q_b[n, c])^2
 *   probs[i, :] = softmax(mean[i, :] / sqrt(1 + pi/8 var[i, :]))
 * Xs: device, m x d FP32; mean: device m x c (required); var, probs: device m x c or
 * NULL.  One fused kernel product against the stacked columns [v | Q]. */
int itergp_predict(const itergp_model* model, const float* Xs, int64_t m, float* mean,
                   float* var, float* probs, itergp_stream stream);

/* Read-only view of the model's device arrays (valid until itergp_model_free). */
typedef struct {
  int64_t n, d;
  int32_t c, buffer_cols;
  itergp_kernel kernel;
  const float* X;   /* n x d                                   */
  const float* v;   /* n x c representer weights v_j           */
  const float* f;   /* n x c latest Newton iterate f_{i+1}     */
  const float* Q;   /* buffer_cols blocks of n x c: root of C_j */
} itergp_model_view;

int itergp_model_get_view(const itergp_model* model, itergp_model_view* view);
void itergp_model_free(itergp_model* model);

/* ----------------------------------------------------------------------------------
 * Instrumentation (off by default).
 * itergp_timing_enable(1): every launch of the fused kernel-product kernel (the tile
 *   kernel inside itergp_kmatvec / itergp_fit / itergp_predict) is bracketed by a pair of
 *   CUDA events recorded on the stream it is launched on.
 * itergp_timing_read: waits for the recorded events, returns the summed device time (ms)
 *   and number of those launches since the previous read, and clears them.
 * itergp_launch_count: total number of CUDA kernels this library has launched in the
 *   process (all kernels, not only the product). */
int itergp_timing_enable(int enable);
int itergp_timing_read(double* kernel_ms, int64_t* launches);
int64_t itergp_launch_count(void);

/* Waits for `stream`, then returns and clears the current device's status word:
 * ITERGP_OK, ITERGP_ETIMEOUT, ITERGP_ENUMERIC or ITERGP_EINVAL (bad label). */
int itergp_sync_status(itergp_stream stream);

const char* itergp_status_string(int status);

/* The CUDA call behind the calling thread's most recent ITERGP_ECUDA: "<call>: <CUDA
 * error string> (<file>:<line>)", or "" if there was none.  The pointer is owned by the
 * library and stays valid until the thread's next failing call.  (Library plumbing; the
 * paper has no counterpart.) */
const char* itergp_last_error(void);

/* ------------------------------------------------------------------------------------
 * Serving (a project addition; the paper has no serving layer).
 *
 * A server owns one GPU's share of models: it fits models from host data and answers
 * predictive queries against them, with continuous batching on two streams driven by two
 * host threads:
 *  - fits: requests waiting when the fit stream frees up are admitted together (in
 *    arrival order, while the HBM budgets allow) and run as ONE batched fit
 *    (itergp_fit_batch semantics: every phase of Alg. 1-3 is one launch over the batch);
 *    each fitted model is then installed in the server's model slab;
 *  - predicts: requests waiting when the predict stream frees up are admitted together,
 *    across models, and answered by one batched product per part (mean: K(X*,X) v;
 *    variance: K(X*,X) Q) over all of them, then one epilogue (Eqs. 9-10, probit).
 * Predicts run while fits are on the GPU.  Every model keeps X (prepared rows), v and the
 * root Q of C_j = Q Q^T resident in the slab until it is released or evicted.
 *
 * Memory: `model_bytes` is the slab, carved into 128-row blocks.  A fit is admitted only
 * when its rows fit in the slab; idle models (no queued or running predicts) are evicted
 * least recently used first to make room.  `work_bytes` bounds the workspace of the fits
 * in flight.  A request that can never fit fails with ITERGP_ENOMEM.
 *
 * All models of a server share kernel.kind, precision and the fit schedule.  Data passed
 * to submit calls is copied before the call returns; predict outputs are written to the
 * caller's host buffers, which must stay valid until the request's completion event. */
typedef struct itergp_server itergp_server;

typedef struct {
  int64_t model_bytes;       /* HBM for resident models (the slab)                      */
  int64_t work_bytes;        /* HBM for the workspaces of fits in flight                */
  int32_t kind;              /* itergp_kernel_kind of every model                       */
  int32_t precision;         /* itergp_precision of fits and predicts                   */
  int32_t d_max;             /* largest input dimension (1..1024)                       */
  int32_t c_max;             /* largest class count (2..16)                             */
  int32_t max_fit_batch;     /* problems per batched fit (>= 1)                         */
  int32_t max_predict_batch; /* requests per batched predict (>= 1)                     */
  int64_t max_predict_rows;  /* query rows per batched predict (>= 4096)                */
  int32_t max_newton, max_iters, rank;   /* fit schedule (Alg. 1-3); CG actions,        */
  int32_t graph;             /* recycling on; graph != 0 captures each fit batch         */
  double tol_abs, tol_rel;   /* inner tolerances (App. B.2)                             */
} itergp_server_config;

typedef enum { ITERGP_REQ_FIT = 0, ITERGP_REQ_PREDICT = 1 } itergp_request_kind;

typedef struct {
  int64_t id;                /* model id (fit) or request id (predict)                 */
  int64_t model;             /* the model the request belongs to                       */
  int32_t kind;              /* itergp_request_kind                                     */
  int32_t status;            /* ITERGP_OK or the request's error                        */
  double submit_s, start_s, done_s;   /* server clock (s): submitted, launched, results ready */
  int32_t batch;             /* requests in the launch batch it ran in                 */
  int32_t reserved;
} itergp_server_event;

typedef struct {
  int64_t resident_models, resident_rows, slab_rows;
  int64_t fits_done, predicts_done, fit_batches, predict_batches, evicted;
  int64_t queued_fits, queued_predicts;
} itergp_server_stats;

/* Creates the server on the current device (allocates the slab, starts its threads).
 * c_max * (1 + buffer capacity of the schedule) must be <= 144 (one mean tile of 16 and
 * one variance tile of 128 weight columns per model). */
int itergp_server_create(const itergp_server_config* config, itergp_server** out);
/* Stops accepting requests, drops those still queued (no events for them), waits for the
 * batches on the GPU, joins the threads and frees the slab. */
int itergp_server_destroy(itergp_server* server);
/* Queues a fit of host X (n x d) with host labels y (n, values in [0, c)).  *model_id
 * identifies the model in predicts and events. */
int itergp_server_submit_fit(itergp_server* server, const float* X, const int32_t* y,
                             int64_t n, int64_t d, int32_t c, float lengthscale,
                             float outputscale, int64_t* model_id);
/* Queues a predict of host Xs (m x d of the model) against a model that is resident or
 * still being fitted.  mean (m x c) is required; var and probs (m x c) may be NULL. */
int itergp_server_submit_predict(itergp_server* server, int64_t model_id, const float* Xs,
                                 int64_t m, float* mean, float* var, float* probs,
                                 int64_t* request_id);
/* Moves up to `capacity` completion events (oldest first) to `events`; waits up to
 * timeout_us (< 0: forever) for the first one.  *count may be 0 after a timeout. */
int itergp_server_poll(itergp_server* server, itergp_server_event* events, int32_t capacity,
                       int32_t* count, int64_t timeout_us);
/* Releases a model's slab rows once its queued predicts are done (later predicts on it
 * fail with ITERGP_EGONE). */
int itergp_server_release(itergp_server* server, int64_t model_id);
int itergp_server_get_stats(itergp_server* server, itergp_server_stats* stats);

/* ------------------------------------------------------------------------------------
 * Autotuning of the tensor-core product (a project addition; the paper has no such part).
 * A launch variant is the number of epilogue warps (4, or 8 with two warps per TMEM lane
 * quadrant splitting the columns), the depth of the TMA stage ring (2-4 stages of A and B
 * tiles), where D fits one 64-wide slice of BF16 rows a resident-A ring (the row
 * tile's A stays in shared memory; 3 or 5 stages of B tiles; not for TF32 rows, which
 * take two slices per 64 columns), and for the single-problem schedule the CTA-pair form
 * (clusters of two CTAs on two SMs sharing 256-row tiles through cta_group::2 MMAs of
 * M = 256; by default on wherever A is streamed), with chunks of 128 rows of B (MMA
 * N = 128) or, where all of P fits one tile of <= 80 columns, wide chunks of 192 rows
 * (MMA N = 192, three stages; the default there).  The library
 * keeps a process-wide table keyed by (precision, kernel kind, D padded to 64, P tile,
 * schedule); launches not in the table use 4 warps and the deepest ring that fits.
 *
 * itergp_autotune times every variant that fits on synthetic operands of the given shape
 * (n rows of dimension d, p weight columns; items = 0: the single-problem schedule of
 * itergp_kmatvec and fits, items = 1: the batched/served item schedule, p <= 128), records
 * the fastest in the table and reports all timings (ms per launch; stages < 0 mark the
 * resident-A ring).  It waits for the stream.  Tensor-core precisions only.
 * itergp_tune_save / _load write / merge the table as text lines
 * "precision kind d_pad p_tile items epilogue_warps stages resident_a cta_pair"
 * (resident_a: 1, 0, or -1 = where possible; cta_pair: 1 pair form, 2 pair form with wide
 * chunks, 0 off, -1 where possible; missing last columns read as -1); _clear empties it. */
#define ITERGP_TUNE_MAX 20
typedef struct {
  int32_t epilogue_warps, stages, cta_pair;   /* stages < 0: resident-A ring; cta_pair 1: pair
                                               form, 2: pair form with wide chunks */
  double ms;
} itergp_tune_variant;
typedef struct {
  int32_t count, best;
  itergp_tune_variant variants[ITERGP_TUNE_MAX];
} itergp_tune_result;
int itergp_autotune(const itergp_kernel* kernel, int32_t precision, int64_t n, int64_t d, int64_t p,
                    int32_t items, itergp_tune_result* result, itergp_stream stream);
int itergp_tune_save(const char* path);
int itergp_tune_load(const char* path);
int itergp_tune_clear(void);

/* Self-test of failure detection (a project addition): launches one CTA that waits, with
 * the same bounded mbarrier wait the tensor-core kernel uses, on a barrier nothing ever
 * arrives on.  After limit_ns (1e5 .. 5e9) the wait gives up, the kernel records
 * ITERGP_ETIMEOUT in the device status word (read and cleared by itergp_sync_status) and
 * returns; the context stays usable.  No fault, trap or hang is involved. */
int itergp_selftest_wait(uint64_t limit_ns, itergp_stream stream);

/* Throughput probes: measurement tooling of the bench, in libitergp_probe.so (include/itergp_probe.h). */

/* Library version "major.minor.patch". */
const char* itergp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ITERGP_H_ */
