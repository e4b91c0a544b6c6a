/*
 * qr.h -- C-ABI of libqrmc, a B300 (sm_103a) implementation of the
 * Quasi-Regression Monte-Carlo (QRMC) scheme of Gobet, Lopez-Salas and
 * Vazquez, "Quasi-Regression Monte-Carlo scheme for semi-linear PDEs and
 * BSDEs with large scale parallelization on GPUs" (arXiv 2407.21084).
 *
 * The library solves the dynamic programming equation of Sec. 2.1.1,
 *     y_i(x) = E[ g(X_N) + sum_{j=i}^{N-1} f(t_j, X_j, y_{j+1}(X_{j+1})) dt | X_i = x ],
 * on the grid t_j = j dt, dt = T/N, with X the Euler scheme of Sec. 2.1.1
 * (constant drift b and constant diffusion matrix sigma). Each y_i is
 * represented by its coefficients alpha_{i,k}, k in an index set Gamma of
 * Z^d, on the nu-orthonormal basis phi_k(x) = prod_l e^{2 pi i k_l F_nu(x_l)}
 * (Sec. 2.2 with complex exponentials in place of cosines):
 *     ybar_i(x) = Re sum_{k in Gamma} alpha_{i,k} phi_k(x),
 * or on the paper's own cosine basis over an N^d set (index-set kinds 3-5
 * below), optionally with the damping exponent q of eq. (yqi).
 * One Picard iteration recomputes every row i from the previous iterate at
 * once; each row is the Monte-Carlo projection of Algorithm 1 (Sec. 2.3):
 *     alpha_{i,k} = (1/M) sum_m S_i^m conj(phi_k(X_i^{i,m})),  X_i^{i,m} ~ nu,
 *     S_i = g(X_N) + sum_{j=i}^{N-1} f(t_j, X_j, T_L(ybar_{j+1}(X_{j+1}))) dt,
 * with no linear solve.
 *
 * Conventions for every call:
 *  - Every call returns a qr_status and never aborts or exits. Errors found
 *    on the device (a bounded wait that ran out, non-finite responses) are
 *    recorded in the context and returned by the call that launched the
 *    work; qr_last_error() gives a text.
 *  - The caller owns every array it passes. The context owns its device
 *    buffers (allocated at qr_init, freed by qr_destroy, on the context's
 *    stream: by the caller's allocator when qr_opts gives one, else by
 *    cudaMallocAsync / cudaFreeAsync).
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Host arrays are plain C arrays; "device" arrays are CUDA device
 *    pointers of the current device.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with
 *   key = (seed & 0xffffffff, seed >> 32),
 *   counter = (m, c, j, (instance << 20) | (tag << 16) | i),
 * tag 0 = start point (j = 0xffffffff), 1 = Brownian increment of step j,
 * 2 = test point. A uniform is u = (2n+1) 2^-53 with the 52-bit integer
 * n = (w0 << 20) ^ (w1 >> 12) of two words; call c of a path gives
 * coordinates 2c and 2c+1 (start: words (0,1) and (2,3); increments: one
 * Box-Muller pair z = sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b)).
 */
#ifndef QR_H
#define QR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qr_ctx qr_ctx;

typedef enum {
    QR_OK = 0,
    QR_EINVAL = 1,      /* bad argument; nothing was launched */
    QR_ENOMEM = 2,      /* device or host allocation failed */
    QR_ECUDA = 3,       /* a CUDA runtime call failed (text in qr_last_error) */
    QR_ETIMEOUT = 4,    /* a bounded device wait ran out; results are invalid */
    QR_ENONFINITE = 5,  /* some responses were NaN/Inf; results are invalid */
    QR_ENOTIMPL = 6     /* combination not supported by this build */
} qr_status;

/* sampling density nu of the start points (Sec. 2.1.2), same 1-D marginal
 * in every coordinate */
enum {
    QR_NU_LOMAX = 0,    /* (mu/2)(1+|x|)^-(mu+1)                  mu > 0 */
    QR_NU_STUDENT2 = 1, /* 0.5 (1+x^2)^-3/2  (Student mu = 2, Sec. 5) */
    QR_NU_CAUCHY = 2    /* 1/(pi (1+x^2))    (Student mu = 1, Sec. 5) */
};
typedef struct {
    int kind;
    double mu;          /* used by QR_NU_LOMAX */
} qr_nu;

/* Index sets and basis. Kinds 0-2 are sets of Z^d, symmetric under k -> -k,
 * with the complex Fourier basis phi_k(x) = e^{2 pi i k.F_nu(x)}. Kinds 3-5
 * are the N^d sets of Sec. 2.4.2 with the paper's cosine basis
 * phi_k(x) = prod_l C_{k_l}(F_nu(x_l)), C_0 = 1, C_k = sqrt(2) cos(k pi u)
 * (Lemma ortho:dim1). A cosine context runs one of two routes (see
 * qr_opts.path_kernel):
 *   direct: real kernels on Gamma itself, each factor C_k stepped by one
 *     complex product along the canonical order (runs of k_d = 0, 1, ...
 *     under a common prefix; the next run's prefix has one coordinate one
 *     larger and the later ones 0, true of every downward-closed set);
 *     prefix coordinates k_1..k_{d-1} <= 255 and k_d <= 65532;
 *   unfolded: the set {m in Z^d : |m| in Gamma} (Gamma_F(n) -> kind 0,
 *     Gamma_T(n) -> kind 1, Gamma_H(n) -> kind 2, same n) on the Fourier
 *     kernels with half-angle phases e^{i pi m.F_nu(x)}: a cosine series
 *     sum_k a_k phi_k equals Re sum_m c_m e^{i pi m.F_nu(x)} with real,
 *     sign-symmetric c_m = a_|m| 2^{-d'(m)/2}, d'(m) = #{l : m_l != 0}, and
 *     after every projection the coefficients are averaged over the sign
 *     orbits, which is the cosine projection of eq. (Aqi:bar:M) in these
 *     coordinates; its per-lane power tables of d (max|k_l| + 1) complex
 *     values must fit in shared memory (QR_ENOTIMPL otherwise).
 * Either way qr_gamma_size/list, qr_get/set_coefs and a QR_GT_TRIGPOLY g
 * use Gamma itself (the N^d set) and the cosine coefficients a_k: real
 * values in the interleaved complex layout (imaginary parts 0 on output,
 * ignored on input). Canonical order: lexicographic, k_1 most significant. */
enum {
    QR_G_LINF = 0,      /* max_l |k_l| <= n */
    QR_G_L1 = 1,        /* sum_l |k_l| <= n */
    QR_G_HYP = 2,       /* prod_l max(|k_l|,1) <= n */
    QR_G_FULL_N = 3,    /* Gamma_F(n,...,n) = {k in N^d : k_l <= n}, cosine basis */
    QR_G_TOTAL_N = 4,   /* Gamma_T(n) = {k in N^d : sum_l k_l <= n}, cosine basis */
    QR_G_HYP_N = 5      /* Gamma_H(n) = {k in N^d : prod_l max(k_l,1) <= n}, cosine basis */
};
typedef struct {
    int kind;
    int n;
} qr_gamma;

/* driver f(t, x, y) and terminal condition g(x) */
enum {
    QR_F_ZERO = 0,        /* f = 0                                  params: none */
    QR_F_LINEAR = 1,      /* f = lambda y                           params: {lambda} */
    QR_F_CUBIC_MANUF = 2, /* f = -y^3 + r(t,x), r = (a + |sigma^T s|^2/2) u + u^3,
                             u = e^{a(T-t)} cos(s.x)                params: {a, s_1..s_d} */
    QR_F_PAPER_MIN = 3    /* Sec. 5: min(1, [y-kappa-1-sin(lambda sum x) e^{lambda^2 d (t-T)/2}]^2)
                                                                    params: {kappa, lambda} */
};
enum {
    QR_GT_COS = 0,        /* g = cos(s.x)                           params: {s_1..s_d} */
    QR_GT_TRIGPOLY = 1,   /* g = Re sum_{k in Gamma} c_k phi_k(x)   params: 2|Gamma| doubles
                             (re, im interleaved, canonical order, c_{-k} = conj(c_k);
                             cosine contexts: the real cosine coefficients on Gamma) */
    QR_GT_PAPER_SIN = 2   /* Sec. 5: g = 1 + kappa + sin(lambda sum x)  params: {kappa, lambda} */
};
typedef struct {
    int kind;
    const double* params; /* host array, copied by qr_init */
    int n_params;
} qr_fn;

enum { QR_FP64 = 0, QR_FP32 = 1 };
enum { QR_U_PHILOX = 0, QR_U_LATTICE = 1 };
enum { QR_HOST = 0, QR_DEVICE = 1 };

typedef struct {
    long long M;              /* paths per time index, 1 <= M <= 2^32 */
    unsigned long long seed;  /* Philox key */
    int precision;            /* QR_FP64 (plain form) or QR_FP32 (precision form:
                                 FP32 path/basis math, FP64 cross-block sums and alpha) */
    double clamp_L;           /* truncation T_L (eq. TL:2) at the constant level L; <= 0: off */
    void* stream;             /* cudaStream_t for all work; NULL: the context makes its own */
    int uniform_source;       /* QR_U_PHILOX, or QR_U_LATTICE: start uniforms on the centred
                                 lattice u_l = (digit_l(m) + 1/2)/lattice_n, M = lattice_n^d
                                 (test hook: lattice sums integrate trigonometric
                                 polynomials exactly) */
    int lattice_n;
    int instance;             /* Philox counter field, 0 <= instance < 4096 */
    int path_kernel;          /* 0: the compile-time tree kernel when one is built for this
                                 index set (|k|_1 or |k|_inf sets of the benchmark workloads),
                                 else the table-driven kernel; cosine sets: the unfolded
                                 route when a tree kernel covers the unfolded set, else
                                 the direct route. 1: always the table-driven kernel
                                 (cosine: the unfolded route). 2: the direct route (cosine
                                 sets only; QR_EINVAL for kinds 0-2). Other values: QR_EINVAL */
    double damping_q;         /* damping exponent q >= 0 of eq. (yqi), 0 = none: the
                                 coefficients represent ybar^q = y / (1 + |x|^2)^{q/2};
                                 responses follow eq. (Sqi:bar:M) (the series at X_{j+1}
                                 is multiplied by the weight before T_L and f, the
                                 response divided by the weight at X_i^i); qr_eval
                                 returns ybar^q. A QR_GT_TRIGPOLY g stays undamped. */
    /* Device memory of the context (and of a batch built on it): when both
     * are set, every device buffer the context owns is obtained by
     * dev_alloc(bytes, stream, alloc_user) and returned by
     * dev_free(ptr, stream, alloc_user), stream being the context's stream
     * (all use of the buffer is ordered on it); dev_alloc returns NULL on
     * failure (qr_init then fails with QR_ENOMEM). Both NULL (the default):
     * cudaMallocAsync / cudaFreeAsync on the context's stream. A caller
     * running under another allocator (a framework's caching allocator, a
     * fixed pool) passes its own pair; the Python binding passes PyTorch's. */
    void* (*dev_alloc)(size_t bytes, void* stream, void* alloc_user);
    void (*dev_free)(void* ptr, void* stream, void* alloc_user);
    void* alloc_user;
} qr_opts;

/* Creates a context: validates the problem, enumerates Gamma, allocates the
 * device state and sets alpha = 0 (ybar == 0 start).
 *   d in [1, 12] (index sets of Z^d, kinds 0-2, and the unfolded cosine route:
 *   d <= 8; a cosine set with d > 8 runs on the direct route); N in [1, 256];
 *   T > 0; b: d doubles (host); sigma: d*d doubles,
 *   row-major (host), X_{j+1} = X_j + b dt + sigma sqrt(dt) Z; every |k_l| <= 32767
 *   for d <= 4 and <= 127 above (QR_ENOTIMPL otherwise, or when the generic
 *   kernels' per-lane power tables and coefficient rows exceed shared memory);
 *   the direct cosine route has its own limits (see the index-set kinds).
 *   opts may be NULL: M = 2^14, seed 1, QR_FP64, no truncation. */
qr_status qr_init(qr_ctx** out, int d, int N, double T, const qr_nu* nu, const qr_gamma* gamma,
                  const double* b, const double* sigma, const qr_fn* f, const qr_fn* g,
                  const qr_opts* opts);

/* Runs n_iter Jacobi-Picard iterations: every row i in [0, N) is recomputed
 * from the previous iterate (Algorithm 1's projection for all i at once).
 * residual_out (host, nullable): max_{i,k} |alpha^(q) - alpha^(q-1)| of the
 * last iteration. Blocks until the work is done. */
qr_status qr_picard_step(qr_ctx* ctx, int n_iter, double* residual_out);

/* Algorithm 1 as printed: backward sweep i = N-1 .. 0, each row projected
 * with the rows above it already final. Equals N Picard iterations. */
qr_status qr_backward_sweep(qr_ctx* ctx);

/* ybar_i at n points: y[p] = Re sum_k alpha_{i,k} phi_k(x_p) for 0 <= i < N,
 * g(x_p) for i = N. x: n*d doubles (row per point), y: n doubles; both host
 * (ptr_kind = QR_HOST) or both device (QR_DEVICE). Blocks until done. */
qr_status qr_eval(qr_ctx* ctx, int i, const double* x, long long n, double* y_out, int ptr_kind);

/* |Gamma| and the list of k (|Gamma|*d ints, host, canonical order). */
qr_status qr_gamma_size(const qr_ctx* ctx, int* n_gamma);
qr_status qr_gamma_list(const qr_ctx* ctx, int* k_out);

/* alpha: N*|Gamma| complex as interleaved (re, im) doubles, row i = time index
 * i, canonical Gamma order (host). set_coefs expects conjugate symmetry
 * alpha_{-k} = conj(alpha_k) and reads only k = 0 and the half k > 0. For a
 * cosine context (kinds 3-5) the values are the real cosine coefficients a_k
 * on Gamma (imaginary parts 0 on output, ignored on input). */
qr_status qr_get_coefs(const qr_ctx* ctx, double* alpha_out);
qr_status qr_set_coefs(qr_ctx* ctx, const double* alpha_in);

/* Responses S_i^m (m = 0..M-1) of row i from the last iteration (host). */
qr_status qr_get_responses(const qr_ctx* ctx, int i, double* S_out);

typedef struct {
    long long iterations;       /* Picard iterations (or sweeps) run */
    long long clamp_hits;       /* truncations T_L applied, all iterations */
    long long nonfinite;        /* non-finite responses, all iterations */
    double ms_paths;            /* device time of the path-and-series kernel (events) */
    double ms_project;          /* device time of the projection kernel */
    double ms_reduce;           /* device time of the cross-block reduction */
    long long launches_paths, launches_project, launches_reduce;
} qr_stats_t;
/* Kernel timing is recorded only when enabled (events cost a little). */
qr_status qr_set_profiling(qr_ctx* ctx, int on);
qr_status qr_get_stats(const qr_ctx* ctx, qr_stats_t* out);

const char* qr_last_error(const qr_ctx* ctx);
const char* qr_status_string(qr_status s);
void qr_destroy(qr_ctx* ctx);

/* n test points of time index i, nu-distributed and independent of the
 * clouds (Philox tag 2, counter (p, c, 0xffffffff, ...)): x_out is n*d
 * doubles, host. They serve the accuracy reports of Sec. 5, eq. (mse):
 * MSE over 10^3 nu-points per time index. */
qr_status qr_test_points(const qr_ctx* ctx, int i, long long n, double* x_out);

/* Test hook (the paper has no counterpart): runs, on the context's stream,
 * one kernel whose bounded mbarrier wait cannot complete (an expected
 * transaction with no copy behind it). The wait gives up after about 2^31
 * SM cycles (~1 s), the kernel records the timeout in the context's status
 * word and returns, and this call returns QR_ETIMEOUT with the message of a
 * timed-out wait, exactly as a Picard step would. The status word is then
 * cleared: the context stays usable. Any other status is a failure of the
 * mechanism. */
qr_status qr_selftest_wait_timeout(qr_ctx* ctx);

/* Host-side fault injection (the paper has no counterpart): arms one fault
 * on the context, taken once by the next call that reaches it, so that the
 * library's failure paths run without faulting the GPU:
 *   QR_FAULT_ALLOC   the context's next device allocation fails: that call
 *                    returns QR_ENOMEM (qr_init, qr_eval with host points,
 *                    qr_shard, qr_batch_create, ...);
 *   QR_FAULT_LAUNCH  the next qr_picard_step / qr_backward_sweep returns
 *                    QR_ECUDA before it launches anything;
 *   QR_FAULT_NAN     the next qr_picard_step / qr_backward_sweep first sets
 *                    the k = 0 coefficient of row N-1 to NaN (master row and
 *                    packed copies, the context's own buffers), so that the
 *                    path kernel's non-finite guard makes the call return
 *                    QR_ENONFINITE; qr_set_coefs then restores a state (with
 *                    N = 1 no series reads a coefficient row and the call
 *                    succeeds).
 * QR_FAULT_NONE disarms. The environment variable QR_FAULT = alloc, launch
 * or nan arms the same fault on every context at qr_init. A batch's
 * iteration (qr_batch_picard_step) does not take the iteration faults.
 * QR_EINVAL for a NULL context or an unknown kind. */
enum { QR_FAULT_NONE = 0, QR_FAULT_ALLOC = 1, QR_FAULT_LAUNCH = 2, QR_FAULT_NAN = 3 };
qr_status qr_inject_fault(qr_ctx* ctx, int kind);

/* ---- many instances in one iteration ----------------------------------
 * A batch advances n contexts (created by qr_init with QR_FP32, sharing one
 * stream, each with one of the compiled index-set classes: |k|_inf <= 4 in
 * d = 2; |k|_1 <= 5 (d = 3), 4 (d = 4, 5, 6), 3 (d = 6, 7, 8)) by Picard
 * iterations together. The path-and-series phase of all instances is one
 * persistent kernel launch pulling (instance, time index, path tiles) work
 * items, class by class and longest first within a class; instances that
 * share their sample points run the tensor-core kernel below; then ONE
 * finishing launch projects every (instance, row, chunk of paths), and the
 * last chunk of each row to finish reduces it (the same fixed-order sum as
 * qr_picard_step, so an instance on the persistent kernel ends with its single
 * run's coefficients bit for bit) and repacks its working rows. One iteration is one CUDA graph
 * launch of three kernels. Coefficients set with qr_set_coefs between batch
 * iterations are picked up by the next one. The first qr_batch_picard_step times a
 * few item sizes and grids and keeps the fastest (autotuning). The batch
 * does not own the contexts: destroy it before them. Results per instance
 * are read with qr_get_coefs etc. max_residual (nullable): the largest
 * residual over the instances. Contexts of the cosine basis (kinds 3-5)
 * are refused with QR_ENOTIMPL. */
typedef struct qr_batch qr_batch;
qr_status qr_batch_create(qr_batch** out, qr_ctx* const* ctxs, int n);
qr_status qr_batch_picard_step(qr_batch* b, int n_iter, double* max_residual);
/* the autotuned choice and the timings of the candidates (6 doubles, ms) */
qr_status qr_batch_info(const qr_batch* b, int* tiles_per_item, int* grid, double* tune_ms);
/* Instances that share their sample points -- same d, N, M, sigma, b, index
 * set, density, seed, Philox instance and start-point source, driver
 * QR_F_CUBIC_MANUF and g = QR_GT_COS, so that only a, s and the
 * coefficients differ -- see the same Euler paths and basis values. Sets of
 * at least min_group such instances (default 16; 0 turns grouping off) whose
 * index set has a compiled shared-point kernel (|k|_inf <= 4 in d = 2,
 * |k|_1 <= 3 in d = 6; N <= 64) are run by a tensor-core kernel: the series
 * of 32 instances at a tile of 128 points is one product Phi A with BF16
 * hi/lo split operands and FP32 accumulation (about 2^-16 relative error per
 * product), instead of one tree evaluation per instance. Such instances do
 * not count clamp hits (qr_stats_t.clamp_hits stays 0 for them). Must be
 * called before the first qr_batch_picard_step; QR_EINVAL after it. */
qr_status qr_batch_set_grouping(qr_batch* b, int min_group);
/* number of shared-point groups and of the instances they hold */
qr_status qr_batch_groups(const qr_batch* b, int* n_groups, int* n_grouped);
const char* qr_batch_last_error(const qr_batch* b);
void qr_batch_destroy(qr_batch* b);

/* ---- learned warm start (no counterpart in the paper's algorithm) -------
 * A multilayer perceptron y = W_L(...gelu(x W_1 + b_1)...) + b_L with `depth`
 * hidden layers of `width` units (GELU, erf form) maps a row of inputs (for
 * the benchmark family: the wave vector s, sigma0, a and t_i) to a
 * coefficient row alpha_i (|Gamma| reals: alpha_0 and (re, im) of the half
 * set), used as the Picard iteration's start in place of y == 0. Training
 * is plain Adam on the mean squared error, in FP32, with the library's own
 * kernels (tiled GEMM with fused bias/GELU, GELU backward, Adam).
 * Buffers X (B x n_in), T and Y (B x n_out) are row-major FP32 device
 * arrays of the caller; B <= max_batch. Parameters are one flat FP32 array:
 * for each layer W (n_in x n_out, row-major) then b. All device work runs on
 * `stream` (NULL: the legacy default stream), so X and T must be ready in
 * that stream's order; qr_mlp_train_step returns without waiting (unless
 * loss_out is given), the other calls wait for the stream before returning.
 * Every call returns a qr_status; qr_mlp_last_error gives text. */
typedef struct qr_mlp qr_mlp;
qr_status qr_mlp_create(qr_mlp** out, int n_in, int width, int depth, int n_out, int max_batch,
                        unsigned long long seed, void* stream);
long long qr_mlp_num_params(const qr_mlp* m);
qr_status qr_mlp_get_params(const qr_mlp* m, float* out /* host, num_params */);
qr_status qr_mlp_set_params(qr_mlp* m, const float* in /* host, num_params */);
qr_status qr_mlp_forward(qr_mlp* m, const float* X, int B, float* Y);
/* gradient of mean((Y - T)^2) with respect to the parameters (host array
 * grad_out, nullable) and the loss (host, nullable); parameters unchanged */
qr_status qr_mlp_gradients(qr_mlp* m, const float* X, const float* T, int B, float* grad_out, float* loss_out);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on a batch */
qr_status qr_mlp_train_step(qr_mlp* m, const float* X, const float* T, int B, float lr, float* loss_out);
const char* qr_mlp_last_error(const qr_mlp* m);
void qr_mlp_destroy(qr_mlp* m);

/* ---- test hooks (no context) ------------------------------------------ */

/* Host-only test hook: the coefficient layout of the compile-time tree
 * kernels for the |k|_inf <= n (kind QR_G_LINF) or |k|_1 <= n (QR_G_L1) set
 * of Z^d, d in [1, 8], n in [1, 31]. Slot s of a packed row is the pair
 * (x, y) with x = sum_t coef[(2s)T + t] a[idx[(2s)T + t]] and y likewise at
 * 2s+1, T = *n_terms terms (idx -1: unused), where a is the master row as
 * 2|Gamma| doubles (re, im of alpha_k in canonical order). The slots follow
 * the traversal of the kernels: the root, then per dimension the chain
 * tree in Horner form, +-1 leaf pairs and mirrored chains of the last
 * dimension as coefficient pairs, the mirrored chains of the
 * QR_TREE_PAIR_LEVELS dimensions before it as sum and difference subtrees.
 * Call with idx = coef = NULL for *n_slots; then idx and coef hold
 * n_slots * 2 * n_terms entries. No device work. */
qr_status qr_tree_layout(int kind, int d, int n, int* n_slots, int* n_terms, int* idx, double* coef);

/* Philox4x32-10 on the device: ctr_key is n rows of 6 words (ctr0..3, key0,1),
 * out is n rows of 4 words (host arrays). */
qr_status qr_philox_words(const uint32_t* ctr_key, long long n, uint32_t* out);

/* The device sampler of paths m0 .. m0+n-1 of row i: d start uniforms
 * (u_out, n*d, exact doubles), d start points F_nu^{-1}(u) (x_out, n*d)
 * and the d normals of Euler step j (z_out, n*d), computed in `precision`
 * (QR_FP32 results are widened to double). Host arrays; any may be NULL.
 * QR_EINVAL for d outside 1..8. */
qr_status qr_sample(int d, const qr_nu* nu, unsigned long long seed, int instance, int i,
                    long long m0, long long n, int j, int precision, double* u_out,
                    double* x_out, double* z_out);

/* The d normals of Euler step j for paths m0 .. m0+n-1 of row i exactly as
 * the FP32 compile-time tree path kernels and the shared-point group kernel
 * draw them (Box-Muller on the same Philox words as qr_sample, Sec. 5
 * sampling; their own FP32 logarithm), widened to double: z_out is a host
 * array of n*d values. QR_EINVAL for d outside 1..8 or a NULL z_out. */
qr_status qr_sample_normals_tree(int d, unsigned long long seed, int instance, int i, long long m0, long long n,
                                 int j, double* z_out);

/* ---- one problem over several GPUs (Sec. 4's multi-GPU scheme) -------------
 * The paper splits the Monte-Carlo sum of eq. (Aqi:bar:M) over GPUs by paths
 * and reduces the per-GPU partial sums in a second level (Sec. 4). Here the
 * M paths of every row are cut into the projection's chunks, the chunks into
 * 8 fixed groups (group g = chunks [floor(g C/8), floor((g+1) C/8)), C chunks),
 * and the cross-chunk sum is always taken as: chunks in order within each
 * group, then the 8 group sums in order. A rank of a world of W ranks (W in
 * {1, 2, 4, 8}) owns groups [rank 8/W, (rank+1) 8/W): it simulates and projects
 * only the paths of those chunks, and the W ranks exchange their group sums
 * (kShardGroups x N x |Gamma_+| complex doubles, e.g. by an all-gather) once per
 * iteration. Every rank then holds the coefficients a single GPU computes,
 * bit for bit, whatever W.
 *
 * qr_shard_plan: the chunk and group ranges of `rank` (host arithmetic only;
 *   QR_EINVAL unless W divides 8, 0 <= rank < W and n_chunks >= 1).
 * qr_shard: restricts a context (Fourier basis) to its rank's chunks; W = 1
 *   undoes it. A context with W > 1 iterates by qr_picard_begin (paths,
 *   projection and the group sums of its own groups, asynchronous on the
 *   context's stream), the exchange of the group sums by the caller, and
 *   qr_picard_finish (the reduction from all 8 group sums, repack; blocks;
 *   residual_out as qr_picard_step). qr_picard_step, qr_backward_sweep,
 *   qr_project_static and batches refuse sharded contexts (QR_EINVAL).
 * qr_shard_groups: the device array of group sums (8 groups of
 *   bytes_per_group bytes, group-major, each N x |Gamma_+| double2 in
 *   canonical half-set order; nullable until qr_shard with W > 1) and this
 *   rank's groups [g_lo, g_hi). Before qr_picard_finish the caller fills the
 *   groups of the other ranks with theirs. Clamp and non-finite counts in
 *   qr_get_stats are this rank's share. */
qr_status qr_shard_plan(int n_chunks, int rank, int world, int* c_lo, int* c_hi, int* g_lo, int* g_hi);
qr_status qr_shard(qr_ctx* ctx, int rank, int world);
qr_status qr_shard_groups(const qr_ctx* ctx, void** gsum, long long* bytes_per_group, int* g_lo, int* g_hi);
qr_status qr_picard_begin(qr_ctx* ctx);
qr_status qr_picard_finish(qr_ctx* ctx, double* residual_out);

/* Test hook (the paper has no counterpart): one 128 x 32 x 64 product
 * D = A B^T on the 5th-generation tensor cores (tcgen05.mma, BF16 operands
 * staged in 128-byte swizzled shared memory, FP32 accumulator in tensor
 * memory, read back by tcgen05.ld) -- the building block of the shared-point
 * group kernel, checked against a product computed on the host.
 *   A: 128 x 64 BF16 (raw 16-bit patterns), row-major, host.
 *   B: 32 x 64 BF16, row-major, host.   D: 128 x 32 floats, row-major, host.
 * QR_ETIMEOUT if the tensor core never signalled completion (bounded wait),
 * QR_ECUDA on a CUDA error or misplaced tiles. Blocks until done. */
qr_status qr_tc_selftest(const uint16_t* A, const uint16_t* B, float* D);

/* ---- arithmetic peaks of this device (the paper has no counterpart) -----
 * The denominators of the rooflines the benchmark reports: the rate at which
 * the SMs of the current device retire fused multiply-adds, measured, not
 * derived from a lane count and a clock. A grid that fills every SM
 * (resident 256-thread CTAs x multiprocessors) runs 8 independent FMA chains
 * per thread, in launches of about 20 ms repeated for about `ms`
 * milliseconds (a few tens of ms: the burst rate; seconds: the rate the
 * power and thermal limits sustain), timed with CUDA events on `stream`
 * (cudaStream_t, NULL = default stream). No device setting is touched.
 *   kind:        QR_PEAK_FP32 (scalar FP32 FMA), QR_PEAK_FP32X2 (packed
 *                two-lane FP32 FMA, counted as two), QR_PEAK_FP64,
 *                QR_PEAK_FP32MIX (half the chains scalar, half packed,
 *                interleaved: both FP32 instruction forms in flight).
 *   tflops_out:  2 flop per FMA / elapsed time, in TFLOP/s (host, nullable).
 *   ms_out:      elapsed device time of the timed launches (host, nullable).
 *   sm_count_out: multiprocessors of the current device (host, nullable).
 * Allocates a small result buffer on the stream (one value per thread).
 * Blocks until done. QR_EINVAL for an unknown kind or ms outside (0, 60000]. */
enum { QR_PEAK_FP32 = 0, QR_PEAK_FP32X2 = 1, QR_PEAK_FP64 = 2, QR_PEAK_FP32MIX = 3 };
qr_status qr_fma_peak(int kind, double ms, void* stream, double* tflops_out, double* ms_out, int* sm_count_out);

/* ---- projection without device allocation -----------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory when they run it: code that owns a fixed
 * memory budget handed out up front, code running where a cudaMalloc could
 * block or fail at an unpredictable moment (a latency-bound serving loop, a
 * driver running under another framework's allocator). qr_picard_step keeps
 * its cross-block partial sums in memory the context allocated; this call
 * keeps them in a fixed array compiled into libqrmc instead (16 MiB per GPU
 * that loads the library, held until the process exits), so it allocates
 * nothing itself.
 *
 * Computes coefficient rows i in [i_lo, i_hi) from responses S given by the
 * caller: alpha_{i,k} = (1/M) sum_m S_i^m conj(phi_k(U_i^m)), with the start
 * uniforms U regenerated from the context's seed, by the same kernel the
 * projection inside qr_picard_step runs for this context (the compiled tiled
 * projection when one covers the index set, else the table-driven one).
 * The work runs on the context's device, which the call makes current for
 * its duration (the caller's current device is restored).
 *   S:         device array, (i_hi - i_lo) rows of M responses, row-major, in
 *              the context's precision (float for QR_FP32, double for QR_FP64).
 *   alpha_out: device array, (i_hi - i_lo) rows of |Gamma| complex values as
 *              interleaved (re, im) doubles, canonical order.
 * Requires (i_hi - i_lo) * n_chunks * (|Gamma|+1)/2 <= 2^20 partial sums,
 * n_chunks = ceil(M / chunk) <= 256; otherwise returns QR_EINVAL with the
 * sizes in qr_last_error (project fewer rows per call). Contexts of the
 * cosine basis (kinds 3-5) return QR_ENOTIMPL.
 * The call is asynchronous on the context's stream. The first call on a
 * device looks up the device address of the fixed array (once per device);
 * make that first call before any stream capture. Every call on a GPU shares
 * the one array, and each call overwrites every slot it reads, so nothing
 * carries over between calls; calls that can overlap on the GPU (different
 * streams or contexts, or several host threads) race on it. */
qr_status qr_project_static(qr_ctx* ctx, const void* S, int i_lo, int i_hi, double* alpha_out);

#ifdef __cplusplus
}
#endif
#endif
