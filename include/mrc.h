/*
 * mrc.h -- C ABI of libmrc: FFT-Newton inversion of matrix-valued sequences
 * and the Markov renewal functionals derived from it, on one NVIDIA GB300.
 *
 * Method: Kordalis & Trevezas, "Algebraic and FFT-Based Methods for
 * Discrete-Time Matrix Convolutions with Applications to Semi-Markov Models"
 * (arXiv 2605.30379).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - A matrix-valued sequence X in S_{r,c} (Section 2) truncated to k < N is an
 *   array of N*r*c doubles, row-major per coefficient, time slowest:
 *       X[k*r*c + i*c + j] = X(k)_{ij}.
 * - Array arguments are DEVICE pointers owned by the caller unless stated
 *   otherwise.  They must stay valid until the work queued on `stream` has
 *   finished.  Outputs must not alias inputs.
 * - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *   stream.  Every call only enqueues work on `stream` and returns, except
 *   where `report` (host pointer) is non-NULL: then the call synchronises the
 *   stream, reads the device status word and fills `report`.
 * - Host-side argument errors are returned before anything is enqueued.
 *   Errors found on the device (a singular A(0)) are written to a status word
 *   in the context; they are returned by a call with a non-NULL report, or by
 *   mrc_sync_status().  No C++ exception crosses this boundary.
 * - One context per host thread; a context is bound to the device it was
 *   created on.  The context owns its workspace (device memory, grown on
 *   demand up to max_workspace_bytes) and the twiddle tables.
 * - Sizes: 1 <= d <= 512, 1 <= N <= 2^20; calls whose workspace would exceed
 *   the context cap return MRC_ERR_NO_MEMORY.
 */
#ifndef MRC_H
#define MRC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrc_ctx mrc_ctx;

typedef enum {
    MRC_OK = 0,
    MRC_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer or option */
    MRC_ERR_SINGULAR_A0 = 2,   /* A(0) singular: no convolutional inverse (Theorem 2.2) */
    MRC_ERR_NO_MEMORY = 3,     /* workspace above the context cap or cudaMalloc failed */
    MRC_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed */
    MRC_ERR_NOT_CONVERGED = 5, /* refinement left max|rho| above target_residual */
    MRC_ERR_TIMEOUT = 6,       /* a bounded device wait gave up (the tensor-core product's mbarrier waits) */
    MRC_ERR_UNIMPLEMENTED = 7
} mrc_status;

typedef enum {
    MRC_FP64 = 0,  /* every stage in IEEE binary64 on the FP64 pipes */
    MRC_MIXED = 1  /* FP32 Newton + double-float (FP32-pair) residual refinement */
} mrc_precision;

typedef struct {
    int prec;               /* mrc_precision */
    int refine_sweeps;      /* MRC_MIXED: residual/correction sweeps (default 1, max 4) */
    double target_residual; /* MRC_MIXED with a report: max|rho_L| bound checked after refinement (0 = no check) */
    int autotune;           /* 1: pick the per-frequency product kernel (FP32-pipe tile 16/32/64, or the
                               tensor-core kernel for double-float) by timing each candidate once per
                               (precision, shape, transform size) on the call's own stream; choices are
                               kept in the context and, if MRC_AUTOTUNE_CACHE names a file, loaded at
                               mrc_create and written at mrc_destroy.  Batched calls tune before capture. */
} mrc_options;

typedef struct {
    double res_left_l1;   /* sum_k ||rho_L(k)||_F over k < N (Frobenius form of ||.||_{1,N}) */
    double res_right_l1;  /* same for rho_R, when computed; else -1 */
    double res_max_abs;   /* max_{k,i,j} |rho_L(k)_{ij}| (or of rho_R when only R was asked) */
    int levels;           /* Newton doubling levels run */
    int sweeps;           /* refinement sweeps run */
    double ms;            /* device time of the call (CUDA events) */
} mrc_report;

/* Library and status helpers. */
const char *mrc_status_string(mrc_status s);
const char *mrc_version(void);

/* Create a context on `device` (cudaSetDevice is called).  max_workspace_bytes
 * caps the device workspace (0 = no cap).  *ctx receives an owned handle. */
mrc_status mrc_create(mrc_ctx **ctx, int device, size_t max_workspace_bytes);

/* Free the context's workspace and handle.  Synchronises the device first. */
mrc_status mrc_destroy(mrc_ctx *ctx);

/* Synchronise `stream`, return and clear the context's device status word. */
mrc_status mrc_sync_status(mrc_ctx *ctx, void *stream);

/* Bytes of workspace mrc_inverse would use for (d, N, prec). */
size_t mrc_inverse_workspace_bytes(int d, int64_t N, int prec);

/*
 * mrc_inverse -- psi = A^{(-1)} mod x^N in the truncated algebra A_{d,N}
 * (Proposition 2.3), by Newton doubling B_{r+1} = B_r * (2 e0 - A * B_r)
 * mod x^{2^{r+1}} (Eq. (newton), Appendix D "Newton inversion") with the
 * products done by zero-padded FFT (Eq. (fft-convolution)) and B_0(0) = A(0)^{-1}
 * by Gauss-Jordan with partial pivoting.
 *   d, N    : matrix dimension and horizon.
 *   A       : device, [N][d][d] doubles, the sequence to invert; A(0) must be
 *             nonsingular.  For the Markov renewal sequence pass A = e0 - q.
 *   psi     : device, [N][d][d] doubles, receives the inverse.
 *   opt     : host, may be NULL (= MRC_FP64).  MRC_MIXED runs the Newton levels
 *             in FP32 and then `refine_sweeps` sweeps of
 *             psi <- psi + psi * (e0 - A * psi) with the residual in double-float.
 *   stream  : cudaStream_t.
 *   report  : host, may be NULL; if set, the call synchronises, fills levels,
 *             sweeps and ms, and (MRC_MIXED with target_residual > 0) the final
 *             left residual norms.
 * Errors: MRC_ERR_INVALID_ARG, MRC_ERR_NO_MEMORY, MRC_ERR_CUDA, and with a
 * report MRC_ERR_SINGULAR_A0 / MRC_ERR_NOT_CONVERGED.
 */
mrc_status mrc_inverse(mrc_ctx *ctx, int d, int64_t N, const double *A, double *psi,
                       const mrc_options *opt, void *stream, mrc_report *report);

/*
 * mrc_inverse_gj -- the same inverse psi = A^{(-1)} mod x^N by Gauss-Jordan
 * elimination on the augmented matrix [P_A(x) | I] over C[[x]]/<x^N>
 * (Appendix D "Gauss-Jordan inversion"; cost O(d^3 N log N), Proposition 2.4),
 * in FP64.  At column i the row r >= i whose series at (r, i) has the largest
 * constant coefficient in absolute value becomes row i (partial pivoting on
 * A(0), which ordinary Gauss-Jordan on A(0) shows to exist); the pivot series
 * is inverted by scalar Newton doubling (Eq. (newton) with d = 1), the row is
 * normalised and eliminated from the other rows, every truncated series
 * product by zero-padded FFT of length 2 pow2ceil(N) (Eq. (fft-convolution)).
 *   d       : 1 .. MRC_GJ_DMAX (the method's cost grows as d^3).
 *   N, A, psi, stream : as mrc_inverse.
 *   opt     : host, may be NULL; prec must be MRC_FP64; autotune as mrc_inverse.
 *   report  : host, may be NULL; if set the call synchronises and fills ms and
 *             levels (= d, the pivot steps).
 * Workspace: 2 N d^2 doubles for the augmented matrix, spectra of length
 * pow2ceil(N) for 2 d^2 + 3 d + 1 series, and the scalar inverse's buffers.
 * Errors: MRC_ERR_INVALID_ARG, MRC_ERR_NO_MEMORY, MRC_ERR_CUDA; a singular
 * A(0) fills psi with NaN and sets the status word (returned with a report,
 * else by mrc_sync_status).
 */
#define MRC_GJ_DMAX 64
mrc_status mrc_inverse_gj(mrc_ctx *ctx, int d, int64_t N, const double *A, double *psi,
                          const mrc_options *opt, void *stream, mrc_report *report);

/*
 * mrc_mre_solve -- the continuous-time Markov renewal equation
 * K = L + Q (Stieltjes-convolved) K on the grid t = m h (Section 4),
 * discretised by the endpoint mean-value rule (scheme 0, Eq. (mre-discrete)),
 *     K_h = (e0 - Qbar_h)^(-1) * [L_h - (1/2) Delta+ Q_h * (L_h(0) e0)]
 *                                                      (Eq. (mre-solution)),
 * with Delta Q_h(0) = O, Delta Q_h(m) = Q_h(m) - Q_h(m-1), Delta+ Q_h(m) =
 * Delta Q_h(m+1), Qbar_h = (Delta Q_h + Delta+ Q_h) / 2; or by the
 * process discretisation (scheme 1, Eq. (process-discretization)),
 *     K_h = (e0 - Delta Q_h)^(-1) * L_h.
 * L = Hbar (diag(1 - H_i)) gives the transition function P; the up-state
 * block of Q with L_i = 1 - H_i (i up) gives reliability; A(t) = alpha P 1_U
 * availability.
 *   d, c   : kernel dimension and number of right-hand-side columns (<= 512).
 *   N      : number of output coefficients m = 0 .. N-1.
 *   Q      : device, [N+1][d][d] doubles: Q_h(m) = Q(m h), m = 0 .. N (the
 *            extra sample feeds Delta+ Q_h(N-1)); Q(0) = O expected.
 *   L      : device, [N][d][c] doubles: L_h(m) = L(m h).
 *   scheme : 0 mean-value rule, 1 process discretisation.
 *   K      : device, [N][d][c] doubles, receives K_h.
 *   opt    : as mrc_inverse (MRC_MIXED: FP32 Newton levels, double-float
 *            residual sweep and product).
 * Errors: MRC_ERR_INVALID_ARG, MRC_ERR_NO_MEMORY, MRC_ERR_CUDA; a singular
 * e0 - Qbar_h(0) shows in the status word (mrc_sync_status).
 */
mrc_status mrc_mre_solve(mrc_ctx *ctx, int d, int c, int64_t N, const double *Q, const double *L, int scheme,
                         double *K, const mrc_options *opt, void *stream);

/*
 * mrc_inverse_host -- the same inverse as mrc_inverse (same kernels, same
 * results) for a sequence that lives in host memory, with the transfers in
 * the call: A is uploaded in the row ranges the Newton doubling consumes
 * (level m of Eq. (newton) reads A(0) .. A(2m-1), Section 3), on an
 * internal copy stream, so that the first levels start while the rest of A
 * is still in transit; psi is copied back on `stream` after the last sweep.
 *   A_host  : host, [N][d][d] doubles.  Pinned (page-locked) memory lets the
 *             uploads overlap the kernels; pageable memory works too, with
 *             the copies serialised by the CUDA runtime.
 *   psi_host: host, [N][d][d] doubles, written when the call's work on
 *             `stream` completes (synchronise `stream`, or pass a report).
 *   d, N, opt, stream, report: as mrc_inverse.  The device copies of A and
 *             psi live in the context workspace (2 N d^2 doubles more than
 *             mrc_inverse_workspace_bytes).
 * Errors: as mrc_inverse.
 */
mrc_status mrc_inverse_host(mrc_ctx *ctx, int d, int64_t N, const double *A_host, double *psi_host,
                            const mrc_options *opt, void *stream, mrc_report *report);

/*
 * mrc_inverse_batched -- mrc_inverse over `nmodels` independent models with
 * their own d[b] and N[b] (host arrays), A[b]/psi[b] device pointers held in
 * HOST arrays of pointers (no counterpart in the paper beyond applying
 * Eq. (newton) to each model).
 * Scheduling, stage by stage: every launch covers all models of a wave at
 * one stage -- one launch per FFT pass of each Newton level size m (every
 * model with m0 <= m < N at once, whatever its d), one per FP32-pipe product
 * tile configuration, one for all Gauss-Jordan inverses of the A(0), one for
 * the direct recursions, one per conversion; the tensor-core products
 * (square 32 <= d, one CTA per SM) run model after model.  The residual and
 * correction stages group models by transform length pow2ceil(N).  Models
 * enter waves in decreasing cost (~ N d^2 (log2 N + d)) while the waves'
 * buffers (mrc_inverse_workspace_bytes per model) fit the budget: the
 * context cap if set, else min(192 GB, three quarters of the device memory
 * free besides the workspace), at least the largest model.  The whole batch is captured once into a CUDA
 * graph; a later call with the same (d, N, A, psi, prec, sweeps) lists
 * replays it with one launch on `stream`.  The context keeps the 8 most
 * recent graphs, and a workspace reallocation discards them.  The
 * launch-count counter counts kernels at capture time only.
 * report (nullable, host) receives one mrc_report per model (ms = the whole
 * batch); with a report the call synchronises and returns the first nonzero
 * per-model status (e.g. MRC_ERR_SINGULAR_A0).
 */
mrc_status mrc_inverse_batched(mrc_ctx *ctx, int nmodels, const int *d, const int64_t *N,
                               const double *const *A, double *const *psi,
                               const mrc_options *opt, void *stream, mrc_report *report);

/*
 * mrc_residual -- left and right residuals of a computed inverse
 * (Proposition 2.6; the accuracy check of Section 5):
 *   rho_L = e0 - A * psi,  rho_R = e0 - psi * A,  k < N,
 * computed by FFT in double-float (prec MRC_MIXED) or FP64 (MRC_FP64).
 *   sides     : 1 = left only, 2 = right only, 3 = both.
 *   rho_left, rho_right : device [N][d][d] doubles or NULL (norms only).
 *   report    : host, may be NULL; if set the call synchronises and fills
 *               res_left_l1 / res_right_l1 / res_max_abs.
 */
mrc_status mrc_residual(mrc_ctx *ctx, int d, int64_t N, const double *A, const double *psi, int sides,
                        double *rho_left, double *rho_right, int prec, void *stream, mrc_report *report);

/*
 * mrc_transition -- transition probabilities P = psi * Hbar
 * (Eq. (transition-discrete)), with the survival diagonal
 * Hbar(k) = diag(1 - sum_j sum_{l=1..k} q_ij(l)) built on the device.
 *   psi : device [N][d][d], the Markov renewal sequence (e0 - q)^{(-1)}.
 *   q   : device [N][d][d], the discrete semi-Markov kernel (q(0) = 0).
 *   P   : device [N][d][d], output.
 *   prec: MRC_FP64 or MRC_MIXED (double-float convolution).
 */
mrc_status mrc_transition(mrc_ctx *ctx, int d, int64_t N, const double *psi, const double *q, double *P,
                          int prec, void *stream);

/*
 * mrc_first_entrance -- first entrance into D (Eqs. (first-entrance-mass),
 * (first-entrance-cdf)): g_D = (e0^C - q_CC)^{(-1)} * q_CD,
 * G_D(k) = sum_{l<=k} g_D(l), F_D(k) = alpha_C G_D(k) 1_D, S_D = 1 - F_D.
 * Reliability is S_D with D the failed states.
 *   q       : device [N][d][d] kernel.
 *   D, nD   : HOST array of nD distinct state indices in [0, d); C is the
 *             complement in increasing order.  1 <= nD < d.
 *   alpha_C : device [|C|] initial distribution on C.
 *   g       : device [N][|C|][|D|] or NULL.
 *   F, S    : device [N] or NULL.
 *   opt     : precision of the inverse of e0^C - q_CC (as mrc_inverse) and of
 *             the product with q_CD.
 */
mrc_status mrc_first_entrance(mrc_ctx *ctx, int d, int64_t N, const double *q, const int *D, int nD,
                              const double *alpha_C, double *g, double *F, double *S,
                              const mrc_options *opt, void *stream);

/*
 * mrc_occupation -- occupation probability A_B(k) = alpha P(k) 1_{E,B}
 * (Table 2); availability when B is the set of up states.
 *   P     : device [N][d][d];  alpha : device [d];
 *   B, nB : HOST list of states in B;  out : device [N].
 */
mrc_status mrc_occupation(mrc_ctx *ctx, int d, int64_t N, const double *P, const double *alpha,
                          const int *B, int nB, double *out, void *stream);

/*
 * mrc_reward -- reward-type functional V = psi * r (Eq. (reward)): the
 * solution of V = r + q * V with a rectangular right-hand side.
 *   psi : device [N][d][d], the Markov renewal sequence.
 *   r   : device [N][d][c] reward sequence (c >= 1 columns).
 *   V   : device [N][d][c] output.
 *   prec: MRC_FP64 or MRC_MIXED (double-float convolution).
 */
mrc_status mrc_reward(mrc_ctx *ctx, int d, int c, int64_t N, const double *psi, const double *r, double *V,
                      int prec, void *stream);

/*
 * mrc_renewal_visits -- expected renewal visits to B counted from time 0,
 * Eq. (renewal-visits): out(k) = alpha sum_{l<=k} psi(l) I_B 1_s.
 *   psi   : device [N][d][d];  alpha : device [d];
 *   B, nB : HOST list of states in B;  out : device [N].
 */
mrc_status mrc_renewal_visits(mrc_ctx *ctx, int d, int64_t N, const double *psi, const double *alpha,
                              const int *B, int nB, double *out, void *stream);

/*
 * mrc_inverse_noalloc -- the FP64 inverse of mrc_inverse for callers that
 * cannot let a library allocate device memory: a process whose device memory
 * is already owned by another allocator's pool, code that forbids dynamic
 * allocation after initialisation, or a plugin host that only hands out
 * fixed buffers.  The paper has no counterpart; this is an interface variant
 * only.  It runs mrc_inverse's Newton schedule with the same FFT kernels and
 * the default FP64 product kernel (never an autotuned one), so its results
 * agree with mrc_inverse's to rounding.
 *   d, N, A, psi, stream : as mrc_inverse with prec = MRC_FP64.
 * Scratch: one fixed 64 MiB device array inside the library.  The call uses
 * 256 B + 512 KiB (twiddles) + 16 d^2 + 4 * 16 d^2 * M bytes of it, M being
 * the largest Newton level (< N); N must be <= 2^14.  Larger requests return
 * MRC_ERR_NO_MEMORY at once, with the limit printed to stderr.
 * No cudaMalloc/cudaFree or allocating library routine is called.
 * Initialisation: under CUDA's default lazy module loading, the array (and
 * the library's kernels) are mapped on a device only when first used there.
 * The first call on each device is therefore the initialisation step: it
 * resolves the array's device address (cudaGetSymbolAddress), which maps it,
 * and fills the twiddle table, synchronously.  Make that first call before
 * another allocator reserves the device's memory and before any stream
 * capture (or set CUDA_MODULE_LOADING=EAGER, which maps the array when the
 * library is loaded).  Once mapped, the array stays on that device until the
 * process exits.
 * Every call then clears the status word, enqueues the work on `stream`,
 * synchronises `stream` and returns MRC_OK or MRC_ERR_SINGULAR_A0.  All calls
 * share the array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU (two host threads, or two streams) race on it and must
 * be serialised by the caller.
 */
mrc_status mrc_inverse_noalloc(int d, int64_t N, const double *A, double *psi, void *stream);

/*
 * mrc_selftest_timeout -- failure-detection self-test (no counterpart in the
 * paper).  Enqueues on `stream` one thread that runs the bounded mbarrier
 * wait of the tensor-core product kernels on a barrier nothing arrives on;
 * after `spins` rounds of try_wait (each suspending for at most about 1 us)
 * it gives up and writes MRC_ERR_TIMEOUT to the context's status word, which
 * the next mrc_sync_status (or call with a report) returns and clears.
 * Nothing asynchronous is in flight in that kernel, so the context stays
 * usable afterwards.  1 <= spins <= 2^20, else MRC_ERR_INVALID_ARG.
 */
mrc_status mrc_selftest_timeout(mrc_ctx *ctx, int spins, void *stream);

/*
 * Instrumentation (no counterpart in the paper; used to report the roofline
 * of one kernel class measured inside a timed region).
 *
 * mrc_launch_count: number of CUDA kernel launches this library has issued
 * since it was loaded (all contexts).
 *
 * mrc_profile_begin(kclass): from now on, record a CUDA event pair on the
 * launching stream around every launch of kernel class `kclass`
 * (MRC_K_* below; 0 switches recording off) and accumulate the algorithmic
 * bytes and flops each launch is charged with (the per-unit figures in the
 * design notes).  mrc_profile_end synchronises the recorded events and returns
 * the summed device time (ms), the number of timed launches and the charged
 * bytes and flops, then switches recording off.  At most 8192 launches are
 * timed per begin/end; later launches are counted by mrc_launch_count only.
 * Launches on the context's side stream (the double-float spectrum of A and
 * the residual product's prepared X that a mixed inverse computes while its
 * Newton levels run) are not timed: they overlap the critical path, so their event
 * durations would include time spent waiting for SMs.  Not thread safe.
 */
#define MRC_K_FFT_F64 1
#define MRC_K_FFT_F32 2
#define MRC_K_FFT_DD 3
#define MRC_K_PAIR_F64 4
#define MRC_K_PAIR_F32 5
#define MRC_K_PAIR_DD 6
#define MRC_K_MISC 7
#define MRC_KCLASS_MAX 7
unsigned long long mrc_launch_count(void);
mrc_status mrc_profile_begin(int kclass);
mrc_status mrc_profile_end(double *ms_total, long long *launches, double *bytes, double *flops);

#ifdef __cplusplus
}
#endif
#endif /* MRC_H */
