// api.cu -- C ABI of libmrc and the host-side Newton driver.
//
// The driver only sequences kernels on the caller's stream; every arithmetic
// step of the method runs in the CUDA kernels of k_*.cu and misc.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <vector>

#include "../../include/mrc.h"
#include "mrc_internal.h"

#define MRC_TW_LOG 21  // twiddle tables cover transform lengths up to 2^21

// One captured batch: the CUDA graph of every model's kernels on the
// context's internal streams, replayed while the configuration is unchanged.
struct BatchGraph {
    std::vector<int> d;
    std::vector<int64_t> N;
    std::vector<const double *> A;
    std::vector<double *> psi;
    int prec = 0, sweeps = 0;
    void *ws = nullptr;  // the workspace the graph's buffers live in
    cudaGraphExec_t exec = nullptr;
};

#define MRC_BATCH_STREAMS 8

struct mrc_ctx {
    int device = 0;
    size_t cap = 0;        // 0 = unlimited
    void *ws = nullptr;    // workspace
    size_t ws_size = 0;
    void *tw[3] = {nullptr, nullptr, nullptr};
    int *d_status = nullptr;
    double *d_acc = nullptr;  // [4] norm accumulators
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // streams of the single-model mixed inverse, created on first use: the
    // FP32 Newton levels on `lvl` while the double-float spectrum of A (and
    // its prepared digit tiles) are computed on `aux`, both at the highest
    // priority
    cudaStream_t aux = nullptr, lvl = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    // host-buffer inverse: copy stream and one event per uploaded row range
    cudaStream_t cpy = nullptr;
    cudaEvent_t ev_cpy_fork = nullptr;
    cudaEvent_t ev_rows[32] = {};
    // batching
    cudaStream_t bst[MRC_BATCH_STREAMS] = {};
    cudaEvent_t bev[MRC_BATCH_STREAMS] = {};
    std::vector<BatchGraph> graphs;  // most recent last
    // autotuner of the per-frequency product kernel: key -> choice
    // (0..2: FP32-pipe tile configuration 16/32/64, 3: tensor-core kernel)
    std::map<uint64_t, int> tune;
    bool autotune = false;   // the current call asked for it
    bool capturing = false;  // a batch graph is being captured: no timing
    bool tune_dirty = false;
    // status word of the call being enqueued: d_status, or a batched model's
    // own word (bounded device waits write MRC_ERR_TIMEOUT there)
    int *cur_status = nullptr;
};

void mrc_prof_set_capturing(bool on);
void mrc_prof_set_untimed(cudaStream_t st);
bool mrc_prof_timing();
static mrc_status ensure_split_streams(mrc_ctx *c);

namespace {

struct PrecOps {
    cudaError_t (*fft)(const FftSrc &, const FftDst &, int64_t, int, int, void *, const void *, int, cudaStream_t,
                       int);
    cudaError_t (*pairmul)(const void *, const void *, void *, int64_t, int, int, int, const void *, int, cudaStream_t);
    cudaError_t (*pairmul_cfg)(const void *, const void *, void *, int64_t, int, int, int, int, const void *, int,
                               cudaStream_t);
    cudaError_t (*pairdiag)(const void *, const void *, void *, int64_t, int, int, const void *, int, cudaStream_t);
    cudaError_t (*twiddles)(void *, int, cudaStream_t);
    cudaError_t (*init)(void);
    size_t cxb;
};

const PrecOps OPS[3] = {
    {mrc_fft_f64, mrc_pairmul_f64, mrc_pairmul_cfg_f64, mrc_pairdiag_f64, mrc_twiddles_f64, mrc_init_f64, 16},
    {mrc_fft_f32, mrc_pairmul_f32, mrc_pairmul_cfg_f32, mrc_pairdiag_f32, mrc_twiddles_f32, mrc_init_f32, 8},
    {mrc_fft_dd, mrc_pairmul_dd, mrc_pairmul_cfg_dd, mrc_pairdiag_dd, mrc_twiddles_dd, mrc_init_dd, 16},
};

int64_t pow2ceil(int64_t x)
{
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Bump allocator over the context workspace.
struct Arena {
    char *base;
    size_t off = 0;
    void *take(size_t bytes)
    {
        void *p = base + off;
        off += align_up(bytes);
        return p;
    }
};

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) {                          \
            fprintf(stderr, "libmrc: %s -> %s\n", #call, cudaGetErrorString(e_)); \
            return MRC_ERR_CUDA;                          \
        }                                                 \
    } while (0)

mrc_status ensure_tw(mrc_ctx *c, int prec, cudaStream_t st)
{
    if (c->tw[prec]) return MRC_OK;
    void *p = nullptr;
    if (cudaMalloc(&p, OPS[prec].cxb << MRC_TW_LOG) != cudaSuccess) return MRC_ERR_NO_MEMORY;
    CK(OPS[prec].twiddles(p, MRC_TW_LOG, st));
    c->tw[prec] = p;
    return MRC_OK;
}

mrc_status ensure_ws(mrc_ctx *c, size_t need)
{
    if (need <= c->ws_size) return MRC_OK;
    if (c->cap && need > c->cap) return MRC_ERR_NO_MEMORY;
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);  // graphs hold workspace addresses
    c->graphs.clear();
    if (c->ws) {
        cudaDeviceSynchronize();
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_size = 0;
    }
    if (cudaMalloc(&c->ws, need) != cudaSuccess) {
        cudaGetLastError();
        return MRC_ERR_NO_MEMORY;
    }
    c->ws_size = need;
    return MRC_OK;
}

// ---------------------------------------------------------------------------
// Workspace plans
int64_t base_size(int d, int64_t N) { return mrc_base_size(d, N); }
int64_t newton_maxM(int d, int64_t N) { return mrc_newton_maxM(d, N); }

size_t ws_newton(int d, int64_t N, int prec)
{
    const size_t E = (size_t)d * d;
    size_t b = align_up(sizeof(double) * 2 * E);  // Gauss-Jordan work
    const int64_t M = newton_maxM(d, N);
    b += 3 * align_up((size_t)M * E * OPS[prec].cxb) + align_up(mrc_fft_scratch_elems(M, (int)E) * OPS[prec].cxb);
    return b;
}

size_t ws_product(int64_t Mr, size_t EX, size_t EY, size_t EC, int prec)
{
    size_t cxb = OPS[prec].cxb;
    size_t emax = std::max(EX, std::max(EY, EC));
    return align_up(Mr * EX * cxb) + align_up(Mr * EY * cxb) + align_up(Mr * EC * cxb) +
           align_up(mrc_fft_scratch_elems(Mr, (int)emax) * cxb);
}

// Mixed inverse layout: [Gauss-Jordan work | double-float spectrum of A |
// its FFT scratch | psi_0 in binary32 | then either A in binary32 and the
// FP32 Newton buffers or, afterwards, rho_L (binary32) followed by the
// residual's two other double-float spectra or the FP32 correction's
// product buffers].
// The mixed inverse's residual product with X prepared once (the
// tensor-core double-float product, square 32 <= d <= 64)
bool xpre_used(int d) { return mrc_tcp_supported(d, d, d); }

size_t ws_inverse(int d, int64_t N, int prec)
{
    const size_t E = (size_t)d * d;
    if (prec == MRC_FP64) return ws_newton(d, N, PREC_F64);
    const int64_t Mr = pow2ceil(N);
    const size_t gj = align_up(sizeof(double) * 2 * E);
    const size_t ahat = align_up((size_t)Mr * E * 16) + align_up(mrc_fft_scratch_elems(Mr, (int)E) * 16);
    // psi_0 in binary32 (the FP32 Newton levels' output), kept to the end
    const size_t psi32 = align_up((size_t)N * E * sizeof(float));
    // the FP32 Newton levels: their binary32 copy of A and their buffers
    const size_t newton = align_up((size_t)N * E * sizeof(float)) + ws_newton(d, N, PREC_F32) - gj;
    // rho_L (binary32), the FP32 spectrum of psi_0 (hi parts of its
    // double-float one), then the residual's spectra of psi_0 and of the
    // product (double-float) or the correction's FP32 spectrum of rho,
    // product and FFT scratch
    const size_t refine = align_up((size_t)N * E * sizeof(float)) + align_up((size_t)Mr * E * 8) +
                          std::max(2 * align_up((size_t)Mr * E * 16),
                                   2 * align_up((size_t)Mr * E * 8) + align_up(mrc_fft_scratch_elems(Mr, (int)E) * 8));
    // the residual product's prepared X (digit tiles and scales of A's spectrum)
    const size_t xpre = xpre_used(d) ? align_up(mrc_tcp_prep_bytes(Mr, d)) + align_up(mrc_tcp_prep_scale_bytes(Mr)) : 0;
    return gj + ahat + xpre + psi32 + std::max(newton, refine);
}

// Product kernel choices: 0..2 and 4 the FP32-pipe tile configurations
// 16/32/64 and 24 (pairmul_cfg), 3 the tensor-core digit kernel: for square 32 <= d <= 64
// the pipelined one (pair_tc.cu; double-float or FP32), for double-float
// 64 < d <= 512 the tiled one (ozaki_tc.cu).
bool tensor_choice_exists(int prec, int r, int m, int c)
{
    if (prec == PREC_DD) return mrc_tc_supported(r, m, c);
    return prec == PREC_F32 && mrc_tcp_supported(r, m, c);
}

cudaError_t launch_tensor(mrc_ctx *cx, int prec, const void *zx, const void *zy, void *zc, int64_t M, int d,
                          const void *tw, cudaStream_t st)
{
    if (prec == PREC_F32) return mrc_pairmul_f32_tcp(zx, zy, zc, M, d, tw, MRC_TW_LOG, cx->cur_status, st);
    if (d <= 64) return mrc_pairmul_dd_tcp(zx, zy, zc, M, d, tw, MRC_TW_LOG, cx->cur_status, st);
    return mrc_pairmul_dd_tc(zx, zy, zc, M, d, tw, MRC_TW_LOG, cx->cur_status, st);
}

cudaError_t launch_choice(mrc_ctx *cx, int prec, int choice, const void *zx, const void *zy, void *zc, int64_t M,
                          int r, int m, int c, const void *tw, cudaStream_t st)
{
    if (choice == 3) return launch_tensor(cx, prec, zx, zy, zc, M, r, tw, st);
    return OPS[prec].pairmul_cfg(zx, zy, zc, M, r, m, c, choice, tw, MRC_TW_LOG, st);
}

uint64_t tune_key(int prec, int r, int m, int c, int64_t M)
{
    int l = 0;
    while (((int64_t)1 << l) < M) ++l;
    return ((uint64_t)prec << 40) | ((uint64_t)r << 30) | ((uint64_t)m << 20) | ((uint64_t)c << 10) | (uint64_t)l;
}

// Autotuned product kernel for (precision, r, m, c, log2 M): every candidate
// runs once to warm up and twice under CUDA events on the call's own buffers
// and stream; the fastest is cached in the context.  Candidates compute the
// same product (the tensor-core kernel only for double-float, where its
// accuracy matches), so whichever ran last leaves a valid result behind.
// Returns -1 (use the built-in choice) when tuning is off or a graph is being
// captured.
int tuned_choice(mrc_ctx *cx, int prec, const void *zx, const void *zy, void *zc, int64_t M, int r, int m, int c,
                 const void *tw, cudaStream_t st)
{
    if (!cx || !cx->autotune) return -1;
    const uint64_t key = tune_key(prec, r, m, c, M);
    auto it = cx->tune.find(key);
    if (it != cx->tune.end()) return it->second;
    if (cx->capturing) return -1;
    int cands[5] = {0, 1, 2, 4, 3};
    const int nc = tensor_choice_exists(prec, r, m, c) ? 5 : 4;
    float best = 1e30f;
    int pick = -1;
    for (int k = 0; k < nc; ++k) {
        if (launch_choice(cx, prec, cands[k], zx, zy, zc, M, r, m, c, tw, st) != cudaSuccess) continue;
        cudaEventRecord(cx->ev0, st);
        launch_choice(cx, prec, cands[k], zx, zy, zc, M, r, m, c, tw, st);
        launch_choice(cx, prec, cands[k], zx, zy, zc, M, r, m, c, tw, st);
        cudaEventRecord(cx->ev1, st);
        if (cudaEventSynchronize(cx->ev1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, cx->ev0, cx->ev1);
        if (ms < best) { best = ms; pick = cands[k]; }
    }
    cudaGetLastError();
    if (pick >= 0) {
        cx->tune[key] = pick;
        cx->tune_dirty = true;
    }
    return pick;
}

// Autotuned FFT plan for (precision, direction, source and destination
// kinds, entries, log2 M): the candidate radix splits (each pass at most
// 2^10 points) with the default or four entries per CTA, each run once to
// warm up and twice under CUDA events on the call's own buffers and stream,
// the fastest kept in the context.  Transforms whose destination accumulates
// (DST_REAL64_ADD) are not re-run and keep the built-in plan, as do calls
// while a graph is being captured.
uint64_t fft_key(int prec, const FftSrc &sx, const FftDst &dx, int64_t M, int E, int dir)
{
    int l = 0;
    while (((int64_t)1 << l) < M) ++l;
    return ((uint64_t)1 << 62) | ((uint64_t)prec << 56) | ((uint64_t)(dir > 0) << 55) | ((uint64_t)sx.mode << 52) |
           ((uint64_t)dx.mode << 48) | ((uint64_t)E << 8) | (uint64_t)l;
}

int fft_plan_choice(mrc_ctx *cx, int prec, const FftSrc &sx, const FftDst &dx, int64_t M, int E, int dir,
                    void *scratch, const void *tw, cudaStream_t st)
{
    if (!cx || !cx->autotune) return -1;
    const uint64_t key = fft_key(prec, sx, dx, M, E, dir);
    auto it = cx->tune.find(key);
    if (it != cx->tune.end()) return it->second;
    if (cx->capturing || dx.mode == DST_REAL64_ADD || (cx->aux && st == cx->aux)) return -1;
    int l = 0;
    while (((int64_t)1 << l) < M) ++l;
    std::vector<int> cands;
    const bool ec4_alt = (prec == PREC_F32 ? E >= 16 : E >= 8);  // four entries per CTA differ from the default
    if (l <= 10) {
        cands.push_back(0);
        if (ec4_alt) cands.push_back(256);
    } else {
        for (int a = std::max(1, l - 10); a <= std::min(10, l - 1); ++a) {
            cands.push_back(a);
            if (ec4_alt) cands.push_back(a | 256);
        }
    }
    float best = 1e30f;
    int pick = -1;
    for (int pl : cands) {
        if (OPS[prec].fft(sx, dx, M, E, dir, scratch, tw, MRC_TW_LOG, st, pl) != cudaSuccess) continue;
        cudaEventRecord(cx->ev0, st);
        OPS[prec].fft(sx, dx, M, E, dir, scratch, tw, MRC_TW_LOG, st, pl);
        OPS[prec].fft(sx, dx, M, E, dir, scratch, tw, MRC_TW_LOG, st, pl);
        cudaEventRecord(cx->ev1, st);
        if (cudaEventSynchronize(cx->ev1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, cx->ev0, cx->ev1);
        if (ms < best) { best = ms; pick = pl; }
    }
    cudaGetLastError();
    if (pick >= 0) {
        cx->tune[key] = pick;
        cx->tune_dirty = true;
    }
    return pick;
}

cudaError_t fft_any(mrc_ctx *cx, int prec, const FftSrc &sx, const FftDst &dx, int64_t M, int E, int dir,
                    void *scratch, const void *tw, cudaStream_t st)
{
    const int plan = fft_plan_choice(cx, prec, sx, dx, M, E, dir, scratch, tw, st);
    return OPS[prec].fft(sx, dx, M, E, dir, scratch, tw, MRC_TW_LOG, st, plan);
}

// The per-frequency product of one precision: the autotuned choice when the
// call asked for tuning, else the tensor-core digit kernels for square
// double-float products with 32 <= d <= 512 and square FP32 products with
// 32 <= d <= 64 on transforms of at least 256 points (fewer pairs than SMs
// below that), the FP32-pipe tiles elsewhere.
cudaError_t pairmul_any(mrc_ctx *cx, int prec, const void *zx, const void *zy, void *zc, int64_t M, int r, int m,
                        int c, const void *tw, cudaStream_t st)
{
    const int ch = tuned_choice(cx, prec, zx, zy, zc, M, r, m, c, tw, st);
    if (ch >= 0) return launch_choice(cx, prec, ch, zx, zy, zc, M, r, m, c, tw, st);
    if (tensor_choice_exists(prec, r, m, c) && (prec == PREC_DD || M >= 256))
        return launch_tensor(cx, prec, zx, zy, zc, M, r, tw, st);
    return OPS[prec].pairmul(zx, zy, zc, M, r, m, c, tw, MRC_TW_LOG, st);
}

// ---------------------------------------------------------------------------
// C = X * Y truncated to rows [0, N) (linear convolution via L = 2 Mr,
// Mr = pow2ceil(N)), X: [NX rows][r][m], Y: [NY rows][m][c] real FP64.
// Output: REAL64 rows [0, N) into `out` with scale s (and +I at row 0 if eye).
// preX / preT (optional): the spectrum of X already computed into preX (length
// Mr, EX entries, this precision) and the FFT scratch to use instead of a new
// one; y_hi (double-float only, optional): also write the hi parts of Y's
// spectrum there as FP32 complex values.
// y_mode: SRC_REAL64 or SRC_REAL32 rows of Y; out_mode >= 0 overrides the
// destination (DST_REAL32, or DST_REAL64_BASE32 with out_base).
mrc_status conv_product(mrc_ctx *c, Arena &ar, int prec, const double *X, int64_t NX, const void *Y, int64_t NY,
                        int r, int m, int cc, int64_t N, void *out, double sign, int eye_d, int add,
                        bool diag, cudaStream_t st, void *preX = nullptr, void *preT = nullptr,
                        void *y_hi = nullptr, int y_mode = SRC_REAL64, int out_mode = -1,
                        const float *out_base = nullptr, const void *xpt = nullptr, const void *xps = nullptr)
{
    const PrecOps &op = OPS[prec];
    const int64_t Mr = pow2ceil(N);
    // diag: X is r x cc, Y is a cc-vector per time index
    const size_t EX = diag ? (size_t)r * cc : (size_t)r * m, EY = diag ? (size_t)cc : (size_t)m * cc;
    const size_t EC = (size_t)r * cc;
    const size_t emax = std::max(EX, std::max(EY, EC));
    void *bX = preX ? preX : ar.take(Mr * EX * op.cxb);
    void *bY = ar.take(Mr * EY * op.cxb);
    void *bC = ar.take(Mr * EC * op.cxb);
    void *bT = preT ? preT : ar.take(mrc_fft_scratch_elems(Mr, (int)emax) * op.cxb);
    const void *tw = c->tw[prec];
    FftSrc sx{SRC_REAL64, X, 0, std::min(NX, N), (int)EX, 0};
    FftSrc sy{y_mode, Y, 0, std::min(NY, N), (int)EY, 0};
    FftDst dx{DST_CPLX, bX, (int)EX, 0, 0, 0, 1.0, 0};
    FftDst dy{DST_CPLX, bY, (int)EY, 0, 0, 0, 1.0, 0, y_hi};
    if (!preX) CK(fft_any(c, prec, sx, dx, Mr, (int)EX, -1, bT, tw, st));
    CK(fft_any(c, prec, sy, dy, Mr, (int)EY, -1, bT, tw, st));
    if (diag) {
        CK(op.pairdiag(bX, bY, bC, Mr, r, cc, tw, MRC_TW_LOG, st));
    } else if (xpt) {  // double-float with X prepared (xpt: tiles, xps: scales)
        SegParams<PairArgs> P{};
        P.nseg = 1;
        P.a[0] = mrc_tcp_args(xpt, bY, bC, Mr, r, tw, MRC_TW_LOG);
        P.a[0].xs = xps;
        CK(mrc_tcp_seg(1, P, c->cur_status, st));
    } else {
        CK(pairmul_any(c, prec, bX, bY, bC, Mr, r, m, cc, tw, st));
    }
    FftSrc sc{SRC_CPLX, bC, 0, Mr, (int)EC, 0};
    FftDst dc{out_mode >= 0 ? out_mode : (add ? DST_REAL64_ADD : DST_REAL64), out, (int)EC, 0, N, 0,
              sign / (double)Mr, eye_d, nullptr, out_base};
    CK(fft_any(c, prec, sc, dc, Mr, (int)EC, +1, bT, tw, st));
    return MRC_OK;
}

// The level transforms and products through the context: autotuned or built-in choices.
cudaError_t level_fft(void *user, int prec, const FftSrc &sx, const FftDst &dx, int64_t M, int E, int dir,
                      void *scratch, const void *tw, int, cudaStream_t st)
{
    return fft_any((mrc_ctx *)user, prec, sx, dx, M, E, dir, scratch, tw, st);
}

cudaError_t level_product(void *user, int prec, const void *zx, const void *zy, void *zc, int64_t M, int d,
                          const void *tw, int, cudaStream_t st)
{
    return pairmul_any((mrc_ctx *)user, prec, zx, zy, zc, M, d, d, d, tw, st);
}

// Newton doubling levels in working precision `prec` over buffers taken
// from the context workspace (the schedule itself is mrc_newton_levels).
mrc_status newton_levels(mrc_ctx *c, Arena &ar, int prec, int d, int64_t N, const double *A, double *psi,
                         int64_t m0, int *levels, cudaStream_t st, const RowWait *rw = nullptr,
                         float *A32 = nullptr, float *psi32 = nullptr, int64_t a32_rows = 0)
{
    const PrecOps &op = OPS[prec];
    const int E = d * d;
    const int64_t Mmax = newton_maxM(d, N);
    if (levels) *levels = 0;
    if (Mmax == 0) return MRC_OK;
    NewtonBufs b;
    b.b0 = ar.take((size_t)Mmax * E * op.cxb);
    b.b1 = ar.take((size_t)Mmax * E * op.cxb);
    b.b2 = ar.take((size_t)Mmax * E * op.cxb);
    b.bt = ar.take(mrc_fft_scratch_elems(Mmax, E) * op.cxb);
    return (mrc_status)mrc_newton_levels(prec, d, N, A, psi, m0, b, c->tw[prec], MRC_TW_LOG, level_fft,
                                         level_product, c, st, rw, A32, psi32, levels, a32_rows);
}

bool valid_dN(int d, int64_t N) { return d >= 1 && d <= 512 && N >= 1 && N <= ((int64_t)1 << 20); }

// Mixed precision: the double-float spectrum of A that every residual sweep
// uses, and the residual product's prepared X, depend on A alone.  With
// `split` (single-model calls) they are computed on the context's side
// stream while the FP32 Newton levels run on its other one -- the
// double-float FFT and the digit split keep the FP32 pipes busy, the FP32
// passes mostly wait on memory; at equal priorities (d = 64, N = 2^18: step
// 209.9 ms, against 216.7 with the side stream at the lowest priority, where
// its work ran only in the gaps the levels left and finished late) -- and
// `st` waits for both before the first residual.  Without `split` everything
// runs on `st`.
mrc_status inverse_impl(mrc_ctx *c, Arena &ar, int d, int64_t N, const double *A, double *psi, int prec, int sweeps,
                        int *levels, cudaStream_t st, int *status = nullptr, bool split = false,
                        const RowWait *rw = nullptr)
{
    const size_t E = (size_t)d * d;
    struct StatusScope {  // bounded waits of this model report to its own word
        mrc_ctx *c;
        int *old;
        ~StatusScope() { c->cur_status = old; }
    } sscope{c, c->cur_status};
    c->cur_status = status ? status : c->d_status;
    double *gjw = (double *)ar.take(sizeof(double) * 2 * E);
    void *ahat = nullptr, *ascr = nullptr, *xpt = nullptr, *xps = nullptr;
    float *psi32 = nullptr, *A32 = nullptr;
    size_t mark = 0;
    int64_t a32_rows = 0;
    cudaStream_t sn = st;  // Newton levels
    if (prec == MRC_MIXED) {
        const int64_t Mr = pow2ceil(N);
        ahat = ar.take((size_t)Mr * E * 16);
        ascr = ar.take(mrc_fft_scratch_elems(Mr, (int)E) * 16);
        if (xpre_used(d)) {
            xpt = ar.take(mrc_tcp_prep_bytes(Mr, d));
            xps = ar.take(mrc_tcp_prep_scale_bytes(Mr));
        }
        // psi_0 is kept in binary32 (every entry the FP32 levels write is a
        // binary32 number; the first m0 rows are rounded to it), and the FP32
        // levels read a binary32 copy of A
        psi32 = (float *)ar.take((size_t)N * E * sizeof(float));
        mark = ar.off;
        A32 = (float *)ar.take((size_t)N * E * sizeof(float));
        if (!rw) {
            // A is resident: one conversion before the side stream starts (level by
            // level it ran beside the side stream's kernels and waited for SMs)
            CK(mrc_f64_to_f32(A, A32, N * (int64_t)E, st));
            a32_rows = N;
        }
        cudaStream_t sa = st;
        if (split) {
            CK(cudaEventRecord(c->ev_fork, st));
            CK(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
            CK(cudaStreamWaitEvent(c->lvl, c->ev_fork, 0));
            sa = c->aux;
            sn = c->lvl;
        }
        if (rw) CK(rw->wait(sa, N));
        FftSrc sx{SRC_REAL64, A, 0, N, (int)E, 0};
        FftDst dx{DST_CPLX, ahat, (int)E, 0, 0, 0, 1.0, 0};
        CK(fft_any(c, PREC_DD, sx, dx, Mr, (int)E, -1, ascr, c->tw[PREC_DD], sa));
        if (xpt) {  // the residual product's X: digit tiles and scales of A's spectrum
            SegParams<PairArgs> P{};
            P.nseg = 1;
            P.a[0] = mrc_tcp_args(ahat, nullptr, xpt, Mr, d, c->tw[PREC_DD], MRC_TW_LOG);
            P.a[0].xs = xps;
            CK(mrc_tcp_prep(P, sa));
        }
        if (split) CK(cudaEventRecord(c->ev_join, c->aux));
    }
    const int64_t m0 = base_size(d, N);
    if (rw) CK(rw->wait(sn, m0));
    CK(mrc_gauss_jordan(A, psi, gjw, d, status ? status : c->d_status, sn));
    CK(mrc_base_case(A, psi, d, m0, sn));
    if (psi32) CK(mrc_f64_to_f32(psi, psi32, m0 * (int64_t)E, sn));
    if (!psi32) mark = ar.off;
    mrc_status s = newton_levels(c, ar, prec == MRC_FP64 ? PREC_F64 : PREC_F32, d, N, A, psi, m0, levels, sn, rw,
                                 A32, psi32, a32_rows);
    if (s != MRC_OK) return s;
    ar.off = mark;
    if (prec == MRC_MIXED) {
        if (split) {
            CK(cudaEventRecord(c->ev_join2, c->lvl));
            CK(cudaStreamWaitEvent(st, c->ev_join2, 0));
            CK(cudaStreamWaitEvent(st, c->ev_join, 0));
        }
        float *rho32 = (float *)ar.take(sizeof(float) * (size_t)N * E);
        void *psi_hat32 = ar.take((size_t)pow2ceil(N) * E * 8);
        const size_t mark2 = ar.off;
        for (int sw = 0; sw < sweeps; ++sw) {
            ar.off = mark2;
            // rho_L = e0 - A * psi in double-float (Proposition 2.6), stored
            // in binary32 (the precision the FP32 correction reads it in);
            // the FFT of psi also leaves the FP32 spectrum the correction
            // needs.  The first sweep reads psi_0 from its binary32 copy.
            const bool first = sw == 0;
            s = conv_product(c, ar, PREC_DD, A, N, first ? (const void *)psi32 : psi, N, d, d, d, N, rho32, -1.0, d,
                             0, false, st, ahat, ascr, psi_hat32, first ? SRC_REAL32 : SRC_REAL64, DST_REAL32, nullptr,
                             xpt, xps);
            if (s != MRC_OK) return s;
            ar.off = mark2;
            // psi <- psi + psi * rho_L (Eq. (newton) from a full-length
            // approximation), FP32 product; the first sweep writes
            // psi = psi_0 + psi_0 * rho_L in FP64 from the binary32 psi_0
            s = conv_product(c, ar, PREC_F32, psi, N, rho32, N, d, d, d, N, psi, 1.0, 0, 1, false, st, psi_hat32,
                             nullptr, nullptr, SRC_REAL32, first ? DST_REAL64_BASE32 : DST_REAL64_ADD,
                             first ? psi32 : nullptr);
            if (s != MRC_OK) return s;
        }
    }
    return MRC_OK;
}

// Gauss-Jordan elimination over C[[x]]/<x^N> (Appendix D, "Gauss-Jordan
// inversion"; cost Proposition 2.4): W = [P_A(x) | I] in FP64, [N][d][2d].
// Column i: the row with the largest |constant coefficient| among rows >= i
// becomes row i; its pivot series u = W[i][i] is inverted by scalar Newton
// (the d = 1 Newton doubling of Eq. (newton)); the row is normalised,
// W[i][.] <- u^(-1) * W[i][.] mod x^N, and eliminated from every other row,
// W[r][.] <- W[r][.] - W[r][i] * W[i][.] mod x^N.  Every truncated product is
// a zero-padded FFT product of length 2 pow2ceil(N) (Eq. (fft-convolution)),
// over the whole augmented row (2d entries).  After d columns the right block
// is P_A(x)^(-1) mod x^N.
size_t ws_gj_series(int d, int64_t N)
{
    const int64_t Mr = pow2ceil(N);
    const size_t n2 = 2 * (size_t)d, EW = (size_t)d * n2;
    return align_up(256) + align_up(sizeof(double) * N * EW) + 2 * align_up(sizeof(double) * N) +
           align_up(sizeof(double) * N * d) + align_up((size_t)Mr * 16) + align_up((size_t)Mr * n2 * 16) +
           align_up((size_t)Mr * d * 16) + align_up((size_t)Mr * EW * 16) +
           align_up(mrc_fft_scratch_elems(Mr, (int)EW) * 16) + ws_inverse(1, N, MRC_FP64);
}

mrc_status gj_series_impl(mrc_ctx *c, Arena &ar, int d, int64_t N, const double *A, double *psi, cudaStream_t st)
{
    const int n2 = 2 * d, EW = d * n2;
    const int64_t Mr = pow2ceil(N);
    const void *tw = c->tw[PREC_F64];
    int *flags = (int *)ar.take(256);  // [0] pivot row, [1] singular flag
    double *W = (double *)ar.take(sizeof(double) * N * EW);
    double *u = (double *)ar.take(sizeof(double) * N), *v = (double *)ar.take(sizeof(double) * N);
    double *cv = (double *)ar.take(sizeof(double) * N * d);
    void *hv = ar.take((size_t)Mr * 16), *hr = ar.take((size_t)Mr * n2 * 16);
    void *hc = ar.take((size_t)Mr * d * 16), *hp = ar.take((size_t)Mr * EW * 16);
    void *bt = ar.take(mrc_fft_scratch_elems(Mr, EW) * 16);
    CK(mrc_gjs_init(A, W, d, N, flags + 1, st));
    for (int col = 0; col < d; ++col) {
        double *row = W + (size_t)col * n2;  // row col at every k: 2d entries, row stride EW
        CK(mrc_gjs_pivot(A, W, d, N, col, flags, u, cv, flags + 1, c->cur_status, st));
        // v = u^(-1) mod x^N (scalar Newton; its own workspace above this call's)
        const size_t mark = ar.off;
        mrc_status s = inverse_impl(c, ar, 1, N, u, v, MRC_FP64, 0, nullptr, st);
        if (s != MRC_OK) return s;
        ar.off = mark;
        // normalise: row <- v * row mod x^N
        FftSrc sv{SRC_REAL64, v, 0, N, 1, 0};
        FftSrc sr{SRC_REAL64, row, 0, N, EW, 0};
        FftDst dv{DST_CPLX, hv, 1, 0, 0, 0, 1.0, 0};
        FftDst dr{DST_CPLX, hr, n2, 0, 0, 0, 1.0, 0};
        CK(fft_any(c, PREC_F64, sv, dv, Mr, 1, -1, bt, tw, st));
        CK(fft_any(c, PREC_F64, sr, dr, Mr, n2, -1, bt, tw, st));
        CK(pairmul_any(c, PREC_F64, hv, hr, hp, Mr, 1, 1, n2, tw, st));
        FftSrc sp{SRC_CPLX, hp, 0, Mr, n2, 0};
        FftDst drow{DST_REAL64, row, EW, 0, N, 0, 1.0 / (double)Mr, 0};
        CK(fft_any(c, PREC_F64, sp, drow, Mr, n2, +1, bt, tw, st));
        // eliminate: W[r][.] -= cv[r] * row mod x^N for r != col (cv[col] = 0)
        FftSrc sc{SRC_REAL64, cv, 0, N, d, 0};
        FftDst dc{DST_CPLX, hc, d, 0, 0, 0, 1.0, 0};
        CK(fft_any(c, PREC_F64, sc, dc, Mr, d, -1, bt, tw, st));
        CK(fft_any(c, PREC_F64, sr, dr, Mr, n2, -1, bt, tw, st));
        CK(pairmul_any(c, PREC_F64, hc, hr, hp, Mr, d, 1, n2, tw, st));
        FftSrc se{SRC_CPLX, hp, 0, Mr, EW, 0};
        FftDst dw{DST_REAL64_ADD, W, EW, 0, N, 0, -1.0 / (double)Mr, 0};
        CK(fft_any(c, PREC_F64, se, dw, Mr, EW, +1, bt, tw, st));
    }
    CK(mrc_gjs_extract(W, psi, d, N, flags + 1, st));
    return MRC_OK;
}

mrc_status read_status(mrc_ctx *c, cudaStream_t st)
{
    int h = 0;
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(c->d_status, 0, sizeof(int)));
    return (mrc_status)h;
}

mrc_status residual_impl(mrc_ctx *c, Arena &ar, int d, int64_t N, const double *A, const double *psi, int sides,
                         double *rl, double *rr, int prec, cudaStream_t st, mrc_report *rep)
{
    const size_t E = (size_t)d * d;
    const int p = prec == MRC_FP64 ? PREC_F64 : PREC_DD;
    double *tmp = nullptr;
    if ((sides & 1 && !rl) || (sides & 2 && !rr)) tmp = (double *)ar.take(sizeof(double) * N * E);
    double h[4] = {-1, -1, -1, -1};
    if (sides & 1) {
        double *o = rl ? rl : tmp;
        const size_t mk = ar.off;
        mrc_status s = conv_product(c, ar, p, A, N, psi, N, d, d, d, N, o, -1.0, d, 0, false, st);
        if (s != MRC_OK) return s;
        ar.off = mk;
        if (rep) {
            CK(mrc_norms(o, (int)E, N, c->d_acc, st));
            CK(cudaMemcpyAsync(h, c->d_acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            rep->res_left_l1 = h[0];
            rep->res_max_abs = h[1];
        }
    }
    if (sides & 2) {
        double *o = rr ? rr : tmp;
        const size_t mk = ar.off;
        mrc_status s = conv_product(c, ar, p, psi, N, A, N, d, d, d, N, o, -1.0, d, 0, false, st);
        if (s != MRC_OK) return s;
        ar.off = mk;
        if (rep) {
            CK(mrc_norms(o, (int)E, N, c->d_acc, st));
            CK(cudaMemcpyAsync(h + 2, c->d_acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            rep->res_right_l1 = h[2];
            if (!(sides & 1)) rep->res_max_abs = h[3];
        }
    }
    return MRC_OK;
}

size_t ws_residual(int d, int64_t N, int prec, bool need_tmp)
{
    const size_t E = (size_t)d * d;
    const int p = prec == MRC_FP64 ? PREC_F64 : PREC_DD;
    return ws_product(pow2ceil(N), E, E, E, p) + (need_tmp ? align_up(sizeof(double) * N * E) : 0);
}

// The options' autotune flag holds for one API call.
struct TuneScope {
    mrc_ctx *cx;
    TuneScope(mrc_ctx *c, const mrc_options *o) : cx(c) { cx->autotune = o && o->autotune; }
    ~TuneScope() { cx->autotune = false; }
};

// Tune every product shape one model's inverse uses, on workspace buffers,
// before a batch graph is captured (timing is impossible during capture).
void pretune_model(mrc_ctx *cx, int prec, int d, int64_t N, char *buf, size_t bytes, cudaStream_t st)
{
    const size_t E = (size_t)d * d;
    auto one = [&](int p, int64_t M) {
        const size_t sz = align_up((size_t)M * E * OPS[p].cxb);
        if (3 * sz > bytes) return;
        tuned_choice(cx, p, buf, buf + sz, buf + 2 * sz, M, d, d, d, cx->tw[p], st);
    };
    const int pl = prec == MRC_FP64 ? PREC_F64 : PREC_F32;
    for (int64_t m = base_size(d, N); m < N; m <<= 1) one(pl, m);
    if (prec == MRC_MIXED) {
        one(PREC_DD, pow2ceil(N));
        one(PREC_F32, pow2ceil(N));
    }
}

void tune_load(mrc_ctx *cx)
{
    const char *path = getenv("MRC_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    unsigned long long k;
    int ch;
    while (fscanf(f, "%llu %d", &k, &ch) == 2)
        if (ch >= 0 && ch <= ((k >> 62) ? 511 : 4)) cx->tune[(uint64_t)k] = ch;  // FFT plans / product choices
    fclose(f);
}

void tune_save(mrc_ctx *cx)
{
    const char *path = getenv("MRC_AUTOTUNE_CACHE");
    if (!path || !cx->tune_dirty) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    for (auto &kv : cx->tune) fprintf(f, "%llu %d\n", (unsigned long long)kv.first, kv.second);
    fclose(f);
    cx->tune_dirty = false;
}

// ===========================================================================
// The batched inverse, stage by stage (mrc_inverse_batched): each launch of a
// stage covers every model of a wave at that stage -- one segmented launch
// per FFT pass and per product tile configuration, one batched launch for
// the Gauss-Jordan inverses of the A(0), one for the direct recursions and
// one per conversion.  The tensor-core products (persistent kernels over one
// product's frequency pairs, one CTA per SM) run model after model.  Models
// are taken in decreasing cost into waves whose buffers fit the workspace
// budget; inside a wave each model owns the buffers inverse_impl would give
// it, laid out the same way.

struct SegOps {
    cudaError_t (*build)(const FftSrc &, const FftDst &, int64_t, int, int, void *, const void *, int, FftPasses &);
    cudaError_t (*fft_seg)(int, const SegParams<FftArgs> &, unsigned, double, double, cudaStream_t);
    cudaError_t (*pair_seg)(int, const SegParams<PairArgs> &, unsigned, double, double, cudaStream_t);
};
const SegOps SOPS[3] = {
    {mrc_fft_build_f64, mrc_fft_seg_f64, mrc_pairmul_seg_f64},
    {mrc_fft_build_f32, mrc_fft_seg_f32, mrc_pairmul_seg_f32},
    {mrc_fft_build_dd, mrc_fft_seg_dd, mrc_pairmul_seg_dd},
};

struct BModel {
    int d = 0, E = 0;
    int64_t N = 0, m0 = 0, Mr = 0, Mmax = 0;
    const double *A = nullptr;
    double *psi = nullptr;
    int *status = nullptr;
    double cost = 0;
    size_t ws = 0;
    double *gjw = nullptr;
    float *A32 = nullptr, *psi32 = nullptr, *rho32 = nullptr;
    void *b0 = nullptr, *b1 = nullptr, *b2 = nullptr, *bt = nullptr;  // Newton level spectra and scratch
    void *ahat = nullptr, *ascr = nullptr;                              // double-float spectrum of A, scratch
    void *xpt = nullptr, *xps = nullptr;                                // its prepared digit tiles and scales
    void *psihat32 = nullptr, *rY = nullptr, *rC = nullptr;             // residual
    void *cY = nullptr, *cC = nullptr, *cT = nullptr;                   // correction
};

// the model's buffers from `base`, in inverse_impl's order (ws_inverse bytes)
void bmodel_layout(BModel &m, int prec, char *base)
{
    const size_t E = (size_t)m.E, Mr = (size_t)m.Mr, Mm = (size_t)m.Mmax, N = (size_t)m.N;
    Arena ar{base};
    m.gjw = (double *)ar.take(sizeof(double) * 2 * E);
    if (prec == MRC_FP64) {
        m.b0 = ar.take(Mm * E * 16);
        m.b1 = ar.take(Mm * E * 16);
        m.b2 = ar.take(Mm * E * 16);
        m.bt = ar.take(mrc_fft_scratch_elems(m.Mmax, m.E) * 16);
        return;
    }
    m.ahat = ar.take(Mr * E * 16);
    m.ascr = ar.take(mrc_fft_scratch_elems(m.Mr, m.E) * 16);
    if (xpre_used(m.d)) {
        m.xpt = ar.take(mrc_tcp_prep_bytes(m.Mr, m.d));
        m.xps = ar.take(mrc_tcp_prep_scale_bytes(m.Mr));
    }
    m.psi32 = (float *)ar.take(N * E * sizeof(float));
    const size_t mark = ar.off;
    m.A32 = (float *)ar.take(N * E * sizeof(float));
    m.b0 = ar.take(Mm * E * 8);
    m.b1 = ar.take(Mm * E * 8);
    m.b2 = ar.take(Mm * E * 8);
    m.bt = ar.take(mrc_fft_scratch_elems(m.Mmax, m.E) * 8);
    ar.off = mark;  // the levels' buffers are free once the levels are done
    m.rho32 = (float *)ar.take(N * E * sizeof(float));
    m.psihat32 = ar.take(Mr * E * 8);
    const size_t mark2 = ar.off;
    m.rY = ar.take(Mr * E * 16);
    m.rC = ar.take(Mr * E * 16);
    ar.off = mark2;  // the residual's spectra are free before the correction
    m.cY = ar.take(Mr * E * 8);
    m.cC = ar.take(Mr * E * 8);
    m.cT = ar.take(mrc_fft_scratch_elems(m.Mr, m.E) * 8);
}

struct FftJob {
    FftSrc src;
    FftDst dst;
    int E;
    void *scratch;
};

// One transform per job, all of packed length M and direction dir: one
// segmented launch per pass (in groups of MRC_SEG_MAX transforms)
mrc_status fft_stage(mrc_ctx *c, int prec, int64_t M, int dir, const std::vector<FftJob> &jobs, cudaStream_t st)
{
    if (jobs.empty()) return MRC_OK;
    std::vector<FftPasses> ps(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i)
        CK(SOPS[prec].build(jobs[i].src, jobs[i].dst, M, jobs[i].E, dir, jobs[i].scratch, c->tw[prec], MRC_TW_LOG,
                            ps[i]));
    auto P = std::make_unique<SegParams<FftArgs>>();
    for (int k = 0; k < ps[0].np; ++k)
        for (size_t i0 = 0; i0 < jobs.size(); i0 += MRC_SEG_MAX) {
            const size_t i1 = std::min(jobs.size(), i0 + (size_t)MRC_SEG_MAX);
            unsigned total = 0;
            double by = 0, fl = 0;
            P->nseg = (int)(i1 - i0);
            for (size_t i = i0; i < i1; ++i) {
                P->first[i - i0] = total;
                P->a[i - i0] = ps[i].a[k];
                total += ps[i].nchunk * ps[i].nrow[k];
                by += ps[i].bytes[k];
                fl += ps[i].flops[k];
            }
            CK(SOPS[prec].fft_seg(ps[0].logR[k], *P, total, by, fl, st));
        }
    return MRC_OK;
}

// the product kernel choice pairmul_any makes for a square d x d product of M points
int product_choice(mrc_ctx *cx, int prec, int64_t M, int d)
{
    if (cx->autotune) {
        auto it = cx->tune.find(tune_key(prec, d, d, d, M));
        if (it != cx->tune.end()) return it->second;
    }
    if (tensor_choice_exists(prec, d, d, d) && (prec == PREC_DD || M >= 256)) return 3;
    return d <= 16 ? 0 : (d <= 24 ? 4 : (d <= 32 ? 1 : 2));
}

struct PairJob {
    const void *zx, *zy;
    void *zc;
    int d;
    int *status;
    const void *xs = nullptr;  // double-float with X prepared: zx the tiles, xs the scales
};

// One square product per job, all of M points: the tensor-core ones of
// d <= 64 in one persistent segmented launch per K-chunk count ceil(d / 16),
// a timeout reported in the first product's status word;
// d > 64 model by model; the FP32-pipe ones in one segmented launch per tile
// configuration
mrc_status product_stage(mrc_ctx *c, int prec, int64_t M, const std::vector<PairJob> &jobs, cudaStream_t st)
{
    std::vector<size_t> bycfg[5], tcp[10];  // tensor-core groups: K-chunk count, + 5 with X prepared
    int *const old = c->cur_status;
    for (size_t i = 0; i < jobs.size(); ++i) {
        const int ch = jobs[i].xs ? 3 : product_choice(c, prec, M, jobs[i].d);
        if (ch == 3 && jobs[i].d <= 64) {
            tcp[(jobs[i].d + 15) / 16 + (jobs[i].xs ? 5 : 0)].push_back(i);
        } else if (ch == 3) {
            c->cur_status = jobs[i].status;
            const cudaError_t e = launch_tensor(c, prec, jobs[i].zx, jobs[i].zy, jobs[i].zc, M, jobs[i].d, c->tw[prec], st);
            c->cur_status = old;
            CK(e);
        } else {
            bycfg[ch].push_back(i);
        }
    }
    auto P = std::make_unique<SegParams<PairArgs>>();
    for (int g = 0; g < 10; ++g)
        for (size_t i0 = 0; i0 < tcp[g].size(); i0 += MRC_SEG_MAX) {
            const size_t i1 = std::min(tcp[g].size(), i0 + (size_t)MRC_SEG_MAX);
            P->nseg = (int)(i1 - i0);
            for (size_t q = i0; q < i1; ++q) {
                const PairJob &j = jobs[tcp[g][q]];
                P->first[q - i0] = 0;  // every product has the same pair count (same M)
                P->a[q - i0] = mrc_tcp_args(j.zx, j.zy, j.zc, M, j.d, c->tw[prec], MRC_TW_LOG);
                P->a[q - i0].xs = j.xs;
            }
            CK(mrc_tcp_seg(prec == PREC_DD, *P, jobs[tcp[g][i0]].status, st));
        }
    const int bsz[5] = {16, 32, 64, 0, 24};
    for (int cfg = 0; cfg < 5; ++cfg)
        for (size_t i0 = 0; i0 < bycfg[cfg].size(); i0 += MRC_SEG_MAX) {
            const size_t i1 = std::min(bycfg[cfg].size(), i0 + (size_t)MRC_SEG_MAX);
            unsigned total = 0;
            double by = 0, fl = 0;
            P->nseg = (int)(i1 - i0);
            for (size_t q = i0; q < i1; ++q) {
                const PairJob &j = jobs[bycfg[cfg][q]];
                PairArgs a{};
                a.zx = j.zx; a.zy = j.zy; a.zc = j.zc; a.tw = c->tw[prec]; a.tw_log = MRC_TW_LOG; a.M = M;
                int l = 0;
                while (((int64_t)1 << l) < M) ++l;
                a.logM = l;
                a.npairs = M >= 2 ? M / 2 + 1 : 1;
                a.r = a.m = a.c = j.d;
                const int nt = (j.d + bsz[cfg] - 1) / bsz[cfg];
                P->first[q - i0] = total;
                P->a[q - i0] = a;
                total += (unsigned)a.npairs * (unsigned)(nt * nt);
                by += (double)M * 3.0 * j.d * j.d * OPS[prec].cxb;
                fl += 8.0 * (double)j.d * j.d * j.d * (double)(M + 1);
            }
            CK(SOPS[prec].pair_seg(cfg, *P, total, by, fl, st));
        }
    return MRC_OK;
}

// The whole inverse of one wave of models, stage by stage
mrc_status batch_wave(mrc_ctx *c, std::vector<BModel> &W, int prec, int sweeps, cudaStream_t st)
{
    const int pl = prec == MRC_FP64 ? PREC_F64 : PREC_F32;
    const bool f32 = prec == MRC_MIXED;
    const size_t n = W.size();
    int dmax = 1;
    int64_t mmin = INT64_MAX, nmax = 0;  // mmin: the smallest first level (m0 < N: a power of two)
    for (auto &m : W) {
        dmax = std::max(dmax, m.d);
        if (m.m0 < m.N) mmin = std::min(mmin, m.m0);
        nmax = std::max(nmax, m.N);
    }
    // psi(0) = A(0)^(-1) and the direct recursion for psi(1 .. m0-1)
    {
        auto G = std::make_unique<SegParams<GjArgs>>();
        auto B = std::make_unique<SegParams<BaseArgs>>();
        for (size_t i0 = 0; i0 < n; i0 += MRC_SEG_MAX) {
            const size_t i1 = std::min(n, i0 + (size_t)MRC_SEG_MAX);
            G->nseg = B->nseg = (int)(i1 - i0);
            for (size_t i = i0; i < i1; ++i) {
                G->first[i - i0] = B->first[i - i0] = (unsigned)(i - i0);
                G->a[i - i0] = GjArgs{W[i].A, W[i].psi, W[i].gjw, W[i].d, W[i].status};
                B->a[i - i0] = BaseArgs{W[i].A, W[i].psi, W[i].d, (int)W[i].m0};
            }
            CK(mrc_gauss_jordan_batch(*G, dmax, st));
            CK(mrc_base_case_batch(*B, dmax, st));
        }
    }
    if (f32) {
        // binary32 copies of A and of psi(0 .. m0-1) for the FP32 levels
        auto C = std::make_unique<SegParams<CvtArgs>>();
        std::vector<CvtArgs> cv;
        for (auto &m : W) {
            cv.push_back(CvtArgs{m.A, m.A32, m.N * m.E});
            cv.push_back(CvtArgs{m.psi, m.psi32, m.m0 * m.E});
        }
        for (size_t i0 = 0; i0 < cv.size(); i0 += MRC_SEG_MAX) {
            const size_t i1 = std::min(cv.size(), i0 + (size_t)MRC_SEG_MAX);
            unsigned total = 0;
            C->nseg = (int)(i1 - i0);
            for (size_t i = i0; i < i1; ++i) {
                C->first[i - i0] = total;
                C->a[i - i0] = cv[i];
                total += (unsigned)((cv[i].n + MRC_CVT_CHUNK - 1) / MRC_CVT_CHUNK);
            }
            CK(mrc_f64_to_f32_batch(*C, total, st));
        }
        // the double-float spectra of A that every residual sweep uses, by
        // transform length, on the side stream while the FP32
        // levels run (as in the single-model inverse)
        mrc_status s = ensure_split_streams(c);
        if (s != MRC_OK) return s;
        CK(cudaEventRecord(c->ev_fork, st));
        CK(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
        for (int64_t Mr = pow2ceil(nmax); Mr >= 1; Mr >>= 1) {
            std::vector<FftJob> jobs;
            for (auto &m : W)
                if (m.Mr == Mr)
                    jobs.push_back({FftSrc{SRC_REAL64, m.A, 0, m.N, m.E, 0}, FftDst{DST_CPLX, m.ahat, m.E, 0, 0, 0, 1.0, 0},
                                    m.E, m.ascr});
            if ((s = fft_stage(c, PREC_DD, Mr, -1, jobs, c->aux)) != MRC_OK) return s;
            // the prepared X of the tensor-core residual products, per K-chunk count
            std::vector<PairArgs> pj[5];
            for (auto &m : W)
                if (m.Mr == Mr && m.xpt) {
                    PairArgs a = mrc_tcp_args(m.ahat, nullptr, m.xpt, Mr, m.d, c->tw[PREC_DD], MRC_TW_LOG);
                    a.xs = m.xps;
                    pj[(m.d + 15) / 16].push_back(a);
                }
            auto P = std::make_unique<SegParams<PairArgs>>();
            for (int g = 0; g < 5; ++g)
                for (size_t i0 = 0; i0 < pj[g].size(); i0 += MRC_SEG_MAX) {
                    const size_t i1 = std::min(pj[g].size(), i0 + (size_t)MRC_SEG_MAX);
                    P->nseg = (int)(i1 - i0);
                    for (size_t q = i0; q < i1; ++q) {
                        P->first[q - i0] = 0;
                        P->a[q - i0] = pj[g][q];
                    }
                    CK(mrc_tcp_prep(*P, c->aux));
                }
        }
        CK(cudaEventRecord(c->ev_join, c->aux));
    }
    // Newton levels m -> min(2m, N) of Eq. (newton), every model at level m at once
    for (int64_t m = mmin; mmin < INT64_MAX && m < nmax; m <<= 1) {
        std::vector<size_t> act;
        for (size_t i = 0; i < n; ++i)
            if (W[i].m0 <= m && m < W[i].N) act.push_back(i);
        if (act.empty()) continue;
        const int64_t M = m;
        std::vector<FftJob> ja, jb, ji, jr, jo;
        std::vector<PairJob> p1, p2;
        for (size_t i : act) {
            BModel &b = W[i];
            const int64_t m2 = std::min<int64_t>(2 * m, b.N);
            const void *Asrc = f32 ? (const void *)b.A32 : (const void *)b.A;
            const void *Bsrc = f32 ? (const void *)b.psi32 : (const void *)b.psi;
            const int sm = f32 ? SRC_REAL32 : SRC_REAL64;
            ja.push_back({FftSrc{sm, Asrc, 0, m2, b.E, 0}, FftDst{DST_CPLX, b.b0, b.E, 0, 0, 0, 1.0, 0}, b.E, b.bt});
            jb.push_back({FftSrc{sm, Bsrc, 0, m, b.E, 0}, FftDst{DST_CPLX, b.b1, b.E, 0, 0, 0, 1.0, 0}, b.E, b.bt});
            p1.push_back({b.b0, b.b1, b.b2, b.d, b.status});
            ji.push_back({FftSrc{SRC_CPLX, b.b2, 0, M, b.E, 0}, FftDst{DST_CPLX, b.b0, b.E, 0, 0, 0, 1.0 / (double)M, 0},
                          b.E, b.bt});
            jr.push_back({FftSrc{SRC_CPLX, b.b0, M / 2, M / 2, b.E, 1}, FftDst{DST_CPLX, b.b2, b.E, 0, 0, 0, 1.0, 0}, b.E,
                          b.bt});
            p2.push_back({b.b1, b.b2, b.b0, b.d, b.status});
            jo.push_back({FftSrc{SRC_CPLX, b.b0, 0, M, b.E, 0},
                          FftDst{f32 ? DST_REAL32 : DST_REAL64, f32 ? (void *)b.psi32 : (void *)b.psi, b.E, 0, m2 - m, m,
                                 1.0 / (double)M, 0},
                          b.E, b.bt});
        }
        mrc_status s;
        if ((s = fft_stage(c, pl, M, -1, ja, st)) != MRC_OK) return s;      // A-hat
        if ((s = fft_stage(c, pl, M, -1, jb, st)) != MRC_OK) return s;      // B-hat
        if ((s = product_stage(c, pl, M, p1, st)) != MRC_OK) return s;      // (A B)-hat
        if ((s = fft_stage(c, pl, M, +1, ji, st)) != MRC_OK) return s;      // A*B, packed time
        if ((s = fft_stage(c, pl, M, -1, jr, st)) != MRC_OK) return s;      // R-hat, R = -(A*B)[m, 2m)
        if ((s = product_stage(c, pl, M, p2, st)) != MRC_OK) return s;      // (B R)-hat
        if ((s = fft_stage(c, pl, M, +1, jo, st)) != MRC_OK) return s;      // B[m, m2)
    }
    if (!f32) return MRC_OK;
    CK(cudaStreamWaitEvent(st, c->ev_join, 0));  // the spectra of A
    // residual rho_L = e0 - A * psi in double-float (Proposition 2.6) and the
    // FP32 correction psi <- psi + psi * rho_L, by transform length
    for (int sw = 0; sw < sweeps; ++sw) {
        const bool first = sw == 0;
        for (int64_t Mr = pow2ceil(nmax); Mr >= 1; Mr >>= 1) {
            std::vector<FftJob> fy, fc, gy, gc;
            std::vector<PairJob> pr, pc;
            for (auto &b : W) {
                if (b.Mr != Mr) continue;
                fy.push_back({FftSrc{first ? SRC_REAL32 : SRC_REAL64, first ? (const void *)b.psi32 : (const void *)b.psi,
                                     0, b.N, b.E, 0},
                              FftDst{DST_CPLX, b.rY, b.E, 0, 0, 0, 1.0, 0, b.psihat32}, b.E, b.ascr});
                if (b.xpt) pr.push_back({b.xpt, b.rY, b.rC, b.d, b.status, b.xps});
                else pr.push_back({b.ahat, b.rY, b.rC, b.d, b.status});
                fc.push_back({FftSrc{SRC_CPLX, b.rC, 0, Mr, b.E, 0},
                              FftDst{DST_REAL32, b.rho32, b.E, 0, b.N, 0, -1.0 / (double)Mr, b.d}, b.E, b.ascr});
                gy.push_back({FftSrc{SRC_REAL32, b.rho32, 0, b.N, b.E, 0}, FftDst{DST_CPLX, b.cY, b.E, 0, 0, 0, 1.0, 0},
                              b.E, b.cT});
                pc.push_back({b.psihat32, b.cY, b.cC, b.d, b.status});
                gc.push_back({FftSrc{SRC_CPLX, b.cC, 0, Mr, b.E, 0},
                              FftDst{first ? DST_REAL64_BASE32 : DST_REAL64_ADD, b.psi, b.E, 0, b.N, 0, 1.0 / (double)Mr, 0,
                                     nullptr, first ? (const void *)b.psi32 : nullptr},
                              b.E, b.cT});
            }
            if (fy.empty()) continue;
            mrc_status s;
            if ((s = fft_stage(c, PREC_DD, Mr, -1, fy, st)) != MRC_OK) return s;
            if ((s = product_stage(c, PREC_DD, Mr, pr, st)) != MRC_OK) return s;
            if ((s = fft_stage(c, PREC_DD, Mr, +1, fc, st)) != MRC_OK) return s;
            if ((s = fft_stage(c, PREC_F32, Mr, -1, gy, st)) != MRC_OK) return s;
            if ((s = product_stage(c, PREC_F32, Mr, pc, st)) != MRC_OK) return s;
            if ((s = fft_stage(c, PREC_F32, Mr, +1, gc, st)) != MRC_OK) return s;
        }
    }
    return MRC_OK;
}

} // namespace

// ===========================================================================
// The Newton schedule shared by the inverse entry points.
int64_t mrc_base_size(int d, int64_t N)
{
    int64_t m0 = d <= 8 ? 32 : (d <= 32 ? 8 : 2);
    return std::min<int64_t>(m0, N);
}

int64_t mrc_newton_maxM(int d, int64_t N)
{
    int64_t m0 = mrc_base_size(d, N), M = 0;
    for (int64_t m = m0; m < N; m <<= 1) M = m;
    return M;
}

// Each level m -> min(2m, N) follows Eq. (newton) with the middle product
// (L = 2m): E = A*B (cyclic), R = -E[m, 2m), B[m, 2m) = (B*R)[0, m).
int mrc_newton_levels(int prec, int d, int64_t N, const double *A, double *psi, int64_t m0, const NewtonBufs &b,
                      const void *tw, int tw_log, mrc_level_fft_fn fft, mrc_level_product_fn product, void *user,
                      cudaStream_t st, const RowWait *rw, float *A32, float *psi32, int *levels, int64_t a32_rows)
{
    const int E = d * d;
    const bool f32 = A32 && psi32;
    int64_t conv = a32_rows;  // rows of A32 converted so far
    int lv = 0;
    for (int64_t m = m0; m < N; m <<= 1, ++lv) {
        const int64_t M = m, m2 = std::min<int64_t>(2 * m, N);
        if (rw) CK(rw->wait(st, m2));  // this level reads A[0, 2m)
        if (f32 && conv < m2) {
            CK(mrc_f64_to_f32(A + conv * E, A32 + conv * E, (m2 - conv) * E, st));
            conv = m2;
        }
        FftSrc sA{f32 ? SRC_REAL32 : SRC_REAL64, f32 ? (const void *)A32 : A, 0, m2, E, 0};
        FftSrc sB{f32 ? SRC_REAL32 : SRC_REAL64, f32 ? (const void *)psi32 : psi, 0, m, E, 0};
        FftDst to0{DST_CPLX, b.b0, E, 0, 0, 0, 1.0, 0};
        FftDst to1{DST_CPLX, b.b1, E, 0, 0, 0, 1.0, 0};
        CK(fft(user, prec, sA, to0, M, E, -1, b.bt, tw, tw_log, st));        // A-hat
        CK(fft(user, prec, sB, to1, M, E, -1, b.bt, tw, tw_log, st));        // B-hat
        CK(product(user, prec, b.b0, b.b1, b.b2, M, d, tw, tw_log, st));      // (A B)-hat
        FftSrc s2{SRC_CPLX, b.b2, 0, M, E, 0};
        FftDst t0s{DST_CPLX, b.b0, E, 0, 0, 0, 1.0 / (double)M, 0};
        CK(fft(user, prec, s2, t0s, M, E, +1, b.bt, tw, tw_log, st));        // A*B, packed time
        FftSrc sR{SRC_CPLX, b.b0, M / 2, M / 2, E, 1};                         // R = -(A*B)[m, 2m)
        FftDst to2{DST_CPLX, b.b2, E, 0, 0, 0, 1.0, 0};
        CK(fft(user, prec, sR, to2, M, E, -1, b.bt, tw, tw_log, st));        // R-hat
        CK(product(user, prec, b.b1, b.b2, b.b0, M, d, tw, tw_log, st));      // (B R)-hat
        FftSrc s0{SRC_CPLX, b.b0, 0, M, E, 0};
        FftDst toP{f32 ? DST_REAL32 : DST_REAL64, f32 ? (void *)psi32 : psi, E, 0, m2 - m, m, 1.0 / (double)M, 0};
        CK(fft(user, prec, s0, toP, M, E, +1, b.bt, tw, tw_log, st));        // B[m, m2)
    }
    if (levels) *levels = lv;
    return MRC_OK;
}

// the single-model mixed inverse's two internal streams (created on first use)
static mrc_status ensure_split_streams(mrc_ctx *c)
{
    if (c->aux) return MRC_OK;
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, greatest));
    mrc_prof_set_untimed(c->aux);
    CK(cudaStreamCreateWithPriority(&c->lvl, cudaStreamNonBlocking, greatest));
    CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming));
    return MRC_OK;
}

extern "C" {

const char *mrc_status_string(mrc_status s)
{
    switch (s) {
    case MRC_OK: return "ok";
    case MRC_ERR_INVALID_ARG: return "invalid argument";
    case MRC_ERR_SINGULAR_A0: return "A(0) is singular";
    case MRC_ERR_NO_MEMORY: return "out of workspace memory";
    case MRC_ERR_CUDA: return "CUDA error";
    case MRC_ERR_NOT_CONVERGED: return "refinement did not reach the target residual";
    case MRC_ERR_TIMEOUT: return "device wait timed out";
    case MRC_ERR_UNIMPLEMENTED: return "unimplemented";
    }
    return "unknown status";
}

const char *mrc_version(void) { return "libmrc 0.1 (sm_103a)"; }

mrc_status mrc_create(mrc_ctx **out, int device, size_t max_workspace_bytes)
{
    if (!out) return MRC_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return MRC_ERR_CUDA;
    for (int p = 0; p < 3; ++p)
        if (OPS[p].init() != cudaSuccess) return MRC_ERR_CUDA;
    if (mrc_tc_init() != cudaSuccess || mrc_tcp_init() != cudaSuccess) return MRC_ERR_CUDA;
    mrc_ctx *c = new mrc_ctx();
    c->device = device;
    c->cap = max_workspace_bytes;
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess || cudaMalloc(&c->d_acc, 4 * sizeof(double)) != cudaSuccess) {
        delete c;
        return MRC_ERR_NO_MEMORY;
    }
    cudaMemset(c->d_status, 0, sizeof(int));
    c->cur_status = c->d_status;
    tune_load(c);
    cudaEventCreate(&c->ev0);
    cudaEventCreate(&c->ev1);
    *out = c;
    return MRC_OK;
}

mrc_status mrc_destroy(mrc_ctx *c)
{
    if (!c) return MRC_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    tune_save(c);
    cudaFree(c->ws);
    for (int p = 0; p < 3; ++p) cudaFree(c->tw[p]);
    cudaFree(c->d_status);
    cudaFree(c->d_acc);
    cudaEventDestroy(c->ev0);
    cudaEventDestroy(c->ev1);
    if (c->aux) {
        mrc_prof_set_untimed(nullptr);
        cudaStreamDestroy(c->aux);
    }
    if (c->lvl) cudaStreamDestroy(c->lvl);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_join2) cudaEventDestroy(c->ev_join2);
    if (c->cpy) cudaStreamDestroy(c->cpy);
    if (c->ev_cpy_fork) cudaEventDestroy(c->ev_cpy_fork);
    for (auto e : c->ev_rows)
        if (e) cudaEventDestroy(e);
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    for (int k = 0; k < MRC_BATCH_STREAMS; ++k) {
        if (c->bst[k]) cudaStreamDestroy(c->bst[k]);
        if (c->bev[k]) cudaEventDestroy(c->bev[k]);
    }
    delete c;
    return MRC_OK;
}

mrc_status mrc_sync_status(mrc_ctx *c, void *stream)
{
    if (!c) return MRC_ERR_INVALID_ARG;
    return read_status(c, (cudaStream_t)stream);
}

size_t mrc_inverse_workspace_bytes(int d, int64_t N, int prec)
{
    if (!valid_dN(d, N)) return 0;
    return ws_inverse(d, N, prec);
}

mrc_status mrc_inverse(mrc_ctx *c, int d, int64_t N, const double *A, double *psi, const mrc_options *opt,
                       void *stream, mrc_report *report)
{
    if (!c || !A || !psi || !valid_dN(d, N)) return MRC_ERR_INVALID_ARG;
    TuneScope tscope(c, opt);
    const int prec = opt ? opt->prec : MRC_FP64;
    if (prec != MRC_FP64 && prec != MRC_MIXED) return MRC_ERR_INVALID_ARG;
    int sweeps = opt ? opt->refine_sweeps : 1;
    if (prec == MRC_MIXED && sweeps <= 0) sweeps = 1;
    if (sweeps > 4) return MRC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    mrc_status s;
    if ((s = ensure_tw(c, prec == MRC_FP64 ? PREC_F64 : PREC_F32, st)) != MRC_OK) return s;
    if (prec == MRC_MIXED && (s = ensure_tw(c, PREC_DD, st)) != MRC_OK) return s;
    const bool check = report && prec == MRC_MIXED && opt && opt->target_residual > 0;
    size_t need = ws_inverse(d, N, prec);
    if (check) need = std::max(need, ws_residual(d, N, MRC_MIXED, true));
    if ((s = ensure_ws(c, need)) != MRC_OK) return s;
    Arena ar{(char *)c->ws};
    int levels = 0;
    if (report) CK(cudaEventRecord(c->ev0, st));
    if (prec == MRC_MIXED && (s = ensure_split_streams(c)) != MRC_OK) return s;
    s = inverse_impl(c, ar, d, N, A, psi, prec, sweeps, &levels, st, nullptr, prec == MRC_MIXED);
    if (s != MRC_OK) return s;
    if (report) {
        CK(cudaEventRecord(c->ev1, st));
        memset(report, 0, sizeof(*report));
        report->res_left_l1 = report->res_right_l1 = report->res_max_abs = -1.0;
        report->levels = levels;
        report->sweeps = prec == MRC_MIXED ? sweeps : 0;
        s = read_status(c, st);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        report->ms = ms;
        if (s != MRC_OK) return s;
        if (check) {
            Arena ar2{(char *)c->ws};
            s = residual_impl(c, ar2, d, N, A, psi, 1, nullptr, nullptr, MRC_MIXED, st, report);
            if (s != MRC_OK) return s;
            if (!(report->res_max_abs <= opt->target_residual)) return MRC_ERR_NOT_CONVERGED;
        }
    }
    return MRC_OK;
}

mrc_status mrc_inverse_gj(mrc_ctx *c, int d, int64_t N, const double *A, double *psi, const mrc_options *opt,
                          void *stream, mrc_report *report)
{
    if (!c || !A || !psi || d < 1 || d > MRC_GJ_DMAX || N < 1 || N > ((int64_t)1 << 20)) return MRC_ERR_INVALID_ARG;
    if (opt && opt->prec != MRC_FP64) return MRC_ERR_INVALID_ARG;
    TuneScope tscope(c, opt);
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    mrc_status s;
    if ((s = ensure_tw(c, PREC_F64, st)) != MRC_OK) return s;
    if ((s = ensure_ws(c, ws_gj_series(d, N))) != MRC_OK) return s;
    Arena ar{(char *)c->ws};
    if (report) CK(cudaEventRecord(c->ev0, st));
    c->cur_status = c->d_status;
    if ((s = gj_series_impl(c, ar, d, N, A, psi, st)) != MRC_OK) return s;
    if (report) {
        CK(cudaEventRecord(c->ev1, st));
        memset(report, 0, sizeof(*report));
        report->res_left_l1 = report->res_right_l1 = report->res_max_abs = -1.0;
        report->levels = d;
        s = read_status(c, st);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        report->ms = ms;
        if (s != MRC_OK) return s;
    }
    return MRC_OK;
}

mrc_status mrc_inverse_host(mrc_ctx *c, int d, int64_t N, const double *A_host, double *psi_host,
                            const mrc_options *opt, void *stream, mrc_report *report)
{
    if (!c || !A_host || !psi_host || !valid_dN(d, N)) return MRC_ERR_INVALID_ARG;
    TuneScope tscope(c, opt);
    const int prec = opt ? opt->prec : MRC_FP64;
    if (prec != MRC_FP64 && prec != MRC_MIXED) return MRC_ERR_INVALID_ARG;
    int sweeps = opt ? opt->refine_sweeps : 1;
    if (prec == MRC_MIXED && sweeps <= 0) sweeps = 1;
    if (sweeps > 4) return MRC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    mrc_status s;
    if ((s = ensure_tw(c, prec == MRC_FP64 ? PREC_F64 : PREC_F32, st)) != MRC_OK) return s;
    if (prec == MRC_MIXED && (s = ensure_tw(c, PREC_DD, st)) != MRC_OK) return s;
    const size_t E = (size_t)d * d, bytes = (size_t)N * E * sizeof(double), seq = align_up(bytes);
    const bool check = report && prec == MRC_MIXED && opt && opt->target_residual > 0;
    size_t need = ws_inverse(d, N, prec);
    if (check) need = std::max(need, ws_residual(d, N, MRC_MIXED, true));
    if ((s = ensure_ws(c, 2 * seq + need)) != MRC_OK) return s;
    double *dA = (double *)c->ws, *dpsi = (double *)((char *)c->ws + seq);
    if (!c->cpy) {
        CK(cudaStreamCreateWithFlags(&c->cpy, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->ev_cpy_fork, cudaEventDisableTiming));
        for (auto &e : c->ev_rows) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (prec == MRC_MIXED && (s = ensure_split_streams(c)) != MRC_OK) return s;
    // upload A in the row ranges the Newton levels consume: [0, 2 m0), then doubling
    if (report) CK(cudaEventRecord(c->ev0, st));
    CK(cudaEventRecord(c->ev_cpy_fork, st));  // earlier work on st may still use the workspace
    CK(cudaStreamWaitEvent(c->cpy, c->ev_cpy_fork, 0));
    RowWait rw;
    int64_t r0 = 0, r1 = std::min<int64_t>(2 * base_size(d, N), N);
    while (r0 < N && rw.n < 32) {
        if (rw.n == 31) r1 = N;
        CK(cudaMemcpyAsync(dA + r0 * E, A_host + r0 * E, (size_t)(r1 - r0) * E * sizeof(double),
                           cudaMemcpyHostToDevice, c->cpy));
        CK(cudaEventRecord(c->ev_rows[rw.n], c->cpy));
        rw.end[rw.n] = r1;
        rw.ev[rw.n] = c->ev_rows[rw.n];
        ++rw.n;
        r0 = r1;
        r1 = std::min<int64_t>(2 * r1, N);
    }
    Arena ar{(char *)c->ws + 2 * seq};
    int levels = 0;
    s = inverse_impl(c, ar, d, N, dA, dpsi, prec, sweeps, &levels, st, nullptr, prec == MRC_MIXED, &rw);
    if (s != MRC_OK) return s;
    CK(rw.wait(st, N));
    CK(cudaMemcpyAsync(psi_host, dpsi, bytes, cudaMemcpyDeviceToHost, st));
    if (report) {
        CK(cudaEventRecord(c->ev1, st));
        memset(report, 0, sizeof(*report));
        report->res_left_l1 = report->res_right_l1 = report->res_max_abs = -1.0;
        report->levels = levels;
        report->sweeps = prec == MRC_MIXED ? sweeps : 0;
        s = read_status(c, st);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        report->ms = ms;
        if (s != MRC_OK) return s;
        if (check) {
            Arena ar2{(char *)c->ws + 2 * seq};
            s = residual_impl(c, ar2, d, N, dA, dpsi, 1, nullptr, nullptr, MRC_MIXED, st, report);
            if (s != MRC_OK) return s;
            if (!(report->res_max_abs <= opt->target_residual)) return MRC_ERR_NOT_CONVERGED;
        }
    }
    return MRC_OK;
}

mrc_status mrc_inverse_batched(mrc_ctx *c, int nmodels, const int *d, const int64_t *N, const double *const *A,
                               double *const *psi, const mrc_options *opt, void *stream, mrc_report *report)
{
    if (!c || nmodels < 0 || (nmodels > 0 && (!d || !N || !A || !psi))) return MRC_ERR_INVALID_ARG;
    for (int b = 0; b < nmodels; ++b)
        if (!valid_dN(d[b], N[b]) || !A[b] || !psi[b]) return MRC_ERR_INVALID_ARG;
    if (nmodels == 0) return MRC_OK;
    TuneScope tscope(c, opt);
    const int prec = opt ? opt->prec : MRC_FP64;
    if (prec != MRC_FP64 && prec != MRC_MIXED) return MRC_ERR_INVALID_ARG;
    int sweeps = opt ? opt->refine_sweeps : 1;
    if (prec == MRC_MIXED && sweeps <= 0) sweeps = 1;
    if (prec == MRC_FP64) sweeps = 0;
    if (sweeps > 4) return MRC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    mrc_status s;
    if ((s = ensure_tw(c, prec == MRC_FP64 ? PREC_F64 : PREC_F32, st)) != MRC_OK) return s;
    if (prec == MRC_MIXED && (s = ensure_tw(c, PREC_DD, st)) != MRC_OK) return s;

    // Models in decreasing cost (~ N d^2 (log2 N + d), the FFT and product
    // terms of Prop 2.4) into waves whose buffers fit the budget: the context
    // cap if set, else at most 192 GB and three quarters of the device memory
    // free besides the workspace (but always room for the largest model)
    std::vector<BModel> bm(nmodels);
    size_t wmax = 0;
    for (int b = 0; b < nmodels; ++b) {
        BModel &m = bm[b];
        m.d = d[b];
        m.E = d[b] * d[b];
        m.N = N[b];
        m.m0 = base_size(d[b], N[b]);
        m.Mr = pow2ceil(N[b]);
        m.Mmax = newton_maxM(d[b], N[b]);
        m.A = A[b];
        m.psi = psi[b];
        double lg = 1.0;
        for (int64_t x = 1; x < N[b]; x <<= 1) lg += 1.0;
        m.cost = (double)N[b] * d[b] * d[b] * (lg + d[b]);
        m.ws = align_up(ws_inverse(d[b], N[b], prec));
        wmax = std::max(wmax, m.ws);
    }
    std::vector<int> order(nmodels);
    for (int b = 0; b < nmodels; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return bm[x].cost > bm[y].cost; });
    size_t budget = (size_t)192 << 30;
    {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) budget = std::min(budget, (fr + c->ws_size) / 4 * 3);
    }
    const size_t head = align_up(sizeof(int) * nmodels);
    if (c->cap) budget = std::min(budget, c->cap > head ? c->cap - head : 0);
    budget = std::max(budget, wmax);
    std::vector<std::vector<int>> waves;
    std::vector<size_t> woff(nmodels, 0);
    size_t used = 0, wsneed = 0;
    for (int b : order) {
        if (waves.empty() || used + bm[b].ws > budget) {
            waves.emplace_back();
            used = 0;
        }
        woff[b] = used;
        used += bm[b].ws;
        waves.back().push_back(b);
        wsneed = std::max(wsneed, used);
    }
    if ((s = ensure_ws(c, head + wsneed)) != MRC_OK) return s;
    if (prec == MRC_MIXED && (s = ensure_split_streams(c)) != MRC_OK) return s;
    int *status = (int *)c->ws;
    for (int b = 0; b < nmodels; ++b) bm[b].status = status + b;

    auto run_waves = [&](cudaStream_t s0) -> mrc_status {
        for (size_t w = 0; w < waves.size(); ++w) {
            std::vector<BModel> W;
            for (int b : waves[w]) {
                W.push_back(bm[b]);
                bmodel_layout(W.back(), prec, (char *)c->ws + head + woff[b]);
            }
            mrc_status r = batch_wave(c, W, prec, sweeps, s0);
            if (r != MRC_OK) return r;
        }
        return MRC_OK;
    };
    if (mrc_prof_timing()) {
        // a kernel class is being timed: run the stages eagerly on `stream`
        // (a graph replay would not pass through the per-launch events)
        if (report) CK(cudaEventRecord(c->ev0, st));
        CK(cudaMemsetAsync(status, 0, sizeof(int) * nmodels, st));
        if ((s = run_waves(st)) != MRC_OK) return s;
    }
    BatchGraph *hit = nullptr;
    for (auto &g : c->graphs) {
        if (mrc_prof_timing()) break;
        if (g.prec != prec || g.sweeps != sweeps || (int)g.d.size() != nmodels || g.ws != c->ws) continue;
        bool same = true;
        for (int b = 0; b < nmodels && same; ++b)
            same = g.d[b] == d[b] && g.N[b] == N[b] && g.A[b] == A[b] && g.psi[b] == psi[b];
        if (same) { hit = &g; break; }
    }
    if (!hit && !mrc_prof_timing()) {
        if (c->autotune) {
            // tune each distinct shape now: the graph capture below cannot time kernels
            std::vector<std::pair<int, int64_t>> seen;
            for (int b = 0; b < nmodels; ++b) {
                std::pair<int, int64_t> key{d[b], N[b]};
                if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
                seen.push_back(key);
                pretune_model(c, prec, d[b], N[b], (char *)c->ws + head, c->ws_size - head, st);
            }
        }
        if (!c->bst[0]) CK(cudaStreamCreateWithFlags(&c->bst[0], cudaStreamNonBlocking));
        cudaStream_t s0 = c->bst[0];
        CK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
        mrc_prof_set_capturing(true);
        c->capturing = true;
        mrc_status cs = MRC_OK;
        if (cudaMemsetAsync(status, 0, sizeof(int) * nmodels, s0) != cudaSuccess) cs = MRC_ERR_CUDA;
        if (cs == MRC_OK) cs = run_waves(s0);
        mrc_prof_set_capturing(false);
        c->capturing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t ee = cudaStreamEndCapture(s0, &graph);
        if (cs != MRC_OK || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return cs != MRC_OK ? cs : MRC_ERR_CUDA;
        }
        BatchGraph g;
        g.d.assign(d, d + nmodels);
        g.N.assign(N, N + nmodels);
        g.A.assign(A, A + nmodels);
        g.psi.assign(psi, psi + nmodels);
        g.prec = prec;
        g.sweeps = sweeps;
        g.ws = c->ws;
        cudaError_t ce = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return MRC_ERR_CUDA;
        if (c->graphs.size() >= 8) {
            cudaGraphExecDestroy(c->graphs.front().exec);
            c->graphs.erase(c->graphs.begin());
        }
        c->graphs.push_back(std::move(g));
        hit = &c->graphs.back();
    }
    if (hit) {
        if (report) CK(cudaEventRecord(c->ev0, st));
        CK(cudaGraphLaunch(hit->exec, st));
    }
    if (!report) return MRC_OK;
    CK(cudaEventRecord(c->ev1, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    std::vector<int> hs(nmodels, 0);
    CK(cudaMemcpy(hs.data(), status, sizeof(int) * nmodels, cudaMemcpyDeviceToHost));
    mrc_status first = MRC_OK;
    for (int b = 0; b < nmodels; ++b) {
        mrc_report &r = report[b];
        memset(&r, 0, sizeof(r));
        r.res_left_l1 = r.res_right_l1 = r.res_max_abs = -1.0;
        int lv = 0;
        for (int64_t m = base_size(d[b], N[b]); m < N[b]; m <<= 1) ++lv;
        r.levels = lv;
        r.sweeps = sweeps;
        r.ms = ms;
        if (hs[b] && first == MRC_OK) first = (mrc_status)hs[b];
    }
    return first;
}

mrc_status mrc_residual(mrc_ctx *c, int d, int64_t N, const double *A, const double *psi, int sides, double *rho_left,
                        double *rho_right, int prec, void *stream, mrc_report *report)
{
    if (!c || !A || !psi || !valid_dN(d, N) || sides < 1 || sides > 3) return MRC_ERR_INVALID_ARG;
    if (prec != MRC_FP64 && prec != MRC_MIXED) return MRC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    mrc_status s;
    const int p = prec == MRC_FP64 ? PREC_F64 : PREC_DD;
    if ((s = ensure_tw(c, p, st)) != MRC_OK) return s;
    const bool need_tmp = ((sides & 1) && !rho_left) || ((sides & 2) && !rho_right);
    if ((s = ensure_ws(c, ws_residual(d, N, prec, need_tmp))) != MRC_OK) return s;
    Arena ar{(char *)c->ws};
    if (report) {
        memset(report, 0, sizeof(*report));
        report->res_left_l1 = report->res_right_l1 = report->res_max_abs = -1.0;
    }
    return residual_impl(c, ar, d, N, A, psi, sides, rho_left, rho_right, prec, st, report);
}

mrc_status mrc_transition(mrc_ctx *c, int d, int64_t N, const double *psi, const double *q, double *P, int prec,
                          void *stream)
{
    if (!c || !psi || !q || !P || !valid_dN(d, N)) return MRC_ERR_INVALID_ARG;
    if (prec != MRC_FP64 && prec != MRC_MIXED) return MRC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    const int p = prec == MRC_FP64 ? PREC_F64 : PREC_DD;
    mrc_status s;
    if ((s = ensure_tw(c, p, st)) != MRC_OK) return s;
    const size_t E = (size_t)d * d;
    const int64_t nch = (N + 1023) / 1024;
    size_t need = align_up(sizeof(double) * N * d) + align_up(sizeof(double) * nch * d) +
                  ws_product(pow2ceil(N), E, d, E, p);
    if ((s = ensure_ws(c, need)) != MRC_OK) return s;
    Arena ar{(char *)c->ws};
    double *h = (double *)ar.take(sizeof(double) * N * d);
    double *work = (double *)ar.take(sizeof(double) * nch * d);
    CK(mrc_row_sums(q, h, d, N, st));
    CK(mrc_scan_cols(h, d, N, work, -1.0, 1.0, st));  // Hbar_j(k) = 1 - sum_{l<=k} sum_j' q_jj'(l)
    return conv_product(c, ar, p, psi, N, h, N, d, 1, d, N, P, 1.0, 0, 0, true, st);
}

mrc_status mrc_first_entrance(mrc_ctx *c, int d, int64_t N, const double *q, const int *D, int nD,
                              const double *alpha_C, double *g, double *F, double *S, const mrc_options *opt,
                              void *stream)
{
    if (!c || !q || !D || !alpha_C || !valid_dN(d, N) || nD < 1 || nD >= d) return MRC_ERR_INVALID_ARG;
    TuneScope tscope(c, opt);
    std::vector<int> inD(d, 0), Ci, Di;
    for (int t = 0; t < nD; ++t) {
        if (D[t] < 0 || D[t] >= d || inD[D[t]]) return MRC_ERR_INVALID_ARG;
        inD[D[t]] = 1;
    }
    for (int i = 0; i < d; ++i) (inD[i] ? Di : Ci).push_back(i);
    const int nC = (int)Ci.size();
    const int prec = opt ? opt->prec : MRC_FP64;
    if (prec != MRC_FP64 && prec != MRC_MIXED) return MRC_ERR_INVALID_ARG;
    int sweeps = opt && opt->refine_sweeps > 0 ? opt->refine_sweeps : 1;
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    mrc_status s;
    const int pc = prec == MRC_FP64 ? PREC_F64 : PREC_DD;
    if ((s = ensure_tw(c, prec == MRC_FP64 ? PREC_F64 : PREC_F32, st)) != MRC_OK) return s;
    if ((s = ensure_tw(c, pc, st)) != MRC_OK) return s;
    const size_t ECC = (size_t)nC * nC, ECD = (size_t)nC * nD;
    size_t fixed = align_up(sizeof(double) * N * ECC) * 2 + align_up(sizeof(double) * N * ECD) * 2 +
                   align_up(sizeof(double) * N) * 2 + align_up(sizeof(double) * ((N + 1023) / 1024));
    size_t need = fixed + std::max(ws_inverse(nC, N, prec), ws_product(pow2ceil(N), ECC, ECD, ECD, pc));
    if ((s = ensure_ws(c, need)) != MRC_OK) return s;
    Arena ar{(char *)c->ws};
    double *ACC = (double *)ar.take(sizeof(double) * N * ECC);
    double *psiC = (double *)ar.take(sizeof(double) * N * ECC);
    double *QCD = (double *)ar.take(sizeof(double) * N * ECD);
    double *gw = (double *)ar.take(sizeof(double) * N * ECD);
    double *Fw = (double *)ar.take(sizeof(double) * N);
    double *fk = (double *)ar.take(sizeof(double) * N);
    double *work = (double *)ar.take(sizeof(double) * ((N + 1023) / 1024));
    CK(mrc_gather_blocks(q, d, N, Ci.data(), nC, Di.data(), nD, ACC, QCD, st));
    const size_t mark = ar.off;
    s = inverse_impl(c, ar, nC, N, ACC, psiC, prec, sweeps, nullptr, st);
    if (s != MRC_OK) return s;
    ar.off = mark;
    double *gout = g ? g : gw;
    s = conv_product(c, ar, pc, psiC, N, QCD, N, nC, nC, nD, N, gout, 1.0, 0, 0, false, st);
    if (s != MRC_OK) return s;
    if (F || S) {
        double *Fo = F ? F : Fw;
        CK(mrc_weighted_rowsum(gout, nC, nD, N, alpha_C, fk, st));
        CK(cudaMemcpyAsync(Fo, fk, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        CK(mrc_scan_cols(Fo, 1, N, work, 1.0, 0.0, st));
        if (S) CK(mrc_one_minus(Fo, S, N, st));
    }
    return MRC_OK;
}

mrc_status mrc_occupation(mrc_ctx *c, int d, int64_t N, const double *P, const double *alpha, const int *B, int nB,
                          double *out, void *stream)
{
    if (!c || !P || !alpha || !B || !out || !valid_dN(d, N) || nB < 0 || nB > d) return MRC_ERR_INVALID_ARG;
    std::vector<int> inB(d, 0);
    for (int t = 0; t < nB; ++t) {
        if (B[t] < 0 || B[t] >= d) return MRC_ERR_INVALID_ARG;
        inB[B[t]] = 1;
    }
    cudaSetDevice(c->device);
    CK(mrc_occupation_k(P, d, N, alpha, inB.data(), out, (cudaStream_t)stream));
    return MRC_OK;
}

mrc_status mrc_reward(mrc_ctx *c, int d, int cc, int64_t N, const double *psi, const double *r, double *V, int prec,
                      void *stream)
{
    if (!c || !psi || !r || !V || !valid_dN(d, N) || cc < 1 || cc > 512) return MRC_ERR_INVALID_ARG;
    if (prec != MRC_FP64 && prec != MRC_MIXED) return MRC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    const int p = prec == MRC_FP64 ? PREC_F64 : PREC_DD;
    mrc_status s;
    if ((s = ensure_tw(c, p, st)) != MRC_OK) return s;
    const size_t E = (size_t)d * d, EV = (size_t)d * cc;
    if ((s = ensure_ws(c, ws_product(pow2ceil(N), E, EV, EV, p))) != MRC_OK) return s;
    Arena ar{(char *)c->ws};
    // V = psi * r: d x d times d x c at every frequency (Eq. (reward))
    return conv_product(c, ar, p, psi, N, r, N, d, d, cc, N, V, 1.0, 0, 0, false, st);
}

mrc_status mrc_mre_solve(mrc_ctx *c, int d, int cc, int64_t N, const double *Q, const double *L, int scheme,
                         double *K, const mrc_options *opt, void *stream)
{
    if (!c || !Q || !L || !K || !valid_dN(d, N) || cc < 1 || cc > 512 || (scheme != 0 && scheme != 1))
        return MRC_ERR_INVALID_ARG;
    const int prec = opt ? opt->prec : MRC_FP64;
    if (prec != MRC_FP64 && prec != MRC_MIXED) return MRC_ERR_INVALID_ARG;
    int sweeps = opt ? opt->refine_sweeps : 1;
    if (prec == MRC_MIXED && sweeps <= 0) sweeps = 1;
    if (sweeps > 4) return MRC_ERR_INVALID_ARG;
    TuneScope tscope(c, opt);
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    const int p = prec == MRC_FP64 ? PREC_F64 : PREC_DD;
    mrc_status s;
    if ((s = ensure_tw(c, prec == MRC_FP64 ? PREC_F64 : PREC_F32, st)) != MRC_OK) return s;
    if (prec == MRC_MIXED && (s = ensure_tw(c, PREC_DD, st)) != MRC_OK) return s;
    const size_t E = (size_t)d * d, EL = (size_t)d * cc;
    const size_t fixed = 2 * align_up(sizeof(double) * N * E) + align_up(sizeof(double) * N * EL);
    if ((s = ensure_ws(c, fixed + std::max(ws_inverse(d, N, prec), ws_product(pow2ceil(N), E, EL, EL, p)))) != MRC_OK)
        return s;
    Arena ar{(char *)c->ws};
    double *A = (double *)ar.take(sizeof(double) * N * E);
    double *psi = (double *)ar.take(sizeof(double) * N * E);
    double *R = (double *)ar.take(sizeof(double) * N * EL);
    const size_t mark = ar.off;
    // e0 - Qbar_h (or e0 - Delta Q_h) and its inverse
    CK(mrc_mre_operator(Q, A, d, N, scheme, st));
    s = inverse_impl(c, ar, d, N, A, psi, prec, sweeps, nullptr, st);
    if (s != MRC_OK) return s;
    ar.off = mark;
    // right-hand side: L_h - (1/2) Delta+ Q_h L_h(0) (mean-value rule) or L_h, then K = psi * R
    const double *rhs = L;
    if (scheme == 0) {
        CK(mrc_mre_rhs(Q, L, R, d, cc, N, st));
        rhs = R;
    }
    return conv_product(c, ar, p, psi, N, rhs, N, d, d, cc, N, K, 1.0, 0, 0, false, st);
}

mrc_status mrc_selftest_timeout(mrc_ctx *c, int spins, void *stream)
{
    if (!c || spins < 1 || spins > (1 << 20)) return MRC_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    CK(mrc_tc_wait_selftest(c->d_status, spins, (cudaStream_t)stream));
    return MRC_OK;
}

mrc_status mrc_renewal_visits(mrc_ctx *c, int d, int64_t N, const double *psi, const double *alpha, const int *B,
                              int nB, double *out, void *stream)
{
    if (!c || !psi || !alpha || !B || !out || !valid_dN(d, N) || nB < 0 || nB > d) return MRC_ERR_INVALID_ARG;
    std::vector<int> inB(d, 0);
    for (int t = 0; t < nB; ++t) {
        if (B[t] < 0 || B[t] >= d) return MRC_ERR_INVALID_ARG;
        inB[B[t]] = 1;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    const int64_t nch = (N + 1023) / 1024;
    mrc_status s;
    if ((s = ensure_ws(c, align_up(sizeof(double) * nch))) != MRC_OK) return s;
    // alpha psi(k) 1_B per k, then the running sum over k (Eq. (renewal-visits))
    CK(mrc_occupation_k(psi, d, N, alpha, inB.data(), out, st));
    CK(mrc_scan_cols(out, 1, N, (double *)c->ws, 1.0, 0.0, st));
    return MRC_OK;
}

} // extern "C"
