// mrc_internal.h -- argument blocks and launcher declarations shared by the
// per-precision kernel units and the host driver.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Real sources and destinations hold pairs of rows (2k, 2k+1) per packed
// complex point.  REAL32: binary32 rows.  DST_REAL64_BASE32: out = base + x
// with base the binary32 rows of FftArgs::dst_base (same indexing as out).
enum { SRC_CPLX = 0, SRC_REAL64 = 1, SRC_REAL32 = 2 };
enum { DST_CPLX = 0, DST_REAL64 = 1, DST_REAL64_ADD = 2, DST_REAL32 = 3, DST_REAL64_BASE32 = 4 };
enum { PREC_F64 = 0, PREC_F32 = 1, PREC_DD = 2 };

struct FftArgs {
    int64_t M;      // transform length, power of two
    int logR;       // this pass: radix 2^logR
    int logNs;      // product of earlier radices = 2^logNs
    int64_t Ns;
    int E;          // entries per row processed
    int ec;         // entries per CTA
    int dir;        // -1 forward (exp(-2 pi i ...)), +1 inverse (no 1/M; see dst_scale)
    const void *tw; // forward twiddle table of 2^tw_log entries (working precision)
    int tw_log;
    // source
    int src_mode;
    const void *src;
    int64_t src_row0;   // first row read
    int64_t src_nvalid; // CPLX: valid packed rows; REAL64: valid real rows; beyond: zero
    int src_ld;         // row stride (elements)
    int src_neg;
    // destination
    int dst_mode;
    void *dst;
    int dst_ld;
    int64_t dst_lo, dst_hi; // REAL64*: kept window of real rows
    int64_t dst_row0;       // REAL64*: destination row of real row dst_lo
    double dst_scale;       // signed power of two
    float dst_scale_f;      // the same, for the FP32-based precisions
    int dst_scaled;         // dst_scale != 1 (decided on the host: no FP64 compare in the kernels)
    int dst_eye_d;          // REAL64*: if > 0 add 1 to the diagonal of real row 0 (d = this)
    void *dst2;             // double-float DST_CPLX only: also write the hi parts here as FP32 complex (or null)
    const void *dst_base;   // DST_REAL64_BASE32: binary32 rows added to the result
    int src_off32, dst_off32; // every source / destination element offset of the pass fits 32 bits
};

struct PairArgs {
    const void *zx, *zy;
    void *zc;
    const void *tw;
    int tw_log;
    int64_t M;
    int logM;
    int64_t npairs;
    int r, m, c; // X: r x m, Y: m x c (pairdiag: Y is a c-vector, m unused)
    // tensor-core double-float product with X prepared (mrc_tcp_prep): zx
    // holds X's digit tiles, xs its per-pair scale factors; else null
    const void *xs;
};

// Source / destination descriptors used by the host-side FFT driver.
struct FftSrc {
    int mode;
    const void *ptr;
    int64_t row0, nvalid;
    int ld;
    int neg;
};
struct FftDst {
    int mode;
    void *ptr;
    int ld;
    int64_t lo, hi, row0;
    double scale;
    int eye_d;
    void *ptr2 = nullptr;  // double-float DST_CPLX: FP32 copy of the hi parts (FftArgs::dst2)
    const void *base = nullptr;  // DST_REAL64_BASE32: binary32 rows (FftArgs::dst_base)
};

// Segmented launches: one launch over several independent pieces of work of
// one shape class (the models of a batch at one stage).  The pieces'
// argument blocks travel in the kernel's parameter space as one
// __grid_constant__ block (at most 32764 bytes: MRC_SEG_MAX x
// (sizeof(FftArgs) + 4)), read through the constant cache like a single
// launch's arguments.  CTA b belongs to segment s = max{s : first[s] <= b}.
#define MRC_SEG_MAX 144
template <class A>
struct SegParams {
    int nseg;
    unsigned first[MRC_SEG_MAX];
    A a[MRC_SEG_MAX];
};

template <class A>
__device__ __forceinline__ int seg_find(const SegParams<A> &P, unsigned b)
{
    int lo = 0, hi = P.nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.first[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// argument blocks of the batched Gauss-Jordan, base-case and conversion kernels
struct GjArgs {
    const double *A0;
    double *out, *W;
    int d;
    int *status;
};
struct BaseArgs {
    const double *A;
    double *psi;
    int d, m0;
};
struct CvtArgs {
    const double *x;
    float *y;
    int64_t n;
};
#define MRC_CVT_CHUNK 8192  // elements per CTA of the segmented conversion

// The passes of one transform (at most two): argument blocks, radices, the
// algorithmic charge of each, and the launch shape (nchunk entry chunks of ec
// entries x nrow rows per pass)
struct FftPasses {
    int np;
    int logR[2];
    FftArgs a[2];
    double bytes[2], flops[2];
    unsigned nchunk, nrow[2];
    int ec;
};

// elements of FFT scratch a transform of M points over E entries needs
static inline size_t mrc_fft_scratch_elems(int64_t M, int E) { return (size_t)M * (size_t)E; }

// prof.cu: every launch is bracketed by these (launch counter, optional timing)
void mrc_prof_pre(int kclass, cudaStream_t st);
void mrc_prof_post(int kclass, cudaStream_t st, double bytes, double flops);

// Per-precision launchers (k_f64.cu, k_f32.cu, k_dd.cu).
// An FFT plan: -1 the built-in one (one pass up to 2^10 points, else two
// passes of 2^ceil(l/2) and 2^floor(l/2); the default entries per CTA), or
// plan bits 0-4 = log2 of the first pass's radix (0: one pass), bit 8 = four
// entries per CTA.  Plans that do not fit the transform fall back to the
// built-in one.
#define MRC_DECLARE_PREC(SUF)                                                                         \
    cudaError_t mrc_fft_##SUF(const FftSrc &src, const FftDst &dst, int64_t M, int E, int dir,        \
                              void *scratch, const void *tw, int tw_log, cudaStream_t st,             \
                              int plan = -1);                                                         \
    cudaError_t mrc_pairmul_##SUF(const void *zx, const void *zy, void *zc, int64_t M, int r, int m,  \
                                  int c, const void *tw, int tw_log, cudaStream_t st);                \
    cudaError_t mrc_pairmul_cfg_##SUF(const void *zx, const void *zy, void *zc, int64_t M, int r,     \
                                      int m, int c, int cfg, const void *tw, int tw_log,              \
                                      cudaStream_t st);                                               \
    cudaError_t mrc_pairdiag_##SUF(const void *zx, const void *zy, void *zc, int64_t M, int r, int c, \
                                   const void *tw, int tw_log, cudaStream_t st);                      \
    cudaError_t mrc_twiddles_##SUF(void *tw, int tw_log, cudaStream_t st);                            \
    cudaError_t mrc_init_##SUF(void);                                                                 \
    cudaError_t mrc_fft_build_##SUF(const FftSrc &src, const FftDst &dst, int64_t M, int E, int dir,    \
                                    void *scratch, const void *tw, int tw_log, FftPasses &ps);        \
    cudaError_t mrc_fft_seg_##SUF(int logR, const SegParams<FftArgs> &P, unsigned nctas, double bytes,  \
                                  double flops, cudaStream_t st);                                     \
    cudaError_t mrc_pairmul_seg_##SUF(int cfg, const SegParams<PairArgs> &P, unsigned nctas,            \
                                      double bytes, double flops, cudaStream_t st);

MRC_DECLARE_PREC(f64)
MRC_DECLARE_PREC(f32)
MRC_DECLARE_PREC(dd)

// Element sizes of one complex value per precision.
static inline size_t mrc_cx_bytes(int prec) { return prec == PREC_F32 ? 8 : 16; }

// ozaki_tc.cu: double-float square products (32 <= d <= 512) as exact digit
// products on the tcgen05 tensor cores (TMEM accumulators); a bounded wait
// that gives up writes MRC_ERR_TIMEOUT (6) to *status
bool mrc_tc_supported(int r, int m, int c);
cudaError_t mrc_tc_init(void);
cudaError_t mrc_pairmul_dd_tc(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                              int *status, cudaStream_t st);
// pair_tc.cu: the pipelined, warp-specialised tcgen05 digit products for
// square 32 <= d <= 64, double-float (the residual) and FP32 (Newton levels
// and correction); timeouts as above
bool mrc_tcp_supported(int r, int m, int c);
cudaError_t mrc_tcp_init(void);
cudaError_t mrc_pairmul_dd_tcp(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                               int *status, cudaStream_t st);
cudaError_t mrc_pairmul_f32_tcp(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                                int *status, cudaStream_t st);
// the same over the products of one segmented launch (all of the same M and
// of the same ceil(d / 16)); a timeout is reported in *status
cudaError_t mrc_tcp_seg(int dd_prec, const SegParams<PairArgs> &P, int *status, cudaStream_t st);
PairArgs mrc_tcp_args(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log);
// The double-float product with X prepared once (X is the spectrum of A,
// the same in every residual sweep): mrc_tcp_prep writes, for every product
// of P (zx: X's packed spectrum, zc: tiles out, xs: scales out;
// mrc_tcp_prep_bytes and mrc_tcp_prep_scale_bytes each), X's digit tiles and
// row scales; a product whose PairArgs carry xs (zx: the tiles) then splits
// only Y.
size_t mrc_tcp_prep_bytes(int64_t M, int d);
size_t mrc_tcp_prep_scale_bytes(int64_t M);
cudaError_t mrc_tcp_prep(const SegParams<PairArgs> &P, cudaStream_t st);
// the kernels' bounded mbarrier wait on a barrier nothing arrives on: writes 6 to *status
cudaError_t mrc_tc_wait_selftest(int *status, int spins, cudaStream_t st);

// api.cu: the Newton doubling schedule of Eq. (newton), shared by every
// inverse entry point (mrc_inverse* and mrc_inverse_noalloc).
//   mrc_base_size: the first m0 coefficients come from the direct recursion;
//   mrc_newton_maxM: the largest level m (its transforms have M = m points).
int64_t mrc_base_size(int d, int64_t N);
int64_t mrc_newton_maxM(int d, int64_t N);
// Row ranges of A still being uploaded (mrc_inverse_host): rows
// [end[i-1], end[i]) complete at ev[i]; wait(s, rows) makes stream s wait
// until rows [0, rows) are on the device.  n == 0: everything is there.
struct RowWait {
    int n = 0;
    int64_t end[32] = {};
    cudaEvent_t ev[32] = {};
    cudaError_t wait(cudaStream_t s, int64_t rows) const
    {
        for (int i = 0; i < n; ++i)
            if (end[i] >= rows) return cudaStreamWaitEvent(s, ev[i], 0);
        return n ? cudaStreamWaitEvent(s, ev[n - 1], 0) : cudaSuccess;
    }
};
// The transform a level uses (an mrc_fft_<prec> call, perhaps with a tuned plan)
typedef cudaError_t (*mrc_level_fft_fn)(void *user, int prec, const FftSrc &src, const FftDst &dst, int64_t M, int E,
                                        int dir, void *scratch, const void *tw, int tw_log, cudaStream_t st);
// The per-frequency product a level uses: zc = zx * zy at the M/2 + 1
// frequency pairs of (PREC_F64 or PREC_F32) spectra of length M, d x d.
typedef cudaError_t (*mrc_level_product_fn)(void *user, int prec, const void *zx, const void *zy, void *zc,
                                            int64_t M, int d, const void *tw, int tw_log, cudaStream_t st);
// Buffers of the levels: three spectra and the FFT scratch, each
// mrc_newton_maxM(d, N) * d^2 complex values of the working precision.
struct NewtonBufs {
    void *b0, *b1, *b2, *bt;
};
// Levels m0 -> N on `st`: psi rows [0, m0) are already correct.  With A32 /
// psi32 (FP32 levels of the mixed path) A is read from its binary32 copy,
// converted here row range by row range, and psi is read and written in
// binary32.  rw (nullable) delays each level until its rows of A arrived.
// Returns 0 or 4 (a CUDA error, printed); *levels (nullable) = levels run.
// a32_rows: rows of A32 already converted by the caller (the rest are
// converted level by level, as each level first reads them)
int mrc_newton_levels(int prec, int d, int64_t N, const double *A, double *psi, int64_t m0, const NewtonBufs &b,
                      const void *tw, int tw_log, mrc_level_fft_fn fft, mrc_level_product_fn product, void *user,
                      cudaStream_t st, const RowWait *rw, float *A32, float *psi32, int *levels,
                      int64_t a32_rows = 0);

// misc.cu
cudaError_t mrc_gauss_jordan(const double *A0, double *out, double *work, int d, int *status, cudaStream_t st);
cudaError_t mrc_base_case(const double *A, double *psi, int d, int64_t m0, cudaStream_t st);
cudaError_t mrc_row_sums(const double *q, double *rs, int d, int64_t N, cudaStream_t st);
cudaError_t mrc_scan_cols(double *x, int ncol, int64_t N, double *work, double scale, double offset,
                          cudaStream_t st);
cudaError_t mrc_norms(const double *rho, int E, int64_t N, double *acc, cudaStream_t st);
cudaError_t mrc_gather_blocks(const double *q, int d, int64_t N, const int *Cidx, int nC, const int *Didx,
                              int nD, double *ACC, double *QCD, cudaStream_t st);
cudaError_t mrc_weighted_rowsum(const double *g, int nC, int nD, int64_t N, const double *alpha, double *out,
                                cudaStream_t st);
cudaError_t mrc_occupation_k(const double *P, int d, int64_t N, const double *alpha, const int *inB, double *out,
                             cudaStream_t st);
cudaError_t mrc_one_minus(const double *x, double *y, int64_t n, cudaStream_t st);
cudaError_t mrc_f64_to_f32(const double *x, float *y, int64_t n, cudaStream_t st);
// batched: Gauss-Jordan of every segment's A(0) (one CTA each, dmax the
// largest d), the direct recursion (dmax x nseg CTAs), and conversions
// (P.first: CTA starts in MRC_CVT_CHUNK elements; nctas in all)
cudaError_t mrc_gauss_jordan_batch(const SegParams<GjArgs> &P, int dmax, cudaStream_t st);
cudaError_t mrc_base_case_batch(const SegParams<BaseArgs> &P, int dmax, cudaStream_t st);
cudaError_t mrc_f64_to_f32_batch(const SegParams<CvtArgs> &P, unsigned nctas, cudaStream_t st);
// series Gauss-Jordan on W = [P_A | I] ([N][d][2d]): build W (clearing the
// call's singular flag), choose the pivot of column col and exchange rows
// (with the pivot series u [N] and the elimination factors cv [N][d]), take
// psi from the right block (NaN if the flag is set)
cudaError_t mrc_gjs_init(const double *A, double *W, int d, int64_t N, int *flag, cudaStream_t st);
cudaError_t mrc_gjs_pivot(const double *A0, double *W, int d, int64_t N, int col, int *piv, double *u, double *cv,
                          int *flag, int *status, cudaStream_t st);
cudaError_t mrc_gjs_extract(const double *W, double *psi, int d, int64_t N, const int *flag, cudaStream_t st);
cudaError_t mrc_mre_operator(const double *Q, double *A, int d, int64_t N, int scheme, cudaStream_t st);
cudaError_t mrc_mre_rhs(const double *Q, const double *L, double *R, int d, int c, int64_t N, cudaStream_t st);
