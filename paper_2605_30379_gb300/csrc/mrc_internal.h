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
    int tma;                // CPLX source staged into shared memory by bulk copies (first stage)
    int chunk_fast;         // grid order: 1 = entry chunk in blockIdx.x, row offset j in blockIdx.y
    int *status;            // device status word: MRC_ERR_TIMEOUT (6) if a bounded wait gives up
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

// prof.cu: device status word that bounded in-kernel waits report timeouts to
// (the most recently created context's), and the FFT staging switch
// (MRC_FFT_TMA=1 turns bulk-copy staging of complex sources on; measured
// slower on the d = 64 workload, so off by default)
int *mrc_status_word(void);
void mrc_set_status_word(int *p);
bool mrc_fft_tma_enabled(void);
// elements of FFT scratch a transform of M points over E entries needs
static inline size_t mrc_fft_scratch_elems(int64_t M, int E) { return (size_t)M * (size_t)E; }

// prof.cu: every launch is bracketed by these (launch counter, optional timing)
void mrc_prof_pre(int kclass, cudaStream_t st);
void mrc_prof_post(int kclass, cudaStream_t st, double bytes, double flops);

// Per-precision launchers (k_f64.cu, k_f32.cu, k_dd.cu).
#define MRC_DECLARE_PREC(SUF)                                                                         \
    cudaError_t mrc_fft_##SUF(const FftSrc &src, const FftDst &dst, int64_t M, int E, int dir,        \
                              void *scratch, const void *tw, int tw_log, cudaStream_t st);            \
    cudaError_t mrc_pairmul_##SUF(const void *zx, const void *zy, void *zc, int64_t M, int r, int m,  \
                                  int c, const void *tw, int tw_log, cudaStream_t st);                \
    cudaError_t mrc_pairmul_cfg_##SUF(const void *zx, const void *zy, void *zc, int64_t M, int r,     \
                                      int m, int c, int cfg, const void *tw, int tw_log,              \
                                      cudaStream_t st);                                               \
    cudaError_t mrc_pairdiag_##SUF(const void *zx, const void *zy, void *zc, int64_t M, int r, int c, \
                                   const void *tw, int tw_log, cudaStream_t st);                      \
    cudaError_t mrc_twiddles_##SUF(void *tw, int tw_log, cudaStream_t st);                            \
    cudaError_t mrc_init_##SUF(void);

MRC_DECLARE_PREC(f64)
MRC_DECLARE_PREC(f32)
MRC_DECLARE_PREC(dd)

// Element sizes of one complex value per precision.
static inline size_t mrc_cx_bytes(int prec) { return prec == PREC_F32 ? 8 : 16; }

// ozaki.cu: double-float and FP32 square products (32 <= d <= 64) on BF16 tensor cores
bool mrc_ozaki_supported(int r, int m, int c);
cudaError_t mrc_ozaki_init(void);
cudaError_t mrc_pairmul_dd_ozaki(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw,
                                 int tw_log, cudaStream_t st);
cudaError_t mrc_pairmul_f32_ozaki(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw,
                                  int tw_log, cudaStream_t st);

// ozaki_tc.cu: the same digit products on the tcgen05 tensor cores (TMEM accumulators)
bool mrc_tc_supported(int r, int m, int c);
cudaError_t mrc_tc_init(void);
cudaError_t mrc_pairmul_dd_tc(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                              cudaStream_t st);
cudaError_t mrc_pairmul_f32_tc(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                               cudaStream_t st);

// tf32x3.cu: FP32 square products (16 <= d <= 64) as three TF32 tensor-core products
bool mrc_tf32x3_supported(int r, int m, int c);
cudaError_t mrc_tf32x3_init(void);
cudaError_t mrc_pairmul_f32_tf32x3(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw,
                                   int tw_log, cudaStream_t st);

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
cudaError_t mrc_mre_operator(const double *Q, double *A, int d, int64_t N, int scheme, cudaStream_t st);
cudaError_t mrc_mre_rhs(const double *Q, const double *L, double *R, int d, int c, int64_t N, cudaStream_t st);
