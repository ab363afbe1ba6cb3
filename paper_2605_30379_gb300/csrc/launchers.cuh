// launchers.cuh -- host-side launchers for one working precision T.  Each
// k_<prec>.cu includes this file once with MRC_T / MRC_SUF defined.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <type_traits>
#include <utility>
#include "kernels.cuh"

// table[ec_index][logR] (ec_index 0: default entries per CTA, 1: 4), filled by
// the two FFT translation units of this precision (low and high radices);
// specialised once per precision by MRC_DEFINE_PREC.
template <class T>
const FftEntry (&fft_table())[2][11];
template <class T>
const FftSegEntry (&fft_seg_table())[11];

namespace {

inline int ilog2_i64(int64_t x)
{
    int l = 0;
    while (((int64_t)1 << l) < x) ++l;
    return l;
}

template <class T> constexpr int kclass_fft();
template <> constexpr int kclass_fft<double>() { return 1; }
template <> constexpr int kclass_fft<float>() { return 2; }
template <> constexpr int kclass_fft<dd>() { return 3; }
template <class T> constexpr int kclass_pair() { return kclass_fft<T>() + 3; }

template <class T>
constexpr int default_ec() { return fft_default_ec<T>(); }

// entries per CTA: the full default when E allows, else 4 (>= 32-byte row
// segments; lanes beyond E idle)
template <class T>
int pick_ec(int E) { return E >= default_ec<T>() ? default_ec<T>() : 4; }

template <class T>
size_t fft_smem_bytes(int logR, int ec)
{
    const size_t R = (size_t)1 << logR;
    return (R * ec + 2 * R) * sizeof(cx<T>);
}

template <class T>
int ec_index(int ec) { return ec == default_ec<T>() ? 0 : 1; }

// Radix plan: one pass up to 2^10, else two passes of sizes 2^ceil(l/2), 2^floor(l/2).
inline int fft_plan(int logM, int *logRs)
{
    if (logM <= 10) { logRs[0] = logM; return 1; }
    logRs[0] = (logM + 1) / 2;
    logRs[1] = logM / 2;
    return 2;
}

// The passes and entries per CTA of `plan` (see mrc_internal.h), or the
// built-in ones when the plan does not fit logM.
inline int fft_plan_apply(int logM, int plan, int *logRs, bool *ec4)
{
    *ec4 = plan >= 0 && ((plan >> 8) & 1);
    const int a = plan >= 0 ? (plan & 31) : -1;
    if (a == 0 && logM <= 10) { logRs[0] = logM; return 1; }
    if (a >= 1 && a <= 10 && logM - a >= 1 && logM - a <= 10) {
        logRs[0] = a;
        logRs[1] = logM - a;
        return 2;
    }
    *ec4 = false;
    return fft_plan(logM, logRs);
}

// The argument blocks of a transform's passes and the algorithmic charge of
// each (the valid source rows read once, the kept output written once,
// 5 M log2(R) real flops per entry, radix-2 convention).  seg: the default
// entries per CTA whatever E (the segmented passes exist for it only).
template <class T>
cudaError_t fft_build(const FftSrc &src, const FftDst &dst, int64_t M, int E, int dir, void *scratch, const void *tw,
                      int tw_log, int plan, bool seg, FftPasses &ps)
{
    const int logM = ilog2_i64(M);
    if (((int64_t)1 << logM) != M || logM > 20 || logM + 1 > tw_log) return cudaErrorInvalidValue;
    bool ec4 = false;
    ps.np = fft_plan_apply(logM, seg ? -1 : plan, ps.logR, &ec4);
    const int ec = seg ? default_ec<T>() : (ec4 ? 4 : pick_ec<T>(E));
    ps.ec = ec;
    const int sld = E;  // scratch row length (complex elements)
    int logNs = 0;
    for (int k = 0; k < ps.np; ++k) {
        FftArgs &a = ps.a[k];
        a = FftArgs{};
        a.M = M;
        a.logR = ps.logR[k];
        a.logNs = logNs;
        a.Ns = (int64_t)1 << logNs;
        a.E = E;
        a.ec = ec;
        a.dir = dir;
        a.tw = tw;
        a.tw_log = tw_log;
        if (k == 0) {
            a.src_mode = src.mode; a.src = src.ptr; a.src_row0 = src.row0; a.src_nvalid = src.nvalid;
            a.src_ld = src.ld; a.src_neg = src.neg;
        } else {
            a.src_mode = SRC_CPLX; a.src = scratch; a.src_row0 = 0; a.src_nvalid = M; a.src_ld = sld; a.src_neg = 0;
        }
        if (k == ps.np - 1) {
            a.dst_mode = dst.mode; a.dst = dst.ptr; a.dst_ld = dst.ld; a.dst_lo = dst.lo; a.dst_hi = dst.hi;
            a.dst_row0 = dst.row0; a.dst_scale = dst.scale; a.dst_eye_d = dst.eye_d;
            a.dst2 = (std::is_same<T, dd>::value && dst.mode == DST_CPLX) ? dst.ptr2 : nullptr;
            a.dst_base = dst.base;
        } else {
            a.dst_mode = DST_CPLX; a.dst = scratch; a.dst_ld = sld; a.dst_lo = 0; a.dst_hi = 0; a.dst_row0 = 0;
            a.dst_scale = 1.0; a.dst_eye_d = 0;
        }
        // 32-bit element offsets when every offset a pass forms fits
        {
            const int64_t lim = (int64_t)1 << 32;
            const int64_t src_span = (a.src_mode == SRC_CPLX ? M : 2 * M + 1) * (int64_t)a.src_ld + ec;
            const int64_t dst_span = a.dst_mode == DST_CPLX ? M * (int64_t)a.dst_ld + ec
                                                            : (a.dst_row0 + (a.dst_hi - a.dst_lo) + 1) * a.dst_ld + ec;
            a.src_off32 = src_span < lim;
            a.dst_off32 = dst_span < lim && a.dst_row0 >= 0 && a.dst_hi >= a.dst_lo;
        }
        a.dst_scale_f = (float)a.dst_scale;
        a.dst_scaled = a.dst_scale != 1.0;
        // entry chunk in blockIdx.x, row offset j in blockIdx.y: CTAs launched
        // together cover whole rows j + rho M / R (d = 64, N = 2^18: double-float
        // FFT 67.9 -> 66.6 ms against the other order, FP32 unchanged);
        // nrow = M / R <= 2^10 in every plan
        ps.nrow[k] = (unsigned)(M >> a.logR);
        ps.nchunk = (unsigned)((E + ec - 1) / ec);
        double rd, wr;
        if (a.src_mode == SRC_REAL64) rd = (double)std::min<int64_t>(a.src_nvalid, 2 * M) * E * 8.0;
        else if (a.src_mode == SRC_REAL32) rd = (double)std::min<int64_t>(a.src_nvalid, 2 * M) * E * 4.0;
        else rd = (double)std::min<int64_t>(a.src_nvalid, M) * E * sizeof(cx<T>);
        const double rows = (double)(a.dst_hi - a.dst_lo) * E;
        if (a.dst_mode == DST_CPLX) wr = (double)M * E * (sizeof(cx<T>) + (a.dst2 ? 8 : 0));
        else if (a.dst_mode == DST_REAL32) wr = rows * 4.0;
        else if (a.dst_mode == DST_REAL64_BASE32) wr = rows * 12.0;
        else wr = rows * 8.0 * (a.dst_mode == DST_REAL64_ADD ? 2.0 : 1.0);
        ps.bytes[k] = rd + wr;
        ps.flops[k] = 5.0 * (double)M * a.logR * E;
        logNs += a.logR;
    }
    return cudaSuccess;
}

template <class T>
cudaError_t fft_run(const FftSrc &src, const FftDst &dst, int64_t M, int E, int dir, void *scratch,
                    const void *tw, int tw_log, cudaStream_t st, int plan)
{
    FftPasses ps;
    cudaError_t e = fft_build<T>(src, dst, M, E, dir, scratch, tw, tw_log, plan, false, ps);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < ps.np; ++k) {
        const FftEntry &kn = fft_table<T>()[ec_index<T>(ps.ec)][ps.logR[k]];
        mrc_prof_pre(kclass_fft<T>(), st);
        kn.fn<<<dim3(ps.nchunk, ps.nrow[k]), kn.nt, fft_smem_bytes<T>(ps.logR[k], ps.ec), st>>>(ps.a[k]);
        mrc_prof_post(kclass_fft<T>(), st, ps.bytes[k], ps.flops[k]);
    }
    return cudaGetLastError();
}

// One segmented pass of radix 2^logR over nseg transforms (device tables of
// their argument blocks and first CTAs; nctas CTAs in all)
template <class T>
cudaError_t fft_seg_run(int logR, const SegParams<FftArgs> &P, unsigned nctas, double bytes, double flops,
                        cudaStream_t st)
{
    if (P.nseg <= 0 || nctas == 0) return cudaSuccess;
    const FftSegEntry &kn = fft_seg_table<T>()[logR];
    mrc_prof_pre(kclass_fft<T>(), st);
    kn.fn<<<nctas, kn.nt, fft_smem_bytes<T>(logR, default_ec<T>()), st>>>(P);
    mrc_prof_post(kclass_fft<T>(), st, bytes, flops);
    return cudaGetLastError();
}

template <class T, int BM, int BN, int BK, int TM, int TN>
cudaError_t pairmul_launch(const PairArgs &a, cudaStream_t st)
{
    const int tiles = ((a.r + BM - 1) / BM) * ((a.c + BN - 1) / BN);
    dim3 grid((unsigned)a.npairs, (unsigned)tiles);
    const double bytes = (double)a.M * ((double)a.r * a.m + (double)a.m * a.c + (double)a.r * a.c) * sizeof(cx<T>);
    const double flops = 8.0 * a.r * a.m * a.c * (double)(a.M + 1);
    mrc_prof_pre(kclass_pair<T>(), st);
    pairmul_kernel<T, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(a);
    mrc_prof_post(kclass_pair<T>(), st, bytes, flops);
    return cudaGetLastError();
}

template <class T, int BM, int BN, int BK, int TM, int TN>
cudaError_t pairmul2_launch(const PairArgs &a, cudaStream_t st)
{
    const int tiles = ((a.r + BM - 1) / BM) * ((a.c + BN - 1) / BN);
    dim3 grid((unsigned)a.npairs, (unsigned)tiles);
    const double bytes = (double)a.M * ((double)a.r * a.m + (double)a.m * a.c + (double)a.r * a.c) * sizeof(cx<T>);
    const double flops = 8.0 * a.r * a.m * a.c * (double)(a.M + 1);
    mrc_prof_pre(kclass_pair<T>(), st);
    pairmul2_kernel<T, BM, BN, BK, TM, TN><<<grid, 2 * (BM / TM) * (BN / TN), 0, st>>>(a);
    mrc_prof_post(kclass_pair<T>(), st, bytes, flops);
    return cudaGetLastError();
}

// product argument block and tile configuration: 0 = 16x16 (64 threads),
// 1 = 32x32 (256), 2 = 64x64 (256), 4 = 24x24 (96: 17 <= d <= 24 fills 50 .. 100 %
// of it against 28 .. 56 % of a 32x32 tile); cfg < 0 picks by the larger output dimension
inline PairArgs pairmul_args(const void *zx, const void *zy, void *zc, int64_t M, int r, int m, int c, const void *tw,
                             int tw_log)
{
    PairArgs a{};
    a.zx = zx; a.zy = zy; a.zc = zc; a.tw = tw; a.tw_log = tw_log; a.M = M; a.logM = ilog2_i64(M);
    a.npairs = M >= 2 ? M / 2 + 1 : 1;
    a.r = r; a.m = m; a.c = c;
    return a;
}
inline int pairmul_cfg_for(int r, int c, int cfg)
{
    const int mx = r > c ? r : c;
    return cfg >= 0 ? cfg : (mx <= 16 ? 0 : (mx <= 24 ? 4 : (mx <= 32 ? 1 : 2)));
}
// CTAs of one product: pairs x output tiles
inline unsigned pairmul_ctas(const PairArgs &a, int cfg)
{
    const int b = cfg == 0 ? 16 : (cfg == 1 ? 32 : (cfg == 4 ? 24 : 64));
    return (unsigned)a.npairs * (unsigned)(((a.r + b - 1) / b) * ((a.c + b - 1) / b));
}

template <class T>
cudaError_t pairmul_run(const void *zx, const void *zy, void *zc, int64_t M, int r, int m, int c, int cfg, const void *tw,
                        int tw_log, cudaStream_t st)
{
    const PairArgs a = pairmul_args(zx, zy, zc, M, r, m, c, tw, tw_log);
    cfg = pairmul_cfg_for(r, c, cfg);
    if (cfg == 0) return pairmul_launch<T, 16, 16, 16, 2, 2>(a, st);
    if (cfg == 1) return pairmul_launch<T, 32, 32, 16, 2, 2>(a, st);
    if (cfg == 4) return pairmul_launch<T, 24, 24, 8, 3, 2>(a, st);
    // FP32, 64 x 64 tiles: the frequencies of a pair on two halves of the CTA
    // (half the registers per thread, two CTAs per SM: pairmul_f32 54.9 ->
    // 49.4 ms at d = 64, N = 2^18 against both frequencies in every thread)
    if constexpr (std::is_same<T, float>::value) return pairmul2_launch<T, 64, 64, 8, 4, 4>(a, st);
    else return pairmul_launch<T, 64, 64, 8, 4, 4>(a, st);
}

// One segmented product launch of tile configuration cfg (resolved) over
// nseg products (device tables; nctas CTAs in all)
template <class T>
cudaError_t pairmul_seg_run(int cfg, const SegParams<PairArgs> &P, unsigned nctas, double bytes, double flops,
                            cudaStream_t st)
{
    if (P.nseg <= 0 || nctas == 0) return cudaSuccess;
    mrc_prof_pre(kclass_pair<T>(), st);
    if (cfg == 0) pairmul_seg_kernel<T, 16, 16, 16, 2, 2><<<nctas, 64, 0, st>>>(P);
    else if (cfg == 1) pairmul_seg_kernel<T, 32, 32, 16, 2, 2><<<nctas, 256, 0, st>>>(P);
    else if (cfg == 4) pairmul_seg_kernel<T, 24, 24, 8, 3, 2><<<nctas, 96, 0, st>>>(P);
    else if constexpr (std::is_same<T, float>::value) pairmul2_seg_kernel<T, 64, 64, 8, 4, 4><<<nctas, 512, 0, st>>>(P);
    else pairmul_seg_kernel<T, 64, 64, 8, 4, 4><<<nctas, 256, 0, st>>>(P);
    mrc_prof_post(kclass_pair<T>(), st, bytes, flops);
    return cudaGetLastError();
}

template <class T>
cudaError_t pairdiag_run(const void *zx, const void *zy, void *zc, int64_t M, int r, int c, const void *tw,
                         int tw_log, cudaStream_t st)
{
    PairArgs a{};
    a.zx = zx; a.zy = zy; a.zc = zc; a.tw = tw; a.tw_log = tw_log; a.M = M; a.logM = ilog2_i64(M);
    a.npairs = M >= 2 ? M / 2 + 1 : 1;
    a.r = r; a.m = 0; a.c = c;
    const int64_t total = a.npairs * (int64_t)r * c;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    const double bytes = (double)M * (2.0 * r * c + c) * sizeof(cx<T>);
    mrc_prof_pre(kclass_pair<T>(), st);
    pairdiag_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(a);
    mrc_prof_post(kclass_pair<T>(), st, bytes, 6.0 * r * c * (double)(M + 1));
    return cudaGetLastError();
}

template <class T>
cudaError_t twiddles_run(void *tw, int tw_log, cudaStream_t st)
{
    mrc_prof_pre(7, st);
    twiddle_kernel<T><<<152 * 8, 256, 0, st>>>(reinterpret_cast<cx<T> *>(tw), tw_log);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

template <class T>
cudaError_t init_run()
{
    const auto &t = fft_table<T>();
    for (int i = 0; i < 2; ++i)
        for (int l = 0; l < 11; ++l) {
            cudaError_t e = cudaFuncSetAttribute(t[i][l].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (e != cudaSuccess) return e;
        }
    const auto &ts = fft_seg_table<T>();
    for (int l = 0; l < 11; ++l) {
        cudaError_t e = cudaFuncSetAttribute(ts[l].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

} // namespace

#define MRC_DEFINE_PREC(T, SUF)                                                                             \
    void mrc_fft_fill_##SUF##_lo(FftEntry (*t)[11], FftSegEntry *ts);                                       \
    void mrc_fft_fill_##SUF##_hi(FftEntry (*t)[11], FftSegEntry *ts);                                       \
    struct FftTables_##SUF {                                                                                \
        FftEntry t[2][11];                                                                                  \
        FftSegEntry ts[11];                                                                                 \
        FftTables_##SUF()                                                                                   \
        {                                                                                                   \
            mrc_fft_fill_##SUF##_lo(t, ts);                                                                 \
            mrc_fft_fill_##SUF##_hi(t, ts);                                                                 \
        }                                                                                                   \
    };                                                                                                      \
    static const FftTables_##SUF &fft_tables_##SUF()                                                        \
    {                                                                                                       \
        static const FftTables_##SUF tb;                                                                    \
        return tb;                                                                                          \
    }                                                                                                       \
    template <>                                                                                             \
    const FftEntry (&fft_table<T>())[2][11] { return fft_tables_##SUF().t; }                                \
    template <>                                                                                             \
    const FftSegEntry (&fft_seg_table<T>())[11] { return fft_tables_##SUF().ts; }                           \
    cudaError_t mrc_fft_build_##SUF(const FftSrc &src, const FftDst &dst, int64_t M, int E, int dir,          \
                                    void *scratch, const void *tw, int tw_log, FftPasses &ps)               \
    {                                                                                                       \
        return fft_build<T>(src, dst, M, E, dir, scratch, tw, tw_log, -1, true, ps);                        \
    }                                                                                                       \
    cudaError_t mrc_fft_seg_##SUF(int logR, const SegParams<FftArgs> &P, unsigned nctas, double bytes,       \
                                  double flops, cudaStream_t st)                                            \
    {                                                                                                       \
        return fft_seg_run<T>(logR, P, nctas, bytes, flops, st);                                            \
    }                                                                                                       \
    cudaError_t mrc_pairmul_seg_##SUF(int cfg, const SegParams<PairArgs> &P, unsigned nctas, double bytes,   \
                                      double flops, cudaStream_t st)                                        \
    {                                                                                                       \
        return pairmul_seg_run<T>(cfg, P, nctas, bytes, flops, st);                                         \
    }                                                                                                       \
    cudaError_t mrc_fft_##SUF(const FftSrc &src, const FftDst &dst, int64_t M, int E, int dir, void *scratch, \
                              const void *tw, int tw_log, cudaStream_t st, int plan)                        \
    {                                                                                                       \
        return fft_run<T>(src, dst, M, E, dir, scratch, tw, tw_log, st, plan);                              \
    }                                                                                                       \
    cudaError_t mrc_pairmul_##SUF(const void *zx, const void *zy, void *zc, int64_t M, int r, int m, int c,   \
                                  const void *tw, int tw_log, cudaStream_t st)                              \
    {                                                                                                       \
        return pairmul_run<T>(zx, zy, zc, M, r, m, c, -1, tw, tw_log, st);                                  \
    }                                                                                                       \
    cudaError_t mrc_pairmul_cfg_##SUF(const void *zx, const void *zy, void *zc, int64_t M, int r, int m,      \
                                      int c, int cfg, const void *tw, int tw_log, cudaStream_t st)          \
    {                                                                                                       \
        return pairmul_run<T>(zx, zy, zc, M, r, m, c, cfg, tw, tw_log, st);                                 \
    }                                                                                                       \
    cudaError_t mrc_pairdiag_##SUF(const void *zx, const void *zy, void *zc, int64_t M, int r, int c,         \
                                   const void *tw, int tw_log, cudaStream_t st)                             \
    {                                                                                                       \
        return pairdiag_run<T>(zx, zy, zc, M, r, c, tw, tw_log, st);                                        \
    }                                                                                                       \
    cudaError_t mrc_twiddles_##SUF(void *tw, int tw_log, cudaStream_t st) { return twiddles_run<T>(tw, tw_log, st); } \
    cudaError_t mrc_init_##SUF(void) { return init_run<T>(); }
