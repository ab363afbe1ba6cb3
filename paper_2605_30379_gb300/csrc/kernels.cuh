// kernels.cuh -- FFT stages and per-frequency matrix products of the
// FFT-Newton inversion, templated on the working precision T (float, double,
// dd).  Included by one translation unit per precision.
//
// Layout.  A matrix sequence in time or frequency is a 2-D array [rows][E]
// with E = r*c matrix entries contiguous per row (time / frequency slowest).
// FFTs run down the slow axis for all E entries at once, so every global
// access is a row segment of contiguous entries, coalesced for any transform
// stride, and no transpose pass is ever needed.
//
// Real sequences of length L = 2M are transformed by one complex FFT of length
// M of the packed sequence z_k = x_{2k} + i x_{2k+1}.  Splitting the packed
// spectrum into the real-input spectrum needs the partner frequency M-f; that
// split (and its inverse) is fused into the product kernel, which handles the
// frequency pair {f, M-f} in one CTA.  Frequency-domain products then cover
// exactly the L/2+1 frequencies of the half spectrum (Eq. (fft-convolution)
// restricted to Hermitian spectra).
#pragma once
#include <type_traits>
#include <utility>

#include "arith.cuh"
#include "mrc_internal.h"

// ---------------------------------------------------------------------------
// FFT pass: one radix-R Stockham step of a length-M transform (R = 2^logR,
// Ns = product of the earlier radices).  CTA (j, chunk) loads the R elements
// j + r*M/R of EC consecutive entries, applies the inter-pass twiddles
// W_{Ns R}^{(j mod Ns) r}, runs the length-R DFT as in-CTA Stockham stages of
// radix 2/4 then 8 with the points of each butterfly in registers and one
// shared-memory exchange per stage, and writes element f to
// (j/Ns)*Ns*R + (j mod Ns) + f*Ns.  After the last pass the output is in
// natural frequency order.  The global loads and stores of a pass are in
// fft_gather and fft_stage's store_global below.

// multiply by the (signed power of two) output scale in the working precision
template <class T>
__device__ __forceinline__ cx<T> scale_out(const FftArgs &a, cx<T> v)
{
    if constexpr (sizeof(T) == 8 && sizeof(cx<T>) == 16 && !__is_same(T, dd)) return c_scal(v, a.dst_scale);
    else return {Ar<T>::scal_f(v.re, a.dst_scale_f), Ar<T>::scal_f(v.im, a.dst_scale_f)};
}

// Small DFTs in registers, natural order in and out.  INV selects the sign
// of the exponent (+ for the inverse transform).
template <class T, bool INV>
__device__ __forceinline__ cx<T> mul_mi(cx<T> a)  // a * (-i) forward, a * (+i) inverse
{
    return INV ? cx<T>{Ar<T>::neg(a.im), a.re} : cx<T>{a.im, Ar<T>::neg(a.re)};
}

template <class T, bool INV>
__device__ __forceinline__ void dft2(cx<T> *v)
{
    cx<T> t = v[0];
    v[0] = c_add_nn(t, v[1]);
    v[1] = c_sub_nn(t, v[1]);
}

template <class T, bool INV>
__device__ __forceinline__ void dft4(cx<T> *v)
{
    cx<T> c0 = c_add_nn(v[0], v[2]), c2 = c_sub_nn(v[0], v[2]);
    cx<T> c1 = c_add_nn(v[1], v[3]), c3 = mul_mi<T, INV>(c_sub_nn(v[1], v[3]));
    v[0] = c_add_nn(c0, c1);
    v[2] = c_sub_nn(c0, c1);
    v[1] = c_add_nn(c2, c3);
    v[3] = c_sub_nn(c2, c3);
}

// radix-8 = one radix-2 step (decimation in frequency) + two radix-4 DFTs
template <class T, bool INV>
__device__ __forceinline__ void dft8(cx<T> *v)
{
    const T s = Ar<T>::rsqrt2();
    cx<T> a[4], b[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        a[n] = c_add_nn(v[n], v[n + 4]);
        b[n] = c_sub_nn(v[n], v[n + 4]);
    }
    // b_n *= W_8^{n} (forward) or W_8^{-n} (inverse)
    {
        cx<T> x = b[1];
        b[1] = INV ? cx<T>{Ar<T>::mul(Ar<T>::sub_nn(x.re, x.im), s), Ar<T>::mul(Ar<T>::add_nn(x.re, x.im), s)}
                   : cx<T>{Ar<T>::mul(Ar<T>::add_nn(x.re, x.im), s), Ar<T>::mul(Ar<T>::sub_nn(x.im, x.re), s)};
        b[2] = mul_mi<T, INV>(b[2]);
        x = b[3];
        b[3] = INV ? cx<T>{Ar<T>::mul(Ar<T>::neg(Ar<T>::add_nn(x.re, x.im)), s), Ar<T>::mul(Ar<T>::sub_nn(x.re, x.im), s)}
                   : cx<T>{Ar<T>::mul(Ar<T>::sub_nn(x.im, x.re), s), Ar<T>::mul(Ar<T>::neg(Ar<T>::add_nn(x.re, x.im)), s)};
    }
    dft4<T, INV>(a);
    dft4<T, INV>(b);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = a[k];
        v[2 * k + 1] = b[k];
    }
}

// The adds inside one small DFT skip the double-float normalisation
// (c_add_nn); dft_r normalises its outputs once.
template <class T, bool INV, int LR, bool NORM = true>
__device__ __forceinline__ void dft_r(cx<T> *v)
{
    if constexpr (LR == 0) return;
    else {
        if constexpr (LR == 1) dft2<T, INV>(v);
        else if constexpr (LR == 2) dft4<T, INV>(v);
        else dft8<T, INV>(v);
        if constexpr (__is_same(T, dd) && NORM) {
#pragma unroll
            for (int q = 0; q < (1 << LR); ++q) v[q] = c_norm(v[q]);
        }
    }
}

// Entries per CTA of the passes: for 8-byte complex values (FP32) 16, i.e.
// 128-byte row segments and 16 points per thread in the radix-2^9 and 2^10
// passes.  At d = 64, N = 2^18, once the passes' index arithmetic was
// strength-reduced, the FP32 FFT took 55.4 ms with 16 against 74.9 ms with 8
// (with 8 the passes were bound by the L1 / shared-memory pipe at 86 % of
// peak); before that, 8 had been the faster (103.5 against 111.6 ms).  For
// 16-byte values (FP64, double-float) 8: double-float with 16 went
// 50.9 -> 59.8 ms.
#ifndef MRC_F32_EC
#define MRC_F32_EC 16
#endif
#ifndef MRC_DD_EC
#define MRC_DD_EC 8
#endif
// Double-float passes normalise their points only after the last in-CTA
// stage (before the store): the adds and dot products of the earlier stages
// accept unnormalised operands, and the low parts stay within a few ulps of
// the high parts (error a small multiple of 2^-48 |x|).  d = 64, N = 2^18:
// double-float FFT 51.0 -> 49.6 ms against normalising after every stage,
// max |rho_L| 7.51e-14 either way.
template <class T>
constexpr int fft_default_ec() { return sizeof(cx<T>) == 8 ? MRC_F32_EC : MRC_DD_EC; }

// Threads per CTA at most: 1024 for the FP32 passes (the radix-2^9 pass at
// 16 entries then runs 1024 threads of 8 points, two CTAs per SM, instead
// of 512 threads of 16 points: FP32 FFT 55.4 -> 53.3 ms at d = 64,
// N = 2^18), 512 for the others.
#ifndef MRC_FFT32_NTMAX
#define MRC_FFT32_NTMAX 1024
#endif

// Compile-time plan of one pass: R = 2^LOGR points split into in-CTA stages
// of radix 2^FIRST then 8, 8, ...; EC entries per CTA; NT threads, each
// holding EPT points in registers.
template <class T, int LOGR, int EC>
struct FftPlan {
    static constexpr int R = 1 << LOGR;
    static constexpr int FIRST = (LOGR < 3) ? LOGR : ((LOGR % 3) == 0 ? 3 : (LOGR % 3));
    static constexpr int NSTAGE = (LOGR < 3) ? 1 : 1 + (LOGR - FIRST) / 3;
    static constexpr int LRMAX = (LOGR < 3) ? LOGR : 3;
    static constexpr int UNITS = (R >> LRMAX) * EC;        // butterflies in a max-radix stage
    static constexpr int NTMAX = (sizeof(cx<T>) == 8) ? MRC_FFT32_NTMAX : 512;
    static constexpr int UB = UNITS > NTMAX ? UNITS / NTMAX : 1;
    static constexpr int NT = UNITS / UB;
    static constexpr int EPT = UB << LRMAX;               // points per thread
    static constexpr int LEC = EC == 1 ? 0 : EC == 2 ? 1 : EC == 4 ? 2 : EC == 8 ? 3 : 4;
};

// Element offsets of the first-stage loads and last-stage stores: a CTA's
// points sit at offset o0 + q * dq from a per-CTA base pointer (q the point
// index inside a thread's butterfly), so each point costs one multiply-add
// and one address formation.  With OFF32 (every offset of the launch below
// 2^32 elements, decided on the host) the offsets are 32-bit.
template <bool OFF32>
using fft_off_t = typename std::conditional<OFF32, unsigned, int64_t>::type;

// The first stage's global loads: x[u * r + q] = point rho = b + q R / r of
// unit u, i.e. packed row k = j + rho M / R (a complex row, or the real rows
// 2k and 2k + 1); zero past the valid rows and past the entry count.
template <class T, int LOGR, int EC, int SRC, bool OFF32>
__device__ __forceinline__ void fft_gather(const FftArgs &a, cx<T> *x, int64_t j, int e0, int ecount)
{
    using P = FftPlan<T, LOGR, EC>;
    using Off = fft_off_t<OFF32>;
    using Elt = typename std::conditional<SRC == SRC_CPLX, cx<T>,
                                          typename std::conditional<SRC == SRC_REAL32, float, double>::type>::type;
    constexpr int R = P::R, NT = P::NT, r = 1 << P::FIRST, UPT = P::EPT / r;
    constexpr int ROWS = SRC == SRC_CPLX ? 1 : 2;  // stored rows per packed point
    const int tid = threadIdx.x;
    const int S = (int)(a.M >> LOGR);
    const int ld = a.src_ld;
    const int nv = (int)(a.src_nvalid < 0x7fffffff ? a.src_nvalid : 0x7fffffff);
    const Elt *base = reinterpret_cast<const Elt *>(a.src) + a.src_row0 * (int64_t)ld + e0;
    const Off dq = (Off)((int64_t)ROWS * (R / r) * S * ld);
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
        const int unit = tid + u * NT;
        const int e = unit & (EC - 1), b = unit >> P::LEC;
        const bool live = e < ecount;
        const int k0 = (int)j + b * S;
        const Off o0 = (Off)((int64_t)ROWS * k0 * ld + e);
#pragma unroll
        for (int q = 0; q < r; ++q) {
            const int k = k0 + q * (R / r) * S;
            const Off o = o0 + (Off)q * dq;
            cx<T> v;
            if constexpr (SRC == SRC_CPLX) {
                v = (live && k < nv) ? base[o] : c_zero<T>();
            } else if constexpr (SRC == SRC_REAL32) {
                const float x0 = (live && 2 * k < nv) ? base[o] : 0.0f;
                const float x1 = (live && 2 * k + 1 < nv) ? base[o + (Off)ld] : 0.0f;
                v = c_from_f<T>(x0, x1);
            } else {
                const double x0 = (live && 2 * k < nv) ? base[o] : 0.0;
                const double x1 = (live && 2 * k + 1 < nv) ? base[o + (Off)ld] : 0.0;
                v = c_from_d<T>(x0, x1);
            }
            x[u * r + q] = a.src_neg ? c_neg(v) : v;
        }
    }
}

template <class T, int LOGR, int EC, int SRC>
__device__ __forceinline__ void fft_gather_any(const FftArgs &a, cx<T> *x, int64_t j, int e0, int ecount)
{
    if (a.src_off32) fft_gather<T, LOGR, EC, SRC, true>(a, x, j, e0, ecount);
    else fft_gather<T, LOGR, EC, SRC, false>(a, x, j, e0, ecount);
}

// One in-CTA stage S.  Stage 0 takes its points from `pre` (loaded from
// global memory by fft_gather before the CTA filled its twiddle tables, so
// that both latencies overlap) and applies the inter-pass twiddles of spt;
// later stages read the previous stage's output from sm.
template <class T, int LOGR, int EC, int S, bool INV>
__device__ __forceinline__ void fft_stage(const FftArgs &a, cx<T> *sm, const cx<T> *stw, const cx<T> *spt,
                                          int e0, int ecount, int64_t base_out, const cx<T> *pre)
{
    using P = FftPlan<T, LOGR, EC>;
    constexpr int R = P::R, NT = P::NT;
    constexpr int LR = (S == 0) ? P::FIRST : 3;
    constexpr int r = 1 << LR;
    constexpr int LNS = (S == 0) ? 0 : P::FIRST + 3 * (S - 1);
    constexpr int Ns = 1 << LNS;
    constexpr int UPT = P::EPT / r;
    constexpr bool FIRST = (S == 0), LAST = (S == P::NSTAGE - 1);
    const int tid = threadIdx.x;
    cx<T> v[UPT][r];
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
        const int unit = tid + u * NT;
        const int e = unit & (EC - 1), b = unit >> P::LEC;
#pragma unroll
        for (int q = 0; q < r; ++q) {
            const int rho = b + q * (R / r);
            if constexpr (FIRST) {
                cx<T> x = pre[u * r + q];
                if (a.Ns > 1) x = c_mul(x, spt[rho]);
                v[u][q] = x;
            } else {
                v[u][q] = sm[rho * EC + e];
            }
        }
    }
    if (!FIRST) __syncthreads();  // every read of sm done before the in-place writes
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
        const int b = (tid + u * NT) >> P::LEC;
        if constexpr (Ns > 1) {
            const int bm = b & (Ns - 1);
#pragma unroll
            for (int q = 1; q < r; ++q) v[u][q] = c_mul(v[u][q], stw[(bm * q) << (LOGR - LNS - LR)]);
        }
        dft_r<T, INV, LR, LAST>(v[u]);
    }
    // Output point q of unit u goes to row k = k0 + q Ns a.Ns.  Complex rows
    // sit at k ld + e; the real rows 2k + h (kept in the window [lo, hi)) at
    // (row0 - lo + 2k + h) ld + e, offsets relative to the CTA's entry e0.
    auto store_global = [&](auto dst_tag, auto off_tag) {
        constexpr int DST = decltype(dst_tag)::value;
        constexpr bool OFF32 = decltype(off_tag)::value;
        using Off = fft_off_t<OFF32>;
        const int ld = a.dst_ld;
        const int64_t kst = (int64_t)Ns * a.Ns;
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
            const int unit = tid + u * NT;
            const int e = unit & (EC - 1), b = unit >> P::LEC;
            if (e >= ecount) continue;
            const int ob = ((b >> LNS) << (LNS + LR)) + (b & (Ns - 1));
            const int64_t k0 = base_out + (int64_t)ob * a.Ns;
            if constexpr (DST == DST_CPLX) {
                cx<T> *d = reinterpret_cast<cx<T> *>(a.dst) + e0;
                const Off o0 = (Off)(k0 * ld + e), dq = (Off)(kst * ld);
#pragma unroll
                for (int q = 0; q < r; ++q) {
                    cx<T> y = v[u][q];
                    if (a.dst_scaled) y = scale_out(a, y);
                    d[o0 + (Off)q * dq] = y;
                    if constexpr (__is_same(T, dd))
                        if (a.dst2)
                            (reinterpret_cast<cx<float> *>(a.dst2) + e0)[o0 + (Off)q * dq] = {y.re.hi, y.im.hi};
                }
            } else {
                const int lo = (int)a.dst_lo, hi = (int)a.dst_hi;
                const Off o0 = (Off)((a.dst_row0 - a.dst_lo + 2 * k0) * ld + e), dq = (Off)(2 * kst * ld);
                const bool eye_e = a.dst_eye_d > 0 && (e0 + e) % (a.dst_eye_d + 1) == 0;
#pragma unroll
                for (int q = 0; q < r; ++q) {
                    const cx<T> y = scale_out(a, v[u][q]);
                    const T vals[2] = {y.re, y.im};
                    const int r0 = (int)(k0 + q * kst) * 2;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int rr = r0 + h;
                        if (rr < lo || rr >= hi) continue;
                        T z = vals[h];
                        if (eye_e && rr == 0) z = Ar<T>::add(z, Ar<T>::one());
                        const Off o = o0 + (Off)q * dq + (Off)(h * ld);
                        if constexpr (DST == DST_REAL32) {
                            (reinterpret_cast<float *>(a.dst) + e0)[o] = Ar<T>::to_f(z);
                        } else {
                            const double xz = Ar<T>::to_d(z);
                            double *pz = reinterpret_cast<double *>(a.dst) + e0 + o;
                            if constexpr (DST == DST_REAL64_ADD) *pz += xz;
                            else if constexpr (DST == DST_REAL64_BASE32)
                                *pz = f32_to_f64((reinterpret_cast<const float *>(a.dst_base) + e0)[o]) + xz;
                            else *pz = xz;
                        }
                    }
                }
            }
        }
    };
    auto store_mode = [&](auto off_tag) {
        if (a.dst_mode == DST_CPLX) store_global(std::integral_constant<int, DST_CPLX>{}, off_tag);
        else if (a.dst_mode == DST_REAL64) store_global(std::integral_constant<int, DST_REAL64>{}, off_tag);
        else if (a.dst_mode == DST_REAL32) store_global(std::integral_constant<int, DST_REAL32>{}, off_tag);
        else if (a.dst_mode == DST_REAL64_BASE32)
            store_global(std::integral_constant<int, DST_REAL64_BASE32>{}, off_tag);
        else store_global(std::integral_constant<int, DST_REAL64_ADD>{}, off_tag);
    };
    if constexpr (LAST) {
        if (a.dst_off32) store_mode(std::true_type{});
        else store_mode(std::false_type{});
    } else {
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
            const int unit = tid + u * NT;
            const int e = unit & (EC - 1), b = unit >> P::LEC;
            const int ob = ((b >> LNS) << (LNS + LR)) + (b & (Ns - 1));
#pragma unroll
            for (int q = 0; q < r; ++q) sm[(ob + q * Ns) * EC + e] = v[u][q];
        }
        __syncthreads();
    }
}

template <class T, int LOGR, int EC, bool INV>
__device__ __forceinline__ void fft_pass_body(const FftArgs &a, int64_t j, int e0)
{
    using P = FftPlan<T, LOGR, EC>;
    constexpr int R = P::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);  // [R][EC]
    cx<T> *stw = sm + R * EC;                         // [R]  W_R^t
    cx<T> *spt = stw + R;                             // [R]  inter-pass twiddles
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw);
    const int tid = threadIdx.x;
    const int ecount = min(EC, a.E - e0);
    const int64_t jm = j & (a.Ns - 1);
    // first-stage global loads before the twiddle tables are filled (both latencies overlap)
    cx<T> pre[P::EPT];
    if (a.src_mode == SRC_CPLX) fft_gather_any<T, LOGR, EC, SRC_CPLX>(a, pre, j, e0, ecount);
    else if (a.src_mode == SRC_REAL32) fft_gather_any<T, LOGR, EC, SRC_REAL32>(a, pre, j, e0, ecount);
    else fft_gather_any<T, LOGR, EC, SRC_REAL64>(a, pre, j, e0, ecount);
    if constexpr (P::NSTAGE > 1)
        for (int t = tid; t < R; t += P::NT) {
            cx<T> w = tw[(int64_t)t << (a.tw_log - LOGR)];
            stw[t] = INV ? c_conj(w) : w;
        }
    if (a.Ns > 1) {
        const int sh = a.tw_log - (a.logNs + LOGR);
        for (int t = tid; t < R; t += P::NT) {
            cx<T> w = tw[(jm * t) << sh];
            spt[t] = INV ? c_conj(w) : w;
        }
    }
    __syncthreads();
    const int64_t base_out = (j >> a.logNs << (a.logNs + LOGR)) + jm;
    fft_stage<T, LOGR, EC, 0, INV>(a, sm, stw, spt, e0, ecount, base_out, pre);
    if constexpr (P::NSTAGE > 1) fft_stage<T, LOGR, EC, 1, INV>(a, sm, stw, spt, e0, ecount, base_out, nullptr);
    if constexpr (P::NSTAGE > 2) fft_stage<T, LOGR, EC, 2, INV>(a, sm, stw, spt, e0, ecount, base_out, nullptr);
    if constexpr (P::NSTAGE > 3) fft_stage<T, LOGR, EC, 3, INV>(a, sm, stw, spt, e0, ecount, base_out, nullptr);
}

// One Stockham pass of radix R = 2^LOGR over EC entries per CTA.
// (Only the thread count is bounded: with an explicit minimum of CTAs per SM
// ptxas chose more registers for the FP32 passes of radix <= 2^8 and fewer
// CTAs fitted; d = 64, N = 2^18 FP32 FFT time went from 110 to 124 ms.)
template <class T, int LOGR, int EC>
__global__ void __launch_bounds__(FftPlan<T, LOGR, EC>::NT) fft_pass_kernel(FftArgs a)
{
    // entry chunk fastest: CTAs launched together cover whole rows
    if (a.dir > 0) fft_pass_body<T, LOGR, EC, true>(a, blockIdx.y, blockIdx.x * EC);
    else fft_pass_body<T, LOGR, EC, false>(a, blockIdx.y, blockIdx.x * EC);
}

// The same pass with a minimum of resident CTAs per SM (MRC_FFT32_MINB x 512
// threads; 0 at build time = off), used for the FP32 passes of at most 8
// points per thread.  With 4 (2048 threads: 32 registers, a 40-byte spill)
// the FP32 passes are latency-bound at full occupancy instead of 75 %: FP32
// FFT 89.5 -> 83.5 ms at d = 64, N = 2^18.  Not for the double-float passes:
// there an explicit minimum, even of 1, raised ptxas's register choice from
// 64 to 96-109.
#ifndef MRC_FFT32_MINB
#define MRC_FFT32_MINB 4
#endif
template <class T, int LOGR, int EC>
__global__ void __launch_bounds__(FftPlan<T, LOGR, EC>::NT,
                                  MRC_FFT32_MINB > 0 ? (MRC_FFT32_MINB * 512) / FftPlan<T, LOGR, EC>::NT : 1)
    fft_pass_kernel_mb(FftArgs a)
{
    if (a.dir > 0) fft_pass_body<T, LOGR, EC, true>(a, blockIdx.y, blockIdx.x * EC);
    else fft_pass_body<T, LOGR, EC, false>(a, blockIdx.y, blockIdx.x * EC);
}

// ---------------------------------------------------------------------------
// Segmented launches: one launch covers several independent transforms (or
// products) of one shape class -- the models of a batch at one Newton level.
// The segments' argument blocks travel in the kernel's parameter space (a
// __grid_constant__ block of at most MRC_SEG_MAX segments, read through the
// constant cache like a single launch's arguments); CTA b runs CTA
// b - first[s] of segment s = max{s : first[s] <= b}, in the order of the
// single-segment launch.
template <class T, int LOGR, int EC>
__device__ __forceinline__ void fft_seg_run(const SegParams<FftArgs> &P)
{
    const int s = seg_find(P, blockIdx.x);
    const FftArgs &a = P.a[s];
    const unsigned loc = blockIdx.x - P.first[s];
    const unsigned nchunk = (unsigned)((a.E + EC - 1) / EC);
    const unsigned j = loc / nchunk;
    const int e0 = (int)(loc - j * nchunk) * EC;
    if (a.dir > 0) fft_pass_body<T, LOGR, EC, true>(a, j, e0);
    else fft_pass_body<T, LOGR, EC, false>(a, j, e0);
}

template <class T, int LOGR, int EC>
__global__ void __launch_bounds__(FftPlan<T, LOGR, EC>::NT) fft_seg_kernel(const __grid_constant__ SegParams<FftArgs> P)
{
    fft_seg_run<T, LOGR, EC>(P);
}

template <class T, int LOGR, int EC>
__global__ void __launch_bounds__(FftPlan<T, LOGR, EC>::NT,
                                  MRC_FFT32_MINB > 0 ? (MRC_FFT32_MINB * 512) / FftPlan<T, LOGR, EC>::NT : 1)
    fft_seg_kernel_mb(const __grid_constant__ SegParams<FftArgs> P)
{
    fft_seg_run<T, LOGR, EC>(P);
}

// ---------------------------------------------------------------------------
// Frequency-pair matrix product.  For the real sequences X (r x m entries)
// and Y (m x c) with packed spectra ZX, ZY of length M (L = 2M):
//   Xh(f) = 1/2 [Z(f) + conj Z(M-f)] - (i/2) W_L^f [Z(f) - conj Z(M-f)],
// Ch(f) = Xh(f) Yh(f) for f and its partner g = M - f, then the packed
// spectrum of C = X (*) Y (cyclic, length L):
//   ZC(f) = 1/2 [Ch(f) + conj Ch(g)] + (i/2) W_L^{-f} [Ch(f) - conj Ch(g)].
// One CTA: one pair p (f = p, g = M - p), an output tile BM x BN, both
// frequencies accumulated together.
template <class T>
__device__ __forceinline__ cx<T> split_real(cx<T> za, cx<T> zb, cx<T> w)
{
    // 1/2 (za + conj zb) + w * (-(i/2)) (za - conj zb)
    cx<T> s = {Ar<T>::add(za.re, zb.re), Ar<T>::sub(za.im, zb.im)};
    cx<T> dlt = {Ar<T>::sub(za.re, zb.re), Ar<T>::add(za.im, zb.im)};
    cx<T> o = {dlt.im, Ar<T>::neg(dlt.re)};  // -i * dlt
    return c_scal(c_add(s, c_mul(w, o)), 0.5);
}

template <class T>
__device__ __forceinline__ cx<T> merge_real(cx<T> cf, cx<T> cg, cx<T> wconj)
{
    // 1/2 (cf + conj cg) + (i/2) wconj (cf - conj cg)
    cx<T> s = {Ar<T>::add(cf.re, cg.re), Ar<T>::sub(cf.im, cg.im)};
    cx<T> dlt = {Ar<T>::sub(cf.re, cg.re), Ar<T>::add(cf.im, cg.im)};
    return c_scal(c_add(s, c_mul_i(c_mul(wconj, dlt))), 0.5);
}

template <class T, int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void pairmul_body(const PairArgs &a, int64_t p, int tile)
{
    constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
    __shared__ cx<T> Xf[BK][BM + 1], Xg[BK][BM + 1];
    __shared__ cx<T> Yf[BK][BN], Yg[BK][BN];
    const cx<T> *ZX = reinterpret_cast<const cx<T> *>(a.zx);
    const cx<T> *ZY = reinterpret_cast<const cx<T> *>(a.zy);
    cx<T> *ZC = reinterpret_cast<cx<T> *>(a.zc);
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw);

    const int64_t M = a.M;
    const int64_t f = p;
    const int64_t gL = M - p;        // partner frequency of the length-L spectrum
    const int64_t gZ = gL & (M - 1);  // its packed index
    const int ntile_c = (a.c + BN - 1) / BN;
    const int i0 = (tile / ntile_c) * BM;
    const int j0 = (tile % ntile_c) * BN;
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    // W_L^f with L = 2M; W_L^{gL} = -conj(W_L^f)
    const cx<T> wf = tw[f << (a.tw_log - a.logM - 1)];
    const cx<T> wg = c_neg(c_conj(wf));

    const int64_t EX = (int64_t)a.r * a.m, EY = (int64_t)a.m * a.c, EC = (int64_t)a.r * a.c;
    const cx<T> *xf = ZX + f * EX, *xg = ZX + gZ * EX;
    const cx<T> *yf = ZY + f * EY, *yg = ZY + gZ * EY;

    cx<T> accf[TM][TN], accg[TM][TN];
#pragma unroll
    for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TN; ++v) { accf[u][v] = c_zero<T>(); accg[u][v] = c_zero<T>(); }

    for (int k0 = 0; k0 < a.m; k0 += BK) {
        for (int idx = threadIdx.x; idx < BM * BK; idx += NT) {
            int ii = idx / BK, kk = idx - ii * BK;
            int i = i0 + ii, k = k0 + kk;
            cx<T> vf = c_zero<T>(), vg = c_zero<T>();
            if (i < a.r && k < a.m) {
                cx<T> za = xf[(int64_t)i * a.m + k], zb = xg[(int64_t)i * a.m + k];
                vf = split_real(za, zb, wf);
                vg = split_real(zb, za, wg);
            }
            Xf[kk][ii] = vf;
            Xg[kk][ii] = vg;
        }
        for (int idx = threadIdx.x; idx < BK * BN; idx += NT) {
            int kk = idx / BN, jj = idx - kk * BN;
            int k = k0 + kk, jx = j0 + jj;
            cx<T> vf = c_zero<T>(), vg = c_zero<T>();
            if (k < a.m && jx < a.c) {
                cx<T> za = yf[(int64_t)k * a.c + jx], zb = yg[(int64_t)k * a.c + jx];
                vf = split_real(za, zb, wf);
                vg = split_real(zb, za, wg);
            }
            Yf[kk][jj] = vf;
            Yg[kk][jj] = vg;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            cx<T> xa[TM], xb[TM], ya[TN], yb[TN];
#pragma unroll
            for (int u = 0; u < TM; ++u) { xa[u] = Xf[kk][ty + u * NTY]; xb[u] = Xg[kk][ty + u * NTY]; }
#pragma unroll
            for (int v = 0; v < TN; ++v) { ya[v] = Yf[kk][tx + v * NTX]; yb[v] = Yg[kk][tx + v * NTX]; }
#pragma unroll
            for (int u = 0; u < TM; ++u)
#pragma unroll
                for (int v = 0; v < TN; ++v) {
                    c_mac(accf[u][v], xa[u], ya[v]);
                    c_mac(accg[u][v], xb[u], yb[v]);
                }
        }
        __syncthreads();
    }

    const cx<T> wfc = c_conj(wf), wgc = c_conj(wg);
    const bool two = (gZ != f);
#pragma unroll
    for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TN; ++v) {
            int i = i0 + ty + u * NTY, jx = j0 + tx + v * NTX;
            if (i >= a.r || jx >= a.c) continue;
            int64_t e = (int64_t)i * a.c + jx;
            ZC[f * EC + e] = merge_real(accf[u][v], accg[u][v], wfc);
            if (two) ZC[gZ * EC + e] = merge_real(accg[u][v], accf[u][v], wgc);
        }
}

template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) pairmul_kernel(PairArgs a)
{
    pairmul_body<T, BM, BN, BK, TM, TN>(a, blockIdx.x, blockIdx.y);
}

// segmented: CTA (pair p, tile) of segment s at local index tile * npairs + p
template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) pairmul_seg_kernel(const __grid_constant__ SegParams<PairArgs> P)
{
    const int s = seg_find(P, blockIdx.x);
    const PairArgs &a = P.a[s];
    const unsigned loc = blockIdx.x - P.first[s], np = (unsigned)a.npairs;
    pairmul_body<T, BM, BN, BK, TM, TN>(a, loc % np, (int)(loc / np));
}

// The same product with the two frequencies of the pair on two halves of
// the CTA (2 x NTX x NTY threads): thread group fq in {0: f, 1: g} keeps only
// its own TM x TN accumulators, which halves the registers per thread and
// lets two CTAs share an SM.  Each thread's TM rows and TN columns are
// contiguous in shared memory; the Y tile stores column tx * TN + v at
// (v / 2) * 2 NTX + 2 tx + v % 2, so that the 16-byte loads of the FP32
// kernel fall on consecutive addresses across tx.  The k tiles are double
// buffered: the next tile's spectra are loaded into registers before the
// current tile is multiplied and split into the other buffer after it.
// After the k loop the g half hands C(g) to the f half through shared memory
// (the tiles' space), which merges both into the packed output spectrum.
template <int NTX, int TN>
__device__ __forceinline__ int pm2_ycol(int jj)
{
    const int tx = jj / TN, v = jj - (jj / TN) * TN;
    return (v >> 1) * (2 * NTX) + 2 * tx + (v & 1);
}

template <class T, int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void pairmul2_body(const PairArgs &a, int64_t p, int tile)
{
    constexpr int NTX = BN / TN, NTY = BM / TM, NTF = NTX * NTY, NT = 2 * NTF;
    constexpr int XLD = BM + (sizeof(cx<T>) == 8 ? 2 : 1), YLD = BN + (sizeof(cx<T>) == 8 ? 2 : 1);
    constexpr int TILE = 2 * BK * (XLD + YLD);  // complex values: X and Y tiles of both frequencies
    constexpr int XCH = BM * YLD;               // the C(g) exchange
    constexpr int XPT = (BM * BK + NT - 1) / NT, YPT = (BK * BN + NT - 1) / NT;  // fill items per thread
    static_assert(TN % 2 == 0, "column pairs");
    __shared__ __align__(16) cx<T> sbuf[2 * TILE > XCH ? 2 * TILE : XCH];  // two tile buffers
    const cx<T> *ZX = reinterpret_cast<const cx<T> *>(a.zx);
    const cx<T> *ZY = reinterpret_cast<const cx<T> *>(a.zy);
    cx<T> *ZC = reinterpret_cast<cx<T> *>(a.zc);
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw);

    const int64_t M = a.M;
    const int64_t f = p, gL = M - p, gZ = gL & (M - 1);
    const int ntile_c = (a.c + BN - 1) / BN;
    const int i0 = (tile / ntile_c) * BM, j0 = (tile % ntile_c) * BN;
    const int fq = threadIdx.x / NTF, lt = threadIdx.x - fq * NTF;
    const int tx = lt % NTX, ty = lt / NTX;
    const cx<T> wf = tw[f << (a.tw_log - a.logM - 1)];
    const cx<T> wg = c_neg(c_conj(wf));
    const int64_t EX = (int64_t)a.r * a.m, EY = (int64_t)a.m * a.c, EC = (int64_t)a.r * a.c;
    const cx<T> *xf = ZX + f * EX, *xg = ZX + gZ * EX;
    const cx<T> *yf = ZY + f * EY, *yg = ZY + gZ * EY;

    // raw spectra of the next k tile, held in registers while the current one is multiplied
    cx<T> rx[XPT][2], ry[YPT][2];
    auto load = [&](int k0) {
#pragma unroll
        for (int n = 0; n < XPT; ++n) {
            const int idx = threadIdx.x + n * NT;
            const int ii = idx / BK, kk = idx - (idx / BK) * BK;
            const int i = i0 + ii, k = k0 + kk;
            const bool ok = idx < BM * BK && i < a.r && k < a.m;
            rx[n][0] = ok ? xf[(int64_t)i * a.m + k] : c_zero<T>();
            rx[n][1] = ok ? xg[(int64_t)i * a.m + k] : c_zero<T>();
        }
#pragma unroll
        for (int n = 0; n < YPT; ++n) {
            const int idx = threadIdx.x + n * NT;
            const int kk = idx / BN, jj = idx - (idx / BN) * BN;
            const int k = k0 + kk, jx = j0 + jj;
            const bool ok = idx < BK * BN && k < a.m && jx < a.c;
            ry[n][0] = ok ? yf[(int64_t)k * a.c + jx] : c_zero<T>();
            ry[n][1] = ok ? yg[(int64_t)k * a.c + jx] : c_zero<T>();
        }
    };
    auto store = [&](cx<T> *buf) {
        cx<T> *Xs = buf, *Ys = buf + 2 * BK * XLD;
#pragma unroll
        for (int n = 0; n < XPT; ++n) {
            const int idx = threadIdx.x + n * NT;
            if (idx >= BM * BK) break;
            const int ii = idx / BK, kk = idx - (idx / BK) * BK;
            Xs[kk * XLD + ii] = split_real(rx[n][0], rx[n][1], wf);
            Xs[(BK + kk) * XLD + ii] = split_real(rx[n][1], rx[n][0], wg);
        }
#pragma unroll
        for (int n = 0; n < YPT; ++n) {
            const int idx = threadIdx.x + n * NT;
            if (idx >= BK * BN) break;
            const int kk = idx / BN, jj = idx - (idx / BN) * BN;
            const int pc = pm2_ycol<NTX, TN>(jj);
            Ys[kk * YLD + pc] = split_real(ry[n][0], ry[n][1], wf);
            Ys[(BK + kk) * YLD + pc] = split_real(ry[n][1], ry[n][0], wg);
        }
    };

    cx<T> acc[TM][TN];
#pragma unroll
    for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TN; ++v) acc[u][v] = c_zero<T>();

    load(0);
    store(sbuf);
    __syncthreads();
    int cur = 0;
    for (int k0 = 0; k0 < a.m; k0 += BK) {
        const bool more = k0 + BK < a.m;
        if (more) load(k0 + BK);  // in flight while this tile is multiplied
        const cx<T> *Xs = sbuf + cur * TILE, *Ys = Xs + 2 * BK * XLD;
        const cx<T> *xb = Xs + fq * BK * XLD + ty * TM;
        const cx<T> *yb = Ys + fq * BK * YLD + 2 * tx;
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            cx<T> xa[TM], ya[TN];
#pragma unroll
            for (int u = 0; u < TM; ++u) xa[u] = xb[kk * XLD + u];
#pragma unroll
            for (int h = 0; h < TN / 2; ++h) {
                ya[2 * h] = yb[kk * YLD + h * 2 * NTX];
                ya[2 * h + 1] = yb[kk * YLD + h * 2 * NTX + 1];
            }
#pragma unroll
            for (int u = 0; u < TM; ++u)
#pragma unroll
                for (int v = 0; v < TN; ++v) c_mac(acc[u][v], xa[u], ya[v]);
        }
        if (more) store(sbuf + (cur ^ 1) * TILE);  // the other buffer: last read two tiles ago
        __syncthreads();
        cur ^= 1;
    }

    // C(g) to shared memory, then the f half merges both
    if (fq == 1) {
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
            for (int v = 0; v < TN; ++v) sbuf[(ty * TM + u) * YLD + tx * TN + v] = acc[u][v];
    }
    __syncthreads();
    if (fq == 0) {
        const cx<T> wfc = c_conj(wf), wgc = c_conj(wg);
        const bool two = (gZ != f);
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
            for (int v = 0; v < TN; ++v) {
                const int i = i0 + ty * TM + u, jx = j0 + tx * TN + v;
                if (i >= a.r || jx >= a.c) continue;
                const cx<T> cg = sbuf[(ty * TM + u) * YLD + tx * TN + v];
                const int64_t e = (int64_t)i * a.c + jx;
                ZC[f * EC + e] = merge_real(acc[u][v], cg, wfc);
                if (two) ZC[gZ * EC + e] = merge_real(cg, acc[u][v], wgc);
            }
    }
}

template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(2 * (BM / TM) * (BN / TN), 2) pairmul2_kernel(PairArgs a)
{
    pairmul2_body<T, BM, BN, BK, TM, TN>(a, blockIdx.x, blockIdx.y);
}

template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(2 * (BM / TM) * (BN / TN), 2)
    pairmul2_seg_kernel(const __grid_constant__ SegParams<PairArgs> P)
{
    const int s = seg_find(P, blockIdx.x);
    const PairArgs &a = P.a[s];
    const unsigned loc = blockIdx.x - P.first[s], np = (unsigned)a.npairs;
    pairmul2_body<T, BM, BN, BK, TM, TN>(a, loc % np, (int)(loc / np));
}

// Frequency-pair product with a diagonal right factor:
//   Ch(f)_{ij} = Xh(f)_{ij} * Yh(f)_j   (X: [E = r*c], Y: [c]),
// the per-entry scalar convolutions P_ij = psi_ij * h_j of Eq. (transition-discrete).
template <class T>
__global__ void __launch_bounds__(256) pairdiag_kernel(PairArgs a)
{
    const cx<T> *ZX = reinterpret_cast<const cx<T> *>(a.zx);
    const cx<T> *ZY = reinterpret_cast<const cx<T> *>(a.zy);
    cx<T> *ZC = reinterpret_cast<cx<T> *>(a.zc);
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw);
    const int64_t E = (int64_t)a.r * a.c;
    const int64_t total = a.npairs * E;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / E, e = t - p * E;
        const int jx = (int)(e % a.c);
        const int64_t f = p, gZ = (a.M - p) & (a.M - 1);
        const cx<T> wf = tw[f << (a.tw_log - a.logM - 1)];
        const cx<T> wg = c_neg(c_conj(wf));
        cx<T> za = ZX[f * E + e], zb = ZX[gZ * E + e];
        cx<T> ya = ZY[f * a.c + jx], yb = ZY[gZ * a.c + jx];
        cx<T> cf = c_mul(split_real(za, zb, wf), split_real(ya, yb, wf));
        cx<T> cg = c_mul(split_real(zb, za, wg), split_real(yb, ya, wg));
        ZC[f * E + e] = merge_real(cf, cg, c_conj(wf));
        if (gZ != f) ZC[gZ * E + e] = merge_real(cg, cf, c_conj(wg));
    }
}

// Twiddle table: tw[t] = exp(-2 pi i t / 2^log) from FP64 sincospi (called,
// not re-derived), rounded to the working precision.
template <class T>
__global__ void twiddle_kernel(cx<T> *tw, int log)
{
    const int64_t n = (int64_t)1 << log;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)t / (double)n, &s, &c);
        tw[t] = c_from_d<T>(c, s);
    }
}

// ---------------------------------------------------------------------------
// Launch table of the FFT pass instantiations: entry [ec_index][logR], where
// ec_index 0 is the default entries per CTA (MRC_F32_EC for 8-byte complex
// values, MRC_DD_EC for 16-byte ones) and 1 is 4 entries per CTA.
using FftKernel = void (*)(FftArgs);
struct FftEntry {
    FftKernel fn;
    int nt;
};
using FftSegKernel = void (*)(SegParams<FftArgs>);
struct FftSegEntry {
    FftSegKernel fn;
    int nt;
};

template <class T, int L, int EC>
constexpr FftKernel fft_pass_or_mb()
{
    if constexpr (MRC_FFT32_MINB > 0 && sizeof(cx<T>) == 8 && FftPlan<T, L, EC>::EPT <= 8 &&
                  FftPlan<T, L, EC>::NT <= MRC_FFT32_MINB * 512)
        return fft_pass_kernel_mb<T, L, EC>;
    else return fft_pass_kernel<T, L, EC>;
}

template <class T, int L, int EC>
constexpr FftSegKernel fft_seg_or_mb()
{
    if constexpr (MRC_FFT32_MINB > 0 && sizeof(cx<T>) == 8 && FftPlan<T, L, EC>::EPT <= 8 &&
                  FftPlan<T, L, EC>::NT <= MRC_FFT32_MINB * 512)
        return fft_seg_kernel_mb<T, L, EC>;
    else return fft_seg_kernel<T, L, EC>;
}

// t: the single-transform passes; ts: the segmented ones (default entries per CTA)
template <class T, int OFF, int... L>
void fft_fill_shifted(FftEntry (*t)[11], FftSegEntry *ts, std::integer_sequence<int, L...>)
{
    constexpr int ECD = fft_default_ec<T>();
    ((t[0][OFF + L] = FftEntry{fft_pass_or_mb<T, OFF + L, ECD>(), FftPlan<T, OFF + L, ECD>::NT}), ...);
    ((t[1][OFF + L] = FftEntry{fft_pass_kernel<T, OFF + L, 4>, FftPlan<T, OFF + L, 4>::NT}), ...);
    ((ts[OFF + L] = FftSegEntry{fft_seg_or_mb<T, OFF + L, ECD>(), FftPlan<T, OFF + L, ECD>::NT}), ...);
}
