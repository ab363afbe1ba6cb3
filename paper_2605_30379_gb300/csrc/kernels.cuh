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
#include "arith.cuh"
#include "mrc_internal.h"

// ---------------------------------------------------------------------------
// FFT pass: one radix-R Stockham step of a length-M transform (R = 2^logR,
// Ns = product of the earlier radices).  CTA (j, chunk) loads the R elements
// j + r*M/R of `ec` consecutive entries, applies the inter-pass twiddles
// W_{Ns R}^{(j mod Ns) r}, runs the length-R DFT in shared memory (radix-2,
// bit-reversed load), and writes element f to (j/Ns)*Ns*R + (j mod Ns) + f*Ns.
// After the last pass the output is in natural frequency order.
template <class T>
__device__ __forceinline__ cx<T> fft_load(const FftArgs &a, int64_t k, int e)
{
    if (a.src_mode == SRC_CPLX) {
        if (k >= a.src_nvalid) return c_zero<T>();
        const cx<T> *s = reinterpret_cast<const cx<T> *>(a.src);
        cx<T> v = s[(a.src_row0 + k) * (int64_t)a.src_ld + e];
        return a.src_neg ? c_neg(v) : v;
    }
    // SRC_REAL64: packed pair of real rows 2k, 2k+1
    const double *s = reinterpret_cast<const double *>(a.src);
    int64_t r0 = 2 * k, r1 = 2 * k + 1;
    double x0 = (r0 < a.src_nvalid) ? s[(a.src_row0 + r0) * (int64_t)a.src_ld + e] : 0.0;
    double x1 = (r1 < a.src_nvalid) ? s[(a.src_row0 + r1) * (int64_t)a.src_ld + e] : 0.0;
    if (a.src_neg) { x0 = -x0; x1 = -x1; }
    return c_from_d<T>(x0, x1);
}

template <class T>
__device__ __forceinline__ void fft_store(const FftArgs &a, int64_t k, int e, cx<T> v)
{
    if (a.dst_mode == DST_CPLX) {
        cx<T> *d = reinterpret_cast<cx<T> *>(a.dst);
        if (a.dst_scale != 1.0) v = c_scal(v, a.dst_scale);
        d[k * (int64_t)a.dst_ld + e] = v;
        return;
    }
    // real rows 2k (re) and 2k+1 (im), window [lo, hi)
    double *d = reinterpret_cast<double *>(a.dst);
    double vals[2] = {Ar<T>::to_d(v.re), Ar<T>::to_d(v.im)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int64_t r = 2 * k + h;
        if (r < a.dst_lo || r >= a.dst_hi) continue;
        double x = vals[h] * a.dst_scale;
        if (a.dst_eye_d > 0 && r == 0 && (e % (a.dst_eye_d + 1)) == 0) x += 1.0;
        double *p = d + (a.dst_row0 + (r - a.dst_lo)) * (int64_t)a.dst_ld + e;
        if (a.dst_mode == DST_REAL64_ADD) *p += x;
        else *p = x;
    }
}

template <class T>
__global__ void __launch_bounds__(256) fft_pass_kernel(FftArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int logR = a.logR;
    const int R = 1 << logR;
    const int ec = a.ec;
    cx<T> *s = reinterpret_cast<cx<T> *>(smem_raw);  // [R][ec]
    cx<T> *stw = s + (size_t)R * ec;                  // [R/2]  W_R^t
    cx<T> *spt = stw + (R >> 1);                      // [R]    inter-pass twiddle
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t j = blockIdx.x;
    const int e0 = blockIdx.y * ec;
    const int ecount = min(ec, a.E - e0);
    const int64_t jm = j & (a.Ns - 1);
    const bool inv = a.dir > 0;

    for (int t = tid; t < (R >> 1); t += nt) {
        cx<T> w = tw[(int64_t)t << (a.tw_log - logR)];
        stw[t] = inv ? c_conj(w) : w;
    }
    const bool has_pt = a.Ns > 1;
    if (has_pt) {
        // W_{Ns R}^{jm r} = table[(jm r) << (tw_log - log2(Ns R))]
        const int sh = a.tw_log - (a.logNs + logR);
        for (int r = tid; r < R; r += nt) {
            cx<T> w = tw[(jm * r) << sh];
            spt[r] = inv ? c_conj(w) : w;
        }
    }
    __syncthreads();

    const int64_t stride_in = a.M >> logR;
    for (int idx = tid; idx < R * ec; idx += nt) {
        int r = idx / ec, e = idx - r * ec;
        cx<T> v = c_zero<T>();
        if (e < ecount) {
            v = fft_load<T>(a, j + (int64_t)r * stride_in, e0 + e);
            if (has_pt) v = c_mul(v, spt[r]);
        }
        int rb = logR ? (int)(__brev((unsigned)r) >> (32 - logR)) : 0;
        s[rb * ec + e] = v;
    }
    __syncthreads();

    for (int lh = 0; lh < logR; ++lh) {
        const int h = 1 << lh;
        const int tsh = logR - 1 - lh;  // W_{2h}^pos = W_R^{pos * R/(2h)}
        for (int idx = tid; idx < (R >> 1) * ec; idx += nt) {
            int b = idx / ec, e = idx - b * ec;
            int pos = b & (h - 1);
            int i0 = ((b >> lh) << (lh + 1)) + pos;
            int i1 = i0 + h;
            cx<T> w = stw[pos << tsh];
            cx<T> x0 = s[i0 * ec + e];
            cx<T> x1 = c_mul(s[i1 * ec + e], w);
            s[i0 * ec + e] = c_add(x0, x1);
            s[i1 * ec + e] = c_sub(x0, x1);
        }
        __syncthreads();
    }

    const int64_t base = (j >> a.logNs << (a.logNs + logR)) + jm;
    for (int idx = tid; idx < R * ec; idx += nt) {
        int f = idx / ec, e = idx - f * ec;
        if (e < ecount) fft_store<T>(a, base + (int64_t)f * a.Ns, e0 + e, s[f * ec + e]);
    }
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
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) pairmul_kernel(PairArgs a)
{
    constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
    __shared__ cx<T> Xf[BK][BM + 1], Xg[BK][BM + 1];
    __shared__ cx<T> Yf[BK][BN], Yg[BK][BN];
    const cx<T> *ZX = reinterpret_cast<const cx<T> *>(a.zx);
    const cx<T> *ZY = reinterpret_cast<const cx<T> *>(a.zy);
    cx<T> *ZC = reinterpret_cast<cx<T> *>(a.zc);
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw);

    const int64_t p = blockIdx.x;
    const int64_t M = a.M;
    const int64_t f = p;
    const int64_t gL = M - p;        // partner frequency of the length-L spectrum
    const int64_t gZ = gL & (M - 1);  // its packed index
    const int ntile_c = (a.c + BN - 1) / BN;
    const int i0 = (blockIdx.y / ntile_c) * BM;
    const int j0 = (blockIdx.y % ntile_c) * BN;
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
