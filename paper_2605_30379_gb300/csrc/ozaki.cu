// ozaki.cu -- double-float per-frequency complex matrix products on the
// tensor cores (the residual product of the mixed path, d in [32, 64]).
//
// The frequency-pair product of kernels.cuh computes, at each frequency,
// C = X Y with X, Y complex d x d in double-float.  Here the two real
// products that make up C,
//     [C_r | C_i] = [X_r | X_i] . [[Y_r, Y_i], [-Y_i, Y_r]],
// run as exact integer products on BF16 tensor cores:
//   * every row i of [X_r | X_i] is scaled by 2^-sigma_i and every column j of
//     Y by 2^-tau_j (powers of two with all scaled magnitudes <= 1/2);
//   * each scaled value v = hi + lo is written as six balanced base-256 digits
//     v ~ sum_s q_s 2^(8s-48), |q_s| <= 128, each exactly a BF16 integer
//     (the rounding of the last digit is below 2^-49);
//   * for every digit pair (s, t) with s + t >= 5 the product of the digit
//     matrices is formed with mma.sync (BF16 in, FP32 accumulate).  Products
//     are <= 2^14, a 128-term dot product <= 2^21 and a weight group
//     g = s + t holds at most 6 of them, so each group sum is an exact integer
//     below 2^24 in FP32;
//   * the six group sums are combined exactly in int64 with shifts 8(g-5),
//     converted to double-float and scaled back by 2^(sigma_i + tau_j - 56).
// Dropped pairs (s + t < 5) weigh below 2^-48 of the row/column scale.  This
// is the error-free splitting idea of Ozaki et al. (2012) specialised to
// this product; the paper's error model (Proposition 2.1) only needs the
// product error to be a small multiple of the unit roundoff of the result
// precision times |X||Y|.
//
// One CTA owns one frequency pair {f, M-f} (the real-FFT split and merge of
// kernels.cuh), computes C(f) (stored unmerged in its output rows), then
// C(M-f), then merges both into the packed output spectrum.
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace {

constexpr int OZ_D = 64;       // padded matrix size
constexpr int OZ_S = 6;        // digits per value
constexpr int OZ_LD = 72;      // shared-memory row length (bf16), padded against bank conflicts
constexpr int OZ_GMIN = 5;     // smallest digit-pair weight group kept
constexpr int OZ_THREADS = 256;
constexpr int OZ_SLICE = OZ_D * OZ_LD;
constexpr size_t OZ_SMEM = (size_t)4 * OZ_S * OZ_SLICE * sizeof(unsigned short) + 4 * OZ_D * sizeof(int);

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Six balanced base-256 digits of v = hi + lo, |v| <= 1/2: digit s has weight
// 2^(8s-48) and |q_s| <= 128.  t = (x + C) - C with C = 1.5 * 2^k rounds x to
// the nearest multiple of 2^(k-23) (|x| <= 2^(k-1)) and x - t is exact.  lo
// joins after two digits through an exact TwoSum (y + e = rest + lo, |y| <=
// 2^-17 + 2^-26, |e| <= 2^-41); e joins after four digits, where the rest is
// <= 2^-33.  Each digit therefore stays within 128 (+ at most 1/2 before
// rounding to an integer).
__device__ __forceinline__ void digits6(float hi, float lo, float (&q)[OZ_S])
{
    float x = hi, t;
    t = __fsub_rn(__fadd_rn(x, 49152.0f), 49152.0f);            // grid 2^-8
    q[5] = t * 256.0f;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 192.0f), 192.0f);                // grid 2^-16
    q[4] = t * 65536.0f;
    x = __fsub_rn(x, t);
    const dd ye = dd_two_sum(x, lo);                            // exact: x + lo = y + e
    x = ye.hi;
    t = __fsub_rn(__fadd_rn(x, 0.75f), 0.75f);                  // grid 2^-24
    q[3] = t * 16777216.0f;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 0x1.8p-9f), 0x1.8p-9f);          // grid 2^-32
    q[2] = t * 0x1p32f;
    x = __fadd_rn(__fsub_rn(x, t), ye.lo);
    t = __fsub_rn(__fadd_rn(x, 0x1.8p-17f), 0x1.8p-17f);        // grid 2^-40
    q[1] = t * 0x1p40f;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 0x1.8p-25f), 0x1.8p-25f);        // grid 2^-48
    q[0] = t * 0x1p48f;
}

__device__ __forceinline__ unsigned short bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

// 2^e as a float for e in [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((unsigned)(e + 127) << 23); }

// multiply by 2^e with e possibly outside one float exponent's range
__device__ __forceinline__ float scale2(float x, int e)
{
    int e1 = e / 2, e2 = e - e1;
    e1 = max(-126, min(127, e1));
    e2 = max(-126, min(127, e2));
    return x * pow2f(e1) * pow2f(e2);
}

// exponent sigma with max|.| <= b < 2^(sigma - 1), i.e. scaled values <= 1/2
__device__ __forceinline__ int scale_exp(float b)
{
    if (!(b > 0x1p-120f)) return 0;  // zero (or negligible) row: all digits vanish
    int e;
    frexpf(b * (1.0f + 0x1p-20f), &e);  // b < 2^e
    return e + 1;
}

__global__ void __launch_bounds__(OZ_THREADS, 1) ozaki_pairmul_kernel(PairArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned short *Xr = reinterpret_cast<unsigned short *>(smem_raw);  // [S][64][72]
    unsigned short *Xi = Xr + OZ_S * OZ_SLICE;
    unsigned short *YrT = Xi + OZ_S * OZ_SLICE;  // transposed: [S][j][k]
    unsigned short *YiT = YrT + OZ_S * OZ_SLICE;
    unsigned *bx = reinterpret_cast<unsigned *>(YiT + OZ_S * OZ_SLICE);  // [64] row bounds (float bits)
    unsigned *by = bx + OZ_D;
    int *sig = reinterpret_cast<int *>(by + OZ_D);
    int *tau = sig + OZ_D;

    const cx<dd> *ZX = reinterpret_cast<const cx<dd> *>(a.zx);
    const cx<dd> *ZY = reinterpret_cast<const cx<dd> *>(a.zy);
    cx<dd> *ZC = reinterpret_cast<cx<dd> *>(a.zc);
    const cx<dd> *tw = reinterpret_cast<const cx<dd> *>(a.tw);
    const int d = a.r;  // square: r = m = c = d <= 64
    const int64_t E = (int64_t)d * d;
    const int64_t p = blockIdx.x, M = a.M;
    const int64_t f = p, gL = M - p, gZ = gL & (M - 1);
    const cx<dd> wf = tw[f << (a.tw_log - a.logM - 1)];
    const cx<dd> wg = c_neg(c_conj(wf));
    const int tid = threadIdx.x;

    // ---- row (X) and column (Y) magnitude bounds: |Xh(f)|, |Xh(g)| <= |Z(f)| + |Z(g)|
    for (int t = tid; t < 2 * OZ_D; t += OZ_THREADS) bx[t] = 0u;  // bx and by
    __syncthreads();
    for (int t = tid; t < d * d; t += OZ_THREADS) {
        const int i = t / d, k = t - i * d;
        const cx<dd> xa = ZX[f * E + t], xb = ZX[gZ * E + t];
        const cx<dd> ya = ZY[f * E + t], yb = ZY[gZ * E + t];
        const float mx = fabsf(xa.re.hi) + fabsf(xa.im.hi) + fabsf(xb.re.hi) + fabsf(xb.im.hi);
        const float my = fabsf(ya.re.hi) + fabsf(ya.im.hi) + fabsf(yb.re.hi) + fabsf(yb.im.hi);
        atomicMax(&bx[i], __float_as_uint(mx));  // X row i
        atomicMax(&by[k], __float_as_uint(my));  // Y entry (i=k row, k=column): column index is k here
    }
    __syncthreads();
    for (int t = tid; t < OZ_D; t += OZ_THREADS) {
        sig[t] = scale_exp(__uint_as_float(bx[t]));
        tau[t] = scale_exp(__uint_as_float(by[t]));
    }
    __syncthreads();

    const int lane = tid & 31, warp = tid >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int i0 = (warp & 3) * 16, j0 = (warp >> 2) * 32;
    const bool two = (gZ != f);
    const int nfreq = (gL == f) ? 1 : 2;  // p = M/2 pairs with itself

    cx<dd> keep[16];  // C(f) of this thread's outputs while C(g) is formed
    for (int phase = 0; phase < nfreq; ++phase) {
        // ---- split, scale and slice X(phi), Y(phi) into digit matrices
        const int64_t ra = phase == 0 ? f : gZ, rb = phase == 0 ? gZ : f;
        const cx<dd> w = phase == 0 ? wf : wg;
        for (int t = tid; t < OZ_D * OZ_D; t += OZ_THREADS) {
            const int i = t >> 6, k = t & 63;
            float qr[OZ_S], qi[OZ_S];
            // X entry (i, k)
            if (i < d && k < d) {
                const int64_t e = (int64_t)i * d + k;
                cx<dd> x = split_real(ZX[ra * E + e], ZX[rb * E + e], w);
                const float sc = pow2f(-sig[i]);
                digits6(x.re.hi * sc, x.re.lo * sc, qr);
                digits6(x.im.hi * sc, x.im.lo * sc, qi);
            } else {
#pragma unroll
                for (int s = 0; s < OZ_S; ++s) qr[s] = qi[s] = 0.0f;
            }
#pragma unroll
            for (int s = 0; s < OZ_S; ++s) {
                Xr[s * OZ_SLICE + i * OZ_LD + k] = bf16_bits(qr[s]);
                Xi[s * OZ_SLICE + i * OZ_LD + k] = bf16_bits(qi[s]);
            }
            // Y entry (row i -> k index of the product, column k -> j); stored transposed [j][k]
            if (i < d && k < d) {
                const int64_t e = (int64_t)i * d + k;
                cx<dd> y = split_real(ZY[ra * E + e], ZY[rb * E + e], w);
                const float sc = pow2f(-tau[k]);
                digits6(y.re.hi * sc, y.re.lo * sc, qr);
                digits6(y.im.hi * sc, y.im.lo * sc, qi);
            } else {
#pragma unroll
                for (int s = 0; s < OZ_S; ++s) qr[s] = qi[s] = 0.0f;
            }
#pragma unroll
            for (int s = 0; s < OZ_S; ++s) {
                YrT[s * OZ_SLICE + k * OZ_LD + i] = bf16_bits(qr[s]);
                YiT[s * OZ_SLICE + k * OZ_LD + i] = bf16_bits(qi[s]);
            }
        }
        __syncthreads();

        // ---- exact digit-pair products, grouped by weight
        long long acc64[8][4];
#pragma unroll
        for (int n = 0; n < 8; ++n)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc64[n][r] = 0;
        for (int g = 2 * (OZ_S - 1); g >= OZ_GMIN; --g) {
            float acc[8][4];
#pragma unroll
            for (int n = 0; n < 8; ++n)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[n][r] = 0.0f;
            for (int s = max(0, g - (OZ_S - 1)); s <= min(OZ_S - 1, g); ++s) {
                const int tt = g - s;
                const unsigned short *xr = Xr + s * OZ_SLICE, *xi = Xi + s * OZ_SLICE;
                const unsigned short *yr = YrT + tt * OZ_SLICE, *yi = YiT + tt * OZ_SLICE;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const unsigned short *xa = half == 0 ? xr : xi;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const int k0 = ks * 16 + tig * 2;
                        unsigned af[4];
                        af[0] = *reinterpret_cast<const unsigned *>(xa + (i0 + gid) * OZ_LD + k0);
                        af[1] = *reinterpret_cast<const unsigned *>(xa + (i0 + gid + 8) * OZ_LD + k0);
                        af[2] = *reinterpret_cast<const unsigned *>(xa + (i0 + gid) * OZ_LD + k0 + 8);
                        af[3] = *reinterpret_cast<const unsigned *>(xa + (i0 + gid + 8) * OZ_LD + k0 + 8);
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt) {
                            const int jn = j0 + nt * 8 + gid;
                            // C_r: X_r Y_r (half 0) + X_i (-Y_i) (half 1)
                            const unsigned short *br = half == 0 ? yr : yi;
                            unsigned b0 = *reinterpret_cast<const unsigned *>(br + jn * OZ_LD + k0);
                            unsigned b1 = *reinterpret_cast<const unsigned *>(br + jn * OZ_LD + k0 + 8);
                            if (half == 1) { b0 ^= 0x80008000u; b1 ^= 0x80008000u; }
                            mma_bf16(acc[nt], af, b0, b1);
                            // C_i: X_r Y_i (half 0) + X_i Y_r (half 1)
                            const unsigned short *bi = half == 0 ? yi : yr;
                            b0 = *reinterpret_cast<const unsigned *>(bi + jn * OZ_LD + k0);
                            b1 = *reinterpret_cast<const unsigned *>(bi + jn * OZ_LD + k0 + 8);
                            mma_bf16(acc[4 + nt], af, b0, b1);
                        }
                    }
                }
            }
            const int sh = 8 * (g - OZ_GMIN);
#pragma unroll
            for (int n = 0; n < 8; ++n)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc64[n][r] += (long long)__float2ll_rn(acc[n][r]) << sh;
        }
        __syncthreads();  // digit matrices are rewritten by the next phase

        // ---- back to double-float, scaled by 2^(sigma_i + tau_j - 56)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = i0 + gid + ((r >> 1) << 3), j = j0 + nt * 8 + tig * 2 + (r & 1);
                const int ex = sig[i] + tau[j] - 56;
                cx<dd> v;
                const long long sr = acc64[nt][r], si = acc64[4 + nt][r];
                float h = __ll2float_rn(sr);
                float l = __ll2float_rn(sr - __float2ll_rn(h));
                v.re = dd_fast_two_sum(scale2(h, ex), scale2(l, ex));
                h = __ll2float_rn(si);
                l = __ll2float_rn(si - __float2ll_rn(h));
                v.im = dd_fast_two_sum(scale2(h, ex), scale2(l, ex));
                const int o = nt * 4 + r;
                if (phase == 0) keep[o] = v;
                if (i >= d || j >= d) continue;
                const int64_t e = (int64_t)i * d + j;
                if (nfreq == 1) {
                    // p = M/2: C(g) = C(f)
                    ZC[f * E + e] = merge_real(v, v, c_conj(wf));
                } else if (phase == 1) {
                    const cx<dd> cf = keep[o];
                    ZC[f * E + e] = merge_real(cf, v, c_conj(wf));
                    if (two) ZC[gZ * E + e] = merge_real(v, cf, c_conj(wg));
                }
            }
    }
}

} // namespace

bool mrc_ozaki_supported(int r, int m, int c) { return r == m && m == c && r >= 32 && r <= OZ_D; }

cudaError_t mrc_ozaki_init(void)
{
    return cudaFuncSetAttribute(ozaki_pairmul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
}

cudaError_t mrc_pairmul_dd_ozaki(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                                 cudaStream_t st)
{
    PairArgs a{};
    a.zx = zx; a.zy = zy; a.zc = zc; a.tw = tw; a.tw_log = tw_log; a.M = M;
    int l = 0;
    while (((int64_t)1 << l) < M) ++l;
    a.logM = l;
    a.npairs = M >= 2 ? M / 2 + 1 : 1;
    a.r = a.m = a.c = d;
    const double bytes = (double)M * 3.0 * d * d * sizeof(cx<dd>);
    const double flops = 8.0 * d * d * d * (double)(M + 1);
    mrc_prof_pre(6, st);
    ozaki_pairmul_kernel<<<(unsigned)a.npairs, OZ_THREADS, OZ_SMEM, st>>>(a);
    mrc_prof_post(6, st, bytes, flops);
    return cudaGetLastError();
}
