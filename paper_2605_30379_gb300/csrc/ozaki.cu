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
// kernels.cuh), computes C(f) (kept in registers), then C(M-f), then merges
// both into the packed output spectrum.
#include <cuda_bf16.h>

#include "digits.cuh"

namespace {

using namespace mrc_digits;

constexpr int OZ_D = 64;       // padded matrix size
constexpr int OZ_LD = 72;      // shared-memory row length (bf16), padded against bank conflicts
constexpr int OZ_THREADS = 512;
constexpr int OZ_SLICE = OZ_D * OZ_LD;

template <class T>
constexpr size_t oz_smem() { return (size_t)4 * OzP<T>::S * OZ_SLICE * sizeof(unsigned short) + 4 * OZ_D * sizeof(int); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

// 16 warps: warp w owns rows 16 (w & 3) .. +16 and columns 16 (w >> 2) .. +16
// of both C_r and C_i (two n-tiles of 8 each).  Digit tiles are row-major
// [row][k] for X and [k][j] for Y (72-element rows: the 8 rows an ldmatrix
// phase touches fall in distinct banks).
template <class T>
__global__ void __launch_bounds__(OZ_THREADS, 1) ozaki_pairmul_kernel(PairArgs a)
{
    constexpr int OZ_S = OzP<T>::S, OZ_GMIN = OzP<T>::GMIN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned short *Xr = reinterpret_cast<unsigned short *>(smem_raw);  // [S][64][72]  X_r digits [i][k]
    unsigned short *Xi = Xr + OZ_S * OZ_SLICE;
    unsigned short *Yr = Xi + OZ_S * OZ_SLICE;  // [S][64][72]  Y_r digits [k][j]
    unsigned short *Yi = Yr + OZ_S * OZ_SLICE;
    unsigned *bx = reinterpret_cast<unsigned *>(Yi + OZ_S * OZ_SLICE);  // [64] row bounds (float bits)
    unsigned *by = bx + OZ_D;
    int *sig = reinterpret_cast<int *>(by + OZ_D);
    int *tau = sig + OZ_D;

    const cx<T> *ZX = reinterpret_cast<const cx<T> *>(a.zx);
    const cx<T> *ZY = reinterpret_cast<const cx<T> *>(a.zy);
    cx<T> *ZC = reinterpret_cast<cx<T> *>(a.zc);
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw);
    const int d = a.r;  // square: r = m = c = d <= 64
    const int64_t E = (int64_t)d * d;
    const int64_t p = blockIdx.x, M = a.M;
    const int64_t f = p, gL = M - p, gZ = gL & (M - 1);
    const cx<T> wf = tw[f << (a.tw_log - a.logM - 1)];
    const cx<T> wg = c_neg(c_conj(wf));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- magnitude bounds: |Xh(f)|, |Xh(g)| <= |Z(f)| + |Z(g)| entrywise.
    // The 64 x 64 (padded) grid is walked as t = tid + 512 n: a thread keeps
    // one column k = tid & 63, a warp one row per step.
    for (int t = tid; t < 2 * OZ_D; t += OZ_THREADS) bx[t] = 0u;
    __syncthreads();
    {
        const int k = tid & 63;
        float my = 0.0f;
        for (int t = tid; t < OZ_D * OZ_D; t += OZ_THREADS) {
            const int i = t >> 6;
            float mx = 0.0f;
            if (i < d && k < d) {
                const int64_t e = (int64_t)i * d + k;
                const cx<T> xa = ZX[f * E + e], xb = ZX[gZ * E + e];
                const cx<T> ya = ZY[f * E + e], yb = ZY[gZ * E + e];
                mx = fabsf(hi_part(xa.re)) + fabsf(hi_part(xa.im)) + fabsf(hi_part(xb.re)) + fabsf(hi_part(xb.im));
                my = fmaxf(my, fabsf(hi_part(ya.re)) + fabsf(hi_part(ya.im)) + fabsf(hi_part(yb.re)) +
                                   fabsf(hi_part(yb.im)));
            }
            const unsigned wmx = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));  // one row per warp
            if (lane == 0) atomicMax(&bx[i], wmx);
        }
        atomicMax(&by[k], __float_as_uint(my));
    }
    __syncthreads();
    for (int t = tid; t < OZ_D; t += OZ_THREADS) {
        sig[t] = scale_exp(__uint_as_float(bx[t]));
        tau[t] = scale_exp(__uint_as_float(by[t]));
    }
    __syncthreads();

    const int gid = lane >> 2, tig = lane & 3;
    const int i0 = (warp & 3) * 16, j0 = (warp >> 2) * 16;
    const bool two = (gZ != f);
    const int nfreq = (gL == f) ? 1 : 2;  // p = M/2 pairs with itself
    // ldmatrix lane addresses (element offsets inside one digit tile)
    const int a_off = (i0 + (lane & 15)) * OZ_LD + ((lane >> 4) << 3);               // + k0
    const int b_off = ((lane & 7) + (((lane >> 3) & 1) << 3)) * OZ_LD + j0 + ((lane >> 4) << 3);  // + k0 * OZ_LD

    cx<T> keep[8];  // C(f) of this thread's outputs while C(g) is formed
    for (int phase = 0; phase < nfreq; ++phase) {
        // ---- split, scale and slice X(phi), Y(phi) into digit tiles
        const int64_t ra = phase == 0 ? f : gZ, rb = phase == 0 ? gZ : f;
        const cx<T> w = phase == 0 ? wf : wg;
        for (int t = tid; t < OZ_D * OZ_D; t += OZ_THREADS) {
            const int i = t >> 6, k = t & 63;
            float qr[OZ_S], qi[OZ_S];
            const bool in = i < d && k < d;
            const int64_t e = (int64_t)i * d + k;
            if (in) {
                const cx<T> x = split_real(ZX[ra * E + e], ZX[rb * E + e], w);
                const float sc = pow2f(-sig[i]);
                split_digits(x.re, sc, qr);
                split_digits(x.im, sc, qi);
            } else {
#pragma unroll
                for (int s = 0; s < OZ_S; ++s) qr[s] = qi[s] = 0.0f;
            }
#pragma unroll
            for (int s = 0; s < OZ_S; ++s) {
                Xr[s * OZ_SLICE + i * OZ_LD + k] = bf16_bits(qr[s]);
                Xi[s * OZ_SLICE + i * OZ_LD + k] = bf16_bits(qi[s]);
            }
            // Y entry: row i is the product's k index, column k is j
            if (in) {
                const cx<T> y = split_real(ZY[ra * E + e], ZY[rb * E + e], w);
                const float sc = pow2f(-tau[k]);
                split_digits(y.re, sc, qr);
                split_digits(y.im, sc, qi);
            } else {
#pragma unroll
                for (int s = 0; s < OZ_S; ++s) qr[s] = qi[s] = 0.0f;
            }
#pragma unroll
            for (int s = 0; s < OZ_S; ++s) {
                Yr[s * OZ_SLICE + i * OZ_LD + k] = bf16_bits(qr[s]);
                Yi[s * OZ_SLICE + i * OZ_LD + k] = bf16_bits(qi[s]);
            }
        }
        __syncthreads();

        // ---- exact digit-pair products, grouped by weight
        long long acc64[4][4];
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc64[n][r] = 0;
        for (int g = 2 * (OZ_S - 1); g >= OZ_GMIN; --g) {
            float acc[4][4];  // [0..1]: C_r n-tiles, [2..3]: C_i n-tiles
#pragma unroll
            for (int n = 0; n < 4; ++n)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[n][r] = 0.0f;
            for (int s = max(0, g - (OZ_S - 1)); s <= min(OZ_S - 1, g); ++s) {
                const int tt = g - s;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    // half 0: X_r with (Y_r -> C_r, Y_i -> C_i); half 1: X_i with (-Y_i -> C_r, Y_r -> C_i)
                    const unsigned short *xa = (half == 0 ? Xr : Xi) + s * OZ_SLICE + a_off;
                    const unsigned short *ybr = (half == 0 ? Yr : Yi) + tt * OZ_SLICE + b_off;
                    const unsigned short *ybi = (half == 0 ? Yi : Yr) + tt * OZ_SLICE + b_off;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        unsigned af[4], br[4], bi[4];
                        ldsm_x4(af, xa + ks * 16);
                        ldsm_x4_t(br, ybr + ks * 16 * OZ_LD);
                        ldsm_x4_t(bi, ybi + ks * 16 * OZ_LD);
                        if (half == 1) {
#pragma unroll
                            for (int u = 0; u < 4; ++u) br[u] ^= 0x80008000u;
                        }
                        mma_bf16(acc[0], af, br[0], br[1]);
                        mma_bf16(acc[1], af, br[2], br[3]);
                        mma_bf16(acc[2], af, bi[0], bi[1]);
                        mma_bf16(acc[3], af, bi[2], bi[3]);
                    }
                }
            }
            const int sh = 8 * (g - OZ_GMIN);
#pragma unroll
            for (int n = 0; n < 4; ++n)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc64[n][r] += (long long)__float2ll_rn(acc[n][r]) << sh;
        }
        __syncthreads();  // digit tiles are rewritten by the next phase

        // ---- back to the working precision, scaled by 2^(sigma_i + tau_j + 8 GMIN - 16 S)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = i0 + gid + ((r >> 1) << 3), j = j0 + nt * 8 + tig * 2 + (r & 1);
                const int ex = sig[i] + tau[j] + 8 * OZ_GMIN - 16 * OZ_S;
                const cx<T> v = {from_int<T>(acc64[nt][r], ex), from_int<T>(acc64[2 + nt][r], ex)};
                const int o = nt * 4 + r;
                if (phase == 0) keep[o] = v;
                if (i >= d || j >= d) continue;
                const int64_t e = (int64_t)i * d + j;
                if (nfreq == 1) {
                    ZC[f * E + e] = merge_real(v, v, c_conj(wf));  // p = M/2: C(g) = C(f)
                } else if (phase == 1) {
                    const cx<T> cf = keep[o];
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
    cudaError_t e = cudaFuncSetAttribute(ozaki_pairmul_kernel<dd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)oz_smem<dd>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(ozaki_pairmul_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)oz_smem<float>());
}

template <class T>
cudaError_t ozaki_run(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                      cudaStream_t st, int kclass)
{
    PairArgs a{};
    a.zx = zx; a.zy = zy; a.zc = zc; a.tw = tw; a.tw_log = tw_log; a.M = M;
    int l = 0;
    while (((int64_t)1 << l) < M) ++l;
    a.logM = l;
    a.npairs = M >= 2 ? M / 2 + 1 : 1;
    a.r = a.m = a.c = d;
    const double bytes = (double)M * 3.0 * d * d * sizeof(cx<T>);
    const double flops = 8.0 * d * d * d * (double)(M + 1);
    mrc_prof_pre(kclass, st);
    ozaki_pairmul_kernel<T><<<(unsigned)a.npairs, OZ_THREADS, oz_smem<T>(), st>>>(a);
    mrc_prof_post(kclass, st, bytes, flops);
    return cudaGetLastError();
}

cudaError_t mrc_pairmul_dd_ozaki(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                                 cudaStream_t st)
{
    return ozaki_run<dd>(zx, zy, zc, M, d, tw, tw_log, st, 6);
}

cudaError_t mrc_pairmul_f32_ozaki(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw,
                                  int tw_log, cudaStream_t st)
{
    return ozaki_run<float>(zx, zy, zc, M, d, tw, tw_log, st, 5);
}
