// tf32x3.cu -- FP32 per-frequency complex matrix products on the tensor cores
// (square 16 <= d <= 64), for the Newton levels and the refinement
// correction of the mixed path.
//
// Every FP32 operand value v is split into two TF32 numbers, big = tf32(v)
// and small = tf32(v - big), so that v = big + small up to 2^-22 |v| (each
// keeps its own exponent: the split is relative per entry, unlike the
// row-scaled integer digits of ozaki.cu).  The product is formed as
//     X Y ~ Xb Yb + Xb Ys + Xs Yb
// with mma.sync m16n8k8 TF32 (FP32 accumulation); the dropped Xs Ys term
// weighs 2^-22 relative.  This matches the accuracy of an FP32 dot product,
// which is what the FP32 Newton levels and the correction need (error model
// of Proposition 2.1 with gamma_s = O(s u_32)).
//
// The complex product is the real product
//     [C_r | C_i] = [X_r | X_i] . [[Y_r, Y_i], [-Y_i, Y_r]]   (K = 2d).
// One CTA owns one frequency pair {f, M-f} and handles the real-FFT split
// and merge like the other product kernels: C(f) is kept in registers while
// C(M-f) is formed, then both are merged into the packed output spectrum.
#include "kernels.cuh"

namespace {

constexpr int TX_D = 64;       // padded matrix size
// Shared row lengths (words) that make every fragment load conflict-free:
// A reads 8 rows x 4 consecutive words (row stride 68: banks 4 gid + tig),
// B reads 4 rows x 8 consecutive words (row stride 72: banks 8 tig + gid).
constexpr int TX_LDX = 68;
constexpr int TX_LDY = 72;
constexpr int TX_THREADS = 512;
constexpr int TX_TX = TX_D * TX_LDX, TX_TY = TX_D * TX_LDY;
// shared: X_r, X_i ([i][k]) and Y_r, Y_i ([k][j]), each as big and small parts
constexpr size_t TX_SMEM = (size_t)(4 * TX_TX + 4 * TX_TY) * sizeof(unsigned);

__device__ __forceinline__ unsigned to_tf32(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// 16 warps: warp w owns rows 16 (w & 3) .. +16 and columns 16 (w >> 2) .. +16
// of both C_r and C_i (two n-tiles of 8 each).  Tiles are row-major as in
// global memory: X [i][k], Y [k][j].
__global__ void __launch_bounds__(TX_THREADS, 1) tf32x3_pairmul_kernel(PairArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned *sm = reinterpret_cast<unsigned *>(smem_raw);
    unsigned *Xrb = sm, *Xrs = sm + TX_TX, *Xib = sm + 2 * TX_TX, *Xis = sm + 3 * TX_TX;
    unsigned *Yb0 = sm + 4 * TX_TX;
    unsigned *Yrb = Yb0, *Yrs = Yb0 + TX_TY, *Yib = Yb0 + 2 * TX_TY, *Yis = Yb0 + 3 * TX_TY;

    const cx<float> *ZX = reinterpret_cast<const cx<float> *>(a.zx);
    const cx<float> *ZY = reinterpret_cast<const cx<float> *>(a.zy);
    cx<float> *ZC = reinterpret_cast<cx<float> *>(a.zc);
    const cx<float> *tw = reinterpret_cast<const cx<float> *>(a.tw);
    const int d = a.r;
    const int64_t E = (int64_t)d * d;
    const int64_t p = blockIdx.x, M = a.M;
    const int64_t f = p, gL = M - p, gZ = gL & (M - 1);
    const cx<float> wf = tw[f << (a.tw_log - a.logM - 1)];
    const cx<float> wg = c_neg(c_conj(wf));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int i0 = (warp & 3) * 16, j0 = (warp >> 2) * 16;
    const bool two = (gZ != f);
    const int nfreq = (gL == f) ? 1 : 2;
    const int dp = (d + 15) & ~15;  // padded size actually multiplied

    cx<float> keep[8];
    for (int phase = 0; phase < nfreq; ++phase) {
        const int64_t ra = phase == 0 ? f : gZ, rb = phase == 0 ? gZ : f;
        const cx<float> w = phase == 0 ? wf : wg;
        for (int t = tid; t < TX_D * TX_D; t += TX_THREADS) {
            const int i = t >> 6, k = t & 63;
            if (i >= dp || k >= dp) continue;
            cx<float> x = c_zero<float>(), y = c_zero<float>();
            if (i < d && k < d) {
                const int64_t e = (int64_t)i * d + k;
                x = split_real(ZX[ra * E + e], ZX[rb * E + e], w);
                y = split_real(ZY[ra * E + e], ZY[rb * E + e], w);
            }
            unsigned b;
            const int ox = i * TX_LDX + k, oy = i * TX_LDY + k;  // Y row i is the product's k index
            b = to_tf32(x.re); Xrb[ox] = b; Xrs[ox] = to_tf32(x.re - __uint_as_float(b));
            b = to_tf32(x.im); Xib[ox] = b; Xis[ox] = to_tf32(x.im - __uint_as_float(b));
            b = to_tf32(y.re); Yrb[oy] = b; Yrs[oy] = to_tf32(y.re - __uint_as_float(b));
            b = to_tf32(y.im); Yib[oy] = b; Yis[oy] = to_tf32(y.im - __uint_as_float(b));
        }
        __syncthreads();

        float acc[4][4];  // [0..1]: C_r n-tiles, [2..3]: C_i n-tiles
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[n][r] = 0.0f;
        if (i0 < dp && j0 < dp) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                // half 0: X_r with (Y_r -> C_r, Y_i -> C_i); half 1: X_i with (-Y_i -> C_r, Y_r -> C_i)
                const unsigned *xb = half == 0 ? Xrb : Xib, *xs = half == 0 ? Xrs : Xis;
                const unsigned *yrb = half == 0 ? Yrb : Yib, *yrs = half == 0 ? Yrs : Yis;
                const unsigned *yib = half == 0 ? Yib : Yrb, *yis = half == 0 ? Yis : Yrs;
                const unsigned neg = half == 1 ? 0x80000000u : 0u;
                for (int k0 = 0; k0 < dp; k0 += 8) {
                    const int ra0 = (i0 + gid) * TX_LDX + k0 + tig, ra1 = ra0 + 8 * TX_LDX;
                    const unsigned ab0 = xb[ra0], ab1 = xb[ra1], ab2 = xb[ra0 + 4], ab3 = xb[ra1 + 4];
                    const unsigned as0 = xs[ra0], as1 = xs[ra1], as2 = xs[ra0 + 4], as3 = xs[ra1 + 4];
                    // each k-step accumulates in a fresh tensor-core accumulator and is
                    // added to the running sums with round-to-nearest FP32 adds, so the
                    // tensor core's accumulation rounding never chains over K
                    float tk[4][4];
#pragma unroll
                    for (int n = 0; n < 4; ++n)
#pragma unroll
                        for (int r = 0; r < 4; ++r) tk[n][r] = 0.0f;
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        // B fragment: b0 = Y[k0 + tig][j], b1 = Y[k0 + tig + 4][j], j = j0 + 8 nt + gid
                        const int rbb = (k0 + tig) * TX_LDY + j0 + nt * 8 + gid, rb4 = rbb + 4 * TX_LDY;
                        // C_r
                        unsigned bb0 = yrb[rbb] ^ neg, bb1 = yrb[rb4] ^ neg;
                        unsigned bs0 = yrs[rbb] ^ neg, bs1 = yrs[rb4] ^ neg;
                        mma_tf32(tk[nt], as0, as1, as2, as3, bb0, bb1);
                        mma_tf32(tk[nt], ab0, ab1, ab2, ab3, bs0, bs1);
                        mma_tf32(tk[nt], ab0, ab1, ab2, ab3, bb0, bb1);
                        // C_i
                        bb0 = yib[rbb]; bb1 = yib[rb4];
                        bs0 = yis[rbb]; bs1 = yis[rb4];
                        mma_tf32(tk[2 + nt], as0, as1, as2, as3, bb0, bb1);
                        mma_tf32(tk[2 + nt], ab0, ab1, ab2, ab3, bs0, bs1);
                        mma_tf32(tk[2 + nt], ab0, ab1, ab2, ab3, bb0, bb1);
                    }
#pragma unroll
                    for (int n = 0; n < 4; ++n)
#pragma unroll
                        for (int r = 0; r < 4; ++r) acc[n][r] = __fadd_rn(acc[n][r], tk[n][r]);
                }
            }
        }
        __syncthreads();  // tiles are rewritten by the next phase

#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = i0 + gid + ((r >> 1) << 3), j = j0 + nt * 8 + tig * 2 + (r & 1);
                const cx<float> v = {acc[nt][r], acc[2 + nt][r]};
                const int o = nt * 4 + r;
                if (phase == 0) keep[o] = v;
                if (i >= d || j >= d) continue;
                const int64_t e = (int64_t)i * d + j;
                if (nfreq == 1) {
                    ZC[f * E + e] = merge_real(v, v, c_conj(wf));
                } else if (phase == 1) {
                    const cx<float> cf = keep[o];
                    ZC[f * E + e] = merge_real(cf, v, c_conj(wf));
                    if (two) ZC[gZ * E + e] = merge_real(v, cf, c_conj(wg));
                }
            }
    }
}

} // namespace

bool mrc_tf32x3_supported(int r, int m, int c) { return r == m && m == c && r >= 16 && r <= TX_D; }

cudaError_t mrc_tf32x3_init(void)
{
    return cudaFuncSetAttribute(tf32x3_pairmul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TX_SMEM);
}

cudaError_t mrc_pairmul_f32_tf32x3(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw,
                                   int tw_log, cudaStream_t st)
{
    PairArgs a{};
    a.zx = zx; a.zy = zy; a.zc = zc; a.tw = tw; a.tw_log = tw_log; a.M = M;
    int l = 0;
    while (((int64_t)1 << l) < M) ++l;
    a.logM = l;
    a.npairs = M >= 2 ? M / 2 + 1 : 1;
    a.r = a.m = a.c = d;
    const double bytes = (double)M * 3.0 * d * d * sizeof(cx<float>);
    const double flops = 8.0 * d * d * d * (double)(M + 1);
    mrc_prof_pre(5, st);
    tf32x3_pairmul_kernel<<<(unsigned)a.npairs, TX_THREADS, TX_SMEM, st>>>(a);
    mrc_prof_post(5, st, bytes, flops);
    return cudaGetLastError();
}
