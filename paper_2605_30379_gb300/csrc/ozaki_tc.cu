// ozaki_tc.cu -- per-frequency complex matrix products of the FFT-Newton path
// (Eq. (fft-convolution): C(phi) = X(phi) Y(phi) at every frequency of the
// half spectrum) as exact digit products on the fifth-generation tensor
// cores: tcgen05.mma, BF16 operands in shared memory, FP32 accumulators in
// tensor memory (TMEM).  Square d x d with 32 <= d <= 512: 64 x 64 output
// tiles (padded), K in chunks of 64 whose group sums are exact and are added
// in the working precision; the row and column scalings are taken once per
// frequency pair over whole rows and columns.
//
// For the frequency pair {f, M-f} one CTA forms, at each frequency phi and
// for each output tile and K chunk,
//     D = A1 . Y_r + A2 . Y_i = [C_r; C_i]                      (128 x 64),
//     A1 = [X_r; X_i],  A2 = [-X_i; X_r],
// i.e. C_r = X_r Y_r - X_i Y_i and C_i = X_i Y_r + X_r Y_i in one
// accumulator.  The rows of X are scaled by 2^-sigma_i and the columns of Y
// by 2^-tau_j, every value is split into S balanced base-256 digits
// (digits.cuh), and each digit of X is stored once as a 192-row MN-major
// tile [-X_i; X_r; X_i]: A1 is its rows 64..191 and A2 its rows 0..127, two
// descriptors into the same tile.  Y_r and Y_i digits are K-major 64-row
// tiles.  All digit pairs (s, t) of one weight group g = s + t >= GMIN
// accumulate into one 64-column FP32 accumulator in TMEM -- exact, since a
// group holds at most 6 pairs of two 64-term dot products of digits <= 128
// (below 2^24).  The group sums are then scaled by their powers of two
// (exact) and added top group first in the working precision: a compensated
// double-float sum for the residual product, plain FP32 for the FP32 one.
// Nothing here converts to or from 64-bit integers: on this GPU those
// conversions share the narrow FP64 pipe.
//
// Schedule per frequency, in two halves of K (k < 32, k >= 32; 120 KB of
// digit tiles each for double-float): every thread splits four entries of X
// and then four of Y into digit tiles; one thread issues the MMAs (every kept
// pair, two K = 16 steps, A1 with Y_r and A2 with Y_i, M = 128, N = 64) and
// commits them to an mbarrier; all threads wait (bounded) before the tiles
// are rewritten.  After the second half every warp reads its lanes of the
// accumulators with tcgen05.ld and folds them; C_r and C_i meet in shared
// memory and each thread forms 8 complex outputs.  C(f) is stored unmerged
// and read back by the same thread once C(M-f) is known, when both are
// merged into the packed output spectrum (the real-FFT merge of
// kernels.cuh).  The kernel is persistent: CTA b takes pairs b, b + grid, ...
//
// A bounded wait that gives up sets MRC_ERR_TIMEOUT in the status word; the
// CTA then waits (bounded) for its MMAs in flight, frees its TMEM and exits.
#include "digits.cuh"

namespace {

using namespace mrc_digits;

constexpr int TC_THREADS = 512;
constexpr int TC_KH = 32;                  // K per half
constexpr int TC_SBO = (TC_KH / 8) * 128;  // bytes between 8-row groups of a tile (4 K groups of 128 bytes)
constexpr int TC_A_TILE = 192 * TC_KH * 2; // bytes of one [-X_i; X_r; X_i] digit tile (one K half)
constexpr int TC_B_TILE = 64 * TC_KH * 2;  // bytes of one Y_r or Y_i digit tile (one K half)
constexpr int TC_XLD = 65;                 // row length (values) of the C_r / C_i exchange
constexpr unsigned TC_TMEM_COLS = 512;
constexpr int TC_SPIN = 1 << 24;

template <class T>
__host__ __device__ constexpr size_t tc_tiles() { return (size_t)OzP<T>::S * (TC_A_TILE + 2 * TC_B_TILE); }
constexpr int TC_DMAX = 512;  // largest d (rows of X / columns of Y whose scalings are kept)
// digit tiles | the 128 x 64 output-tile accumulator (C_r; C_i rows) | row and column bounds and exponents
template <class T>
__host__ __device__ constexpr size_t tc_xs_off() { return tc_tiles<T>(); }
template <class T>
__host__ __device__ constexpr size_t tc_small_bounds_off() { return tc_tiles<T>(); }
template <class T>
__host__ __device__ constexpr size_t tc_small_smem() { return tc_tiles<T>() + 4 * 64 * sizeof(int); }
static_assert((size_t)128 * TC_XLD * sizeof(dd) <= (size_t)5 * (TC_A_TILE + 2 * TC_B_TILE), "exchange fits the tiles");
template <class T>
__host__ __device__ constexpr size_t tc_smem() { return tc_tiles<T>() + (size_t)128 * TC_XLD * sizeof(T) + 4 * TC_DMAX * sizeof(int); }

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Byte offset of (m, k) in an MN-major tile (one K half): 8 consecutive m in
// 16 bytes, core matrices of 8 k rows, k groups 128 bytes apart, m groups
// TC_SBO apart.
__device__ __forceinline__ int mn_off(int m, int k) { return (m >> 3) * TC_SBO + (k >> 3) * 128 + (k & 7) * 16 + (m & 7) * 2; }
// Byte offset of (n, k) in a K-major tile: 8 consecutive k in 16 bytes, core
// matrices of 8 n rows, k groups 128 bytes apart, n groups TC_SBO apart.
__device__ __forceinline__ int k_off(int n, int k) { return (n >> 3) * TC_SBO + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2; }

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset 128 (next 8-element K group), stride byte offset TC_SBO (next 8
// rows of M or N), the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(unsigned addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(TC_SBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), A MN-major (bit 15), B K-major, N >> 3 at bit 17,
// M >> 4 at bit 24: M = 128, N = 64.
constexpr unsigned TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(unsigned dtm, uint64_t ad, uint64_t bd, unsigned acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
                 "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Bounded wait for the completion of phase `parity` of an mbarrier: at most
// `spins` rounds of try_wait, each suspending the thread for at most about
// TC_SUSPEND_NS nanoseconds, so the wait gives up after about spins x 1 us.
constexpr unsigned TC_SUSPEND_NS = 1000;
__device__ __forceinline__ bool tc_wait(unsigned mbar, unsigned parity, int spins = TC_SPIN)
{
    for (int it = 0; it < spins; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity), "r"(TC_SUSPEND_NS)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives on (no asynchronous copy or MMA is in flight), gives up after
// `spins` rounds and reports MRC_ERR_TIMEOUT (6) to *status.
__global__ void tc_wait_selftest_kernel(int *status, int spins)
{
    __shared__ __align__(8) unsigned long long mbar;
    const unsigned mb = smem_u32(&mbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (!tc_wait(mb, 0, spins) && status) atomicExch(status, 6);
}

// 32 TMEM lanes x 8 consecutive 32-bit columns: thread `lane` of the warp
// receives lane (base lane + lane), columns col .. col + 7.
__device__ __forceinline__ void tc_ld8(unsigned taddr, unsigned (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// MMAs of one K half of D = A1 . Y_r + A2 . Y_i over every kept digit pair:
// group g accumulates in TMEM columns 64 (g - GMIN) .. +63; `fresh` makes
// the first MMA of each group overwrite (the first K half).
template <int S, int GMIN>
__device__ __forceinline__ void tc_issue(unsigned tmem, unsigned a0, unsigned br0, unsigned bi0, bool fresh)
{
    for (int g = GMIN; g <= 2 * (S - 1); ++g) {
        const unsigned dcol = tmem + (unsigned)(g - GMIN) * 64u;
        unsigned acc = fresh ? 0u : 1u;
        for (int s = max(0, g - (S - 1)); s <= min(S - 1, g); ++s) {
            const int t = g - s;
            const unsigned as = a0 + s * TC_A_TILE;
#pragma unroll
            for (int ks = 0; ks < TC_KH / 16; ++ks) {
                tc_mma(dcol, tc_desc(as + 8 * TC_SBO + ks * 256), tc_desc(br0 + t * TC_B_TILE + ks * 256), acc);
                acc = 1;
                tc_mma(dcol, tc_desc(as + ks * 256), tc_desc(bi0 + t * TC_B_TILE + ks * 256), 1u);
            }
        }
    }
}

// value + v for a float v: one TwoSum of the high parts, lo parts added once
// (the sloppy double-float add of arith.cuh with a float operand)
__device__ __forceinline__ dd tc_add(dd a, float v)
{
    const dd s = dd_two_sum(a.hi, v);
    return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ float tc_add(float a, float v) { return __fadd_rn(a, v); }

// Fold the NG group accumulators of TMEM lanes 32 q + lane, columns
// cb .. cb + 15: sum over g of acc_g 2^(8 (g - NG + 1)), every term an exact
// FP32 value.  The top three groups are added as a compensated double-float
// sum; below them (weights 2^-24 and less of the top group) plain FP32 adds
// suffice -- their rounding, under 2^-46 of the magnitudes, is of the order
// of the digit pairs the split drops -- and the low sum joins once.
template <class T, int NG>
__device__ __forceinline__ void tc_fold(unsigned tmem, int q, int cb, T (&out)[16])
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // two halves of 8 columns: fewer live registers
        float lo[8];
#pragma unroll
        for (int g = NG - 1; g >= 0; --g) {
            unsigned r[8];
            tc_ld8(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(g * 64 + cb + 8 * h), r);
            const float w = __uint_as_float((unsigned)(127 - 8 * (NG - 1 - g)) << 23);  // 2^(8 (g - NG + 1))
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float v = __uint_as_float(r[c]) * w;
                T &o = out[8 * h + c];
                if constexpr (__is_same(T, dd)) {
                    if (g == NG - 1) o = dd{v, 0.0f};
                    else if (g >= NG - 3) o = tc_add(o, v);
                    else if (g == NG - 4) lo[c] = v;
                    else lo[c] = __fadd_rn(lo[c], v);
                } else {
                    if (g == NG - 1) o = v;
                    else o = tc_add(o, v);
                }
            }
        }
        if constexpr (__is_same(T, dd) && NG > 3) {
#pragma unroll
            for (int c = 0; c < 8; ++c) out[8 * h + c] = tc_add(out[8 * h + c], lo[c]);
        }
    }
}

// BF16 bits of two exact small integers (|q| <= 128 has at most 8
// significant bits, so the high half of the binary32 is the BF16 value),
// packed low | high
__device__ __forceinline__ unsigned tc_pack2(float lo, float hi)
{
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// Digit tiles of X(phi) for the K half k0 .. k0 + 31 (phi: packed rows ra,
// partner rb, twiddle w): thread t (i4 = t / 32, k = t % 32) splits
// X[4 i4 .. 4 i4 + 3][k0 + k] (lanes read consecutive k: coalesced) and
// writes, per digit, 8 bytes of 4 consecutive rows into each of the three
// blocks of the MN-major tile: -X_i (rows 0..63), X_r (64..127), X_i
// (128..191).  All warps run this, then tc_split_y, in the same order.
template <class T>
__device__ __forceinline__ void tc_split_x(const PairArgs &a, unsigned char *sA, const int *sig, int64_t ra,
                                           int64_t rb, cx<T> w, int i0, int k0, int t)
{
    constexpr int S = OzP<T>::S;
    const cx<T> *ZX = reinterpret_cast<const cx<T> *>(a.zx);
    const int d = a.r;
    const int64_t E = (int64_t)d * d;
    const int k = t & 31, i4 = t >> 5, kg = k0 + k;
    cx<T> z[4][2];
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {  // loads first
        const int i = i0 + 4 * i4 + ii;
        const int64_t e = (int64_t)i * d + kg;
        z[ii][0] = (i < d && kg < d) ? ZX[ra * E + e] : c_zero<T>();
        z[ii][1] = (i < d && kg < d) ? ZX[rb * E + e] : c_zero<T>();
    }
    unsigned wr[S][2], wi[S][2];
    float pr[S], pi[S];  // digits of the even entry of each pair
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
        const int i = i0 + 4 * i4 + ii;
        float qr[S], qi[S];
        const cx<T> x = split_real(z[ii][0], z[ii][1], w);
        const float sc = i < d ? pow2f(-sig[i]) : 0.0f;
        split_digits(x.re, sc, qr);
        split_digits(x.im, sc, qi);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (ii & 1) {
                wr[s][ii >> 1] = tc_pack2(pr[s], qr[s]);
                wi[s][ii >> 1] = tc_pack2(pi[s], qi[s]);
            } else {
                pr[s] = qr[s];
                pi[s] = qi[s];
            }
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        unsigned char *tl = sA + s * TC_A_TILE;
        *reinterpret_cast<uint2 *>(tl + mn_off(4 * i4, k)) =
            make_uint2(wi[s][0] ^ 0x80008000u, wi[s][1] ^ 0x80008000u);
        *reinterpret_cast<uint2 *>(tl + mn_off(64 + 4 * i4, k)) = make_uint2(wr[s][0], wr[s][1]);
        *reinterpret_cast<uint2 *>(tl + mn_off(128 + 4 * i4, k)) = make_uint2(wi[s][0], wi[s][1]);
    }
}

// Digit tiles of Y(phi) for the K half k0 .. k0 + 31: thread t (k4 = t / 64,
// j = t % 64) splits Y[k0 + 4 k4 .. + 3][j] (lanes read consecutive j:
// coalesced) and writes, per digit, 8 bytes of 4 consecutive k into the
// K-major tiles of Y_r and Y_i (row n = j).
template <class T>
__device__ __forceinline__ void tc_split_y(const PairArgs &a, unsigned char *sBr, unsigned char *sBi, const int *tau,
                                           int64_t ra, int64_t rb, cx<T> w, int j0, int k0, int t)
{
    constexpr int S = OzP<T>::S;
    const cx<T> *ZY = reinterpret_cast<const cx<T> *>(a.zy);
    const int d = a.r;
    const int64_t E = (int64_t)d * d;
    const int jt = t & 63, k4 = t >> 6, j = j0 + jt;
    cx<T> z[4][2];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {  // loads first
        const int k = k0 + 4 * k4 + kk;
        const int64_t e = (int64_t)k * d + j;
        z[kk][0] = (k < d && j < d) ? ZY[ra * E + e] : c_zero<T>();
        z[kk][1] = (k < d && j < d) ? ZY[rb * E + e] : c_zero<T>();
    }
    unsigned wr[S][2], wi[S][2];
    float pr[S], pi[S];
    const float sc = j < d ? pow2f(-tau[j]) : 0.0f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        float qr[S], qi[S];
        const cx<T> y = split_real(z[kk][0], z[kk][1], w);
        split_digits(y.re, sc, qr);
        split_digits(y.im, sc, qi);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (kk & 1) {
                wr[s][kk >> 1] = tc_pack2(pr[s], qr[s]);
                wi[s][kk >> 1] = tc_pack2(pi[s], qi[s]);
            } else {
                pr[s] = qr[s];
                pi[s] = qi[s];
            }
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        *reinterpret_cast<uint2 *>(sBr + s * TC_B_TILE + k_off(jt, 4 * k4)) = make_uint2(wr[s][0], wr[s][1]);
        *reinterpret_cast<uint2 *>(sBi + s * TC_B_TILE + k_off(jt, 4 * k4)) = make_uint2(wi[s][0], wi[s][1]);
    }
}

__device__ __forceinline__ dd tc_scale(dd x, int e) { return {scale2(x.hi, e), scale2(x.lo, e)}; }
__device__ __forceinline__ float tc_scale(float x, int e) { return scale2(x, e); }

// d <= 64: one output tile and one K chunk per frequency; the exchange of
// C_r and C_i reuses the digit tiles and the bounds sit right after them
// (a smaller and tighter kernel than the tiled one below, which it matches
// result for result).
template <class T>
__global__ void __launch_bounds__(TC_THREADS, 1) oztc_pairmul_kernel(PairArgs a, int *status)
{
    constexpr int S = OzP<T>::S, GMIN = OzP<T>::GMIN, NG = 2 * (S - 1) - GMIN + 1;
    static_assert(NG * 64 <= (int)TC_TMEM_COLS, "group accumulators fit in TMEM");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                 // [S] 192 x 32 MN-major: -X_i, X_r, X_i
    unsigned char *sBr = sA + S * TC_A_TILE;  // [S] 64 x 32 K-major (Y_r)
    unsigned char *sBi = sBr + S * TC_B_TILE; // [S] 64 x 32 K-major (Y_i)
    T *xs = reinterpret_cast<T *>(smem);      // C_r | C_i exchange (reuses the tiles)
    unsigned *bx = reinterpret_cast<unsigned *>(smem + tc_small_bounds_off<T>());
    unsigned *by = bx + 64;
    int *sig = reinterpret_cast<int *>(by + 64);
    int *tau = sig + 64;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tslot;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned mb = smem_u32(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tslot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tslot;
    unsigned parity = 0;
    bool failed = false;

    const cx<T> *ZX = reinterpret_cast<const cx<T> *>(a.zx);
    const cx<T> *ZY = reinterpret_cast<const cx<T> *>(a.zy);
    cx<T> *ZC = reinterpret_cast<cx<T> *>(a.zc);
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw);
    const int d = a.r;
    const int64_t E = (int64_t)d * d, M = a.M;
    const int q = warp & 3, cb = (warp >> 2) * 16;  // TMEM lanes 32 q .., columns cb .. cb + 15

    for (int64_t p = blockIdx.x; p < a.npairs && !failed; p += gridDim.x) {
        const int64_t f = p, gL = M - p, gZ = gL & (M - 1);
        const cx<T> wf = tw[f << (a.tw_log - a.logM - 1)];
        const cx<T> wg = c_neg(c_conj(wf));
        const bool two = (gZ != f);
        const int nfreq = (gL == f) ? 1 : 2;  // p = M/2 pairs with itself

        // ---- row bounds of X and column bounds of Y over both frequencies:
        // |Xh(f)|, |Xh(g)| <= |Z(f)| + |Z(g)| entrywise
        for (int t = tid; t < 128; t += TC_THREADS) bx[t] = 0u;
        __syncthreads();
        {
            const int k = tid & 63;
            float my = 0.0f;
            for (int t = tid; t < 64 * 64; t += TC_THREADS) {
                const int i = t >> 6;
                float mx = 0.0f;
                if (i < d && k < d) {
                    const int64_t e = (int64_t)i * d + k;
                    const cx<T> xa = ZX[f * E + e], xb = ZX[gZ * E + e];
                    const cx<T> ya = ZY[f * E + e], yb = ZY[gZ * E + e];
                    mx = fabsf(hi_part(xa.re)) + fabsf(hi_part(xa.im)) + fabsf(hi_part(xb.re)) +
                         fabsf(hi_part(xb.im));
                    my = fmaxf(my, fabsf(hi_part(ya.re)) + fabsf(hi_part(ya.im)) + fabsf(hi_part(yb.re)) +
                                       fabsf(hi_part(yb.im)));
                }
                const unsigned wmx = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));  // one row per warp
                if (lane == 0) atomicMax(&bx[i], wmx);
            }
            atomicMax(&by[k], __float_as_uint(my));
        }
        __syncthreads();
        if (tid < 64) {
            sig[tid] = scale_exp(__uint_as_float(bx[tid]));
            tau[tid] = scale_exp(__uint_as_float(by[tid]));
        }
        __syncthreads();

        for (int phase = 0; phase < nfreq && !failed; ++phase) {
            const int64_t ra = phase == 0 ? f : gZ, rb = phase == 0 ? gZ : f;
            const cx<T> w = phase == 0 ? wf : wg;
            for (int kh = 0; kh < 64 / TC_KH; ++kh) {
                tc_split_x<T>(a, sA, sig, ra, rb, w, 0, kh * TC_KH, tid);
                tc_split_y<T>(a, sBr, sBi, tau, ra, rb, w, 0, kh * TC_KH, tid);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // digit tiles visible to the MMAs
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    tc_issue<S, GMIN>(tmem, smem_u32(sA), smem_u32(sBr), smem_u32(sBi), kh == 0);
                    tc_commit(mb);
                }
                const bool ok = tc_wait(mb, parity);  // before the tiles are rewritten or the sums read
                parity ^= 1u;
                if (__syncthreads_or(!ok)) {
                    failed = true;
                    break;
                }
            }
            if (failed) break;

            // ---- fold the group sums of D = [C_r; C_i]; C_r and C_i meet in shared memory
            T dv[16];
            tc_fence_after();
            tc_fold<T, NG>(tmem, q, cb, dv);
            tc_fence_before();
            __syncthreads();  // accumulators read before the next MMAs
            {
                const int row = 32 * q + lane;
#pragma unroll
                for (int c = 0; c < 16; ++c) xs[row * TC_XLD + cb + c] = dv[c];
            }
            __syncthreads();
            {
                const int i = tid & 63, jb = tid >> 6;
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int j = 8 * jb + jj;
                    if (i >= d || j >= d) continue;
                    // the fold factored out 2^(8 (NG - 1)) of the group weights 2^(8 (g - GMIN))
                    const int ex = sig[i] + tau[j] + 8 * GMIN - 16 * S + 8 * (NG - 1);
                    const cx<T> v = {tc_scale(xs[i * TC_XLD + j], ex), tc_scale(xs[(64 + i) * TC_XLD + j], ex)};
                    const int64_t e = (int64_t)i * d + j;
                    if (nfreq == 1) {
                        ZC[f * E + e] = merge_real(v, v, c_conj(wf));  // p = M/2: C(g) = C(f)
                    } else if (phase == 0) {
                        ZC[f * E + e] = v;  // C(f), merged once C(g) is known (same thread)
                    } else {
                        const cx<T> cf = ZC[f * E + e];
                        ZC[f * E + e] = merge_real(cf, v, c_conj(wf));
                        if (two) ZC[gZ * E + e] = merge_real(v, cf, c_conj(wg));
                    }
                }
            }
            __syncthreads();  // exchange read before the next digit tiles
        }
    }

    if (failed) {
        if (tid == 0 && status) atomicExch(status, 6);
        tc_wait(mb, parity);  // let MMAs still in flight finish before the TMEM is freed
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// d > 64: 64 x 64 output tiles and 64-deep K chunks.
template <class T>
__global__ void __launch_bounds__(TC_THREADS, 1) oztc_tiled_kernel(PairArgs a, int *status)
{
    constexpr int S = OzP<T>::S, GMIN = OzP<T>::GMIN, NG = 2 * (S - 1) - GMIN + 1;
    static_assert(NG * 64 <= (int)TC_TMEM_COLS, "group accumulators fit in TMEM");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                 // [S] 192 x 32 MN-major: -X_i, X_r, X_i
    unsigned char *sBr = sA + S * TC_A_TILE;  // [S] 64 x 32 K-major (Y_r)
    unsigned char *sBi = sBr + S * TC_B_TILE; // [S] 64 x 32 K-major (Y_i)
    T *xs = reinterpret_cast<T *>(smem + tc_xs_off<T>());  // [C_r; C_i] of one output tile, summed over K chunks
    unsigned *bx = reinterpret_cast<unsigned *>(xs + 128 * TC_XLD);
    unsigned *by = bx + TC_DMAX;
    int *sig = reinterpret_cast<int *>(by + TC_DMAX);
    int *tau = sig + TC_DMAX;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tslot;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned mb = smem_u32(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tslot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tslot;
    unsigned parity = 0;
    bool failed = false;

    const cx<T> *ZX = reinterpret_cast<const cx<T> *>(a.zx);
    const cx<T> *ZY = reinterpret_cast<const cx<T> *>(a.zy);
    cx<T> *ZC = reinterpret_cast<cx<T> *>(a.zc);
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw);
    const int d = a.r, nt = (d + 63) / 64;  // 64 x 64 output tiles per side, 64-deep K chunks
    const int64_t E = (int64_t)d * d, M = a.M;
    const int q = warp & 3, cb = (warp >> 2) * 16;  // TMEM lanes 32 q .., columns cb .. cb + 15

    for (int64_t p = blockIdx.x; p < a.npairs && !failed; p += gridDim.x) {
        const int64_t f = p, gL = M - p, gZ = gL & (M - 1);
        const cx<T> wf = tw[f << (a.tw_log - a.logM - 1)];
        const cx<T> wg = c_neg(c_conj(wf));
        const bool two = (gZ != f);
        const int nfreq = (gL == f) ? 1 : 2;  // p = M/2 pairs with itself

        // ---- row bounds of X (a warp per row) and column bounds of Y (eight
        // threads per column, rows k = kq, kq + 8, ...) over both
        // frequencies: |Xh(f)|, |Xh(g)| <= |Z(f)| + |Z(g)| entrywise
        for (int j = tid; j < d; j += TC_THREADS) by[j] = 0u;
        __syncthreads();
        for (int i = warp; i < d; i += TC_THREADS / 32) {
            float mx = 0.0f;
            for (int k = lane; k < d; k += 32) {
                const int64_t e = (int64_t)i * d + k;
                const cx<T> xa = ZX[f * E + e], xb = ZX[gZ * E + e];
                mx = fmaxf(mx, fabsf(hi_part(xa.re)) + fabsf(hi_part(xa.im)) + fabsf(hi_part(xb.re)) +
                                   fabsf(hi_part(xb.im)));
            }
            mx = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
            if (lane == 0) sig[i] = scale_exp(mx);
        }
        for (int jb = 0; jb < nt; ++jb) {
            const int j = 64 * jb + (tid & 63);
            if (j >= d) continue;
            float my = 0.0f;
            for (int k = tid >> 6; k < d; k += TC_THREADS / 64) {
                const int64_t e = (int64_t)k * d + j;
                const cx<T> ya = ZY[f * E + e], yb = ZY[gZ * E + e];
                my = fmaxf(my, fabsf(hi_part(ya.re)) + fabsf(hi_part(ya.im)) + fabsf(hi_part(yb.re)) +
                                   fabsf(hi_part(yb.im)));
            }
            atomicMax(&by[j], __float_as_uint(my));  // nonnegative floats order as their bits
        }
        __syncthreads();
        for (int j = tid; j < d; j += TC_THREADS) tau[j] = scale_exp(__uint_as_float(by[j]));
        __syncthreads();

        for (int tile = 0; tile < nt * nt && !failed; ++tile) {
            const int i0 = (tile / nt) * 64, j0 = (tile % nt) * 64;
            for (int phase = 0; phase < nfreq && !failed; ++phase) {
                const int64_t ra = phase == 0 ? f : gZ, rb = phase == 0 ? gZ : f;
                const cx<T> w = phase == 0 ? wf : wg;
                for (int kc = 0; kc < nt && !failed; ++kc) {
                    for (int kh = 0; kh < 64 / TC_KH; ++kh) {
                        const int k0 = 64 * kc + kh * TC_KH;
                        tc_split_x<T>(a, sA, sig, ra, rb, w, i0, k0, tid);
                        tc_split_y<T>(a, sBr, sBi, tau, ra, rb, w, j0, k0, tid);
                        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // tiles visible to the MMAs
                        __syncthreads();
                        if (tid == 0) {
                            tc_fence_after();
                            tc_issue<S, GMIN>(tmem, smem_u32(sA), smem_u32(sBr), smem_u32(sBi), kh == 0);
                            tc_commit(mb);
                        }
                        const bool ok = tc_wait(mb, parity);  // before the tiles are rewritten or the sums read
                        parity ^= 1u;
                        if (__syncthreads_or(!ok)) {
                            failed = true;
                            break;
                        }
                    }
                    if (failed) break;
                    // ---- fold this K chunk's group sums (exact per chunk) into the tile accumulator
                    T dv[16];
                    tc_fence_after();
                    tc_fold<T, NG>(tmem, q, cb, dv);
                    tc_fence_before();
                    T *xr = xs + (32 * q + lane) * TC_XLD + cb;
                    if (kc == 0) {
#pragma unroll
                        for (int c = 0; c < 16; ++c) xr[c] = dv[c];
                    } else {
#pragma unroll
                        for (int c = 0; c < 16; ++c) xr[c] = Ar<T>::add(xr[c], dv[c]);
                    }
                }
                if (failed) break;
                __syncthreads();  // the tile's C_r and C_i complete in shared memory
                {
                    const int i = tid & 63, jb = tid >> 6;
                    const int gi = i0 + i;
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const int gj = j0 + 8 * jb + jj;
                        if (gi >= d || gj >= d) continue;
                        // the fold factored out 2^(8 (NG - 1)) of the group weights 2^(8 (g - GMIN))
                        const int ex = sig[gi] + tau[gj] + 8 * GMIN - 16 * S + 8 * (NG - 1);
                        const cx<T> v = {tc_scale(xs[i * TC_XLD + 8 * jb + jj], ex),
                                         tc_scale(xs[(64 + i) * TC_XLD + 8 * jb + jj], ex)};
                        const int64_t e = (int64_t)gi * d + gj;
                        if (nfreq == 1) {
                            ZC[f * E + e] = merge_real(v, v, c_conj(wf));  // p = M/2: C(g) = C(f)
                        } else if (phase == 0) {
                            ZC[f * E + e] = v;  // C(f), merged once C(g) is known (same thread)
                        } else {
                            const cx<T> cf = ZC[f * E + e];
                            ZC[f * E + e] = merge_real(cf, v, c_conj(wf));
                            if (two) ZC[gZ * E + e] = merge_real(v, cf, c_conj(wg));
                        }
                    }
                }
                __syncthreads();  // the tile accumulator is read before the next tile's first fold
            }
        }
        __syncthreads();  // bounds of this pair are read before the next pair's
    }

    if (failed) {
        if (tid == 0 && status) atomicExch(status, 6);
        tc_wait(mb, parity);  // let MMAs still in flight finish before the TMEM is freed
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

} // namespace

bool mrc_tc_supported(int r, int m, int c) { return r == m && m == c && r >= 32 && r <= TC_DMAX; }

cudaError_t mrc_tc_wait_selftest(int *status, int spins, cudaStream_t st)
{
    mrc_prof_pre(7, st);
    tc_wait_selftest_kernel<<<1, 1, 0, st>>>(status, spins);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_tc_init(void)
{
    cudaError_t e = cudaFuncSetAttribute(oztc_pairmul_kernel<dd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_small_smem<dd>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(oztc_tiled_kernel<dd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc_smem<dd>());
    return e;
}

cudaError_t mrc_pairmul_dd_tc(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                              int *status, cudaStream_t st)
{
    using T = dd;
    PairArgs a{};
    a.zx = zx; a.zy = zy; a.zc = zc; a.tw = tw; a.tw_log = tw_log; a.M = M;
    int l = 0;
    while (((int64_t)1 << l) < M) ++l;
    a.logM = l;
    a.npairs = M >= 2 ? M / 2 + 1 : 1;
    a.r = a.m = a.c = d;
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    const unsigned grid = (unsigned)std::min<int64_t>(a.npairs, nsm);
    const double bytes = (double)M * 3.0 * d * d * sizeof(cx<T>);
    const double flops = 8.0 * d * d * d * (double)(M + 1);
    mrc_prof_pre(6, st);
    if (d <= 64) oztc_pairmul_kernel<T><<<grid, TC_THREADS, tc_small_smem<T>(), st>>>(a, status);
    else oztc_tiled_kernel<T><<<grid, TC_THREADS, tc_smem<T>(), st>>>(a, status);
    mrc_prof_post(6, st, bytes, flops);
    return cudaGetLastError();
}
