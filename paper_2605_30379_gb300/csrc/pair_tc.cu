// pair_tc.cu -- per-frequency complex matrix products of the FFT-Newton path
// (Eq. (fft-convolution): C(phi) = X(phi) Y(phi) at every frequency of the
// half spectrum, square d x d with 32 <= d <= 64) as exact digit products on
// the tcgen05 tensor cores, for two working precisions:
//
//   double-float (the residual product of Proposition 2.6): six balanced
//     base-256 digits per value, digit pairs of weight s + t >= 5 (21 pairs
//     in 6 weight groups), about 2^-41 relative to the row and column bounds;
//   FP32 (the Newton-level products of Eq. (newton) and the correction):
//     four digits, pairs s + t >= 3 (10 pairs in 4 groups), about 2^-26
//     relative to the row and column bounds.  Three digits (6 pairs, about
//     2^-21) made the product 1.27x faster at d = 64, N = 2^18 but left
//     e_rel at 1.7e-9 after the sweep (gate 1e-10).
//
// The rows of X are scaled by 2^-sigma_i and the columns of Y by 2^-tau_j
// (powers of two from bounds over both frequencies of the pair) and every
// value v is split into S digits t_s, each a multiple of 2^(8s - 8S) of at
// most 8 significant bits (an exact BF16 value; digits.cuh's rounding steps,
// kept at their own scale).  Every digit pair of weight group g = s + t has
// the quantum 2^(8g - 16S), so all pairs of one group accumulate exactly in
// one FP32 accumulator in TMEM: a group holds at most 6 pairs of two 64-term
// dot products of digits <= 128 quanta each (below 2^24 quanta).  One MMA of
// M = 128, N = 64 forms [C_r; C_i] from the 192-row MN-major A tile
// [-X_i; X_r; X_i] of a digit: D += [X_r; X_i] Y_r (rows 64..191) and
// D += [-X_i; X_r] Y_i (rows 0..127).  The group sums add top group first.
//
// The kernels are persistent (one CTA per SM, pairs p = blockIdx.x, + grid,
// ...) and warp-specialised, with every hand-off on an mbarrier:
//   warps 0-7  (split): per frequency pair the row / column bounds, then per
//              K chunk of 16 the real-FFT split of the packed spectra (the
//              fused split of kernels.cuh) and the digit tiles, into a ring
//              of NSLOT chunk slots (full / empty barriers);
//   warp 12    (MMA): one thread issues every kept digit pair's MMAs of a
//              chunk and releases the slot with tcgen05.commit; after the
//              last chunk it signals the epilogue;
//   warps 8-11 (epilogue): tcgen05.ld of the group accumulators and the fold
//              (a compensated double-float sum of the top three groups for
//              the residual product, FP32 below and for FP32), then, through
//              a shared-memory transpose, the scaling by 2^(sigma + tau), the
//              real-FFT merge of the pair and coalesced stores.
// FP32 takes both frequencies of a pair at once: the split of f and M - f
// shares its loads and its twiddle product (2 Xh(M - f) = conj(s - t) where
// 2 Xh(f) = s + t), both accumulator sets fill the 512 TMEM columns
// (4 x 64 each), and the epilogue merges C(f) and C(M - f) directly.
// Double-float (6 x 64 columns per frequency) takes the two frequencies one
// after the other and keeps the unmerged C(f) in the output until C(M - f)
// is known.
//
// Every wait is bounded: a wait that gives up sets MRC_ERR_TIMEOUT (6) in the
// status word and a shared abort flag; all roles then leave their loops, the
// MMA thread waits (bounded) for its MMAs in flight, and the TMEM is freed.
#include "digits.cuh"
#include "tcgen05.cuh"

namespace {

using namespace mrc_digits;
using namespace mrc_tc;

// S digits, smallest group kept, ring slots, frequencies per pass (2: both
// of a pair at once)
template <class T> struct TcP;
// PF: pairs ahead whose spectra are prefetched into L2 (each pair's four
// rows X(f), X(M-f), Y(f), Y(M-f) are 4 E sizeof(cx<T>) bytes); with PF = 1
// the next pair's bounds would be gathered during the second half of the
// current pair's chunks, once the prefetch has landed.  Measured at d = 64,
// N = 2^18: FP32 two pairs ahead 39.2 -> 38.8 ms; double-float one pair
// ahead 41.4 -> 46.4 ms (256 KB per pair and SM crowd L2), so none.
template <> struct TcP<dd> { static constexpr int S = 6, GMIN = 5, NSLOT = 3, NF = 1, PF = 0; };
template <> struct TcP<float> { static constexpr int S = 4, GMIN = 3, NSLOT = 2, NF = 2, PF = 2; };

constexpr int KC = 16;                // K per chunk: one MMA K step
constexpr int NCH = 64 / KC;          // chunks per frequency
constexpr int SBO = (KC / 8) * 128;   // bytes between 8-row groups of a tile
constexpr int A_TILE = 192 * KC * 2;  // bytes of one [-X_i; X_r; X_i] digit tile
constexpr int B_TILE = 64 * KC * 2;   // bytes of one Y_r or Y_i digit tile
// 13 warps: 8 split, 4 epilogue (TMEM lane quarters 0..3), 1 MMA; at most
// four warps per SM sub-partition leaves each thread 128 registers
constexpr int NSPLIT = 256, NEPI = 128;
constexpr int WEPI0 = 8, WMMA = 12;
constexpr int NTHREADS = 13 * 32;
constexpr int XLD = 33;               // row length (values) of the epilogue transpose
constexpr unsigned TMEM_COLS = 512;
constexpr int BAR_SPLIT = 1, BAR_EPI = 2;
constexpr unsigned IDESC = idesc_bf16<128, 64>();

template <class T>
struct TcL {
    static constexpr int S = TcP<T>::S, GMIN = TcP<T>::GMIN, NG = 2 * (S - 1) - GMIN + 1;
    static constexpr int NSLOT = TcP<T>::NSLOT, NF = TcP<T>::NF, PF = TcP<T>::PF;
    static constexpr int SUB = S * (A_TILE + 2 * B_TILE);  // digit tiles of one frequency and chunk
    static constexpr int XT = S * A_TILE;                   // the X part of them (the sub-slot's start)
    static constexpr int SLOT = NF * SUB;
    static constexpr int XCH = 2 * NF * 64 * XLD * (int)sizeof(T);  // [NF][C_r, C_i][64][XLD]
    static constexpr int OFF_XCH = NSLOT * SLOT;
    // Per-pair scale factors scx[i] = 2^-sigma_i, scy[j] = 2^-tau_j (the
    // split) and fx[i] = 2^(sigma_i - 1), fy[j] = 2^(tau_j - 1) (the output:
    // fx fy = 2^(sigma + tau) / 4 undoes the scalings and the split's factor
    // 2 on both operands) in NB buffers by pair counter, then two bound
    // buffers bx[64], by[64] (a pair's, and the next pair's being gathered).
    // The split warps run at most NSLOT chunks ahead of the MMAs and those
    // at most one pass ahead of the epilogue, so the epilogue is fewer than
    // NB pairs behind the split.
    static constexpr int NB = 8;
    static constexpr int OFF_SC = OFF_XCH + XCH;
    static constexpr int SMEM = OFF_SC + (4 * NB + 4) * 64 * 4;
    static constexpr int TCOLS = NG * 64;  // TMEM columns of one frequency's groups
    static_assert(NF * TCOLS <= (int)TMEM_COLS, "accumulators fit in TMEM");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ int mn_off(int m, int k) { return (m >> 3) * SBO + (k >> 3) * 128 + (k & 7) * 16 + (m & 7) * 2; }
__device__ __forceinline__ int k_off(int n, int k) { return (n >> 3) * SBO + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2; }

// 2^e clamped to the normal float exponents
__device__ __forceinline__ float pow2c(int e) { return pow2f(max(-126, min(127, e))); }

// s and t of the real-FFT split (kernels.cuh: split_real without its factor
// 1/2) for packed values a = Z(f), b = Z(M - f), w = W_L^f: 2 Xh(f) = s + t
// and 2 Xh(M - f) = conj(s - t), with s = a + conj b, t = w (-i) (a - conj b).
template <class T>
__device__ __forceinline__ void split_st(cx<T> za, cx<T> zb, cx<T> w, cx<T> &s, cx<T> &t)
{
    s = {Ar<T>::add(za.re, zb.re), Ar<T>::sub(za.im, zb.im)};
    const cx<T> dlt = {Ar<T>::sub(za.re, zb.re), Ar<T>::add(za.im, zb.im)};
    t = c_mul(w, cx<T>{dlt.im, Ar<T>::neg(dlt.re)});
}

// Read-only loads as volatile inline PTX: issued where they stand
// (the compiler keeps volatile asm in order), so that the next chunk's
// values are in flight during the current chunk's digit work instead of
// being requested just before their use
template <class T>
__device__ __forceinline__ cx<T> ldv_cx(const cx<T> *p);
template <>
__device__ __forceinline__ cx<dd> ldv_cx<dd>(const cx<dd> *p)
{
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];\n" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return {{v.x, v.y}, {v.z, v.w}};
}
template <>
__device__ __forceinline__ cx<float> ldv_cx<float>(const cx<float> *p)
{
    float2 v;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return {v.x, v.y};
}

// High parts of one packed value (re, im): the bounds use them only
template <class T>
__device__ __forceinline__ float2 ldg_hi(const cx<T> *p);
template <>
__device__ __forceinline__ float2 ldg_hi<dd>(const cx<dd> *p)
{
    const float *q = reinterpret_cast<const float *>(p);
    return make_float2(__ldg(q), __ldg(q + 2));
}
template <>
__device__ __forceinline__ float2 ldg_hi<float>(const cx<float> *p)
{
    return __ldg(reinterpret_cast<const float2 *>(p));
}

// Bounds of a pair: row bounds bx[i] = max_k (|Z_X(f)_ik|_1 + |Z_X(M-f)_ik|_1)
// and column bounds by[j] = max_k (|Z_Y(f)_kj|_1 + |Z_Y(M-f)_kj|_1), which
// bound |Xh| and |Yh| at both frequencies entrywise.  Split thread t covers
// column t & 63 of rows (t >> 6) + 4 n, n = 0 .. 15, in slices of two n:
// bnd_issue loads a slice, bnd_reduce folds it into bx (a warp reduction, one
// shared atomic per row) and into the thread's running column maximum my.
struct BndIn {
    float2 xa[2], xb[2], ya[2], yb[2];
};

template <class T>
__device__ __forceinline__ void bnd_issue(BndIn &b, const cx<T> *ZX, const cx<T> *ZY, int64_t f, int64_t g, int d,
                                          int t, int n0)
{
    const int64_t E = (int64_t)d * d;
    const int k = t & 63;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int i = (t >> 6) + 4 * (n0 + u);
        const float2 z = make_float2(0.0f, 0.0f);
        b.xa[u] = b.xb[u] = b.ya[u] = b.yb[u] = z;
        if (i < d && k < d) {
            const int64_t e = (int64_t)i * d + k;
            b.xa[u] = ldg_hi(ZX + f * E + e);
            b.xb[u] = ldg_hi(ZX + g * E + e);
            b.ya[u] = ldg_hi(ZY + f * E + e);
            b.yb[u] = ldg_hi(ZY + g * E + e);
        }
    }
}

__device__ __forceinline__ void bnd_reduce(const BndIn &b, unsigned *bx, float &my, int t, int n0)
{
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int i = (t >> 6) + 4 * (n0 + u);  // one row per pair of warps
        const float mx = fabsf(b.xa[u].x) + fabsf(b.xa[u].y) + fabsf(b.xb[u].x) + fabsf(b.xb[u].y);
        my = fmaxf(my, fabsf(b.ya[u].x) + fabsf(b.ya[u].y) + fabsf(b.yb[u].x) + fabsf(b.yb[u].y));
        const unsigned wmx = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));  // nonnegative: bits order
        if ((t & 31) == 0) atomicMax(&bx[i], wmx);
    }
}

// The pair's scale factors from its bounds (2 Xh and 2 Yh are split: bound
// 2 |.|, scaled values <= 1/2)
__device__ __forceinline__ void bnd_scales(const unsigned *bx, const unsigned *by, float *sc, int d, int t)
{
    const int sx = t < d ? scale_exp(2.0f * __uint_as_float(bx[t])) : 0;
    const int sy = t < d ? scale_exp(2.0f * __uint_as_float(by[t])) : 0;
    sc[t] = t < d ? pow2c(-sx) : 0.0f;
    sc[64 + t] = t < d ? pow2c(-sy) : 0.0f;
    sc[128 + t] = pow2c(sx - 1);
    sc[192 + t] = pow2c(sy - 1);
}

// Raw packed-spectrum values of one chunk held by a split thread: X rows
// 4 i4 .. 4 i4 + 3 at column k0 + (t & 15); Y rows k0 + 4 k4 .. + 3 at
// column j = 8 (t / 32) + (t & 7), k4 = (t & 31) / 8; both rows ra and rb.
template <class T>
struct Raw {
    cx<T> xa[4], xb[4], ya[4], yb[4];
};

template <class T>
__device__ __forceinline__ void load_x(Raw<T> &r, const cx<T> *ZX, int64_t ra, int64_t rb, int d, int k0, int t)
{
    const int64_t E = (int64_t)d * d;
    const int k = k0 + (t & 15), i4 = t >> 4;
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
        const int i = 4 * i4 + ii;
        const bool ok = i < d && k < d;
        const int64_t e = (int64_t)i * d + k;
        r.xa[ii] = c_zero<T>();
        r.xb[ii] = c_zero<T>();
        if (ok) {
            r.xa[ii] = ldv_cx(ZX + ra * E + e);
            r.xb[ii] = ldv_cx(ZX + rb * E + e);
        }
    }
}

template <class T>
__device__ __forceinline__ void load_y(Raw<T> &r, const cx<T> *ZY, int64_t ra, int64_t rb, int d, int k0, int t)
{
    const int64_t E = (int64_t)d * d;
    const int lane = t & 31, j = 8 * (t >> 5) + (lane & 7), k4 = lane >> 3;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int k = k0 + 4 * k4 + kk;
        const bool ok = k < d && j < d;
        const int64_t e = (int64_t)k * d + j;
        r.ya[kk] = c_zero<T>();
        r.yb[kk] = c_zero<T>();
        if (ok) {
            r.ya[kk] = ldv_cx(ZY + ra * E + e);
            r.yb[kk] = ldv_cx(ZY + rb * E + e);
        }
    }
}

// Double-float digits value by value (the order the double-float split
// runs fastest in: d = 64, N = 2^18, pairmul_dd 40.6 ms against 51.7 ms in
// digit-major order): hi + lo into six digits on the grids 2^-8 .. 2^-48 by
// the rounding steps described below, lo joining through an exact TwoSum
// after the second digit and that sum's error after the fourth.
__device__ __forceinline__ void digits(dd v, float sc, float (&q)[6])
{
    float x = v.hi * sc, t;
    t = __fsub_rn(__fadd_rn(x, 49152.0f), 49152.0f);  // grid 2^-8
    q[5] = t;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 192.0f), 192.0f);      // grid 2^-16
    q[4] = t;
    x = __fsub_rn(x, t);
    const dd ye = dd_two_sum(x, v.lo * sc);           // exact: x + lo = y + e
    x = ye.hi;
    t = __fsub_rn(__fadd_rn(x, 0.75f), 0.75f);        // grid 2^-24
    q[3] = t;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 0x1.8p-9f), 0x1.8p-9f);  // grid 2^-32
    q[2] = t;
    x = __fadd_rn(__fsub_rn(x, t), ye.lo);
    t = __fsub_rn(__fadd_rn(x, 0x1.8p-17f), 0x1.8p-17f);  // grid 2^-40
    q[1] = t;
    x = __fsub_rn(x, t);
    q[0] = __fsub_rn(__fadd_rn(x, 0x1.8p-25f), 0x1.8p-25f);  // grid 2^-48
}
// Packed BF16 digits of 4 values (two uint per digit and component) of one
// frequency: v[n] = 2 Xh or 2 Yh, scaled by sc[n]
template <class T, int S>
__device__ __forceinline__ void pack4(const cx<T> (&v)[4], const float (&sc)[4], unsigned (&wr)[S][2],
                                      unsigned (&wi)[S][2])
{
    float pr[S], pi[S];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        float qr[S], qi[S];
        digits(v[n].re, sc[n], qr);
        digits(v[n].im, sc[n], qi);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (n & 1) {
                wr[s][n >> 1] = pack2(pr[s], qr[s]);
                wi[s][n >> 1] = pack2(pi[s], qi[s]);
            } else {
                pr[s] = qr[s];
                pi[s] = qi[s];
            }
        }
    }
}

// digit tiles of X for one frequency's sub-slot: per digit, 8 bytes (4
// consecutive rows) into each of the blocks -X_i (rows 0..63), X_r
// (64..127), X_i (128..191)
template <int S>
__device__ __forceinline__ void store_x(unsigned char *sub, const unsigned (&wr)[S][2], const unsigned (&wi)[S][2],
                                        int t)
{
    const int k = t & 15, i4 = t >> 4;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        unsigned char *tl = sub + s * A_TILE;
        *reinterpret_cast<uint2 *>(tl + mn_off(4 * i4, k)) = make_uint2(wi[s][0] ^ 0x80008000u, wi[s][1] ^ 0x80008000u);
        *reinterpret_cast<uint2 *>(tl + mn_off(64 + 4 * i4, k)) = make_uint2(wr[s][0], wr[s][1]);
        *reinterpret_cast<uint2 *>(tl + mn_off(128 + 4 * i4, k)) = make_uint2(wi[s][0], wi[s][1]);
    }
}

// digit tiles of Y_r and Y_i (K-major, row n = j): 8 bytes of 4 consecutive k per digit
template <int S>
__device__ __forceinline__ void store_y(unsigned char *sub, const unsigned (&wr)[S][2], const unsigned (&wi)[S][2],
                                        int t)
{
    const int lane = t & 31, j = 8 * (t >> 5) + (lane & 7), k4 = lane >> 3;
    unsigned char *br = sub + S * A_TILE, *bi = br + S * B_TILE;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        *reinterpret_cast<uint2 *>(br + s * B_TILE + k_off(j, 4 * k4)) = make_uint2(wr[s][0], wr[s][1]);
        *reinterpret_cast<uint2 *>(bi + s * B_TILE + k_off(j, 4 * k4)) = make_uint2(wi[s][0], wi[s][1]);
    }
}

// Balanced digits at their own scale: t = (x + C) - C with C = 1.5 * 2^k
// rounds x to the nearest multiple of 2^(k-23) and x - t is exact, so digit
// s of a value |v| <= 1/2 is a multiple of 2^(8s - 8S) within 128 of its
// quanta (digits.cuh).  FP32 takes four digits on the grids 2^-8 .. 2^-32 in
// digit-major order: the running remainders of all values a split thread
// holds advance one digit at a time together, and each digit is packed and
// stored as soon as it exists (pairmul_f32 38.3 -> 37.7 ms at d = 64,
// N = 2^18 against value by value).
template <class T> struct DState;
template <> struct DState<float> { float x; };
__device__ __forceinline__ DState<float> dstart(float v, float sc) { return {v * sc}; }

constexpr float pow2_ce(int e) { return e >= 0 ? (e == 0 ? 1.0f : 2.0f * pow2_ce(e - 1)) : 0.5f * pow2_ce(e + 1); }

// digit s (grid 2^(8s - 8S)) of the state; the remainder moves on
template <int S, int s>
__device__ __forceinline__ float dstep(DState<float> &st)
{
    constexpr float C = 1.5f * pow2_ce(8 * (s - S) + 23);
    const float t = __fsub_rn(__fadd_rn(st.x, C), C);
    if constexpr (s > 0) st.x = __fsub_rn(st.x, t);
    return t;
}
// X digit tiles of the chunk: per frequency fq of the pass and digit, 8
// bytes (4 consecutive rows) into each of the blocks -X_i (rows 0..63), X_r
// (64..127), X_i (128..191) of sub-slot fq
template <class T, int NFQ, int s>
__device__ __forceinline__ void xdigit(DState<T> (&st)[NFQ][4][2], unsigned char *slot, int off_n, int off_r, int off_p)
{
    using L = TcL<T>;
#pragma unroll
    for (int fq = 0; fq < NFQ; ++fq) {
        float q[4][2];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            q[n][0] = dstep<L::S, s>(st[fq][n][0]);
            q[n][1] = dstep<L::S, s>(st[fq][n][1]);
        }
        const unsigned r0 = pack2(q[0][0], q[1][0]), r1 = pack2(q[2][0], q[3][0]);
        const unsigned i0 = pack2(q[0][1], q[1][1]), i1 = pack2(q[2][1], q[3][1]);
        unsigned char *tl = slot + fq * L::SUB + s * A_TILE;
        *reinterpret_cast<uint2 *>(tl + off_n) = make_uint2(i0 ^ 0x80008000u, i1 ^ 0x80008000u);
        *reinterpret_cast<uint2 *>(tl + off_r) = make_uint2(r0, r1);
        *reinterpret_cast<uint2 *>(tl + off_p) = make_uint2(i0, i1);
    }
}

// Y_r and Y_i digit tiles (K-major, row n = j): 8 bytes of 4 consecutive k per digit
template <class T, int NFQ, int s>
__device__ __forceinline__ void ydigit(DState<T> (&st)[NFQ][4][2], unsigned char *slot, int off)
{
    using L = TcL<T>;
#pragma unroll
    for (int fq = 0; fq < NFQ; ++fq) {
        float q[4][2];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            q[n][0] = dstep<L::S, s>(st[fq][n][0]);
            q[n][1] = dstep<L::S, s>(st[fq][n][1]);
        }
        unsigned char *br = slot + fq * L::SUB + L::S * A_TILE + s * B_TILE;
        *reinterpret_cast<uint2 *>(br + off) = make_uint2(pack2(q[0][0], q[1][0]), pack2(q[2][0], q[3][0]));
        *reinterpret_cast<uint2 *>(br + L::S * B_TILE + off) = make_uint2(pack2(q[0][1], q[1][1]), pack2(q[2][1], q[3][1]));
    }
}

template <class T, int NFQ, int... s>
__device__ __forceinline__ void xdigits(DState<T> (&st)[NFQ][4][2], unsigned char *slot, int on, int orr, int op,
                                        std::integer_sequence<int, s...>)
{
    (xdigit<T, NFQ, TcL<T>::S - 1 - s>(st, slot, on, orr, op), ...);
}
template <class T, int NFQ, int... s>
__device__ __forceinline__ void ydigits(DState<T> (&st)[NFQ][4][2], unsigned char *slot, int off,
                                        std::integer_sequence<int, s...>)
{
    (ydigit<T, NFQ, TcL<T>::S - 1 - s>(st, slot, off), ...);
}

// The split of one chunk into the slot.  NF == 1: the frequency with
// twiddle w of the raw rows (ra, rb); NF == 2: f (sub-slot 0) and M - f (1).
template <class T>
__device__ __forceinline__ void split_chunk_x(const Raw<T> &r, unsigned char *slot, const float *scx, cx<T> w, int t)
{
    using L = TcL<T>;
    constexpr int NF = L::NF;
    const int k = t & 15, i4 = t >> 4;
    if constexpr (__is_same(T, dd)) {  // value by value
        float sc[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) sc[n] = scx[4 * i4 + n];
        cx<T> vf[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            cx<T> s, tt;
            split_st(r.xa[n], r.xb[n], w, s, tt);
            vf[n] = c_add(s, tt);
        }
        unsigned wr[L::S][2], wi[L::S][2];
        pack4<T, L::S>(vf, sc, wr, wi);
        store_x<L::S>(slot, wr, wi, t);
    } else {  // digit-major
        DState<T> st[NF][4][2];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            const float sc = scx[4 * i4 + n];
            cx<T> s, tt;
            split_st(r.xa[n], r.xb[n], w, s, tt);
            const cx<T> vf = c_add(s, tt);
            st[0][n][0] = dstart(vf.re, sc);
            st[0][n][1] = dstart(vf.im, sc);
            if constexpr (NF == 2) {
                st[NF - 1][n][0] = dstart(Ar<T>::sub(s.re, tt.re), sc);
                st[NF - 1][n][1] = dstart(Ar<T>::sub(tt.im, s.im), sc);
            }
        }
        xdigits<T, NF>(st, slot, mn_off(4 * i4, k), mn_off(64 + 4 * i4, k), mn_off(128 + 4 * i4, k),
                       std::make_integer_sequence<int, L::S>{});
    }
}

template <class T>
__device__ __forceinline__ void split_chunk_y(const Raw<T> &r, unsigned char *slot, const float *scy, cx<T> w, int t)
{
    using L = TcL<T>;
    constexpr int NF = L::NF;
    const int lane = t & 31, j = 8 * (t >> 5) + (lane & 7), k4 = lane >> 3;
    const float sc = scy[j];
    if constexpr (__is_same(T, dd)) {  // value by value
        const float scv[4] = {sc, sc, sc, sc};
        cx<T> vf[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            cx<T> s, tt;
            split_st(r.ya[n], r.yb[n], w, s, tt);
            vf[n] = c_add(s, tt);
        }
        unsigned wr[L::S][2], wi[L::S][2];
        pack4<T, L::S>(vf, scv, wr, wi);
        store_y<L::S>(slot, wr, wi, t);
    } else {  // digit-major
        DState<T> st[NF][4][2];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            cx<T> s, tt;
            split_st(r.ya[n], r.yb[n], w, s, tt);
            const cx<T> vf = c_add(s, tt);
            st[0][n][0] = dstart(vf.re, sc);
            st[0][n][1] = dstart(vf.im, sc);
            if constexpr (NF == 2) {
                st[NF - 1][n][0] = dstart(Ar<T>::sub(s.re, tt.re), sc);
                st[NF - 1][n][1] = dstart(Ar<T>::sub(tt.im, s.im), sc);
            }
        }
        ydigits<T, NF>(st, slot, k_off(j, 4 * k4), std::make_integer_sequence<int, L::S>{});
    }
}

// value + v for a float v: one TwoSum of the high parts, lo parts added once
__device__ __forceinline__ dd add_f(dd a, float v)
{
    const dd s = dd_two_sum(a.hi, v);
    return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// Fold the NG group accumulators of TMEM lanes 32 q + lane, columns
// col .. col + 7 (every group sum an exact FP32 value at its own scale), top
// group first.  Double-float: the top three groups as a compensated sum, the
// groups below (2^-24 and less of the top one) in FP32, joining once; FP32:
// plain FP32 adds.
template <class T, int NG>
__device__ __forceinline__ void fold8(unsigned tbase, T (&out)[8])
{
    float lo[8];
#pragma unroll
    for (int g = NG - 1; g >= 0; --g) {
        unsigned r[8];
        ld8(tbase + (unsigned)(g * 64), r);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float v = __uint_as_float(r[c]);
            if constexpr (__is_same(T, dd)) {
                if (g == NG - 1) out[c] = dd{v, 0.0f};
                else if (g >= NG - 3) out[c] = add_f(out[c], v);
                else if (g == NG - 4) lo[c] = v;
                else lo[c] = __fadd_rn(lo[c], v);
            } else {
                if (g == NG - 1) out[c] = v;
                else out[c] = __fadd_rn(out[c], v);
            }
        }
    }
    if constexpr (__is_same(T, dd) && NG > 3) {
#pragma unroll
        for (int c = 0; c < 8; ++c) out[c] = add_f(out[c], lo[c]);
    }
}

__device__ __forceinline__ dd mul_f(dd x, float f) { return {x.hi * f, x.lo * f}; }
__device__ __forceinline__ float mul_f(float x, float f) { return x * f; }

template <class T>
__device__ __forceinline__ void st_cx(cx<T> *p, cx<T> v);
template <>
__device__ __forceinline__ void st_cx<dd>(cx<dd> *p, cx<dd> v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo);
}
template <>
__device__ __forceinline__ void st_cx<float>(cx<float> *p, cx<float> v)
{
    *reinterpret_cast<float2 *>(p) = make_float2(v.re, v.im);
}

// P: the products of one launch, all of M points (a single one, or every
// model of a batch at one stage); global pair gp is pair gp % npairs of
// product gp / npairs.  NCK: the K chunks of KC per frequency, ceil(d / KC)
// for every product of the launch (the chunks that hold k < d; d = 48 runs 3
// of 4).  With the chunk count a run-time value the double-float product took
// 46.9 ms at d = 64, N = 2^18 against 41.4.
// XPRE (double-float): X's digit tiles and row scales were prepared once
// (tcp_prep_kernel: X is the spectrum of A, the same in every residual
// sweep); the split warps bulk-copy them into the slot (on xfull[slot]) and
// split only Y.
template <class T, int NCK, bool XPRE>
__global__ void __launch_bounds__(NTHREADS, 1) tcp_kernel(const __grid_constant__ SegParams<PairArgs> P, int *status)
{
    using L = TcL<T>;
    constexpr int S = L::S, GMIN = L::GMIN, NG = L::NG, NSLOT = L::NSLOT, NF = L::NF;
    extern __shared__ __align__(1024) unsigned char smem[];
    T *xch = reinterpret_cast<T *>(smem + L::OFF_XCH);          // [NF][C_r, C_i][64][XLD]
    float *scb = reinterpret_cast<float *>(smem + L::OFF_SC);  // [NB][scx, scy, fx, fy][64]
    unsigned *bxy = reinterpret_cast<unsigned *>(scb + 4 * 64 * L::NB);  // [2][bx, by][64]
    __shared__ __align__(8) unsigned long long bar_full[NSLOT], bar_empty[NSLOT], bar_tfull, bar_tempty, bar_done;
    __shared__ __align__(8) unsigned long long bar_xfull[NSLOT];  // XPRE: the slot's X tiles landed
    __shared__ unsigned tslot;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) {
            mbar_init(smem_u32(&bar_full[s]), NSPLIT);
            mbar_init(smem_u32(&bar_empty[s]), 1);
            mbar_init(smem_u32(&bar_xfull[s]), 1);
        }
        mbar_init(smem_u32(&bar_tfull), 1);
        mbar_init(smem_u32(&bar_tempty), NEPI);
        mbar_init(smem_u32(&bar_done), 1);
        abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == WMMA) tmem_alloc(smem_u32(&tslot), TMEM_COLS);
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = tslot;

    const PairArgs &a = P.a[0];  // M, twiddles: common to the launch
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw);
    const int64_t M = a.M;
    // pair indices in 32 bits (a launch holds fewer than 2^32 pairs)
    const unsigned npairs = (unsigned)a.npairs, total = npairs * (unsigned)P.nseg;
    // product sg's spectra, output and d, read from the parameter block at
    // each use (no registers held across the chunk loop)
    auto zx_of = [&](int sg) { return reinterpret_cast<const cx<T> *>(P.a[sg].zx); };
    auto zy_of = [&](int sg) { return reinterpret_cast<const cx<T> *>(P.a[sg].zy); };
    auto zc_of = [&](int sg) { return reinterpret_cast<cx<T> *>(P.a[sg].zc); };
    auto d_of = [&](int sg) { return P.a[sg].r; };
    // the spectrum the X bounds come from: X's own, or (XPRE: X's scales are
    // prepared) Y's again, whose X half of the bounds is then replaced
    auto bx_of = [&](int sg) { return XPRE ? zy_of(sg) : zx_of(sg); };
    auto xs_of = [&](int sg) { return reinterpret_cast<const float *>(P.a[sg].xs); };
    constexpr int nck = NCK;
    bool failed = false;
    auto give_up = [&]() {
        failed = true;
        abort_flag = 1;
        if (status) atomicExch(status, 6);
    };
    // passes of pair p: its frequencies one at a time (NF == 1; one for the
    // self-paired p = M/2), or both at once (NF == 2)
    auto npass = [&](int64_t p) { return NF == 2 ? 1 : (((M - p) == p) ? 1 : 2); };

    if (warp < WEPI0) {
        // ------------------------------------------------------------ split
        // The bounds of pair p + grid are gathered during pair p's chunks, in
        // slices (their loads, first touches of those spectra, overlap the
        // digit work); the first pair's before its chunks.
        const int t = tid;
        int it = 0;  // chunk counter: slot it % NSLOT, use it / NSLOT
        int pl = 0;  // pair counter (mod NB selects the scale buffers)
        Raw<T> raw;
        BndIn bi;
        // the four spectrum rows of pair q into L2, one bulk prefetch per row
        // over its 16-byte aligned interior (a bulk copy must start on a
        // 16-byte boundary and span a multiple of 16 bytes; FP32 rows of odd
        // E start and end on 8-byte ones), so it never leaves the row
        auto prefetch_pair = [&](unsigned gq) {
            if (t < 4 && gq < total) {
                const int sq = (int)(gq / npairs);
                const int64_t q = gq - (unsigned)sq * npairs, E = (int64_t)d_of(sq) * d_of(sq);
                const int64_t r = (t & 1) ? ((M - q) & (M - 1)) : q;
                const uintptr_t b0 = (uintptr_t)((t < 2 ? zx_of(sq) : zy_of(sq)) + r * E);
                const uintptr_t lo = (b0 + 15) & ~(uintptr_t)15, hi = (b0 + E * sizeof(cx<T>)) & ~(uintptr_t)15;
                if (hi > lo) prefetch_l2((const void *)lo, (unsigned)(hi - lo));
            }
        };
        for (int k = 1; k < L::PF; ++k) prefetch_pair(blockIdx.x + (unsigned)k * gridDim.x);
        bxy[t] = 0u;  // both bound buffers (256 threads, 256 words)
        bar_sync(BAR_SPLIT, NSPLIT);
        if (blockIdx.x < total) {
            const int s0 = (int)(blockIdx.x / npairs);
            const int64_t f = blockIdx.x - (unsigned)s0 * npairs, gZ = (M - f) & (M - 1);
            float my = 0.0f;
            for (int n0 = 0; n0 < 4 * nck; n0 += 2) {
                bnd_issue(bi, bx_of(s0), zy_of(s0), f, gZ, d_of(s0), t, n0);
                bnd_reduce(bi, bxy, my, t, n0);
            }
            atomicMax(&bxy[64 + (t & 63)], __float_as_uint(my));
        }
        bar_sync(BAR_SPLIT, NSPLIT);
        if (t < 64 && blockIdx.x < total) {
            const int s0 = (int)(blockIdx.x / npairs);
            bnd_scales(bxy, bxy + 64, scb, d_of(s0), t);
            if (XPRE) scb[128 + t] = xs_of(s0)[(int64_t)(blockIdx.x - (unsigned)s0 * npairs) * 128 + 64 + t];
        }
        bar_sync(BAR_SPLIT, NSPLIT);
        unsigned nx = 0;  // XPRE: X tile copies issued (chunk it's copy goes to slot it % NSLOT)
        for (unsigned gp = blockIdx.x; gp < total; gp += gridDim.x, ++pl) {
            const int sg = (int)(gp / npairs);
            const int64_t p = gp - (unsigned)sg * npairs, f = p, gZ = (M - p) & (M - 1);
            const cx<T> wf = tw[f << (a.tw_log - a.logM - 1)];
            const cx<T> wg = c_neg(c_conj(wf));
            const float *sc = scb + 4 * 64 * (pl % L::NB);
            const unsigned gpn = gp + gridDim.x;
            const bool next = gpn < total;
            const int sn = next ? (int)(gpn / npairs) : sg;
            const int64_t pn = gpn - (unsigned)sn * npairs, fn = pn, gn = (M - pn) & (M - 1);
            unsigned *bn = bxy + 128 * ((pl + 1) & 1);  // the next pair's bounds
            float myn = 0.0f;
            const int nch = npass(p) * nck;
            const int cb = L::PF == 1 ? nch / 2 : 0;  // first chunk that gathers the next pair's bounds
            if (L::PF > 0) prefetch_pair(gp + (unsigned)L::PF * gridDim.x);
            // bound rows n per gathering chunk (2, 4 or 8): the 4 nck row steps that cover
            // k < d over the nch - cb gathering chunks (nck per pass, half of them with PF = 1)
            const int ns = (L::PF == 1 ? 8 : 4) >> (npass(p) - 1);
            if (!XPRE) load_x(raw, zx_of(sg), f, gZ, d_of(sg), 0, t);
            load_y(raw, zy_of(sg), f, gZ, d_of(sg), 0, t);
            for (int c = 0; c < nch; ++c, ++it) {
                const cx<T> w = c < nck ? wf : wg;
                const int slot = it % NSLOT, use = it / NSLOT;
                unsigned char *sp = smem + slot * L::SLOT;
                // bound slices of the next pair (in L2 by now): rows n0 .. n0 + ns - 1,
                // two at a time, loads issued before the digit work they overlap
                const bool gather = next && c >= cb;
                const int n0 = (c - cb) * ns;
                if (!failed && use > 0 && (abort_flag || !mbar_wait(smem_u32(&bar_empty[slot]), (use - 1) & 1)))
                    give_up();
                const int cn = c + 1;  // next chunk of this pair: the first pass while cn < nck
                const bool first = cn < nck;
                const int64_t na = first ? f : gZ, nb = first ? gZ : f;
                const int kn = (first ? cn : cn - nck) * KC;
                if (gather) bnd_issue(bi, bx_of(sn), zy_of(sn), fn, gn, d_of(sn), t, n0);
                if constexpr (XPRE) {
                    if (t == 0 && !failed) {  // X tiles of this chunk: pass c / nck, chunk c % nck
                        const int ps = c < nck ? 0 : 1, cc = c - ps * nck;
                        const unsigned char *src = reinterpret_cast<const unsigned char *>(P.a[sg].zx) +
                                                   ((size_t)(p * 2 + ps) * NCK + cc) * (size_t)L::XT;
                        mbar_arrive_expect_tx(smem_u32(&bar_xfull[slot]), L::XT);
                        bulk_g2s(smem_u32(sp), src, L::XT, smem_u32(&bar_xfull[slot]));
                        ++nx;
                    }
                } else {
                    if (!failed) split_chunk_x<T>(raw, sp, sc, w, t);
                    if (cn < nch) load_x(raw, zx_of(sg), na, nb, d_of(sg), kn, t);
                }
                asm volatile("" ::: "memory");  // the loads above stay ahead of the Y digit stores
                if (gather) {
                    bnd_reduce(bi, bn, myn, t, n0);
                    for (int u = 2; u < ns - 2; u += 2) {
                        bnd_issue(bi, bx_of(sn), zy_of(sn), fn, gn, d_of(sn), t, n0 + u);
                        bnd_reduce(bi, bn, myn, t, n0 + u);
                    }
                    if (ns > 2) bnd_issue(bi, bx_of(sn), zy_of(sn), fn, gn, d_of(sn), t, n0 + ns - 2);
                }
                if (!failed) split_chunk_y<T>(raw, sp, sc + 64, w, t);
                if (cn < nch) load_y(raw, zy_of(sg), na, nb, d_of(sg), kn, t);
                asm volatile("" ::: "memory");
                if (gather && ns > 2) bnd_reduce(bi, bn, myn, t, n0 + ns - 2);
                if (!failed) {
                    fence_async_smem();  // digit tiles visible to the tensor cores
                    mbar_arrive(smem_u32(&bar_full[slot]));
                }
            }
            if (next) atomicMax(&bn[64 + (t & 63)], __float_as_uint(myn));
            if (bar_or(BAR_SPLIT, NSPLIT, failed || abort_flag)) break;  // the next pair's bounds complete
            if (next && t < 64) {
                float *scn = scb + 4 * 64 * ((pl + 1) % L::NB);
                bnd_scales(bn, bn + 64, scn, d_of(sn), t);
                if (XPRE) scn[128 + t] = xs_of(sn)[pn * 128 + 64 + t];
            }
            if (t < 128) bxy[128 * (pl & 1) + t] = 0u;  // this pair's buffer: free for pair p + 2 grid
            bar_sync(BAR_SPLIT, NSPLIT);
        }
        if (XPRE && t == 0) {
            // every X tile copy has landed before the CTA may exit (bounded waits)
            for (int sl = 0; sl < NSLOT; ++sl)
                if (nx > (unsigned)sl && !mbar_wait(smem_u32(&bar_xfull[sl]), ((nx - 1 - sl) / NSLOT) & 1)) give_up();
        }
    } else if (warp < WMMA) {
        // --------------------------------------------------------- epilogue
        const int et = tid - WEPI0 * 32;
        const int q = warp & 3;  // TMEM lanes 32 q .. 32 q + 31
        int fi = 0, pl = 0;      // passes drained, pairs
        for (unsigned gp = blockIdx.x; gp < total; gp += gridDim.x, ++pl) {
            const int sg = (int)(gp / npairs);
            const int64_t p = gp - (unsigned)sg * npairs, f = p, gZ = (M - p) & (M - 1);
            cx<T> *ZC = zc_of(sg);
            const int d = d_of(sg);
            const int64_t E = (int64_t)d * d;
            const int np = npass(p);
            const bool self = (M - p) == p;  // p = M/2 pairs with itself
            const bool two = (gZ != f);
            const cx<T> wf = tw[f << (a.tw_log - a.logM - 1)];
            const cx<T> wg = c_neg(c_conj(wf));
            const float *fx = scb + 4 * 64 * (pl % L::NB) + 128, *fy = fx + 64;
            bool stop = false;
            for (int phase = 0; phase < np; ++phase, ++fi) {
                bool ok = !failed && !abort_flag && mbar_wait(smem_u32(&bar_tfull), fi & 1);
                if (bar_or(BAR_EPI, NEPI, !ok)) {
                    if (!failed) give_up();
                    stop = true;
                    break;
                }
                fence_after();
                const unsigned tb = tmem + ((unsigned)(32 * q) << 16);
                // two rounds of 32 columns: fold them into the transpose (lanes
                // along i), release the accumulators after the second fold, then
                // lanes along j for coalesced global accesses
#pragma unroll 1
                for (int r = 0; r < 2; ++r) {
#pragma unroll
                    for (int fq = 0; fq < NF; ++fq) {
                        T *xr = xch + ((fq * 2 + (q >> 1)) * 64 + 32 * (q & 1) + lane) * XLD;  // C_r or C_i rows
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            T o8[8];
                            fold8<T, NG>(tb + (unsigned)(fq * L::TCOLS + 32 * r + 8 * m), o8);
#pragma unroll
                            for (int c = 0; c < 8; ++c) xr[8 * m + c] = o8[c];
                        }
                    }
                    if (r == 1) {
                        fence_before();
                        mbar_arrive(smem_u32(&bar_tempty));  // accumulators read: the next MMAs may overwrite them
                    }
                    bar_sync(BAR_EPI, NEPI);
                    const int jl = et & 31, j = 32 * r + jl;
                    const float sj = fy[j];
                    // four outputs at a time, their loads first
#pragma unroll 1
                    for (int m0 = 0; m0 < 16; m0 += 4) {
                        cx<T> v[4], vg[4], cf[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int i = (et >> 5) + 4 * (m0 + u);
                            const float s_ = fx[i] * sj;  // 2^(sigma_i + tau_j - 2), exact
                            v[u] = {mul_f(xch[i * XLD + jl], s_), mul_f(xch[(64 + i) * XLD + jl], s_)};
                            if constexpr (NF == 2)
                                vg[u] = {mul_f(xch[(128 + i) * XLD + jl], s_), mul_f(xch[(192 + i) * XLD + jl], s_)};
                            else if (phase == 1 && i < d && j < d)
                                cf[u] = ZC[f * E + (int64_t)i * d + j];  // C(f), stored unmerged by this thread
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int i = (et >> 5) + 4 * (m0 + u);
                            if (i >= d || j >= d) continue;
                            cx<T> *zf = ZC + f * E + (int64_t)i * d + j;
                            if constexpr (NF == 2) {
                                st_cx(zf, merge_real(v[u], vg[u], c_conj(wf)));
                                if (two) st_cx(ZC + gZ * E + (int64_t)i * d + j, merge_real(vg[u], v[u], c_conj(wg)));
                            } else if (self) {
                                st_cx(zf, merge_real(v[u], v[u], c_conj(wf)));  // C(M - f) = C(f)
                            } else if (phase == 0) {
                                st_cx(zf, v[u]);  // C(f), merged once C(M - f) is known
                            } else {
                                st_cx(zf, merge_real(cf[u], v[u], c_conj(wf)));
                                if (two) st_cx(ZC + gZ * E + (int64_t)i * d + j, merge_real(v[u], cf[u], c_conj(wg)));
                            }
                        }
                    }
                    bar_sync(BAR_EPI, NEPI);  // transpose read before it is rewritten
                }
            }
            if (stop) break;
        }
    } else if (lane == 0) {  // the MMA warp's other lanes go straight to the final barrier (below)
        // -------------------------------------------------------------- MMA
        int it = 0, fi = 0;
        bool issued = false;
        for (unsigned gp = blockIdx.x; gp < total && !failed; gp += gridDim.x) {
            const int np = npass(gp % npairs);
            for (int phase = 0; phase < np && !failed; ++phase, ++fi) {
                if (fi > 0 && (abort_flag || !mbar_wait(smem_u32(&bar_tempty), (fi - 1) & 1))) {
                    give_up();
                    break;
                }
                fence_after();
                for (int c = 0; c < nck; ++c, ++it) {
                    const int slot = it % NSLOT, use = it / NSLOT;
                    if (abort_flag || !mbar_wait(smem_u32(&bar_full[slot]), use & 1) ||
                        (XPRE && !mbar_wait(smem_u32(&bar_xfull[slot]), use & 1))) {
                        give_up();
                        break;
                    }
                    fence_after();
#pragma unroll
                    for (int fq = 0; fq < NF; ++fq) {
                        const unsigned sa = smem_u32(smem + slot * L::SLOT + fq * L::SUB);
                        const unsigned sbr = sa + S * A_TILE, sbi = sbr + S * B_TILE;
                        const unsigned dbase = tmem + (unsigned)(fq * L::TCOLS);
#pragma unroll
                        for (int g = GMIN; g <= 2 * (S - 1); ++g) {
                            const unsigned dcol = dbase + (unsigned)(g - GMIN) * 64u;
                            unsigned acc = c == 0 ? 0u : 1u;
#pragma unroll
                            for (int s = (g - (S - 1) > 0 ? g - (S - 1) : 0); s <= (g < S - 1 ? g : S - 1); ++s) {
                                const int tt = g - s;
                                const unsigned as = sa + s * A_TILE;
                                mma<IDESC>(dcol, desc<SBO>(as + 8 * SBO), desc<SBO>(sbr + tt * B_TILE), acc);
                                acc = 1u;
                                mma<IDESC>(dcol, desc<SBO>(as), desc<SBO>(sbi + tt * B_TILE), 1u);
                            }
                        }
                    }
                    issued = true;
                    commit(smem_u32(&bar_empty[slot]));  // the slot is free once these MMAs completed
                }
                if (failed) break;
                commit(smem_u32(&bar_tfull));  // the pass's accumulators are complete
            }
        }
        if (issued) {
            commit(smem_u32(&bar_done));
            if (!mbar_wait(smem_u32(&bar_done), 0)) give_up();  // every MMA finished before the TMEM is freed
        }
    }
    if (warp == WMMA) __syncwarp();  // lane 0 rejoins its warp before the CTA-wide barrier

    fence_before();
    __syncthreads();
    if (warp == WMMA) {
        fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

int sm_count()
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    return nsm;
}

template <class T>
using TcpKernel = void (*)(SegParams<PairArgs>, int *);
template <class T, bool XPRE>
TcpKernel<T> tcp_kernel_for(int nck)
{
    return nck <= 2 ? tcp_kernel<T, 2, XPRE> : (nck == 3 ? tcp_kernel<T, 3, XPRE> : tcp_kernel<T, 4, XPRE>);
}

template <class T>
cudaError_t tcp_launch(const SegParams<PairArgs> &P, int *status, cudaStream_t st, int kclass)
{
    if (P.nseg <= 0) return cudaSuccess;
    const int64_t total = P.a[0].npairs * P.nseg;
    const unsigned grid = (unsigned)std::min<int64_t>(total, sm_count());
    double bytes = 0, flops = 0;
    for (int s = 0; s < P.nseg; ++s) {
        const double d = P.a[s].r, M = (double)P.a[s].M;
        bytes += M * 3.0 * d * d * sizeof(cx<T>);
        flops += 8.0 * d * d * d * (M + 1);
    }
    const int nck = (P.a[0].r + KC - 1) / KC;
    TcpKernel<T> k = tcp_kernel_for<T, false>(nck);
    if constexpr (__is_same(T, dd))
        if (P.a[0].xs) k = tcp_kernel_for<T, true>(nck);
    mrc_prof_pre(kclass, st);
    k<<<grid, NTHREADS, TcL<T>::SMEM, st>>>(P, status);
    mrc_prof_post(kclass, st, bytes, flops);
    return cudaGetLastError();
}

// The double-float X operand prepared once: for every pair of every product
// of P (zx: X's packed spectrum; zc: the tiles out; xs: the scales out), its
// row scales (xs[p][0..63] = 2^-sigma_i for the split, [64..127] =
// 2^(sigma_i - 1) for the output, from the same bounds as the product's) and
// per pass and chunk the X digit tiles exactly as the split warps would
// leave them in a slot.  One CTA per pair: the bounds and each chunk's raw
// rows are read once for both passes (the second pass swaps the two rows and
// takes the partner twiddle); one staging sub-slot in shared memory.
template <int NCK>
__global__ void __launch_bounds__(NSPLIT) tcp_prep_kernel(const __grid_constant__ SegParams<PairArgs> P)
{
    using L = TcL<dd>;
    extern __shared__ __align__(1024) unsigned char stage[];  // [XT]
    __shared__ unsigned bxy[128];
    __shared__ float scb[256];
    const PairArgs &a = P.a[0];
    const int64_t M = a.M;
    const unsigned npairs = (unsigned)a.npairs, gp = blockIdx.x;
    const int t = threadIdx.x;
    const int sg = (int)(gp / npairs);
    const int64_t p = gp - (unsigned)sg * npairs, f = p, gZ = (M - p) & (M - 1);
    const int np = (M - p) == p ? 1 : 2;  // the self-paired frequency has one pass
    const PairArgs &as = P.a[sg];
    const cx<dd> *ZX = reinterpret_cast<const cx<dd> *>(as.zx);
    const int d = as.r;
    if (t < 128) bxy[t] = 0u;
    __syncthreads();
    BndIn bi;
    float my = 0.0f;
    for (int n0 = 0; n0 < 4 * NCK; n0 += 2) {
        bnd_issue(bi, ZX, ZX, f, gZ, d, t, n0);
        bnd_reduce(bi, bxy, my, t, n0);
    }
    __syncthreads();
    if (t < 64) bnd_scales(bxy, bxy + 64, scb, d, t);  // bxy + 64: unused column bounds
    __syncthreads();
    if (t < 64) {
        float *xs = reinterpret_cast<float *>(const_cast<void *>(as.xs)) + p * 128;
        xs[t] = scb[t];
        xs[64 + t] = scb[128 + t];
    }
    const cx<dd> *tw = reinterpret_cast<const cx<dd> *>(a.tw);
    const cx<dd> wf = tw[f << (a.tw_log - a.logM - 1)];
    const cx<dd> wg = c_neg(c_conj(wf));
    unsigned char *out = reinterpret_cast<unsigned char *>(as.zc) + (size_t)p * 2 * NCK * (size_t)L::XT;
    Raw<dd> raw;
    for (int c = 0; c < NCK; ++c) {
        load_x(raw, ZX, f, gZ, d, c * KC, t);
        for (int ps = 0; ps < np; ++ps) {
            if (ps == 1)  // the second pass: rows M - f and f
                for (int n = 0; n < 4; ++n) {
                    const cx<dd> v = raw.xa[n];
                    raw.xa[n] = raw.xb[n];
                    raw.xb[n] = v;
                }
            split_chunk_x<dd>(raw, stage, scb, ps ? wg : wf, t);
            __syncthreads();
            unsigned char *o = out + ((size_t)ps * NCK + c) * L::XT;
            for (int q = t * 16; q < L::XT; q += NSPLIT * 16)
                *reinterpret_cast<uint4 *>(o + q) = *reinterpret_cast<const uint4 *>(stage + q);
            __syncthreads();
        }
    }
}

PairArgs tcp_args(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log)
{
    PairArgs a{};
    a.zx = zx; a.zy = zy; a.zc = zc; a.tw = tw; a.tw_log = tw_log; a.M = M;
    int l = 0;
    while (((int64_t)1 << l) < M) ++l;
    a.logM = l;
    a.npairs = M >= 2 ? M / 2 + 1 : 1;
    a.r = a.m = a.c = d;
    return a;
}

template <class T>
cudaError_t tcp_run(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                    int *status, cudaStream_t st, int kclass)
{
    SegParams<PairArgs> P{};  // the launch's parameter block (one product)
    P.nseg = 1;
    P.first[0] = 0;
    P.a[0] = tcp_args(zx, zy, zc, M, d, tw, tw_log);
    return tcp_launch<T>(P, status, st, kclass);
}

} // namespace

bool mrc_tcp_supported(int r, int m, int c) { return r == m && m == c && r >= 32 && r <= 64; }

cudaError_t mrc_tcp_init(void)
{
    for (int k = 2; k <= 4; ++k) {
        cudaError_t e = cudaFuncSetAttribute(tcp_kernel_for<dd, false>(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             TcL<dd>::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(tcp_kernel_for<dd, true>(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     TcL<dd>::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(tcp_kernel_for<float, false>(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     TcL<float>::SMEM);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t mrc_tcp_prep_bytes(int64_t M, int d)
{
    const int64_t npairs = M >= 2 ? M / 2 + 1 : 1;
    const size_t nck = (size_t)(d + KC - 1) / KC;
    return (size_t)npairs * 2 * nck * (size_t)TcL<dd>::XT;
}

size_t mrc_tcp_prep_scale_bytes(int64_t M)
{
    const int64_t npairs = M >= 2 ? M / 2 + 1 : 1;
    return (size_t)npairs * 128 * sizeof(float);
}

cudaError_t mrc_tcp_prep(const SegParams<PairArgs> &P, cudaStream_t st)
{
    if (P.nseg <= 0) return cudaSuccess;
    const int nck = (P.a[0].r + KC - 1) / KC;
    const unsigned grid = (unsigned)(P.a[0].npairs * P.nseg);
    mrc_prof_pre(6, st);
    if (nck <= 2) tcp_prep_kernel<2><<<grid, NSPLIT, TcL<dd>::XT, st>>>(P);
    else if (nck == 3) tcp_prep_kernel<3><<<grid, NSPLIT, TcL<dd>::XT, st>>>(P);
    else tcp_prep_kernel<4><<<grid, NSPLIT, TcL<dd>::XT, st>>>(P);
    double bytes = 0;
    for (int s = 0; s < P.nseg; ++s) bytes += (double)P.a[s].M * P.a[s].r * P.a[s].r * 16.0 + mrc_tcp_prep_bytes(P.a[s].M, P.a[s].r);
    mrc_prof_post(6, st, bytes, 0);
    return cudaGetLastError();
}

cudaError_t mrc_pairmul_dd_tcp(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                               int *status, cudaStream_t st)
{
    return tcp_run<dd>(zx, zy, zc, M, d, tw, tw_log, status, st, 6);
}

cudaError_t mrc_pairmul_f32_tcp(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log,
                                int *status, cudaStream_t st)
{
    return tcp_run<float>(zx, zy, zc, M, d, tw, tw_log, status, st, 5);
}

cudaError_t mrc_tcp_seg(int dd_prec, const SegParams<PairArgs> &P, int *status, cudaStream_t st)
{
    return dd_prec ? tcp_launch<dd>(P, status, st, 6) : tcp_launch<float>(P, status, st, 5);
}

PairArgs mrc_tcp_args(const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw, int tw_log)
{
    return tcp_args(zx, zy, zc, M, d, tw, tw_log);
}
