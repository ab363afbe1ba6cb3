// misc.cu -- FP64 kernels around the FFT-Newton core: Gauss-Jordan inverse of
// A(0), the direct recursion for the first m0 coefficients, survival
// diagonal scans, residual norms, block gathers for first-entrance kernels and
// the occupation / first-entrance reductions.
#include <math.h>
#include "arith.cuh"
#include "mrc_internal.h"

#define MRC_ST_SINGULAR 2

namespace {

__device__ __forceinline__ void warp_argmax(double &v, int &i)
{
    for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_down_sync(0xffffffffu, v, o);
        int i2 = __shfl_down_sync(0xffffffffu, i, o);
        if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
    }
}

// Block-wide argmax of (v, i); the result is broadcast through shared memory.
__device__ void block_argmax(double &v, int &i, double *sv, int *si)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    warp_argmax(v, i);
    if (lane == 0) { sv[wid] = v; si[wid] = i; }
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? sv[lane] : -1.0;
        i = lane < nw ? si[lane] : 0x7fffffff;
        warp_argmax(v, i);
        if (lane == 0) { sv[0] = v; si[0] = i; }
    }
    __syncthreads();
    v = sv[0];
    i = si[0];
    __syncthreads();
}

// Gauss-Jordan with partial pivoting on [A0 | I] (d x 2d, row-major in W).
// One CTA.  A pivot with |p| <= d 2^-52 max|A0| marks A0 singular: the
// status word is set, `out` is filled with NaN and the kernel returns.
__device__ __forceinline__ void gj_run(const double *__restrict__ A0, double *__restrict__ out,
                                       double *__restrict__ W, int d, int *status)
{
    __shared__ double sv[32];
    __shared__ int si[32];
    extern __shared__ double fac[];  // [d]
    const int n2 = 2 * d, tid = threadIdx.x, nt = blockDim.x;
    double amax = 0.0;
    for (int t = tid; t < d * n2; t += nt) {
        int i = t / n2, j = t - i * n2;
        double v = j < d ? A0[i * d + j] : ((j - d) == i ? 1.0 : 0.0);
        W[t] = v;
        if (j < d) amax = fmax(amax, fabs(v));
    }
    int dummy = 0;
    block_argmax(amax, dummy, sv, si);
    const double tol = (double)d * 0x1p-52 * amax;
    for (int col = 0; col < d; ++col) {
        double best = -1.0;
        int piv = 0x7fffffff;
        for (int i = col + tid; i < d; i += nt) {
            double v = fabs(W[i * n2 + col]);
            if (v > best || (v == best && i < piv)) { best = v; piv = i; }
        }
        block_argmax(best, piv, sv, si);
        if (!(best > tol)) {
            if (tid == 0) atomicExch(status, MRC_ST_SINGULAR);
            for (int t = tid; t < d * d; t += nt) out[t] = __longlong_as_double(0x7ff8000000000000ll);
            return;
        }
        if (piv != col)
            for (int j = tid; j < n2; j += nt) {
                double t = W[col * n2 + j];
                W[col * n2 + j] = W[piv * n2 + j];
                W[piv * n2 + j] = t;
            }
        __syncthreads();
        const double p = W[col * n2 + col];
        __syncthreads();
        for (int j = tid; j < n2; j += nt) W[col * n2 + j] /= p;
        __syncthreads();
        for (int i = tid; i < d; i += nt) fac[i] = W[i * n2 + col];
        __syncthreads();
        for (int t = tid; t < d * n2; t += nt) {
            int i = t / n2, j = t - i * n2;
            if (i != col) W[t] = fma(-fac[i], W[col * n2 + j], W[t]);
        }
        __syncthreads();
    }
    for (int t = tid; t < d * d; t += nt) {
        int i = t / d, j = t - i * d;
        out[t] = W[i * n2 + d + j];
    }
}

__global__ void __launch_bounds__(1024) gj_kernel(const double *__restrict__ A0, double *__restrict__ out,
                                                  double *__restrict__ W, int d, int *status)
{
    gj_run(A0, out, W, d, status);
}

// one CTA per model of a batch
__global__ void __launch_bounds__(1024) gj_batch_kernel(const __grid_constant__ SegParams<GjArgs> P)
{
    const GjArgs &g = P.a[blockIdx.x];
    gj_run(g.A0, g.out, g.W, g.d, g.status);
}

// Direct recursion for the first m0 coefficients (left form, Theorem 2.2):
//   psi(k) = A(0)^{-1} [ - sum_{l=1..k} A(l) psi(k-l) ],  k = 1..m0-1,
// with psi(0) = A(0)^{-1} already in place.  CTA j owns column j (columns
// are independent in the left recursion), thread i owns row i.
__device__ __forceinline__ void base_case_run(const double *__restrict__ A, double *__restrict__ psi, int d, int m0,
                                              int j)
{
    extern __shared__ double t[];  // [d]
    const int64_t E = (int64_t)d * d;
    for (int k = 1; k < m0; ++k) {
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            double s = 0.0;
            for (int l = 1; l <= k; ++l) {
                const double *Al = A + l * E + (int64_t)i * d;
                const double *Pk = psi + (int64_t)(k - l) * E + j;
                for (int u = 0; u < d; ++u) s = fma(-Al[u], Pk[(int64_t)u * d], s);
            }
            t[i] = s;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            double v = 0.0;
            for (int u = 0; u < d; ++u) v = fma(psi[(int64_t)i * d + u], t[u], v);
            psi[(int64_t)k * E + (int64_t)i * d + j] = v;
        }
        __syncthreads();
    }
}

__global__ void base_case_kernel(const double *__restrict__ A, double *__restrict__ psi, int d, int m0)
{
    base_case_run(A, psi, d, m0, blockIdx.x);
}

// column blockIdx.x of model blockIdx.y of a batch
__global__ void base_case_batch_kernel(const __grid_constant__ SegParams<BaseArgs> P)
{
    const BaseArgs &g = P.a[blockIdx.y];
    if ((int)blockIdx.x >= g.d || g.m0 <= 1) return;
    base_case_run(g.A, g.psi, g.d, g.m0, blockIdx.x);
}

// rs[k][i] = sum_j q[k][i][j] for k >= 1, rs[0][i] = 0.
__global__ void row_sums_kernel(const double *__restrict__ q, double *__restrict__ rs, int d, int64_t N)
{
    const int64_t n = N * d;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = t / d;
        int i = (int)(t - k * d);
        double s = 0.0;
        if (k >= 1)
            for (int j = 0; j < d; ++j) s += q[k * d * d + (int64_t)i * d + j];
        rs[t] = s;
    }
}

constexpr int SCAN_CH = 1024;

__global__ void scan_chunk_sums(const double *__restrict__ x, int ncol, int64_t N, double *__restrict__ work)
{
    const int64_t nch = (N + SCAN_CH - 1) / SCAN_CH;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nch * ncol; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t ch = t / ncol;
        int c = (int)(t - ch * ncol);
        int64_t k1 = min(N, (ch + 1) * SCAN_CH);
        double s = 0.0;
        for (int64_t k = ch * SCAN_CH; k < k1; ++k) s += x[k * ncol + c];
        work[t] = s;
    }
}

__global__ void scan_chunk_offsets(double *work, int ncol, int64_t nch)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += gridDim.x * blockDim.x) {
        double run = 0.0;
        for (int64_t ch = 0; ch < nch; ++ch) {
            double v = work[ch * ncol + c];
            work[ch * ncol + c] = run;
            run += v;
        }
    }
}

__global__ void scan_apply(double *__restrict__ x, int ncol, int64_t N, const double *__restrict__ work, double scale,
                           double offset)
{
    const int64_t nch = (N + SCAN_CH - 1) / SCAN_CH;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nch * ncol; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t ch = t / ncol;
        int c = (int)(t - ch * ncol);
        int64_t k1 = min(N, (ch + 1) * SCAN_CH);
        double run = work[t];
        for (int64_t k = ch * SCAN_CH; k < k1; ++k) {
            run += x[k * ncol + c];
            x[k * ncol + c] = offset + scale * run;
        }
    }
}

// acc[0] += sum_k ||rho(k)||_F ; acc[1] = max |rho| (as ordered bits of a nonnegative double)
__global__ void norms_kernel(const double *__restrict__ rho, int E, int64_t N, double *acc)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double fro_sum = 0.0, mx = 0.0;
    for (int64_t k = warp; k < N; k += nwarps) {
        double s = 0.0;
        for (int e = lane; e < E; e += 32) {
            double v = rho[k * E + e];
            s = fma(v, v, s);
            mx = fmax(mx, fabs(v));
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) fro_sum += sqrt(s);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if (lane == 0) {
        atomicAdd(&acc[0], fro_sum);
        atomicMax(reinterpret_cast<unsigned long long *>(&acc[1]), (unsigned long long)__double_as_longlong(mx));
    }
}

struct IdxList {
    int n;
    int idx[512];
};

// ACC(k) = delta(k) I - q_CC(k), QCD(k) = q_CD(k)  (Eq. (first-entrance-mass))
__global__ void gather_blocks_kernel(const double *__restrict__ q, int d, int64_t N, IdxList C, IdxList D,
                                     double *__restrict__ ACC, double *__restrict__ QCD)
{
    const int nC = C.n, nD = D.n;
    const int64_t per = (int64_t)nC * (nC + nD);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N * per; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = t / per;
        int rem = (int)(t - k * per);
        int a = rem / (nC + nD), b = rem - a * (nC + nD);
        if (b < nC) {
            double v = -q[k * d * d + (int64_t)C.idx[a] * d + C.idx[b]];
            if (k == 0 && a == b) v += 1.0;
            ACC[k * nC * nC + (int64_t)a * nC + b] = v;
        } else {
            b -= nC;
            QCD[k * nC * nD + (int64_t)a * nD + b] = q[k * d * d + (int64_t)C.idx[a] * d + D.idx[b]];
        }
    }
}

// out[k] = sum_{a,b} alpha[a] g[k][a][b]
__global__ void weighted_rowsum_kernel(const double *__restrict__ g, int nC, int nD, int64_t N,
                                       const double *__restrict__ alpha, double *__restrict__ out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int a = 0; a < nC; ++a) {
            double r = 0.0;
            for (int b = 0; b < nD; ++b) r += g[k * nC * nD + (int64_t)a * nD + b];
            s = fma(alpha[a], r, s);
        }
        out[k] = s;
    }
}

// out[k] = alpha P(k) 1_B
__global__ void occupation_kernel(const double *__restrict__ P, int d, int64_t N, const double *__restrict__ alpha,
                                  IdxList B, double *__restrict__ out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < d; ++i) {
            double r = 0.0;
            for (int b = 0; b < B.n; ++b) r += P[k * d * d + (int64_t)i * d + B.idx[b]];
            s = fma(alpha[i], r, s);
        }
        out[k] = s;
    }
}

__global__ void one_minus_kernel(const double *__restrict__ x, double *__restrict__ y, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        y[t] = 1.0 - x[t];
}

// Endpoint mean-value rule (Section 4): from the kernel samples Q_h(m),
// m = 0 .. N, with Delta Q_h(0) = O, Delta Q_h(m) = Q_h(m) - Q_h(m-1) and
// Delta+ Q_h(m) = Delta Q_h(m+1): A(m) = delta(m) I - Qbar_h(m) with
// Qbar_h = (Delta Q_h + Delta+ Q_h) / 2 (scheme 0, Eq. (mre-solution)), or
// A(m) = delta(m) I - Delta Q_h(m) (scheme 1, Eq. (process-discretization)).
__global__ void mre_operator_kernel(const double *__restrict__ Q, double *__restrict__ A, int d, int64_t N,
                                    int scheme)
{
    const int64_t E = (int64_t)d * d, n = N * E;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = t / E, e = t - m * E;
        const double dQ = m > 0 ? Q[m * E + e] - Q[(m - 1) * E + e] : 0.0;
        const double v = scheme == 0 ? 0.5 * (dQ + (Q[(m + 1) * E + e] - Q[m * E + e])) : dQ;
        const int i = (int)(e / d), j = (int)(e - (e / d) * d);
        A[t] = (m == 0 && i == j ? 1.0 : 0.0) - v;
    }
}

// Right-hand side of Eq. (mre-solution): R(m) = L_h(m) - (1/2) Delta+ Q_h(m) L_h(0)
// ([d][c] per m; Delta+ Q_h * (L_h(0) e0) is Delta+ Q_h(m) L_h(0) at every m).
__global__ void mre_rhs_kernel(const double *__restrict__ Q, const double *__restrict__ L, double *__restrict__ R,
                               int d, int c, int64_t N)
{
    const int64_t E = (int64_t)d * d, EL = (int64_t)d * c, n = N * EL;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = t / EL, e = t - m * EL;
        const int i = (int)(e / c), j = (int)(e - (e / c) * c);
        const double *q1 = Q + (m + 1) * E + (int64_t)i * d, *q0 = Q + m * E + (int64_t)i * d;
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += (q1[k] - q0[k]) * L[(int64_t)k * c + j];
        R[t] = L[t] - 0.5 * s;
    }
}

// ---------------------------------------------------------------------------
// Gauss-Jordan elimination over the truncated series ring C[[x]]/<x^N>
// (Appendix D, "Gauss-Jordan inversion"), on the augmented matrix
// W = [P_A(x) | I] stored as W(k) = [A(k) | delta_k0 I], [N][d][2d].

// W(k)[i][j] = A(k)[i][j] (j < d), delta_k0 delta_i(j-d) (j >= d)
// (and clears the call's singular flag)
__global__ void gjs_init_kernel(const double *__restrict__ A, double *__restrict__ W, int d, int64_t N, int *flag)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *flag = 0;
    const int n2 = 2 * d;
    const int64_t E = (int64_t)d * n2, n = N * E;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / E, e = t - k * E;
        const int i = (int)(e / n2), j = (int)(e - (int64_t)i * n2);
        W[t] = j < d ? A[k * d * d + (int64_t)i * d + j] : (k == 0 && j - d == i ? 1.0 : 0.0);
    }
}

// Pivot of column `col`: the row r >= col with the largest |W(0)[r][col]|
// (the constant coefficients follow ordinary Gauss-Jordan on A(0)).  A pivot
// with |p| <= d 2^-52 max|A(0)| marks A(0) singular (status word and the
// call's flag); the column is then left in place.  One CTA.
__global__ void __launch_bounds__(256) gjs_pivot_kernel(const double *__restrict__ A0, const double *__restrict__ W,
                                                        int d, int col, int *__restrict__ piv, int *flag, int *status)
{
    __shared__ double sv[32];
    __shared__ int si[32];
    double amax = 0.0;
    for (int t = threadIdx.x; t < d * d; t += blockDim.x) amax = fmax(amax, fabs(A0[t]));
    int dummy = 0;
    block_argmax(amax, dummy, sv, si);
    double best = -1.0;
    int p = 0x7fffffff;
    for (int r = col + threadIdx.x; r < d; r += blockDim.x) {
        const double v = fabs(W[(int64_t)r * 2 * d + col]);
        if (v > best || (v == best && r < p)) { best = v; p = r; }
    }
    block_argmax(best, p, sv, si);
    if (threadIdx.x == 0) {
        const bool sing = !(best > (double)d * 0x1p-52 * amax);
        if (sing) {
            atomicExch(status, MRC_ST_SINGULAR);
            *flag = 1;
        }
        *piv = sing ? col : p;
    }
}

// Row exchange col <-> piv at every k, and the two series the pivot step
// needs, both read before the exchange (each thread owns one k, so no other
// thread touches its values): u(k) = W(k)[piv][col] (the pivot series) and
// cv(k)[r] = W(k)[r][col] after the exchange for r != col, 0 for r = col
// (the elimination factors; the pivot row is not eliminated from itself).
__global__ void gjs_swap_kernel(double *__restrict__ W, int d, int64_t N, int col, const int *__restrict__ piv,
                                double *__restrict__ u, double *__restrict__ cv)
{
    const int n2 = 2 * d, p = *piv;
    const int64_t E = (int64_t)d * n2;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        double *w = W + k * E;
        u[k] = w[(int64_t)p * n2 + col];
        for (int r = 0; r < d; ++r) {
            const int src = r == p ? col : r;
            cv[k * d + r] = r == col ? 0.0 : w[(int64_t)src * n2 + col];
        }
        if (p != col)
            for (int j = 0; j < n2; ++j) {
                const double a = w[(int64_t)col * n2 + j];
                w[(int64_t)col * n2 + j] = w[(int64_t)p * n2 + j];
                w[(int64_t)p * n2 + j] = a;
            }
    }
}

// psi(k) = right block of W(k); NaN everywhere if A(0) was found singular
__global__ void gjs_extract_kernel(const double *__restrict__ W, double *__restrict__ psi, int d, int64_t N,
                                   const int *flag)
{
    const int64_t E = (int64_t)d * d, n = N * E;
    const bool bad = *flag != 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / E, e = t - k * E;
        const int i = (int)(e / d), j = (int)(e - (int64_t)i * d);
        psi[t] = bad ? __longlong_as_double(0x7ff8000000000000ll) : W[k * 2 * E + (int64_t)i * 2 * d + d + j];
    }
}

inline unsigned grid_for(int64_t n, int bs = 256)
{
    int64_t b = (n + bs - 1) / bs;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

} // namespace

cudaError_t mrc_gauss_jordan(const double *A0, double *out, double *work, int d, int *status, cudaStream_t st)
{
    mrc_prof_pre(7, st);
    gj_kernel<<<1, 1024, sizeof(double) * d, st>>>(A0, out, work, d, status);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_base_case(const double *A, double *psi, int d, int64_t m0, cudaStream_t st)
{
    if (m0 <= 1) return cudaSuccess;
    int bs = d < 32 ? 32 : (d > 512 ? 512 : ((d + 31) / 32) * 32);
    mrc_prof_pre(7, st);
    base_case_kernel<<<d, bs, sizeof(double) * d, st>>>(A, psi, d, (int)m0);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_row_sums(const double *q, double *rs, int d, int64_t N, cudaStream_t st)
{
    mrc_prof_pre(7, st);
    row_sums_kernel<<<grid_for(N * d), 256, 0, st>>>(q, rs, d, N);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_scan_cols(double *x, int ncol, int64_t N, double *work, double scale, double offset, cudaStream_t st)
{
    const int64_t nch = (N + SCAN_CH - 1) / SCAN_CH;
    mrc_prof_pre(7, st);
    scan_chunk_sums<<<grid_for(nch * ncol), 256, 0, st>>>(x, ncol, N, work);
    mrc_prof_post(7, st, 0, 0);
    mrc_prof_pre(7, st);
    scan_chunk_offsets<<<grid_for(ncol), 256, 0, st>>>(work, ncol, nch);
    mrc_prof_post(7, st, 0, 0);
    mrc_prof_pre(7, st);
    scan_apply<<<grid_for(nch * ncol), 256, 0, st>>>(x, ncol, N, work, scale, offset);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_norms(const double *rho, int E, int64_t N, double *acc, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    mrc_prof_pre(7, st);
    norms_kernel<<<grid_for(N * 32), 256, 0, st>>>(rho, E, N, acc);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_gather_blocks(const double *q, int d, int64_t N, const int *Cidx, int nC, const int *Didx, int nD,
                              double *ACC, double *QCD, cudaStream_t st)
{
    IdxList C{}, D{};
    C.n = nC;
    D.n = nD;
    for (int i = 0; i < nC; ++i) C.idx[i] = Cidx[i];
    for (int i = 0; i < nD; ++i) D.idx[i] = Didx[i];
    mrc_prof_pre(7, st);
    gather_blocks_kernel<<<grid_for(N * nC * (nC + nD)), 256, 0, st>>>(q, d, N, C, D, ACC, QCD);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_weighted_rowsum(const double *g, int nC, int nD, int64_t N, const double *alpha, double *out,
                                cudaStream_t st)
{
    mrc_prof_pre(7, st);
    weighted_rowsum_kernel<<<grid_for(N), 256, 0, st>>>(g, nC, nD, N, alpha, out);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_occupation_k(const double *P, int d, int64_t N, const double *alpha, const int *inB, double *out,
                             cudaStream_t st)
{
    IdxList B{};
    B.n = 0;
    for (int j = 0; j < d; ++j)
        if (inB[j]) B.idx[B.n++] = j;
    mrc_prof_pre(7, st);
    occupation_kernel<<<grid_for(N), 256, 0, st>>>(P, d, N, alpha, B, out);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_mre_operator(const double *Q, double *A, int d, int64_t N, int scheme, cudaStream_t st)
{
    mrc_prof_pre(7, st);
    mre_operator_kernel<<<grid_for(N * (int64_t)d * d), 256, 0, st>>>(Q, A, d, N, scheme);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_mre_rhs(const double *Q, const double *L, double *R, int d, int c, int64_t N, cudaStream_t st)
{
    mrc_prof_pre(7, st);
    mre_rhs_kernel<<<grid_for(N * (int64_t)d * c), 256, 0, st>>>(Q, L, R, d, c, N);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

// y = x rounded to binary32 (nearest, ties to even; integer operations only),
// for the FP32 Newton levels' copy of A.  Four independent elements per
// thread and iteration, consecutive across the warp.
__global__ void f64_to_f32_kernel(const double *__restrict__ x, float *__restrict__ y, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = x[i + u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) y[i + u * stride] = f64_to_f32_rn(v[u]);
    }
    for (; i < n; i += stride) y[i] = f64_to_f32_rn(x[i]);
}

// conversion of segment s's elements [loc C, (loc + 1) C) by CTA loc of the segment
__global__ void f64_to_f32_batch_kernel(const __grid_constant__ SegParams<CvtArgs> P)
{
    const int s = seg_find(P, blockIdx.x);
    const CvtArgs &g = P.a[s];
    const int64_t e0 = (int64_t)(blockIdx.x - P.first[s]) * MRC_CVT_CHUNK;
    const int64_t e1 = min(g.n, e0 + MRC_CVT_CHUNK);
    for (int64_t i = e0 + threadIdx.x; i < e1; i += blockDim.x) g.y[i] = f64_to_f32_rn(g.x[i]);
}

cudaError_t mrc_gauss_jordan_batch(const SegParams<GjArgs> &P, int dmax, cudaStream_t st)
{
    if (P.nseg <= 0) return cudaSuccess;
    mrc_prof_pre(7, st);
    gj_batch_kernel<<<P.nseg, 1024, sizeof(double) * dmax, st>>>(P);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_base_case_batch(const SegParams<BaseArgs> &P, int dmax, cudaStream_t st)
{
    if (P.nseg <= 0) return cudaSuccess;
    const int bs = dmax < 32 ? 32 : (dmax > 512 ? 512 : ((dmax + 31) / 32) * 32);
    mrc_prof_pre(7, st);
    base_case_batch_kernel<<<dim3(dmax, P.nseg), bs, sizeof(double) * dmax, st>>>(P);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_f64_to_f32_batch(const SegParams<CvtArgs> &P, unsigned nctas, cudaStream_t st)
{
    if (P.nseg <= 0 || nctas == 0) return cudaSuccess;
    double n = 0;
    for (int s = 0; s < P.nseg; ++s) n += (double)P.a[s].n;
    mrc_prof_pre(7, st);
    f64_to_f32_batch_kernel<<<nctas, 256, 0, st>>>(P);
    mrc_prof_post(7, st, n * 12.0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_f64_to_f32(const double *x, float *y, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    mrc_prof_pre(7, st);
    f64_to_f32_kernel<<<grid_for(n), 256, 0, st>>>(x, y, n);
    mrc_prof_post(7, st, (double)n * 12.0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_one_minus(const double *x, double *y, int64_t n, cudaStream_t st)
{
    mrc_prof_pre(7, st);
    one_minus_kernel<<<grid_for(n), 256, 0, st>>>(x, y, n);
    mrc_prof_post(7, st, 0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_gjs_init(const double *A, double *W, int d, int64_t N, int *flag, cudaStream_t st)
{
    const int64_t n = N * 2 * (int64_t)d * d;
    mrc_prof_pre(7, st);
    gjs_init_kernel<<<grid_for(n), 256, 0, st>>>(A, W, d, N, flag);
    mrc_prof_post(7, st, (double)n * 12.0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_gjs_pivot(const double *A0, double *W, int d, int64_t N, int col, int *piv, double *u, double *cv,
                          int *flag, int *status, cudaStream_t st)
{
    mrc_prof_pre(7, st);
    gjs_pivot_kernel<<<1, 256, 0, st>>>(A0, W, d, col, piv, flag, status);
    mrc_prof_post(7, st, 0, 0);
    mrc_prof_pre(7, st);
    gjs_swap_kernel<<<grid_for(N, 128), 128, 0, st>>>(W, d, N, col, piv, u, cv);
    mrc_prof_post(7, st, (double)N * (4.0 * d + 1 + d) * 8.0, 0);
    return cudaGetLastError();
}

cudaError_t mrc_gjs_extract(const double *W, double *psi, int d, int64_t N, const int *flag, cudaStream_t st)
{
    const int64_t n = N * (int64_t)d * d;
    mrc_prof_pre(7, st);
    gjs_extract_kernel<<<grid_for(n), 256, 0, st>>>(W, psi, d, N, flag);
    mrc_prof_post(7, st, (double)n * 16.0, 0);
    return cudaGetLastError();
}
