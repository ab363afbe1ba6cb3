// noalloc.cu -- mrc_inverse_noalloc: the FP64 inverse for callers that must
// not allocate device memory.
//
// Some host programs cannot let a library call cudaMalloc: a process whose
// device memory is owned up front by another allocator (a framework's caching
// pool that has reserved the free memory), firmware-style or certified code
// that forbids dynamic allocation once initialisation is over, or a plugin
// host that hands its plugins fixed buffers only.  For them this entry point
// runs the FP64 FFT-Newton schedule of mrc_inverse (the same level loop, FFT
// kernels and default FP64 product kernel), but its scratch (the spectra of
// the Newton levels, the Gauss-Jordan work area, the twiddle table and the
// status word) lives in one file-scope __device__ array of fixed size, so
// nothing is allocated at call time.  The caller still passes A and psi.
//
// Under CUDA's default lazy module loading the array, like the library's
// kernels, is mapped on a device only when this file's module is first used
// there -- by the first call's cudaGetSymbolAddress.  That first call on each
// device is therefore the initialisation step: make it before another
// allocator reserves the device memory (or load modules eagerly with
// CUDA_MODULE_LOADING=EAGER, which maps the array when the library is
// loaded).
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "../../include/mrc.h"
#include "mrc_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;  // 64 MiB
constexpr int kTwLog = 15;                           // transforms up to 2^14 points (N <= 2^14)
constexpr int kMaxDevices = 64;

// Once mapped on a GPU (see above), the array stays there until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch layout: [status int | twiddles | Gauss-Jordan work | 4 spectra]
constexpr size_t kStatusOff = 0;
constexpr size_t kTwOff = 256;
constexpr size_t kTwBytes = (size_t)16 << kTwLog;
constexpr size_t kWorkOff = kTwOff + kTwBytes;

int64_t max_level(int d, int64_t N) { return mrc_newton_maxM(d, N); }

// the level transforms and products: the built-in FFT plans and the default
// FP64 product kernel (no autotuning here)
cudaError_t fft_f64(void *, int, const FftSrc &sx, const FftDst &dx, int64_t M, int E, int dir, void *scratch,
                    const void *tw, int tw_log, cudaStream_t st)
{
    return mrc_fft_f64(sx, dx, M, E, dir, scratch, tw, tw_log, st, -1);
}

// the level product: the default FP64 product kernel (no autotuning here)
cudaError_t product_f64(void *, int, const void *zx, const void *zy, void *zc, int64_t M, int d, const void *tw,
                        int tw_log, cudaStream_t st)
{
    return mrc_pairmul_f64(zx, zy, zc, M, d, d, d, tw, tw_log, st);
}

size_t need_bytes(int d, int64_t N)
{
    const size_t E = (size_t)d * d;
    return kWorkOff + up256(sizeof(double) * 2 * E) + 3 * up256((size_t)max_level(d, N) * E * 16) +
           up256(mrc_fft_scratch_elems(max_level(d, N), (int)E) * 16);
}

// Once per device, with that device current: resolve the array's device
// address (the host-side symbol is only a stand-in), fill the twiddle table
// and raise the FFT kernel's shared-memory limit.  Synchronous.
mrc_status setup(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_addr[dev]) {
        *out = g_addr[dev];
        return MRC_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        fprintf(stderr, "libmrc: cudaGetSymbolAddress(scratch) failed: %s\n", cudaGetErrorString(e));
        return MRC_ERR_CUDA;
    }
    unsigned char *base = (unsigned char *)p;
    if (mrc_init_f64() != cudaSuccess) return MRC_ERR_CUDA;
    if (mrc_twiddles_f64(base + kTwOff, kTwLog, 0) != cudaSuccess) return MRC_ERR_CUDA;
    if (cudaStreamSynchronize(0) != cudaSuccess) return MRC_ERR_CUDA;
    g_addr[dev] = base;
    *out = base;
    return MRC_OK;
}

#define CKN(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            fprintf(stderr, "libmrc: %s -> %s\n", #call, cudaGetErrorString(e_));         \
            return MRC_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)

} // namespace

extern "C" mrc_status mrc_inverse_noalloc(int d, int64_t N, const double *A, double *psi, void *stream)
{
    if (!A || !psi || d < 1 || d > 512 || N < 1) return MRC_ERR_INVALID_ARG;
    if (N > ((int64_t)1 << (kTwLog - 1)) || need_bytes(d, N) > kScratchBytes) {
        fprintf(stderr,
                "libmrc: mrc_inverse_noalloc(d=%d, N=%lld) needs %zu bytes of scratch; the fixed array holds %zu "
                "and N may not exceed %lld\n",
                d, (long long)N, need_bytes(d, N), kScratchBytes, (long long)1 << (kTwLog - 1));
        return MRC_ERR_NO_MEMORY;
    }
    int dev = 0;
    CKN(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return MRC_ERR_CUDA;
    unsigned char *base = nullptr;
    mrc_status s = setup(dev, &base);
    if (s != MRC_OK) return s;

    cudaStream_t st = (cudaStream_t)stream;
    const int E = d * d;
    int *status = (int *)(base + kStatusOff);
    const void *tw = base + kTwOff;
    double *gjw = (double *)(base + kWorkOff);
    unsigned char *spec = base + kWorkOff + up256(sizeof(double) * 2 * E);
    const int64_t Mmax = max_level(d, N);
    const size_t sb = up256((size_t)Mmax * E * 16);
    void *b0 = spec, *b1 = spec + sb, *b2 = spec + 2 * sb, *bt = spec + 3 * sb;

    // the status word keeps the previous call's value: clear it first
    CKN(cudaMemsetAsync(status, 0, sizeof(int), st));
    CKN(mrc_gauss_jordan(A, psi, gjw, d, status, st));
    const int64_t m0 = mrc_base_size(d, N);
    CKN(mrc_base_case(A, psi, d, m0, st));
    const NewtonBufs nb{b0, b1, b2, bt};
    if (mrc_newton_levels(PREC_F64, d, N, A, psi, m0, nb, tw, kTwLog, fft_f64, product_f64, nullptr, st, nullptr,
                          nullptr, nullptr, nullptr) != 0)
        return MRC_ERR_CUDA;
    CKN(cudaStreamSynchronize(st));
    int h = 0;
    CKN(cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost));
    return h ? (mrc_status)h : MRC_OK;
}
