// prof.cu -- launch counting and optional per-kernel-class timing.
//
// Every kernel launch of the library goes through mrc_prof_pre / _post.  The
// counter is always on.  When a kernel class is selected with
// mrc_profile_begin, CUDA events are recorded around each launch of that class
// on its own stream, together with the algorithmic bytes and flops the launch
// is charged with; mrc_profile_end sums them.  Launches on an untimed stream
// (mrc_prof_set_untimed: the side stream whose kernels overlap
// the critical path, so that their event durations include time spent
// waiting for SMs) are counted but not timed.  Not thread safe: profile one
// host thread at a time.
#include <atomic>
#include <vector>

#include "../../include/mrc.h"
#include "mrc_internal.h"

namespace {
std::atomic<unsigned long long> g_launches{0};
struct Prof {
    int kclass = 0;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    double bytes = 0, flops = 0;
    long long n = 0;
    bool capturing = false;  // no event records while a stream capture is open
} g_prof;
constexpr size_t kPool = 16384;
} // namespace

void mrc_prof_set_capturing(bool on) { g_prof.capturing = on; }
bool mrc_prof_timing() { return g_prof.kclass != 0; }

namespace {
cudaStream_t g_untimed = nullptr;
}
void mrc_prof_set_untimed(cudaStream_t st) { g_untimed = st; }


void mrc_prof_pre(int kclass, cudaStream_t st)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_prof.capturing || (g_untimed && st == g_untimed)) return;
    if (g_prof.kclass && kclass == g_prof.kclass && g_prof.used + 2 <= g_prof.pool.size())
        cudaEventRecord(g_prof.pool[g_prof.used], st);
}

void mrc_prof_post(int kclass, cudaStream_t st, double bytes, double flops)
{
    if (g_prof.capturing || (g_untimed && st == g_untimed)) return;
    if (g_prof.kclass && kclass == g_prof.kclass && g_prof.used + 2 <= g_prof.pool.size()) {
        cudaEventRecord(g_prof.pool[g_prof.used + 1], st);
        g_prof.used += 2;
        g_prof.bytes += bytes;
        g_prof.flops += flops;
        g_prof.n += 1;
    }
}

extern "C" {

unsigned long long mrc_launch_count(void) { return g_launches.load(); }

mrc_status mrc_profile_begin(int kclass)
{
    if (kclass < 0 || kclass > MRC_KCLASS_MAX) return MRC_ERR_INVALID_ARG;
    if (g_prof.pool.empty()) {
        g_prof.pool.resize(kPool);
        for (auto &e : g_prof.pool)
            if (cudaEventCreate(&e) != cudaSuccess) return MRC_ERR_CUDA;
    }
    g_prof.kclass = kclass;
    g_prof.used = 0;
    g_prof.bytes = g_prof.flops = 0;
    g_prof.n = 0;
    return MRC_OK;
}

mrc_status mrc_profile_end(double *ms_total, long long *launches, double *bytes, double *flops)
{
    double ms = 0;
    for (size_t i = 0; i + 1 < g_prof.used; i += 2) {
        if (cudaEventSynchronize(g_prof.pool[i + 1]) != cudaSuccess) return MRC_ERR_CUDA;
        float t = 0;
        cudaEventElapsedTime(&t, g_prof.pool[i], g_prof.pool[i + 1]);
        ms += t;
    }
    if (ms_total) *ms_total = ms;
    if (launches) *launches = g_prof.n;
    if (bytes) *bytes = g_prof.bytes;
    if (flops) *flops = g_prof.flops;
    g_prof.kclass = 0;
    g_prof.used = 0;
    return MRC_OK;
}

} // extern "C"
