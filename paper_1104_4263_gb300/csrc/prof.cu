// Kernel timing aid (see prof.cuh) and its C ABI.
#include <mutex>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace die {

std::atomic<bool> g_prof_on{false};
thread_local int g_prof_override = -1;

namespace {
struct Rec {
    int id;
    cudaEvent_t a, b;
};
std::vector<cudaEvent_t> g_pool;         // reusable events
size_t g_used = 0;
std::vector<Rec> g_recs;
std::mutex g_mu;                         // the pool and the records: host threads of the
                                         // concurrent solvers launch at the same time
thread_local int g_open_id = -1;         // the launch bracketed by this thread
thread_local cudaEvent_t g_open_ev = nullptr;
long long g_launches[PK_COUNT];
double g_ms[PK_COUNT];
bool g_overflow = false;
constexpr size_t kMaxEvents = 1 << 19;

cudaEvent_t next_event() {
    if (g_used == g_pool.size()) {
        if (g_pool.size() >= kMaxEvents) return nullptr;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        try {
            g_pool.push_back(e);
        } catch (...) {
            cudaEventDestroy(e);
            return nullptr;
        }
    }
    return g_pool[g_used++];
}
const char* kNames[PK_COUNT] = {"rows_fwd", "cols_green", "rows_inv", "rows_inv_fwd", "dots", "dots32",
                                "cgs_update_norm", "dots_reorth", "update_reorth", "scale",
                                "defl_update", "lincomb", "small_dense", "givens", "other"};
}  // namespace

void prof_mark(int id, cudaStream_t st, int stop) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!stop) {
        g_open_ev = next_event();
        g_open_id = id;
        if (!g_open_ev) { g_overflow = true; return; }
        cudaEventRecord(g_open_ev, st);
        return;
    }
    if (!g_open_ev || g_open_id != id) return;
    cudaEvent_t e = next_event();
    if (!e) { g_overflow = true; g_open_ev = nullptr; return; }
    cudaEventRecord(e, st);
    try {
        g_recs.push_back(Rec{id, g_open_ev, e});
    } catch (...) {
        g_overflow = true;
    }
    g_open_ev = nullptr;
}

}  // namespace die

using namespace die;

extern "C" {

die_status die_prof_begin(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    for (int i = 0; i < PK_COUNT; i++) { g_launches[i] = 0; g_ms[i] = 0; }
    g_recs.clear();
    g_used = 0;
    g_overflow = false;
    g_prof_on = true;
    return DIE_OK;
}

die_status die_prof_end(void) {
    g_prof_on = false;
    DIE_CUDA_TRY(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lock(g_mu);
    for (const Rec& r : g_recs) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_launches[r.id]++;
            g_ms[r.id] += ms;
        } else {
            cudaGetLastError();
        }
    }
    g_recs.clear();
    g_used = 0;
    return g_overflow ? DIE_ENOMEM : DIE_OK;
}

int die_prof_kernels(void) { return PK_COUNT; }

const char* die_prof_name(int id) { return (id >= 0 && id < PK_COUNT) ? kNames[id] : "?"; }

die_status die_prof_read(int id, long long* launches, double* total_ms) {
    if (id < 0 || id >= PK_COUNT || !launches || !total_ms) return DIE_EINVAL;
    *launches = g_launches[id];
    *total_ms = g_ms[id];
    return DIE_OK;
}

}  // extern "C"

// FP64 throughput probe: every thread advances 8 independent chains of dependent FMAs,
// so the FP64 pipe, not the FMA latency, bounds the kernel; the grid covers every SM.
namespace die {
constexpr int kProbeChains = 8;
__global__ void fp64_probe_kernel(double* sink, int iters, double a, double b) {
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) x[c] = 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kProbeChains; c++) x[c] = fma(x[c], a, b);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) s += x[c];
    if (s == 1234.5678) sink[blockIdx.x] = s;     // keeps the chains alive
}
}  // namespace die

extern "C" die_status die_fp64_peak(double* tflops, void* stream) {
    using namespace die;
    if (!tflops) return DIE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    DIE_CUDA_TRY(cudaGetDevice(&dev));
    DIE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 8 * sms, threads = 256, iters = 8192;
    double* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc((void**)&sink, blocks * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return DIE_ENOMEM; }
    die_status s = DIE_OK;
    double best = 0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = DIE_ECUDA;
    for (int rep = 0; s == DIE_OK && rep < 4; rep++) {     // the first run is a warm-up
        cudaEventRecord(e0, st);
        fp64_probe_kernel<<<blocks, threads, 0, st>>>(sink, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, st);
        float ms = 0;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            s = DIE_ECUDA;
            break;
        }
        const double flops = 2.0 * kProbeChains * (double)iters * blocks * threads;
        if (rep > 0 && ms > 0) best = fmax(best, flops / (ms * 1e-3) / 1e12);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    *tflops = best;
    return s;
}
