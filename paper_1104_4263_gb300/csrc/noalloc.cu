// deflation_apply_noalloc: z = P^-1 x = x + V (M (V^* x)) without any device
// allocation.  It runs the same two kernels as deflation_apply (batched projections
// with a deterministic two-level reduction, then the rank-r update), but their
// scratch -- the per-block and per-group partial sums, the r projections and the
// arrival counters of the reduction -- lives in the file-scope array below instead of
// buffers allocated by deflation_build.
#include <mutex>

#include "solver.cuh"

namespace die {

constexpr int kNoAllocMaxR = 128;                // largest deflation rank accepted
constexpr int kNoAllocMaxDevices = 64;
constexpr long kNoAllocPartials = (long)kNoAllocMaxR * kRedBlocksMax;
constexpr long kNoAllocPartials2 = (long)kNoAllocMaxR * kRedGroupsMax;
constexpr long kNoAllocCounterSlots = (kRedCounters * sizeof(unsigned) + sizeof(double2) - 1) / sizeof(double2);
// block partials | group partials | projections s | counters
constexpr long kNoAllocSlots = kNoAllocPartials + kNoAllocPartials2 + kNoAllocMaxR + kNoAllocCounterSlots;

// (128 * 640 + 128 * 40 + 128 + 11) * 16 bytes (about 1.4 MB), held by every GPU that
// loads the library until the process exits.
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocSlots];

static std::mutex g_noalloc_mu;
static double2* g_noalloc_addr[kNoAllocMaxDevices];

// Device address of the array on device `dev`, the current one (looked up once per
// device and kept; a cudaDeviceReset makes the kept address stale).
static die_status noalloc_scratch(int dev, double2** out) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return DIE_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_last_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
            return DIE_ECUDA;
        }
        g_noalloc_addr[dev] = reinterpret_cast<double2*>(p);
    }
    *out = g_noalloc_addr[dev];
    return DIE_OK;
}

}  // namespace die

using namespace die;

extern "C" die_status deflation_apply_noalloc(defl_t d, const void* x, void* z, void* stream) {
    if (!d || !x || !z) return DIE_EINVAL;
    if (d->r < 1 || d->r > kNoAllocMaxR) return DIE_EINVAL;
    int dev = 0;
    DIE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != d->device) return DIE_EINVAL;      // V and M live on another device
    double2* base = nullptr;
    DIE_TRY(noalloc_scratch(dev, &base));
    cudaStream_t st = (cudaStream_t)stream;
    RedScratch rs;
    rs.partial = base;
    rs.partial2 = base + kNoAllocPartials;
    double2* s = base + kNoAllocPartials + kNoAllocPartials2;
    rs.counter = reinterpret_cast<unsigned*>(s + kNoAllocMaxR);
    // the reduction's arrival counters must start at zero
    DIE_CUDA_TRY(cudaMemsetAsync(rs.counter, 0, kRedCounters * sizeof(unsigned), st));
    DIE_TRY(k_dots(d->V, d->n, d->r, (const double2*)x, d->n, 0, s, rs, nullptr, st));
    DIE_TRY(k_defl_update(d->V, d->n, d->r, d->M, s, (const double2*)x, (double2*)z, d->n, nullptr, st));
    return DIE_OK;
}
