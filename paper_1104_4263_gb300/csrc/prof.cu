// Kernel timing aid (see prof.cuh) and its C ABI.
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace die {

bool g_prof_on = false;
thread_local int g_prof_override = -1;

namespace {
struct Rec {
    int id;
    cudaEvent_t a, b;
};
std::vector<cudaEvent_t> g_pool;         // reusable events
size_t g_used = 0;
std::vector<Rec> g_recs;
int g_open_id = -1;
cudaEvent_t g_open_ev = nullptr;
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
