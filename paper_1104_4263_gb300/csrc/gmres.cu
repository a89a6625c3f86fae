// Restarted GMRES(m) (Saad & Schultz) on Atilde = A or A_R A (Section 5), with the
// deflating right preconditioner of Eq. (4.12): Atilde P^-1 v = btilde, x = P^-1 v.
//
// One cycle runs entirely on the device without host round trips.  Each Arnoldi
// vector is orthogonalised by classical Gram-Schmidt with the DGKS criterion: a second
// pass only when the first left less than eta of ||w|| (unless the caller sets eta: 0.01
// for cycles of up to 64 steps, the classical 1/sqrt(2) for longer ones).  Cycles start
// single-pass (the second-pass kernels are not launched); a
// cycle in which the criterion fires stops and runs again with the second passes, and
// the solve keeps them.  The passes use the three-multiplication form of the complex
// products (Re - Im of every basis vector is stored when the vector is normalised).
// The new Hessenberg column is rotated by Givens rotations on the device, on a side
// stream one step behind, since the next Arnoldi step does not need the rotations; the
// normalisation of the new vector uses 1 / ||w|| from the last Gram-Schmidt kernel.
// When the residual estimate reaches tol the Givens step sets a device flag that makes
// the kernels of the remaining steps skip their work.  The host reads one flag set per
// cycle.  Between cycles the residual btilde - Atilde x is recomputed in FP64 (in the
// FP32-inner form this is the iterative-refinement step).
//
// FP32-inner form: the products with Atilde inside a cycle run in complex64 and the
// deflation P^-1 uses a complex64 copy of V and M with FP32 sums (P^-1 is one fixed
// preconditioner for the whole solve, so its rounding only changes the
// preconditioner, and the FP64 restart residual corrects the iterate).  Arnoldi,
// least squares and the restart residual are FP64 in both forms.
//
// A solve runs in a context (SolverCache): buffers, streams, deflation scratch and,
// for the right-hand sides of gmres_solve_batch, a product workspace of its own, so
// that several solves can run at once on one operator.  With gmres_opts.graph a
// cycle's Arnoldi steps (and the side-stream Givens steps) are captured once into a
// CUDA graph per configuration and replayed with one launch per cycle; what changes
// from cycle to cycle (the history slot of the first step, ||btilde||) is read from
// device memory, so the replay is the same launch sequence.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "prof.cuh"
#include "solver.cuh"

namespace die {

die_status alloc_red_scratch(RedScratch* rs) {
    if (cudaMalloc((void**)&rs->partial, (size_t)kMaxBasis * (kRedBlocksMax + kRedGroupsMax) * sizeof(double2)) !=
        cudaSuccess) {
        cudaGetLastError();
        return DIE_ENOMEM;
    }
    rs->partial2 = rs->partial + (size_t)kMaxBasis * kRedBlocksMax;
    if (cudaMalloc((void**)&rs->counter, kRedCounters * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return DIE_ENOMEM;
    }
    DIE_CUDA_TRY(cudaMemset(rs->counter, 0, kRedCounters * sizeof(unsigned)));
    return DIE_OK;
}

void free_red_scratch(RedScratch* rs) {
    if (rs->partial) cudaFree(rs->partial);
    if (rs->counter) cudaFree(rs->counter);
    rs->partial = nullptr;
    rs->partial2 = nullptr;
    rs->counter = nullptr;
}

SolverCache* solver_cache(dieop_s* op) { return reinterpret_cast<SolverCache*>(op->solver); }

static void free_cache(SolverCache* c) {
    if (!c) return;
    void* ptrs[] = {c->V, c->Vm, c->btil, c->tmp, c->z, c->v32, c->z32, c->small, c->hist, c->ints, c->one,
                    c->ds.s, c->ds.c32, c->ws.W, c->ws.v};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    free_red_scratch(&c->rs);
    free_red_scratch(&c->ds.rs);
    if (c->host) cudaFreeHost(c->host);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : {c->join[0], c->join[1], c->fork, c->back})
        if (e) cudaEventDestroy(e);
    for (CycleGraph& g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->side) cudaStreamDestroy(c->side);
    delete c;
}

void free_solver_cache(dieop_s* op) {
    free_cache(solver_cache(op));
    op->solver = nullptr;
    for (void*& p : op->batch) {
        free_cache(reinterpret_cast<SolverCache*>(p));
        p = nullptr;
    }
}

// H, cs, sn, g, h1 and h2 (m slots of m+3), y, nrm (2 per step), scale factors, scalars
static size_t small_count(int m) { return (size_t)(m + 1) * m + 2 * m + 2 * (m + 3) + 2 * (size_t)m * (m + 3) + 3 * m + 16; }
static int ints_count(int m) { return 8 + m; }

// Buffers, streams and events of a new context for GMRES(m) with hist_cap history
// entries; on failure the caller frees what was made (free_cache handles any subset).
static die_status init_cache(SolverCache* c, dieop_s* op, int m, int hist_cap, bool own_ws) {
    const long n = vec_len(op);
    c->m_cap = m;
    c->n = n;
    c->hist_cap = hist_cap;
    auto al = [](void** p, size_t b) { return cudaMalloc(p, b) == cudaSuccess; };
    bool ok = al((void**)&c->V, (size_t)(m + 1) * n * sizeof(double2)) &&
              al((void**)&c->Vm, (size_t)(m + 1) * n * sizeof(double)) && al((void**)&c->btil, n * sizeof(double2)) &&
              al((void**)&c->tmp, n * sizeof(double2)) && al((void**)&c->z, n * sizeof(double2)) &&
              al((void**)&c->v32, n * sizeof(float2)) && al((void**)&c->z32, n * sizeof(float2)) &&
              al((void**)&c->small, small_count(m) * sizeof(double2)) &&
              al((void**)&c->hist, (size_t)hist_cap * sizeof(double)) &&
              al((void**)&c->ints, ints_count(m) * sizeof(int)) && al((void**)&c->one, sizeof(double2)) &&
              al((void**)&c->ds.s, (size_t)(kMaxBasis + 2) * sizeof(double2)) &&
              al((void**)&c->ds.c32, (size_t)kMaxBasis * sizeof(float2));
    if (ok && own_ws) {
        c->ws.W_bytes = op->ws.W_bytes;
        c->ws.v_bytes = op->ws.v_bytes;
        ok = al(&c->ws.W, c->ws.W_bytes) && al(&c->ws.v, c->ws.v_bytes);
    }
    if (!ok || cudaHostAlloc((void**)&c->host, 64 * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return DIE_ENOMEM;
    }
    DIE_TRY(alloc_red_scratch(&c->rs));
    DIE_TRY(alloc_red_scratch(&c->ds.rs));
    DIE_TRY(krylov_prepare(m));
    const double2 one = make_double2(1.0, 0.0);
    DIE_CUDA_TRY(cudaMemcpy(c->one, &one, sizeof one, cudaMemcpyHostToDevice));
    DIE_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    DIE_CUDA_TRY(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    for (auto& e : c->join) DIE_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    DIE_CUDA_TRY(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    DIE_CUDA_TRY(cudaEventCreateWithFlags(&c->back, cudaEventDisableTiming));
    return DIE_OK;      // the timing events (gmres_opts.timing) are created on first use
}

// Timing events of gmres_opts.timing: four per Arnoldi step of a cycle.
static die_status ensure_events(SolverCache* c) {
    const size_t need = 4 * (size_t)(c->m_cap + 1);
    if (c->ev.size() >= need) return DIE_OK;
    const size_t have = c->ev.size();
    try {
        c->ev.resize(need);       // null handles until created
    } catch (...) {
        return DIE_ENOMEM;
    }
    for (size_t i = have; i < need; i++) DIE_CUDA_TRY(cudaEventCreate(&c->ev[i]));
    return DIE_OK;
}

die_status ensure_cache(SolverCache** slot, dieop_s* op, int m, int hist_cap, bool own_ws) {
    SolverCache* c = *slot;
    if (c && c->m_cap >= m && c->hist_cap >= hist_cap) return DIE_OK;
    if (c) {
        m = m > c->m_cap ? m : c->m_cap;
        hist_cap = hist_cap > c->hist_cap ? hist_cap : c->hist_cap;
        free_cache(c);
        *slot = nullptr;
    }
    c = new (std::nothrow) SolverCache();
    if (!c) return DIE_ENOMEM;
    const die_status s = init_cache(c, op, m, hist_cap, own_ws);
    if (s != DIE_OK) {            // a context is published only once complete
        free_cache(c);
        return s;
    }
    *slot = c;
    return DIE_OK;
}

die_status ensure_solver_cache(dieop_s* op, int m, int hist_cap) {
    SolverCache* c = solver_cache(op);
    const die_status s = ensure_cache(&c, op, m, hist_cap, false);
    op->solver = c;
    return s;
}

die_status defl_apply(defl_s* d, const double2* x, double2* z, const int* skip, cudaStream_t st, bool live,
                      const DeflScratch* sc) {
    double2* s = sc ? sc->s : d->s;
    const RedScratch& rs = sc ? sc->rs : d->rs;
    DIE_TRY(k_dots(d->V, d->n, d->r, x, d->n, 0, s, rs, skip, st, live));
    DIE_TRY(k_defl_update(d->V, d->n, d->r, d->M, s, x, z, d->n, skip, st));
    return DIE_OK;
}

die_status defl_apply32(defl_s* d, float2* x, double2* w, const double* inv, float2* z, const int* skip,
                        cudaStream_t st, bool live, const DeflScratch* sc) {
    double2* s = sc ? sc->s : d->s;
    float2* c32 = sc ? sc->c32 : d->c32;
    const RedScratch& rs = sc ? sc->rs : d->rs;
    DIE_TRY(k_dots32(d->V32, d->n, d->r, x, w, inv, d->n, s, d->M32, c32, rs, skip, st, live));
    DIE_TRY(k_defl_update32(d->V32, d->n, d->r, c32, x, z, d->n, skip, st));
    return DIE_OK;
}

// Atilde in FP64 (restart residuals, right-hand side).
static die_status apply64(dieop_s* op, bool reg, const double2* in, double2* out, cudaStream_t st,
                          const Workspace* ws) {
    return reg ? apply_reg<double, double2>(op, in, out, st, ws)
               : apply_op<double, double2>(op, Contrast::Chi, in, out, st, ws);
}

static die_status apply_inner(dieop_s* op, bool reg, bool mixed, const double2* in, double2* out, const int* skip,
                              cudaStream_t st, const Workspace* ws) {
    if (mixed)
        return reg ? apply_reg_skip<float, double2>(op, in, out, skip, st, ws)
                   : apply_op_skip<float, double2>(op, Contrast::Chi, in, out, skip, st, ws);
    return reg ? apply_reg_skip<double, double2>(op, in, out, skip, st, ws)
               : apply_op_skip<double, double2>(op, Contrast::Chi, in, out, skip, st, ws);
}

// ||v||^2 read back to the host (synchronises the stream).
static die_status norm2_host(SolverCache* c, const double2* v, long n, double2* dev_out, double* host_out,
                             cudaStream_t st) {
    DIE_TRY(k_dots(v, 0, 0, v, n, 1, dev_out, c->rs, nullptr, st));
    DIE_CUDA_TRY(cudaMemcpyAsync(c->host, dev_out, sizeof(double2), cudaMemcpyDeviceToHost, st));
    DIE_CUDA_TRY(cudaStreamSynchronize(st));
    *host_out = c->host[0];
    return DIE_OK;
}

// Keeps a buffer resident in L2 while a solve runs: a persisting access-policy window
// on the solve's stream (a per-context reservation, released and restored on exit).
// Best effort: any refusal leaves caching as it was.
struct L2Pin {
    cudaStream_t st = nullptr;
    bool on = false;
    size_t old_limit = 0;
    L2Pin(cudaStream_t s, const void* base, size_t bytes) : st(s) {
        int dev = 0, max_persist = 0, max_window = 0;
        const char* env = getenv("DIE_L2PIN");
        if (env && env[0] == '0') return;        // DIE_L2PIN=0: no window (A/B timing)
        if (!base || bytes == 0 || cudaGetDevice(&dev) != cudaSuccess) return;
        if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev) != cudaSuccess ||
            max_persist <= 0 || max_window <= 0) {
            cudaGetLastError();
            return;
        }
        if (cudaDeviceGetLimit(&old_limit, cudaLimitPersistingL2CacheSize) != cudaSuccess) { cudaGetLastError(); return; }
        const size_t win = bytes < (size_t)max_window ? bytes : (size_t)max_window;
        const size_t res = win < (size_t)max_persist ? win : (size_t)max_persist;
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, res) != cudaSuccess) { cudaGetLastError(); return; }
        cudaStreamAttrValue a = {};
        a.accessPolicyWindow.base_ptr = const_cast<void*>(base);
        a.accessPolicyWindow.num_bytes = win;
        a.accessPolicyWindow.hitRatio = (float)((double)res / (double)win);
        a.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        a.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        if (cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &a) != cudaSuccess) {
            cudaGetLastError();
            cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
            return;
        }
        on = true;
    }
    ~L2Pin() {
        if (!on) return;
        cudaStreamAttrValue a = {};
        a.accessPolicyWindow.num_bytes = 0;
        cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &a);
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
        cudaGetLastError();
    }
};

static double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace die

using namespace die;

static bool opts_valid(const dieop_s* op, const defl_s* defl, const gmres_opts* o) {
    if (o->restart < 1 || o->restart > kMaxRestart || o->max_iters < 0 || !(o->tol >= 0)) return false;
    if (o->inner != DIE_FP64 && o->inner != DIE_FP32_INNER) return false;
    if (defl && (defl->op_id != op->id || defl->regularized != (o->regularized ? 1 : 0))) return false;
    return true;
}

static int hist_cap_of(const gmres_opts* o) {
    return o->max_iters < (1 << 22) ? (o->max_iters > 0 ? o->max_iters : 1) : (1 << 22);
}

// One solve in context c (its buffers, streams, deflation scratch and, for a batch
// context, its product workspace); pin: use the L2 window for the deflation basis.
// Captured cycles.  A context records the configurations (CycleKey) of the cycles it
// runs; a graph is captured only for a configuration that has already run directly, so
// every kernel of the cycle has been launched once (first-use attribute calls stay out of
// the capture).
static CycleGraph* find_cycle(SolverCache* c, const CycleKey& key) {
    for (CycleGraph& g : c->graphs)
        if (g.used && g.key == key) return &g;
    return nullptr;
}

static void note_cycle(SolverCache* c, const CycleKey& key) {
    CycleGraph& slot = c->graphs[c->next_graph];
    if (slot.exec) cudaGraphExecDestroy(slot.exec);
    slot.exec = nullptr;
    slot.key = key;
    slot.used = true;
    c->next_graph = (c->next_graph + 1) % kCycleGraphs;
}

// Captures `steps` from `st` (with the side stream they fork to and join back from) into
// g->exec.
template <typename F>
static die_status capture_cycle(CycleGraph* g, cudaStream_t st, F&& steps) {
    DIE_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const die_status s = steps();
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s != DIE_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (s != DIE_OK) return s;
        set_last_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        return DIE_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        set_last_cuda_error(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
        return DIE_ECUDA;
    }
    g->exec = exec;
    return DIE_OK;
}

static die_status solve_ctx(dieop_s* op, defl_s* defl, const gmres_opts* o, const void* b_, void* x_,
                            gmres_report* rep, cudaStream_t ust, SolverCache* c, bool pin) {
    const auto t0 = std::chrono::steady_clock::now();
    const bool reg = o->regularized != 0, mixed = o->inner == DIE_FP32_INNER;
    const double eta = o->reorth_eta > 0 ? o->reorth_eta : default_reorth_eta(o->restart);
    const double eta2 = eta >= 1.0 ? 1.0 : eta * eta;
    const int m = o->restart;
    const long n = vec_len(op);
    const Workspace* pws = c->ws.W ? &c->ws : nullptr;
    // The solve runs on the library's own stream, ordered after the caller's stream at
    // entry and before it at every exit (a stream of its own can carry the L2
    // access-policy window below, which the legacy default stream cannot).
    cudaStream_t st = c->stream, side = c->side;
    DIE_CUDA_TRY(cudaEventRecord(c->join[0], ust));
    DIE_CUDA_TRY(cudaStreamWaitEvent(st, c->join[0], 0));
    // at every exit: the side stream joins the solve's stream, which joins the caller's
    struct Join {
        cudaStream_t side, from, to;
        cudaEvent_t back, ev;
        ~Join() {
            if (cudaEventRecord(back, side) == cudaSuccess) cudaStreamWaitEvent(from, back, 0);
            if (cudaEventRecord(ev, from) == cudaSuccess) cudaStreamWaitEvent(to, ev, 0);
        }
    } join{side, st, ust, c->back, c->join[1]};
    const double2* b = (const double2*)b_;
    double2* x = (double2*)x_;

    // device state of a cycle
    double2* sm = c->small;
    GmresDev S;
    S.H = sm; sm += (size_t)(m + 1) * m;
    S.cs = sm; sm += m;
    S.sn = sm; sm += m;
    S.g = sm; sm += m + 3;
    S.h1 = sm; sm += (size_t)m * (m + 3);
    S.h2 = sm; sm += (size_t)m * (m + 3);
    S.y = sm; sm += m + 3;
    S.nrm = sm; sm += 2 * m;
    S.inv = reinterpret_cast<double*>(sm); sm += m;
    double2* scal = sm;            // scalars: [0] residual norm^2, [1].x ||btilde||
    S.bnorm = &scal[1].x;
    S.hist = c->hist;
    S.done = c->ints;
    S.k = c->ints + 1;
    S.flags = c->ints + 2;
    S.skip2 = c->ints + 3;
    S.nreorth = c->ints + 4;
    S.step0 = c->ints + 5;
    S.reorth = c->ints + 8;
    S.m = m;
    S.jmax = m;
    S.hist_cap = c->hist_cap;
    S.tol = o->tol;
    DIE_CUDA_TRY(cudaMemsetAsync(c->ints, 0, ints_count(m) * sizeof(int), st));
    if (o->timing) DIE_TRY(ensure_events(c));

    // right-hand side of the solved system
    const double2* bt = b;
    int n_apply = 0;
    if (reg) {
        DIE_TRY(apply_op<double, double2>(op, Contrast::ChiReg, b, c->btil, st, pws));
        bt = c->btil;
        n_apply++;
    }
    double bn2 = 0;
    DIE_TRY(norm2_host(c, bt, n, scal, &bn2, st));
    const double bnorm = sqrt(bn2);
    if (!isfinite(bnorm)) return DIE_ENAN;
    if (!o->use_x0) DIE_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double2), st));
    const double bnorm_ref = bnorm > 0 ? bnorm : 1.0;

    die_status status = DIE_ENOCONV;
    int iters = 0, cycles = 0, hist_len = 0, graph_cycles = 0;
    // per-launch event timing cannot be captured into a graph
    const bool use_graph = o->graph && !o->timing && !g_prof_on;
    double rel = 0, t_mv = 0, t_orth = 0, t_defl = 0;
    const long ldv = n;
    double2* V = c->V;
    // FP32-inner with deflation: P^-1 v_j and the product input stay complex64; the
    // deflation projections of step j normalise v_j (scaled by 1 / ||w|| of step j-1)
    // and keep its complex64 copy.
    const bool defl32 = defl && mixed;
    float2* v32 = defl32 ? c->v32 : nullptr;
    // For r <= kDeflFoldMax the deflation projections of v_{j+1} are folded into the
    // Gram-Schmidt update of step j (which produces cf for step j+1), and the deflation
    // update of step j+1 normalises v_{j+1}; otherwise they run as their own pass.
    const bool fold = defl32 && defl->r <= kDeflFoldMax;
    const bool fold_product = fold && defl_product_ok(op);   // deflation inside the first row pass
    // Update passes in the three-multiplication form: every kernel that normalises a basis
    // vector also stores its Re - Im in c->Vm (all paths but the separate complex64
    // projection pass of r > kDeflFoldMax).
    double* Vm = (defl32 && !fold) ? nullptr : c->Vm;
    DeflProj dp;
    if (fold) {
        dp.V32 = defl->V32;
        dp.ld = n;
        dp.r = defl->r;
        dp.M32 = defl->M32;
        dp.s = c->ds.s;
        dp.cf = c->ds.c32;
    }
    // the complex64 deflation basis is read twice per Arnoldi step: keep it in L2
    L2Pin l2pin(st, pin && defl32 ? defl->V32 : nullptr, defl32 ? (size_t)defl->r * n * sizeof(float2) : 0);
    if (bnorm == 0.0) {
        DIE_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double2), st));
        status = DIE_OK;
    }
    // Cycles start single-pass: the second Gram-Schmidt pass is almost never needed, so
    // its kernels are not launched; a cycle in which one would have been needed stops and
    // runs again with the DGKS passes (identical to running it that way from the start),
    // and the solve keeps them from then on.
    bool optimistic = eta2 < 1.0;
    while (status == DIE_ENOCONV) {
        // r = btilde - Atilde x in FP64 into V_0
        if (cycles == 0 && !o->use_x0) {
            DIE_CUDA_TRY(cudaMemcpyAsync(V, bt, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        } else {
            DIE_TRY(apply64(op, reg, x, c->tmp, st, pws));
            n_apply += reg ? 2 : 1;
            DIE_TRY(k_sub(bt, c->tmp, V, n, st));
        }
        double beta2 = 0;
        DIE_TRY(norm2_host(c, V, n, scal, &beta2, st));
        rel = sqrt(beta2) / bnorm;
        if (!isfinite(rel)) { status = DIE_ENAN; break; }
        if (rel <= o->tol) { status = DIE_OK; break; }
        if (iters >= o->max_iters) break;
        DIE_TRY(k_scale_inv_sqrt(V, n, scal, nullptr, st, v32, Vm));
        int hk[8];
        const int jmax = m < o->max_iters - iters ? m : o->max_iters - iters;
        S.jmax = jmax;
        DIE_TRY(k_cycle_scalars(S, bnorm_ref, iters, st));
        for (;;) {   // one cycle; a single-pass cycle that met a needed second pass runs again
        // The Arnoldi steps of the cycle: launched directly, or captured once as a graph.
        auto steps = [&]() -> die_status {
        if (fold)   // cf for v_0
            DIE_TRY(k_dots32(defl->V32, n, defl->r, c->v32, nullptr, nullptr, n, c->ds.s, defl->M32, c->ds.c32,
                             c->ds.rs, nullptr, st));
        DIE_TRY(k_gmres_init(S, scal, st));
        // Step j: v_j = w_{j-1} / ||w_{j-1}|| (j > 0), w = Atilde P^-1 v_j, Gram-Schmidt
        // against v_0..v_j on this stream; the Givens step of j then runs on the side
        // stream while step j+1 starts.  The done flag it sets is read by the kernels
        // of later steps as a live skip flag.
        for (int j = 0; j < jmax; j++) {
            double2* vj = V + (long)j * ldv;
            double2* w = V + (long)(j + 1) * ldv;
            const double* inv_prev = j > 0 ? S.inv + (j - 1) : nullptr;
            if (o->timing) DIE_CUDA_TRY(cudaEventRecord(c->ev[4 * j], st));
            if (fold_product) {
                DeflIn din;
                din.V32 = defl->V32;
                din.ld = n;
                din.r = defl->r;
                din.cf = c->ds.c32;
                din.x = c->v32;
                din.w = j > 0 ? vj : nullptr;
                din.inv = inv_prev;
                din.wm = j > 0 && Vm ? Vm + (long)j * ldv : nullptr;
                if (o->timing) DIE_CUDA_TRY(cudaEventRecord(c->ev[4 * j + 1], st));
                DIE_TRY(apply_defl_xy(op, din, c->z32, w, reg, S.done, st, pws));
            } else if (fold) {
                DIE_TRY(k_defl_update32(defl->V32, n, defl->r, c->ds.c32, c->v32, c->z32, n, S.done, st,
                                        j > 0 ? vj : nullptr, inv_prev, j > 0 && Vm ? Vm + (long)j * ldv : nullptr));
                if (o->timing) DIE_CUDA_TRY(cudaEventRecord(c->ev[4 * j + 1], st));
                DIE_TRY(reg ? apply_reg_skip_xy<float, float2, double2>(op, c->z32, w, S.done, st, pws)
                            : apply_op_skip_xy<float, float2, double2>(op, Contrast::Chi, c->z32, w, S.done, st, pws));
            } else if (defl32) {
                DIE_TRY(defl_apply32(defl, c->v32, j > 0 ? vj : nullptr, inv_prev, c->z32, S.done, st, true, &c->ds));
                if (o->timing) DIE_CUDA_TRY(cudaEventRecord(c->ev[4 * j + 1], st));
                DIE_TRY(reg ? apply_reg_skip_xy<float, float2, double2>(op, c->z32, w, S.done, st, pws)
                            : apply_op_skip_xy<float, float2, double2>(op, Contrast::Chi, c->z32, w, S.done, st, pws));
            } else {
                if (inv_prev) DIE_TRY(k_scale_by(vj, n, inv_prev, S.done, st, nullptr, Vm ? Vm + (long)j * ldv : nullptr));
                const double2* src = vj;
                if (defl) {
                    DIE_TRY(defl_apply(defl, vj, c->z, S.done, st, true, &c->ds));
                    src = c->z;
                }
                if (o->timing) DIE_CUDA_TRY(cudaEventRecord(c->ev[4 * j + 1], st));
                DIE_TRY(apply_inner(op, reg, mixed, src, w, S.done, st, pws));
            }
            if (o->timing) DIE_CUDA_TRY(cudaEventRecord(c->ev[4 * j + 2], st));
            DIE_TRY(cgs_dgks(V, ldv, j + 1, w, n, S.h1 + (long)j * (m + 3), S.h2 + (long)j * (m + 3), S.nrm + 2 * j,
                             S.reorth + j, S.skip2, S.done, eta2, c->rs, st, S.inv + j, fold ? &dp : nullptr,
                             Vm, optimistic ? S.flags : nullptr, optimistic ? S.done : nullptr));
            if (o->timing) DIE_CUDA_TRY(cudaEventRecord(c->ev[4 * j + 3], st));
            DIE_CUDA_TRY(cudaEventRecord(c->fork, st));
            DIE_CUDA_TRY(cudaStreamWaitEvent(side, c->fork, 0));
            DIE_TRY(k_arnoldi_finish(S, j, side));
        }
        DIE_CUDA_TRY(cudaEventRecord(c->back, side));
        DIE_CUDA_TRY(cudaStreamWaitEvent(st, c->back, 0));
        return DIE_OK;
        };
        CycleKey key;
        key.defl = defl ? defl->id : 0;
        key.jmax = jmax;
        key.m = m;
        key.optimistic = optimistic ? 1 : 0;
        key.reg = reg ? 1 : 0;
        key.mixed = mixed ? 1 : 0;
        key.fold = fold ? 1 : 0;
        key.fold_product = fold_product ? 1 : 0;
        key.vm = Vm ? 1 : 0;
        key.tol = o->tol;
        key.eta2 = eta2;
        CycleGraph* g = find_cycle(c, key);
        if (use_graph && g) {
            if (!g->exec) DIE_TRY(capture_cycle(g, st, steps));
            DIE_CUDA_TRY(cudaGraphLaunch(g->exec, st));
            graph_cycles++;
        } else {
            DIE_TRY(steps());
            if (!g) note_cycle(c, key);
        }
        DIE_CUDA_TRY(cudaMemcpyAsync(c->host, c->ints, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
        DIE_CUDA_TRY(cudaStreamSynchronize(st));
        memcpy(hk, c->host, sizeof hk);
        if (optimistic && (hk[2] & 8)) {   // v_0 and the residual are intact: rerun with DGKS passes
            optimistic = false;
            continue;
        }
        break;
        }
        const int k = hk[1], flags = hk[2];
        if (o->timing) {
            for (int j = 0; j < k; j++) {
                float a = 0, bb = 0, cc = 0;
                cudaEventElapsedTime(&a, c->ev[4 * j], c->ev[4 * j + 1]);
                cudaEventElapsedTime(&bb, c->ev[4 * j + 1], c->ev[4 * j + 2]);
                cudaEventElapsedTime(&cc, c->ev[4 * j + 2], c->ev[4 * j + 3]);
                t_defl += a * 1e-3; t_mv += bb * 1e-3; t_orth += cc * 1e-3;
            }
        }
        iters += k;
        n_apply += k * (reg ? 2 : 1);
        hist_len = iters < c->hist_cap ? iters : c->hist_cap;
        cycles++;
        if (flags & 1) { status = DIE_ENAN; break; }
        if (k == 0) { status = DIE_EBREAKDOWN; break; }
        DIE_TRY(k_gmres_lsq(S, st));
        if (defl) {
            DIE_TRY(k_lincomb(V, ldv, k, S.y, nullptr, c->tmp, n, c->rs, st, Vm));
            DIE_TRY(defl_apply(defl, c->tmp, c->tmp, nullptr, st, false, &c->ds));
            DIE_TRY(k_basis_axpy(c->tmp, ldv, 1, c->one, 1.0, x, x, n, nullptr, nullptr, c->rs, nullptr, st));
        } else {
            DIE_TRY(k_lincomb(V, ldv, k, S.y, x, x, n, c->rs, st, Vm));
        }
        // a singular triangular factor (breakdown with no exact solution) shows up after the LSQ
        DIE_CUDA_TRY(cudaMemcpyAsync(c->host, c->ints, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
        DIE_CUDA_TRY(cudaStreamSynchronize(st));
        memcpy(hk, c->host, sizeof hk);
        if (hk[2] & 4) { status = DIE_EBREAKDOWN; break; }
    }
    double rel_orig = rel;
    if (reg && (status == DIE_OK || status == DIE_ENOCONV)) {
        DIE_TRY(apply_op<double, double2>(op, Contrast::Chi, x, c->tmp, st, pws));
        n_apply++;
        DIE_TRY(k_sub(b, c->tmp, c->tmp, n, st));
        double r2 = 0, b2 = 0;
        DIE_TRY(norm2_host(c, c->tmp, n, scal, &r2, st));
        DIE_TRY(norm2_host(c, b, n, scal, &b2, st));
        rel_orig = b2 > 0 ? sqrt(r2 / b2) : 0.0;
    }
    int nre = 0;
    DIE_CUDA_TRY(cudaMemcpyAsync(&nre, S.nreorth, sizeof(int), cudaMemcpyDeviceToHost, st));
    DIE_CUDA_TRY(cudaStreamSynchronize(st));
    if (rep) {
        rep->cycles = cycles;
        rep->iters = iters;
        rep->n_apply = n_apply;
        rep->rel_res_solved = rel;
        rep->rel_res_orig = rel_orig;
        rep->t_matvec = t_mv;
        rep->t_orth = t_orth;
        rep->t_defl = t_defl;
        rep->t_total = seconds_since(t0);
        rep->history_len = 0;
        rep->n_reorth = nre;
        rep->graph_cycles = graph_cycles;
        if (rep->history && rep->history_cap > 0 && hist_len > 0) {
            const int cnt = hist_len < rep->history_cap ? hist_len : rep->history_cap;
            DIE_CUDA_TRY(cudaMemcpy(rep->history, c->hist, cnt * sizeof(double), cudaMemcpyDeviceToHost));
            rep->history_len = cnt;
        }
    }
    return status;
}

extern "C" die_status gmres_basis(dieop_t op, int first, int count, void* out, void* stream) {
    if (!op || !out || first < 0 || count < 1) return DIE_EINVAL;
    SolverCache* c = solver_cache(op);
    if (!c || (long)first + count > (long)c->m_cap + 1) return DIE_EINVAL;
    DIE_CUDA_TRY(cudaMemcpyAsync(out, c->V + (long)first * c->n, (size_t)count * c->n * sizeof(double2),
                                 cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return DIE_OK;
}

extern "C" die_status gmres_solve(dieop_t op, defl_t defl, const gmres_opts* o, const void* b_, void* x_,
                                  gmres_report* rep, void* stream) {
    if (!op || !o || !b_ || !x_) return DIE_EINVAL;
    if (!opts_valid(op, defl, o)) return DIE_EINVAL;
    try {                         // host allocation failure: no exception crosses the C ABI
        DIE_TRY(ensure_solver_cache(op, o->restart, hist_cap_of(o)));
        return solve_ctx(op, defl, o, b_, x_, rep, (cudaStream_t)stream, solver_cache(op), true);
    } catch (...) {
        return DIE_ENOMEM;
    }
}

// Right-hand sides solved concurrently: one context (buffers, product workspace, deflation
// scratch, streams) and one host thread per right-hand side, so that the FP64-bound
// Gram-Schmidt passes of one system and the FFT passes of another share the GPU.
static die_status solve_batch_impl(dieop_s* op, defl_s* defl, const gmres_opts* o, int nrhs, const void* b_,
                                   void* x_, gmres_report* reps, void* stream) {
    const long n = vec_len(op);
    for (int k = 0; k < nrhs; k++) {
        SolverCache* c = reinterpret_cast<SolverCache*>(op->batch[k]);
        const die_status s = ensure_cache(&c, op, o->restart, hist_cap_of(o), true);
        op->batch[k] = c;
        if (s != DIE_OK) return s;
    }
    int dev = 0;
    DIE_CUDA_TRY(cudaGetDevice(&dev));
    std::vector<die_status> status(nrhs, DIE_OK);
    std::vector<std::thread> threads;
    threads.reserve(nrhs);
    for (int k = 0; k < nrhs; k++) {
        try {
            threads.emplace_back([&, k] {
                try {
                    if (cudaSetDevice(dev) != cudaSuccess) { status[k] = DIE_ECUDA; return; }
                    status[k] = solve_ctx(op, defl, o, (const double2*)b_ + k * n, (double2*)x_ + k * n,
                                          reps ? reps + k : nullptr, (cudaStream_t)stream,
                                          reinterpret_cast<SolverCache*>(op->batch[k]), false);
                } catch (...) {
                    status[k] = DIE_ENOMEM;
                }
            });
        } catch (...) {           // no thread for systems k .. nrhs - 1
            for (int q = k; q < nrhs; q++) status[q] = DIE_ENOMEM;
            break;
        }
    }
    for (auto& t : threads) t.join();
    die_status out = DIE_OK;
    for (die_status s : status)
        if (s != DIE_OK && s != DIE_ENOCONV) return s;
        else if (s == DIE_ENOCONV) out = DIE_ENOCONV;
    return out;
}

extern "C" die_status gmres_solve_batch(dieop_t op, defl_t defl, const gmres_opts* o, int nrhs, const void* b_,
                                        void* x_, gmres_report* reps, void* stream) {
    if (!op || !o || !b_ || !x_ || nrhs < 1 || nrhs > kMaxBatchSolve) return DIE_EINVAL;
    if (!opts_valid(op, defl, o)) return DIE_EINVAL;
    try {                         // host allocation failure before the threads start
        return solve_batch_impl(op, defl, o, nrhs, b_, x_, reps, stream);
    } catch (...) {
        return DIE_ENOMEM;
    }
}

// Systems of different operators (grid sizes) solved concurrently: up to kMaxBatchSolve
// host threads take the systems in order from a shared counter.  A thread solves in the
// first batch context of the system's operator that no other thread holds at that
// moment, so an operator keeps only as many contexts as it had systems in flight.
static die_status solve_many_impl(int count, const dieop_t* ops, const defl_t* defls, const gmres_opts* o,
                                  const void* const* b, void* const* x, gmres_report* reps, void* stream) {
    int dev = 0;
    DIE_CUDA_TRY(cudaGetDevice(&dev));
    std::vector<dieop_s*> uniq;             // distinct operators, and the slots held in each
    std::vector<unsigned> held;
    std::vector<int> which(count);
    for (int k = 0; k < count; k++) {
        int u = 0;
        while (u < (int)uniq.size() && uniq[u] != ops[k]) u++;
        if (u == (int)uniq.size()) {
            uniq.push_back(ops[k]);
            held.push_back(0u);
        }
        which[k] = u;
    }
    const int nthreads = count < kMaxBatchSolve ? count : kMaxBatchSolve;
    std::mutex mu;
    std::vector<die_status> status(count, DIE_OK);
    std::atomic<int> next{0};
    std::atomic<bool> no_device{false};
    std::vector<std::thread> threads;
    threads.reserve(nthreads);
    for (int w = 0; w < nthreads; w++) {
        try {
            threads.emplace_back([&] {
                if (cudaSetDevice(dev) != cudaSuccess) { no_device = true; return; }
                for (int k = next.fetch_add(1); k < count; k = next.fetch_add(1)) {
                    dieop_s* op = ops[k];
                    const int u = which[k];
                    int slot = 0;
                    {   // at most nthreads <= kMaxBatchSolve slots are held at once: one is free
                        std::lock_guard<std::mutex> lock(mu);
                        while (held[u] & (1u << slot)) slot++;
                        held[u] |= 1u << slot;
                    }
                    die_status s;
                    try {
                        SolverCache* c = reinterpret_cast<SolverCache*>(op->batch[slot]);
                        s = ensure_cache(&c, op, o->restart, hist_cap_of(o), true);
                        op->batch[slot] = c;
                        if (s == DIE_OK)
                            s = solve_ctx(op, defls ? defls[k] : nullptr, o, b[k], x[k], reps ? reps + k : nullptr,
                                          (cudaStream_t)stream, c, false);
                    } catch (...) {
                        s = DIE_ENOMEM;
                    }
                    status[k] = s;
                    std::lock_guard<std::mutex> lock(mu);
                    held[u] &= ~(1u << slot);
                }
            });
        } catch (...) {           // fewer threads: the ones running take every system
            break;
        }
    }
    if (threads.empty()) return DIE_ENOMEM;
    for (auto& t : threads) t.join();
    if (no_device) return DIE_ECUDA;
    die_status out = DIE_OK;
    for (die_status s : status)
        if (s != DIE_OK && s != DIE_ENOCONV) return s;
        else if (s == DIE_ENOCONV) out = DIE_ENOCONV;
    return out;
}

extern "C" die_status gmres_solve_many(int count, const dieop_t* ops, const defl_t* defls, const gmres_opts* o,
                                       const void* const* b, void* const* x, gmres_report* reps, void* stream) {
    if (count < 1 || !ops || !o || !b || !x) return DIE_EINVAL;
    for (int k = 0; k < count; k++) {
        if (!ops[k] || !b[k] || !x[k]) return DIE_EINVAL;
        if (!opts_valid(ops[k], defls ? defls[k] : nullptr, o)) return DIE_EINVAL;
    }
    try {                         // host allocation failure before the threads start
        return solve_many_impl(count, ops, defls, o, b, x, reps, stream);
    } catch (...) {
        return DIE_ENOMEM;
    }
}
