// Workspaces of restarted GMRES and the deflation handle.
#pragma once

#include <vector>

#include "krylov.cuh"
#include "op.cuh"

namespace die {

// Scratch of one deflation apply: projections (r + 2), complex64 coefficients (r) and
// the reduction scratch.  A solver context owns one, so that concurrent solves can share
// a deflation handle.
struct DeflScratch {
    double2* s = nullptr;
    float2* c32 = nullptr;
    RedScratch rs;
};

constexpr int kMaxBatchSolve = 16;   // right-hand sides of one gmres_solve_batch call

// Device buffers reused across gmres_solve calls on one operator (one context), or by one
// right-hand side of gmres_solve_batch (a batch context, with its own product workspace).
// What a captured cycle (gmres_opts.graph) depends on besides the context's own buffers.
struct CycleKey {
    uint64_t defl = 0;          // deflation handle identity (0: none)
    int jmax = 0, m = 0, optimistic = 0, reg = 0, mixed = 0, fold = 0, fold_product = 0, vm = 0;
    double tol = 0, eta2 = 0;
    bool operator==(const CycleKey& o) const {
        return defl == o.defl && jmax == o.jmax && m == o.m && optimistic == o.optimistic && reg == o.reg &&
               mixed == o.mixed && fold == o.fold && fold_product == o.fold_product && vm == o.vm &&
               tol == o.tol && eta2 == o.eta2;
    }
};
struct CycleGraph {
    bool used = false;              // key holds a configuration this context has run
    CycleKey key;
    cudaGraphExec_t exec = nullptr; // its captured cycle, once one has been captured
};
constexpr int kCycleGraphs = 4;

struct SolverCache {
    int m_cap = 0;          // Krylov dimension the buffers hold
    long n = 0;             // vector length 2N
    int hist_cap = 0;
    double2* V = nullptr;   // (m_cap + 1) * n
    double* Vm = nullptr;   // (m_cap + 1) * n: Re - Im of each basis vector (three-multiplication form)
    double2* btil = nullptr;
    double2* tmp = nullptr;
    double2* z = nullptr;
    float2* v32 = nullptr;      // complex64 copy of the current Arnoldi vector (FP32-inner + deflation)
    float2* z32 = nullptr;      // complex64 P^-1 v of the FP32-inner form
    double2* small = nullptr;   // H, cs, sn, g, per-step h1, h2, nrm, scale factors, y, scalars
    double* hist = nullptr;
    int* ints = nullptr;        // done, k, flags, skip2, nreorth, then the per-step DGKS flags
    double2* one = nullptr;     // device constant 1 + 0i
    RedScratch rs;
    double* host = nullptr;     // pinned readback area
    std::vector<cudaEvent_t> ev;
    cudaStream_t stream = nullptr;  // internal stream of the solves (joined to the caller's)
    cudaStream_t side = nullptr;    // Givens steps, one step behind the Arnoldi steps
    cudaEvent_t join[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, back = nullptr;   // stream -> side, side -> stream
    DeflScratch ds;                 // deflation scratch (kMaxBasis + 2 projections)
    Workspace ws;                   // batch contexts: own product workspace (else W == NULL)
    CycleGraph graphs[kCycleGraphs];  // configurations run and their captured cycles, replaced round-robin
    int next_graph = 0;
};

void free_solver_cache(dieop_s* op);   // the operator's context and its batch contexts
SolverCache* solver_cache(dieop_s* op);
die_status ensure_solver_cache(dieop_s* op, int m, int hist_cap);
// A context in *slot with room for GMRES(m) and hist_cap history entries; own_ws: with
// its own product workspace.
die_status ensure_cache(SolverCache** slot, dieop_s* op, int m, int hist_cap, bool own_ws);
die_status alloc_red_scratch(RedScratch* rs);
void free_red_scratch(RedScratch* rs);

}  // namespace die

// Deflation handle: V (r orthonormal vectors of length n) and M = T^-1 - I (Eq. (4.12)).
struct defl_s {
    uint64_t id = 0;            // unique identity of this handle
    uint64_t op_id = 0;
    int device = -1;            // CUDA device the handle's arrays live on
    int r = 0;
    long n = 0;
    int regularized = 0;
    double2* V = nullptr;       // r * n, vector i at V + i * n
    float2* V32 = nullptr;      // complex64 copy of V (FP32-inner solves)
    float2* M32 = nullptr;      // complex64 copy of M (FP32-inner solves)
    float2* c32 = nullptr;      // r coefficients M (V^* x), complex64 (scratch)
    double2* M = nullptr;       // r * r, column-major
    double2* s = nullptr;       // r projections (scratch)
    die::RedScratch rs;
    std::vector<double> eigs;   // (re, im) pairs, |lambda| descending
};

namespace die {
// z = P^-1 x = x + V (M (V^* x)); z may equal x.  `skip`, `live` as for the Krylov kernels;
// sc: scratch (NULL: the handle's own).
die_status defl_apply(defl_s* d, const double2* x, double2* z, const int* skip, cudaStream_t st, bool live = false,
                      const DeflScratch* sc = nullptr);
// The same entirely in complex64 (copy of V, FP32 sums), for the FP32-inner solves.  With
// inv != NULL the input is first formed from the FP64 vector w: w *= *inv, x = complex64(w).
die_status defl_apply32(defl_s* d, float2* x, double2* w, const double* inv, float2* z, const int* skip,
                        cudaStream_t st, bool live = false, const DeflScratch* sc = nullptr);
}  // namespace die
