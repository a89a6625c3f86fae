// Flexible GMRES (Saad, SIAM J. Sci. Comput. 14, 1993) on A x = b with the learned right
// preconditioner of die_fno.h: step j applies z_j = M(v_j) (the network), keeps z_j,
// and extends the Arnoldi relation A Z_j = V_{j+1} H_j; the cycle ends with
// x += Z_k y, y the minimiser of || beta e1 - H y ||.  Products and Arnoldi are FP64 on
// the device (the product kernels and classical Gram-Schmidt with the DGKS criterion of
// the restarted solver); the Givens rotations of the small least-squares problem run on
// the host (one step per network evaluation, which synchronises anyway).  If the flexible
// iteration has not converged within its budget, the regularised and deflated restarted
// GMRES of Sections 4-5 continues from its iterate.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/die_fno.h"
#include "solver.cuh"

namespace die {
die_status fno_apply_precond(fno_s* f, dieop_s* op, const double2* v, double2* z, cudaStream_t st);
bool fno_matches(const fno_s* f, const dieop_s* op);
}  // namespace die

using namespace die;

namespace {

struct FgmresWork {
    double2 *V = nullptr, *Z = nullptr, *tmp = nullptr, *small = nullptr;
    double* inv = nullptr;
    int* ints = nullptr;
    RedScratch rs;
    ~FgmresWork() {
        for (void* p : {(void*)V, (void*)Z, (void*)tmp, (void*)small, (void*)inv, (void*)ints})
            if (p) cudaFree(p);
        free_red_scratch(&rs);
    }
};

die_status norm2(FgmresWork& w, const double2* v, long n, cudaStream_t st, double* out) {
    DIE_TRY(k_dots(v, 0, 0, v, n, 1, w.small, w.rs, nullptr, st));
    double2 h;
    DIE_CUDA_TRY(cudaMemcpyAsync(&h, w.small, sizeof h, cudaMemcpyDeviceToHost, st));
    DIE_CUDA_TRY(cudaStreamSynchronize(st));
    *out = h.x;
    return DIE_OK;
}

die_status fgmres_impl(dieop_s* op, fno_s* net, const gmres_opts* o, const double2* b, double2* x,
                       gmres_report* rep, cudaStream_t st, bool* nan_out) {
    const int m = o->restart;
    const long n = vec_len(op);
    FgmresWork w;
    auto al = [](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    if (!al((void**)&w.V, (size_t)(m + 1) * n * sizeof(double2)) || !al((void**)&w.Z, (size_t)m * n * sizeof(double2)) ||
        !al((void**)&w.tmp, n * sizeof(double2)) || !al((void**)&w.small, (size_t)(3 * m + 16) * sizeof(double2)) ||
        !al((void**)&w.inv, sizeof(double)) || !al((void**)&w.ints, 4 * sizeof(int))) {
        cudaGetLastError();
        return DIE_ENOMEM;
    }
    DIE_TRY(alloc_red_scratch(&w.rs));
    DIE_CUDA_TRY(cudaMemsetAsync(w.ints, 0, 4 * sizeof(int), st));
    double2* h1 = w.small + 4;           // m + 3 slots each
    double2* h2 = h1 + (m + 3);
    double2* nrm = h2 + (m + 3);         // 2 slots
    const double eta = o->reorth_eta > 0 ? o->reorth_eta : default_reorth_eta(m);
    const double eta2 = eta >= 1.0 ? 1.0 : eta * eta;

    double bn2 = 0;
    DIE_TRY(norm2(w, b, n, st, &bn2));
    const double bnorm = sqrt(bn2);
    *nan_out = false;
    if (!isfinite(bnorm)) { *nan_out = true; return DIE_ENAN; }
    if (!o->use_x0) {
        if (net && bnorm > 0) DIE_TRY(fno_apply_precond(net, op, b, x, st));
        else DIE_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double2), st));
    }
    if (bnorm == 0) {
        DIE_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double2), st));
        if (rep) { rep->rel_res_solved = rep->rel_res_orig = 0; }
        return DIE_OK;
    }
    std::vector<double2> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 2), col(m + 2), y(m);
    int iters = 0, cycles = 0;
    die_status status = DIE_ENOCONV;
    double rel = 0;
    for (;;) {
        DIE_TRY(apply_op<double, double2>(op, Contrast::Chi, x, w.tmp, st));
        DIE_TRY(k_sub(b, w.tmp, w.V, n, st));
        double beta2 = 0;
        DIE_TRY(norm2(w, w.V, n, st, &beta2));
        rel = sqrt(beta2) / bnorm;
        if (!isfinite(rel)) { *nan_out = true; status = DIE_ENAN; break; }
        if (rel <= o->tol) { status = DIE_OK; break; }
        if (iters >= o->max_iters) break;
        DIE_TRY(k_scale_inv_sqrt(w.V, n, w.small, nullptr, st));
        std::fill(g.begin(), g.end(), make_double2(0, 0));
        g[0] = make_double2(sqrt(beta2), 0);
        int k = 0;
        bool bad = false;
        for (int j = 0; j < m && iters < o->max_iters; j++) {
            double2* vj = w.V + (long)j * n;
            double2* zj = w.Z + (long)j * n;
            double2* wv = w.V + (long)(j + 1) * n;
            if (net) DIE_TRY(fno_apply_precond(net, op, vj, zj, st));
            else DIE_CUDA_TRY(cudaMemcpyAsync(zj, vj, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            DIE_TRY(apply_op<double, double2>(op, Contrast::Chi, zj, wv, st));
            iters++;
            DIE_TRY(cgs_dgks(w.V, n, j + 1, wv, n, h1, h2, nrm, w.ints, w.ints + 1, nullptr, eta2, w.rs, st, w.inv));
            // the new column: h1 (+ h2 when the second pass ran), ||w|| after the last pass
            int re = 0;
            DIE_CUDA_TRY(cudaMemcpyAsync(col.data(), h1, (j + 2) * sizeof(double2), cudaMemcpyDeviceToHost, st));
            DIE_CUDA_TRY(cudaMemcpyAsync(&re, w.ints, sizeof(int), cudaMemcpyDeviceToHost, st));
            double2 nr[2];
            DIE_CUDA_TRY(cudaMemcpyAsync(nr, nrm, sizeof nr, cudaMemcpyDeviceToHost, st));
            std::vector<double2> c2;
            DIE_CUDA_TRY(cudaStreamSynchronize(st));
            if (re) {
                c2.resize(j + 1);
                DIE_CUDA_TRY(cudaMemcpy(c2.data(), h2, (j + 1) * sizeof(double2), cudaMemcpyDeviceToHost));
                for (int i = 0; i <= j; i++) col[i] = make_double2(col[i].x + c2[i].x, col[i].y + c2[i].y);
            }
            const double hn = sqrt(fmax(re ? nr[1].x : nr[0].x, 0.0));
            double2* Hc = &H[(size_t)j * (m + 1)];
            for (int i = 0; i <= j; i++) Hc[i] = col[i];
            givens_column(Hc, cs.data(), sn.data(), j, hn, &cs[j], &sn[j], g.data());
            k = j + 1;
            const double est = hypot(g[j + 1].x, g[j + 1].y) / bnorm;
            if (!isfinite(est) || !isfinite(hn)) { bad = true; break; }
            if (est <= o->tol || hn == 0.0) break;
            DIE_TRY(k_scale_by(wv, n, w.inv, nullptr, st));
        }
        cycles++;
        if (bad) { *nan_out = true; status = DIE_ENAN; break; }
        if (k == 0) break;
        // R y = g, back substitution (R: the rotated H)
        for (int i = k - 1; i >= 0; i--) {
            double2 s = g[i];
            for (int q = i + 1; q < k; q++) s = csub(s, cmul(H[(size_t)q * (m + 1) + i], y[q]));
            const double2 d = H[(size_t)i * (m + 1) + i];
            const double dd = d.x * d.x + d.y * d.y;
            if (dd == 0.0) return DIE_EBREAKDOWN;
            y[i] = cmul(s, make_double2(d.x / dd, -d.y / dd));
        }
        DIE_CUDA_TRY(cudaMemcpyAsync(w.small, y.data(), k * sizeof(double2), cudaMemcpyHostToDevice, st));
        DIE_TRY(k_lincomb(w.Z, n, k, w.small, x, x, n, w.rs, st));
    }
    if (rep) {
        rep->cycles = cycles;
        rep->iters = iters;
        rep->n_apply = iters + cycles + 1;
        rep->rel_res_solved = rel;
        rep->rel_res_orig = rel;
        rep->history_len = 0;
        rep->n_reorth = 0;
        rep->graph_cycles = 0;
    }
    return status;
}

}  // namespace

extern "C" die_status fgmres_solve(dieop_t op, fno_t net, defl_t defl, const gmres_opts* o, int fallback_restart,
                                   int fallback_iters, const void* b, void* x, gmres_report* rep, int* used_fallback,
                                   void* stream) {
    if (!op || !o || !b || !x) return DIE_EINVAL;
    if (o->restart < 1 || o->restart > 256 || o->max_iters < 0 || !(o->tol >= 0)) return DIE_EINVAL;
    if (net && !fno_matches(net, op)) return DIE_EINVAL;
    if (fallback_iters > 0 && (fallback_restart < 1 || fallback_restart > kMaxRestart)) return DIE_EINVAL;
    if (defl && (defl->op_id != op->id || !defl->regularized)) return DIE_EINVAL;
    if (used_fallback) *used_fallback = 0;
    cudaStream_t st = (cudaStream_t)stream;
    gmres_report r1{};
    bool nan = false;
    die_status s;
    try {
        s = fgmres_impl(op, net, o, (const double2*)b, (double2*)x, &r1, st, &nan);
    } catch (...) {
        return DIE_ENOMEM;
    }
    if (s != DIE_OK && s != DIE_ENOCONV && s != DIE_ENAN) return s;
    if (s != DIE_OK && fallback_iters > 0) {
        if (used_fallback) *used_fallback = 1;
        gmres_opts fo = *o;
        fo.restart = fallback_restart;
        fo.max_iters = fallback_iters;
        fo.regularized = 1;
        fo.inner = DIE_FP32_INNER;
        fo.use_x0 = nan ? 0 : 1;       // a NaN iterate is not a starting point
        fo.graph = 0;
        fo.timing = 0;
        // the regularised solve stops on its own residual ||A_R (b - A x)|| / ||A_R b||: tighten
        // its tolerance (up to 1000x) until ||b - A x|| / ||b|| meets tol
        int left = fallback_iters;
        for (int tries = 0; tries < 4 && left > 0; tries++) {
            gmres_report r2{};
            fo.max_iters = left;
            s = gmres_solve(op, defl, &fo, b, x, &r2, stream);
            if (s != DIE_OK && s != DIE_ENOCONV) return s;
            r1.cycles += r2.cycles;
            r1.iters += r2.iters;
            r1.n_apply += r2.n_apply;
            r1.rel_res_solved = r2.rel_res_orig;
            r1.rel_res_orig = r2.rel_res_orig;
            left -= r2.iters;
            if (r2.rel_res_orig <= o->tol || s == DIE_ENOCONV) break;
            fo.tol *= 0.1;
            fo.use_x0 = 1;
        }
        s = r1.rel_res_orig <= o->tol ? DIE_OK : DIE_ENOCONV;
    }
    if (rep) {
        double* hist = rep->history;
        const int cap = rep->history_cap;
        *rep = r1;
        rep->history = hist;
        rep->history_cap = cap;
        rep->history_len = 0;
    }
    return s;
}
