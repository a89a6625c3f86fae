// Deflating right preconditioner of Eqs. (4.12)-(4.13):
//   P^-1 = I + V (T^-1 - I) V^*,  T = V^* Atilde V,
// V = orthonormal basis of the invariant subspace of the r largest-magnitude
// eigenvalues of Atilde.  The paper obtains the eigenvectors with Matlab's eigs at
// tolerance 1e-4 and orthonormalises them (Section 5); here the Krylov-Schur method
// (Stewart 2002) computes the Schur vectors of that subspace directly, which span
// the same space: Arnoldi expansion with the device products and CGS2, a small
// FP64 Schur decomposition of the Rayleigh quotient on the device, reordering by
// |lambda|, truncation and basis rotation, until the leading r Schur vectors have
// residual coefficients |b_i| <= tol |T_ii|.
#include <math.h>
#include <string.h>

#include <vector>

#include "small_dense.cuh"
#include "solver.cuh"

namespace die {

// counter-based start vector: splitmix64 of (seed, index) -> uniform(-1, 1) parts
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void random_vector_kernel(double2* v, long n, uint64_t seed) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const uint64_t a = splitmix64(seed * 0x100000001B3ull + 2 * (uint64_t)i);
        const uint64_t b = splitmix64(seed * 0x100000001B3ull + 2 * (uint64_t)i + 1);
        v[i] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, (double)(b >> 11) * 0x1.0p-52 - 1.0);
    }
}

// out_l = sum_i Q_i Z(i, l) for l < k (out-of-place basis rotation), Z p x k column-major, ld = ldz.
__global__ void rotate_basis_kernel(const double2* __restrict__ Q, long ldq, int p, const double2* __restrict__ Z,
                                    int ldz, int k, double2* __restrict__ out, long n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* zs = reinterpret_cast<double2*>(smem_raw);    // p * k
    for (int e = threadIdx.x; e < p * k; e += blockDim.x) {
        const int i = e % p, l = e / p;
        zs[e] = Z[(long)l * ldz + i];
    }
    __syncthreads();
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
        for (int l = 0; l < k; l++) {
            double2 acc = make_double2(0, 0);
            for (int i = 0; i < p; i++) acc = cadd(acc, cmul(Q[(long)i * ldq + idx], zs[(long)l * p + i]));
            out[(long)l * ldq + idx] = acc;
        }
    }
}

// out_l = sum_i Q_i Z(i, l) for l < k (Z: p x k, column-major, ld = p), in column chunks
// whose p x chunk block of Z fits the kernel's shared memory (so any p, k up to the
// largest Krylov dimension run).
static die_status rotate_basis(const double2* Q, long n, int p, const double2* Z, int k, double2* out, cudaStream_t st) {
    constexpr size_t kSmemCap = 200 * 1024;
    int kc = (int)(kSmemCap / ((size_t)p * sizeof(double2)));
    if (kc < 1) return DIE_EINVAL;
    DIE_CUDA_TRY(cudaFuncSetAttribute(rotate_basis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    for (int l0 = 0; l0 < k; l0 += kc) {
        const int cnt = k - l0 < kc ? k - l0 : kc;
        const size_t smem = (size_t)p * cnt * sizeof(double2);
        rotate_basis_kernel<<<1216, 256, smem, st>>>(Q, n, p, Z + (long)l0 * p, p, cnt, out + (long)l0 * n, n);
        DIE_LAUNCH_CHECK();
    }
    return DIE_OK;
}

// Small eigenproblem of one Krylov-Schur restart, on the host (FP64; the same textbook
// routines run on one GPU thread were 10x slower and made builds with Krylov dimensions
// of a few hundred take minutes).
//   B: (p+1) x p Rayleigh matrix (column-major, ld = p+1); row p holds beta e_{p-1}.
//   Outputs: T (p x p Schur form, |T_ii| descending, ld = p), Z (p x p, ld = p),
//   bvec (p): residual coefficients beta Z(p-1, :).  Returns 0, or -1 if the QR iteration
//   did not converge.
static int ks_small_host(const double2* B, int p, double2* T, double2* Z, double2* bvec, std::vector<sd::cd>& work) {
    using sd::cd;
    cd* t = reinterpret_cast<cd*>(T);
    cd* z = reinterpret_cast<cd*>(Z);
    for (int j = 0; j < p; j++)
        for (int i = 0; i < p; i++) {
            const double2 v = B[(long)j * (p + 1) + i];
            t[(long)j * p + i] = cd{v.x, v.y};
            z[(long)j * p + i] = cd{i == j ? 1.0 : 0.0, 0.0};
        }
    work.resize(p);
    sd::hessenberg(t, p, z, p, p, work.data());
    const int rc = sd::schur_qr(t, p, z, p, p, 60);
    if (rc == 0) sd::schur_sort_desc(t, p, z, p, p);
    const double2 beta = B[(long)(p - 1) * (p + 1) + p];
    for (int l = 0; l < p; l++) {
        const cd zz = z[(long)l * p + (p - 1)];
        bvec[l] = make_double2(beta.x * zz.re - beta.y * zz.im, beta.x * zz.im + beta.y * zz.re);
    }
    return rc;
}

// M = T^-1 - I for the r x r matrix T (column-major); status[0] = 0 / -1 (singular).
__global__ void inverse_minus_identity_kernel(double2* T, int r, int* piv, int* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    using sd::cd;
    cd* t = reinterpret_cast<cd*>(T);
    const int rc = sd::invert(t, r, r, piv);
    if (rc == 0)
        for (int i = 0; i < r; i++) t[(long)i * r + i] = t[(long)i * r + i] - cd{1.0, 0.0};
    status[0] = rc;
}

// B(0:k, 0:k) = T(0:k, 0:k), B(k, 0:k) = b(0:k), everything else 0.
__global__ void ks_truncate_kernel(double2* B, int p, const double2* T, const double2* bvec, int k) {
    const long total = (long)(p + 1) * p;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e % (p + 1)), j = (int)(e / (p + 1));
        double2 v = make_double2(0, 0);
        if (j < k) {
            if (i < k) v = T[(long)j * p + i];
            else if (i == k) v = bvec[j];
        }
        B[e] = v;
    }
}

// B(0:j+1, j) = h(0:j+1) (+ h2), B(j+1, j) = sqrt(nrm2)
__global__ void ks_column_kernel(double2* B, int p, int j, const double2* h1, const double2* h2, const double2* nrm2) {
    const int i = threadIdx.x;
    for (int q = i; q <= j; q += blockDim.x) B[(long)j * (p + 1) + q] = cadd(h1[q], h2[q]);
    if (i == 0) B[(long)j * (p + 1) + j + 1] = make_double2(sqrt(fmax(nrm2->x, 0.0)), 0.0);
}

static die_status dalloc(void** p, size_t b) {
    if (cudaMalloc(p, b) != cudaSuccess) { cudaGetLastError(); *p = nullptr; return DIE_ENOMEM; }
    return DIE_OK;
}

}  // namespace die

using namespace die;

static void free_defl(defl_s* d) {
    if (!d) return;
    if (d->V) cudaFree(d->V);
    if (d->M) cudaFree(d->M);
    if (d->V32) cudaFree(d->V32);
    if (d->c32) cudaFree(d->c32);
    if (d->M32) cudaFree(d->M32);
    if (d->s) cudaFree(d->s);
    free_red_scratch(&d->rs);
    delete d;
}

namespace {

struct KsWork {
    double2 *Q = nullptr, *Q2 = nullptr, *B = nullptr, *T = nullptr, *Z = nullptr, *bvec = nullptr, *work = nullptr;
    double2 *h1 = nullptr, *h2 = nullptr, *nrm = nullptr;
    int* ist = nullptr;
    ~KsWork() {
        void* ps[] = {Q, Q2, B, T, Z, bvec, work, h1, h2, nrm, ist};
        for (void* p : ps)
            if (p) cudaFree(p);
    }
};

}  // namespace

static die_status build_impl(dieop_s* op, const defl_opts* o, cudaStream_t st, defl_s* d, double* eig_out,
                             int* r_out) {
    const long n = vec_len(op);
    const bool reg = o->regularized != 0, mixed = o->inner == DIE_FP32_INNER;
    int r = o->r;
    int rmax = o->r_max > 0 ? o->r_max : 64;
    const bool auto_r = r == 0;
    if (auto_r) r = rmax;
    int p = o->krylov_dim > 0 ? o->krylov_dim : (2 * r + 16 > r + 32 ? 2 * r + 16 : r + 32);
    if (o->krylov_dim <= 0 && p + 2 > kMaxBasis) p = kMaxBasis - 2;   // large r: the largest basis
    if (p <= r + 1) p = r + 2;
    if (p + 2 > kMaxBasis) return DIE_EINVAL;
    const double tol = o->tol > 0 ? o->tol : 1e-4;
    const int max_restarts = o->max_restarts > 0 ? o->max_restarts : 200;

    DIE_TRY(ensure_solver_cache(op, 1, 1));
    SolverCache* sc = solver_cache(op);
    KsWork w;
    DIE_TRY(dalloc((void**)&w.Q, (size_t)(p + 1) * n * sizeof(double2)));
    DIE_TRY(dalloc((void**)&w.Q2, (size_t)(p + 1) * n * sizeof(double2)));
    DIE_TRY(dalloc((void**)&w.B, (size_t)(p + 1) * p * sizeof(double2)));
    DIE_TRY(dalloc((void**)&w.T, (size_t)p * p * sizeof(double2)));
    DIE_TRY(dalloc((void**)&w.Z, (size_t)p * p * sizeof(double2)));
    DIE_TRY(dalloc((void**)&w.bvec, (size_t)p * sizeof(double2)));
    DIE_TRY(dalloc((void**)&w.work, (size_t)(p + 1) * sizeof(double2)));
    DIE_TRY(dalloc((void**)&w.h1, (size_t)(p + 2) * sizeof(double2)));
    DIE_TRY(dalloc((void**)&w.h2, (size_t)(p + 2) * sizeof(double2)));
    DIE_TRY(dalloc((void**)&w.nrm, 4 * sizeof(double2)));
    DIE_TRY(dalloc((void**)&w.ist, (size_t)(p + 8) * sizeof(int)));
    DIE_CUDA_TRY(cudaMemsetAsync(w.B, 0, (size_t)(p + 1) * p * sizeof(double2), st));
    const RedScratch& rs = sc->rs;

    auto apply = [&](const double2* in, double2* out) -> die_status {
        if (mixed) return reg ? apply_reg<float, double2>(op, in, out, st) : apply_op<float, double2>(op, Contrast::Chi, in, out, st);
        return reg ? apply_reg<double, double2>(op, in, out, st) : apply_op<double, double2>(op, Contrast::Chi, in, out, st);
    };

    // q_0: seeded random unit vector
    random_vector_kernel<<<1216, 256, 0, st>>>(w.Q, n, o->seed + 1);
    // TM: a start vector in the first plane keeps the Krylov space there (the second plane
    // of a TM field is zero), so every deflated eigenvector is a TM field
    if (op->pol == DIE_TM) DIE_CUDA_TRY(cudaMemsetAsync(w.Q + n / 2, 0, (n / 2) * sizeof(double2), st));
    DIE_LAUNCH_CHECK();
    DIE_TRY(k_dots(w.Q, 0, 0, w.Q, n, 1, w.nrm, rs, nullptr, st));
    DIE_TRY(k_scale_inv_sqrt(w.Q, n, w.nrm, nullptr, st));

    std::vector<double2> T(p * (size_t)p), bv(p), Bh((size_t)(p + 1) * p), Zh(p * (size_t)p);
    std::vector<sd::cd> swork;
    double R_defl = -1.0;             // Section 5 deflation radius (r = 0), computed once
    int k = 0, nconv = 0;
    bool converged = false;
    for (int it = 0; it < max_restarts; it++) {
        for (int j = k; j < p; j++) {
            double2* qj = w.Q + (long)j * n;
            double2* wv = w.Q + (long)(j + 1) * n;
            DIE_TRY(apply(qj, wv));
            DIE_TRY(cgs_dgks(w.Q, n, j + 1, wv, n, w.h1, w.h2, w.nrm, w.ist + 1, w.ist + 2, nullptr, 1.0, rs, st));
            ks_column_kernel<<<1, 128, 0, st>>>(w.B, p, j, w.h1, w.h2, w.nrm + 1);
            DIE_LAUNCH_CHECK();
            DIE_TRY(k_scale_inv_sqrt(wv, n, w.nrm + 1, nullptr, st));
        }
        DIE_CUDA_TRY(cudaMemcpyAsync(Bh.data(), w.B, Bh.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
        DIE_CUDA_TRY(cudaStreamSynchronize(st));
        const int rc = ks_small_host(Bh.data(), p, T.data(), Zh.data(), bv.data(), swork);
        if (rc != 0) return DIE_ENOCONV;
        DIE_CUDA_TRY(cudaMemcpyAsync(w.T, T.data(), T.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
        DIE_CUDA_TRY(cudaMemcpyAsync(w.Z, Zh.data(), Zh.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
        DIE_CUDA_TRY(cudaMemcpyAsync(w.bvec, bv.data(), bv.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
        DIE_CUDA_TRY(cudaStreamSynchronize(st));     // the host buffers are refilled next restart
        if (auto_r) {
            // Section 5: deflate the eigenvalues outside the deflation radius (capped at r_max)
            if (R_defl < 0) {
                std::vector<double> eps(2 * (size_t)op->N);
                DIE_CUDA_TRY(cudaMemcpy(eps.data(), op->chi_d, op->N * sizeof(double2), cudaMemcpyDeviceToHost));
                for (long i = 0; i < op->N; i++) eps[2 * i] += 1.0;                 // eps_r = chi + 1
                R_defl = die_deflation_radius(eps.data(), op->N, 1000);
                if (!reg) {
                    R_defl = 0;                                                    // unregularised: |eps_r| max
                    for (long i = 0; i < op->N; i++) R_defl = fmax(R_defl, hypot(eps[2 * i], eps[2 * i + 1]));
                }
            }
            const double R = R_defl;
            int cnt = 0;
            while (cnt < rmax && cnt < p - 1 && hypot(T[(size_t)cnt * p + cnt].x, T[(size_t)cnt * p + cnt].y) > R) cnt++;
            if (cnt < 1) cnt = 1;
            r = cnt;
        }
        nconv = 0;
        while (nconv < r) {
            const double lam = hypot(T[(size_t)nconv * p + nconv].x, T[(size_t)nconv * p + nconv].y);
            if (hypot(bv[nconv].x, bv[nconv].y) > tol * lam) break;
            nconv++;
        }
        if (nconv >= r) { converged = true; break; }
        if (it == max_restarts - 1) break;
        // keep the wanted r plus half of the rest
        int kk = r + (p - r) / 2;
        if (kk >= p) kk = p - 1;
        if (kk < r) kk = r;
        DIE_TRY(rotate_basis(w.Q, n, p, w.Z, kk, w.Q2, st));
        DIE_CUDA_TRY(cudaMemcpyAsync(w.Q2 + (long)kk * n, w.Q + (long)p * n, n * sizeof(double2),
                                     cudaMemcpyDeviceToDevice, st));
        std::swap(w.Q, w.Q2);
        ks_truncate_kernel<<<64, 256, 0, st>>>(w.B, p, w.T, w.bvec, kk);
        DIE_LAUNCH_CHECK();
        k = kk;
    }
    // V = first r Schur vectors
    d->r = r;
    d->n = n;
    d->regularized = reg ? 1 : 0;
    d->op_id = op->id;
    DIE_CUDA_TRY(cudaGetDevice(&d->device));
    d->id = next_handle_id();
    DIE_TRY(dalloc((void**)&d->V, (size_t)r * n * sizeof(double2)));
    DIE_TRY(dalloc((void**)&d->M, (size_t)r * r * sizeof(double2)));
    DIE_TRY(dalloc((void**)&d->s, (size_t)(r + 2) * sizeof(double2)));
    DIE_TRY(alloc_red_scratch(&d->rs));
    DIE_TRY(rotate_basis(w.Q, n, p, w.Z, r, d->V, st));
    // re-orthonormalise V (CGS2) so that V^* V = I to FP64 accuracy
    for (int j = 0; j < r; j++) {
        double2* vj = d->V + (long)j * n;
        if (j > 0) {
            DIE_TRY(cgs_dgks(d->V, n, j, vj, n, w.h1, w.h2, w.nrm, w.ist + 1, w.ist + 2, nullptr, 1.0, rs, st));
            DIE_TRY(k_scale_inv_sqrt(vj, n, w.nrm + 1, nullptr, st));
        } else {
            DIE_TRY(k_dots(vj, 0, 0, vj, n, 1, w.nrm, rs, nullptr, st));
            DIE_TRY(k_scale_inv_sqrt(vj, n, w.nrm, nullptr, st));
        }
    }
    // T = V^* Atilde V in FP64 (Eq. (4.13)); column l: V^* (Atilde v_l)
    double2* AV = w.Q2;          // reuse: r vectors
    for (int l = 0; l < r; l++) {
        DIE_TRY(reg ? apply_reg<double, double2>(op, d->V + (long)l * n, AV, st)
                    : apply_op<double, double2>(op, Contrast::Chi, d->V + (long)l * n, AV, st));
        DIE_TRY(k_dots(d->V, n, r, AV, n, 0, d->M + (long)l * r, rs, nullptr, st));
    }
    DIE_TRY(dalloc((void**)&d->V32, (size_t)r * n * sizeof(float2)));
    DIE_TRY(dalloc((void**)&d->c32, (size_t)r * sizeof(float2)));
    DIE_TRY(k_to_c64(d->V, d->V32, (long)r * n, st));
    inverse_minus_identity_kernel<<<1, 32, 0, st>>>(d->M, r, w.ist + 4, w.ist);
    DIE_LAUNCH_CHECK();
    DIE_TRY(dalloc((void**)&d->M32, (size_t)r * r * sizeof(float2)));
    DIE_TRY(k_to_c64(d->M, d->M32, (long)r * r, st));
    int rc = 0;
    DIE_CUDA_TRY(cudaMemcpyAsync(&rc, w.ist, sizeof(int), cudaMemcpyDeviceToHost, st));
    DIE_CUDA_TRY(cudaStreamSynchronize(st));
    d->eigs.resize(2 * (size_t)r);
    for (int i = 0; i < r; i++) {
        d->eigs[2 * i] = T[(size_t)i * p + i].x;
        d->eigs[2 * i + 1] = T[(size_t)i * p + i].y;
    }
    if (eig_out) memcpy(eig_out, d->eigs.data(), 2 * (size_t)r * sizeof(double));
    if (r_out) *r_out = r;
    if (rc != 0) return DIE_ESINGULAR;
    return converged ? DIE_OK : DIE_ENOCONV;
}

extern "C" die_status deflation_build(dieop_t op, const defl_opts* o, void* stream, defl_t* out, double* eig_out,
                                      int* r_out) {
    if (!out) return DIE_EINVAL;
    *out = nullptr;
    if (!op || !o) return DIE_EINVAL;
    if (o->r < 0 || o->r > kMaxDeflation || o->r_max > kMaxDeflation || o->krylov_dim < 0 || o->max_restarts < 0)
        return DIE_EINVAL;
    if (o->inner != DIE_FP64 && o->inner != DIE_FP32_INNER) return DIE_EINVAL;
    if (o->r > 0 && vec_len(op) <= o->r + 2) return DIE_EINVAL;
    defl_s* d = new (std::nothrow) defl_s();
    if (!d) return DIE_ENOMEM;
    die_status s;
    try {
        s = build_impl(op, o, (cudaStream_t)stream, d, eig_out, r_out);
    } catch (...) {               // host allocation failure: no exception crosses the C ABI
        s = DIE_ENOMEM;
    }
    if (s != DIE_OK && s != DIE_ENOCONV) {
        free_defl(d);
        return s;
    }
    *out = d;
    return s;
}

extern "C" die_status deflation_apply(defl_t d, const void* x, void* z, void* stream) {
    if (!d || !x || !z) return DIE_EINVAL;
    return defl_apply(d, (const double2*)x, (double2*)z, nullptr, (cudaStream_t)stream);
}

extern "C" void deflation_destroy(defl_t d) {
    if (!d) return;
    cudaDeviceSynchronize();
    free_defl(d);
}
