// Krylov-space kernels shared by restarted GMRES and the deflation eigensolver:
// batched complex dot products with a deterministic two-level reduction, the fused
// sweeps of classical Gram-Schmidt with one re-orthogonalisation (CGS2), linear
// combinations and the deflation apply.  Vectors are complex128 (double2) of length
// n; a basis is stored as consecutive vectors V_i = V + i * ldv.
#pragma once

#include "common.cuh"

namespace die {

constexpr int kRedBlocks = 304;      // 2 blocks per SM on a 152-SM GB300; fixed => deterministic sums
constexpr int kRedThreads = 256;
constexpr int kMaxBasis = 320;       // largest basis a single reduction handles

// Reduction scratch: per-block partial sums, [vector][block].
struct RedScratch {
    double2* partial = nullptr;      // kMaxBasis * kRedBlocks
    unsigned* counter = nullptr;     // arrival counter of the last-block reduction (left at 0)
};

// State of one GMRES cycle on the device (all FP64).
struct GmresDev {
    double2* H;        // (m+1) x m, column-major, ld = m+1: Hessenberg, rotated in place to R
    double2* cs;       // m rotation cosines (real part used)
    double2* sn;       // m rotation sines
    double2* g;        // m+1: rotated beta e1
    double2* h1;       // m+2: first projection (+ ||w||^2 in the last slot)
    double2* h2;       // m+2: second projection
    double2* y;        // m: least-squares solution
    double* hist;      // per-step residual estimates (relative), indexed by global step
    int* done;         // 1 when the cycle must stop (converged / breakdown / NaN)
    int* k;            // steps completed in the current cycle
    int* flags;        // bit 0: NaN/Inf met, bit 1: Arnoldi breakdown, bit 2: singular R
    double* wnorm;     // ||w|| after orthogonalisation (= H(j+1, j))
    double bnorm, tol;
    int m, jmax, hist_cap;
};

// Host launchers (blas.cu).  `skip` (device int, may be NULL) makes every launched
// kernel return immediately when *skip != 0.
die_status k_dots(const double2* V, long ldv, int nv, const double2* w, long n, double2* out,
                  const RedScratch& rs, const int* skip, cudaStream_t st);
die_status k_cgs_update_dots(const double2* V, long ldv, int nv, double2* w, long n, const double2* h,
                             double2* out, const RedScratch& rs, const int* skip, cudaStream_t st);
// w -= V h2; then the Givens step for column j (writes H, g, hist, done, k).
die_status k_cgs_update_norm_givens(const double2* V, long ldv, int nv, double2* w, long n, GmresDev S, int j,
                                    int step, const RedScratch& rs, cudaStream_t st);
// w -= V h (no norm) and ||w||^2 into out[0]  (used by the eigensolver)
die_status k_cgs_update_norm(const double2* V, long ldv, int nv, double2* w, long n, const double2* h,
                             double2* out, const RedScratch& rs, const int* skip, cudaStream_t st);
// v *= 1 / sqrt(max(re(*nrm2), 0)) if the norm is positive (nrm2 on the device)
die_status k_scale_inv_sqrt(double2* v, long n, const double2* nrm2, const int* skip, cudaStream_t st);
die_status k_scale_inv_real(double2* v, long n, const double* s, const int* skip, cudaStream_t st);
// r = b - y
die_status k_sub(const double2* b, const double2* y, double2* r, long n, cudaStream_t st);
// x += sum_i V_i c_i  (c on the device, k entries)
die_status k_lincomb_add(const double2* V, long ldv, int k, const double2* c, double2* x, long n, cudaStream_t st);
// out = sum_i V_i c_i
die_status k_lincomb(const double2* V, long ldv, int k, const double2* c, double2* out, long n, cudaStream_t st);
// z = x + V (M s): M is r x r column-major on the device, s the projections V^* x
die_status k_defl_update(const double2* V, long ldv, int r, const double2* M, const double2* s, const double2* x,
                         double2* z, long n, const int* skip, cudaStream_t st);
// Solve the k x k upper-triangular R y = g of the current cycle (k read from S.k).
die_status k_gmres_lsq(GmresDev S, cudaStream_t st);
die_status k_gmres_init(GmresDev S, const double2* beta2, cudaStream_t st);

}  // namespace die
