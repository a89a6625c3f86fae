// Krylov-space kernels shared by restarted GMRES and the deflation eigensolver:
// batched complex projections V^* w with a deterministic two-level reduction,
// basis updates out = base + sign * V c (with an optional norm and a DGKS
// re-orthogonalisation decision), the deflation apply, and the small per-step
// kernels of GMRES (Givens, least squares).  Vectors are complex128 (double2) of
// length n; a basis is stored as consecutive vectors V_i = V + i * ldv, complex128 or,
// for the FP32 deflation apply, complex64.
#pragma once

#include "common.cuh"

namespace die {

constexpr int kRedBlocks = 304;      // 2 blocks per SM on a 152-SM GB300; fixed => deterministic sums
constexpr int kRedThreads = 256;
constexpr int kMaxBasis = 320;       // largest basis a single call handles

// Reduction scratch: per-block partial sums, [vector][block], and the arrival counter
// of the last-block reduction (left at 0 by every kernel that uses it).
struct RedScratch {
    double2* partial = nullptr;      // kMaxBasis * kRedBlocks
    unsigned* counter = nullptr;
};

// DGKS decision taken by the last block of a norm-computing update: reorth = always ||
// ||w'||^2 < eta^2 ||w||^2; skip2 = done || !reorth (makes the second pass return at once).
struct Dgks {
    const double2* before2 = nullptr;  // ||w||^2 before the first pass (real part)
    int* reorth = nullptr;
    int* skip2 = nullptr;
    const int* done = nullptr;         // may be NULL
    int always = 0;
    double eta2 = 0.5;
};

// State of one GMRES cycle on the device (all FP64).
struct GmresDev {
    double2* H;        // (m+1) x m, column-major, ld = m+1: Hessenberg, rotated in place to R
    double2* cs;       // m rotation cosines (real part used)
    double2* sn;       // m rotation sines
    double2* g;        // m+1: rotated beta e1
    double2* h1;       // m+3: first projections (+ ||w||^2 at index j+1)
    double2* h2;       // m+3: second projections (re-orthogonalisation)
    double2* y;        // m: least-squares solution
    double2* nrm;      // [0]: ||w||^2 after pass 1, [1]: after pass 2
    double* hist;      // per-step residual estimates (relative), indexed by global step
    int* done;         // 1 when the cycle must stop (converged / breakdown / NaN)
    int* k;            // steps completed in the current cycle
    int* flags;        // bit 0: NaN/Inf met, bit 1: Arnoldi breakdown, bit 2: singular R
    int* reorth;       // 1 if the second Gram-Schmidt pass ran this step
    int* skip2;        // done || !reorth
    int* nreorth;      // second passes run (counter over the solve)
    double* wnorm;     // ||w|| after orthogonalisation (= H(j+1, j))
    double bnorm, tol;
    int m, jmax, hist_cap;
};

// out[i] = V_i^* w for i < nv; with_norm: out[nv] = ||w||^2 (real part).
die_status k_dots(const double2* V, long ldv, int nv, const double2* w, long n, int with_norm, double2* out,
                  const RedScratch& rs, const int* skip, cudaStream_t st);
// The same with a complex64 basis and vector, FP32 accumulation within each lane.
die_status k_dots32(const float2* V, long ldv, int nv, const float2* w, long n, double2* out,
                    const RedScratch& rs, const int* skip, cudaStream_t st);
// out = base + sign * sum_i V_i c_i (base may be NULL = 0, out may equal base), c = coef.
// nrm2 != NULL: ||out||^2 into nrm2[0] (device), and the DGKS decision if dec != NULL.
die_status k_basis_axpy(const double2* V, long ldv, int k, const double2* coef, double sign, const double2* base,
                        double2* out, long n, double2* nrm2, const Dgks* dec, const RedScratch& rs,
                        const int* skip, cudaStream_t st);
// z = x + V (M s); M r x r column-major; s the projections V^* x.  z may equal x.
die_status k_defl_update(const double2* V, long ldv, int r, const double2* M, const double2* s, const double2* x,
                         double2* z, long n, const int* skip, cudaStream_t st);
// All-complex64 deflation update (FP32-inner solves): cf = M s (rounded, r entries of
// device scratch), then z = x + V cf.
die_status k_defl_update32(const float2* V, long ldv, int r, const double2* M, const double2* s, float2* cf,
                           const float2* x, float2* z, long n, const int* skip, cudaStream_t st);

// Classical Gram-Schmidt of w against V_0..V_{nv-1} with the DGKS criterion:
// h1 = V^* w (||w||^2 in h1[nv]); w -= V h1 (||w||^2 -> nrm[0]); if ||w||^2 < eta2
// ||w_before||^2 (always when eta2 >= 1): h2 = V^* w; w -= V h2 (||w||^2 -> nrm[1]).
die_status cgs_dgks(const double2* V, long ldv, int nv, double2* w, long n, double2* h1, double2* h2,
                    double2* nrm, int* reorth, int* skip2, const int* done, double eta2, const RedScratch& rs,
                    cudaStream_t st);

// v *= 1 / sqrt(re(*nrm2)) if positive; v *= 1 / *s if non-zero.  v32 != NULL also
// receives the scaled vector rounded to complex64.
die_status k_scale_inv_sqrt(double2* v, long n, const double2* nrm2, const int* skip, cudaStream_t st,
                            float2* v32 = nullptr);
die_status k_scale_inv_real(double2* v, long n, const double* s, const int* skip, cudaStream_t st,
                            float2* v32 = nullptr);
// r = b - y
die_status k_sub(const double2* b, const double2* y, double2* r, long n, cudaStream_t st);
// complex128 -> complex64 copy
die_status k_to_c64(const double2* x, float2* y, long n, cudaStream_t st);

// GMRES step j after Gram-Schmidt: H(:, j) = h1 (+ h2), H(j+1, j) = ||w||, Givens.
die_status k_arnoldi_finish(GmresDev S, int j, int step, cudaStream_t st);
// Solve the k x k upper-triangular R y = g of the current cycle (k read from S.k).
die_status k_gmres_lsq(GmresDev S, cudaStream_t st);
die_status k_gmres_init(GmresDev S, const double2* beta2, cudaStream_t st);

}  // namespace die
