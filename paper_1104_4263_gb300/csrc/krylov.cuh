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

constexpr int kRedThreads = 256;
constexpr int kRedGroup = 16;        // blocks per first-level group of the final sums
constexpr int kRedBlocksMax = 640;   // the reduction scratch holds partials of up to this many blocks
constexpr int kRedGroupsMax = kRedBlocksMax / kRedGroup;
// Blocks of every reduction launch: two per SM of the current device, a multiple of
// kRedGroup (queried once per device).  The count is fixed for a device, so the
// fixed-order sums are bitwise reproducible on it.
int red_blocks();
constexpr int kMaxBasis = 320;       // largest basis a single projection / update launch handles
constexpr int kBasisChunk = 256;     // longer bases are swept in chunks of this many vectors
constexpr int kMaxRestart = 2048;    // largest GMRES restart (Krylov dimension per cycle)
constexpr int kMaxDeflation = 256;   // largest deflation rank (Krylov-Schur basis <= kMaxBasis - 2)
// Default DGKS threshold: a second classical Gram-Schmidt pass when the first left
// ||w'|| < eta ||w||.  The loss of orthogonality of single-pass steps accumulates over a
// cycle: cycles of up to kShortCycle vectors take eta = 0.01 (measured on the 512^2
// core-shell with no second pass firing: max |V* V - I| 1.6e-13, 6.6e-13 and 2.3e-11
// after cycles of 40, 48 and 64 steps with complex64 products and deflation, 2.9e-9
// after 96), longer ones the classical 1/sqrt(2), which keeps the basis orthonormal to
// working precision at any length (the same measurement at 300 steps and eta = 0.01 gave
// 3e-6).
constexpr int kShortCycle = 64;
constexpr double kShortCycleEta = 0.01;
constexpr double kDefaultReorthEta = 0.70710678118654752440;
inline double default_reorth_eta(int restart) { return restart <= kShortCycle ? kShortCycleEta : kDefaultReorthEta; }
static_assert(kRedBlocksMax % kRedGroup == 0, "reduction groups must tile the grid");
static_assert(kBasisChunk + 1 <= kMaxBasis, "a chunk and the norm fit the reduction scratch");

// Reduction scratch.  Each block writes one partial per vector ([vector][block]); the
// last block of each group of kRedGroup consecutive blocks to arrive sums the group's
// partials in block order ([vector][group]); the last group to finish sums those in
// group order.  The arrival counters (one per group, then the top one) are left at 0
// by every kernel that uses them.
struct RedScratch {
    double2* partial = nullptr;      // kMaxBasis * kRedBlocksMax
    double2* partial2 = nullptr;     // kMaxBasis * kRedGroupsMax
    unsigned* counter = nullptr;     // kRedCounters
};
constexpr int kRedCounters = 1 + kRedGroupsMax;

// DGKS decision taken by the last block of a norm-computing update: reorth = always ||
// ||w'||^2 < eta^2 ||w||^2; skip2 = done || !reorth (makes the second pass return at once).
// When inv != NULL the block that holds the final norm of w also stores 1 / ||w|| there
// (1 when the norm is zero or not finite), for the normalisation of the next basis vector.
struct Dgks {
    const double2* before2 = nullptr;  // ||w||^2 before the first pass (real part)
    int* reorth = nullptr;
    int* skip2 = nullptr;
    const int* done = nullptr;         // may be NULL
    double* inv = nullptr;             // may be NULL
    int always = 0;
    double eta2 = 0.5;
    // Single-pass (optimistic) cycles: no second pass is launched; when one would be
    // needed the deciding block sets bit 3 of *abort_flags and *abort_done = 1 (the
    // cycle is then run again with second passes).  NULL: normal DGKS.
    int* abort_flags = nullptr;
    int* abort_done = nullptr;
};

// Deflation projections folded into a Gram-Schmidt update (FP32-inner deflated solves):
// while the update kernel writes the new vector w, it also accumulates V32^* w in FP32
// (w rounded to complex64); the block that finishes its sums forms
// cf = M32 (V32^* w / ||w||) for the deflation update of the next Arnoldi step.
struct DeflProj {
    const float2* V32 = nullptr;   // r complex64 basis vectors, vector i at V32 + i * ld
    long ld = 0;
    int r = 0;                     // 1 <= r <= kDeflFoldMax
    const float2* M32 = nullptr;   // r x r, column-major (M = T^-1 - I in complex64)
    double2* s = nullptr;          // 1 + r scratch: ||w||^2, then V32^* w
    float2* cf = nullptr;          // r coefficients (complex64)
};
constexpr int kDeflFoldMax = 32;   // largest r folded into the update

// State of one GMRES cycle on the device (all FP64).  The per-step arrays (projections,
// norms, DGKS flag, scale factor) have one slot per Arnoldi step, so that the Givens
// step of step j, which runs on a side stream, reads values that step j+1 does not
// overwrite.
struct GmresDev {
    double2* H;        // (m+1) x m, column-major, ld = m+1: Hessenberg, rotated in place to R
    double2* cs;       // m rotation cosines (real part used)
    double2* sn;       // m rotation sines
    double2* g;        // m+1: rotated beta e1
    double2* h1;       // m x (m+3): step j's first projections at h1 + j (m+3) (+ ||w||^2 at index j+1)
    double2* h2;       // m x (m+3): second projections (re-orthogonalisation)
    double2* y;        // m: least-squares solution
    double2* nrm;      // 2 m: step j: [2j] ||w||^2 after pass 1, [2j+1] after pass 2
    double* inv;       // m: step j: 1 / ||w|| after orthogonalisation (scales v_{j+1})
    double* hist;      // per-step residual estimates (relative), indexed by global step
    int* done;         // 1 when the cycle must stop (converged / breakdown / NaN)
    int* k;            // steps completed in the current cycle
    int* flags;        // bit 0: NaN/Inf met, bit 1: Arnoldi breakdown, bit 2: singular R
    int* reorth;       // m: 1 if the second Gram-Schmidt pass ran at step j
    int* skip2;        // done || !reorth of the current step
    int* nreorth;      // second passes run (counter over the solve)
    int* step0;        // global index of the cycle's first step: step j's history slot is *step0 + j
    double* bnorm;     // ||btilde|| (the residual estimates are relative to it)
    double tol;
    int m, jmax, hist_cap;
};

// One Givens step of the GMRES least-squares problem min || beta e1 - H y || (Saad &
// Schultz): Hc[0..j] holds column j of H (the projections of step j) and hn = ||w|| its
// subdiagonal entry.  The j earlier rotations (cosine csv[i].x, complex sine snv[i]) are
// applied to the column; the rotation that zeroes the subdiagonal is formed, stored in
// *cs_j, *sn_j, and applied to g[j], g[j + 1].  Hc then holds column j of R (Hc[j + 1] =
// 0) and |g[j + 1]| is the least-squares residual after j + 1 steps.  Host and device.
__host__ __device__ inline void givens_column(double2* Hc, const double2* csv, const double2* snv, int j, double hn,
                                              double2* cs_j, double2* sn_j, double2* g) {
    Hc[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; i++) {
        const double c = csv[i].x;
        const double2 s = snv[i];
        const double2 a = Hc[i], b = Hc[i + 1];
        Hc[i] = make_double2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
        // -conj(s) a + c b
        Hc[i + 1] = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
    }
    const double2 a = Hc[j];
    const double b = Hc[j + 1].x;
    const double an = hypot(a.x, a.y);
    double c;
    double2 s;
    if (an == 0.0) { c = 0.0; s = make_double2(1.0, 0.0); Hc[j] = make_double2(b, 0.0); }
    else {
        const double rho = hypot(an, b);
        c = an / rho;
        s = make_double2(a.x / an * b / rho, a.y / an * b / rho);
        Hc[j] = make_double2(a.x / an * rho, a.y / an * rho);
    }
    Hc[j + 1] = make_double2(0.0, 0.0);
    *cs_j = make_double2(c, 0.0);
    *sn_j = s;
    const double2 gj = g[j];
    g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    g[j] = make_double2(c * gj.x, c * gj.y);
}

// Skip flags: the kernels return at once when *skip != 0.  A "live" flag is one that
// another stream may set while the kernel runs (the GMRES done flag, set by the Givens
// step on its side stream): the reduction kernels then skip only their own work and
// still take part in the final sums, so that the arrival counters stay consistent.
//
// out[i] = V_i^* w for i < nv; with_norm: out[nv] = ||w||^2 (real part).
// VM != NULL: the three-multiplication form, with m = Re - Im of every V_i in VM.
die_status k_dots(const double2* V, long ldv, int nv, const double2* w, long n, int with_norm, double2* out,
                  const RedScratch& rs, const int* skip, cudaStream_t st, bool live = false,
                  const double* VM = nullptr);
// Deflation projections of the FP32-inner solves: s = V^* x with a complex64 basis and
// vector (FP32 products and in-block sums, FP64 across blocks), then cf = M s rounded to
// complex64 (M32: the r x r matrix M in complex64, column-major).  With inv != NULL, x
// is first formed from the FP64 vector w: w *= *inv (written back) and x = w in complex64.
die_status k_dots32(const float2* V, long ldv, int nv, float2* x, double2* w, const double* inv, long n,
                    double2* out, const float2* M32, float2* cf, const RedScratch& rs, const int* skip,
                    cudaStream_t st, bool live = false);
// out = base + sum_i V_i coef_i for any k (chunks of kBasisChunk vectors; base may be NULL
// = 0, out may equal base); no norm, no skip flag.  VM as for k_basis_axpy.
die_status k_lincomb(const double2* V, long ldv, int k, const double2* coef, const double2* base, double2* out,
                     long n, const RedScratch& rs, cudaStream_t st, const double* VM = nullptr);
// Sets the dynamic shared-memory limits of the per-step GMRES kernels for restarts up to
// m (call once per device, outside any stream capture, before the first solve).
die_status krylov_prepare(int m);
// out = base + sign * sum_i V_i c_i (base may be NULL = 0, out may equal base), c = coef.
// nrm2 != NULL: ||out||^2 into nrm2[0] (device), and the DGKS decision if dec != NULL.
// VM != NULL: the three-multiplication form, with Re - Im of every V_i in VM.
die_status k_basis_axpy(const double2* V, long ldv, int k, const double2* coef, double sign, const double2* base,
                        double2* out, long n, double2* nrm2, const Dgks* dec, const RedScratch& rs,
                        const int* skip, cudaStream_t st, bool live = false, const double* VM = nullptr);
// z = x + V (M s); M r x r column-major; s the projections V^* x.  z may equal x.
die_status k_defl_update(const double2* V, long ldv, int r, const double2* M, const double2* s, const double2* x,
                         double2* z, long n, const int* skip, cudaStream_t st);
// All-complex64 deflation update (FP32-inner solves): z = x + V cf, cf from k_dots32 or
// from a folded update.  With inv != NULL the input is formed from the FP64 vector w:
// w *= *inv (written back) and x = complex64(w) (x itself is then not read).
die_status k_defl_update32(const float2* V, long ldv, int r, const float2* cf, const float2* x, float2* z, long n,
                           const int* skip, cudaStream_t st, double2* w = nullptr, const double* inv = nullptr,
                           double* wm = nullptr);

// Classical Gram-Schmidt of w against V_0..V_{nv-1} with the DGKS criterion (done is a
// live flag, see above); any nv up to kMaxRestart + 1 (bases longer than kBasisChunk
// are swept in chunks: the projections of all chunks use the same w, as classical
// Gram-Schmidt requires, and the update subtracts chunk after chunk):
// h1 = V^* w (||w||^2 in h1[nv]); w -= V h1 (||w||^2 -> nrm[0]); if ||w||^2 < eta2
// ||w_before||^2 (always when eta2 >= 1): h2 = V^* w; w -= V h2 (||w||^2 -> nrm[1]).
// inv != NULL receives 1 / ||w|| of the final w (1 if that norm is zero or not finite).
// dp != NULL folds the deflation projections of the final w into the update passes.
// abort_flags != NULL: single pass only (see Dgks::abort_flags; abort_done = done).
// VM != NULL: both passes in the three-multiplication form, with m = Re - Im of each basis
// vector V_i stored in VM (same stride as V) by whatever normalised V_i.
die_status cgs_dgks(const double2* V, long ldv, int nv, double2* w, long n, double2* h1, double2* h2,
                    double2* nrm, int* reorth, int* skip2, const int* done, double eta2, const RedScratch& rs,
                    cudaStream_t st, double* inv = nullptr, const DeflProj* dp = nullptr, double* VM = nullptr,
                    int* abort_flags = nullptr, int* abort_done = nullptr);

// v *= 1 / sqrt(re(*nrm2)) if positive; v *= *inv.  v32 != NULL also receives the
// scaled vector rounded to complex64.
// vm != NULL also receives Re - Im of the scaled vector (three-multiplication form).
die_status k_scale_inv_sqrt(double2* v, long n, const double2* nrm2, const int* skip, cudaStream_t st,
                            float2* v32 = nullptr, double* vm = nullptr);
die_status k_scale_by(double2* v, long n, const double* inv, const int* skip, cudaStream_t st,
                      float2* v32 = nullptr, double* vm = nullptr);
// r = b - y
die_status k_sub(const double2* b, const double2* y, double2* r, long n, cudaStream_t st);
// complex128 -> complex64 copy
die_status k_to_c64(const double2* x, float2* y, long n, cudaStream_t st);

// GMRES step j after Gram-Schmidt: H(:, j) = h1 (+ h2), H(j+1, j) = ||w||, Givens.
// Reads only step j's slots, so it may run on a side stream behind the next step.
die_status k_arnoldi_finish(GmresDev S, int j, cudaStream_t st);
// The per-cycle scalars the cycle's kernels read from device memory (so that a captured
// cycle replays unchanged): *S.step0 = step0, *S.bnorm = bnorm.
die_status k_cycle_scalars(GmresDev S, double bnorm, int step0, cudaStream_t st);
// Solve the k x k upper-triangular R y = g of the current cycle (k read from S.k).
die_status k_gmres_lsq(GmresDev S, cudaStream_t st);
die_status k_gmres_init(GmresDev S, const double2* beta2, cudaStream_t st);

}  // namespace die
