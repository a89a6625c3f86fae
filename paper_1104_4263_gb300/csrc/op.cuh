// Operator handle of libdie and the device view passed to the FFT-convolution kernels.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace die {

// Everything a product kernel needs, by value.
template <typename T>
struct OpDev {
    using C = C_t<T>;
    int n1, n2, M1, M2, Q1, Q2;   // grid, FFT sizes, quarter-spectrum extents (M/2 + 1)
    FftPlan f1, i1, f2, i2;       // forward / inverse plans along x1 (length M1) and x2 (M2)
    const C* tw1;                 // exp(-2 pi i m / M1), m < M1
    const C* tw2;                 // exp(-2 pi i m / M2)
    const C* twx1;                // stage tables of the compile-time plans along x1 (2 M1)
    const C* twx2;                // the same along x2 (2 M2)
    const C* gq;                  // quarter spectra of G11, G22, G12 (and, with three planes, G13,
                                  // G23, G33): [plane][k1q][k2q], pre-scaled
    const C* chim;                // magnetic contrast chi_m (three planes; null otherwise)
    long xs;                      // batched products: elements per field vector (planes n1 n2)
    long ws;                      // batched products: elements per set of row spectra (planes M1 n2)
    int tr;                       // tile height of the fast row passes (0: default)
    int planes;                   // field planes: 2 (E1, E2), or 3 (E1, E2, H3) for DIE_TE_MAG
};

constexpr int kRowsMaxThreads = 512;    // threads per block of the row passes

// Tile heights (rows per block) of the complex64 fast row passes, M1 = L: the default
// (4 rows, or as many as 512 threads allow) and the alternatives with kernels of their own.
constexpr int kTileRowsAlt[] = {1, 2, 8};
inline int default_tile_rows_c64(int L) { return 4 * (L / 16) <= kRowsMaxThreads ? 4 : kRowsMaxThreads / (L / 16); }
// The code the launchers use for height tr at length L: tr when it is a valid alternative,
// else 0 (the default).
inline int tile_rows_code(int tr, int L) {
    if (tr <= 0 || tr == default_tile_rows_c64(L) || tr * (L / 16) > kRowsMaxThreads) return 0;
    for (int a : kTileRowsAlt)
        if (a == tr) return tr;
    return 0;
}

struct Workspace {
    void* W = nullptr;            // 2 x M1 x n2 complex (compute precision), transposed row spectra
    void* v = nullptr;            // 2 x N complex: intermediate of the regularised product
    size_t W_bytes = 0, v_bytes = 0;
};

}  // namespace die

struct dieop_s {
    int device = 0;
    int n1 = 0, n2 = 0, M1 = 0, M2 = 0, N = 0, Q1 = 0, Q2 = 0;
    double h = 0, k = 0;
    die_precision prec = DIE_FP64;
    die_polarization pol = DIE_TE;
    die::FftPlan f1{}, i1{}, f2{}, i2{};
    double2 *tw1_d = nullptr, *tw2_d = nullptr;   // 3 M entries: natural table, then the
    float2 *tw1_f = nullptr, *tw2_f = nullptr;    // forward and inverse stage tables
    int planes = 2;                // field planes: 3 for DIE_TE_MAG (E1, E2, H3)
    double2* gq_d = nullptr;       // (planes == 3 ? 6 : 3) * Q1 * Q2
    float2* gq_f = nullptr;
    double2 *chi_d = nullptr, *chir_d = nullptr;   // chi = eps_r - 1, chi' = 1/eps_r - 1
    float2 *chi_f = nullptr, *chir_f = nullptr;
    double2* chim_d = nullptr;     // chi_m = mu_r - 1 (DIE_TE_MAG only)
    float2* chim_f = nullptr;
    die::Workspace ws;             // FP64-sized; the complex64 path uses the first half
    die::Workspace wsb;            // batched products: grown to the largest batch seen
    int wsb_cap = 0;
    int* dflag = nullptr;          // device status word (create-time checks)
    uint64_t id = 0;               // identity for deflation handles
    void* solver = nullptr;        // die::SolverCache, created by the first gmres_solve
    void* batch[16] = {};          // die::SolverCache of each right-hand side of gmres_solve_batch
    int tile_rows_c64 = 0;         // tile height of the complex64 fast row passes (0: default)
};

namespace die {
uint64_t next_handle_id();   // process-wide unique identities of operator and deflation handles

// Quarter spectra kept by an operator: G11, G22, G12, and G13, G23, G33 with three planes.
inline int green_plane_count(const dieop_s* op) { return op->planes == 3 ? 6 : 3; }
// Complex entries of one field vector.
inline long vec_len(const dieop_s* op) { return (long)op->planes * op->N; }

OpDev<double> view_d(const dieop_s* op);
OpDev<float> view_f(const dieop_s* op);

enum class Contrast { Chi, ChiReg };

// y = (I - G X(contrast)) x with compute type T and element type IO for x and y.  Every
// product takes an optional workspace (row spectra W, middle vector v); NULL = the
// operator's own (op->ws).  Concurrent products on one operator need one each.
template <typename T, typename IO>
die_status apply_op(dieop_s* op, Contrast c, const IO* x, IO* y, cudaStream_t st, const Workspace* ws = nullptr);

// y = A(chi') A(chi) x.
template <typename T, typename IO>
die_status apply_reg(dieop_s* op, const IO* x, IO* y, cudaStream_t st, const Workspace* ws = nullptr);

// The same with a device flag: every kernel returns at once when *skip != 0.
template <typename T, typename IO>
die_status apply_op_skip(dieop_s* op, Contrast c, const IO* x, IO* y, const int* skip, cudaStream_t st,
                         const Workspace* ws = nullptr);
template <typename T, typename IO>
die_status apply_reg_skip(dieop_s* op, const IO* x, IO* y, const int* skip, cudaStream_t st,
                          const Workspace* ws = nullptr);

// nb products over consecutive field vectors, with a workspace of nb sets of row spectra
// (Wws) and nb middle vectors (vws, used when reg).
template <typename T, typename IO>
die_status apply_batch(dieop_s* op, bool reg, const IO* x, IO* y, int nb, void* Wws, void* vws, cudaStream_t st);

// Input and output of different element types (complex64 in, complex128 out).
template <typename T, typename IX, typename IY>
die_status apply_op_skip_xy(dieop_s* op, Contrast c, const IX* x, IY* y, const int* skip, cudaStream_t st,
                            const Workspace* ws = nullptr);
template <typename T, typename IX, typename IY>
die_status apply_reg_skip_xy(dieop_s* op, const IX* x, IY* y, const int* skip, cudaStream_t st,
                             const Workspace* ws = nullptr);

// Input of a product whose first row pass also applies the deflation preconditioner of
// the FP32-inner solves: z = v + V32 cf, with v = w * (*inv) (the FP64 Arnoldi vector,
// normalised in place) or, when w is NULL, v = x (complex64).
struct DeflIn {
    const float2* V32 = nullptr;   // r vectors, vector i at V32 + i * ld
    long ld = 0;
    int r = 0;                     // 1 <= r <= 32
    const float2* cf = nullptr;    // r coefficients
    const float2* x = nullptr;
    double2* w = nullptr;
    const double* inv = nullptr;
    double* wm = nullptr;          // may be NULL: receives Re - Im of the normalised w
};
// y = Atilde z with z = P^-1 v formed inside the first row pass (z is also stored, for
// the later passes); Atilde = A_R A when reg, else A.  Only for grids on the
// compile-time FFT path along x1 (defl_product_ok).
bool defl_product_ok(const dieop_s* op);
die_status apply_defl_xy(dieop_s* op, const DeflIn& d, float2* z, double2* y, bool reg, const int* skip,
                         cudaStream_t st, const Workspace* ws = nullptr);

die_status set_kernel_attributes(const dieop_s* op);

}  // namespace die
