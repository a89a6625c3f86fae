// FFT-speed products with the discretised TE operator A = I - G X (Eqs. (4.3)-(4.5)).
//
// G is block-Toeplitz (its entries depend on x_n - x_m only), so G w is a 2-D
// linear convolution of the 2 x 2 Green's tensor table with the contrast current
// w = chi u; it is computed with zero padding to M1 x M2 >= (2 n1) x (2 n2):
//
//   K1  per grid row i2 and component: w = chi * u, zero-pad to M1, FFT along x1,
//       written transposed: W[c][k1][i2]                    (rows i2 < n2 only)
//   K2  per column k1: FFT along x2 (inputs i2 >= n2 are zero), multiply by the
//       Green spectra  z1 = G11 w1 + G12 w2, z2 = G12 w1 + G22 w2, inverse FFT,
//       keep i2 < n2, written back in place
//   K3  per grid row: inverse FFT along x1, keep i1 < n1, y = u - z
//   K3K1 (regularised product A(chi') A(chi), Section 5) finishes row i2 of the
//       first product (v = u - z, kept in a buffer for the final subtraction) and
//       immediately starts the second product on the same row: chi' * v, FFT.
//
// The spectra are stored for k1 <= M1/2, k2 <= M2/2 only: G11, G22 are even and
// G12 is odd in each offset coordinate (a symmetry of Eqs. (4.3)-(4.5)), so the
// other quadrants follow by sign.  They carry the 1/(M1 M2) of the inverse FFTs.
#include "op.cuh"
#include "prof.cuh"

namespace die {

// Rows per block of the row passes: enough for 32-byte segments in the transposed
// accesses (4 complex64 / 2 complex128), at most 512 threads per block.
template <typename C> constexpr int tile_rows() { return sizeof(C) == 8 ? 4 : 2; }
constexpr int kRowsMaxThreads = 512;

template <typename C> __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

// ------------------------------------------------------------------------- K1
template <typename T, typename IO, int EPT>
__global__ void __launch_bounds__(512) k1_rows_fwd(OpDev<T> op, const IO* __restrict__ u,
                                                    const C_t<T>* __restrict__ chi, C_t<T>* __restrict__ W,
                                                    const int* __restrict__ skip) {
    using C = C_t<T>;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int L = op.M1, G = L / EPT, TR = blockDim.x / G;
    const int rs = threadIdx.x / G, t = threadIdx.x - rs * G;
    const int c = blockIdx.y;
    const int i2_0 = blockIdx.x * TR;
    const int i2 = i2_0 + rs;
    const bool active = i2 < op.n2;
    const long N = (long)op.n1 * op.n2;
    C* buf = tile + rs * L;
    const FftPlan& pl = op.f1;
    int Ns = 1;
    {
        const int R = pl.radix[0];
        C x[EPT];
        if (active) {
            const IO* urow = u + c * N + (long)i2 * op.n1;
            const C* crow = chi + (long)i2 * op.n1;
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                const int idx = reg_index<EPT>(e, R, L, t, G);
                x[e] = idx < op.n1 ? cmul(cvt<C>(urow[idx]), crow[idx]) : czero<C>();
            }
            compute_any<C, EPT, false>(R, x, L, 1, t, G, op.tw1);
            store_any<C, EPT>(R, buf, x, L, 1, t, G);
        }
        __syncthreads();
        Ns = R;
    }
    run_stages<C, EPT, false>(buf, pl, 1, pl.ns, Ns, op.tw1, t, G, active);
    for (int e = threadIdx.x; e < L * TR; e += blockDim.x) {
        const int k1 = e / TR, r = e - k1 * TR;
        const int row = i2_0 + r;
        if (row < op.n2) W[((long)c * L + k1) * op.n2 + row] = tile[r * L + k1];
    }
}

// ------------------------------------------------------------------------- K2
template <typename T, int EPT>
__global__ void __launch_bounds__(256) k2_cols(OpDev<T> op, C_t<T>* __restrict__ W, const int* __restrict__ skip) {
    using C = C_t<T>;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + op.M2;
    const int L = op.M2, G = L / EPT, t = threadIdx.x;
    const int k1 = blockIdx.x;
    C* col0 = W + (long)k1 * op.n2;
    C* col1 = W + ((long)op.M1 + k1) * op.n2;
    C x0[EPT], x1[EPT];
    const FftPlan& f = op.f2;
    int Ns = 1;
    for (int s = 0; s < f.ns; s++) {
        const int R = f.radix[s];
        if (s == 0) {
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                const int idx = reg_index<EPT>(e, R, L, t, G);
                const bool in = idx < op.n2;
                x0[e] = in ? col0[idx] : czero<C>();
                x1[e] = in ? col1[idx] : czero<C>();
            }
        } else {
            load_any<C, EPT>(R, b0, x0, L, t, G);
            load_any<C, EPT>(R, b1, x1, L, t, G);
            __syncthreads();
        }
        compute_any<C, EPT, false>(R, x0, L, Ns, t, G, op.tw2);
        compute_any<C, EPT, false>(R, x1, L, Ns, t, G, op.tw2);
        if (s < f.ns - 1) {
            store_any<C, EPT>(R, b0, x0, L, Ns, t, G);
            store_any<C, EPT>(R, b1, x1, L, Ns, t, G);
            __syncthreads();
        }
        Ns *= R;
    }
    {   // 2 x 2 Green-spectrum multiply at frequencies (k1, k2)
        const int R = f.radix[f.ns - 1];
        const int h1 = op.M1 >> 1, h2 = op.M2 >> 1;
        const int k1q = k1 <= h1 ? k1 : op.M1 - k1;
        const bool neg1 = k1 > h1;
        const long plane = (long)op.Q1 * op.Q2;
        const C* g = op.gq + (long)k1q * op.Q2;
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            const int k2 = reg_index<EPT>(e, R, L, t, G);
            const int k2q = k2 <= h2 ? k2 : op.M2 - k2;
            const bool neg = neg1 != (k2 > h2);
            const C g11 = g[k2q], g22 = g[plane + k2q];
            C g12 = g[2 * plane + k2q];
            if (neg) { g12.x = -g12.x; g12.y = -g12.y; }
            const C w0 = x0[e], w1 = x1[e];
            x0[e] = cadd(cmul(g11, w0), cmul(g12, w1));
            x1[e] = cadd(cmul(g12, w0), cmul(g22, w1));
        }
    }
    const FftPlan& iv = op.i2;
    Ns = 1;
    for (int s = 0; s < iv.ns; s++) {
        const int R = iv.radix[s];
        if (s > 0) {
            load_any<C, EPT>(R, b0, x0, L, t, G);
            load_any<C, EPT>(R, b1, x1, L, t, G);
            __syncthreads();
        }
        compute_any<C, EPT, true>(R, x0, L, Ns, t, G, op.tw2);
        compute_any<C, EPT, true>(R, x1, L, Ns, t, G, op.tw2);
        if (s < iv.ns - 1) {
            store_any<C, EPT>(R, b0, x0, L, Ns, t, G);
            store_any<C, EPT>(R, b1, x1, L, Ns, t, G);
            __syncthreads();
        } else {
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                const int idx = reg_index<EPT>(e, R, L, t, G);
                if (idx < op.n2) { col0[idx] = x0[e]; col1[idx] = x1[e]; }
            }
        }
        Ns *= R;
    }
}

// Load the transposed tile W[c][0..M1)[i2_0 .. i2_0+TR) into shared memory rows.
template <typename C>
__device__ __forceinline__ void load_tile(C* tile, const C* __restrict__ W, int c, int i2_0, int M1, int n2, int TR) {
    for (int e = threadIdx.x; e < M1 * TR; e += blockDim.x) {
        const int k1 = e / TR, r = e - k1 * TR;
        const int row = i2_0 + r;
        tile[r * M1 + k1] = row < n2 ? W[((long)c * M1 + k1) * n2 + row] : czero<C>();
    }
    __syncthreads();
}

// ------------------------------------------------------------------------- K3
// y = u - z for one tile of rows; u of element type U, y of IO.
template <typename T, typename U, typename IO, int EPT>
__global__ void __launch_bounds__(512) k3_rows_inv(OpDev<T> op, const C_t<T>* __restrict__ W,
                                                    const U* __restrict__ u, IO* __restrict__ y,
                                                    const int* __restrict__ skip) {
    using C = C_t<T>;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int L = op.M1, G = L / EPT, TR = blockDim.x / G;
    const int rs = threadIdx.x / G, t = threadIdx.x - rs * G;
    const int c = blockIdx.y;
    const int i2_0 = blockIdx.x * TR;
    const int i2 = i2_0 + rs;
    const bool active = i2 < op.n2;
    const long N = (long)op.n1 * op.n2;
    C* buf = tile + rs * L;
    load_tile<C>(tile, W, c, i2_0, L, op.n2, TR);
    const FftPlan& iv = op.i1;
    int Ns = 1;
    C x[EPT];
    for (int s = 0; s < iv.ns; s++) {
        const int R = iv.radix[s];
        if (active) load_any<C, EPT>(R, buf, x, L, t, G);
        __syncthreads();
        if (active) compute_any<C, EPT, true>(R, x, L, Ns, t, G, op.tw1);
        if (s < iv.ns - 1) {
            if (active) store_any<C, EPT>(R, buf, x, L, Ns, t, G);
            __syncthreads();
        } else if (active) {
            const long off = c * N + (long)i2 * op.n1;
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                const int idx = reg_index<EPT>(e, R, L, t, G);
                if (idx < op.n1) y[off + idx] = csub(cvt<IO>(u[off + idx]), cvt<IO>(x[e]));
            }
        }
        Ns *= R;
    }
}

// ----------------------------------------------------------------------- K3K1
template <typename T, typename IO, int EPT>
__global__ void __launch_bounds__(512) k3k1_rows(OpDev<T> op, C_t<T>* __restrict__ W, const IO* __restrict__ u,
                                                  const C_t<T>* __restrict__ chir, C_t<T>* __restrict__ vbuf,
                                                  const int* __restrict__ skip) {
    using C = C_t<T>;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int L = op.M1, G = L / EPT, TR = blockDim.x / G;
    const int rs = threadIdx.x / G, t = threadIdx.x - rs * G;
    const int c = blockIdx.y;
    const int i2_0 = blockIdx.x * TR;
    const int i2 = i2_0 + rs;
    const bool active = i2 < op.n2;
    const long N = (long)op.n1 * op.n2;
    C* buf = tile + rs * L;
    load_tile<C>(tile, W, c, i2_0, L, op.n2, TR);
    const FftPlan& iv = op.i1;
    int Ns = 1;
    C x[EPT];
    for (int s = 0; s < iv.ns; s++) {
        const int R = iv.radix[s];
        if (active) load_any<C, EPT>(R, buf, x, L, t, G);
        __syncthreads();
        if (active) compute_any<C, EPT, true>(R, x, L, Ns, t, G, op.tw1);
        if (s < iv.ns - 1) {
            if (active) store_any<C, EPT>(R, buf, x, L, Ns, t, G);
            __syncthreads();
        }
        Ns *= R;
    }
    // v = u - z (first product), kept for the final subtraction; then chi' v -> FFT.
    const FftPlan& f = op.f1;
    {
        const int R = iv.radix[iv.ns - 1];      // == f.radix[0]: inverse plan is the reversed forward plan
        if (active) {
            const long off = c * N + (long)i2 * op.n1;
            const C* crow = chir + (long)i2 * op.n1;
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                const int idx = reg_index<EPT>(e, R, L, t, G);
                if (idx < op.n1) {
                    const C v = csub(cvt<C>(u[off + idx]), x[e]);
                    vbuf[off + idx] = v;
                    x[e] = cmul(v, crow[idx]);
                } else {
                    x[e] = czero<C>();
                }
            }
            compute_any<C, EPT, false>(R, x, L, 1, t, G, op.tw1);
            store_any<C, EPT>(R, buf, x, L, 1, t, G);
        }
        __syncthreads();
        Ns = R;
    }
    run_stages<C, EPT, false>(buf, f, 1, f.ns, Ns, op.tw1, t, G, active);
    for (int e = threadIdx.x; e < L * TR; e += blockDim.x) {
        const int k1 = e / TR, r = e - k1 * TR;
        const int row = i2_0 + r;
        if (row < op.n2) W[((long)c * L + k1) * op.n2 + row] = tile[r * L + k1];
    }
}

// --------------------------------------------------------------------- launch
template <typename T> struct Sel;
template <> struct Sel<double> {
    static const double2* chi(const dieop_s* o, Contrast c) { return c == Contrast::Chi ? o->chi_d : o->chir_d; }
};
template <> struct Sel<float> {
    static const float2* chi(const dieop_s* o, Contrast c) { return c == Contrast::Chi ? o->chi_f : o->chir_f; }
};

template <typename T> OpDev<T> view(const dieop_s* op);
template <> OpDev<double> view<double>(const dieop_s* op) { return view_d(op); }
template <> OpDev<float> view<float>(const dieop_s* op) { return view_f(op); }

OpDev<double> view_d(const dieop_s* op) {
    OpDev<double> v;
    v.n1 = op->n1; v.n2 = op->n2; v.M1 = op->M1; v.M2 = op->M2; v.Q1 = op->Q1; v.Q2 = op->Q2;
    v.f1 = op->f1; v.i1 = op->i1; v.f2 = op->f2; v.i2 = op->i2;
    v.tw1 = op->tw1_d; v.tw2 = op->tw2_d; v.gq = op->gq_d;
    return v;
}
OpDev<float> view_f(const dieop_s* op) {
    OpDev<float> v;
    v.n1 = op->n1; v.n2 = op->n2; v.M1 = op->M1; v.M2 = op->M2; v.Q1 = op->Q1; v.Q2 = op->Q2;
    v.f1 = op->f1; v.i1 = op->i1; v.f2 = op->f2; v.i2 = op->i2;
    v.tw1 = op->tw1_f; v.tw2 = op->tw2_f; v.gq = op->gq_f;
    return v;
}

struct Launch { dim3 grid, block; size_t smem; };

template <typename T>
static Launch rows_launch(const OpDev<T>& v) {
    using C = C_t<T>;
    const int G = v.M1 / v.f1.ept;
    int TR = tile_rows<C>();
    while (TR > 1 && TR * G > kRowsMaxThreads) TR /= 2;
    return Launch{dim3((v.n2 + TR - 1) / TR, 2), dim3(TR * G), (size_t)TR * v.M1 * sizeof(C)};
}
template <typename T>
static Launch cols_launch(const OpDev<T>& v) {
    using C = C_t<T>;
    return Launch{dim3(v.M1), dim3(v.M2 / v.f2.ept), (size_t)2 * v.M2 * sizeof(C)};
}

template <typename T, typename IO>
static void launch_k1(const OpDev<T>& v, const IO* u, const C_t<T>* chi, C_t<T>* W, const int* skip, cudaStream_t st) {
    Launch l = rows_launch(v);
    DIE_PROF(PK_ROWS_FWD, st,
             if (v.f1.ept == 16) k1_rows_fwd<T, IO, 16><<<l.grid, l.block, l.smem, st>>>(v, u, chi, W, skip);
             else k1_rows_fwd<T, IO, 12><<<l.grid, l.block, l.smem, st>>>(v, u, chi, W, skip));
}
template <typename T>
static void launch_k2(const OpDev<T>& v, C_t<T>* W, const int* skip, cudaStream_t st) {
    Launch l = cols_launch(v);
    DIE_PROF(PK_COLS, st,
             if (v.f2.ept == 16) k2_cols<T, 16><<<l.grid, l.block, l.smem, st>>>(v, W, skip);
             else k2_cols<T, 12><<<l.grid, l.block, l.smem, st>>>(v, W, skip));
}
template <typename T, typename U, typename IO>
static void launch_k3(const OpDev<T>& v, const C_t<T>* W, const U* u, IO* y, const int* skip, cudaStream_t st) {
    Launch l = rows_launch(v);
    DIE_PROF(PK_ROWS_INV, st,
             if (v.f1.ept == 16) k3_rows_inv<T, U, IO, 16><<<l.grid, l.block, l.smem, st>>>(v, W, u, y, skip);
             else k3_rows_inv<T, U, IO, 12><<<l.grid, l.block, l.smem, st>>>(v, W, u, y, skip));
}
template <typename T, typename IO>
static void launch_k3k1(const OpDev<T>& v, C_t<T>* W, const IO* u, const C_t<T>* chir, C_t<T>* vb, const int* skip,
                        cudaStream_t st) {
    Launch l = rows_launch(v);
    DIE_PROF(PK_ROWS_INV_FWD, st,
             if (v.f1.ept == 16) k3k1_rows<T, IO, 16><<<l.grid, l.block, l.smem, st>>>(v, W, u, chir, vb, skip);
             else k3k1_rows<T, IO, 12><<<l.grid, l.block, l.smem, st>>>(v, W, u, chir, vb, skip));
}

template <typename T, typename IO>
die_status apply_op_skip(dieop_s* op, Contrast which, const IO* x, IO* y, const int* skip, cudaStream_t st) {
    using C = C_t<T>;
    OpDev<T> v = view<T>(op);
    C* W = reinterpret_cast<C*>(op->ws.W);
    launch_k1<T, IO>(v, x, Sel<T>::chi(op, which), W, skip, st);
    launch_k2<T>(v, W, skip, st);
    launch_k3<T, IO, IO>(v, W, x, y, skip, st);
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

template <typename T, typename IO>
die_status apply_reg_skip(dieop_s* op, const IO* x, IO* y, const int* skip, cudaStream_t st) {
    using C = C_t<T>;
    OpDev<T> v = view<T>(op);
    C* W = reinterpret_cast<C*>(op->ws.W);
    C* vb = reinterpret_cast<C*>(op->ws.v);
    launch_k1<T, IO>(v, x, Sel<T>::chi(op, Contrast::Chi), W, skip, st);
    launch_k2<T>(v, W, skip, st);
    launch_k3k1<T, IO>(v, W, x, Sel<T>::chi(op, Contrast::ChiReg), vb, skip, st);
    launch_k2<T>(v, W, skip, st);
    launch_k3<T, C, IO>(v, W, vb, y, skip, st);
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

template <typename T, typename IO>
die_status apply_op(dieop_s* op, Contrast c, const IO* x, IO* y, cudaStream_t st) {
    return apply_op_skip<T, IO>(op, c, x, y, nullptr, st);
}
template <typename T, typename IO>
die_status apply_reg(dieop_s* op, const IO* x, IO* y, cudaStream_t st) {
    return apply_reg_skip<T, IO>(op, x, y, nullptr, st);
}

template die_status apply_op<double, double2>(dieop_s*, Contrast, const double2*, double2*, cudaStream_t);
template die_status apply_op<float, float2>(dieop_s*, Contrast, const float2*, float2*, cudaStream_t);
template die_status apply_op<float, double2>(dieop_s*, Contrast, const double2*, double2*, cudaStream_t);
template die_status apply_reg<double, double2>(dieop_s*, const double2*, double2*, cudaStream_t);
template die_status apply_reg<float, float2>(dieop_s*, const float2*, float2*, cudaStream_t);
template die_status apply_reg<float, double2>(dieop_s*, const double2*, double2*, cudaStream_t);
template die_status apply_op_skip<double, double2>(dieop_s*, Contrast, const double2*, double2*, const int*, cudaStream_t);
template die_status apply_op_skip<float, double2>(dieop_s*, Contrast, const double2*, double2*, const int*, cudaStream_t);
template die_status apply_reg_skip<double, double2>(dieop_s*, const double2*, double2*, const int*, cudaStream_t);
template die_status apply_reg_skip<float, double2>(dieop_s*, const double2*, double2*, const int*, cudaStream_t);

// Allow up to 227 KB of dynamic shared memory for every instantiation (once per process/device).
template <typename F>
static cudaError_t allow_smem(F f) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

die_status set_kernel_attributes(const dieop_s*) {
#define DIE_ALLOW(k) DIE_CUDA_TRY(allow_smem(k))
    DIE_ALLOW((k1_rows_fwd<double, double2, 16>)); DIE_ALLOW((k1_rows_fwd<double, double2, 12>));
    DIE_ALLOW((k1_rows_fwd<float, float2, 16>)); DIE_ALLOW((k1_rows_fwd<float, float2, 12>));
    DIE_ALLOW((k1_rows_fwd<float, double2, 16>)); DIE_ALLOW((k1_rows_fwd<float, double2, 12>));
    DIE_ALLOW((k2_cols<double, 16>)); DIE_ALLOW((k2_cols<double, 12>));
    DIE_ALLOW((k2_cols<float, 16>)); DIE_ALLOW((k2_cols<float, 12>));
    DIE_ALLOW((k3_rows_inv<double, double2, double2, 16>)); DIE_ALLOW((k3_rows_inv<double, double2, double2, 12>));
    DIE_ALLOW((k3_rows_inv<float, float2, float2, 16>)); DIE_ALLOW((k3_rows_inv<float, float2, float2, 12>));
    DIE_ALLOW((k3_rows_inv<float, double2, double2, 16>)); DIE_ALLOW((k3_rows_inv<float, double2, double2, 12>));
    DIE_ALLOW((k3_rows_inv<float, float2, double2, 16>)); DIE_ALLOW((k3_rows_inv<float, float2, double2, 12>));
    DIE_ALLOW((k3k1_rows<double, double2, 16>)); DIE_ALLOW((k3k1_rows<double, double2, 12>));
    DIE_ALLOW((k3k1_rows<float, float2, 16>)); DIE_ALLOW((k3k1_rows<float, float2, 12>));
    DIE_ALLOW((k3k1_rows<float, double2, 16>)); DIE_ALLOW((k3k1_rows<float, double2, 12>));
#undef DIE_ALLOW
    return DIE_OK;
}

}  // namespace die
