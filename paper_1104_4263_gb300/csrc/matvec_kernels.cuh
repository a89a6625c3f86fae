// FFT-speed products with the discretised TE operator A = I - G X (Eqs. (4.3)-(4.5)):
// kernels and launchers, included by the instantiation units matvec.cu (FP64) and
// matvec_f32.cu (complex64 arithmetic).
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
//
// Every kernel takes a compile-time transform length LS: LS = 0 reads the plan from
// the operator at run time (any 2^a or 3 * 2^a length); LS = 2^a fixes the plan at
// compile time so that radices, strides and indices are constants.
#pragma once

#include <atomic>
#include <type_traits>

#include "fft_fast.cuh"
#include "op.cuh"
#include "prof.cuh"

namespace die {

// Rows per block of the row passes: enough for 32-byte segments in the transposed
// accesses (4 complex64 / 2 complex128), at most 512 threads per block.
template <typename C> constexpr int tile_rows() { return sizeof(C) == 8 ? 4 : 2; }
constexpr size_t kStageGreenMaxSmem = 200 * 1024;

template <typename C> __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

// Row stride of the row-pass tiles: the padded length plus two slots, so that the TR
// rows (whose lengths are multiples of 128 bytes) start in different banks.
__host__ __device__ __forceinline__ int tile_stride(int L) { return padded_len(L) + 2; }

// ------------------------------------------------------------------------- K1
template <typename T, typename IO, int EPT, int LS>
__global__ void __launch_bounds__(512) k1_rows_fwd(OpDev<T> op, const IO* __restrict__ u,
                                                   const C_t<T>* __restrict__ chi, C_t<T>* __restrict__ W,
                                                   const int* __restrict__ skip) {
    using C = C_t<T>;
    pdl_wait();
    if (block_flag(skip)) return;
    u += blockIdx.z * op.xs;            // right-hand side of a batched product
    W += blockIdx.z * op.ws;
    constexpr FftPlan kf = pow2_plan(LS ? LS : 16, false);
    const FftPlan pl = LS ? kf : op.f1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int L = LS ? LS : op.M1, G = L / EPT, TR = blockDim.x / G;
    const int rs = threadIdx.x / G, t = threadIdx.x - rs * G;
    const int c = blockIdx.y;
    const int i2_0 = blockIdx.x * TR;
    const int i2 = i2_0 + rs;
    const bool active = i2 < op.n2;
    const long N = (long)op.n1 * op.n2;
    const int Lp = tile_stride(L);
    C* buf = tile + rs * Lp;
    int Ns = 1;
    {
        const int R = pl.radix[0];
        C x[EPT];
        if (active) {
            const IO* urow = u + c * N + (long)i2 * op.n1;
            const C* crow = (c == 2 ? op.chim : chi) + (long)i2 * op.n1;   // H3 plane: chi_m
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
        if (row < op.n2) W[((long)c * L + k1) * op.n2 + row] = tile[r * Lp + pidx(k1)];
    }
}

// ------------------------------------------------------------------------- K2
// One block per column k1: threads [0, G) transform component 0 and [G, 2G)
// component 1, each holding EPT values.  The forward transforms end in shared memory
// in natural order; at the Green multiply every thread reads both components at the
// indices of its first inverse stage.  The column's quarter spectra are staged into
// shared memory at the start (when they fit), so their latency overlaps the FFT.
template <typename T, int EPT, int LS>
__global__ void __launch_bounds__(512) k2_cols(OpDev<T> op, C_t<T>* __restrict__ W, int stage_g,
                                               const int* __restrict__ skip) {
    using C = C_t<T>;
    pdl_wait();
    if (block_flag(skip)) return;
    W += blockIdx.y * op.ws;            // right-hand side of a batched product
    constexpr FftPlan kf = pow2_plan(LS ? LS : 16, false), ki = pow2_plan(LS ? LS : 16, true);
    const int nsf = LS ? kf.ns : op.f2.ns, nsi = LS ? ki.ns : op.i2.ns;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = LS ? LS : op.M2, G = L / EPT, Lp = padded_len(L);
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + Lp;
    C* gs = buf1 + Lp;                          // 3 x Q2 spectra of this column (if staged)
    const int comp = threadIdx.x >= G ? 1 : 0;
    const int t = threadIdx.x - comp * G;
    C* buf = comp ? buf1 : buf0;
    const int k1 = blockIdx.x;
    C* col = W + ((long)comp * op.M1 + k1) * op.n2;
    const int h1 = op.M1 >> 1, h2 = L >> 1;
    const int Q2 = h2 + 1;
    const int k1q = k1 <= h1 ? k1 : op.M1 - k1;
    const bool neg1 = k1 > h1;
    const long plane = (long)op.Q1 * Q2;
    const C* g = op.gq + (long)k1q * Q2;
    if (stage_g) {
        for (int e = threadIdx.x; e < 3 * Q2; e += blockDim.x) {
            const int pl = e / Q2, q = e - pl * Q2;
            gs[e] = g[pl * plane + q];
        }
    }
    C x[EPT];
    int Ns = 1;
#pragma unroll
    for (int s = 0; s < nsf; s++) {
        const int R = LS ? kf.radix[s] : op.f2.radix[s];
        if (s == 0) {
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                const int idx = reg_index<EPT>(e, R, L, t, G);
                x[e] = idx < op.n2 ? col[idx] : czero<C>();
            }
        } else {
            load_any<C, EPT>(R, buf, x, L, t, G);
            __syncthreads();
        }
        compute_any<C, EPT, false>(R, x, L, Ns, t, G, op.tw2);
        store_any<C, EPT>(R, buf, x, L, Ns, t, G);
        __syncthreads();
        Ns *= R;
    }
    {   // 2 x 2 Green-spectrum multiply at frequencies (k1, k2)
        const int R = LS ? ki.radix[0] : op.i2.radix[0];
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            const int k2 = reg_index<EPT>(e, R, L, t, G);
            const int k2q = k2 <= h2 ? k2 : L - k2;
            const bool neg = neg1 != (k2 > h2);
            const C a = buf0[pidx(k2)], b = buf1[pidx(k2)];
            C gd, go;                           // diagonal (G11 or G22) and off-diagonal G12
            if (stage_g) { gd = gs[comp * Q2 + k2q]; go = gs[2 * Q2 + k2q]; }
            else { gd = g[comp * plane + k2q]; go = g[2 * plane + k2q]; }
            if (neg) { go.x = -go.x; go.y = -go.y; }
            x[e] = comp == 0 ? cadd(cmul(gd, a), cmul(go, b)) : cadd(cmul(go, a), cmul(gd, b));
        }
    }
    __syncthreads();
    Ns = 1;
#pragma unroll
    for (int s = 0; s < nsi; s++) {
        const int R = LS ? ki.radix[s] : op.i2.radix[s];
        if (s > 0) {
            load_any<C, EPT>(R, buf, x, L, t, G);
            __syncthreads();
        }
        compute_any<C, EPT, true>(R, x, L, Ns, t, G, op.tw2);
        if (s < nsi - 1) {
            store_any<C, EPT>(R, buf, x, L, Ns, t, G);
            __syncthreads();
        } else {
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                const int idx = reg_index<EPT>(e, R, L, t, G);
                if (idx < op.n2) col[idx] = x[e];
            }
        }
        Ns *= R;
    }
}

// The column pass of the three-plane operator (DIE_TE_MAG): threads [0, G), [G, 2G) and
// [2G, 3G) transform E1, E2 and H3; the 3 x 3 Green multiply reads the six quarter
// spectra from global memory (planes 0..5: G11, G22, G12, G13, G23, G33).  A spectrum
// at a mirrored frequency is the stored one times the kernel's parity: G12 (odd in x1 and
// x2) flips when exactly one of k1, k2 is mirrored, G13 (odd in x2) when k2 is, G23 (odd
// in x1) when k1 is.
template <typename T, int EPT, int LS, int MAXT>
__global__ void __launch_bounds__(MAXT) k2_cols3(OpDev<T> op, C_t<T>* __restrict__ W, const int* __restrict__ skip) {
    using C = C_t<T>;
    pdl_wait();
    if (block_flag(skip)) return;
    W += blockIdx.y * op.ws;            // right-hand side of a batched product
    constexpr FftPlan kf = pow2_plan(LS ? LS : 16, false), ki = pow2_plan(LS ? LS : 16, true);
    const int nsf = LS ? kf.ns : op.f2.ns, nsi = LS ? ki.ns : op.i2.ns;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = LS ? LS : op.M2, G = L / EPT, Lp = padded_len(L);
    C* bufs = reinterpret_cast<C*>(smem_raw);           // three planes of Lp
    const int comp = threadIdx.x / G;
    const int t = threadIdx.x - comp * G;
    C* buf = bufs + comp * Lp;
    const int k1 = blockIdx.x;
    C* col = W + ((long)comp * op.M1 + k1) * op.n2;
    const int h1 = op.M1 >> 1, h2 = L >> 1;
    const int Q2 = h2 + 1;
    const int k1q = k1 <= h1 ? k1 : op.M1 - k1;
    const bool neg1 = k1 > h1;
    const long plane = (long)op.Q1 * Q2;
    const C* g = op.gq + (long)k1q * Q2;
    C x[EPT];
    int Ns = 1;
#pragma unroll
    for (int s = 0; s < nsf; s++) {
        const int R = LS ? kf.radix[s] : op.f2.radix[s];
        if (s == 0) {
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                const int idx = reg_index<EPT>(e, R, L, t, G);
                x[e] = idx < op.n2 ? col[idx] : czero<C>();
            }
        } else {
            load_any<C, EPT>(R, buf, x, L, t, G);
            __syncthreads();
        }
        compute_any<C, EPT, false>(R, x, L, Ns, t, G, op.tw2);
        store_any<C, EPT>(R, buf, x, L, Ns, t, G);
        __syncthreads();
        Ns *= R;
    }
    {   // 3 x 3 Green-spectrum multiply at frequencies (k1, k2)
        const int R = LS ? ki.radix[0] : op.i2.radix[0];
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            const int k2 = reg_index<EPT>(e, R, L, t, G);
            const int k2q = k2 <= h2 ? k2 : L - k2;
            const bool neg2 = k2 > h2;
            const C a = bufs[pidx(k2)], b = bufs[Lp + pidx(k2)], c = bufs[2 * Lp + pidx(k2)];
            C g12 = g[2 * plane + k2q], g13 = g[3 * plane + k2q], g23 = g[4 * plane + k2q];
            if (neg1 != neg2) { g12.x = -g12.x; g12.y = -g12.y; }
            if (neg2) { g13.x = -g13.x; g13.y = -g13.y; }
            if (neg1) { g23.x = -g23.x; g23.y = -g23.y; }
            if (comp == 0) x[e] = cadd(cadd(cmul(g[k2q], a), cmul(g12, b)), cmul(g13, c));
            else if (comp == 1) x[e] = cadd(cadd(cmul(g12, a), cmul(g[plane + k2q], b)), cmul(g23, c));
            else x[e] = cadd(cadd(cmul(g13, a), cmul(g23, b)), cmul(g[5 * plane + k2q], c));
        }
    }
    __syncthreads();
    Ns = 1;
#pragma unroll
    for (int s = 0; s < nsi; s++) {
        const int R = LS ? ki.radix[s] : op.i2.radix[s];
        if (s > 0) {
            load_any<C, EPT>(R, buf, x, L, t, G);
            __syncthreads();
        }
        compute_any<C, EPT, true>(R, x, L, Ns, t, G, op.tw2);
        if (s < nsi - 1) {
            store_any<C, EPT>(R, buf, x, L, Ns, t, G);
            __syncthreads();
        } else {
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                const int idx = reg_index<EPT>(e, R, L, t, G);
                if (idx < op.n2) col[idx] = x[e];
            }
        }
        Ns *= R;
    }
}

// Load the transposed tile W[c][0..M1)[i2_0 .. i2_0+TR) into shared memory rows.
template <typename C>
__device__ __forceinline__ void load_tile(C* tile, const C* __restrict__ W, int c, int i2_0, int M1, int n2, int TR) {
    const int Lp = tile_stride(M1);
    for (int e = threadIdx.x; e < M1 * TR; e += blockDim.x) {
        const int k1 = e / TR, r = e - k1 * TR;
        const int row = i2_0 + r;
        tile[r * Lp + pidx(k1)] = row < n2 ? W[((long)c * M1 + k1) * n2 + row] : czero<C>();
    }
    __syncthreads();
}

// ------------------------------------------------------------------------- K3
// y = u - z for one tile of rows; u of element type U, y of IO.
template <typename T, typename U, typename IO, int EPT, int LS>
__global__ void __launch_bounds__(512) k3_rows_inv(OpDev<T> op, const C_t<T>* __restrict__ W,
                                                   const U* __restrict__ u, IO* __restrict__ y,
                                                   const int* __restrict__ skip) {
    using C = C_t<T>;
    pdl_wait();
    if (block_flag(skip)) return;
    W += blockIdx.z * op.ws;            // right-hand side of a batched product
    u += blockIdx.z * op.xs;
    y += blockIdx.z * op.xs;
    constexpr FftPlan ki = pow2_plan(LS ? LS : 16, true);
    const FftPlan iv = LS ? ki : op.i1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int L = LS ? LS : op.M1, G = L / EPT, TR = blockDim.x / G;
    const int rs = threadIdx.x / G, t = threadIdx.x - rs * G;
    const int c = blockIdx.y;
    const int i2_0 = blockIdx.x * TR;
    const int i2 = i2_0 + rs;
    const bool active = i2 < op.n2;
    const long N = (long)op.n1 * op.n2;
    C* buf = tile + rs * tile_stride(L);
    load_tile<C>(tile, W, c, i2_0, L, op.n2, TR);
    int Ns = 1;
    C x[EPT];
#pragma unroll
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
template <typename T, typename IO, int EPT, int LS>
__global__ void __launch_bounds__(512) k3k1_rows(OpDev<T> op, C_t<T>* __restrict__ W, const IO* __restrict__ u,
                                                 const C_t<T>* __restrict__ chir, C_t<T>* __restrict__ vbuf,
                                                 const int* __restrict__ skip) {
    using C = C_t<T>;
    pdl_wait();
    if (block_flag(skip)) return;
    W += blockIdx.z * op.ws;            // right-hand side of a batched product
    u += blockIdx.z * op.xs;
    vbuf += blockIdx.z * op.xs;
    constexpr FftPlan kf = pow2_plan(LS ? LS : 16, false), ki = pow2_plan(LS ? LS : 16, true);
    const FftPlan f = LS ? kf : op.f1;
    const FftPlan iv = LS ? ki : op.i1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int L = LS ? LS : op.M1, G = L / EPT, TR = blockDim.x / G;
    const int rs = threadIdx.x / G, t = threadIdx.x - rs * G;
    const int c = blockIdx.y;
    const int i2_0 = blockIdx.x * TR;
    const int i2 = i2_0 + rs;
    const bool active = i2 < op.n2;
    const long N = (long)op.n1 * op.n2;
    C* buf = tile + rs * tile_stride(L);
    load_tile<C>(tile, W, c, i2_0, L, op.n2, TR);
    int Ns = 1;
    C x[EPT];
#pragma unroll
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
    {
        const int R = iv.radix[iv.ns - 1];      // == f.radix[0]: inverse plan is the reversed forward plan
        if (active) {
            const long off = c * N + (long)i2 * op.n1;
            const C* crow = (c == 2 ? op.chim : chir) + (long)i2 * op.n1;  // the regulariser keeps chi_m
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
    const int Lp = tile_stride(L);
    for (int e = threadIdx.x; e < L * TR; e += blockDim.x) {
        const int k1 = e / TR, r = e - k1 * TR;
        const int row = i2_0 + r;
        if (row < op.n2) W[((long)c * L + k1) * op.n2 + row] = tile[r * Lp + pidx(k1)];
    }
}

// ------------------------------------------------------------------ fast path
// Grids with n = L / 2 exactly and L = 2^a in [256, 4096] (the padding is then exactly
// half of every transform): the same passes with the compile-time stages of
// fft_fast.cuh.  The zero inputs (index >= n) of the forward transforms and the
// discarded outputs (index >= n) of the inverse ones are known at compile time.
template <typename C, int L> constexpr int fast_tr() {
    return tile_rows<C>() * (L / 16) <= kRowsMaxThreads ? tile_rows<C>() : kRowsMaxThreads / (L / 16);
}
template <int L> constexpr int tile_stride_c() { return L + (L >> 4) + 2; }

// Asynchronous global -> shared copy of one complex value (no register staging), and the
// wait for all of this thread's copies.
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* smem, const C* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(C) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
    else asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Blocks per SM that the column pass should fit: all M1 = 1024 complex64 columns in one
// wave of 152 SMs needs 7 (at most 72 registers per thread).
template <typename C, int L> constexpr int k2_min_blocks() { return (sizeof(C) == 8 && L == 1024) ? 7 : 1; }

// Transposed tile I/O of the row passes: thread (k0 = tid / TR, r = tid % TR) moves
// elements k1 = k0 + it G, it < 16, of tile row r.
template <typename C, int L, int TR, bool STORE>
__device__ __forceinline__ void tile_io(C* tile, C* __restrict__ W, int c, int i2_0, int n2) {
    constexpr int G = L / 16, Lp = tile_stride_c<L>();
    const int r = threadIdx.x % TR, k0 = threadIdx.x / TR;
    const int row = i2_0 + r;
    C* t = tile + r * Lp + pidx(k0);
    C* g = W + ((long)c * L + k0) * n2 + row;
    const long gs = (long)G * n2;
#pragma unroll
    for (int it = 0; it < 16; it++) {
        const int off = it * G + ((it * G) >> 4);
        if constexpr (STORE) {
            if (row < n2) g[it * gs] = t[off];
        } else {
            t[off] = row < n2 ? g[it * gs] : czero<C>();
        }
    }
}

template <typename T, typename IO, int L, int TR>
__global__ void __launch_bounds__(512) k1_fast(OpDev<T> op, const IO* __restrict__ u, const C_t<T>* __restrict__ chi,
                                               C_t<T>* __restrict__ W, const int* __restrict__ skip) {
    using C = C_t<T>;
    constexpr int G = L / 16, n1 = L / 2;
    using F0 = typename PlanStage<C, L, false, 0>::St;
    pdl_wait();
    if (block_flag(skip)) return;
    u += blockIdx.z * op.xs;            // right-hand side of a batched product
    W += blockIdx.z * op.ws;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int rs = threadIdx.x / G, t = threadIdx.x % G;
    const int c = blockIdx.y, i2_0 = blockIdx.x * TR, i2 = i2_0 + rs;
    const bool active = i2 < op.n2;
    C* buf = tile + rs * tile_stride_c<L>();
    C x[16];
    if (active) {
        const long N = (long)n1 * op.n2;
        const IO* ur = u + c * N + (long)i2 * n1 + t;
        const C* cr = chi + (long)i2 * n1 + t;
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const int idx = F0::index(e);
            x[e] = idx < n1 ? cmul(cvt<C>(ur[idx]), cr[idx]) : czero<C>();
        }
        F0::compute(x, t, op.twx1);
        F0::store(buf, x, t);
    }
    __syncthreads();
    run_fast<C, L, false, 1, P2<L>::fwd.ns, false>(buf, x, t, op.twx1, active);
    tile_io<C, L, TR, true>(tile, W, c, i2_0, op.n2);
}

// First row pass of a deflated FP32-inner product (complex64): per element
// z = v + sum_i V32_i cf_i (v = w / ||w|| written back to the FP64 Arnoldi vector, or
// the complex64 x), stored to zout for the later passes, then chi * z and the forward
// row transform as in k1_fast.  The basis loads go five vectors (40 loads) at a time.
template <int L, int TR>
__global__ void __launch_bounds__(512) k1_defl_fast(OpDev<float> op, DeflIn d, const float2* __restrict__ chi,
                                                    float2* __restrict__ zout, float2* __restrict__ W,
                                                    const int* __restrict__ skip) {
    using C = float2;
    constexpr int G = L / 16, n1 = L / 2;
    using F0 = typename PlanStage<C, L, false, 0>::St;
    __shared__ float2 cs[32];
    pdl_wait();
    if (block_flag(skip)) return;
    for (int i = threadIdx.x; i < d.r; i += blockDim.x) cs[i] = __ldcg(&d.cf[i]);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int rs = threadIdx.x / G, t = threadIdx.x % G;
    const int c = blockIdx.y, i2_0 = blockIdx.x * TR, i2 = i2_0 + rs;
    const bool active = i2 < op.n2;
    C* buf = tile + rs * tile_stride_c<L>();
    __syncthreads();
    C x[16];
    if (active) {
        const long off = c * ((long)n1 * op.n2) + (long)i2 * n1 + t;
        C zq[8];
        if (d.w) {
            const double sc = *d.inv;
#pragma unroll
            for (int e = 0, q = 0; e < 16; e++) {
                const int idx = F0::index(e);
                if (idx < n1) {
                    double2 u = d.w[off + idx];
                    u.x *= sc;
                    u.y *= sc;
                    d.w[off + idx] = u;
                    if (d.wm) d.wm[off + idx] = u.x - u.y;
                    zq[q++] = make_float2((float)u.x, (float)u.y);
                }
            }
        } else {
#pragma unroll
            for (int e = 0, q = 0; e < 16; e++)
                if (F0::index(e) < n1) zq[q++] = d.x[off + F0::index(e)];
        }
        constexpr int VB = 5;                     // basis vectors per round of loads (40 in flight)
        for (int i0 = 0; i0 < d.r; i0 += VB) {
            C a[VB][8];
#pragma unroll
            for (int v = 0; v < VB; v++) {
                const C* p = d.V32 + (long)(i0 + v < d.r ? i0 + v : i0) * d.ld + off;
#pragma unroll
                for (int e = 0, q = 0; e < 16; e++)
                    if (F0::index(e) < n1) a[v][q++] = p[F0::index(e)];
            }
#pragma unroll
            for (int v = 0; v < VB; v++) {
                if (i0 + v < d.r) {
                    const C cv = cs[i0 + v];
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        zq[q].x = fmaf(a[v][q].x, cv.x, zq[q].x);
                        zq[q].x = fmaf(-a[v][q].y, cv.y, zq[q].x);
                        zq[q].y = fmaf(a[v][q].x, cv.y, zq[q].y);
                        zq[q].y = fmaf(a[v][q].y, cv.x, zq[q].y);
                    }
                }
            }
        }
        const C* cr = chi + (long)i2 * n1 + t;
#pragma unroll
        for (int e = 0, q = 0; e < 16; e++) {
            const int idx = F0::index(e);
            if (idx < n1) {
                zout[off + idx] = zq[q];
                x[e] = cmul(zq[q], cr[idx]);
                q++;
            } else {
                x[e] = czero<C>();
            }
        }
        F0::compute(x, t, op.twx1);
        F0::store(buf, x, t);
    }
    __syncthreads();
    run_fast<C, L, false, 1, P2<L>::fwd.ns, false>(buf, x, t, op.twx1, active);
    tile_io<C, L, TR, true>(tile, W, c, i2_0, op.n2);
}

template <typename T, int L>
__global__ void __launch_bounds__(2 * (L / 16), k2_min_blocks<C_t<T>, L>()) k2_fast(OpDev<T> op, C_t<T>* __restrict__ W,
                                                                                 int stage_g, const int* __restrict__ skip) {
    using C = C_t<T>;
    constexpr int G = L / 16, n2 = L / 2, Q2 = L / 2 + 1, Lp = L + (L >> 4);
    constexpr int nsf = P2<L>::fwd.ns, nsi = P2<L>::inv.ns;
    using F0 = typename PlanStage<C, L, false, 0>::St;
    using I0 = typename PlanStage<C, L, true, 0>::St;
    using IL = typename PlanStage<C, L, true, nsi - 1>::St;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + Lp;
    C* gs = buf1 + Lp;
    const int comp = threadIdx.x >= G ? 1 : 0;
    const int t = threadIdx.x - comp * G;
    C* buf = comp ? buf1 : buf0;
    W += blockIdx.y * op.ws;            // right-hand side of a batched product
    const int k1 = blockIdx.x;
    C* col = W + ((long)comp * op.M1 + k1) * n2 + t;
    const int h1 = op.M1 >> 1;
    const int k1q = k1 <= h1 ? k1 : op.M1 - k1;
    const bool neg1 = k1 > h1;
    const long plane = (long)op.Q1 * Q2;
    const C* g = op.gq + (long)k1q * Q2;
    if (stage_g) {   // the column's three quarter-spectrum rows (operator constants), issued
                     // before the wait on the previous kernel; they land during the forward FFT
        for (int e = threadIdx.x; e < 3 * Q2; e += 2 * G) {
            const int pl = e / Q2, q = e - pl * Q2;
            cp_async_elem(gs + e, g + pl * plane + q);
        }
    }
    pdl_wait();
    if (block_flag(skip)) {
        cp_async_wait_all();
        return;
    }
    C x[16];
#pragma unroll
    for (int e = 0; e < 16; e++) {
        const int idx = F0::index(e);
        x[e] = idx < n2 ? col[idx] : czero<C>();
    }
    F0::compute(x, t, op.twx2);
    F0::store(buf, x, t);
    __syncthreads();
    run_fast<C, L, false, 1, nsf, false>(buf, x, t, op.twx2, true);
    if (stage_g) {
        cp_async_wait_all();
        __syncthreads();
    }
    {   // 2 x 2 Green-spectrum multiply at the first inverse stage's indices k2 = t + c
        const long ps = stage_g ? (long)Q2 : plane;
        const C* gsrc = stage_g ? gs : g;
        const C* gdp = gsrc + comp * ps + t;     // k2 <= L/2: quarter index k2
        const C* gop = gsrc + 2 * ps + t;
        const C* gdm = gsrc + comp * ps - t;     // k2 > L/2: quarter index L - k2
        const C* gom = gsrc + 2 * ps - t;
        const C* a0 = buf0 + pidx(t);
        const C* a1 = buf1 + pidx(t);
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const int c = I0::index(e);
            const C a = a0[c + (c >> 4)], b = a1[c + (c >> 4)];
            C gd, go;
            bool neg2;
            if (c < L / 2) { gd = gdp[c]; go = gop[c]; neg2 = false; }
            else { gd = gdm[L - c]; go = gom[L - c]; neg2 = c > L / 2 || t > 0; }
            if (neg1 != neg2) { go.x = -go.x; go.y = -go.y; }
            x[e] = comp == 0 ? cadd(cmul(gd, a), cmul(go, b)) : cadd(cmul(go, a), cmul(gd, b));
        }
    }
    __syncthreads();
    I0::compute(x, t, op.twx2);
    I0::store(buf, x, t);
    __syncthreads();
    run_fast<C, L, true, 1, nsi - 1, false>(buf, x, t, op.twx2, true);
    IL::load(buf, x, t);
    IL::compute(x, t, op.twx2);
#pragma unroll
    for (int e = 0; e < 16; e++) {
        const int idx = IL::index(e);
        if (idx < n2) col[idx] = x[e];
    }
}

// Complex64 column pass with both components in the same thread (G threads per column):
// the last forward stage leaves each thread's values at the indices where the first
// inverse stage (same radix: the inverse plan is the reversed forward plan) wants them,
// so the 2 x 2 Green multiply is done in registers between the two, with no shared-
// memory round trip, and every twiddle serves both components.
template <typename T, int L>
__global__ void __launch_bounds__(L / 16, (L == 1024 ? 7 : 1)) k2_fast2(OpDev<T> op, C_t<T>* __restrict__ W,
                                                                        int stage_g, const int* __restrict__ skip) {
    using C = C_t<T>;
    constexpr int G = L / 16, n2 = L / 2, Q2 = L / 2 + 1, Lp = L + (L >> 4);
    constexpr int nsf = P2<L>::fwd.ns, nsi = P2<L>::inv.ns;
    using F0 = typename PlanStage<C, L, false, 0>::St;
    using FL = typename PlanStage<C, L, false, nsf - 1>::St;
    using I0 = typename PlanStage<C, L, true, 0>::St;
    using IL = typename PlanStage<C, L, true, nsi - 1>::St;
    static_assert(FL::kR == I0::kR, "the inverse plan is the reversed forward plan");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + Lp;
    C* gs = buf1 + Lp;
    const int t = threadIdx.x;
    W += blockIdx.y * op.ws;            // right-hand side of a batched product
    const int k1 = blockIdx.x;
    C* col0 = W + (long)k1 * n2 + t;
    C* col1 = W + ((long)op.M1 + k1) * n2 + t;
    const int h1 = op.M1 >> 1;
    const int k1q = k1 <= h1 ? k1 : op.M1 - k1;
    const bool neg1 = k1 > h1;
    const long plane = (long)op.Q1 * Q2;
    const C* g = op.gq + (long)k1q * Q2;
    if (stage_g) {   // the column's three quarter-spectrum rows (operator constants), issued
                     // before the wait on the previous kernel; they land during the forward FFT
        for (int e = t; e < 3 * Q2; e += G) {
            const int pl = e / Q2, q = e - pl * Q2;
            cp_async_elem(gs + e, g + pl * plane + q);
        }
    }
    pdl_wait();
    if (block_flag(skip)) {
        cp_async_wait_all();
        return;
    }
    C x0[16], x1[16];
#pragma unroll
    for (int e = 0; e < 16; e++) {
        const int idx = F0::index(e);
        x0[e] = idx < n2 ? col0[idx] : czero<C>();
        x1[e] = idx < n2 ? col1[idx] : czero<C>();
    }
    F0::compute2(x0, x1, t, op.twx2);
    F0::store(buf0, x0, t);
    F0::store(buf1, x1, t);
    __syncthreads();
    run_fast2<C, L, false, 1, nsf - 1>(buf0, buf1, x0, x1, t, op.twx2);
    FL::load(buf0, x0, t);
    FL::load(buf1, x1, t);
    FL::compute2(x0, x1, t, op.twx2);
    if (stage_g) cp_async_wait_all();
    __syncthreads();             // spectra visible; every thread has read its last forward stage
    {   // 2 x 2 Green-spectrum multiply at k2 = t + c (c = I0::index(e))
        const long ps = stage_g ? (long)Q2 : plane;
        const C* gsrc = stage_g ? gs : g;
        const C* g11p = gsrc + t;           // k2 <= L/2: quarter index k2
        const C* g22p = gsrc + ps + t;
        const C* g12p = gsrc + 2 * ps + t;
        const C* g11m = gsrc - t;           // k2 > L/2: quarter index L - k2
        const C* g22m = gsrc + ps - t;
        const C* g12m = gsrc + 2 * ps - t;
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const int c = I0::index(e);
            C a, b, go;
            bool neg2;
            if (c < L / 2) { a = g11p[c]; b = g22p[c]; go = g12p[c]; neg2 = false; }
            else { a = g11m[L - c]; b = g22m[L - c]; go = g12m[L - c]; neg2 = c > L / 2 || t > 0; }
            if (neg1 != neg2) { go.x = -go.x; go.y = -go.y; }
            const C u0 = x0[e], u1 = x1[e];
            x0[e] = cadd(cmul(a, u0), cmul(go, u1));
            x1[e] = cadd(cmul(go, u0), cmul(b, u1));
        }
    }
    I0::compute2(x0, x1, t, op.twx2);
    I0::store(buf0, x0, t);
    I0::store(buf1, x1, t);
    __syncthreads();
    run_fast2<C, L, true, 1, nsi - 1>(buf0, buf1, x0, x1, t, op.twx2);
    IL::load(buf0, x0, t);
    IL::load(buf1, x1, t);
    IL::compute2(x0, x1, t, op.twx2);
#pragma unroll
    for (int e = 0; e < 16; e++) {
        const int idx = IL::index(e);
        if (idx < n2) { col0[idx] = x0[e]; col1[idx] = x1[e]; }
    }
}

template <typename T, typename U, typename IO, int L, int TR>
__global__ void __launch_bounds__(512) k3_fast(OpDev<T> op, const C_t<T>* __restrict__ W, const U* __restrict__ u,
                                               IO* __restrict__ y, const int* __restrict__ skip) {
    using C = C_t<T>;
    constexpr int G = L / 16, n1 = L / 2, ns = P2<L>::inv.ns;
    using IL = typename PlanStage<C, L, true, ns - 1>::St;
    pdl_wait();
    if (block_flag(skip)) return;
    W += blockIdx.z * op.ws;            // right-hand side of a batched product
    u += blockIdx.z * op.xs;
    y += blockIdx.z * op.xs;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int rs = threadIdx.x / G, t = threadIdx.x % G;
    const int c = blockIdx.y, i2_0 = blockIdx.x * TR, i2 = i2_0 + rs;
    const bool active = i2 < op.n2;
    C* buf = tile + rs * tile_stride_c<L>();
    const long off = c * ((long)n1 * op.n2) + (long)(active ? i2 : 0) * n1 + t;
    U up[8];                    // u at this thread's output indices, loaded before the FFT
#pragma unroll
    for (int e = 0, q = 0; e < 16; e++)
        if (IL::index(e) < n1) up[q++] = u[off + IL::index(e)];
    tile_io<C, L, TR, false>(tile, const_cast<C*>(W), c, i2_0, op.n2);
    __syncthreads();
    C x[16];
    run_fast<C, L, true, 0, ns - 1, false>(buf, x, t, op.twx1, active);
    if (!active) return;
    IL::load(buf, x, t);
    IL::compute(x, t, op.twx1);
#pragma unroll
    for (int e = 0, q = 0; e < 16; e++) {
        const int idx = IL::index(e);
        if (idx < n1) y[off + idx] = csub(cvt<IO>(up[q++]), cvt<IO>(x[e]));
    }
}

template <typename T, typename IO, int L, int TR>
__global__ void __launch_bounds__(512) k3k1_fast(OpDev<T> op, C_t<T>* __restrict__ W, const IO* __restrict__ u,
                                                 const C_t<T>* __restrict__ chir, C_t<T>* __restrict__ vbuf,
                                                 const int* __restrict__ skip) {
    using C = C_t<T>;
    constexpr int G = L / 16, n1 = L / 2;
    constexpr int nsi = P2<L>::inv.ns, nsf = P2<L>::fwd.ns;
    using IL = typename PlanStage<C, L, true, nsi - 1>::St;
    using F0 = typename PlanStage<C, L, false, 0>::St;
    static_assert(IL::kR == F0::kR, "the inverse plan is the reversed forward plan");
    pdl_wait();
    if (block_flag(skip)) return;
    W += blockIdx.z * op.ws;            // right-hand side of a batched product
    u += blockIdx.z * op.xs;
    vbuf += blockIdx.z * op.xs;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int rs = threadIdx.x / G, t = threadIdx.x % G;
    const int c = blockIdx.y, i2_0 = blockIdx.x * TR, i2 = i2_0 + rs;
    const bool active = i2 < op.n2;
    C* buf = tile + rs * tile_stride_c<L>();
    const long off = c * ((long)n1 * op.n2) + (long)(active ? i2 : 0) * n1 + t;
    const C* cr = chir + (long)(active ? i2 : 0) * n1 + t;
    C up[8], cp[8];             // u and chi' at this thread's indices, loaded before the FFT
#pragma unroll
    for (int e = 0, q = 0; e < 16; e++)
        if (IL::index(e) < n1) { up[q] = cvt<C>(u[off + IL::index(e)]); cp[q] = cr[IL::index(e)]; q++; }
    tile_io<C, L, TR, false>(tile, W, c, i2_0, op.n2);
    __syncthreads();
    C x[16];
    run_fast<C, L, true, 0, nsi - 1, false>(buf, x, t, op.twx1, active);
    if (active) {
        IL::load(buf, x, t);
        IL::compute(x, t, op.twx1);
        // v = u - z (first product), kept for the final subtraction; then chi' v -> FFT
#pragma unroll
        for (int e = 0, q = 0; e < 16; e++) {
            const int idx = IL::index(e);
            if (idx < n1) {
                const C v = csub(up[q], x[e]);
                vbuf[off + idx] = v;
                x[e] = cmul(v, cp[q]);
                q++;
            } else {
                x[e] = czero<C>();
            }
        }
    }
    __syncthreads();            // every thread has read its last inverse stage from the tile
    if (active) {
        F0::compute(x, t, op.twx1);
        F0::store(buf, x, t);
    }
    __syncthreads();
    run_fast<C, L, false, 1, nsf, false>(buf, x, t, op.twx1, active);
    tile_io<C, L, TR, true>(tile, W, c, i2_0, op.n2);
}

// --------------------------------------------------------------------- launch
struct Launch { dim3 grid, block; size_t smem; };
inline Launch with_z(Launch l, int nb) { l.grid.z = nb; return l; }

template <typename T>
inline Launch rows_launch(const OpDev<T>& v) {
    using C = C_t<T>;
    const int G = v.M1 / v.f1.ept;
    int TR = tile_rows<C>();
    while (TR > 1 && TR * G > kRowsMaxThreads) TR /= 2;
    return Launch{dim3((v.n2 + TR - 1) / TR, v.planes), dim3(TR * G), (size_t)TR * tile_stride(v.M1) * sizeof(C)};
}

template <typename T>
inline Launch cols_launch(const OpDev<T>& v, int* stage_g) {
    using C = C_t<T>;
    if (v.planes == 3) {    // three components per column, spectra read from global memory
        *stage_g = 0;
        return Launch{dim3(v.M1), dim3(3 * (v.M2 / v.f2.ept)), (size_t)3 * padded_len(v.M2) * sizeof(C)};
    }
    const size_t base = (size_t)2 * padded_len(v.M2) * sizeof(C);
    const size_t staged = base + (size_t)3 * v.Q2 * sizeof(C);
    *stage_g = staged <= kStageGreenMaxSmem ? 1 : 0;
    return Launch{dim3(v.M1), dim3(2 * (v.M2 / v.f2.ept)), *stage_g ? staged : base};
}

// Launch a kernel instantiation, raising its dynamic shared-memory limit on first use
// to what the 227 KB per block leaves beside the kernel's static shared memory.
template <typename K, typename... Args>
inline void launch_kernel(K kernel, std::atomic<bool>& attr_set, const Launch& l, cudaStream_t st, Args... args) {
    if (!attr_set.load(std::memory_order_acquire)) {
        cudaFuncAttributes fa = {};
        const size_t stat = cudaFuncGetAttributes(&fa, kernel) == cudaSuccess ? fa.sharedSizeBytes : 1024;
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(227 * 1024 - stat));
        attr_set.store(true, std::memory_order_release);
    }
    launch_pdl(kernel, l.grid, l.block, l.smem, st, args...);
}

// Compile-time lengths with a dedicated instantiation; anything else takes the runtime plan.
#define DIE_POW2_SWITCH(M, CASE, DEFAULT) \
    switch (M) {                          \
        case 64: CASE(64); break;         \
        case 128: CASE(128); break;       \
        case 256: CASE(256); break;       \
        case 512: CASE(512); break;       \
        case 1024: CASE(1024); break;     \
        case 2048: CASE(2048); break;     \
        case 4096: CASE(4096); break;     \
        default: DEFAULT; break;          \
    }

// Grids on the fast path: n = L / 2 with L = 2^a in [256, 4096] (per direction).
// (Two-plane operators only: the three-plane one runs on the runtime-plan kernels.)
template <typename T> inline bool fast_rows(const OpDev<T>& v) {
    return v.planes == 2 && 2 * v.n1 == v.M1 && v.M1 >= 256 && v.M1 <= 4096 && (v.M1 & (v.M1 - 1)) == 0;
}
template <typename T> inline bool fast_cols(const OpDev<T>& v) {
    return v.planes == 2 && 2 * v.n2 == v.M2 && v.M2 >= 256 && v.M2 <= 4096 && (v.M2 & (v.M2 - 1)) == 0;
}
template <typename C, int L, int TR> inline Launch rows_launch_fast(int n2) {
    return Launch{dim3((n2 + TR - 1) / TR, 2), dim3(TR * (L / 16)), (size_t)TR * tile_stride_c<L>() * sizeof(C)};
}

#define DIE_FAST_SWITCH(M, CASE)  \
    switch (M) {                  \
        case 256: CASE(256); break;   \
        case 512: CASE(512); break;   \
        case 1024: CASE(1024); break; \
        case 2048: CASE(2048); break; \
        case 4096: CASE(4096); break; \
        default: break;               \
    }

// Tile height of the fast row passes: the rows of one block (TR).  0 selects fast_tr,
// the default of the element type and length; an operator's schedule (dieop_autotune,
// dieop_set_tile_rows) may pick another valid height for its complex64 passes.  Every row
// is transformed by the same threads and stages whatever TR is, so the products are
// bit-identical for all heights.
template <typename C, int L, int TR> constexpr int tile_of() { return TR == 0 ? fast_tr<C, L>() : TR; }
template <typename C, int L, int TR> constexpr bool tile_ok() {
    return TR == 0 || (TR * (L / 16) <= kRowsMaxThreads && TR != fast_tr<C, L>());
}

// The fast row passes at one tile height (definitions in rows_fast.cuh).
template <typename T, typename IO, int TR>
void rows_fwd_fast(const OpDev<T>& v, const IO* u, const C_t<T>* chi, C_t<T>* W, const int* skip, cudaStream_t st,
                   int nb);
template <typename T, typename U, typename IO, int TR>
void rows_inv_fast(const OpDev<T>& v, const C_t<T>* W, const U* u, IO* y, const int* skip, cudaStream_t st, int nb);
template <typename T, typename IO, int TR>
void rows_inv_fwd_fast(const OpDev<T>& v, C_t<T>* W, const IO* u, const C_t<T>* chir, C_t<T>* vb, const int* skip,
                       cudaStream_t st, int nb);
template <int TR>
void rows_defl_fast(const OpDev<float>& v, const DeflIn& d, const float2* chi, float2* z, float2* W, const int* skip,
                    cudaStream_t st);

// Calls F<TR> with the tile height of the view (complex64: the operator's schedule).
template <typename T, typename F>
inline void with_tile_rows(const OpDev<T>& v, F&& f) {
    if constexpr (sizeof(C_t<T>) == 8) {
        switch (tile_rows_code(v.tr, v.M1)) {
            case 1: f(std::integral_constant<int, 1>{}); return;
            case 2: f(std::integral_constant<int, 2>{}); return;
            case 8: f(std::integral_constant<int, 8>{}); return;
            default: break;
        }
    }
    f(std::integral_constant<int, 0>{});
}

// nb > 1: a batched product over nb right-hand sides (grid z: row passes, grid y: columns).
template <typename T, typename IO>
inline void launch_k1(const OpDev<T>& v, const IO* u, const C_t<T>* chi, C_t<T>* W, const int* skip, cudaStream_t st,
                      int nb = 1) {
    if (fast_rows(v)) {
        with_tile_rows(v, [&](auto tr) { rows_fwd_fast<T, IO, decltype(tr)::value>(v, u, chi, W, skip, st, nb); });
        return;
    }
    const Launch l = with_z(rows_launch(v), nb);
#define K1_CASE(LSV) { static std::atomic<bool> a_{false}; launch_kernel(k1_rows_fwd<T, IO, 16, LSV>, a_, l, st, v, u, chi, W, skip); }
#define K1_DEF { static std::atomic<bool> a16{false}, a12{false};                                                     \
                 if (v.f1.ept == 16) launch_kernel(k1_rows_fwd<T, IO, 16, 0>, a16, l, st, v, u, chi, W, skip); \
                 else launch_kernel(k1_rows_fwd<T, IO, 12, 0>, a12, l, st, v, u, chi, W, skip); }
    DIE_PROF(PK_ROWS_FWD, st, DIE_POW2_SWITCH(v.M1, K1_CASE, K1_DEF));
#undef K1_CASE
#undef K1_DEF
}

template <typename T>
inline void launch_k2(const OpDev<T>& v, C_t<T>* W, const int* skip, cudaStream_t st, int nb = 1) {
    int sg = 0;
    Launch l = cols_launch(v, &sg);
    l.grid.y = nb;
    if (v.planes == 3) {   // 3 G threads: at most 384 up to M2 = 2048, 768 beyond (fewer registers)
        static std::atomic<bool> a16{false}, a12{false}, b16{false}, b12{false};
        const bool small = l.block.x <= 384;
        if (v.f2.ept == 16) {
            if (small) DIE_PROF(PK_COLS, st, launch_kernel(k2_cols3<T, 16, 0, 384>, a16, l, st, v, W, skip));
            else DIE_PROF(PK_COLS, st, launch_kernel(k2_cols3<T, 16, 0, 768>, b16, l, st, v, W, skip));
        } else {
            if (small) DIE_PROF(PK_COLS, st, launch_kernel(k2_cols3<T, 12, 0, 384>, a12, l, st, v, W, skip));
            else DIE_PROF(PK_COLS, st, launch_kernel(k2_cols3<T, 12, 0, 768>, b12, l, st, v, W, skip));
        }
        return;
    }
    if (fast_cols(v)) {
        if constexpr (sizeof(C_t<T>) == 8) {     // complex64: both components per thread
            const Launch l2{l.grid, dim3(v.M2 / 16), l.smem};
#define K2F_CASE(LSV) { static std::atomic<bool> a_{false}; launch_kernel(k2_fast2<T, LSV>, a_, l2, st, v, W, sg, skip); }
            DIE_PROF(PK_COLS, st, DIE_FAST_SWITCH(v.M2, K2F_CASE));
#undef K2F_CASE
        } else {
#define K2F_CASE(LSV) { static std::atomic<bool> a_{false}; launch_kernel(k2_fast<T, LSV>, a_, l, st, v, W, sg, skip); }
            DIE_PROF(PK_COLS, st, DIE_FAST_SWITCH(v.M2, K2F_CASE));
#undef K2F_CASE
        }
        return;
    }
#define K2_CASE(LSV) { static std::atomic<bool> a_{false}; launch_kernel(k2_cols<T, 16, LSV>, a_, l, st, v, W, sg, skip); }
#define K2_DEF { static std::atomic<bool> a16{false}, a12{false};                                            \
                 if (v.f2.ept == 16) launch_kernel(k2_cols<T, 16, 0>, a16, l, st, v, W, sg, skip); \
                 else launch_kernel(k2_cols<T, 12, 0>, a12, l, st, v, W, sg, skip); }
    DIE_PROF(PK_COLS, st, DIE_POW2_SWITCH(v.M2, K2_CASE, K2_DEF));
#undef K2_CASE
#undef K2_DEF
}

template <typename T, typename U, typename IO>
inline void launch_k3(const OpDev<T>& v, const C_t<T>* W, const U* u, IO* y, const int* skip, cudaStream_t st,
                      int nb = 1) {
    if (fast_rows(v)) {
        with_tile_rows(v, [&](auto tr) { rows_inv_fast<T, U, IO, decltype(tr)::value>(v, W, u, y, skip, st, nb); });
        return;
    }
    const Launch l = with_z(rows_launch(v), nb);
#define K3_CASE(LSV) { static std::atomic<bool> a_{false}; launch_kernel(k3_rows_inv<T, U, IO, 16, LSV>, a_, l, st, v, W, u, y, skip); }
#define K3_DEF { static std::atomic<bool> a16{false}, a12{false};                                                    \
                 if (v.f1.ept == 16) launch_kernel(k3_rows_inv<T, U, IO, 16, 0>, a16, l, st, v, W, u, y, skip); \
                 else launch_kernel(k3_rows_inv<T, U, IO, 12, 0>, a12, l, st, v, W, u, y, skip); }
    DIE_PROF(PK_ROWS_INV, st, DIE_POW2_SWITCH(v.M1, K3_CASE, K3_DEF));
#undef K3_CASE
#undef K3_DEF
}

template <typename T, typename IO>
inline void launch_k3k1(const OpDev<T>& v, C_t<T>* W, const IO* u, const C_t<T>* chir, C_t<T>* vb, const int* skip,
                        cudaStream_t st, int nb = 1) {
    if (fast_rows(v)) {
        with_tile_rows(v, [&](auto tr) {
            rows_inv_fwd_fast<T, IO, decltype(tr)::value>(v, W, u, chir, vb, skip, st, nb);
        });
        return;
    }
    const Launch l = with_z(rows_launch(v), nb);
#define KK_CASE(LSV) { static std::atomic<bool> a_{false}; launch_kernel(k3k1_rows<T, IO, 16, LSV>, a_, l, st, v, W, u, chir, vb, skip); }
#define KK_DEF { static std::atomic<bool> a16{false}, a12{false};                                                        \
                 if (v.f1.ept == 16) launch_kernel(k3k1_rows<T, IO, 16, 0>, a16, l, st, v, W, u, chir, vb, skip); \
                 else launch_kernel(k3k1_rows<T, IO, 12, 0>, a12, l, st, v, W, u, chir, vb, skip); }
    DIE_PROF(PK_ROWS_INV_FWD, st, DIE_POW2_SWITCH(v.M1, KK_CASE, KK_DEF));
#undef KK_CASE
#undef KK_DEF
}

template <typename T> struct Sel;
template <> struct Sel<double> {
    static const double2* chi(const dieop_s* o, Contrast c) { return c == Contrast::Chi ? o->chi_d : o->chir_d; }
    static OpDev<double> view(const dieop_s* o) { return view_d(o); }
};
template <> struct Sel<float> {
    static const float2* chi(const dieop_s* o, Contrast c) { return c == Contrast::Chi ? o->chi_f : o->chir_f; }
    static OpDev<float> view(const dieop_s* o) { return view_f(o); }
};

template <typename T, typename IO>
die_status apply_op_skip(dieop_s* op, Contrast which, const IO* x, IO* y, const int* skip, cudaStream_t st,
                         const Workspace* ws) {
    if (!ws) ws = &op->ws;
    using C = C_t<T>;
    const OpDev<T> v = Sel<T>::view(op);
    C* W = reinterpret_cast<C*>(ws->W);
    launch_k1<T, IO>(v, x, Sel<T>::chi(op, which), W, skip, st);
    launch_k2<T>(v, W, skip, st);
    launch_k3<T, IO, IO>(v, W, x, y, skip, st);
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

template <typename T, typename IO>
die_status apply_reg_skip(dieop_s* op, const IO* x, IO* y, const int* skip, cudaStream_t st, const Workspace* ws) {
    if (!ws) ws = &op->ws;
    using C = C_t<T>;
    const OpDev<T> v = Sel<T>::view(op);
    C* W = reinterpret_cast<C*>(ws->W);
    C* vb = reinterpret_cast<C*>(ws->v);
    launch_k1<T, IO>(v, x, Sel<T>::chi(op, Contrast::Chi), W, skip, st);
    launch_k2<T>(v, W, skip, st);
    launch_k3k1<T, IO>(v, W, x, Sel<T>::chi(op, Contrast::ChiReg), vb, skip, st);
    launch_k2<T>(v, W, skip, st);
    launch_k3<T, C, IO>(v, W, vb, y, skip, st);
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

// Input and output of different element types (complex64 in, complex128 out: the
// products of the FP32-inner solves whose right preconditioner runs in complex64).
template <typename T, typename IX, typename IY>
die_status apply_op_skip_xy(dieop_s* op, Contrast which, const IX* x, IY* y, const int* skip, cudaStream_t st,
                            const Workspace* ws) {
    if (!ws) ws = &op->ws;
    using C = C_t<T>;
    const OpDev<T> v = Sel<T>::view(op);
    C* W = reinterpret_cast<C*>(ws->W);
    launch_k1<T, IX>(v, x, Sel<T>::chi(op, which), W, skip, st);
    launch_k2<T>(v, W, skip, st);
    launch_k3<T, IX, IY>(v, W, x, y, skip, st);
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

template <typename T, typename IX, typename IY>
die_status apply_reg_skip_xy(dieop_s* op, const IX* x, IY* y, const int* skip, cudaStream_t st,
                             const Workspace* ws) {
    if (!ws) ws = &op->ws;
    using C = C_t<T>;
    const OpDev<T> v = Sel<T>::view(op);
    C* W = reinterpret_cast<C*>(ws->W);
    C* vb = reinterpret_cast<C*>(ws->v);
    launch_k1<T, IX>(v, x, Sel<T>::chi(op, Contrast::Chi), W, skip, st);
    launch_k2<T>(v, W, skip, st);
    launch_k3k1<T, IX>(v, W, x, Sel<T>::chi(op, Contrast::ChiReg), vb, skip, st);
    launch_k2<T>(v, W, skip, st);
    launch_k3<T, C, IY>(v, W, vb, y, skip, st);
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

template <typename T, typename IO>
die_status apply_op(dieop_s* op, Contrast c, const IO* x, IO* y, cudaStream_t st, const Workspace* ws) {
    return apply_op_skip<T, IO>(op, c, x, y, nullptr, st, ws);
}
template <typename T, typename IO>
die_status apply_reg(dieop_s* op, const IO* x, IO* y, cudaStream_t st, const Workspace* ws) {
    return apply_reg_skip<T, IO>(op, x, y, nullptr, st, ws);
}

// nb products y_k = Atilde x_k (Atilde = A_R A when reg, else A) over consecutive field
// vectors, one launch per pass for all of them, with the caller's workspace (nb sets of
// row spectra and, when reg, nb middle vectors).
template <typename T, typename IO>
die_status apply_batch(dieop_s* op, bool reg, const IO* x, IO* y, int nb, void* Wws, void* vws, cudaStream_t st) {
    using C = C_t<T>;
    const OpDev<T> v = Sel<T>::view(op);
    C* W = reinterpret_cast<C*>(Wws);
    C* vb = reinterpret_cast<C*>(vws);
    launch_k1<T, IO>(v, x, Sel<T>::chi(op, Contrast::Chi), W, nullptr, st, nb);
    launch_k2<T>(v, W, nullptr, st, nb);
    if (reg) {
        launch_k3k1<T, IO>(v, W, x, Sel<T>::chi(op, Contrast::ChiReg), vb, nullptr, st, nb);
        launch_k2<T>(v, W, nullptr, st, nb);
        launch_k3<T, C, IO>(v, W, vb, y, nullptr, st, nb);
    } else {
        launch_k3<T, IO, IO>(v, W, x, y, nullptr, st, nb);
    }
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

}  // namespace die
