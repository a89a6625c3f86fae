// Krylov-space kernels (see krylov.cuh).
//
// Projections: one thread per row (grid-stride), holding the row of w in registers and
// the running sums of a group of basis vectors; the loads of a group are issued
// together, so many are in flight.  At the end of a group every warp sums its lanes by
// recursive halving (each level exchanges half as many values as the one before), the
// eight warp sums of each value are added in a fixed order, and the block writes one
// partial per vector.  The partials are summed in two levels (groups of kRedGroup
// blocks, then the groups) by the last block to arrive at each level, in block and
// group order, so results do not depend on scheduling.  Updates: one thread per row,
// sum over the basis with fused multiply-adds (4 per complex term); the optional norm
// uses the same two-level reduction.  Every complex multiply-add is written as four
// FMAs: on GB300 the FP64 pipe (about 2 FMA per clock per SM) bounds the FP64 kernels.
#include "krylov.cuh"
#include "prof.cuh"

namespace die {

template <typename V> struct acc_of;
template <> struct acc_of<double2> { using type = double; };
template <> struct acc_of<float2> { using type = float; };

// Fused multiply-add in the operands' own precision (a bare fma() on floats would be
// promoted to the FP64 pipe, which is narrow on GB300).
__device__ __forceinline__ float fmac(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return fma(a, b, c); }

// Warp sums of K = 2^P values per lane by recursive halving: at offset o = 16, 8, ...
// a lane keeps the half of its current values selected by (lane & o) and adds the
// partner's copy of that half.  Afterwards lane l holds in v[0 .. C) (C = max(K/32, 1))
// the 32-lane sums of the values with index (l >> (5 - H)) * C + c, H = min(P, 5).
template <typename A, int K>
__device__ __forceinline__ void warp_halving_sum(A (&v)[K]) {
    static_assert(K >= 1 && K <= 64 && (K & (K - 1)) == 0, "K must be a power of two <= 64");
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int lvl = 0; lvl < 5; lvl++) {
        const int o = 16 >> lvl;
        const int c = K >> lvl;
        if (c >= 2) {
            const int h = c >> 1;
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < h; i++) {
                const A send = up ? v[i] : v[i + h];
                const A keep = up ? v[i + h] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
}

template <int K> __host__ __device__ constexpr int halving_levels() { return K >= 32 ? 5 : (K >= 16 ? 4 : (K >= 8 ? 3 : (K >= 4 ? 2 : (K >= 2 ? 1 : 0)))); }

// Block partials of one group of CNT vectors: acc[2 v + c] is component c (0: re, 1: im)
// of the running sum of vector g0 + v (entries from 2 CNT on are zero padding up to the
// power of two K).  Writes partial[(g0 + v) * gridDim.x + blockIdx.x] for v < CNT.
// red: K values per warp of shared memory.
template <typename A, int K, int CNT>
__device__ __forceinline__ void block_partials(A (&acc)[K], A* red, int g0, const RedScratch& rs) {
    constexpr int H = halving_levels<K>();
    constexpr int C = K >= 32 ? K / 32 : 1;
    warp_halving_sum<A, K>(acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if ((lane & ((1 << (5 - H)) - 1)) == 0) {
#pragma unroll
        for (int c = 0; c < C; c++) red[warp * K + (lane >> (5 - H)) * C + c] = acc[c];
    }
    __syncthreads();
    double* pp = reinterpret_cast<double*>(rs.partial);
    for (int e = threadIdx.x; e < 2 * CNT; e += blockDim.x) {
        A s = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += red[q * K + e];
        pp[2 * ((long)(g0 + (e >> 1)) * gridDim.x + blockIdx.x) + (e & 1)] = (double)s;
    }
    __syncthreads();
}

// Final sums of the per-block partials partial[i * gridDim.x + b], i < nv (see
// RedScratch).  Every thread of every block calls it after its block's partials are
// written; it returns true in the one block that has written out[0 .. nv), whose
// threads may then read out.
__device__ bool reduce_partials(const RedScratch& rs, int nv, double2* out) {
    __shared__ int s_last;
    const int G = gridDim.x, ng = (G + kRedGroup - 1) / kRedGroup, g = blockIdx.x / kRedGroup;
    const int gsz = min(kRedGroup, G - g * kRedGroup);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool last = atomicAdd(&rs.counter[1 + g], 1u) == (unsigned)(gsz - 1);
        if (last) rs.counter[1 + g] = 0;
        s_last = last;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const double* pp = reinterpret_cast<const double*>(rs.partial);
    double* p2 = reinterpret_cast<double*>(rs.partial2);
    for (int e = threadIdx.x; e < 2 * nv; e += blockDim.x) {   // e = 2 i + component
        const double* src = pp + 2 * ((long)(e >> 1) * G + (long)g * kRedGroup) + (e & 1);
        double s = 0;
        for (int b = 0; b < gsz; b++) s += __ldcg(src + 2 * b);
        p2[2 * ((long)(e >> 1) * ng + g) + (e & 1)] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool last = atomicAdd(&rs.counter[0], 1u) == (unsigned)(ng - 1);
        if (last) rs.counter[0] = 0;
        s_last = last;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double* o = reinterpret_cast<double*>(out);
    for (int e = threadIdx.x; e < 2 * nv; e += blockDim.x) {
        const double* src = p2 + 2 * (long)(e >> 1) * ng + (e & 1);
        double s = 0;
        for (int q = 0; q < ng; q++) s += __ldcg(src + 2 * q);
        o[e] = s;
    }
    __syncthreads();
    return true;
}

// A block that skips its work still writes (zero) partials and takes part in the final
// sums when the skip flag is "live": a flag that another stream may set while the
// kernel runs, so that blocks of one launch may disagree on it.
__device__ __forceinline__ void zero_partials(int g0, int K, int nvt, const RedScratch& rs) {
    double* pp = reinterpret_cast<double*>(rs.partial);
    for (int e = threadIdx.x; e < K; e += blockDim.x)
        if (g0 + (e >> 1) < nvt) pp[2 * ((long)(g0 + (e >> 1)) * gridDim.x + blockIdx.x) + (e & 1)] = 0.0;
}

// conj(a) b accumulated into acc[0] (re), acc[1] (im)
template <typename VT, typename A>
__device__ __forceinline__ void conj_mac(const VT& a, const VT& b, A& re, A& im) {
    re = fmac(a.x, b.x, re); re = fmac(a.y, b.y, re);
    im = fmac(a.x, b.y, im); im = fmac(-a.y, b.x, im);
}

template <int X> __host__ __device__ constexpr int pow2ceil() { return X <= 1 ? 1 : 2 * pow2ceil<(X + 1) / 2>(); }

// One group of CNT projections over this thread's rows (grid-stride), summed into the
// block's partials.  Projection g0 + v is onto V_{g0+v}, or onto the vector itself for
// index nv (the norm).  The basis loads of a row are issued first, then the row of the
// vector: b = xin[idx], or (SCALE) w[idx] *= sc written back and b = its complex64
// copy, also stored to xout.  CNT is a compile-time count: no predicated-off FMAs,
// which would still occupy the FP64 pipe.
template <typename VT, int CNT, bool SCALE>
__device__ __forceinline__ void proj_group(const VT* __restrict__ V, long ldv, int g0, int nv, const VT* xin,
                                           VT* xout, double2* w, double sc, long n,
                                           typename acc_of<VT>::type* red, const RedScratch& rs) {
    using A = typename acc_of<VT>::type;
    constexpr int K = pow2ceil<2 * CNT>();
    // FP64: the a.y b.x terms of the imaginary parts go to their own sums, subtracted at
    // the end, so that every step is a plain FMA (a negated operand costs an extra
    // instruction on the FP64 pipe).
    constexpr bool kSplit = sizeof(A) == 8;
    A acc[K], accn[kSplit ? CNT : 1];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = 0;
#pragma unroll
    for (int v = 0; v < (kSplit ? CNT : 1); v++) accn[v] = 0;
    const VT* src[CNT];
#pragma unroll
    for (int v = 0; v < CNT; v++) src[v] = g0 + v < nv ? V + (long)(g0 + v) * ldv : xin;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += stride) {
        VT a[CNT];
#pragma unroll
        for (int v = 0; v < CNT; v++) a[v] = src[v][idx];
        VT b;
        if constexpr (SCALE) {
            double2 u = w[idx];
            u.x *= sc;
            u.y *= sc;
            w[idx] = u;
            b.x = (A)u.x;
            b.y = (A)u.y;
            xout[idx] = b;
        } else {
            b = xin[idx];
        }
#pragma unroll
        for (int v = 0; v < CNT; v++) {
            if constexpr (kSplit) {
                acc[2 * v] = fmac(a[v].x, b.x, acc[2 * v]);
                acc[2 * v] = fmac(a[v].y, b.y, acc[2 * v]);
                acc[2 * v + 1] = fmac(a[v].x, b.y, acc[2 * v + 1]);
                accn[v] = fmac(a[v].y, b.x, accn[v]);
            } else {
                conj_mac(a[v], b, acc[2 * v], acc[2 * v + 1]);
            }
        }
    }
    if constexpr (kSplit) {
#pragma unroll
        for (int v = 0; v < CNT; v++) acc[2 * v + 1] -= accn[v];
    }
    block_partials<A, K, CNT>(acc, red, g0, rs);
}

// Three-multiplication (Gauss) form of the FP64 projections.  With m = a.x - a.y stored
// beside each basis vector (VM, same stride as V):
//   conj(a) b = (P1 - P2) + i (P2 - P3),  P1 = a.x (b.x + b.y),  P2 = m b.y,  P3 = a.y (b.x - b.y),
// three FMAs per term instead of four; the two sums of b are formed once per row.  The
// vector itself (index nv, the norm) takes m = b.x - b.y.
template <int CNT>
__device__ __forceinline__ void proj_group3(const double2* __restrict__ V, const double* __restrict__ VM, long ldv,
                                            int g0, int nv, const double2* __restrict__ w, long n, double* red,
                                            const RedScratch& rs) {
    constexpr int K = pow2ceil<2 * CNT>();
    double p1[CNT], p2[CNT], p3[CNT];
#pragma unroll
    for (int v = 0; v < CNT; v++) { p1[v] = 0; p2[v] = 0; p3[v] = 0; }
    const long stride = (long)gridDim.x * blockDim.x;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += stride) {
        const double2 b = w[idx];
        double2 a[CNT];
        double m[CNT];
#pragma unroll
        for (int v = 0; v < CNT; v++) {
            const int i = g0 + v;
            a[v] = i < nv ? V[(long)i * ldv + idx] : b;
            m[v] = i < nv ? VM[(long)i * ldv + idx] : b.x - b.y;
        }
        const double sb = b.x + b.y, db = b.x - b.y;
#pragma unroll
        for (int v = 0; v < CNT; v++) {
            p1[v] = fma(a[v].x, sb, p1[v]);
            p2[v] = fma(m[v], b.y, p2[v]);
            p3[v] = fma(a[v].y, db, p3[v]);
        }
    }
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = 0;
#pragma unroll
    for (int v = 0; v < CNT; v++) {
        acc[2 * v] = p1[v] - p2[v];
        acc[2 * v + 1] = p2[v] - p3[v];
    }
    block_partials<double, K, CNT>(acc, red, g0, rs);
}

template <int C>
__device__ __forceinline__ void proj_group3_n(int cnt, const double2* V, const double* VM, long ldv, int g0, int nv,
                                              const double2* w, long n, double* red, const RedScratch& rs) {
    if (cnt == C) proj_group3<C>(V, VM, ldv, g0, nv, w, n, red, rs);
    else if constexpr (C > 1) proj_group3_n<C - 1>(cnt, V, VM, ldv, g0, nv, w, n, red, rs);
}

// FP64 projections in the three-multiplication form, kGroup3 vectors per pass.
constexpr int kGroup3 = 8;
__global__ void __launch_bounds__(kRedThreads, 2) proj3_kernel(const double2* __restrict__ V,
                                                               const double* __restrict__ VM, long ldv, int nv,
                                                               const double2* __restrict__ w, long n, int with_norm,
                                                               double2* out, RedScratch rs, const int* skip,
                                                               int live) {
    constexpr int K = pow2ceil<2 * kGroup3>();
    __shared__ double red[(kRedThreads / 32) * K];
    pdl_wait();
    const bool off = block_flag(skip);
    if (off && !live) return;
    const int nvt = nv + (with_norm ? 1 : 0);
    for (int g0 = 0; g0 < nvt; g0 += kGroup3) {
        if (off) { zero_partials(g0, 2 * kGroup3, nvt, rs); continue; }
        const int cnt = nvt - g0 < kGroup3 ? nvt - g0 : kGroup3;
        proj_group3_n<kGroup3>(cnt, V, VM, ldv, g0, nv, w, n, red, rs);
    }
    reduce_partials(rs, nvt, out);
}

// Runtime count -> compile-time CNT in [1, C].
template <typename VT, int C, bool SCALE>
__device__ __forceinline__ void proj_group_n(int cnt, const VT* V, long ldv, int g0, int nv, const VT* xin, VT* xout,
                                             double2* w, double sc, long n, typename acc_of<VT>::type* red,
                                             const RedScratch& rs) {
    if (cnt == C) proj_group<VT, C, SCALE>(V, ldv, g0, nv, xin, xout, w, sc, n, red, rs);
    else if constexpr (C > 1) proj_group_n<VT, C - 1, SCALE>(cnt, V, ldv, g0, nv, xin, xout, w, sc, n, red, rs);
}

// out[i] = sum_e conj(V_i[e]) w[e] for i < nv; with_norm: out[nv] = ||w||^2 (as the
// projection of w on itself).  Groups of GV vectors; w is re-read once per group.
template <typename VT, int GV>
__global__ void __launch_bounds__(kRedThreads) proj_kernel(const VT* __restrict__ V, long ldv, int nv,
                                                           const VT* __restrict__ w, long n, int with_norm,
                                                           double2* out, RedScratch rs, const int* skip, int live) {
    using A = typename acc_of<VT>::type;
    constexpr int K = 2 * GV;
    __shared__ A red[(kRedThreads / 32) * K];
    pdl_wait();
    const bool off = block_flag(skip);
    if (off && !live) return;
    const int nvt = nv + (with_norm ? 1 : 0);
    for (int g0 = 0; g0 < nvt; g0 += GV) {
        if (off) { zero_partials(g0, K, nvt, rs); continue; }
        const int cnt = nvt - g0 < GV ? nvt - g0 : GV;
        proj_group_n<VT, GV, false>(cnt, V, ldv, g0, nv, w, nullptr, nullptr, 1.0, n, red, rs);
    }
    reduce_partials(rs, nvt, out);
}

// Deflation projections of the FP32-inner solves (see k_dots32): complex64 basis and
// vector, FP32 products and in-block sums; the block that finishes the sums also forms
// cf = M s in FP32.
__global__ void __launch_bounds__(kRedThreads, 2) proj32_kernel(const float2* __restrict__ V, long ldv, int nv,
                                                                float2* x, double2* w, const double* inv, long n,
                                                                double2* out, const float2* __restrict__ M32,
                                                                float2* cf, RedScratch rs, const int* skip, int live) {
    constexpr int GV = 16, K = 2 * GV;     // 16 vectors per pass: 32 running sums, 16 loads in flight
    __shared__ float red[(kRedThreads / 32) * K];
    pdl_wait();
    const bool off = block_flag(skip);
    if (off && !live) return;
    const double sc = inv ? *inv : 1.0;
    for (int g0 = 0; g0 < nv; g0 += GV) {
        if (off) { zero_partials(g0, K, nv, rs); continue; }
        const int cnt = nv - g0 < GV ? nv - g0 : GV;
        if (inv && g0 == 0) proj_group_n<float2, GV, true>(cnt, V, ldv, g0, nv, x, x, w, sc, n, red, rs);
        else proj_group_n<float2, GV, false>(cnt, V, ldv, g0, nv, x, nullptr, nullptr, 1.0, n, red, rs);
    }
    if (reduce_partials(rs, nv, out) && M32) {
        for (int i = threadIdx.x; i < nv; i += blockDim.x) {
            float cx = 0, cy = 0;
            for (int q = 0; q < nv; q++) {
                const float2 m = M32[(long)q * nv + i];
                const double2 sq = __ldcg(&out[q]);
                const float sx = (float)sq.x, sy = (float)sq.y;
                cx = fmaf(m.x, sx, cx); cx = fmaf(-m.y, sy, cx);
                cy = fmaf(m.x, sy, cy); cy = fmaf(m.y, sx, cy);
            }
            cf[i] = make_float2(cx, cy);
        }
    }
}

// z = x + V c (c precomputed, complex64), all complex64: the deflation update of the
// FP32-inner solves.
__global__ void __launch_bounds__(kRedThreads) defl_update32_kernel(const float2* __restrict__ V, long ldv, int r,
                                                                    const float2* __restrict__ cf,
                                                                    const float2* x, float2* z, long n,
                                                                    const int* skip, double2* w, const double* inv,
                                                                    double* wm) {
    pdl_wait();
    if (block_flag(skip)) return;
    __shared__ float2 cs[kMaxBasis];
    for (int i = threadIdx.x; i < r; i += blockDim.x) cs[i] = __ldcg(&cf[i]);
    __syncthreads();
    const double sc = inv ? *inv : 1.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += stride) {
        float2 acc;
        if (inv) {                          // normalise the FP64 vector, take its complex64 copy
            double2 u = w[idx];
            u.x *= sc;
            u.y *= sc;
            w[idx] = u;
            if (wm) wm[idx] = u.x - u.y;
            acc = make_float2((float)u.x, (float)u.y);
        } else {
            acc = x[idx];
        }
        float ex = 0, ey = 0;
        int i = 0;
#pragma unroll 4
        for (; i + 1 < r; i += 2) {
            const float2 a = V[(long)i * ldv + idx], c = cs[i];
            const float2 b = V[(long)(i + 1) * ldv + idx], d = cs[i + 1];
            acc.x = fmaf(a.x, c.x, acc.x); acc.x = fmaf(-a.y, c.y, acc.x);
            acc.y = fmaf(a.x, c.y, acc.y); acc.y = fmaf(a.y, c.x, acc.y);
            ex = fmaf(b.x, d.x, ex); ex = fmaf(-b.y, d.y, ex);
            ey = fmaf(b.x, d.y, ey); ey = fmaf(b.y, d.x, ey);
        }
        if (i < r) {
            const float2 a = V[(long)i * ldv + idx], c = cs[i];
            acc.x = fmaf(a.x, c.x, acc.x); acc.x = fmaf(-a.y, c.y, acc.x);
            acc.y = fmaf(a.x, c.y, acc.y); acc.y = fmaf(a.y, c.x, acc.y);
        }
        z[idx] = make_float2(acc.x + ex, acc.y + ey);
    }
}

// 1 / ||w|| from ||w||^2 (1 when the norm is zero or not finite: the vector is left as it is)
__device__ __forceinline__ double inv_norm(double s2) {
    const double hn = sqrt(fmax(s2, 0.0));
    return (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 1.0;
}

// out = base + sum_i V_i c_i.  Coefficients: c = sign * coef, or c = M s when M != NULL.
// The sum for a row starts from base and runs through the basis in order in one pair of
// accumulators (the FP64 pipe, not the FMA latency, bounds the loop).
template <typename VT, bool NORM>
__global__ void __launch_bounds__(kRedThreads) basis_axpy_kernel(const VT* __restrict__ V, long ldv, int k,
                                                                 const double2* __restrict__ coef, double sign,
                                                                 const double2* __restrict__ M,
                                                                 const double2* __restrict__ s, const double2* base,
                                                                 double2* out, long n, double2* nrm2, Dgks dec,
                                                                 int has_dec, RedScratch rs, const int* skip,
                                                                 int live, const double* VM) {
    using A = typename acc_of<VT>::type;
    pdl_wait();
    const bool off = block_flag(skip);
    if (off && !(NORM && live)) return;
    __shared__ VT cs[kMaxBasis];
    __shared__ A csn[kMaxBasis];            // -Im(c): every step below is a plain FMA
    __shared__ double c3[3][kMaxBasis];     // VM != NULL: Im c, Re c - Im c, Re c + Im c
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double cx = 0, cy = 0;
        if (M) {
            for (int q = 0; q < k; q++) {
                const double2 m = M[(long)q * k + i], sv = s[q];
                cx = fmac(m.x, sv.x, cx); cx = fmac(-m.y, sv.y, cx);
                cy = fmac(m.x, sv.y, cy); cy = fmac(m.y, sv.x, cy);
            }
        } else {
            cx = sign * coef[i].x;
            cy = sign * coef[i].y;
        }
        VT c;
        c.x = (A)cx;
        c.y = (A)cy;
        cs[i] = c;
        csn[i] = -c.y;
        c3[0][i] = cy;
        c3[1][i] = cx - cy;
        c3[2][i] = cx + cy;
    }
    __syncthreads();
    double nacc = 0;
    const long stride = (long)gridDim.x * blockDim.x;
    const long nn = off ? 0 : n;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < nn; idx += stride) {
        A x0 = 0, y0 = 0;
        if (base) { const double2 bv = base[idx]; x0 = (A)bv.x; y0 = (A)bv.y; }
        if (VM) {   // three-multiplication form: c a = (K1 + K2) + i (K1 + K3)
            double k1 = 0, k2 = 0, k3 = 0;
#pragma unroll 4
            for (int i = 0; i < k; i++) {
                const VT a = V[(long)i * ldv + idx];
                const double m = VM[(long)i * ldv + idx];
                k1 = fma(c3[0][i], m, k1);
                k2 = fma(c3[1][i], (double)a.x, k2);
                k3 = fma(c3[2][i], (double)a.y, k3);
            }
            x0 += (A)(k1 + k2);
            y0 += (A)(k1 + k3);
        } else {
#pragma unroll 4
            for (int i = 0; i < k; i++) {
                const VT a = V[(long)i * ldv + idx], c = cs[i];
                x0 = fmac(a.x, c.x, x0); x0 = fmac(a.y, csn[i], x0);
                y0 = fmac(a.x, c.y, y0); y0 = fmac(a.y, c.x, y0);
            }
        }
        const double2 o = make_double2((double)x0, (double)y0);
        out[idx] = o;
        if (NORM) { nacc = fmac(o.x, o.x, nacc); nacc = fmac(o.y, o.y, nacc); }
    }
    if (NORM) {
        A acc[2] = {(A)nacc, (A)0};
        __shared__ A red[(kRedThreads / 32) * 2];
        block_partials<A, 2, 1>(acc, red, 0, rs);
        if (reduce_partials(rs, 1, nrm2) && threadIdx.x == 0) {
            const double tot = __ldcg(&nrm2->x);
            int r = 0;
            if (has_dec) {
                r = dec.always || tot < dec.eta2 * dec.before2->x;
                *dec.reorth = r;
                *dec.skip2 = (dec.done && *dec.done) || !r;
                if (r && dec.abort_flags) {          // single-pass cycle: stop it here
                    *dec.abort_flags |= 8;
                    *dec.abort_done = 1;
                }
            }
            if (dec.inv && !r) *dec.inv = inv_norm(tot);
        }
    }
}

// Gram-Schmidt update w = base - V c with ||w||^2 and the DGKS decision (as
// basis_axpy_kernel<double2, true> with sign -1), and the deflation projections
// V32^* w folded in: NGD groups of 8 complex64 basis vectors, FP32 products and
// in-block sums (the FP32 pipe and the spare memory bandwidth of this FP64-bound
// pass).  Reduction vector 0 is ||w||^2, vectors 1 .. r the projections.  The last
// block writes ||w||^2 to nrm2 and, when no second pass follows, 1 / ||w|| to dec.inv
// and cf = M32 (V32^* w / ||w||) to dp.cf.
template <int NGD>
__global__ void __launch_bounds__(kRedThreads) cgs_update_defl_kernel(const double2* __restrict__ V, long ldv, int k,
                                                                      const double2* __restrict__ coef,
                                                                      const double2* base, double2* out, long n,
                                                                      double2* nrm2, Dgks dec, int has_dec,
                                                                      DeflProj dp, RedScratch rs, const int* skip,
                                                                      int live, const double* VM) {
    pdl_wait();
    const bool off = block_flag(skip);
    if (off && !live) return;
    __shared__ double2 cs[kMaxBasis];
    __shared__ double csn[kMaxBasis];
    __shared__ double c3[3][kMaxBasis];     // VM != NULL: Im c, Re c - Im c, Re c + Im c
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double2 c = make_double2(-coef[i].x, -coef[i].y);
        cs[i] = c;
        csn[i] = -c.y;
        c3[0][i] = c.y;
        c3[1][i] = c.x - c.y;
        c3[2][i] = c.x + c.y;
    }
    __syncthreads();
    double nacc = 0;
    float dacc[NGD][16];
#pragma unroll
    for (int g = 0; g < NGD; g++)
#pragma unroll
        for (int q = 0; q < 16; q++) dacc[g][q] = 0.f;
    const long stride = (long)gridDim.x * blockDim.x;
    const long nn = off ? 0 : n;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < nn; idx += stride) {
        double x0 = 0, y0 = 0;
        if (base) { const double2 bv = base[idx]; x0 = bv.x; y0 = bv.y; }
        if (VM) {   // three-multiplication form: c a = (K1 + K2) + i (K1 + K3)
            double k1 = 0, k2 = 0, k3 = 0;
#pragma unroll 4
            for (int i = 0; i < k; i++) {
                const double2 a = V[(long)i * ldv + idx];
                const double m = VM[(long)i * ldv + idx];
                k1 = fma(c3[0][i], m, k1);
                k2 = fma(c3[1][i], a.x, k2);
                k3 = fma(c3[2][i], a.y, k3);
            }
            x0 += k1 + k2;
            y0 += k1 + k3;
        } else {
#pragma unroll 4
            for (int i = 0; i < k; i++) {
                const double2 a = V[(long)i * ldv + idx], c = cs[i];
                x0 = fma(a.x, c.x, x0); x0 = fma(a.y, csn[i], x0);
                y0 = fma(a.x, c.y, y0); y0 = fma(a.y, c.x, y0);
            }
        }
        const double2 o = make_double2(x0, y0);
        out[idx] = o;
        nacc = fma(o.x, o.x, nacc);
        nacc = fma(o.y, o.y, nacc);
        const float2 of = make_float2((float)o.x, (float)o.y);
#pragma unroll
        for (int g = 0; g < NGD; g++) {
            float2 a[8];
#pragma unroll
            for (int v = 0; v < 8; v++) {
                const int i = 8 * g + v;
                a[v] = i < dp.r ? dp.V32[(long)i * dp.ld + idx] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int v = 0; v < 8; v++) conj_mac(a[v], of, dacc[g][2 * v], dacc[g][2 * v + 1]);
        }
    }
    {
        double acc[2] = {nacc, 0.0};
        __shared__ double red[(kRedThreads / 32) * 2];
        block_partials<double, 2, 1>(acc, red, 0, rs);
    }
    __shared__ float redf[(kRedThreads / 32) * 16];
#pragma unroll
    for (int g = 0; g < NGD; g++) block_partials<float, 16, 8>(dacc[g], redf, 1 + 8 * g, rs);
    if (reduce_partials(rs, 1 + dp.r, dp.s)) {
        __shared__ float s_iv;
        __shared__ int s_fin;
        if (threadIdx.x == 0) {
            const double tot = __ldcg(&dp.s[0].x);
            *nrm2 = make_double2(tot, 0.0);
            int r = 0;
            if (has_dec) {
                r = dec.always || tot < dec.eta2 * dec.before2->x;
                *dec.reorth = r;
                *dec.skip2 = (dec.done && *dec.done) || !r;
                if (r && dec.abort_flags) {          // single-pass cycle: stop it here
                    *dec.abort_flags |= 8;
                    *dec.abort_done = 1;
                }
            }
            const double iv = inv_norm(tot);
            if (dec.inv && !r) *dec.inv = iv;
            s_iv = (float)iv;
            s_fin = !r;
        }
        __syncthreads();
        if (s_fin) {
            for (int i = threadIdx.x; i < dp.r; i += blockDim.x) {
                float cx = 0, cy = 0;
                for (int q = 0; q < dp.r; q++) {
                    const float2 m = dp.M32[(long)q * dp.r + i];
                    const double2 sq = __ldcg(&dp.s[1 + q]);
                    const float sx = (float)sq.x * s_iv, sy = (float)sq.y * s_iv;
                    cx = fmaf(m.x, sx, cx); cx = fmaf(-m.y, sy, cx);
                    cy = fmaf(m.x, sy, cy); cy = fmaf(m.y, sx, cy);
                }
                dp.cf[i] = make_float2(cx, cy);
            }
        }
    }
}

// One Givens step of the restarted GMRES least-squares problem (Saad & Schultz):
// H(:, j) = h1 (+ h2) with H(j+1, j) = ||w||; apply the stored rotations, build the
// rotation that annihilates H(j+1, j), update g; residual estimate |g_{j+1}| / ||b||.
// The column, the stored rotations and g_j are staged in shared memory by the whole
// block (one global round trip instead of one per rotation), then thread 0 computes.
// Everything it reads belongs to step j (its own slots of h1, h2, nrm and reorth).
// Shared memory (dynamic): the column (j + 2 slots), then the j cosines and j sines.
__global__ void arnoldi_finish_kernel(GmresDev S, int j) {
    extern __shared__ double2 fin_smem[];
    double2* col = fin_smem;
    double2* csv = col + (j + 2);
    double2* snv = csv + j;
    if (*S.done) return;
    const int ld = S.m + 1;
    double2* Hgl = S.H + (long)j * ld;
    const double2* h1 = S.h1 + (long)j * (S.m + 3);
    const double2* h2 = S.h2 + (long)j * (S.m + 3);
    const int re = S.reorth[j];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        col[i] = re ? make_double2(h1[i].x + h2[i].x, h1[i].y + h2[i].y) : h1[i];
        if (i < j) { csv[i] = S.cs[i]; snv[i] = S.sn[i]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
    double2* Hc = col;
    if (re) *S.nreorth += 1;
    const double wnorm2 = re ? S.nrm[2 * j + 1].x : S.nrm[2 * j].x;
    const double before2 = h1[j + 1].x;
    const double hn = sqrt(fmax(wnorm2, 0.0));
    givens_column(Hc, csv, snv, j, hn, S.cs + j, S.sn + j, S.g);
    const double est = hypot(S.g[j + 1].x, S.g[j + 1].y) / *S.bnorm;
    const int step = *S.step0 + j;
    if (step < S.hist_cap) S.hist[step] = est;
    *S.k = j + 1;
    const bool bad = !isfinite(est) || !isfinite(hn);
    const bool breakdown = hn <= 1e-14 * sqrt(fmax(before2, 0.0));
    if (bad) *S.flags |= 1;
    if (breakdown) *S.flags |= 2;
    if (bad || breakdown || est <= S.tol || j + 1 >= S.jmax) *S.done = 1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) Hgl[i] = col[i];
}

// v *= inv, with an optional complex64 copy of the result and its Re - Im (vm)
__device__ __forceinline__ void scale_rows(double2* v, long n, double inv, float2* v32, double* vm) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 a = v[i];
        const double2 b = make_double2(a.x * inv, a.y * inv);
        v[i] = b;
        if (v32) v32[i] = make_float2((float)b.x, (float)b.y);
        if (vm) vm[i] = b.x - b.y;
    }
}

__global__ void scale_inv_sqrt_kernel(double2* v, long n, const double2* nrm2, const int* skip, float2* v32,
                                      double* vm) {
    pdl_wait();
    if (block_flag(skip)) return;
    __shared__ double s_inv;
    if (threadIdx.x == 0) s_inv = inv_norm(nrm2->x);
    __syncthreads();
    scale_rows(v, n, s_inv, v32, vm);
}

__global__ void scale_by_kernel(double2* v, long n, const double* inv, const int* skip, float2* v32, double* vm) {
    pdl_wait();
    if (block_flag(skip)) return;
    scale_rows(v, n, *inv, v32, vm);
}

__global__ void sub_kernel(const double2* b, const double2* y, double2* r, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        r[i] = csub(b[i], y[i]);
}

__global__ void to_c64_kernel(const double2* x, float2* y, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = make_float2((float)x[i].x, (float)x[i].y);
}

// Back substitution R y = g (R: the rotated k x k Hessenberg), column by column: the
// reciprocals of the diagonal are formed in parallel first, then y_i = g_i / R_ii and
// the rest of g is updated by all threads at once, so the serial chain is one complex
// multiply per column instead of a row of them.
// Shared memory (dynamic): rhs and rd, m slots each.
__global__ void gmres_lsq_kernel(GmresDev S) {
    extern __shared__ double2 lsq_smem[];
    double2* rhs = lsq_smem;
    double2* rd = lsq_smem + S.m;
    const int k = *S.k, ld = S.m + 1;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        rhs[i] = S.g[i];
        const double2 d = S.H[(long)i * ld + i];
        const double dd = d.x * d.x + d.y * d.y;
        rd[i] = dd == 0.0 ? make_double2(0.0, 0.0) : make_double2(d.x / dd, -d.y / dd);
        if (dd == 0.0) *S.flags |= 4;
    }
    __syncthreads();
    for (int i = k - 1; i >= 0; i--) {
        const double2 yi = cmul(rhs[i], rd[i]);
        __syncthreads();
        for (int q = threadIdx.x; q < i; q += blockDim.x) rhs[q] = csub(rhs[q], cmul(S.H[(long)i * ld + q], yi));
        if (threadIdx.x == 0) S.y[i] = yi;
        __syncthreads();
    }
}

__global__ void cycle_scalars_kernel(GmresDev S, double bnorm, int step0) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *S.step0 = step0;
    *S.bnorm = bnorm;
}

// Start a cycle: g = (beta, 0, ...), counters cleared; beta = sqrt(re(*beta2)).
__global__ void gmres_init_kernel(GmresDev S, const double2* beta2) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i <= S.m; i++) S.g[i] = make_double2(0, 0);
    S.g[0] = make_double2(sqrt(fmax(beta2->x, 0.0)), 0.0);
    *S.done = 0;
    *S.k = 0;
    *S.flags = 0;
}

// ------------------------------------------------------------------ launchers
int red_blocks() {
    static int cache[64] = {};       // per device; a benign race writes the same value
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return 2 * kRedGroup; }
    if (cache[dev]) return cache[dev];
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = kRedGroup;
    }
    int b = 2 * sms / kRedGroup * kRedGroup;
    b = b < kRedGroup ? kRedGroup : (b > kRedBlocksMax ? kRedBlocksMax : b);
    cache[dev] = b;
    return b;
}

static inline int grid_for(long n) {
    long b = (n + kRedThreads - 1) / kRedThreads;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

constexpr int kGroupFp64 = 8;        // FP64 projections per group (16 running sums per thread)

die_status k_dots(const double2* V, long ldv, int nv, const double2* w, long n, int with_norm, double2* out,
                  const RedScratch& rs, const int* skip, cudaStream_t st, bool live, const double* VM) {
    if (nv + 1 > kMaxBasis || nv < 0) return DIE_EINVAL;
    if (VM)
        DIE_PROF(PK_DOTS, st, launch_pdl(proj3_kernel, dim3(red_blocks()), dim3(kRedThreads), 0, st, V, VM, ldv, nv, w, n, with_norm, out, rs, skip, live ? 1 : 0));
    else
        DIE_PROF(PK_DOTS, st, launch_pdl(proj_kernel<double2, kGroupFp64>, dim3(red_blocks()), dim3(kRedThreads), 0, st, V, ldv, nv, w, n, with_norm, out, rs, skip, live ? 1 : 0));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_dots32(const float2* V, long ldv, int nv, float2* x, double2* w, const double* inv, long n,
                    double2* out, const float2* M32, float2* cf, const RedScratch& rs, const int* skip,
                    cudaStream_t st, bool live) {
    if (nv > kMaxBasis || nv < 1 || (inv && !w)) return DIE_EINVAL;
    DIE_PROF(PK_DOTS32, st, launch_pdl(proj32_kernel, dim3(red_blocks()), dim3(kRedThreads), 0, st, V, ldv, nv, x, w, inv, n, out, M32, cf, rs, skip, live ? 1 : 0));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_basis_axpy(const double2* V, long ldv, int k, const double2* coef, double sign, const double2* base,
                        double2* out, long n, double2* nrm2, const Dgks* dec, const RedScratch& rs, const int* skip,
                        cudaStream_t st, bool live, const double* VM) {
    if (k > kMaxBasis || k < 0) return DIE_EINVAL;
    const Dgks d = dec ? *dec : Dgks{};
    const int has_dec = dec && dec->reorth ? 1 : 0;
    if (nrm2) {
        DIE_PROF(PK_UPDATE_NORM, st, launch_pdl(basis_axpy_kernel<double2, true>, dim3(red_blocks()), dim3(kRedThreads), 0, st,
                     V, ldv, k, coef, sign, (const double2*)nullptr, (const double2*)nullptr, base, out, n, nrm2, d, has_dec, rs, skip, live ? 1 : 0, VM));
    } else {
        DIE_PROF(PK_LINCOMB, st, launch_pdl(basis_axpy_kernel<double2, false>, dim3(grid_for(n)), dim3(kRedThreads), 0, st,
                     V, ldv, k, coef, sign, (const double2*)nullptr, (const double2*)nullptr, base, out, n, (double2*)nullptr, d, 0, rs, skip, 0, VM));
    }
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_defl_update(const double2* V, long ldv, int r, const double2* M, const double2* s, const double2* x,
                         double2* z, long n, const int* skip, cudaStream_t st) {
    if (r > kMaxBasis || r < 1) return DIE_EINVAL;
    DIE_PROF(PK_DEFL_UPDATE, st, launch_pdl(basis_axpy_kernel<double2, false>, dim3(grid_for(n)), dim3(kRedThreads), 0, st,
                 V, ldv, r, (const double2*)nullptr, 1.0, M, s, x, z, n, (double2*)nullptr, Dgks{}, 0, RedScratch{}, skip, 0, (const double*)nullptr));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_defl_update32(const float2* V, long ldv, int r, const float2* cf, const float2* x, float2* z, long n,
                           const int* skip, cudaStream_t st, double2* w, const double* inv, double* wm) {
    if (r > kMaxBasis || r < 1 || (inv && !w)) return DIE_EINVAL;
    DIE_PROF(PK_DEFL_UPDATE, st, launch_pdl(defl_update32_kernel, dim3(grid_for(n)), dim3(kRedThreads), 0, st, V, ldv, r, cf, x, z, n, skip, w, inv, wm));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

// Update pass with the deflation projections folded in (see cgs_update_defl_kernel).
static die_status k_update_defl(const double2* V, long ldv, int k, const double2* coef, double2* w, long n,
                                double2* nrm2, const Dgks& dec, int has_dec, const DeflProj& dp, const RedScratch& rs,
                                const int* skip, cudaStream_t st, bool live, const double* VM) {
    if (k > kMaxBasis || k < 0 || dp.r < 1 || dp.r > kDeflFoldMax) return DIE_EINVAL;
    const int ng = (dp.r + 7) / 8;
#define UPD_CASE(NG) DIE_PROF(PK_UPDATE_NORM, st, launch_pdl(cgs_update_defl_kernel<NG>, dim3(red_blocks()), dim3(kRedThreads), 0, st, \
                              V, ldv, k, coef, (const double2*)w, w, n, nrm2, dec, has_dec, dp, rs, skip, live ? 1 : 0, VM))
    switch (ng) {
        case 1: UPD_CASE(1); break;
        case 2: UPD_CASE(2); break;
        case 3: UPD_CASE(3); break;
        default: UPD_CASE(4); break;
    }
#undef UPD_CASE
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

// Projections h = V^* w over a basis of any length, in chunks of kBasisChunk vectors
// (every chunk projects the same w); with_norm: ||w||^2 lands at h[nv].
static die_status dots_chunked(const double2* V, long ldv, int nv, const double2* w, long n, int with_norm,
                               double2* h, const RedScratch& rs, const int* skip, cudaStream_t st, bool live,
                               const double* VM) {
    for (int a = 0; a < nv; a += kBasisChunk) {
        const int cnt = nv - a < kBasisChunk ? nv - a : kBasisChunk;
        const bool last = a + cnt >= nv;
        DIE_TRY(k_dots(V + (long)a * ldv, ldv, cnt, w, n, last ? with_norm : 0, h + a, rs, skip, st, live,
                       VM ? VM + (long)a * ldv : nullptr));
    }
    return DIE_OK;
}

// w -= V h over a basis of any length: the chunks before the last subtract without a norm,
// the last one runs `last_update` (the norm, the DGKS decision, folded projections).
template <typename F>
static die_status update_chunked(const double2* V, long ldv, int nv, const double2* h, double2* w, long n,
                                 const RedScratch& rs, const int* skip, cudaStream_t st, const double* VM,
                                 F&& last_update) {
    int a = 0;
    for (; nv - a > kBasisChunk; a += kBasisChunk)
        DIE_TRY(k_basis_axpy(V + (long)a * ldv, ldv, kBasisChunk, h + a, -1.0, w, w, n, nullptr, nullptr, rs, skip,
                             st, false, VM ? VM + (long)a * ldv : nullptr));
    return last_update(V + (long)a * ldv, nv - a, h + a, VM ? VM + (long)a * ldv : nullptr);
}

die_status cgs_dgks(const double2* V, long ldv, int nv, double2* w, long n, double2* h1, double2* h2, double2* nrm,
                    int* reorth, int* skip2, const int* done, double eta2, const RedScratch& rs, cudaStream_t st,
                    double* inv, const DeflProj* dp, double* VM, int* abort_flags, int* abort_done) {
    if (nv < 1 || nv > kMaxRestart + 1) return DIE_EINVAL;
    Dgks dec;
    dec.before2 = h1 + nv;
    dec.reorth = reorth;
    dec.skip2 = skip2;
    dec.done = done;
    dec.inv = inv;
    dec.always = eta2 >= 1.0 ? 1 : 0;
    dec.eta2 = eta2;
    dec.abort_flags = abort_flags;
    dec.abort_done = abort_done;
    DIE_TRY(dots_chunked(V, ldv, nv, w, n, 1, h1, rs, done, st, true, VM));
    DIE_TRY(update_chunked(V, ldv, nv, h1, w, n, rs, done, st, VM,
                           [&](const double2* Vl, int cnt, const double2* hl, const double* VMl) {
                               return dp ? k_update_defl(Vl, ldv, cnt, hl, w, n, nrm, dec, 1, *dp, rs, done, st, true,
                                                         VMl)
                                         : k_basis_axpy(Vl, ldv, cnt, hl, -1.0, w, w, n, nrm, &dec, rs, done, st,
                                                        true, VMl);
                           }));
    if (abort_flags) return DIE_OK;   // single-pass cycle: no second-pass launches
    Dgks last;                       // second pass: no decision, only the scale factor
    last.inv = inv;
    g_prof_override = PK_DOTS_REORTH;
    die_status s = dots_chunked(V, ldv, nv, w, n, 0, h2, rs, skip2, st, false, VM);
    g_prof_override = PK_UPDATE_REORTH;
    if (s == DIE_OK)
        s = update_chunked(V, ldv, nv, h2, w, n, rs, skip2, st, VM,
                           [&](const double2* Vl, int cnt, const double2* hl, const double* VMl) {
                               return dp ? k_update_defl(Vl, ldv, cnt, hl, w, n, nrm + 1, last, 0, *dp, rs, skip2, st,
                                                         false, VMl)
                                         : k_basis_axpy(Vl, ldv, cnt, hl, -1.0, w, w, n, nrm + 1, &last, rs, skip2,
                                                        st, false, VMl);
                           });
    g_prof_override = -1;
    return s;
}

die_status k_lincomb(const double2* V, long ldv, int k, const double2* coef, const double2* base, double2* out,
                     long n, const RedScratch& rs, cudaStream_t st, const double* VM) {
    if (k < 0) return DIE_EINVAL;
    int a = 0;
    do {        // k == 0: one launch, out = base
        const int cnt = k - a < kBasisChunk ? k - a : kBasisChunk;
        DIE_TRY(k_basis_axpy(V + (long)a * ldv, ldv, cnt, coef + a, 1.0, a == 0 ? base : out, out, n, nullptr,
                             nullptr, rs, nullptr, st, false, VM ? VM + (long)a * ldv : nullptr));
        a += cnt;
    } while (a < k);
    return DIE_OK;
}

die_status k_scale_inv_sqrt(double2* v, long n, const double2* nrm2, const int* skip, cudaStream_t st, float2* v32,
                            double* vm) {
    DIE_PROF(PK_SCALE, st, launch_pdl(scale_inv_sqrt_kernel, dim3(grid_for(n)), dim3(kRedThreads), 0, st, v, n, nrm2, skip, v32, vm));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_scale_by(double2* v, long n, const double* inv, const int* skip, cudaStream_t st, float2* v32,
                      double* vm) {
    DIE_PROF(PK_SCALE, st, launch_pdl(scale_by_kernel, dim3(grid_for(n)), dim3(kRedThreads), 0, st, v, n, inv, skip, v32, vm));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_sub(const double2* b, const double2* y, double2* r, long n, cudaStream_t st) {
    DIE_PROF(PK_OTHER, st, sub_kernel<<<grid_for(n), kRedThreads, 0, st>>>(b, y, r, n));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_to_c64(const double2* x, float2* y, long n, cudaStream_t st) {
    DIE_PROF(PK_OTHER, st, to_c64_kernel<<<grid_for(n), kRedThreads, 0, st>>>(x, y, n));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
static size_t finish_smem_bytes(int j) { return (size_t)(3 * j + 2) * sizeof(double2); }
static size_t lsq_smem_bytes(int m) { return (size_t)2 * m * sizeof(double2); }

die_status krylov_prepare(int m) {
    if (m < 1 || m > kMaxRestart) return DIE_EINVAL;
    DIE_CUDA_TRY(cudaFuncSetAttribute(arnoldi_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)finish_smem_bytes(kMaxRestart)));
    DIE_CUDA_TRY(cudaFuncSetAttribute(gmres_lsq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)lsq_smem_bytes(kMaxRestart)));
    return DIE_OK;
}

die_status k_arnoldi_finish(GmresDev S, int j, cudaStream_t st) {
    if (j < 0 || j >= kMaxRestart) return DIE_EINVAL;
    DIE_PROF(PK_GIVENS, st, arnoldi_finish_kernel<<<1, 128, finish_smem_bytes(j), st>>>(S, j));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_cycle_scalars(GmresDev S, double bnorm, int step0, cudaStream_t st) {
    DIE_PROF(PK_SMALL, st, cycle_scalars_kernel<<<1, 32, 0, st>>>(S, bnorm, step0));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_gmres_lsq(GmresDev S, cudaStream_t st) {
    if (S.m < 1 || S.m > kMaxRestart) return DIE_EINVAL;
    DIE_PROF(PK_SMALL, st, gmres_lsq_kernel<<<1, 64, lsq_smem_bytes(S.m), st>>>(S));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_gmres_init(GmresDev S, const double2* beta2, cudaStream_t st) {
    DIE_PROF(PK_SMALL, st, gmres_init_kernel<<<1, 32, 0, st>>>(S, beta2));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

}  // namespace die
