// Krylov-space kernels (see krylov.cuh).
//
// Projections: each block owns a contiguous slice of the rows; each warp accumulates
// whole vectors over that slice (lanes stride the rows in batches of loads, so basis
// reads are coalesced and many are in flight; w is re-read from L1; there is no
// barrier or reduction until the end), then one warp reduction per vector gives the
// block's partial (stride = the launch's block count).  The last block to arrive
// (atomic counter) sums the partials of each vector in a fixed order, so results do
// not depend on scheduling.  Updates: one thread per row, sum over the basis with
// fused multiply-adds (4 per complex term); the optional norm uses the same
// deterministic two-level reduction.  Every complex multiply-add is written as four
// FMAs: on GB300 the FP64 pipe (about 2 FMA per clock per SM) bounds these kernels.
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

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// True in exactly one block: the last one to finish writing its partials.
__device__ __forceinline__ bool arrive_last(unsigned* counter) {
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// out[i] = sum over blocks of partial[i][b], i < nv (one warp per vector, fixed order).
__device__ __forceinline__ void final_sums(const double2* partial, int nv, double2* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < nv; i += nw) {
        double sx = 0, sy = 0;
        for (int b = lane; b < (int)gridDim.x; b += 32) {
            const double2 p = __ldcg(&partial[(long)i * gridDim.x + b]);
            sx += p.x;
            sy += p.y;
        }
        sx = warp_sum_d(sx);
        sy = warp_sum_d(sy);
        if (lane == 0) out[i] = make_double2(sx, sy);
    }
}

// Rows loaded per batch by each lane: enough independent loads in flight to cover
// HBM latency with two blocks of eight warps per SM.
template <typename VT> constexpr int dot_batch() { return sizeof(VT) == 8 ? 8 : 4; }

// out[i] = sum_e conj(V_i[e]) w[e]; w has the basis' element type (no conversions).
// Warp q of a block handles vectors q, q+8, q+16, ... one at a time over the block's rows.
template <typename VT>
__global__ void __launch_bounds__(kRedThreads) dots_kernel(const VT* __restrict__ V, long ldv, int nv,
                                                           const VT* __restrict__ w, long n, int with_norm,
                                                           double2* out, RedScratch rs, const int* skip) {
    using A = typename acc_of<VT>::type;
    constexpr int U = dot_batch<VT>();
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long r0 = n * (long)blockIdx.x / gridDim.x, r1 = n * (long)(blockIdx.x + 1) / gridDim.x;
    const int nvt = nv + (with_norm ? 1 : 0);
    for (int i = warp; i < nvt; i += 8) {
        A ax = 0, ay = 0, bx = 0, by = 0;
        long idx = r0 + lane;
        if (i < nv) {
            const VT* p = V + (long)i * ldv;
            for (; idx + 32 * (U - 1) < r1; idx += 32 * U) {
                VT a[U], b[U];
#pragma unroll
                for (int u = 0; u < U; u++) { a[u] = p[idx + 32 * u]; b[u] = w[idx + 32 * u]; }
#pragma unroll
                for (int u = 0; u < U; u += 2) {
                    ax = fmac(a[u].x, b[u].x, ax); ax = fmac(a[u].y, b[u].y, ax);
                    ay = fmac(a[u].x, b[u].y, ay); ay = fmac(-a[u].y, b[u].x, ay);
                    bx = fmac(a[u + 1].x, b[u + 1].x, bx); bx = fmac(a[u + 1].y, b[u + 1].y, bx);
                    by = fmac(a[u + 1].x, b[u + 1].y, by); by = fmac(-a[u + 1].y, b[u + 1].x, by);
                }
            }
            for (; idx < r1; idx += 32) {
                const VT a = p[idx], b = w[idx];
                ax = fmac(a.x, b.x, ax); ax = fmac(a.y, b.y, ax);
                ay = fmac(a.x, b.y, ay); ay = fmac(-a.y, b.x, ay);
            }
        } else {                                            // the norm of w
            for (; idx + 32 * (U - 1) < r1; idx += 32 * U) {
                VT b[U];
#pragma unroll
                for (int u = 0; u < U; u++) b[u] = w[idx + 32 * u];
#pragma unroll
                for (int u = 0; u < U; u++) { ax = fmac(b[u].x, b[u].x, ax); bx = fmac(b[u].y, b[u].y, bx); }
            }
            for (; idx < r1; idx += 32) {
                const VT b = w[idx];
                ax = fmac(b.x, b.x, ax);
                bx = fmac(b.y, b.y, bx);
            }
            ax += bx;
            bx = 0;
        }
        const double sx = warp_sum_d((double)ax + (double)bx), sy = warp_sum_d((double)ay + (double)by);
        if (lane == 0) rs.partial[(long)i * gridDim.x + blockIdx.x] = make_double2(sx, sy);
    }
    if (arrive_last(rs.counter)) {
        final_sums(rs.partial, nvt, out);
        if (threadIdx.x == 0) *rs.counter = 0;
    }
}

// c = M s (r x r times r, FP64 sums) rounded to complex64; one warp per coefficient.
__global__ void defl_coef_kernel(const double2* __restrict__ M, const double2* __restrict__ s, int r, float2* cf,
                                 const int* skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < r; i += nw) {
        double cx = 0, cy = 0;
        for (int q = lane; q < r; q += 32) {
            const double2 m = M[(long)q * r + i], sv = s[q];
            cx = fmac(m.x, sv.x, cx); cx = fmac(-m.y, sv.y, cx);
            cy = fmac(m.x, sv.y, cy); cy = fmac(m.y, sv.x, cy);
        }
        cx = warp_sum_d(cx);
        cy = warp_sum_d(cy);
        if (lane == 0) cf[i] = make_float2((float)cx, (float)cy);
    }
}

// z = x + V c (c precomputed, complex64), all complex64: the deflation update of the
// FP32-inner solves.
__global__ void __launch_bounds__(kRedThreads) defl_update32_kernel(const float2* __restrict__ V, long ldv, int r,
                                                                    const float2* __restrict__ cf,
                                                                    const float2* x, float2* z, long n,
                                                                    const int* skip) {
    if (skip && *skip) return;
    __shared__ float2 cs[kMaxBasis];
    for (int i = threadIdx.x; i < r; i += blockDim.x) cs[i] = cf[i];
    __syncthreads();
    const long stride = (long)gridDim.x * blockDim.x;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += stride) {
        float2 acc = x[idx];
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

// out = base + sum_i V_i c_i.  Coefficients: c = sign * coef, or c = M s when M != NULL.
template <typename VT, bool NORM>
__global__ void __launch_bounds__(kRedThreads) basis_axpy_kernel(const VT* __restrict__ V, long ldv, int k,
                                                                 const double2* __restrict__ coef, double sign,
                                                                 const double2* __restrict__ M,
                                                                 const double2* __restrict__ s, const double2* base,
                                                                 double2* out, long n, double2* nrm2, Dgks dec,
                                                                 int has_dec, RedScratch rs, const int* skip) {
    using A = typename acc_of<VT>::type;
    if (skip && *skip) return;
    __shared__ VT cs[kMaxBasis];
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
    }
    __syncthreads();
    double nacc = 0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += stride) {
        A x0 = 0, y0 = 0, x1 = 0, y1 = 0;
        int i = 0;
#pragma unroll 4
        for (; i + 1 < k; i += 2) {
            const VT a = V[(long)i * ldv + idx], c = cs[i];
            const VT b = V[(long)(i + 1) * ldv + idx], d = cs[i + 1];
            x0 = fmac(a.x, c.x, x0); x0 = fmac(-a.y, c.y, x0);
            y0 = fmac(a.x, c.y, y0); y0 = fmac(a.y, c.x, y0);
            x1 = fmac(b.x, d.x, x1); x1 = fmac(-b.y, d.y, x1);
            y1 = fmac(b.x, d.y, y1); y1 = fmac(b.y, d.x, y1);
        }
        if (i < k) {
            const VT a = V[(long)i * ldv + idx], c = cs[i];
            x0 = fmac(a.x, c.x, x0); x0 = fmac(-a.y, c.y, x0);
            y0 = fmac(a.x, c.y, y0); y0 = fmac(a.y, c.x, y0);
        }
        double2 o = make_double2((double)x0 + (double)x1, (double)y0 + (double)y1);
        if (base) { const double2 bv = base[idx]; o.x += bv.x; o.y += bv.y; }
        out[idx] = o;
        if (NORM) { nacc = fmac(o.x, o.x, nacc); nacc = fmac(o.y, o.y, nacc); }
    }
    if (NORM) {
        __shared__ double red[kRedThreads / 32];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        nacc = warp_sum_d(nacc);
        if (lane == 0) red[warp] = nacc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int q = 0; q < kRedThreads / 32; q++) t += red[q];
            rs.partial[blockIdx.x] = make_double2(t, 0.0);
        }
        if (arrive_last(rs.counter)) {
            __shared__ double2 tot;
            final_sums(rs.partial, 1, &tot);
            __syncthreads();
            if (threadIdx.x == 0) {
                *rs.counter = 0;
                *nrm2 = tot;
                if (has_dec) {
                    const int r = dec.always || tot.x < dec.eta2 * dec.before2->x;
                    *dec.reorth = r;
                    *dec.skip2 = (dec.done && *dec.done) || !r;
                }
            }
        }
    }
}

// One Givens step of the restarted GMRES least-squares problem (Saad & Schultz):
// H(:, j) = h1 (+ h2) with H(j+1, j) = ||w||; apply the stored rotations, build the
// rotation that annihilates H(j+1, j), update g; residual estimate |g_{j+1}| / ||b||.
// The column, the stored rotations and g_j are staged in shared memory by the whole
// block (one global round trip instead of one per rotation), then thread 0 computes.
__global__ void arnoldi_finish_kernel(GmresDev S, int j, int step) {
    __shared__ double2 col[kMaxBasis + 2], csv[kMaxBasis], snv[kMaxBasis];
    if (*S.done) return;
    const int ld = S.m + 1;
    double2* Hgl = S.H + (long)j * ld;
    const int re = *S.reorth;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        col[i] = re ? make_double2(S.h1[i].x + S.h2[i].x, S.h1[i].y + S.h2[i].y) : S.h1[i];
        if (i < j) { csv[i] = S.cs[i]; snv[i] = S.sn[i]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
    double2* Hc = col;
    if (re) *S.nreorth += 1;
    const double wnorm2 = re ? S.nrm[1].x : S.nrm[0].x;
    const double before2 = S.h1[j + 1].x;
    const double hn = sqrt(fmax(wnorm2, 0.0));
    *S.wnorm = hn;
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
    S.cs[j] = make_double2(c, 0.0);
    S.sn[j] = s;
    const double2 gj = S.g[j];
    S.g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    S.g[j] = make_double2(c * gj.x, c * gj.y);
    const double est = hypot(S.g[j + 1].x, S.g[j + 1].y) / S.bnorm;
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

// v *= inv, with an optional complex64 copy of the result
__device__ __forceinline__ void scale_rows(double2* v, long n, double inv, float2* v32) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 a = v[i];
        const double2 b = make_double2(a.x * inv, a.y * inv);
        v[i] = b;
        if (v32) v32[i] = make_float2((float)b.x, (float)b.y);
    }
}

__global__ void scale_inv_sqrt_kernel(double2* v, long n, const double2* nrm2, const int* skip, float2* v32) {
    if (skip && *skip) return;
    const double s2 = nrm2->x;
    if (!(s2 > 0.0) || !isfinite(s2)) return;
    scale_rows(v, n, 1.0 / sqrt(s2), v32);
}

__global__ void scale_inv_real_kernel(double2* v, long n, const double* s, const int* skip, float2* v32) {
    if (skip && *skip) return;
    const double d = *s;
    if (!(d != 0.0) || !isfinite(d)) return;
    scale_rows(v, n, 1.0 / d, v32);
}

__global__ void sub_kernel(const double2* b, const double2* y, double2* r, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        r[i] = csub(b[i], y[i]);
}

__global__ void to_c64_kernel(const double2* x, float2* y, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = make_float2((float)x[i].x, (float)x[i].y);
}

__global__ void gmres_lsq_kernel(GmresDev S) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k = *S.k, ld = S.m + 1;
    for (int i = k - 1; i >= 0; i--) {
        double2 acc = S.g[i];
        for (int q = i + 1; q < k; q++) acc = csub(acc, cmul(S.H[(long)q * ld + i], S.y[q]));
        const double2 d = S.H[(long)i * ld + i];
        const double dd = d.x * d.x + d.y * d.y;
        if (dd == 0.0) { S.y[i] = make_double2(0, 0); *S.flags |= 4; continue; }
        S.y[i] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
    }
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
static inline int grid_for(long n) {
    long b = (n + kRedThreads - 1) / kRedThreads;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

die_status k_dots(const double2* V, long ldv, int nv, const double2* w, long n, int with_norm, double2* out,
                  const RedScratch& rs, const int* skip, cudaStream_t st) {
    if (nv + 1 > kMaxBasis || nv < 0) return DIE_EINVAL;
    DIE_PROF(PK_DOTS, st, dots_kernel<double2><<<kRedBlocks, kRedThreads, 0, st>>>(V, ldv, nv, w, n, with_norm, out, rs, skip));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_dots32(const float2* V, long ldv, int nv, const float2* w, long n, double2* out, const RedScratch& rs,
                    const int* skip, cudaStream_t st) {
    if (nv > kMaxBasis || nv < 0) return DIE_EINVAL;
    DIE_PROF(PK_DOTS32, st, dots_kernel<float2><<<kRedBlocks, kRedThreads, 0, st>>>(V, ldv, nv, w, n, 0, out, rs, skip));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_basis_axpy(const double2* V, long ldv, int k, const double2* coef, double sign, const double2* base,
                        double2* out, long n, double2* nrm2, const Dgks* dec, const RedScratch& rs, const int* skip,
                        cudaStream_t st) {
    if (k > kMaxBasis || k < 0) return DIE_EINVAL;
    const Dgks d = dec ? *dec : Dgks{};
    if (nrm2) {
        DIE_PROF(PK_UPDATE_NORM, st, basis_axpy_kernel<double2, true><<<kRedBlocks, kRedThreads, 0, st>>>(
                     V, ldv, k, coef, sign, nullptr, nullptr, base, out, n, nrm2, d, dec ? 1 : 0, rs, skip));
    } else {
        DIE_PROF(PK_LINCOMB, st, basis_axpy_kernel<double2, false><<<grid_for(n), kRedThreads, 0, st>>>(
                     V, ldv, k, coef, sign, nullptr, nullptr, base, out, n, nullptr, d, 0, rs, skip));
    }
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_defl_update(const double2* V, long ldv, int r, const double2* M, const double2* s, const double2* x,
                         double2* z, long n, const int* skip, cudaStream_t st) {
    if (r > kMaxBasis || r < 1) return DIE_EINVAL;
    DIE_PROF(PK_DEFL_UPDATE, st, basis_axpy_kernel<double2, false><<<grid_for(n), kRedThreads, 0, st>>>(
                 V, ldv, r, nullptr, 1.0, M, s, x, z, n, nullptr, Dgks{}, 0, RedScratch{}, skip));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_defl_update32(const float2* V, long ldv, int r, const double2* M, const double2* s, float2* cf,
                           const float2* x, float2* z, long n, const int* skip, cudaStream_t st) {
    if (r > kMaxBasis || r < 1) return DIE_EINVAL;
    DIE_PROF(PK_SMALL, st, defl_coef_kernel<<<1, 256, 0, st>>>(M, s, r, cf, skip));
    DIE_PROF(PK_DEFL_UPDATE, st, defl_update32_kernel<<<grid_for(n), kRedThreads, 0, st>>>(V, ldv, r, cf, x, z, n, skip));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

die_status cgs_dgks(const double2* V, long ldv, int nv, double2* w, long n, double2* h1, double2* h2, double2* nrm,
                    int* reorth, int* skip2, const int* done, double eta2, const RedScratch& rs, cudaStream_t st) {
    Dgks dec;
    dec.before2 = h1 + nv;
    dec.reorth = reorth;
    dec.skip2 = skip2;
    dec.done = done;
    dec.always = eta2 >= 1.0 ? 1 : 0;
    dec.eta2 = eta2;
    DIE_TRY(k_dots(V, ldv, nv, w, n, 1, h1, rs, done, st));
    DIE_TRY(k_basis_axpy(V, ldv, nv, h1, -1.0, w, w, n, nrm, &dec, rs, done, st));
    g_prof_override = PK_DOTS_REORTH;
    die_status s = k_dots(V, ldv, nv, w, n, 0, h2, rs, skip2, st);
    g_prof_override = PK_UPDATE_REORTH;
    if (s == DIE_OK) s = k_basis_axpy(V, ldv, nv, h2, -1.0, w, w, n, nrm + 1, nullptr, rs, skip2, st);
    g_prof_override = -1;
    return s;
}

die_status k_scale_inv_sqrt(double2* v, long n, const double2* nrm2, const int* skip, cudaStream_t st, float2* v32) {
    DIE_PROF(PK_SCALE, st, scale_inv_sqrt_kernel<<<grid_for(n), kRedThreads, 0, st>>>(v, n, nrm2, skip, v32));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_scale_inv_real(double2* v, long n, const double* s, const int* skip, cudaStream_t st, float2* v32) {
    DIE_PROF(PK_SCALE, st, scale_inv_real_kernel<<<grid_for(n), kRedThreads, 0, st>>>(v, n, s, skip, v32));
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
die_status k_arnoldi_finish(GmresDev S, int j, int step, cudaStream_t st) {
    DIE_PROF(PK_SMALL, st, arnoldi_finish_kernel<<<1, 128, 0, st>>>(S, j, step));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_gmres_lsq(GmresDev S, cudaStream_t st) {
    DIE_PROF(PK_SMALL, st, gmres_lsq_kernel<<<1, 32, 0, st>>>(S));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_gmres_init(GmresDev S, const double2* beta2, cudaStream_t st) {
    DIE_PROF(PK_SMALL, st, gmres_init_kernel<<<1, 32, 0, st>>>(S, beta2));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

}  // namespace die
