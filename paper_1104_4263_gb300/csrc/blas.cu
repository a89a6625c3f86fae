// Krylov-space kernels (see krylov.cuh).  Reductions: every block accumulates a
// fixed, grid-strided share of the rows, reduces it with warp shuffles in a fixed
// order and writes one partial per vector; the last block to arrive (atomic
// counter) sums the partials of each vector in a fixed order.  Results therefore
// do not depend on scheduling.
#include "krylov.cuh"
#include "prof.cuh"

namespace die {

__device__ __forceinline__ double2 shfl_down2(double2 v, int off) {
    v.x = __shfl_down_sync(0xffffffffu, v.x, off);
    v.y = __shfl_down_sync(0xffffffffu, v.y, off);
    return v;
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) { double2 o = shfl_down2(v, off); v.x += o.x; v.y += o.y; }
    return v;
}

// Reduce acc[0..cnt) over the block and store the block's partials of vectors vbase + i.
template <int CH>
__device__ __forceinline__ void block_partials(double2 (&acc)[CH], int cnt, double2* partial, int vbase) {
    __shared__ double2 red[kRedThreads / 32][CH];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < CH; i++) acc[i] = warp_sum(acc[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < CH; i++) red[warp][i] = acc[i];
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        double2 s = make_double2(0, 0);
        for (int w = 0; w < kRedThreads / 32; w++) { s.x += red[w][threadIdx.x].x; s.y += red[w][threadIdx.x].y; }
        partial[(long)(vbase + threadIdx.x) * kRedBlocks + blockIdx.x] = s;
    }
    __syncthreads();
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
        double2 s = make_double2(0, 0);
        for (int b = lane; b < (int)gridDim.x; b += 32) {
            const double2 p = __ldcg(&partial[(long)i * kRedBlocks + b]);
            s.x += p.x; s.y += p.y;
        }
        s = warp_sum(s);
        if (lane == 0) out[i] = s;
    }
}

constexpr int kCh = 8;

// acc_i += conj(V_i[idx]) w[idx] for vectors c0 .. c0+cnt over this thread's rows.
__device__ __forceinline__ void dot_chunk(const double2* __restrict__ V, long ldv, int c0, int cnt,
                                          const double2* __restrict__ w, long n, double2 (&acc)[kCh]) {
    const long stride = (long)gridDim.x * blockDim.x;
#pragma unroll
    for (int i = 0; i < kCh; i++) acc[i] = make_double2(0, 0);
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += stride) {
        const double2 wv = w[idx];
#pragma unroll
        for (int i = 0; i < kCh; i++) {
            if (i < cnt) {
                const double2 a = V[(long)(c0 + i) * ldv + idx];
                acc[i].x = fma(a.x, wv.x, fma(a.y, wv.y, acc[i].x));
                acc[i].y = fma(a.x, wv.y, fma(-a.y, wv.x, acc[i].y));
            }
        }
    }
}

__device__ __forceinline__ void all_dots(const double2* V, long ldv, int nv, const double2* w, long n, double2* partial) {
    for (int c0 = 0; c0 < nv; c0 += kCh) {
        const int cnt = imin(kCh, nv - c0);
        double2 acc[kCh];
        dot_chunk(V, ldv, c0, cnt, w, n, acc);
        block_partials<kCh>(acc, cnt, partial, c0);
    }
}

// w[idx] -= sum_i V_i[idx] h_i over this thread's rows (h in shared memory).
__device__ __forceinline__ void update_rows(const double2* __restrict__ V, long ldv, int nv, double2* __restrict__ w,
                                            long n, const double2* hs) {
    const long stride = (long)gridDim.x * blockDim.x;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += stride) {
        double2 wv = w[idx];
        for (int i = 0; i < nv; i++) {
            const double2 a = V[(long)i * ldv + idx];
            const double2 hh = hs[i];
            wv.x -= a.x * hh.x - a.y * hh.y;
            wv.y -= a.x * hh.y + a.y * hh.x;
        }
        w[idx] = wv;
    }
}

__global__ void __launch_bounds__(kRedThreads) dots_kernel(const double2* V, long ldv, int nv, const double2* w,
                                                           long n, double2* out, RedScratch rs, const int* skip) {
    if (skip && *skip) return;
    all_dots(V, ldv, nv, w, n, rs.partial);
    if (arrive_last(rs.counter)) {
        final_sums(rs.partial, nv, out);
        if (threadIdx.x == 0) *rs.counter = 0;
    }
}

__global__ void __launch_bounds__(kRedThreads) update_dots_kernel(const double2* V, long ldv, int nv, double2* w,
                                                                  long n, const double2* h, double2* out,
                                                                  RedScratch rs, const int* skip) {
    if (skip && *skip) return;
    __shared__ double2 hs[kMaxBasis];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    update_rows(V, ldv, nv, w, n, hs);
    all_dots(V, ldv, nv, w, n, rs.partial);   // each thread re-reads only rows it wrote
    if (arrive_last(rs.counter)) {
        final_sums(rs.partial, nv, out);
        if (threadIdx.x == 0) *rs.counter = 0;
    }
}

__global__ void __launch_bounds__(kRedThreads) update_norm_kernel(const double2* V, long ldv, int nv, double2* w,
                                                                  long n, const double2* h, double2* out,
                                                                  RedScratch rs, const int* skip) {
    if (skip && *skip) return;
    __shared__ double2 hs[kMaxBasis];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    update_rows(V, ldv, nv, w, n, hs);
    all_dots(w, 0, 1, w, n, rs.partial);
    if (arrive_last(rs.counter)) {
        final_sums(rs.partial, 1, out);
        if (threadIdx.x == 0) *rs.counter = 0;
    }
}

// One Givens step of the restarted GMRES least-squares problem (Saad & Schultz):
// H(:, j) = h1 + h2 with H(j+1, j) = ||w||; apply the stored rotations, build the
// rotation that annihilates H(j+1, j), update g; residual estimate |g_{j+1}| / ||b||.
__device__ void givens_step(GmresDev S, int j, int step, double wnorm2, double wnorm2_before) {
    const int ld = S.m + 1;
    double2* Hc = S.H + (long)j * ld;
    for (int i = 0; i <= j; i++) Hc[i] = make_double2(S.h1[i].x + S.h2[i].x, S.h1[i].y + S.h2[i].y);
    const double hn = sqrt(fmax(wnorm2, 0.0));
    *S.wnorm = hn;
    Hc[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; i++) {
        const double c = S.cs[i].x;
        const double2 s = S.sn[i];
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
    const bool breakdown = hn <= 1e-14 * sqrt(fmax(wnorm2_before, 0.0));
    if (bad) *S.flags |= 1;
    if (breakdown) *S.flags |= 2;
    if (bad || breakdown || est <= S.tol || j + 1 >= S.jmax) *S.done = 1;
}

__global__ void __launch_bounds__(kRedThreads) update_norm_givens_kernel(const double2* V, long ldv, int nv,
                                                                         double2* w, long n, GmresDev S, int j,
                                                                         int step, RedScratch rs) {
    if (*S.done) return;
    __shared__ double2 hs[kMaxBasis];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = S.h2[i];
    __syncthreads();
    update_rows(V, ldv, nv, w, n, hs);
    all_dots(w, 0, 1, w, n, rs.partial);
    if (arrive_last(rs.counter)) {
        __shared__ double2 nrm;
        final_sums(rs.partial, 1, &nrm);
        __syncthreads();
        if (threadIdx.x == 0) {
            *rs.counter = 0;
            givens_step(S, j, step, nrm.x, S.h1[nv].x);
        }
    }
}

__global__ void scale_inv_sqrt_kernel(double2* v, long n, const double2* nrm2, const int* skip) {
    if (skip && *skip) return;
    const double s2 = nrm2->x;
    if (!(s2 > 0.0) || !isfinite(s2)) return;
    const double inv = 1.0 / sqrt(s2);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 a = v[i];
        v[i] = make_double2(a.x * inv, a.y * inv);
    }
}

__global__ void scale_inv_real_kernel(double2* v, long n, const double* s, const int* skip) {
    if (skip && *skip) return;
    const double d = *s;
    if (!(d != 0.0) || !isfinite(d)) return;
    const double inv = 1.0 / d;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 a = v[i];
        v[i] = make_double2(a.x * inv, a.y * inv);
    }
}

__global__ void sub_kernel(const double2* b, const double2* y, double2* r, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        r[i] = csub(b[i], y[i]);
}

template <bool ADD>
__global__ void lincomb_kernel(const double2* __restrict__ V, long ldv, int k, const double2* __restrict__ c,
                               double2* __restrict__ out, long n) {
    __shared__ double2 cs[kMaxBasis];
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = c[i];
    __syncthreads();
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
        double2 s = ADD ? out[idx] : make_double2(0, 0);
        for (int i = 0; i < k; i++) s = cadd(s, cmul(V[(long)i * ldv + idx], cs[i]));
        out[idx] = s;
    }
}

// z = x + V (M s); M: r x r column-major.  Each block forms c = M s redundantly.
__global__ void defl_update_kernel(const double2* __restrict__ V, long ldv, int r, const double2* __restrict__ M,
                                   const double2* __restrict__ s, const double2* x, double2* z, long n,
                                   const int* skip) {
    if (skip && *skip) return;
    __shared__ double2 cs[kMaxBasis];
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
        double2 acc = make_double2(0, 0);
        for (int q = 0; q < r; q++) acc = cadd(acc, cmul(M[(long)q * r + i], s[q]));
        cs[i] = acc;
    }
    __syncthreads();
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
        double2 acc = x[idx];
        for (int i = 0; i < r; i++) acc = cadd(acc, cmul(V[(long)i * ldv + idx], cs[i]));
        z[idx] = acc;
    }
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
        // acc / d
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

die_status k_dots(const double2* V, long ldv, int nv, const double2* w, long n, double2* out, const RedScratch& rs,
                  const int* skip, cudaStream_t st) {
    if (nv > kMaxBasis) return DIE_EINVAL;
    DIE_PROF(PK_DOTS, st, dots_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(V, ldv, nv, w, n, out, rs, skip));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_cgs_update_dots(const double2* V, long ldv, int nv, double2* w, long n, const double2* h, double2* out,
                             const RedScratch& rs, const int* skip, cudaStream_t st) {
    if (nv > kMaxBasis) return DIE_EINVAL;
    DIE_PROF(PK_UPDATE_DOTS, st, update_dots_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(V, ldv, nv, w, n, h, out, rs, skip));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_cgs_update_norm_givens(const double2* V, long ldv, int nv, double2* w, long n, GmresDev S, int j,
                                    int step, const RedScratch& rs, cudaStream_t st) {
    if (nv > kMaxBasis) return DIE_EINVAL;
    DIE_PROF(PK_UPDATE_NORM, st, update_norm_givens_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(V, ldv, nv, w, n, S, j, step, rs));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_cgs_update_norm(const double2* V, long ldv, int nv, double2* w, long n, const double2* h, double2* out,
                             const RedScratch& rs, const int* skip, cudaStream_t st) {
    if (nv > kMaxBasis) return DIE_EINVAL;
    DIE_PROF(PK_UPDATE_NORM, st, update_norm_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(V, ldv, nv, w, n, h, out, rs, skip));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_scale_inv_sqrt(double2* v, long n, const double2* nrm2, const int* skip, cudaStream_t st) {
    DIE_PROF(PK_SCALE, st, scale_inv_sqrt_kernel<<<grid_for(n), kRedThreads, 0, st>>>(v, n, nrm2, skip));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_scale_inv_real(double2* v, long n, const double* s, const int* skip, cudaStream_t st) {
    DIE_PROF(PK_SCALE, st, scale_inv_real_kernel<<<grid_for(n), kRedThreads, 0, st>>>(v, n, s, skip));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_sub(const double2* b, const double2* y, double2* r, long n, cudaStream_t st) {
    DIE_PROF(PK_OTHER, st, sub_kernel<<<grid_for(n), kRedThreads, 0, st>>>(b, y, r, n));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_lincomb_add(const double2* V, long ldv, int k, const double2* c, double2* x, long n, cudaStream_t st) {
    if (k > kMaxBasis) return DIE_EINVAL;
    DIE_PROF(PK_LINCOMB, st, lincomb_kernel<true><<<grid_for(n), kRedThreads, 0, st>>>(V, ldv, k, c, x, n));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_lincomb(const double2* V, long ldv, int k, const double2* c, double2* out, long n, cudaStream_t st) {
    if (k > kMaxBasis) return DIE_EINVAL;
    DIE_PROF(PK_LINCOMB, st, lincomb_kernel<false><<<grid_for(n), kRedThreads, 0, st>>>(V, ldv, k, c, out, n));
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}
die_status k_defl_update(const double2* V, long ldv, int r, const double2* M, const double2* s, const double2* x,
                         double2* z, long n, const int* skip, cudaStream_t st) {
    if (r > kMaxBasis) return DIE_EINVAL;
    DIE_PROF(PK_DEFL_UPDATE, st, defl_update_kernel<<<grid_for(n), kRedThreads, 0, st>>>(V, ldv, r, M, s, x, z, n, skip));
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
