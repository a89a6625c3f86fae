// Shared-memory Stockham FFT building blocks for lengths 2^a and 3 * 2^a.
//
// A transform of length L is done by a group of G = L / EPT threads; each thread
// holds EPT complex values in registers.  A stage of radix R (R | EPT) lets every
// thread run EPT / R radix-R butterflies.  Butterfly j of the stage with current
// sub-transform length Ns reads x_r = in[j + r L/R] (r < R), multiplies x_r by
// exp(-+ 2 pi i r k / (Ns R)) with k = j mod Ns, does a radix-R DFT and writes
// y_s to out[(j - k) R + k + s Ns].  After all stages (Ns = L) the result is in
// natural order, for any ordering of the radices (Stockham autosort).
//
// Stages exchange data in place through one shared-memory array per transform:
// every stage loads its inputs into registers, the block synchronises, and the
// outputs are stored.  The first stage may load from global memory and the last
// stage may store to global memory directly; the index sets of both are
// j + r L/R, i.e. coalesced across the threads of a group.
//
// Forward transforms use exp(-2 pi i ...), inverse ones exp(+2 pi i ...), both
// unnormalised.  Twiddles come from a table tw[m] = exp(-2 pi i m / L), m < L,
// built on the host in FP64.
#pragma once

#include "common.cuh"

namespace die {

constexpr int kMaxStages = 8;

struct FftPlan {
    int L;                    // transform length
    int ns;                   // number of stages
    int radix[kMaxStages];    // radix of each stage, product = L
    int ept;                  // complex values held per thread (16 for 2^a, 12 for 3*2^a)
};

// ------------------------------------------------------------------ small DFTs
template <typename V, bool INV>
__host__ __device__ __forceinline__ V rot_q(V a) { return INV ? mul_pi(a) : mul_mi(a); }   // * (-+ i)

template <typename V, bool INV>
__host__ __device__ __forceinline__ void dft2(V& a, V& b) { V t = a; a = cadd(t, b); b = csub(t, b); }

template <typename V, bool INV>
__host__ __device__ __forceinline__ void dft4(V& x0, V& x1, V& x2, V& x3) {
    V a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = rot_q<V, INV>(csub(x1, x3));
    x0 = cadd(a, c); x2 = csub(a, c); x1 = cadd(b, d); x3 = csub(b, d);
}

template <typename V, bool INV>
__host__ __device__ __forceinline__ void dft3(V& x0, V& x1, V& x2) {
    using T = typename real_of<V>::type;
    const T h3 = (T)0.86602540378443864676;   // sqrt(3)/2
    V s = cadd(x1, x2), d = csub(x1, x2);
    V m = csub(x0, cscale(s, (T)0.5));
    V t = cscale(rot_q<V, INV>(d), h3);       // -+ i sqrt(3)/2 (x1 - x2)
    x0 = cadd(x0, s); x1 = cadd(m, t); x2 = csub(m, t);
}

// multiply by exp(-+ i pi q / 4), q = 1..3
template <typename V, bool INV>
__host__ __device__ __forceinline__ V w8(V a, int q) {
    using T = typename real_of<V>::type;
    const T r2 = (T)0.70710678118654752440;
    if (q == 1) { V t = INV ? mk((T)(a.x - a.y), (T)(a.x + a.y)) : mk((T)(a.x + a.y), (T)(a.y - a.x)); return cscale(t, r2); }
    if (q == 2) return rot_q<V, INV>(a);
    // q == 3: exp(-+ 3 i pi/4) = (-1 -+ i)/sqrt(2)
    V t = INV ? mk((T)(-a.x - a.y), (T)(a.x - a.y)) : mk((T)(a.y - a.x), (T)(-a.x - a.y));
    return cscale(t, r2);
}

template <typename V, bool INV>
__host__ __device__ __forceinline__ void dft8(V* x) {
    // even/odd split: E = DFT4(x0,x2,x4,x6), O = DFT4(x1,x3,x5,x7); y_s = E_s + w8^s O_s
    V e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    V o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4<V, INV>(e0, e1, e2, e3);
    dft4<V, INV>(o0, o1, o2, o3);
    o1 = w8<V, INV>(o1, 1); o2 = w8<V, INV>(o2, 2); o3 = w8<V, INV>(o3, 3);
    x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
    x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
    x[2] = cadd(e2, o2); x[6] = csub(e2, o2);
    x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
}

template <typename V, bool INV>
__host__ __device__ __forceinline__ void dft16(V* x) {
    using T = typename real_of<V>::type;
    // cos / sin of s pi / 8, s = 0..7
    const T c[8] = {(T)1.0, (T)0.92387953251128675613, (T)0.70710678118654752440, (T)0.38268343236508977173,
                    (T)0.0, (T)-0.38268343236508977173, (T)-0.70710678118654752440, (T)-0.92387953251128675613};
    const T s[8] = {(T)0.0, (T)0.38268343236508977173, (T)0.70710678118654752440, (T)0.92387953251128675613,
                    (T)1.0, (T)0.92387953251128675613, (T)0.70710678118654752440, (T)0.38268343236508977173};
    V e[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; i++) { e[i] = x[2 * i]; o[i] = x[2 * i + 1]; }
    dft8<V, INV>(e);
    dft8<V, INV>(o);
#pragma unroll
    for (int q = 0; q < 8; q++) {
        V w = INV ? mk(c[q], s[q]) : mk(c[q], (T)-s[q]);
        V t = (q == 0) ? o[q] : cmul(o[q], w);
        x[q] = cadd(e[q], t);
        x[q + 8] = csub(e[q], t);
    }
}

template <typename V, int R, bool INV>
__host__ __device__ __forceinline__ void dft(V* x) {
    static_assert(R == 2 || R == 3 || R == 4 || R == 8 || R == 16, "radix 2, 3, 4, 8 or 16");
    if constexpr (R == 2) dft2<V, INV>(x[0], x[1]);
    else if constexpr (R == 3) dft3<V, INV>(x[0], x[1], x[2]);
    else if constexpr (R == 4) dft4<V, INV>(x[0], x[1], x[2], x[3]);
    else if constexpr (R == 8) dft8<V, INV>(x);
    else if constexpr (R == 16) dft16<V, INV>(x);
}

// ------------------------------------------------------------ stage primitives
// Shared-memory arrays are padded by one slot per 16 elements: the stride-R stores of
// the early stages (thread j writes j R + r) then fall in distinct banks.
__host__ __device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int padded_len(int L) { return L + (L >> 4); }

// Twiddle load: read-only cache path on the device, plain load on the host (the stage
// code also runs on the host, where a CPU test checks it against a plain DFT).
template <typename V> __host__ __device__ __forceinline__ V ld_tw(const V* p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// 1 + index of the lowest set bit (0 for x == 0)
__host__ __device__ __forceinline__ int ffs_int(int x) {
#ifdef __CUDA_ARCH__
    return __ffs(x);
#else
    return __builtin_ffs(x);
#endif
}

// j mod Ns (Ns is a power of two for 2^a transforms, possibly 3 * 2^b otherwise)
__host__ __device__ __forceinline__ int mod_ns(int j, int Ns) { return (Ns & (Ns - 1)) == 0 ? (j & (Ns - 1)) : j % Ns; }
// Thread t of a group of G threads handles butterflies j = t + b G, b < EPT/R.
// Register x[b * R + r] holds input r of butterfly b.

template <typename V, int EPT, int R>
__host__ __device__ __forceinline__ void stage_load(const V* __restrict__ buf, V (&x)[EPT], int L, int t, int G) {
    constexpr int B = EPT / R;
    const int LR = L / R;
#pragma unroll
    for (int b = 0; b < B; b++) {
        const int j = t + b * G;
#pragma unroll
        for (int r = 0; r < R; r++) x[b * R + r] = buf[pidx(j + r * LR)];
    }
}

template <typename V, int EPT, int R, bool INV>
__host__ __device__ __forceinline__ void stage_compute(V (&x)[EPT], int L, int Ns, int t, int G, const V* __restrict__ tw) {
    constexpr int B = EPT / R;
#pragma unroll
    for (int b = 0; b < B; b++) {
        const int j = t + b * G;
        if (Ns > 1) {
            const int k = mod_ns(j, Ns);
            const int LR = L / R;
            const int step = ((Ns & (Ns - 1)) == 0 ? (LR >> (ffs_int(Ns) - 1)) : LR / Ns) * k;
#pragma unroll
            for (int r = 1; r < R; r++) {
                V w = ld_tw(&tw[r * step]);
                if (INV) w.y = -w.y;
                x[b * R + r] = cmul(x[b * R + r], w);
            }
        }
        dft<V, R, INV>(&x[b * R]);
    }
}

template <typename V, int EPT, int R>
__host__ __device__ __forceinline__ void stage_store(V* __restrict__ buf, const V (&x)[EPT], int L, int Ns, int t, int G) {
    constexpr int B = EPT / R;
#pragma unroll
    for (int b = 0; b < B; b++) {
        const int j = t + b * G;
        const int k = mod_ns(j, Ns);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; r++) buf[pidx(base + r * Ns)] = x[b * R + r];
    }
}

// Dispatch helpers over the runtime radix (EPT = 16: R in {2,4,8,16}; EPT = 12: R in {2,3,4}).
template <typename V, int EPT, bool INV>
__host__ __device__ __forceinline__ void compute_any(int R, V (&x)[EPT], int L, int Ns, int t, int G, const V* tw) {
    if constexpr (EPT % 16 == 0) { if (R == 16) { stage_compute<V, EPT, 16, INV>(x, L, Ns, t, G, tw); return; } }
    if constexpr (EPT % 8 == 0) { if (R == 8) { stage_compute<V, EPT, 8, INV>(x, L, Ns, t, G, tw); return; } }
    if constexpr (EPT % 4 == 0) { if (R == 4) { stage_compute<V, EPT, 4, INV>(x, L, Ns, t, G, tw); return; } }
    if constexpr (EPT % 3 == 0) { if (R == 3) { stage_compute<V, EPT, 3, INV>(x, L, Ns, t, G, tw); return; } }
    if constexpr (EPT % 2 == 0) { if (R == 2) { stage_compute<V, EPT, 2, INV>(x, L, Ns, t, G, tw); return; } }
}

template <typename V, int EPT>
__host__ __device__ __forceinline__ void load_any(int R, const V* buf, V (&x)[EPT], int L, int t, int G) {
    if constexpr (EPT % 16 == 0) { if (R == 16) { stage_load<V, EPT, 16>(buf, x, L, t, G); return; } }
    if constexpr (EPT % 8 == 0) { if (R == 8) { stage_load<V, EPT, 8>(buf, x, L, t, G); return; } }
    if constexpr (EPT % 4 == 0) { if (R == 4) { stage_load<V, EPT, 4>(buf, x, L, t, G); return; } }
    if constexpr (EPT % 3 == 0) { if (R == 3) { stage_load<V, EPT, 3>(buf, x, L, t, G); return; } }
    if constexpr (EPT % 2 == 0) { if (R == 2) { stage_load<V, EPT, 2>(buf, x, L, t, G); return; } }
}

template <typename V, int EPT>
__host__ __device__ __forceinline__ void store_any(int R, V* buf, const V (&x)[EPT], int L, int Ns, int t, int G) {
    if constexpr (EPT % 16 == 0) { if (R == 16) { stage_store<V, EPT, 16>(buf, x, L, Ns, t, G); return; } }
    if constexpr (EPT % 8 == 0) { if (R == 8) { stage_store<V, EPT, 8>(buf, x, L, Ns, t, G); return; } }
    if constexpr (EPT % 4 == 0) { if (R == 4) { stage_store<V, EPT, 4>(buf, x, L, Ns, t, G); return; } }
    if constexpr (EPT % 3 == 0) { if (R == 3) { stage_store<V, EPT, 3>(buf, x, L, Ns, t, G); return; } }
    if constexpr (EPT % 2 == 0) { if (R == 2) { stage_store<V, EPT, 2>(buf, x, L, Ns, t, G); return; } }
}

// Element e = b*R + r of the register array sits at natural index j + r L/R of the
// stage's input (first stage) or output (last stage, Ns = L/R), j = t + b G.
template <int EPT>
__host__ __device__ __forceinline__ int reg_index(int e, int R, int L, int t, int G) {
    if ((R & (R - 1)) == 0) {
        const int lg = ffs_int(R) - 1;
        return t + (e >> lg) * G + (e & (R - 1)) * (L >> lg);
    }
    const int b = e / R, r = e - b * R;
    return t + b * G + r * (L / R);
}

// Plan of a power-of-two length known at compile time (the same radices as the host
// planner): kernels instantiated for a fixed L use it so that every radix, stride and
// index in the stage code is a constant.
__host__ __device__ constexpr FftPlan pow2_plan(int L, bool reversed) {
    FftPlan p{};
    int a = 0;
    while ((1 << a) < L) a++;
    p.L = L;
    p.ept = 16;
    const int stages = (a + 3) / 4;
    const int base = a / stages, extra = a % stages;
    p.ns = stages;
    for (int s = 0; s < stages; s++) p.radix[reversed ? stages - 1 - s : s] = 1 << (base + (s < extra ? 1 : 0));
    return p;
}

// Run stages [s0, s1) of plan `pl` in place on `buf` (shared memory).  Every thread
// of the block must call this (block-wide barriers); t/G identify the caller's
// position within the group that owns `buf`.
template <typename V, int EPT, bool INV>
__device__ __forceinline__ void run_stages(V* buf, const FftPlan& pl, int s0, int s1, int& Ns, const V* tw,
                                           int t, int G, bool active) {
    V x[EPT];
#pragma unroll
    for (int s = s0; s < s1; s++) {
        const int R = pl.radix[s];
        if (active) load_any<V, EPT>(R, buf, x, pl.L, t, G);
        __syncthreads();
        if (active) {
            compute_any<V, EPT, INV>(R, x, pl.L, Ns, t, G, tw);
            store_any<V, EPT>(R, buf, x, pl.L, Ns, t, G);
        }
        __syncthreads();
        Ns *= R;
    }
}

}  // namespace die
