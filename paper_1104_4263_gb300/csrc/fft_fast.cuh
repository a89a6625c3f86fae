// Stockham stages with every index known at compile time except the thread's own
// position, for transform lengths L = 2^a, 256 <= L <= 4096, 16 values per thread
// (G = L / 16 threads per transform).  Same algorithm, radices and twiddles as the
// general stages of fft.cuh, with two facts used to cut the per-element work:
//
//  * Every shared-memory access of a stage is P(base(t) + c), with P(i) = i + (i >> 4)
//    the bank-conflict padding, base(t) a per-thread value and c a compile-time
//    constant such that (base & 15) + (c & 15) < 16.  Hence P(base + c) =
//    P(base) + c + (c >> 4): one base pointer per stage, immediate offsets after it.
//    (Loads: base = t, c = b G + r L / R, a multiple of 16.  Stores: base =
//    (t - t mod Ns) R + t mod Ns with c = b G R + s Ns, or base = t with
//    c = b G + s Ns in the last stage.  The bound on the low bits is checked at compile
//    time for every stage of every instantiated plan.)
//  * While Ns divides G (every stage but possibly the last), the twiddle index
//    k = (t + b G) mod Ns is the same for all butterflies of a thread, so the R - 1
//    twiddles are loaded once per stage.
//  * Twiddles come from per-stage tables (the `twx` arrays of the operator): the factor
//    exp(-2 pi i r k / (Ns R)) of a stage sits at r Ns + k - 1 of its plan's table
//    (forward plan at [0, L), inverse plan at [L, 2 L)), so the threads of a warp read
//    consecutive entries.  In the natural table the same factors are L r / (Ns R)
//    entries apart and one warp's load touches up to 16 cache lines.
#pragma once

#include "fft.cuh"

namespace die {

template <int L> struct P2 {
    static_assert(L >= 256 && L <= 4096 && (L & (L - 1)) == 0, "fast FFT path: L = 2^a, 256 <= L <= 4096");
    static constexpr int G = L / 16;
    static constexpr FftPlan fwd = pow2_plan(L, false);
    static constexpr FftPlan inv = pow2_plan(L, true);
};


// (base mod 16) + (c mod 16) < 16 for every load and store of a stage (see the top of
// the file).
template <int L, int R, int NS>
constexpr bool padding_linear() {
    constexpr int G = L / 16, B = 16 / R, LR = L / R;
    constexpr bool uniform = (G % NS) == 0;
    for (int t = 0; t < G; t++) {
        const int sb = uniform ? (t & ~(NS - 1)) * R + (t & (NS - 1)) : t;
        for (int b = 0; b < B; b++)
            for (int r = 0; r < R; r++) {
                const int cl = b * G + r * LR;
                const int cs = (uniform ? b * G * R : b * G) + r * NS;
                if ((t & 15) + (cl & 15) >= 16) return false;
                if ((sb & 15) + (cs & 15) >= 16) return false;
            }
    }
    return true;
}

template <typename V, int L, int R, int NS, bool INV>
struct FStage {
    static constexpr int kR = R;
    static constexpr int G = L / 16, B = 16 / R, LR = L / R;
    static constexpr bool kUniformK = (G % NS) == 0;    // twiddle index shared by the thread's butterflies
    static constexpr int kTwBase = INV ? L : 0;          // this plan's part of the stage tables
    static_assert(kUniformK || B * G <= NS, "last-stage layout");
    static_assert(padding_linear<L, R, NS>(), "shared-memory padding is not linear over this stage's accesses");

    // x[b R + r] = buf[P(t + b G + r L / R)]
    __host__ __device__ static __forceinline__ void load(const V* __restrict__ buf, V (&x)[16], int t) {
        const V* p = buf + pidx(t);
#pragma unroll
        for (int b = 0; b < B; b++)
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int c = b * G + r * LR;
                x[b * R + r] = p[c + (c >> 4)];
            }
    }

    // twiddles, then the radix-R DFTs
    __host__ __device__ static __forceinline__ void compute(V (&x)[16], int t, const V* __restrict__ tw) {
        if constexpr (NS > 1) {
            // tw[kTwBase + r NS + k - 1] = exp(-2 pi i r k / (NS R))
            if constexpr (kUniformK) {
                const int k = t & (NS - 1);
                V w[R];
#pragma unroll
                for (int r = 1; r < R; r++) {
                    w[r] = ld_tw(&tw[kTwBase + r * NS + k - 1]);
                    if (INV) w[r].y = -w[r].y;
                }
#pragma unroll
                for (int b = 0; b < B; b++)
#pragma unroll
                    for (int r = 1; r < R; r++) x[b * R + r] = cmul(x[b * R + r], w[r]);
            } else {
#pragma unroll
                for (int b = 0; b < B; b++) {
                    const int k = t + b * G;
#pragma unroll
                    for (int r = 1; r < R; r++) {
                        V w = ld_tw(&tw[kTwBase + r * NS + k - 1]);
                        if (INV) w.y = -w.y;
                        x[b * R + r] = cmul(x[b * R + r], w);
                    }
                }
            }
        }
#pragma unroll
        for (int b = 0; b < B; b++) dft<V, R, INV>(&x[b * R]);
    }

    // buf[P(out)] = x, out = (j - k) R + k + s NS for butterfly j = t + b G, k = j mod NS
    __host__ __device__ static __forceinline__ void store(V* __restrict__ buf, const V (&x)[16], int t) {
        const int base = kUniformK ? (t & ~(NS - 1)) * R + (t & (NS - 1)) : t;
        V* p = buf + pidx(base);
#pragma unroll
        for (int b = 0; b < B; b++)
#pragma unroll
            for (int s = 0; s < R; s++) {
                const int c = (kUniformK ? b * G * R : b * G) + s * NS;
                p[c + (c >> 4)] = x[b * R + s];
            }
    }

    // The same stage on two independent transforms (x0, x1) at the same indices, with the
    // twiddles loaded once for both.
    __host__ __device__ static __forceinline__ void compute2(V (&x0)[16], V (&x1)[16], int t, const V* __restrict__ tw) {
        if constexpr (NS > 1) {
            if constexpr (kUniformK) {
                const int k = t & (NS - 1);
#pragma unroll
                for (int r = 1; r < R; r++) {
                    V w = ld_tw(&tw[kTwBase + r * NS + k - 1]);
                    if (INV) w.y = -w.y;
#pragma unroll
                    for (int b = 0; b < B; b++) {
                        x0[b * R + r] = cmul(x0[b * R + r], w);
                        x1[b * R + r] = cmul(x1[b * R + r], w);
                    }
                }
            } else {
#pragma unroll
                for (int b = 0; b < B; b++) {
                    const int k = t + b * G;
#pragma unroll
                    for (int r = 1; r < R; r++) {
                        V w = ld_tw(&tw[kTwBase + r * NS + k - 1]);
                        if (INV) w.y = -w.y;
                        x0[b * R + r] = cmul(x0[b * R + r], w);
                        x1[b * R + r] = cmul(x1[b * R + r], w);
                    }
                }
            }
        }
#pragma unroll
        for (int b = 0; b < B; b++) {
            dft<V, R, INV>(&x0[b * R]);
            dft<V, R, INV>(&x1[b * R]);
        }
    }

    // Natural index of register e in the stage's input (first stage) or output (last stage).
    static constexpr int index(int e) { return (e / R) * G + (e % R) * LR; }
};

// Stage s of a compile-time plan, with its NS.
template <typename V, int L, bool INV, int S>
struct PlanStage {
    static constexpr FftPlan pl = INV ? P2<L>::inv : P2<L>::fwd;
    static constexpr int R = pl.radix[S];
    static constexpr int ns() {
        int v = 1;
        for (int q = 0; q < S; q++) v *= pl.radix[q];
        return v;
    }
    static constexpr int NS = ns();
    using St = FStage<V, L, R, NS, INV>;
};

// Run stages [S0, S1) of the plan in place on buf: each loads from buf (except the
// first when FROM_REGS: x already holds its inputs), computes, stores back.  All
// threads of the block call it (block barriers); inactive threads pass active=false.
template <typename V, int L, bool INV, int S0, int S1, bool FROM_REGS>
__device__ __forceinline__ void run_fast(V* buf, V (&x)[16], int t, const V* tw, bool active) {
    if constexpr (S0 < S1) {
        using PS = PlanStage<V, L, INV, S0>;
        if constexpr (!FROM_REGS) {
            if (active) PS::St::load(buf, x, t);
            __syncthreads();
        }
        if (active) {
            PS::St::compute(x, t, tw);
            PS::St::store(buf, x, t);
        }
        __syncthreads();
        run_fast<V, L, INV, S0 + 1, S1, false>(buf, x, t, tw, active);
    }
}

// run_fast on two transforms held by the same threads, in buffers buf0 and buf1.
template <typename V, int L, bool INV, int S0, int S1>
__device__ __forceinline__ void run_fast2(V* buf0, V* buf1, V (&x0)[16], V (&x1)[16], int t, const V* tw) {
    if constexpr (S0 < S1) {
        using St = typename PlanStage<V, L, INV, S0>::St;
        St::load(buf0, x0, t);
        St::load(buf1, x1, t);
        __syncthreads();
        St::compute2(x0, x1, t, tw);
        St::store(buf0, x0, t);
        St::store(buf1, x1, t);
        __syncthreads();
        run_fast2<V, L, INV, S0 + 1, S1>(buf0, buf1, x0, x1, t, tw);
    }
}

}  // namespace die
