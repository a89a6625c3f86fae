// Host run of the Stockham stages of the product kernels (fft_fast.cuh, fft.cuh):
// every thread of a transform group executes its stage loads, twiddles, radix-R DFTs and
// stores in turn, with the block barriers between stages taken as phase boundaries.  The
// result is compared with the plain DFT sum in long double.  Prints one line per
// (length, direction, precision): "L dir prec max_rel_err" for the compile-time plans,
// "genL dir prec max_rel_err" for the runtime-plan stages of the general kernels.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>
#include <vector>

#include "../paper_1104_4263_gb300/csrc/fft_fast.cuh"

using namespace die;

template <typename V, int L, bool INV, int S, int NS>
void run_stages(V* buf, std::vector<std::array<V, 16>>& x, const V* tw) {
    if constexpr (S < NS) {
        using St = typename PlanStage<V, L, INV, S>::St;
        constexpr int G = L / 16;
        using Regs = V[16];
        if constexpr (S > 0)
            for (int t = 0; t < G; t++) St::load(buf, *reinterpret_cast<Regs*>(x[t].data()), t);
        for (int t = 0; t < G; t++) St::compute(*reinterpret_cast<Regs*>(x[t].data()), t, tw);
        if constexpr (S + 1 < NS)
            for (int t = 0; t < G; t++) St::store(buf, *reinterpret_cast<const Regs*>(x[t].data()), t);
        run_stages<V, L, INV, S + 1, NS>(buf, x, tw);
    }
}

template <typename V, int L, bool INV>
double max_rel_err() {
    using T = typename real_of<V>::type;
    constexpr int G = L / 16;
    constexpr FftPlan pl = INV ? P2<L>::inv : P2<L>::fwd;
    using F0 = typename PlanStage<V, L, INV, 0>::St;
    using FL = typename PlanStage<V, L, INV, pl.ns - 1>::St;
    const long double pi = 3.141592653589793238462643383279502884L;
    // stage tables as the fast stages read them: the forward plan at [0, L), the inverse
    // plan at [L, 2 L); stage (radix R, sub-transform length Ns) holds
    // exp(-2 pi i r k / (Ns R)) at r Ns + k - 1 for 1 <= r < R, k < Ns
    std::vector<V> tw(2 * L), buf(padded_len(L));
    for (int part = 0; part < 2; part++) {
        const FftPlan p = part ? P2<L>::inv : P2<L>::fwd;
        for (int st = 0, ns = 1; st < p.ns; ns *= p.radix[st], st++)
            for (int r = 1; r < p.radix[st]; r++)
                for (int k = 0; k < ns; k++) {
                    const long double a = -2.0L * pi * (long double)(r * k) / (long double)(ns * p.radix[st]);
                    tw[part * L + r * ns + k - 1] = mk((T)std::cos(a), (T)std::sin(a));
                }
    }
    std::vector<std::complex<long double>> in(L);
    unsigned s = 20110421u;                       // fixed LCG: the input needs no other source
    for (int i = 0; i < L; i++) {
        s = s * 1103515245u + 12345u;
        const double a = (s >> 8) / 16777216.0 - 0.5;
        s = s * 1103515245u + 12345u;
        const double b = (s >> 8) / 16777216.0 - 0.5;
        in[i] = {(long double)(T)a, (long double)(T)b};
    }
    std::vector<std::array<V, 16>> x(G);
    for (int t = 0; t < G; t++)
        for (int e = 0; e < 16; e++) {
            const auto v = in[t + F0::index(e)];
            x[t][e] = mk((T)v.real(), (T)v.imag());
        }
    run_stages<V, L, INV, 0, pl.ns>(buf.data(), x, tw.data());
    long double err = 0, nrm = 0;
    for (int t = 0; t < G; t++)
        for (int e = 0; e < 16; e++) {
            const int k = t + FL::index(e);
            std::complex<long double> acc = 0;
            for (int j = 0; j < L; j++) {
                const long double a = (INV ? 2.0L : -2.0L) * pi * (long double)((long)j * k % L) / L;
                acc += in[j] * std::complex<long double>(std::cos(a), std::sin(a));
            }
            const std::complex<long double> got(x[t][e].x, x[t][e].y);
            err = std::max(err, std::abs(got - acc));
            nrm = std::max(nrm, std::abs(acc));
        }
    return (double)(err / nrm);
}

// The runtime-plan stages (fft.cuh) used by the general kernels: the same transform
// through stage_load / stage_compute / stage_store with the radix known only at run
// time, EPT = 16 (L = 2^a) or 12 (L = 3 * 2^a); the inverse runs the reversed plan.
template <typename V, int EPT, bool INV>
double general_max_rel_err(int L, const std::vector<int>& radices) {
    using T = typename real_of<V>::type;
    const int G = L / EPT;
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<V> tw(L), buf(padded_len(L));
    for (int m = 0; m < L; m++) {
        const long double a = -2.0L * pi * m / L;
        tw[m] = mk((T)std::cos(a), (T)std::sin(a));
    }
    std::vector<std::complex<long double>> in(L);
    unsigned s = 19790101u + (unsigned)L;
    for (int i = 0; i < L; i++) {
        s = s * 1103515245u + 12345u;
        const double a = (s >> 8) / 16777216.0 - 0.5;
        s = s * 1103515245u + 12345u;
        const double b = (s >> 8) / 16777216.0 - 0.5;
        in[i] = {(long double)(T)a, (long double)(T)b};
        buf[pidx(i)] = mk((T)a, (T)b);
    }
    std::vector<std::array<V, EPT>> x(G);
    using Regs = V[EPT];
    int Ns = 1;
    for (size_t st = 0; st < radices.size(); st++) {
        const int R = INV ? radices[radices.size() - 1 - st] : radices[st];
        for (int t = 0; t < G; t++) load_any<V, EPT>(R, buf.data(), *reinterpret_cast<Regs*>(x[t].data()), L, t, G);
        for (int t = 0; t < G; t++) {
            compute_any<V, EPT, INV>(R, *reinterpret_cast<Regs*>(x[t].data()), L, Ns, t, G, tw.data());
            store_any<V, EPT>(R, buf.data(), *reinterpret_cast<const Regs*>(x[t].data()), L, Ns, t, G);
        }
        Ns *= R;
    }
    long double err = 0, nrm = 0;
    for (int k = 0; k < L; k++) {
        std::complex<long double> acc = 0;
        for (int j = 0; j < L; j++) {
            const long double a = (INV ? 2.0L : -2.0L) * pi * (long double)((long)j * k % L) / L;
            acc += in[j] * std::complex<long double>(std::cos(a), std::sin(a));
        }
        const V v = buf[pidx(k)];
        err = std::max(err, std::abs(std::complex<long double>(v.x, v.y) - acc));
        nrm = std::max(nrm, std::abs(acc));
    }
    return (double)(err / nrm);
}

template <int EPT> void report_general(int L, const std::vector<int>& radices) {
    std::printf("gen%d fwd f64 %.3e\n", L, general_max_rel_err<double2, EPT, false>(L, radices));
    std::printf("gen%d inv f64 %.3e\n", L, general_max_rel_err<double2, EPT, true>(L, radices));
    std::printf("gen%d fwd f32 %.3e\n", L, general_max_rel_err<float2, EPT, false>(L, radices));
    std::printf("gen%d inv f32 %.3e\n", L, general_max_rel_err<float2, EPT, true>(L, radices));
}

template <int L> void report() {
    std::printf("%d fwd f64 %.3e\n", L, max_rel_err<double2, L, false>());
    std::printf("%d inv f64 %.3e\n", L, max_rel_err<double2, L, true>());
    std::printf("%d fwd f32 %.3e\n", L, max_rel_err<float2, L, false>());
    std::printf("%d inv f32 %.3e\n", L, max_rel_err<float2, L, true>());
}

int main() {
    report<256>();
    report<512>();
    report<1024>();
    report<2048>();
    report<4096>();
    // the plans of the runtime planner: radix <= 16 for 2^a; a leading radix 3 and
    // radices <= 4 for 3 * 2^a; stages balanced
    report_general<16>(16, {16});
    report_general<16>(32, {8, 4});
    report_general<16>(64, {8, 8});
    report_general<16>(128, {16, 8});
    report_general<16>(512, {8, 8, 8});
    report_general<16>(1024, {16, 8, 8});
    report_general<12>(24, {3, 4, 2});
    report_general<12>(48, {3, 4, 4});
    report_general<12>(96, {3, 4, 4, 2});
    report_general<12>(192, {3, 4, 4, 4});
    report_general<12>(384, {3, 4, 4, 4, 2});
    report_general<12>(768, {3, 4, 4, 4, 4});
    report_general<12>(1536, {3, 4, 4, 4, 4, 2});
    return 0;
}
