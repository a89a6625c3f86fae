// Host run of the small dense FP64 routines of the deflation eigensolver
// (small_dense.cuh): Hessenberg reduction, shifted QR to Schur form, reordering by
// decreasing |T_ii|, and the Gauss-Jordan inverse, on seeded matrices.  Prints, per case,
//   case <name> <n> <rc> <unitarity> <below-diagonal> <reconstruction> <sorted> <inverse>
// (errors relative to max |B_ij|), then the matrix ("b i j re im") and the diagonal of T
// ("t i re im"), for the eigenvalue comparison done by the Python side.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../paper_1104_4263_gb300/csrc/small_dense.cuh"

using namespace die::sd;

static unsigned g_state = 1;
static double uniform() {                      // fixed LCG in [-0.5, 0.5)
    g_state = g_state * 1103515245u + 12345u;
    return (g_state >> 8) / 16777216.0 - 0.5;
}

static std::vector<cd> matrix(const char* kind, int n, unsigned seed) {
    g_state = seed;
    std::vector<cd> B((size_t)n * n);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) B[(size_t)j * n + i] = c_(uniform(), uniform());
    if (std::string(kind) == "upper") {        // already triangular: eigenvalues on the diagonal
        for (int j = 0; j < n; j++)
            for (int i = j + 1; i < n; i++) B[(size_t)j * n + i] = c_(0, 0);
    } else if (std::string(kind) == "shifted") {   // eigenvalues clustered away from 0 (as in T = V* A V)
        for (int i = 0; i < n; i++) B[(size_t)i * n + i] = B[(size_t)i * n + i] + c_(3.0 + 0.1 * i, 0.5);
    }
    return B;
}

static void run(const char* name, const char* kind, int n, unsigned seed) {
    const std::vector<cd> B = matrix(kind, n, seed);
    std::vector<cd> T = B, Z((size_t)n * n, c_(0, 0)), work(n);
    for (int i = 0; i < n; i++) Z[(size_t)i * n + i] = c_(1, 0);
    hessenberg(T.data(), n, Z.data(), n, n, work.data());
    const int rc = schur_qr(T.data(), n, Z.data(), n, n, 60);
    if (rc == 0) schur_sort_desc(T.data(), n, Z.data(), n, n);
    double bmax = 0;
    for (const cd& v : B) bmax = std::max(bmax, cabs(v));
    double unit = 0, below = 0, rec = 0, inv = 0;
    int sorted = 1;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            cd s = c_(0, 0), r = c_(0, 0);
            for (int k = 0; k < n; k++) s = s + conj(Z[(size_t)i * n + k]) * Z[(size_t)j * n + k];   // (Z^* Z)_ij
            for (int k = 0; k < n; k++)
                for (int l = k; l < n; l++)
                    r = r + Z[(size_t)k * n + i] * T[(size_t)l * n + k] * conj(Z[(size_t)l * n + j]);   // (Z T Z^*)_ij
            unit = std::max(unit, cabs(s - c_(i == j ? 1.0 : 0.0, 0.0)));
            rec = std::max(rec, cabs(r - B[(size_t)j * n + i]) / bmax);
            if (i > j) below = std::max(below, cabs(T[(size_t)j * n + i]) / bmax);
        }
    for (int i = 0; i + 1 < n; i++)
        if (cabs(T[(size_t)(i + 1) * n + i + 1]) > cabs(T[(size_t)i * n + i]) * (1 + 1e-12)) sorted = 0;
    std::vector<cd> Ai = B;
    std::vector<int> piv(n);
    const int irc = invert(Ai.data(), n, n, piv.data());
    for (int i = 0; i < n && irc == 0; i++)
        for (int j = 0; j < n; j++) {
            cd s = c_(0, 0);
            for (int k = 0; k < n; k++) s = s + Ai[(size_t)k * n + i] * B[(size_t)j * n + k];   // (A^-1 B)_ij
            inv = std::max(inv, cabs(s - c_(i == j ? 1.0 : 0.0, 0.0)));
        }
    if (irc != 0) inv = -1;
    std::printf("case %s %d %d %.3e %.3e %.3e %d %.3e\n", name, n, rc, unit, below, rec, sorted, inv);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) std::printf("b %d %d %.17g %.17g\n", i, j, B[(size_t)j * n + i].re, B[(size_t)j * n + i].im);
    for (int i = 0; i < n; i++) std::printf("t %d %.17g %.17g\n", i, T[(size_t)i * n + i].re, T[(size_t)i * n + i].im);
}

int main() {
    run("one", "random", 1, 3u);
    run("two", "random", 2, 5u);
    run("random5", "random", 5, 7u);
    run("random17", "random", 17, 11u);
    run("random40", "random", 40, 13u);
    run("shifted64", "shifted", 64, 17u);
    run("upper12", "upper", 12, 19u);
    return 0;
}
