// Host run of the GMRES Givens step (krylov.cuh: givens_column), the arithmetic of the
// device kernel that turns the Hessenberg matrix of each Arnoldi step into R and rotates
// beta e1.  Seeded complex upper Hessenberg matrices H ((m+1) x m, real non-negative
// subdiagonal as Arnoldi produces) are processed column by column.  Prints, per case,
//   case <name> <m> <beta>          then  h <i> <j> <re> <im>   (H)
//   est <j> <|g[j+1]|>              (least-squares residual after j + 1 steps)
//   r <i> <j> <re> <im>             (R, upper triangular m x m)   and   g <i> <re> <im>
#include <cmath>
#include <cstdio>
#include <vector>

#include "../paper_1104_4263_gb300/csrc/krylov.cuh"

using die::givens_column;

static unsigned g_state = 1;
static double uniform() {
    g_state = g_state * 1103515245u + 12345u;
    return (g_state >> 8) / 16777216.0 - 0.5;
}

static void run(const char* name, int m, double beta, unsigned seed, int zero_col) {
    g_state = seed;
    std::vector<double2> H((size_t)(m + 1) * m, make_double2(0, 0));   // column-major, ld = m + 1
    for (int j = 0; j < m; j++) {
        for (int i = 0; i <= j; i++) H[(size_t)j * (m + 1) + i] = make_double2(uniform(), uniform());
        H[(size_t)j * (m + 1) + j + 1] = make_double2(std::fabs(uniform()) + 0.05, 0.0);
    }
    if (zero_col >= 0)          // a column whose diagonal entry after rotation may vanish
        for (int i = 0; i <= zero_col; i++) H[(size_t)zero_col * (m + 1) + i] = make_double2(0, 0);
    std::printf("case %s %d %.17g\n", name, m, beta);
    for (int j = 0; j < m; j++)
        for (int i = 0; i <= j + 1; i++)
            std::printf("h %d %d %.17g %.17g\n", i, j, H[(size_t)j * (m + 1) + i].x, H[(size_t)j * (m + 1) + i].y);
    std::vector<double2> cs(m), sn(m), g(m + 1, make_double2(0, 0)), R((size_t)m * m, make_double2(0, 0));
    std::vector<double2> col(m + 2);
    g[0] = make_double2(beta, 0.0);
    for (int j = 0; j < m; j++) {
        for (int i = 0; i <= j; i++) col[i] = H[(size_t)j * (m + 1) + i];
        givens_column(col.data(), cs.data(), sn.data(), j, H[(size_t)j * (m + 1) + j + 1].x, &cs[j], &sn[j], g.data());
        std::printf("est %d %.17g\n", j, std::hypot(g[j + 1].x, g[j + 1].y));
        for (int i = 0; i <= j; i++) R[(size_t)j * m + i] = col[i];
    }
    for (int j = 0; j < m; j++)
        for (int i = 0; i <= j; i++) std::printf("r %d %d %.17g %.17g\n", i, j, R[(size_t)j * m + i].x, R[(size_t)j * m + i].y);
    for (int i = 0; i <= m; i++) std::printf("g %d %.17g %.17g\n", i, g[i].x, g[i].y);
}

int main() {
    run("m1", 1, 1.0, 3u, -1);
    run("m5", 5, 2.5, 7u, -1);
    run("m30", 30, 1.0, 11u, -1);
    run("m64", 64, 0.3, 13u, -1);
    run("zero_column", 12, 1.0, 17u, 0);
    return 0;
}
