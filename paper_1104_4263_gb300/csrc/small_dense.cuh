// Small dense complex FP64 linear algebra for the deflation eigensolver (one thread;
// matrices of order <= a few hundred, column-major with leading dimension ld).
//   * Householder reduction to upper Hessenberg form, accumulating the unitary Z;
//   * single-shift complex QR iteration (Wilkinson shift, implicit bulge chase with
//     Givens rotations) to a Schur form T = Z^* B Z;
//   * reordering of the Schur form by decreasing |T_ii| (adjacent swaps);
//   * Gauss-Jordan inverse with partial pivoting.
// These are textbook algorithms (Golub & Van Loan, ch. 7) written for this library.
#pragma once

#include <math.h>

#include "common.cuh"

namespace die {
namespace sd {

struct cd {
    double re, im;
};
__host__ __device__ inline cd c_(double r, double i) { return cd{r, i}; }
__host__ __device__ inline cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__host__ __device__ inline cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__host__ __device__ inline cd operator*(cd a, cd b) { return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ inline cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
__host__ __device__ inline cd conj(cd a) { return cd{a.re, -a.im}; }
__host__ __device__ inline double cabs(cd a) { return hypot(a.re, a.im); }
__host__ __device__ inline cd cdiv(cd a, cd b) {
    // scaled division
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, d = b.re + r * b.im;
        return cd{(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    }
    const double r = b.re / b.im, d = b.im + r * b.re;
    return cd{(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
__host__ __device__ inline cd csqrt_(cd z) {
    const double m = cabs(z);
    if (m == 0.0) return cd{0, 0};
    double re = sqrt(0.5 * (m + fabs(z.re)));
    double im = 0.5 * z.im / re;
    if (z.re < 0) { const double t = fabs(im); im = z.im >= 0 ? re : -re; re = t; }
    return cd{re, im};
}

#define SD_AT(A, ld, i, j) (A)[(long)(j) * (ld) + (i)]

// Rotation G = [c s; -conj(s) c] with G [x; y] = [r; 0].
__host__ __device__ inline void givens(cd x, cd y, double& c, cd& s) {
    const double ax = cabs(x), ay = cabs(y);
    if (ay == 0.0) { c = 1.0; s = cd{0, 0}; return; }
    if (ax == 0.0) { c = 0.0; s = (1.0 / ay) * conj(y); return; }
    const double rho = hypot(ax, ay);
    c = ax / rho;
    s = (1.0 / (ax * rho)) * (x * conj(y));
}
// rows i, i+1 of A (columns c0..c1-1) <- G [row i; row i+1]
__host__ __device__ inline void rot_rows(cd* A, int ld, int i, int c0, int c1, double c, cd s) {
    for (int j = c0; j < c1; j++) {
        const cd a = SD_AT(A, ld, i, j), b = SD_AT(A, ld, i + 1, j);
        SD_AT(A, ld, i, j) = c * a + s * b;
        SD_AT(A, ld, i + 1, j) = c * b - conj(s) * a;
    }
}
// columns i, i+1 of A (rows r0..r1-1) <- [col i, col i+1] G^*
__host__ __device__ inline void rot_cols(cd* A, int ld, int i, int r0, int r1, double c, cd s) {
    for (int r = r0; r < r1; r++) {
        const cd a = SD_AT(A, ld, r, i), b = SD_AT(A, ld, r, i + 1);
        SD_AT(A, ld, r, i) = c * a + conj(s) * b;
        SD_AT(A, ld, r, i + 1) = c * b - s * a;
    }
}

// A (n x n) -> upper Hessenberg H = Z^* A Z; Z must hold a unitary matrix on entry
// (identity for a plain decomposition); it is multiplied on the right by the reflectors.
// v: workspace of n entries.
__host__ __device__ inline void hessenberg(cd* A, int lda, cd* Z, int ldz, int n, cd* v) {
    for (int k = 0; k + 2 < n; k++) {
        double xn = 0;
        for (int i = k + 1; i < n; i++) xn = hypot(xn, cabs(SD_AT(A, lda, i, k)));
        if (xn == 0.0) continue;
        const cd x0 = SD_AT(A, lda, k + 1, k);
        const double a0 = cabs(x0);
        const cd ph = a0 > 0 ? (1.0 / a0) * x0 : cd{1, 0};
        const cd alpha = (-xn) * ph;                  // reflect x onto alpha e1
        for (int i = k + 1; i < n; i++) v[i] = SD_AT(A, lda, i, k);
        v[k + 1] = v[k + 1] - alpha;
        double vn = 0;
        for (int i = k + 1; i < n; i++) vn = hypot(vn, cabs(v[i]));
        if (vn == 0.0) continue;
        for (int i = k + 1; i < n; i++) v[i] = (1.0 / vn) * v[i];
        // A <- (I - 2 v v^*) A
        for (int j = 0; j < n; j++) {
            cd d{0, 0};
            for (int i = k + 1; i < n; i++) d = d + conj(v[i]) * SD_AT(A, lda, i, j);
            for (int i = k + 1; i < n; i++) SD_AT(A, lda, i, j) = SD_AT(A, lda, i, j) - 2.0 * (v[i] * d);
        }
        // A <- A (I - 2 v v^*), Z <- Z (I - 2 v v^*)
        for (int r = 0; r < n; r++) {
            cd d{0, 0};
            for (int i = k + 1; i < n; i++) d = d + SD_AT(A, lda, r, i) * v[i];
            for (int i = k + 1; i < n; i++) SD_AT(A, lda, r, i) = SD_AT(A, lda, r, i) - 2.0 * (d * conj(v[i]));
            cd e{0, 0};
            for (int i = k + 1; i < n; i++) e = e + SD_AT(Z, ldz, r, i) * v[i];
            for (int i = k + 1; i < n; i++) SD_AT(Z, ldz, r, i) = SD_AT(Z, ldz, r, i) - 2.0 * (e * conj(v[i]));
        }
        SD_AT(A, lda, k + 1, k) = alpha;
        for (int i = k + 2; i < n; i++) SD_AT(A, lda, i, k) = cd{0, 0};
    }
}

// Upper Hessenberg H -> upper triangular Schur form, accumulating rotations into Z.
// Returns 0 on success, -1 if an eigenvalue failed to converge within maxit iterations.
__host__ __device__ inline int schur_qr(cd* H, int ldh, cd* Z, int ldz, int n, int maxit) {
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, it = 0, total = 0;
    while (hi > 0) {
        int l = hi;
        for (; l > 0; l--) {
            const double s = cabs(SD_AT(H, ldh, l - 1, l - 1)) + cabs(SD_AT(H, ldh, l, l));
            if (cabs(SD_AT(H, ldh, l, l - 1)) <= eps * (s > 0 ? s : 1.0)) { SD_AT(H, ldh, l, l - 1) = cd{0, 0}; break; }
        }
        if (l == hi) { hi--; it = 0; continue; }
        if (++total > maxit * n) return -1;
        // Wilkinson shift from the trailing 2 x 2 block of the active window
        const cd a = SD_AT(H, ldh, hi - 1, hi - 1), b = SD_AT(H, ldh, hi - 1, hi);
        const cd c = SD_AT(H, ldh, hi, hi - 1), d = SD_AT(H, ldh, hi, hi);
        cd mu;
        if (it > 0 && it % 10 == 0) {
            mu = d + c_(1.5 * cabs(c), 0.0);          // exceptional shift
        } else {
            const cd half = 0.5 * (a - d);
            const cd disc = csqrt_(half * half + b * c);
            const cd m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
            mu = cabs(m1 - d) < cabs(m2 - d) ? m1 : m2;
        }
        it++;
        cd x = SD_AT(H, ldh, l, l) - mu, y = SD_AT(H, ldh, l + 1, l);
        for (int k = l; k < hi; k++) {
            double cs;
            cd sn;
            givens(x, y, cs, sn);
            const int c0 = k > l ? k - 1 : l;
            rot_rows(H, ldh, k, c0, n, cs, sn);
            const int r1 = k + 3 < hi + 1 ? k + 3 : hi + 1;
            rot_cols(H, ldh, k, 0, r1, cs, sn);
            rot_cols(Z, ldz, k, 0, n, cs, sn);
            if (k > l) SD_AT(H, ldh, k + 1, k - 1) = cd{0, 0};
            if (k + 1 < hi) { x = SD_AT(H, ldh, k + 1, k); y = SD_AT(H, ldh, k + 2, k); }
        }
    }
    for (int j = 0; j < n; j++)
        for (int i = j + 1; i < n; i++) SD_AT(H, ldh, i, j) = cd{0, 0};
    return 0;
}

// Swap diagonal entries k and k+1 of the upper triangular T (unitary similarity), Z <- Z G^*.
__host__ __device__ inline void schur_swap(cd* T, int ldt, cd* Z, int ldz, int n, int k) {
    const cd a = SD_AT(T, ldt, k, k), b = SD_AT(T, ldt, k + 1, k + 1);
    // eigenvector of b in the 2 x 2 block: (T[k,k+1], b - a)
    double cs;
    cd sn;
    givens(SD_AT(T, ldt, k, k + 1), b - a, cs, sn);
    rot_rows(T, ldt, k, k, n, cs, sn);
    rot_cols(T, ldt, k, 0, k + 2, cs, sn);
    rot_cols(Z, ldz, k, 0, n, cs, sn);
    SD_AT(T, ldt, k + 1, k) = cd{0, 0};
    SD_AT(T, ldt, k, k) = b;
    SD_AT(T, ldt, k + 1, k + 1) = a;
}

// Order the Schur form by decreasing |T_ii| (ties keep their order).
__host__ __device__ inline void schur_sort_desc(cd* T, int ldt, cd* Z, int ldz, int n) {
    for (int i = 0; i < n; i++)
        for (int k = n - 2; k >= i; k--)
            if (cabs(SD_AT(T, ldt, k + 1, k + 1)) > cabs(SD_AT(T, ldt, k, k))) schur_swap(T, ldt, Z, ldz, n, k);
}

// In-place inverse of A (n x n) by Gauss-Jordan with partial pivoting.  piv: n ints.
// Returns 0, or -1 when a pivot is zero (singular).
__host__ __device__ inline int invert(cd* A, int lda, int n, int* piv) {
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = cabs(SD_AT(A, lda, k, k));
        for (int i = k + 1; i < n; i++) {
            const double v = cabs(SD_AT(A, lda, i, k));
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k)
            for (int j = 0; j < n; j++) { const cd t = SD_AT(A, lda, k, j); SD_AT(A, lda, k, j) = SD_AT(A, lda, p, j); SD_AT(A, lda, p, j) = t; }
        const cd inv = cdiv(c_(1, 0), SD_AT(A, lda, k, k));
        SD_AT(A, lda, k, k) = c_(1, 0);
        for (int j = 0; j < n; j++) SD_AT(A, lda, k, j) = SD_AT(A, lda, k, j) * inv;
        for (int i = 0; i < n; i++) {
            if (i == k) continue;
            const cd f = SD_AT(A, lda, i, k);
            if (f.re == 0.0 && f.im == 0.0) continue;
            SD_AT(A, lda, i, k) = c_(0, 0);
            for (int j = 0; j < n; j++) SD_AT(A, lda, i, j) = SD_AT(A, lda, i, j) - f * SD_AT(A, lda, k, j);
        }
    }
    for (int k = n - 1; k >= 0; k--) {
        const int p = piv[k];
        if (p != k)
            for (int i = 0; i < n; i++) { const cd t = SD_AT(A, lda, i, k); SD_AT(A, lda, i, k) = SD_AT(A, lda, i, p); SD_AT(A, lda, i, p) = t; }
    }
    return 0;
}

#undef SD_AT

}  // namespace sd
}  // namespace die
