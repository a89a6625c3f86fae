// Fourier neural operator forward and backward passes (see include/die_fno.h) as chains
// of tcgen05 BF16 GEMMs (tc_gemm.cuh) and small FP32 elementwise kernels.
//
// Spectral convolution of one layer, for activations h[b][c][y][x] (B x C x H x W),
// m modes, MH = 2 m kept frequencies along y (k_h = 0 .. m-1 and H-m .. H-1, index
// khi), m along x (k_w), NM = MH m modes in all:
//   1  T1[bc][n][y]  = sum_x h[bc][y][x] Fw[n][x]        n = 2 k_w + ri (ri: re / im)
//   2  Z2[bc][k_w][n] = sum_{k=(ri,y)} T1[bc][2 k_w + ri][y] Gh[n][k]   n = 2 khi + ri'
//   3  Zmix[mode][b][ri c]  <- Z2 (shuffle; mode = khi m + k_w)
//   4  Ymix[mode][b][n] = sum_k Zmix[mode][b][k] Rr[mode][n][k]   (the complex channel
//      mixing Y = X R as a real 2C x 2C matrix per mode)
//   5  Y2[bo][k_w][ri khi]  <- Ymix (shuffle)
//   6  T3[bo][y][ri'][k_w] = sum_k Y2[bo][k_w][k] Ginv[2 y + ri'][k]
//   7  out[bo][y][x] += sum_{k=(ri',k_w)} T3[bo][y][k] Fwinv[x][k]
// with Fw, Gh the forward real DFT along x and complex DFT along y restricted to the kept
// modes, Ginv, Fwinv the inverse ones (Fwinv carries c(k_w) / (H W), c = 1 at k_w = 0 and
// 2 otherwise: the inverse real DFT of a half spectrum).  The backward pass runs the
// transposed GEMMs in reverse order; dR comes from dRr = dYmix^T Zmix per mode.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/die_fno.h"
#include "op.cuh"
#include "tc_gemm.cuh"

struct fno_s {
    fno_desc d{};
    int C = 0, H = 0, W = 0, m = 0, MH = 0, NM = 0, HW = 0, L = 0, hid = 0, cin = 0, cout = 0, maxB = 0;
    long np = 0;
    long oP = 0, op = 0, oW[8] = {}, ow[8] = {}, oR1[8] = {}, oR2[8] = {}, oQ1 = 0, oq1 = 0, oQ2 = 0, oq2 = 0;
    float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
    long adam_t = 0;
    float *Fw = nullptr, *Gh = nullptr, *Ginv = nullptr, *Fwinv = nullptr;
    float* Rr = nullptr;            // L x NM x (2C)^2
    float* dRr = nullptr;           // NM x (2C)^2
    float* x = nullptr;             // input copy   B x cin x HW
    float* h[9] = {};               // h_0 .. h_{L-1}: B x C x HW (h_L = a_{L-1})
    float* a[8] = {};               // pre-activations
    float *u = nullptr, *s = nullptr;   // B x hid x HW
    float *T1 = nullptr, *Z2 = nullptr, *Ymix = nullptr, *Y2 = nullptr, *T3 = nullptr;
    float* Zmix[8] = {};            // kept for dR
    float *g1 = nullptr, *g2 = nullptr, *g3 = nullptr;   // backward scratch B x max(C, hid) x HW
    float* part = nullptr;          // per-batch weight-gradient partials
    float* loss = nullptr;          // device scalar
    float* ytmp = nullptr;          // B x cout x HW (train step)
    float *pin = nullptr, *pout = nullptr;   // preconditioner staging (1 x cin / cout x HW)
    double* rs = nullptr;           // preconditioner: sum of |v|^2 (device)
    int* err = nullptr;
    float* hostbuf = nullptr;
    int lastB = 0;
};

namespace die {
namespace {

constexpr int kT = 256;
inline int blocks_for(long n) {
    long b = (n + kT - 1) / kT;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

// ------------------------------------------------------------------ elementwise kernels
__device__ __forceinline__ float gelu_f(float v) { return v * normcdff(v); }
__device__ __forceinline__ float gelu_d(float v) {
    return normcdff(v) + v * 0.3989422804014327f * __expf(-0.5f * v * v);
}

__global__ void gelu_kernel(const float* a, float* h, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        h[i] = gelu_f(a[i]);
}
// d *= GELU'(a)
__global__ void gelu_back_kernel(const float* a, float* d, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        d[i] *= gelu_d(a[i]);
}

// grads[c] += sum_{b, p} d[b][c][p]   (one block per channel, fixed order)
__global__ void chan_sum_kernel(const float* d, int B, int C, int HW, float* g) {
    __shared__ float red[kT];
    const int c = blockIdx.x;
    float acc = 0.f;
    for (int b = 0; b < B; b++)
        for (int p = threadIdx.x; p < HW; p += blockDim.x) acc += d[((long)b * C + c) * HW + p];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) g[c] += red[0];
}

// g[e] += sum_b part[b][e]
__global__ void batch_sum_kernel(const float* part, int B, long n, float* g) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int b = 0; b < B; b++) acc += part[(long)b * n + e];
        g[e] += acc;
    }
}

// Shuffle 3 (and its transpose): Zmix[mode][b][ri C + c] <-> Z2[b C + c][k_w][2 khi + ri].
__global__ void shuffle_z_kernel(float* Z2, float* Zmix, int B, int C, int m, int MH, int back) {
    const long n = (long)B * C * m * 2 * MH;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        // e enumerates Z2: ((b C + c) m + kw) (2 MH) + 2 khi + ri
        const int q = (int)(e % (2 * MH));
        long t = e / (2 * MH);
        const int kw = (int)(t % m);
        t /= m;
        const int c = (int)(t % C), b = (int)(t / C);
        const int khi = q >> 1, ri = q & 1;
        const long z = (((long)(khi * m + kw) * B + b) * 2 + ri) * C + c;
        if (back) Z2[e] = Zmix[z];
        else Zmix[z] = Z2[e];
    }
}

// Shuffle 5 (and its transpose): Ymix[mode][b][ri C + o] <-> Y2[b C + o][k_w][ri MH + khi].
__global__ void shuffle_y_kernel(float* Ymix, float* Y2, int B, int C, int m, int MH, int back) {
    const long n = (long)B * C * m * 2 * MH;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        // e enumerates Y2: ((b C + o) m + kw) (2 MH) + ri MH + khi
        const int q = (int)(e % (2 * MH));
        long t = e / (2 * MH);
        const int kw = (int)(t % m);
        t /= m;
        const int o = (int)(t % C), b = (int)(t / C);
        const int ri = q / MH, khi = q % MH;
        const long y = (((long)(khi * m + kw) * B + b) * 2 + ri) * C + o;
        if (back) Ymix[y] = Y2[e];
        else Y2[e] = Ymix[y];
    }
}

// Real 2C x 2C mixing matrix of every mode from the complex weights R1 / R2 (layout
// [i][o][kh][kw] (re, im)): Rr[mode][ri' C + o][ri C + i] such that
// Yre = sum_i Zre Rre - Zim Rim, Yim = sum_i Zre Rim + Zim Rre.
__global__ void expand_r_kernel(const float* R1, const float* R2, float* Rr, int C, int m, int MH) {
    const int C2 = 2 * C;
    const long n = (long)MH * m * C2 * C2;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int k = (int)(e % C2);
        const int nn = (int)((e / C2) % C2);
        const int mode = (int)(e / ((long)C2 * C2));
        const int khi = mode / m, kw = mode % m;
        const int ri = k / C, i = k % C, rio = nn / C, o = nn % C;
        const float* R = khi < m ? R1 : R2;
        const int kh = khi < m ? khi : khi - m;
        const long idx = 2 * ((((long)i * C + o) * m + kh) * m + kw);
        const float re = R[idx], im = R[idx + 1];
        float v;
        if (rio == 0) v = ri == 0 ? re : -im;
        else v = ri == 0 ? im : re;
        Rr[e] = v;
    }
}

// dR1 / dR2 += fold of dRr (the adjoint of expand_r_kernel).
__global__ void fold_r_kernel(const float* dRr, float* dR1, float* dR2, int C, int m, int MH) {
    const int C2 = 2 * C;
    const long n = (long)C * C * MH * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        // e enumerates (i, o, khi, kw) with kw fastest
        const int kw = (int)(e % m);
        long t = e / m;
        const int khi = (int)(t % MH);
        t /= MH;
        const int o = (int)(t % C), i = (int)(t / C);
        const float* D = dRr + (long)(khi * m + kw) * C2 * C2;
        const float dre = D[(long)o * C2 + i] + D[(long)(C + o) * C2 + C + i];
        const float dim = -D[(long)o * C2 + C + i] + D[(long)(C + o) * C2 + i];
        float* G = khi < m ? dR1 : dR2;
        const int kh = khi < m ? khi : khi - m;
        const long idx = 2 * ((((long)i * C + o) * m + kh) * m + kw);
        G[idx] += dre;
        G[idx + 1] += dim;
    }
}

// loss = mean (y - t)^2 (single block, fixed order), g = 2 (y - t) / n
__global__ void mse_kernel(const float* y, const float* t, long n, float* g, float* loss) {
    __shared__ float red[kT];
    float acc = 0.f;
    const float sc = 2.f / (float)n;
    for (long i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = y[i] - t[i];
        acc += d * d;
        g[i] = sc * d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (float)n;
}

__global__ void adam_kernel(float* p, const float* g, float* m1, float* m2, long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

// --------------------------------------------------------------- preconditioner glue
// sum of |v|^2 over n complex128 entries into *out (one block, fixed order)
__global__ void sumsq_kernel(const double2* v, long n, double* out) {
    __shared__ double red[kT];
    double acc = 0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) acc += v[i].x * v[i].x + v[i].y * v[i].y;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// x[6][HW] = (Re chi, Im chi, Re v1 / s, Im v1 / s, Re v2 / s, Im v2 / s), s = rms(v)
__global__ void encode_kernel(const double2* chi, const double2* v, const double* ss, long N, float* x) {
    const double s2 = *ss / (2.0 * N);
    const double inv = s2 > 0 ? 1.0 / sqrt(s2) : 1.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const double2 c = chi[i], a = v[i], b = v[N + i];
        x[i] = (float)c.x;
        x[N + i] = (float)c.y;
        x[2 * N + i] = (float)(a.x * inv);
        x[3 * N + i] = (float)(a.y * inv);
        x[4 * N + i] = (float)(b.x * inv);
        x[5 * N + i] = (float)(b.y * inv);
    }
}

// t[4][N] = (u - b) / s, s = rms(b)
__global__ void target_kernel(const double2* b, const double2* u, const double* ss, long N, float* t) {
    const double s2 = *ss / (2.0 * N);
    const double inv = s2 > 0 ? 1.0 / sqrt(s2) : 1.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const double2 a = b[i], c = b[N + i], ua = u[i], uc = u[N + i];
        t[i] = (float)((ua.x - a.x) * inv);
        t[N + i] = (float)((ua.y - a.y) * inv);
        t[2 * N + i] = (float)((uc.x - c.x) * inv);
        t[3 * N + i] = (float)((uc.y - c.y) * inv);
    }
}

// z = v + s d, d = (y0 + i y1, y2 + i y3)
__global__ void decode_kernel(const double2* v, const float* y, const double* ss, long N, double2* z) {
    const double s2 = *ss / (2.0 * N);
    const double s = s2 > 0 ? sqrt(s2) : 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const double2 a = v[i], b = v[N + i];
        z[i] = make_double2(a.x + s * y[i], a.y + s * y[N + i]);
        z[N + i] = make_double2(b.x + s * y[2 * N + i], b.y + s * y[3 * N + i]);
    }
}

// ------------------------------------------------------------------ GEMM shorthand
struct Mat {
    const float* p;
    long s0, s1, sb;     // strides of the first index (m or n), of k, of the batch
};

die_status gemm(int M, int N, int K, int batch, Mat A, Mat B, float* C, long scm, long scn, long scb, float beta,
                const float* bias, int* err, cudaStream_t st) {
    GemmArgs g;
    g.M = M; g.N = N; g.K = K; g.batch = batch;
    g.A = A.p; g.sam = A.s0; g.sak = A.s1; g.sab = A.sb;
    g.B = B.p; g.sbn = B.s0; g.sbk = B.s1; g.sbb = B.sb;
    g.C = C; g.scm = scm; g.scn = scn; g.scb = scb;
    g.alpha = 1.f; g.beta = beta; g.bias = bias; g.err = err;
    return tc_gemm(g, st);
}

// ------------------------------------------------------------------ network passes
// a = W h + w (pointwise) + K h (spectral) for layer l; Zmix[l] kept.
die_status layer_forward(fno_s* f, int l, int B, const float* hin, float* a, cudaStream_t st) {
    const int C = f->C, H = f->H, W = f->W, m = f->m, MH = f->MH, HW = f->HW, C2 = 2 * C;
    const long CHW = (long)C * HW;
    float* prm = f->params;
    // pointwise
    DIE_TRY(gemm(HW, C, C, B, {hin, 1, HW, CHW}, {prm + f->oW[l], C, 1, 0}, a, 1, HW, CHW, 0.f, prm + f->ow[l],
                 f->err, st));
    // 1: along x
    DIE_TRY(gemm(H, 2 * m, W, B * C, {hin, W, 1, HW}, {f->Fw, W, 1, 0}, f->T1, 1, H, 2L * m * H, 0.f, nullptr,
                 f->err, st));
    // 2: along y
    DIE_TRY(gemm(m, 2 * MH, 2 * H, B * C, {f->T1, 2L * H, 1, 2L * m * H}, {f->Gh, 2L * H, 1, 0}, f->Z2, 2L * MH, 1,
                 2L * m * MH, 0.f, nullptr, f->err, st));
    // 3
    shuffle_z_kernel<<<blocks_for((long)B * C * m * 2 * MH), kT, 0, st>>>(f->Z2, f->Zmix[l], B, C, m, MH, 0);
    DIE_LAUNCH_CHECK();
    // 4: channel mixing per mode
    DIE_TRY(gemm(B, C2, C2, f->NM, {f->Zmix[l], C2, 1, (long)B * C2}, {f->Rr + (long)l * f->NM * C2 * C2, C2, 1,
                 (long)C2 * C2}, f->Ymix, C2, 1, (long)B * C2, 0.f, nullptr, f->err, st));
    // 5
    shuffle_y_kernel<<<blocks_for((long)B * C * m * 2 * MH), kT, 0, st>>>(f->Ymix, f->Y2, B, C, m, MH, 0);
    DIE_LAUNCH_CHECK();
    // 6: inverse along y
    DIE_TRY(gemm(m, 2 * H, 2 * MH, B * C, {f->Y2, 2L * MH, 1, 2L * m * MH}, {f->Ginv, 2L * MH, 1, 0}, f->T3, 1, m,
                 2L * H * m, 0.f, nullptr, f->err, st));
    // 7: inverse along x, added to the pointwise part
    DIE_TRY(gemm(H, W, 2 * m, B * C, {f->T3, 2L * m, 1, 2L * H * m}, {f->Fwinv, 2L * m, 1, 0}, a, W, 1, HW, 1.f,
                 nullptr, f->err, st));
    return DIE_OK;
}

// Backward of layer l given da (B x C x HW; overwritten as scratch is not needed):
// grads of W_l, w_l, R1_l, R2_l accumulated, dh (B x C x HW) written.
die_status layer_backward(fno_s* f, int l, int B, const float* hin, const float* da, float* dh, cudaStream_t st) {
    const int C = f->C, H = f->H, W = f->W, m = f->m, MH = f->MH, HW = f->HW, C2 = 2 * C;
    const long CHW = (long)C * HW;
    float* prm = f->params;
    float* grd = f->grads;
    // dW = sum_b da h^T (per-batch partials), dw = channel sums
    DIE_TRY(gemm(C, C, HW, B, {da, HW, 1, CHW}, {hin, HW, 1, CHW}, f->part, C, 1, (long)C * C, 0.f, nullptr, f->err,
                 st));
    batch_sum_kernel<<<blocks_for((long)C * C), kT, 0, st>>>(f->part, B, (long)C * C, grd + f->oW[l]);
    DIE_LAUNCH_CHECK();
    chan_sum_kernel<<<C, kT, 0, st>>>(da, B, C, HW, grd + f->ow[l]);
    DIE_LAUNCH_CHECK();
    // dh = W^T da
    DIE_TRY(gemm(HW, C, C, B, {da, 1, HW, CHW}, {prm + f->oW[l], 1, C, 0}, dh, 1, HW, CHW, 0.f, nullptr, f->err, st));
    // spectral, 7^T: dT3 = da Fwinv
    DIE_TRY(gemm(H, 2 * m, W, B * C, {da, W, 1, HW}, {f->Fwinv, 1, 2L * m, 0}, f->T3, 2L * m, 1, 2L * H * m, 0.f,
                 nullptr, f->err, st));
    // 6^T: dY2 = dT3 Ginv
    DIE_TRY(gemm(m, 2 * MH, 2 * H, B * C, {f->T3, 1, m, 2L * H * m}, {f->Ginv, 1, 2L * MH, 0}, f->Y2, 2L * MH, 1,
                 2L * m * MH, 0.f, nullptr, f->err, st));
    // 5^T
    shuffle_y_kernel<<<blocks_for((long)B * C * m * 2 * MH), kT, 0, st>>>(f->Ymix, f->Y2, B, C, m, MH, 1);
    DIE_LAUNCH_CHECK();
    // 4^T: dRr = dYmix^T Zmix, dZmix = dYmix Rr
    DIE_TRY(gemm(C2, C2, B, f->NM, {f->Ymix, 1, C2, (long)B * C2}, {f->Zmix[l], 1, C2, (long)B * C2}, f->dRr, C2, 1,
                 (long)C2 * C2, 0.f, nullptr, f->err, st));
    fold_r_kernel<<<blocks_for((long)C * C * MH * m), kT, 0, st>>>(f->dRr, grd + f->oR1[l], grd + f->oR2[l], C, m, MH);
    DIE_LAUNCH_CHECK();
    DIE_TRY(gemm(B, C2, C2, f->NM, {f->Ymix, C2, 1, (long)B * C2},
                 {f->Rr + (long)l * f->NM * C2 * C2, 1, C2, (long)C2 * C2}, f->Zmix[l], C2, 1, (long)B * C2, 0.f,
                 nullptr, f->err, st));
    // 3^T
    shuffle_z_kernel<<<blocks_for((long)B * C * m * 2 * MH), kT, 0, st>>>(f->Z2, f->Zmix[l], B, C, m, MH, 1);
    DIE_LAUNCH_CHECK();
    // 2^T: dT1 = dZ2 Gh
    DIE_TRY(gemm(m, 2 * H, 2 * MH, B * C, {f->Z2, 2L * MH, 1, 2L * m * MH}, {f->Gh, 1, 2L * H, 0}, f->T1, 2L * H, 1,
                 2L * m * H, 0.f, nullptr, f->err, st));
    // 1^T: dh += dT1 Fw
    DIE_TRY(gemm(H, W, 2 * m, B * C, {f->T1, 1, H, 2L * m * H}, {f->Fw, 1, W, 0}, dh, W, 1, HW, 1.f, nullptr, f->err,
                 st));
    return DIE_OK;
}

die_status expand_weights(fno_s* f, cudaStream_t st) {
    const long per = (long)f->NM * 4 * f->C * f->C;
    for (int l = 0; l < f->L; l++) {
        expand_r_kernel<<<blocks_for(per), kT, 0, st>>>(f->params + f->oR1[l], f->params + f->oR2[l],
                                                        f->Rr + (long)l * per, f->C, f->m, f->MH);
        DIE_LAUNCH_CHECK();
    }
    return DIE_OK;
}

die_status forward(fno_s* f, int B, const float* x, float* y, cudaStream_t st) {
    const int C = f->C, HW = f->HW;
    const long CHW = (long)C * HW, HHW = (long)f->hid * HW;
    float* prm = f->params;
    DIE_TRY(expand_weights(f, st));
    DIE_CUDA_TRY(cudaMemcpyAsync(f->x, x, (size_t)B * f->cin * HW * sizeof(float), cudaMemcpyDeviceToDevice, st));
    // lifting
    DIE_TRY(gemm(HW, C, f->cin, B, {f->x, 1, HW, (long)f->cin * HW}, {prm + f->oP, f->cin, 1, 0}, f->h[0], 1, HW,
                 CHW, 0.f, prm + f->op, f->err, st));
    for (int l = 0; l < f->L; l++) {
        DIE_TRY(layer_forward(f, l, B, f->h[l], f->a[l], st));
        if (l < f->L - 1) {
            gelu_kernel<<<blocks_for(B * CHW), kT, 0, st>>>(f->a[l], f->h[l + 1], B * CHW);
            DIE_LAUNCH_CHECK();
        }
    }
    const float* hL = f->a[f->L - 1];
    DIE_TRY(gemm(HW, f->hid, C, B, {hL, 1, HW, CHW}, {prm + f->oQ1, C, 1, 0}, f->u, 1, HW, HHW, 0.f, prm + f->oq1,
                 f->err, st));
    gelu_kernel<<<blocks_for(B * HHW), kT, 0, st>>>(f->u, f->s, B * HHW);
    DIE_LAUNCH_CHECK();
    DIE_TRY(gemm(HW, f->cout, f->hid, B, {f->s, 1, HW, HHW}, {prm + f->oQ2, f->hid, 1, 0}, y, 1, HW,
                 (long)f->cout * HW, 0.f, prm + f->oq2, f->err, st));
    f->lastB = B;
    return DIE_OK;
}

die_status backward(fno_s* f, int B, const float* gy, float* gx, cudaStream_t st) {
    const int C = f->C, HW = f->HW, hid = f->hid;
    const long CHW = (long)C * HW, HHW = (long)hid * HW;
    float* prm = f->params;
    float* grd = f->grads;
    // projection: dQ2, dq2, ds
    DIE_TRY(gemm(f->cout, hid, HW, B, {gy, HW, 1, (long)f->cout * HW}, {f->s, HW, 1, HHW}, f->part, hid, 1,
                 (long)f->cout * hid, 0.f, nullptr, f->err, st));
    batch_sum_kernel<<<blocks_for((long)f->cout * hid), kT, 0, st>>>(f->part, B, (long)f->cout * hid, grd + f->oQ2);
    DIE_LAUNCH_CHECK();
    chan_sum_kernel<<<f->cout, kT, 0, st>>>(gy, B, f->cout, HW, grd + f->oq2);
    DIE_LAUNCH_CHECK();
    DIE_TRY(gemm(HW, hid, f->cout, B, {gy, 1, HW, (long)f->cout * HW}, {prm + f->oQ2, 1, hid, 0}, f->g3, 1, HW, HHW,
                 0.f, nullptr, f->err, st));
    gelu_back_kernel<<<blocks_for(B * HHW), kT, 0, st>>>(f->u, f->g3, B * HHW);
    DIE_LAUNCH_CHECK();
    const float* hL = f->a[f->L - 1];
    DIE_TRY(gemm(hid, C, HW, B, {f->g3, HW, 1, HHW}, {hL, HW, 1, CHW}, f->part, C, 1, (long)hid * C, 0.f, nullptr,
                 f->err, st));
    batch_sum_kernel<<<blocks_for((long)hid * C), kT, 0, st>>>(f->part, B, (long)hid * C, grd + f->oQ1);
    DIE_LAUNCH_CHECK();
    chan_sum_kernel<<<hid, kT, 0, st>>>(f->g3, B, hid, HW, grd + f->oq1);
    DIE_LAUNCH_CHECK();
    float* dh = f->g1;   // gradient w.r.t. the current h
    float* da = f->g2;
    DIE_TRY(gemm(HW, C, hid, B, {f->g3, 1, HW, HHW}, {prm + f->oQ1, 1, C, 0}, dh, 1, HW, CHW, 0.f, nullptr, f->err,
                 st));
    for (int l = f->L - 1; l >= 0; l--) {
        // da = dh (last layer) or dh * GELU'(a_l)
        DIE_CUDA_TRY(cudaMemcpyAsync(da, dh, (size_t)B * CHW * sizeof(float), cudaMemcpyDeviceToDevice, st));
        if (l < f->L - 1) {
            gelu_back_kernel<<<blocks_for(B * CHW), kT, 0, st>>>(f->a[l], da, B * CHW);
            DIE_LAUNCH_CHECK();
        }
        DIE_TRY(layer_backward(f, l, B, f->h[l], da, dh, st));
    }
    // lifting
    DIE_TRY(gemm(C, f->cin, HW, B, {dh, HW, 1, CHW}, {f->x, HW, 1, (long)f->cin * HW}, f->part, f->cin, 1,
                 (long)C * f->cin, 0.f, nullptr, f->err, st));
    batch_sum_kernel<<<blocks_for((long)C * f->cin), kT, 0, st>>>(f->part, B, (long)C * f->cin, grd + f->oP);
    DIE_LAUNCH_CHECK();
    chan_sum_kernel<<<C, kT, 0, st>>>(dh, B, C, HW, grd + f->op);
    DIE_LAUNCH_CHECK();
    if (gx)
        DIE_TRY(gemm(HW, f->cin, C, B, {dh, 1, HW, CHW}, {prm + f->oP, 1, f->cin, 0}, gx, 1, HW, (long)f->cin * HW,
                     0.f, nullptr, f->err, st));
    return DIE_OK;
}

// Constant DFT matrices (FP64 on the host, stored FP32).
die_status make_dft(fno_s* f) {
    const int H = f->H, W = f->W, m = f->m, MH = f->MH;
    const double tp = 2.0 * M_PI;
    std::vector<float> Fw((size_t)2 * m * W), Gh((size_t)2 * MH * 2 * H), Gi((size_t)2 * H * 2 * MH),
        Fi((size_t)W * 2 * m);
    for (int kw = 0; kw < m; kw++)
        for (int x = 0; x < W; x++) {
            const double ph = tp * (double)((long)kw * x % W) / W;
            Fw[(size_t)(2 * kw) * W + x] = (float)cos(ph);
            Fw[(size_t)(2 * kw + 1) * W + x] = (float)-sin(ph);
            const double c = (kw == 0 ? 1.0 : 2.0) / ((double)H * W);
            Fi[(size_t)x * 2 * m + kw] = (float)(c * cos(ph));
            Fi[(size_t)x * 2 * m + m + kw] = (float)(-c * sin(ph));
        }
    for (int khi = 0; khi < MH; khi++) {
        const int kh = khi < m ? khi : H - MH + khi;
        for (int y = 0; y < H; y++) {
            const double th = tp * (double)((long)kh * y % H) / H;
            const float c = (float)cos(th), s = (float)sin(th);
            // forward: Zre = sum cos Tre + sin Tim, Zim = sum cos Tim - sin Tre
            Gh[(size_t)(2 * khi) * 2 * H + y] = c;
            Gh[(size_t)(2 * khi) * 2 * H + H + y] = s;
            Gh[(size_t)(2 * khi + 1) * 2 * H + y] = -s;
            Gh[(size_t)(2 * khi + 1) * 2 * H + H + y] = c;
            // inverse: T3re = sum cos Yre - sin Yim, T3im = sum sin Yre + cos Yim
            Gi[(size_t)(2 * y) * 2 * MH + khi] = c;
            Gi[(size_t)(2 * y) * 2 * MH + MH + khi] = -s;
            Gi[(size_t)(2 * y + 1) * 2 * MH + khi] = s;
            Gi[(size_t)(2 * y + 1) * 2 * MH + MH + khi] = c;
        }
    }
    DIE_CUDA_TRY(cudaMemcpy(f->Fw, Fw.data(), Fw.size() * sizeof(float), cudaMemcpyHostToDevice));
    DIE_CUDA_TRY(cudaMemcpy(f->Gh, Gh.data(), Gh.size() * sizeof(float), cudaMemcpyHostToDevice));
    DIE_CUDA_TRY(cudaMemcpy(f->Ginv, Gi.data(), Gi.size() * sizeof(float), cudaMemcpyHostToDevice));
    DIE_CUDA_TRY(cudaMemcpy(f->Fwinv, Fi.data(), Fi.size() * sizeof(float), cudaMemcpyHostToDevice));
    return DIE_OK;
}

void free_fno(fno_s* f) {
    if (!f) return;
    std::vector<void*> ptrs = {f->params, f->grads, f->am, f->av, f->Fw, f->Gh, f->Ginv, f->Fwinv, f->Rr, f->dRr,
                               f->x, f->u, f->s, f->T1, f->Z2, f->Ymix, f->Y2, f->T3, f->g1, f->g2, f->g3, f->part,
                               f->loss, f->ytmp, f->pin, f->pout, f->rs, f->err};
    for (int l = 0; l < 9; l++) ptrs.push_back(f->h[l]);
    for (int l = 0; l < 8; l++) { ptrs.push_back(f->a[l]); ptrs.push_back(f->Zmix[l]); }
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (f->hostbuf) cudaFreeHost(f->hostbuf);
    delete f;
}

die_status create_impl(const fno_desc* d, fno_s* f) {
    f->d = *d;
    f->C = d->width; f->H = d->H; f->W = d->W; f->m = d->modes; f->MH = 2 * d->modes; f->L = d->layers;
    f->hid = d->hidden; f->cin = d->c_in; f->cout = d->c_out; f->maxB = d->max_batch;
    f->HW = f->H * f->W;
    f->NM = f->MH * f->m;
    const int C = f->C, m = f->m;
    long o = 0;
    f->oP = o; o += (long)C * f->cin;
    f->op = o; o += C;
    for (int l = 0; l < f->L; l++) {
        f->oW[l] = o; o += (long)C * C;
        f->ow[l] = o; o += C;
        f->oR1[l] = o; o += 2L * C * C * m * m;
        f->oR2[l] = o; o += 2L * C * C * m * m;
    }
    f->oQ1 = o; o += (long)f->hid * C;
    f->oq1 = o; o += f->hid;
    f->oQ2 = o; o += (long)f->cout * f->hid;
    f->oq2 = o; o += f->cout;
    f->np = o;
    const long B = f->maxB, HW = f->HW, C2 = 2 * C;
    const long wide = (C > f->hid ? C : f->hid);
    auto al = [](float** p, long n) { return cudaMalloc((void**)p, (size_t)(n > 0 ? n : 1) * sizeof(float)) == cudaSuccess; };
    bool ok = al(&f->params, f->np) && al(&f->grads, f->np) && al(&f->am, f->np) && al(&f->av, f->np) &&
              al(&f->Fw, 2L * m * f->W) && al(&f->Gh, 2L * f->MH * 2 * f->H) && al(&f->Ginv, 2L * f->H * 2 * f->MH) &&
              al(&f->Fwinv, (long)f->W * 2 * m) && al(&f->Rr, (long)f->L * f->NM * C2 * C2) &&
              al(&f->dRr, (long)f->NM * C2 * C2) && al(&f->x, B * f->cin * HW) && al(&f->u, B * f->hid * HW) &&
              al(&f->s, B * f->hid * HW) && al(&f->T1, B * C * 2 * m * f->H) && al(&f->Z2, B * C * m * 2 * f->MH) &&
              al(&f->Ymix, (long)f->NM * B * C2) && al(&f->Y2, B * C * m * 2 * f->MH) &&
              al(&f->T3, B * C * f->H * 2 * m) && al(&f->g1, B * wide * HW) && al(&f->g2, B * wide * HW) &&
              al(&f->g3, B * wide * HW) &&
              al(&f->part, B * (wide * wide > (long)C * f->cin ? wide * wide : (long)C * f->cin)) &&
              al(&f->loss, 1) && al(&f->ytmp, B * f->cout * HW) && al(&f->pin, (long)f->cin * HW) &&
              al(&f->pout, (long)f->cout * HW);
    for (int l = 0; ok && l < f->L; l++)
        ok = al(&f->h[l], B * C * HW) && al(&f->a[l], B * C * HW) && al(&f->Zmix[l], (long)f->NM * B * C2);
    ok = ok && cudaMalloc((void**)&f->rs, sizeof(double)) == cudaSuccess &&
         cudaMalloc((void**)&f->err, sizeof(int)) == cudaSuccess &&
         cudaHostAlloc((void**)&f->hostbuf, 16 * sizeof(float), cudaHostAllocDefault) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return DIE_ENOMEM;
    }
    DIE_CUDA_TRY(cudaMemset(f->params, 0, f->np * sizeof(float)));
    DIE_CUDA_TRY(cudaMemset(f->grads, 0, f->np * sizeof(float)));
    DIE_CUDA_TRY(cudaMemset(f->am, 0, f->np * sizeof(float)));
    DIE_CUDA_TRY(cudaMemset(f->av, 0, f->np * sizeof(float)));
    DIE_CUDA_TRY(cudaMemset(f->err, 0, sizeof(int)));
    return make_dft(f);
}

// Reads (and clears) the flag a GEMM sets when one of its bounded waits gave up.
die_status check_err(fno_s* f, cudaStream_t st) {
    int e = 0;
    DIE_CUDA_TRY(cudaMemcpyAsync(&e, f->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DIE_CUDA_TRY(cudaStreamSynchronize(st));
    if (!e) return DIE_OK;
    DIE_CUDA_TRY(cudaMemsetAsync(f->err, 0, sizeof(int), st));
    return DIE_ETIMEOUT;
}

}  // namespace
}  // namespace die

using namespace die;

extern "C" die_status die_gemm_bf16(int M, int N, int K, int batch, float alpha, const float* A, long long sam,
                                    long long sak, long long sab, const float* B, long long sbn, long long sbk,
                                    long long sbb, float beta, float* C, long long scm, long long scn, long long scb,
                                    int check, void* stream) {
    GemmArgs g;
    g.M = M; g.N = N; g.K = K; g.batch = batch; g.alpha = alpha; g.beta = beta;
    g.A = A; g.sam = sam; g.sak = sak; g.sab = sab;
    g.B = B; g.sbn = sbn; g.sbk = sbk; g.sbb = sbb;
    g.C = C; g.scm = scm; g.scn = scn; g.scb = scb;
    cudaStream_t st = (cudaStream_t)stream;
    int* err = nullptr;
    if (check) {
        if (cudaMalloc((void**)&err, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return DIE_ENOMEM; }
        if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) { cudaFree(err); return DIE_ECUDA; }
        g.err = err;
    }
    die_status s = tc_gemm(g, st);
    if (s == DIE_OK && check) {
        int e = 0;
        if (cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            s = DIE_ECUDA;
        else if (e)
            s = DIE_ETIMEOUT;
    }
    if (err) cudaFree(err);
    return s;
}

extern "C" die_status fno_create(const fno_desc* d, fno_t* out) {
    if (!d || !out) return DIE_EINVAL;
    *out = nullptr;
    if (d->c_in < 1 || d->c_in > 64 || d->c_out < 1 || d->c_out > 64 || d->width < 1 || d->width > 64 ||
        d->layers < 1 || d->layers > 8 || d->hidden < 1 || d->hidden > 256 || d->H < 2 || d->H > 512 || d->W < 2 ||
        d->W > 512 || d->modes < 1 || 2 * d->modes > d->H || 2 * d->modes > d->W || d->max_batch < 1 ||
        d->max_batch > 256)
        return DIE_EINVAL;
    fno_s* f = new (std::nothrow) fno_s();
    if (!f) return DIE_ENOMEM;
    die_status s;
    try {
        s = create_impl(d, f);
    } catch (...) {
        s = DIE_ENOMEM;
    }
    if (s != DIE_OK) {
        free_fno(f);
        return s;
    }
    *out = f;
    return DIE_OK;
}

extern "C" void fno_destroy(fno_t f) { free_fno(f); }

extern "C" long long fno_param_count(fno_t f) { return f ? f->np : -1; }

extern "C" die_status fno_set_params(fno_t f, const float* host) {
    if (!f || !host) return DIE_EINVAL;
    DIE_CUDA_TRY(cudaMemcpy(f->params, host, f->np * sizeof(float), cudaMemcpyHostToDevice));
    DIE_CUDA_TRY(cudaMemset(f->am, 0, f->np * sizeof(float)));
    DIE_CUDA_TRY(cudaMemset(f->av, 0, f->np * sizeof(float)));
    f->adam_t = 0;
    return DIE_OK;
}

extern "C" die_status fno_get_params(fno_t f, float* host) {
    if (!f || !host) return DIE_EINVAL;
    DIE_CUDA_TRY(cudaMemcpy(host, f->params, f->np * sizeof(float), cudaMemcpyDeviceToHost));
    return DIE_OK;
}

extern "C" die_status fno_get_grads(fno_t f, float* host) {
    if (!f || !host) return DIE_EINVAL;
    DIE_CUDA_TRY(cudaDeviceSynchronize());
    DIE_CUDA_TRY(cudaMemcpy(host, f->grads, f->np * sizeof(float), cudaMemcpyDeviceToHost));
    return DIE_OK;
}

extern "C" die_status fno_zero_grads(fno_t f, void* stream) {
    if (!f) return DIE_EINVAL;
    DIE_CUDA_TRY(cudaMemsetAsync(f->grads, 0, f->np * sizeof(float), (cudaStream_t)stream));
    return DIE_OK;
}

extern "C" die_status fno_forward(fno_t f, int B, const float* x, float* y, void* stream) {
    if (!f || !x || !y || B < 1 || B > f->maxB) return DIE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    DIE_TRY(forward(f, B, x, y, st));
    return check_err(f, st);
}

extern "C" die_status fno_backward(fno_t f, int B, const float* gy, float* gx, void* stream) {
    if (!f || !gy || B < 1 || B != f->lastB) return DIE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    DIE_TRY(backward(f, B, gy, gx, st));
    return check_err(f, st);
}

extern "C" die_status fno_train_step(fno_t f, int B, const float* x, const float* t, float lr, float* loss,
                                     void* stream) {
    if (!f || !x || !t || B < 1 || B > f->maxB || !(lr >= 0)) return DIE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const long n = (long)B * f->cout * f->HW;
    DIE_TRY(forward(f, B, x, f->ytmp, st));
    mse_kernel<<<1, kT, 0, st>>>(f->ytmp, t, n, f->ytmp, f->loss);   // gradient in place of y
    DIE_LAUNCH_CHECK();
    DIE_CUDA_TRY(cudaMemsetAsync(f->grads, 0, f->np * sizeof(float), st));
    DIE_TRY(backward(f, B, f->ytmp, nullptr, st));
    f->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)f->adam_t), c2 = 1.f - powf(b2, (float)f->adam_t);
    adam_kernel<<<blocks_for(f->np), kT, 0, st>>>(f->params, f->grads, f->am, f->av, f->np, lr, b1, b2, 1e-8f, c1, c2);
    DIE_LAUNCH_CHECK();
    if (loss) {
        DIE_CUDA_TRY(cudaMemcpyAsync(f->hostbuf, f->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        DIE_TRY(check_err(f, st));
        *loss = f->hostbuf[0];
    }
    return DIE_OK;
}

namespace die {
// z = M(v) = v + s * network(encode(chi, v)) for one field of operator op.
die_status fno_apply_precond(fno_s* f, dieop_s* op, const double2* v, double2* z, cudaStream_t st) {
    const long N = op->N;
    sumsq_kernel<<<1, kT, 0, st>>>(v, 2 * N, f->rs);
    DIE_LAUNCH_CHECK();
    encode_kernel<<<blocks_for(N), kT, 0, st>>>(op->chi_d, v, f->rs, N, f->pin);
    DIE_LAUNCH_CHECK();
    DIE_TRY(forward(f, 1, f->pin, f->pout, st));
    decode_kernel<<<blocks_for(N), kT, 0, st>>>(v, f->pout, f->rs, N, z);
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

bool fno_matches(const fno_s* f, const dieop_s* op) {
    return op->planes == 2 && f->cin == 6 && f->cout == 4 && f->H == op->n2 && f->W == op->n1;
}
}  // namespace die

extern "C" die_status fno_precondition(fno_t f, dieop_t op, const void* v, void* z, void* stream) {
    if (!f || !op || !v || !z || !fno_matches(f, op)) return DIE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    DIE_TRY(fno_apply_precond(f, op, (const double2*)v, (double2*)z, st));
    return check_err(f, st);
}

extern "C" die_status fno_encode_pair(dieop_t op, const void* b, const void* u, float* x, float* t, void* stream) {
    if (!op || !b || !x || (t && !u) || op->planes != 2) return DIE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const long N = op->N;
    double* ss = nullptr;
    if (cudaMalloc((void**)&ss, sizeof(double)) != cudaSuccess) { cudaGetLastError(); return DIE_ENOMEM; }
    sumsq_kernel<<<1, kT, 0, st>>>((const double2*)b, 2 * N, ss);
    encode_kernel<<<blocks_for(N), kT, 0, st>>>(op->chi_d, (const double2*)b, ss, N, x);
    if (t) target_kernel<<<blocks_for(N), kT, 0, st>>>((const double2*)b, (const double2*)u, ss, N, t);
    const cudaError_t e = cudaGetLastError();
    cudaFree(ss);                 // waits for the kernels
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "fno_encode_pair", __FILE__, __LINE__);
        return DIE_ECUDA;
    }
    return DIE_OK;
}
