/*
 * libdie -- learned preconditioner: a Fourier neural operator on the GB300 tensor cores,
 * and flexible GMRES that uses it.
 *
 * The paper (Zouros & Budko, arXiv 1104.4263) preconditions GMRES by regularisation and
 * deflation (Sections 4-5) and leaves other preconditioners open (Section 6).  This part
 * adds a learned one: a Fourier neural operator (Li, Kovachki, Azizzadenesheli, Liu,
 * Bhattacharya, Stuart and Anandkumar, "Fourier neural operator for parametric partial
 * differential equations", ICLR 2021) that maps (contrast, right-hand side) to an
 * approximate solution, used as the initial guess and as a step-dependent right
 * preconditioner inside flexible GMRES (Saad, SIAM J. Sci. Comput. 14, 1993), with the
 * regularised and deflated GMRES of die.h as the fallback.
 *
 * Network (real channels on an H x W periodic grid, layout [batch][channel][y][x], x
 * fastest; FP32 in memory, BF16 tensor-core products with FP32 accumulation):
 *   lifting     h_0 = P x + p                                   c_in -> width
 *   layer l     a_l = W_l h_l + w_l + K_l h_l,  h_{l+1} = GELU(a_l)  (h_L = a_{L-1})
 *   projection  y = Q2 GELU(Q1 h_L + q1) + q2                   width -> hidden -> c_out
 *   K_l h: per channel the 2-D real DFT restricted to the modes k_y in [0, m) u [H-m, H),
 *   k_x in [0, m), Y[o, k] = sum_i X[i, k] R[i, o, k] (R1_l for k_y < m, R2_l for
 *   k_y >= H - m), then the inverse real DFT of the half spectrum.  GELU(x) = x Phi(x).
 * Every product of the network -- the pointwise channel maps and the truncated DFTs
 * (dense contractions with DFT matrices) and the per-mode complex channel mixing -- is a
 * tcgen05 BF16 GEMM with FP32 accumulation (die_gemm_bf16); gradients are exact for that
 * arithmetic (hand-derived backward pass).
 *
 * Parameter vector (FP32, this order; complex weights as (re, im) pairs):
 *   P [width][c_in], p [width], for l < layers: W_l [width][width], w_l [width],
 *   R1_l [width][width][m][m] complex, R2_l (same); Q1 [hidden][width], q1 [hidden],
 *   Q2 [c_out][hidden], q2 [c_out].   (R[i][o][k_y][k_x]: input, output, modes.)
 */
#ifndef LIBDIE_DIE_FNO_H
#define LIBDIE_DIE_FNO_H

#include "die.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C = alpha * A B^T + beta * C on the tensor cores, batched: for b < batch, m < M, n < N
 *   C[b*scb + m*scm + n*scn] = alpha * sum_{k<K} A[b*sab + m*sam + k*sak] * B[b*sbb + n*sbn + k*sbk]
 *                              + beta * C[...]            (C not read when beta == 0)
 * A, B, C: device FP32 at any strides (in elements; C must not overlap A or B); A and B are
 * rounded to BF16 on the way into shared memory and the products accumulate in FP32
 * (tcgen05.mma kind::f16 into tensor memory).  DIE_EINVAL: negative sizes, batch outside
 * [1, 65535], NULL operand; DIE_ECUDA on a launch error; DIE_ETIMEOUT if a bounded wait
 * of the kernel gave up (reported after a stream synchronisation, only when
 * check != 0). */
die_status die_gemm_bf16(int M, int N, int K, int batch, float alpha, const float* A, long long sam,
                         long long sak, long long sab, const float* B, long long sbn, long long sbk,
                         long long sbb, float beta, float* C, long long scm, long long scn, long long scb,
                         int check, void* stream);

typedef struct fno_s* fno_t;

typedef struct fno_desc {
    int c_in, c_out;       /* input / output channels                                        */
    int width;             /* channels of the Fourier layers (<= 64)                         */
    int modes;             /* m: 1 <= m, 2 m <= H, m <= W / 2                                */
    int layers;            /* 1 .. 8                                                          */
    int hidden;            /* channels of the projection's hidden layer (<= 256)             */
    int H, W;              /* grid; H, W <= 512                                               */
    int max_batch;         /* largest batch of forward / backward / train calls (<= 256)      */
} fno_desc;

/* Creates a network with zero parameters (set them with fno_set_params).  DIE_EINVAL on
 * sizes outside the ranges above, DIE_ENOMEM, DIE_ECUDA. */
die_status fno_create(const fno_desc* desc, fno_t* out);
void fno_destroy(fno_t net);

/* Number of FP32 entries of the parameter vector (layout above). */
long long fno_param_count(fno_t net);
/* Copy the parameters from / to host memory (fno_param_count floats).  Setting them also
 * clears the Adam moments. */
die_status fno_set_params(fno_t net, const float* host);
die_status fno_get_params(fno_t net, float* host);

/* y = network(x) for `batch` inputs: x device FP32 [batch][c_in][H][W], y device FP32
 * [batch][c_out][H][W].  The activations are kept for fno_backward. */
die_status fno_forward(fno_t net, int batch, const float* x, float* y, void* stream);

/* Gradients of <gy, network(x)> for the x of the last fno_forward (same batch): added to
 * the gradient vector (fno_param_count floats, layout of the parameters; cleared by
 * fno_zero_grads); gx (device [batch][c_in][H][W], or NULL) receives the input gradient. */
die_status fno_backward(fno_t net, int batch, const float* gy, float* gx, void* stream);
die_status fno_zero_grads(fno_t net, void* stream);
/* Copy the gradient vector to host memory. */
die_status fno_get_grads(fno_t net, float* host);

/* One training step on a batch: forward, loss = mean over entries of (y - t)^2, backward,
 * Adam update (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr.  x, t device FP32
 * ([batch][c_in][H][W], [batch][c_out][H][W]); loss (host, may be NULL) receives the loss
 * before the update (this synchronises the stream). */
die_status fno_train_step(fno_t net, int batch, const float* x, const float* t, float lr, float* loss, void* stream);

/* ----------------------------------------------------------------------------
 * The network as a preconditioner of the TE system of die.h.
 * Encoding of a field v (2 n1 n2 complex128, die.h layout) on an operator with n1 = W,
 * n2 = H: input channels (Re chi, Im chi, Re v1 / s, Im v1 / s, Re v2 / s, Im v2 / s) with
 * s the root mean square of v's entries (c_in = 6), output channels (Re d1, Im d1, Re d2,
 * Im d2) (c_out = 4), and the map
 *     M(v) = v + s d,
 * so that M is homogeneous of degree 1 (M(c v) = c M(v) for real c > 0) and the identity
 * when the network outputs zero.  Trained on pairs (v, u = A^-1 v), d approximates
 * (u - v) / s.
 * ------------------------------------------------------------------------- */

/* Training pair of the encoding above for operator op: x (device FP32, 6 x n2 x n1)
 * receives the input channels of the right-hand side b, and t (device FP32, 4 x n2 x n1,
 * or NULL) the target (u - b) / s for the solution u of A u = b (b, u device complex128).
 * A pair from a solve takes a plane wave b and the solved u; a pair from one product takes
 * any field u and b = A u (dieop_apply), for which u = A^-1 b holds exactly. */
die_status fno_encode_pair(dieop_t op, const void* b, const void* u, float* x, float* t, void* stream);

/* z = M(v) for one field; v, z device complex128 (z may equal v).  DIE_EINVAL if the
 * network's grid or channels do not match the operator (c_in 6, c_out 4, H = n2, W = n1). */
die_status fno_precondition(fno_t net, dieop_t op, const void* v, void* z, void* stream);

/* Flexible GMRES(restart) on A x = b (Section 4's system, FP64 products and Arnoldi) with
 * the right preconditioner z_j = M(v_j) (net != NULL) and the initial guess x0 = M(b)
 * (opts->use_x0 == 0 and net != NULL); restart <= 256.  If it has not reached opts->tol
 * after opts->max_iters Arnoldi steps (or met a NaN), the fallback -- gmres_solve with the
 * regularised operator (regularized = 1, inner FP32-inner products) and deflation `defl`
 * (may be NULL), restart `fallback_restart`, from the flexible iterate -- runs for up to
 * `fallback_iters` more steps.  report (may be NULL): cycles, iters (flexible steps plus
 * fallback steps), rel_res_solved / rel_res_orig = FP64 ||b - A x|| / ||b|| at exit;
 * *used_fallback (may be NULL) is set to 1 when the fallback ran.  Returns DIE_OK when
 * converged, DIE_ENOCONV otherwise, or an error as gmres_solve. */
die_status fgmres_solve(dieop_t op, fno_t net, defl_t defl, const gmres_opts* opts, int fallback_restart,
                        int fallback_iters, const void* b, void* x, gmres_report* report, int* used_fallback,
                        void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LIBDIE_DIE_FNO_H */
