// Operator set-up (once per dieop_create): contrasts, the Green's-tensor table of
// Eqs. (4.3)-(4.5) embedded in an M1 x M2 periodic grid, its 2-D FFT and the
// quarter-spectrum extraction used by the column pass.
#include "op.cuh"

namespace die {

// chi = eps_r - 1 (Eq. (2.11)), chi' = 1/eps_r - 1 (Eq. (3.18)); flags |eps_r| <= 1e-12
// (the existence condition eps != 0, Eq. (3.17)) and non-finite values.
__global__ void contrast_kernel(const double2* __restrict__ eps, long N, double2* chi_d, double2* chir_d,
                                float2* chi_f, float2* chir_f, int* flag) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const double2 e = eps[i];
        const double m2 = e.x * e.x + e.y * e.y;
        if (!(m2 > 1e-24) || !isfinite(m2)) { atomicOr(flag, 1); continue; }
        const double2 c = make_double2(e.x - 1.0, e.y);
        const double2 inv = make_double2(e.x / m2, -e.y / m2);
        const double2 cr = make_double2(inv.x - 1.0, inv.y);
        chi_d[i] = c; chir_d[i] = cr;
        chi_f[i] = make_float2((float)c.x, (float)c.y);
        chir_f[i] = make_float2((float)cr.x, (float)cr.y);
    }
}

// Periodic embedding: plane[q_idx][p_idx] holds G(p h, q h) for the signed offsets
// p = p_idx (p_idx <= M1/2) or p_idx - M1, |p| < n1 (same for q); zero elsewhere.
// Off-diagonal entries (Eqs. (4.3), (4.5)), with r = h sqrt(p^2 + q^2), theta = (p, q) h / r:
//   G11 = k^2 h^2 [P theta1^2 + Q],  G22 = k^2 h^2 [P theta2^2 + Q],  G12 = k^2 h^2 P theta1 theta2,
//   P = (i/(2kr)) H1 - (i/4) H0,     Q = (i/4) H0 - (i/(4kr)) H1,      H_m = J_m + i Y_m.
// Self term (Eq. (4.4)): G11 = G22 = -[1 - (i pi/4) k a H1(k a)], a = h/sqrt(pi); G12 = 0.
//
// TM (tm != 0): the scalar kernel of the E-wave equation E3_in = E3 - k^2 g * (chi E3)
// (Section 2) on the same grid, in both diagonal planes: G11 = G22 = k^2 h^2 (i/4) H0(k r)
// off the diagonal, and k^2 times the integral of g over the equal-area disc on it,
// (i pi / 2) k a H1(k a) - 1; G12 = 0, so the two planes never mix.
//
// Three planes (mag != 0, DIE_TE_MAG): also the couplings of the magnetic field, from
// Section 3's compact kernels with eps_b = mu_b = 1, omega = k, d/dx_l g = -(i k/4) H1 theta_l:
//   plane 3: G13 = G31 = i k d2 g h^2 =  (k^2 h^2 / 4) H1(k r) theta2
//   plane 4: G23 = G32 = -i k d1 g h^2 = -(k^2 h^2 / 4) H1(k r) theta1
//   plane 5: G33 = k^2 h^2 (i/4) H0(k r); at r = 0: G13 = G23 = 0 (odd kernels) and G33 =
//            (i pi / 2) k a H1(k a) - 1, the disc integral of k^2 g (Section 4's [A33]_nn).
__global__ void green_planes_kernel(int n1, int n2, int M1, int M2, double h, double k, int tm, int mag,
                                    double2* __restrict__ planes) {
    const long plane = (long)M1 * M2;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < plane; idx += (long)gridDim.x * blockDim.x) {
        const int pi = (int)(idx % M1), qi = (int)(idx / M1);
        const int p = pi <= M1 / 2 ? pi : pi - M1;
        const int q = qi <= M2 / 2 ? qi : qi - M2;
        double2 g11 = make_double2(0, 0), g22 = make_double2(0, 0), g12 = make_double2(0, 0);
        if (tm && abs(p) < n1 && abs(q) < n2) {
            if (p == 0 && q == 0) {
                const double a = h * rsqrt(M_PI);
                const double ka = k * a;
                // (i pi/2) ka (J1 + i Y1) - 1 = (-1 - (pi/2) ka Y1) + i (pi/2) ka J1
                g11 = make_double2(-1.0 - 0.5 * M_PI * ka * y1(ka), 0.5 * M_PI * ka * j1(ka));
            } else {
                const double r = h * sqrt((double)p * p + (double)q * q);
                const double c = k * k * h * h;
                // k^2 h^2 (i/4)(J0 + i Y0)
                g11 = make_double2(-0.25 * c * y0(k * r), 0.25 * c * j0(k * r));
            }
            g22 = g11;
        } else if (abs(p) < n1 && abs(q) < n2) {
            if (p == 0 && q == 0) {
                const double a = h * rsqrt(M_PI);
                const double ka = k * a;
                const double j1v = j1(ka), y1v = y1(ka);
                // -(1 - (i pi/4) ka (J1 + i Y1)) = (-1 - (pi/4) ka Y1) + i (pi/4) ka J1
                g11 = make_double2(-1.0 - 0.25 * M_PI * ka * y1v, 0.25 * M_PI * ka * j1v);
                g22 = g11;
            } else {
                const double d1 = p * h, d2 = q * h;
                const double r = sqrt(d1 * d1 + d2 * d2);
                const double kr = k * r;
                const double J0 = j0(kr), Y0 = y0(kr), J1 = j1(kr), Y1 = y1(kr);
                // P = (i/(2kr))(J1 + iY1) - (i/4)(J0 + iY0)
                const double2 P = make_double2(-Y1 / (2 * kr) + 0.25 * Y0, J1 / (2 * kr) - 0.25 * J0);
                // Q = (i/4)(J0 + iY0) - (i/(4kr))(J1 + iY1)
                const double2 Q = make_double2(-0.25 * Y0 + Y1 / (4 * kr), 0.25 * J0 - J1 / (4 * kr));
                const double t1 = d1 / r, t2 = d2 / r;
                const double c = k * k * h * h;
                g11 = make_double2(c * (P.x * t1 * t1 + Q.x), c * (P.y * t1 * t1 + Q.y));
                g22 = make_double2(c * (P.x * t2 * t2 + Q.x), c * (P.y * t2 * t2 + Q.y));
                g12 = make_double2(c * P.x * t1 * t2, c * P.y * t1 * t2);
            }
        }
        planes[idx] = g11;
        planes[plane + idx] = g22;
        planes[2 * plane + idx] = g12;
        if (mag) {
            double2 g13 = make_double2(0, 0), g23 = make_double2(0, 0), g33 = make_double2(0, 0);
            if (abs(p) < n1 && abs(q) < n2) {
                if (p == 0 && q == 0) {
                    const double ka = k * h * rsqrt(M_PI);
                    g33 = make_double2(-1.0 - 0.5 * M_PI * ka * y1(ka), 0.5 * M_PI * ka * j1(ka));
                } else {
                    const double d1 = p * h, d2 = q * h;
                    const double r = sqrt(d1 * d1 + d2 * d2);
                    const double kr = k * r, c = k * k * h * h;
                    const double J1 = j1(kr), Y1 = y1(kr);
                    // (c/4) (J1 + i Y1) theta2 and -(c/4) (J1 + i Y1) theta1
                    g13 = make_double2(0.25 * c * J1 * d2 / r, 0.25 * c * Y1 * d2 / r);
                    g23 = make_double2(-0.25 * c * J1 * d1 / r, -0.25 * c * Y1 * d1 / r);
                    // c (i/4) (J0 + i Y0)
                    g33 = make_double2(-0.25 * c * y0(kr), 0.25 * c * j0(kr));
                }
            }
            planes[3 * plane + idx] = g13;
            planes[4 * plane + idx] = g23;
            planes[5 * plane + idx] = g33;
        }
    }
}

// In-place forward FFT of `nlines` lines of length pl.L: element e of line l sits at
// data[l * line_stride + e * elem_stride].  One block per line (FP64, set-up only).
template <int EPT>
__global__ void fft_lines_kernel(double2* data, long elem_stride, long line_stride, FftPlan pl, const double2* tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    double2* line = data + blockIdx.x * line_stride;
    for (int e = threadIdx.x; e < pl.L; e += blockDim.x) buf[pidx(e)] = line[e * elem_stride];
    __syncthreads();
    int Ns = 1;
    run_stages<double2, EPT, false>(buf, pl, 0, pl.ns, Ns, tw, threadIdx.x, blockDim.x, true);
    for (int e = threadIdx.x; e < pl.L; e += blockDim.x) line[e * elem_stride] = buf[pidx(e)];
}

// gq[plane][k1q][k2q] = spectrum[plane][k2q][k1q] / (M1 M2), k1q <= M1/2, k2q <= M2/2.
__global__ void quarter_kernel(const double2* __restrict__ spec, int nplanes, int M1, int M2, int Q1, int Q2,
                               double scale, double2* __restrict__ gq_d, float2* __restrict__ gq_f) {
    const long q = (long)Q1 * Q2, plane = (long)M1 * M2;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < nplanes * q;
         idx += (long)gridDim.x * blockDim.x) {
        const int pl = (int)(idx / q);
        const long rem = idx - pl * q;
        const int k1q = (int)(rem / Q2), k2q = (int)(rem % Q2);
        const double2 v = spec[pl * plane + (long)k2q * M1 + k1q];
        const double2 s = make_double2(v.x * scale, v.y * scale);
        gq_d[idx] = s;
        gq_f[idx] = make_float2((float)s.x, (float)s.y);
    }
}

static die_status fft_lines(double2* data, long elem_stride, long line_stride, int nlines, const FftPlan& pl,
                            const double2* tw, cudaStream_t st) {
    const int G = pl.L / pl.ept;
    const size_t smem = (size_t)padded_len(pl.L) * sizeof(double2);
    if (pl.ept == 16) {
        DIE_CUDA_TRY(cudaFuncSetAttribute(fft_lines_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        fft_lines_kernel<16><<<nlines, G, smem, st>>>(data, elem_stride, line_stride, pl, tw);
    } else {
        DIE_CUDA_TRY(cudaFuncSetAttribute(fft_lines_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        fft_lines_kernel<12><<<nlines, G, smem, st>>>(data, elem_stride, line_stride, pl, tw);
    }
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

die_status build_green_spectrum(dieop_s* op, double2* scratch, cudaStream_t st) {
    const int M1 = op->M1, M2 = op->M2;
    const long plane = (long)M1 * M2;
    const int nplanes = green_plane_count(op);
    green_planes_kernel<<<1216, 256, 0, st>>>(op->n1, op->n2, M1, M2, op->h, op->k, op->pol == DIE_TM ? 1 : 0,
                                               op->planes == 3 ? 1 : 0, scratch);
    DIE_LAUNCH_CHECK();
    for (int p = 0; p < nplanes; p++) {
        double2* base = scratch + p * plane;
        DIE_TRY(fft_lines(base, 1, M1, M2, op->f1, op->tw1_d, st));       // rows: along x1
        DIE_TRY(fft_lines(base, M1, 1, M1, op->f2, op->tw2_d, st));       // columns: along x2
    }
    quarter_kernel<<<1216, 256, 0, st>>>(scratch, nplanes, M1, M2, op->Q1, op->Q2, 1.0 / ((double)M1 * M2), op->gq_d,
                                         op->gq_f);
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

// chi_m = mu_r - 1 (Section 2's magnetic contrast, mu_b = 1); flags non-finite values.
__global__ void magnetic_contrast_kernel(const double2* __restrict__ mu, long N, double2* chim_d, float2* chim_f,
                                         int* flag) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const double2 m = mu[i];
        if (!isfinite(m.x) || !isfinite(m.y)) { atomicOr(flag, 1); continue; }
        chim_d[i] = make_double2(m.x - 1.0, m.y);
        chim_f[i] = make_float2((float)(m.x - 1.0), (float)m.y);
    }
}

die_status compute_magnetic_contrast(const dieop_s* op, const double2* mu_dev, double2* chim_d, float2* chim_f,
                                     int* flag, cudaStream_t st) {
    magnetic_contrast_kernel<<<608, 256, 0, st>>>(mu_dev, op->N, chim_d, chim_f, flag);
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

die_status compute_contrasts_into(const dieop_s* op, const double2* eps_dev, double2* chi_d, double2* chir_d,
                                  float2* chi_f, float2* chir_f, int* flag, cudaStream_t st);

die_status compute_contrasts(dieop_s* op, const double2* eps_dev, cudaStream_t st) {
    return compute_contrasts_into(op, eps_dev, op->chi_d, op->chir_d, op->chi_f, op->chir_f, op->dflag, st);
}

die_status compute_contrasts_into(const dieop_s* op, const double2* eps_dev, double2* chi_d, double2* chir_d,
                                  float2* chi_f, float2* chir_f, int* flag, cudaStream_t st) {
    contrast_kernel<<<608, 256, 0, st>>>(eps_dev, op->N, chi_d, chir_d, chi_f, chir_f, flag);
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

}  // namespace die
