// FP64 instantiations of the product kernels (matvec_kernels.cuh) and the operator views.
#include "rows_fast.cuh"

DIE_INSTANTIATE_ROWS_C128

namespace die {

OpDev<double> view_d(const dieop_s* op) {
    OpDev<double> v;
    v.n1 = op->n1; v.n2 = op->n2; v.M1 = op->M1; v.M2 = op->M2; v.Q1 = op->Q1; v.Q2 = op->Q2;
    v.f1 = op->f1; v.i1 = op->i1; v.f2 = op->f2; v.i2 = op->i2;
    v.tw1 = op->tw1_d; v.tw2 = op->tw2_d; v.gq = op->gq_d;
    v.twx1 = op->tw1_d + op->M1; v.twx2 = op->tw2_d + op->M2;
    v.tr = 0;
    v.chim = op->chim_d;
    v.planes = op->planes;
    v.xs = (long)op->planes * op->n1 * op->n2;
    v.ws = (long)op->planes * op->M1 * op->n2;
    return v;
}
OpDev<float> view_f(const dieop_s* op) {
    OpDev<float> v;
    v.n1 = op->n1; v.n2 = op->n2; v.M1 = op->M1; v.M2 = op->M2; v.Q1 = op->Q1; v.Q2 = op->Q2;
    v.f1 = op->f1; v.i1 = op->i1; v.f2 = op->f2; v.i2 = op->i2;
    v.tw1 = op->tw1_f; v.tw2 = op->tw2_f; v.gq = op->gq_f;
    v.twx1 = op->tw1_f + op->M1; v.twx2 = op->tw2_f + op->M2;
    v.tr = op->tile_rows_c64;
    v.chim = op->chim_f;
    v.planes = op->planes;
    v.xs = (long)op->planes * op->n1 * op->n2;
    v.ws = (long)op->planes * op->M1 * op->n2;
    return v;
}

// Shared-memory limits are raised lazily by each launcher on first use.
die_status set_kernel_attributes(const dieop_s*) { return DIE_OK; }

template die_status apply_op<double, double2>(dieop_s*, Contrast, const double2*, double2*, cudaStream_t,
                                  const Workspace*);
template die_status apply_reg<double, double2>(dieop_s*, const double2*, double2*, cudaStream_t,
                                  const Workspace*);
template die_status apply_op_skip<double, double2>(dieop_s*, Contrast, const double2*, double2*, const int*, cudaStream_t,
                                  const Workspace*);
template die_status apply_reg_skip<double, double2>(dieop_s*, const double2*, double2*, const int*, cudaStream_t,
                                  const Workspace*);
template die_status apply_batch<double, double2>(dieop_s*, bool, const double2*, double2*, int, void*, void*,
                                                 cudaStream_t);

}  // namespace die
