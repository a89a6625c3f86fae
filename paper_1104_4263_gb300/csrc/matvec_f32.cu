// Complex64-arithmetic instantiations of the product kernels (matvec_kernels.cuh):
// complex64 I/O (dieop_apply with DIE_FP32_INNER) and complex128 I/O (products inside
// the FP32-inner GMRES cycles).
#include "rows_fast.cuh"

DIE_INSTANTIATE_ROWS_C64(0)

namespace die {

template die_status apply_op<float, float2>(dieop_s*, Contrast, const float2*, float2*, cudaStream_t,
                                  const Workspace*);
template die_status apply_op<float, double2>(dieop_s*, Contrast, const double2*, double2*, cudaStream_t,
                                  const Workspace*);
template die_status apply_reg<float, float2>(dieop_s*, const float2*, float2*, cudaStream_t,
                                  const Workspace*);
template die_status apply_reg<float, double2>(dieop_s*, const double2*, double2*, cudaStream_t,
                                  const Workspace*);
template die_status apply_batch<float, float2>(dieop_s*, bool, const float2*, float2*, int, void*, void*, cudaStream_t);
template die_status apply_op_skip<float, double2>(dieop_s*, Contrast, const double2*, double2*, const int*, cudaStream_t,
                                  const Workspace*);
template die_status apply_reg_skip<float, double2>(dieop_s*, const double2*, double2*, const int*, cudaStream_t,
                                  const Workspace*);
template die_status apply_op_skip_xy<float, float2, double2>(dieop_s*, Contrast, const float2*, double2*, const int*,
                                                             cudaStream_t,
                                  const Workspace*);
template die_status apply_reg_skip_xy<float, float2, double2>(dieop_s*, const float2*, double2*, const int*,
                                                              cudaStream_t,
                                  const Workspace*);

bool defl_product_ok(const dieop_s* op) { return fast_rows(view_f(op)); }

die_status apply_defl_xy(dieop_s* op, const DeflIn& d, float2* z, double2* y, bool reg, const int* skip,
                         cudaStream_t st, const Workspace* ws) {
    if (!ws) ws = &op->ws;
    const OpDev<float> v = view_f(op);
    if (!fast_rows(v) || d.r < 1 || d.r > 32 || !d.V32 || !d.cf || (!d.w && !d.x) || (d.w && !d.inv))
        return DIE_EINVAL;
    float2* W = reinterpret_cast<float2*>(ws->W);
    float2* vb = reinterpret_cast<float2*>(ws->v);
    with_tile_rows(v, [&](auto tr) { rows_defl_fast<decltype(tr)::value>(v, d, op->chi_f, z, W, skip, st); });
    launch_k2<float>(v, W, skip, st);
    if (reg) {
        launch_k3k1<float, float2>(v, W, z, op->chir_f, vb, skip, st);
        launch_k2<float>(v, W, skip, st);
        launch_k3<float, float2, double2>(v, W, vb, y, skip, st);
    } else {
        launch_k3<float, float2, double2>(v, W, z, y, skip, st);
    }
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

}  // namespace die
