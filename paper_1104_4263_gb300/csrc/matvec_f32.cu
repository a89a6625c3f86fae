// Complex64-arithmetic instantiations of the product kernels (matvec_kernels.cuh):
// complex64 I/O (dieop_apply with DIE_FP32_INNER) and complex128 I/O (products inside
// the FP32-inner GMRES cycles).
#include "matvec_kernels.cuh"

namespace die {

template die_status apply_op<float, float2>(dieop_s*, Contrast, const float2*, float2*, cudaStream_t);
template die_status apply_op<float, double2>(dieop_s*, Contrast, const double2*, double2*, cudaStream_t);
template die_status apply_reg<float, float2>(dieop_s*, const float2*, float2*, cudaStream_t);
template die_status apply_reg<float, double2>(dieop_s*, const double2*, double2*, cudaStream_t);
template die_status apply_op_skip<float, double2>(dieop_s*, Contrast, const double2*, double2*, const int*, cudaStream_t);
template die_status apply_reg_skip<float, double2>(dieop_s*, const double2*, double2*, const int*, cudaStream_t);
template die_status apply_op_skip_xy<float, float2, double2>(dieop_s*, Contrast, const float2*, double2*, const int*,
                                                             cudaStream_t);
template die_status apply_reg_skip_xy<float, float2, double2>(dieop_s*, const float2*, double2*, const int*,
                                                              cudaStream_t);

}  // namespace die
