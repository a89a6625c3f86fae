// Launchers of the fast row passes at one tile height TR (declared in matvec_kernels.cuh).
// A translation unit that includes this header instantiates the launchers of one height
// (DIE_INSTANTIATE_ROWS_C64 / _C128), so that the kernels of each height are compiled
// once, in parallel with the others.
#pragma once

#include "matvec_kernels.cuh"

namespace die {

template <typename T, typename IO, int TR>
void rows_fwd_fast(const OpDev<T>& v, const IO* u, const C_t<T>* chi, C_t<T>* W, const int* skip, cudaStream_t st,
                   int nb) {
    using C = C_t<T>;
#define K1F_CASE(LSV)                                                                                        \
    if constexpr (tile_ok<C, LSV, TR>()) {                                                                   \
        constexpr int tr_ = tile_of<C, LSV, TR>();                                                           \
        static std::atomic<bool> a_{false};                                                                  \
        launch_kernel(k1_fast<T, IO, LSV, tr_>, a_, with_z(rows_launch_fast<C, LSV, tr_>(v.n2), nb), st, v, u, \
                      chi, W, skip);                                                                         \
    }
    DIE_PROF(PK_ROWS_FWD, st, DIE_FAST_SWITCH(v.M1, K1F_CASE));
#undef K1F_CASE
}

template <typename T, typename U, typename IO, int TR>
void rows_inv_fast(const OpDev<T>& v, const C_t<T>* W, const U* u, IO* y, const int* skip, cudaStream_t st, int nb) {
    using C = C_t<T>;
#define K3F_CASE(LSV)                                                                                        \
    if constexpr (tile_ok<C, LSV, TR>()) {                                                                   \
        constexpr int tr_ = tile_of<C, LSV, TR>();                                                           \
        static std::atomic<bool> a_{false};                                                                  \
        launch_kernel(k3_fast<T, U, IO, LSV, tr_>, a_, with_z(rows_launch_fast<C, LSV, tr_>(v.n2), nb), st, v, \
                      W, u, y, skip);                                                                        \
    }
    DIE_PROF(PK_ROWS_INV, st, DIE_FAST_SWITCH(v.M1, K3F_CASE));
#undef K3F_CASE
}

template <typename T, typename IO, int TR>
void rows_inv_fwd_fast(const OpDev<T>& v, C_t<T>* W, const IO* u, const C_t<T>* chir, C_t<T>* vb, const int* skip,
                       cudaStream_t st, int nb) {
    using C = C_t<T>;
#define KKF_CASE(LSV)                                                                                        \
    if constexpr (tile_ok<C, LSV, TR>()) {                                                                   \
        constexpr int tr_ = tile_of<C, LSV, TR>();                                                           \
        static std::atomic<bool> a_{false};                                                                  \
        launch_kernel(k3k1_fast<T, IO, LSV, tr_>, a_, with_z(rows_launch_fast<C, LSV, tr_>(v.n2), nb), st, v, \
                      W, u, chir, vb, skip);                                                                 \
    }
    DIE_PROF(PK_ROWS_INV_FWD, st, DIE_FAST_SWITCH(v.M1, KKF_CASE));
#undef KKF_CASE
}

template <int TR>
void rows_defl_fast(const OpDev<float>& v, const DeflIn& d, const float2* chi, float2* z, float2* W, const int* skip,
                    cudaStream_t st) {
#define K1D_CASE(LSV)                                                                                        \
    if constexpr (tile_ok<float2, LSV, TR>()) {                                                              \
        constexpr int tr_ = tile_of<float2, LSV, TR>();                                                      \
        static std::atomic<bool> a_{false};                                                                  \
        launch_kernel(k1_defl_fast<LSV, tr_>, a_, rows_launch_fast<float2, LSV, tr_>(v.n2), st, v, d, chi, z, W, \
                      skip);                                                                                 \
    }
    DIE_PROF(PK_ROWS_FWD, st, DIE_FAST_SWITCH(v.M1, K1D_CASE));
#undef K1D_CASE
}

}  // namespace die

// Every launcher the complex64 products use, at height TR.
#define DIE_INSTANTIATE_ROWS_C64(TR)                                                                          \
    namespace die {                                                                                          \
    template void rows_fwd_fast<float, float2, TR>(const OpDev<float>&, const float2*, const float2*, float2*, \
                                                   const int*, cudaStream_t, int);                          \
    template void rows_fwd_fast<float, double2, TR>(const OpDev<float>&, const double2*, const float2*,       \
                                                    float2*, const int*, cudaStream_t, int);                \
    template void rows_inv_fast<float, float2, float2, TR>(const OpDev<float>&, const float2*, const float2*,  \
                                                           float2*, const int*, cudaStream_t, int);         \
    template void rows_inv_fast<float, double2, double2, TR>(const OpDev<float>&, const float2*,              \
                                                             const double2*, double2*, const int*,          \
                                                             cudaStream_t, int);                            \
    template void rows_inv_fast<float, float2, double2, TR>(const OpDev<float>&, const float2*, const float2*, \
                                                            double2*, const int*, cudaStream_t, int);       \
    template void rows_inv_fwd_fast<float, float2, TR>(const OpDev<float>&, float2*, const float2*,           \
                                                       const float2*, float2*, const int*, cudaStream_t, int); \
    template void rows_inv_fwd_fast<float, double2, TR>(const OpDev<float>&, float2*, const double2*,         \
                                                        const float2*, float2*, const int*, cudaStream_t, int); \
    template void rows_defl_fast<TR>(const OpDev<float>&, const DeflIn&, const float2*, float2*, float2*,     \
                                     const int*, cudaStream_t);                                              \
    }

// The FP64 products (default height only).
#define DIE_INSTANTIATE_ROWS_C128                                                                             \
    namespace die {                                                                                          \
    template void rows_fwd_fast<double, double2, 0>(const OpDev<double>&, const double2*, const double2*,    \
                                                    double2*, const int*, cudaStream_t, int);               \
    template void rows_inv_fast<double, double2, double2, 0>(const OpDev<double>&, const double2*,           \
                                                             const double2*, double2*, const int*,          \
                                                             cudaStream_t, int);                            \
    template void rows_inv_fwd_fast<double, double2, 0>(const OpDev<double>&, double2*, const double2*,      \
                                                        const double2*, double2*, const int*, cudaStream_t,  \
                                                        int);                                                \
    }
