// Shared device/host helpers of libdie: complex arithmetic on float2/double2,
// status plumbing and launch checks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/die.h"

namespace die {

// ---------------------------------------------------------------- complex types
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using C_t = typename cplx<T>::type;

template <typename V> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename V>
__host__ __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V>
__host__ __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V>
__host__ __device__ __forceinline__ V cmul(V a, V b) {
    V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename V, typename S>
__host__ __device__ __forceinline__ V cscale(V a, S s) { V r; r.x = a.x * s; r.y = a.y * s; return r; }
// a * (-i) and a * (+i)
template <typename V>
__host__ __device__ __forceinline__ V mul_mi(V a) { V r; r.x = a.y; r.y = -a.x; return r; }
template <typename V>
__host__ __device__ __forceinline__ V mul_pi(V a) { V r; r.x = -a.y; r.y = a.x; return r; }

// element-type conversion between complex64 and complex128
template <typename To> __device__ __forceinline__ To cvt(float2 a);
template <typename To> __device__ __forceinline__ To cvt(double2 a);
template <> __device__ __forceinline__ float2 cvt<float2>(float2 a) { return a; }
template <> __device__ __forceinline__ double2 cvt<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 cvt<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 cvt<double2>(float2 a) { return make_double2(a.x, a.y); }

__host__ __device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }

// ------------------------------------------------ programmatic dependent launch
// The kernels of an Arnoldi step (and of the products) are launched with programmatic
// stream serialisation: the launch of a kernel's grid overlaps the exit of the previous
// kernel's last blocks, and the kernel waits in pdl_wait for that kernel's completion
// and memory before reading anything an earlier kernel wrote (skip flags included);
// work that needs none of it (staging operator constants) may come before the wait.
// The trigger is the implicit one at block exit: an explicit early trigger made the
// successor's blocks resident while the predecessor still ran and slowed both.  On a
// normal launch pdl_wait is a no-op.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// A skip flag's value for the whole block: thread 0 reads it once and the block shares
// it.  A "live" flag (one that another stream may set while the kernel runs) read by
// every thread could otherwise split a block between threads that skip and threads that
// reach a barrier.
__device__ __forceinline__ bool block_flag(const int* flag) {
    __shared__ int s_flag;
    if (threadIdx.x == 0) s_flag = flag ? *(const volatile int*)flag : 0;
    __syncthreads();
    return s_flag != 0;
}

bool pdl_enabled();   // false when the environment sets DIE_PDL=0

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace die

// ------------------------------------------------------------------ status glue
#define DIE_CUDA_TRY(...)                                                      \
    do {                                                                       \
        cudaError_t e_ = (__VA_ARGS__);                                        \
        if (e_ != cudaSuccess) { die::set_last_cuda_error(e_, #__VA_ARGS__, __FILE__, __LINE__); return DIE_ECUDA; } \
    } while (0)

#define DIE_LAUNCH_CHECK()                                                     \
    do {                                                                       \
        cudaError_t e_ = cudaGetLastError();                                   \
        if (e_ != cudaSuccess) { die::set_last_cuda_error(e_, "kernel launch", __FILE__, __LINE__); return DIE_ECUDA; } \
    } while (0)

#define DIE_TRY(...)                                                           \
    do { die_status s_ = (__VA_ARGS__); if (s_ != DIE_OK) return s_; } while (0)

namespace die {
void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
}
