// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) for the
// learned preconditioner: C(m, n) = alpha * sum_k A(m, k) B(n, k) + beta * C(m, n)
// (+ bias), with FP32 operands in global memory at arbitrary strides, rounded to BF16
// when they are staged into shared memory, and FP32 accumulation in tensor memory.
//
// One CTA of 128 threads computes a 128 x BN tile (BN = 64 or 128):
//   * the operand tiles of a 64-wide K step are copied by all threads into shared
//     memory in the canonical K-major, no-swizzle layout of the tensor cores (8-row x
//     16-byte core matrices; core matrices adjacent in K are BM * 16 bytes apart, the
//     leading-dimension offset; 8-row groups are 128 bytes apart, the stride offset);
//   * one elected thread issues four tcgen05.mma (K = 16 each) into a TMEM accumulator
//     of BN columns and commits them to an mbarrier that every thread waits on (bounded)
//     before the tiles are overwritten;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes
//     32 w .. 32 w + 31, i.e. rows 32 w + lane) and writes C.
// Strides make every transpose of the network's forward and backward passes a plain
// call; the operand sizes of a Fourier neural operator are small, so the copies are not
// pipelined.
#pragma once

#include "common.cuh"

namespace die {

struct GemmArgs {
    int M = 0, N = 0, K = 0, batch = 1;
    const float* A = nullptr;   // A(m, k) of batch b at A[b * sab + m * sam + k * sak]
    long sam = 0, sak = 0, sab = 0;
    const float* B = nullptr;   // B(n, k) at B[b * sbb + n * sbn + k * sbk]
    long sbn = 0, sbk = 0, sbb = 0;
    float* C = nullptr;         // C(m, n) at C[b * scb + m * scm + n * scn]
    long scm = 0, scn = 0, scb = 0;
    float alpha = 1.f, beta = 0.f;   // beta == 0: C is not read
    const float* bias = nullptr;     // optional: + bias[n]
    int* err = nullptr;              // optional device flag: set to 1 when a wait gave up
};

// Launch on `st`.  DIE_EINVAL on bad sizes or a NULL operand, DIE_ECUDA on a launch error.
die_status tc_gemm(const GemmArgs& g, cudaStream_t st);

}  // namespace die
