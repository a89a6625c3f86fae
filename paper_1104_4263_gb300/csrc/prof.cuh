// Kernel timing aid: while enabled (die_prof_begin .. die_prof_end), every kernel
// launch of the library is bracketed by CUDA events recorded on its stream; the
// durations are summed per kernel class when the session ends.  Off by default.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

namespace die {

enum ProfKernel {
    PK_ROWS_FWD = 0,      // K1: contrast multiply + row FFT
    PK_COLS,              // K2: column FFT, Green-spectrum multiply, inverse column FFT
    PK_ROWS_INV,          // K3: row inverse FFT + crop + subtract
    PK_ROWS_INV_FWD,      // K3K1: fused row inverse of A(chi) and row forward of A(chi')
    PK_DOTS,              // batched projections V^* w (FP64 basis)
    PK_DOTS32,            // batched projections with the complex64 deflation basis
    PK_UPDATE_NORM,       // Gram-Schmidt update w -= V h with the norm of the result
    PK_DOTS_REORTH,       // second (re-orthogonalisation) pass: projections
    PK_UPDATE_REORTH,     // second pass: update
    PK_SCALE,             // vector scaling
    PK_DEFL_UPDATE,       // deflation z = x + V (M s)
    PK_LINCOMB,           // x += V y
    PK_SMALL,             // single-thread small dense work
    PK_GIVENS,            // GMRES Givens step (side stream)
    PK_OTHER,
    PK_COUNT
};

extern std::atomic<bool> g_prof_on;
extern thread_local int g_prof_override;      // >= 0: record launches under this class instead
void prof_mark(int id, cudaStream_t st, int stop);

}  // namespace die

#define DIE_PROF(id, st, ...)                                                                    \
    do {                                                                                         \
        const int pid_ = die::g_prof_override >= 0 ? die::g_prof_override : (id);               \
        if (die::g_prof_on) die::prof_mark(pid_, (st), 0);                                       \
        __VA_ARGS__;                                                                             \
        if (die::g_prof_on) die::prof_mark(pid_, (st), 1);                                       \
    } while (0)
