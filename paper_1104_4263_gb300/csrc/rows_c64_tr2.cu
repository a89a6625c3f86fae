// Complex64 fast row passes with 2 rows per block (a tile height of the schedule; see
// matvec_kernels.cuh and dieop_autotune).
#include "rows_fast.cuh"

DIE_INSTANTIATE_ROWS_C64(2)
