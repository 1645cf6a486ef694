// k_cols.cu -- column-stage kernels of the three-kernel path.
//
// Compiled once per variant by build.py with
//   PM_LAZY (1: p < 2^30 regime, 0: word-bound), PM_FWD (1: TFT column
//   stage, 0: ITFT column stage), PM_C (tile width 8 or 128; 32-column tiles run the kernels of
//   k_cols_tma.cu) and
//   PM_COL_FN (the name of the launcher this variant defines),
// so the instantiations (one kernel per column depth t = 1..11) compile in
// parallel.
#include "k_large.cuh"

#if !defined(PM_LAZY) || !defined(PM_FWD) || !defined(PM_C) || !defined(PM_COL_FN)
#error "k_cols.cu is compiled per variant: define PM_LAZY, PM_FWD, PM_C and PM_COL_FN"
#endif

namespace pm {

cudaError_t PM_COL_FN(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    return launch_col_t<Arith<(PM_LAZY != 0)>, PM_C, (PM_FWD != 0)>(d, m, tw, st);
}

}  // namespace pm
