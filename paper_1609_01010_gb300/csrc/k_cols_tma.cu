// k_cols_tma.cu -- the TMA-fed column-stage kernels (32-column tiles).
//
// Compiled once per variant by build.py with PM_LAZY (1: p < 2^30 regime,
// 0: word-bound), PM_FWD (1: TFT column stage, 0: ITFT column stage) and
// PM_TCOL_FN (the name of the launcher this variant defines), so the
// instantiations (one kernel per column depth t = 1..10) compile in parallel.
#include "k_cols_tma.cuh"

#if !defined(PM_LAZY) || !defined(PM_FWD) || !defined(PM_TCOL_FN)
#error "k_cols_tma.cu is compiled per variant: define PM_LAZY, PM_FWD and PM_TCOL_FN"
#endif

namespace pm {

cudaError_t PM_TCOL_FN(const LargeDesc &d, ModParams m, TwTables tw, const ColMaps &cm, cudaStream_t st) {
    return launch_tcol<Arith<(PM_LAZY != 0)>, (PM_FWD != 0)>(d, m, tw, cm, st);
}

}  // namespace pm
