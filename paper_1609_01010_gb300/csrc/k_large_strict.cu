// k_large_strict.cu -- three-kernel product path instantiated for the
// word-bound (2^30 < p < 2^31) arithmetic regime.
#include "k_large.cuh"

namespace pm {

cudaError_t launch_large_strict(const LargeDesc &d, Schedule sch, ModParams m, TwTables tw, cudaStream_t st,
                              cudaEvent_t *ev) {
    return launch_large_t<Arith<false>>(d, sch, m, tw, st, ev);
}

}  // namespace pm
