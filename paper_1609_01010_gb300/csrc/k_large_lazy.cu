// k_large_lazy.cu -- three-kernel product path instantiated for the
// lazy (p < 2^30) arithmetic regime.
#include "k_large.cuh"

namespace pm {

cudaError_t launch_large_lazy(const LargeDesc &d, Schedule sch, ModParams m, TwTables tw, cudaStream_t st,
                              cudaEvent_t *ev) {
    return launch_large_t<Arith<true>>(d, sch, m, tw, st, ev);
}

}  // namespace pm
