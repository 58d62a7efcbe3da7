// The walker update for persistent launches (PERSIST = true), no tunnelling bookkeeping: the kernels of walker_chain.cuh
// instantiated with TUN = false, PERSIST = true.  A translation unit of its
// own, so that it compiles in parallel with the other flavours.
#include "walker_chain.cuh"

namespace mucal {

const void *walker_update_fn_persist(const LaunchShape &shape)
{
    return walker_update_fn_t<false, true>(shape);
}

void walker_update_persist_fns(const void *(&fns)[kWalkerUpdateFns]) { walker_update_fns<false, true>(fns); }

}  // namespace mucal
