// The walker update for persistent launches with the tunnelling bookkeeping of Sec. 4: the kernels of walker_chain.cuh
// instantiated with TUN = true, PERSIST = true.  A translation unit of its
// own, so that it compiles in parallel with the other flavours.
#include "walker_chain.cuh"

namespace mucal {

const void *walker_update_fn_persist_tun(const LaunchShape &shape)
{
    return walker_update_fn_t<true, true>(shape);
}

void walker_update_persist_tun_fns(const void *(&fns)[kWalkerUpdateFns]) { walker_update_fns<true, true>(fns); }

}  // namespace mucal
