// The walker update with tunnelling bookkeeping (Sec. 4): the kernels of
// walker_chain.cuh instantiated with TUN = true.  A translation unit of its
// own, so that it compiles in parallel with walker_kernels.cu.
#include "walker_chain.cuh"

namespace mucal {

const void *walker_update_fn_tunnel(const LaunchShape &shape)
{
    return walker_update_fn_t<true, false>(shape);
}

void walker_update_tunnel_fns(const void *(&fns)[kWalkerUpdateFns]) { walker_update_fns<true, false>(fns); }

}  // namespace mucal
