// The walker update with tunnelling bookkeeping (Sec. 4): the kernels of
// walker_chain.cuh instantiated with TUN = true.  A translation unit of its
// own, so that it compiles in parallel with walker_kernels.cu.
#include "walker_chain.cuh"

namespace mucal {

cudaError_t launch_walker_update_tunnel(const SysParams *dev_sys, const BlockWork *dev_work,
                                        int n_blocks, const LaunchShape &shape, uint64_t sweeps,
                                        uint32_t iteration, cudaStream_t stream)
{
    return launch_walker_update_t<true>(dev_sys, dev_work, n_blocks, shape, sweeps, iteration,
                                        stream);
}

void walker_update_tunnel_fns(const void *(&fns)[24]) { walker_update_fns<true>(fns); }

}  // namespace mucal
