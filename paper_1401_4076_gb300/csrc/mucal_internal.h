// Internal definitions shared by the host driver and the CUDA kernels of
// libmucal.  Nothing here is part of the public C ABI (include/mucal.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mucal {

// Everything a kernel needs to know about one system (one lattice gas with
// its walkers), resident in device memory as an array indexed by system.
struct SysParams {
    int32_t d, L, N, V;        // dimension, linear size, particles, L^d
    int32_t L2;                // L*L
    int32_t e_lo, n_bins;      // energy window [e_lo, e_lo + n_bins - 1]
    int32_t width;             // 4d + 1 thresholds per bin
    int32_t tstride;           // words between threshold rows in thr: width rounded up to a
                               // multiple of 4, so that every row starts on 16 bytes
    int32_t words;             // 32-bit words of one occupation bitset, ceil(V/32)
    int32_t idx16;             // 1: S holds uint16 site indices, 0: uint32
    int32_t n_walkers;
    uint32_t magL;             // ceil(2^32 / L): floor(s / L) = umulhi(s, magL) for s*L < 2^32
    uint64_t seed_base;        // walker w has Philox key seed_base + w
    uint32_t *bits;            // [n_walkers][words] occupation n_i, bit s%32 of word s/32
    void *S;                   // [n_walkers][V] particle sites then empty sites
    int32_t *E;                // [n_walkers] current energy
    unsigned long long *hist;  // [rows][n_bins] histogram rows: one per walker (H_j(E)) when
                               // per-walker histograms are kept, else one per launch block
    int32_t hist_rows;         // rows in use for the current launch shape
    const uint32_t *thr;       // [n_bins][tstride] acceptance thresholds (entries width..tstride-1
                               // of a row unused)
    unsigned long long *accepts; // [n_walkers] accepted moves in the last iteration
    unsigned long long *H;     // [n_bins] summed histogram H(E) (Eq. 2)
    int32_t tun_lo, tun_hi;    // tunnelling ends as bins: a walker at bin <= tun_lo is at the
                               // low end, at bin >= tun_hi at the high end
    uint8_t *tun_state;        // [n_walkers] 0 = no end reached yet, 1 = low end last, 2 = high
                               // end last (NULL: no tunnelling bookkeeping)
    uint32_t *tun_count;       // [n_walkers] tunnelling events (end-to-end travels) so far
    unsigned int *err;         // set non-zero when a bounded wait of a walker kernel ran out
};

// Threshold-row window of the group and field kernels (threshold mode 2):
// each walker keeps kThrWindowRows consecutive rows of the table in shared
// memory as a ring indexed by bin mod kThrWindowRows, rows c - 15 .. c + 16
// around a centre c that follows the walker's energy.
constexpr int kThrWindowRows = 32;

// One block of the walker-update launch works on walkers
// [walker0, walker0 + count) of system sys.
struct BlockWork {
    int32_t sys;
    int32_t walker0;
    int32_t count;
    int32_t hist_row;   // this block's histogram row when rows are per block, else -1
};

// Walker-update kernels of one (tunnelling, persistent) flavour: the thread
// kernel in its shared-memory variants, the group kernel with the bitsets in
// shared or global memory and the thresholds in global memory, in shared
// memory or in a per-walker row window, and the field kernel with the three
// threshold modes.
constexpr int kWalkerUpdateFns = 4 + 5 * 2 * 3 + 5 * 3 + 4 * 6;   // last: multi-commit
                                                                // kernels (NULL where absent)

struct LaunchShape {
    int kernel;             // MUCAL_KERNEL_THREAD / _GROUP / _FIELD
    int lanes;              // lanes per walker
    int walkers_per_block;
    int bits_in_smem;
    int thr_in_smem;        // stage the system's threshold table in shared memory
    size_t smem_bytes;      // dynamic shared memory per block
    int persistent;         // resident blocks pull work items from a counter
    int thr_window;         // (group and field kernels, when the table is not in shared
                            // memory) keep a window of rows per walker in shared memory
    int multi_commit;       // (group and field kernels, 4+ lanes, no window, no tunnelling
                            // bookkeeping) several commits per round
};

// Kernel launchers (walker_kernels.cu).  All are asynchronous on `stream`.
cudaError_t launch_fill_identity(const SysParams *host_sys, const SysParams *dev_sys, int n_sys,
                                 cudaStream_t stream);
cudaError_t launch_init_walkers(const SysParams *host_sys, const SysParams *dev_sys, int n_sys,
                                cudaStream_t stream);
// The walker-update kernel of a launch shape; tunnel selects the flavour with
// the tunnelling bookkeeping (Sec. 4).  Its arguments are (const SysParams *,
// const BlockWork *, uint64_t sweeps, uint32_t iteration, int n_items,
// int *next_item).
const void *walker_update_fn(const LaunchShape &shape, bool tunnel);
// Blocks of a launch over n_items work items: n_items, or for a persistent
// shape the blocks that fit on the device at once (at most n_items).
cudaError_t walker_update_grid(const LaunchShape &shape, bool tunnel, int n_items, int *grid);
// Launch it on `grid` blocks; next_item: a device counter that is 0 at the
// start of the launch (used only by persistent shapes).
cudaError_t launch_walker_update(const SysParams *dev_sys, const BlockWork *dev_work, int n_items,
                                 const LaunchShape &shape, uint64_t sweeps, uint32_t iteration,
                                 bool tunnel, int grid, int *next_item, cudaStream_t stream);
// The other three flavours of the walker update, one translation unit each
// (walker_kernels_tun.cu, walker_kernels_persist.cu,
// walker_kernels_persist_tun.cu): the kernel of a launch shape and all
// kWalkerUpdateFns kernels of the flavour (for their shared-memory
// attributes).
const void *walker_update_fn_tunnel(const LaunchShape &shape);
void walker_update_tunnel_fns(const void *(&fns)[kWalkerUpdateFns]);
const void *walker_update_fn_persist(const LaunchShape &shape);
void walker_update_persist_fns(const void *(&fns)[kWalkerUpdateFns]);
const void *walker_update_fn_persist_tun(const LaunchShape &shape);
void walker_update_persist_tun_fns(const void *(&fns)[kWalkerUpdateFns]);
// Shared-memory layout of a walker-update block: [threshold table][bitsets]
// (group and thread kernels) or [threshold table][count fields] (field
// kernel).
size_t thr_smem_words(const SysParams &p);
// Shared-memory bytes of one walker's threshold-row window and its barrier.
size_t thr_window_bytes(const SysParams &p);
// Shared-memory bytes of one walker's neighbour-count field (field kernel).
size_t field_smem_bytes(const SysParams &p);
cudaError_t launch_hist_reduce(const SysParams *host_sys, const SysParams *dev_sys, int n_sys,
                               cudaStream_t stream);
cudaError_t walker_update_max_smem(int *bytes);

// Replica exchange between neighbouring systems of a tempering ladder
// (walker_kernels.cu): thr holds one row of `width` thresholds per pair.
cudaError_t launch_exchange(const SysParams *dev_sys, int n_sys, int n_walkers, int parity,
                            uint32_t round, const uint32_t *thr, int width,
                            unsigned long long *accepted, cudaStream_t stream);

// Largest-droplet measurement (droplet_kernels.cu).
struct DropletOut {
    unsigned long long *acc;   // [3][n_bins]: count, sum V_D, sum V_D^2 per energy bin
    int32_t *last;             // [n_walkers] V_D at the last measurement
    int *err;                  // set non-zero on a labelling or energy-range failure
};
struct DropletPlan {
    bool shared;               // parent array in shared memory (else global scratch)
    int grid;                  // blocks; each strides over the walkers
    size_t smem;               // dynamic shared memory per block
    size_t scratch_words;      // uint32 words of global scratch the launch needs
};
cudaError_t droplet_plan(const SysParams &p, DropletPlan *plan);
cudaError_t launch_droplets(const SysParams &p, const DropletOut &o, const DropletPlan &plan,
                            uint32_t *scratch, cudaStream_t stream);

// Forward pass of the seeding network with the 128x128 layer on tcgen05
// (mlp_tcgen05.cu): wq the bf16 parameter vector, X [B][4], y [B]; err is set
// non-zero if a tensor-core wait ran out.
cudaError_t mlp_forward_tcgen05(const void *wq, const float *X, float *y, int64_t B, int *err,
                                cudaStream_t stream);
// Gradients of the mean squared error against target[B] written to grad
// (fp32[17281]) and the loss to *loss, every contraction on tcgen05.  part
// holds mlp_train_tcgen05_partial_floats(B) floats: one row per CTA, summed
// in CTA order, so the result does not depend on the CTAs' finishing order.
size_t mlp_train_tcgen05_partial_floats(int64_t B);
cudaError_t mlp_train_tcgen05(const void *wq, const float *X, const float *target, int64_t B,
                              float *part, float *grad, float *loss, int *err, cudaStream_t stream);

// Error message of calls that have no context (mucal_host.cu).
void set_init_error(const char *msg);

}  // namespace mucal
