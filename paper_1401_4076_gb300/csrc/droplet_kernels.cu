// Largest-droplet measurement (Sec. 3): cluster labelling of every walker's
// configuration on the device.
//
// A droplet is a set of occupied sites connected through nearest-neighbour
// bonds of the periodic lattice.  One block labels one walker at a time
// (grid-stride over the walkers of a system) with a concurrent union-find
// over the particle sites S[0..N):
//   1. parent[s] = s for every particle site s;
//   2. for every particle s and every forward neighbour t of s that is
//      occupied, unite(s, t): roots are linked larger index -> smaller index
//      by compare-and-swap, so every parent pointer points to a smaller site
//      and the pointer chains cannot form cycles; finds halve their paths;
//   3. parent[s] = root(s) for every particle (full compression; these
//      finds only read, so that no stale ancestor overwrites a root);
//   4. each root's entry becomes a counter, marked by the top bit, and every
//      particle adds one to the counter of its root;
//   5. V_D = the largest counter (block reduction).
// The parent array (one uint32 per lattice site; only particle sites are
// touched) lives in shared memory when 4 V bytes fit into one block, else in
// a global scratch slice per block (at most 512 MiB for all blocks).  Thread
// 0 then stores V_D and adds (1, V_D, V_D^2) to the system's accumulators at
// the walker's energy bin.
//
// Every compare-and-swap loop has an iteration limit; hitting it (which a
// correct run never does: every failed swap means another thread linked a
// root) sets an error flag that the host reads.

#include <cstdint>

#include "mucal_internal.h"

namespace mucal {
namespace {

constexpr int kDropThreads = 256;
constexpr uint32_t kRootMark = 0x80000000u;
constexpr int kUniteLimit = 1 << 22;
constexpr size_t kDropScratchBytes = size_t(512) << 20;

__device__ __forceinline__ uint32_t particle_site(const SysParams &p, int w, int i)
{
    if (p.idx16) return static_cast<const uint16_t *>(p.S)[(size_t)w * p.V + i];
    return static_cast<const uint32_t *>(p.S)[(size_t)w * p.V + i];
}

// Forward neighbour of site s along axis k (periodic).
__device__ __forceinline__ uint32_t forward(const SysParams &p, uint32_t s, int k)
{
    const uint32_t L = (uint32_t)p.L;
    if (k == 0) return (s % L == L - 1) ? s + 1 - L : s + 1;
    if (k == 1) return ((s / L) % L == L - 1) ? s + L - (uint32_t)p.L2 : s + L;
    const uint32_t L2 = (uint32_t)p.L2;
    return (s / L2 == L - 1) ? s + L2 - (uint32_t)p.V : s + L2;
}

__device__ __forceinline__ uint32_t find_root(volatile uint32_t *P, uint32_t x)
{
    uint32_t px = P[x];
    while (px != x) {
        const uint32_t gp = P[px];
        if (gp != px) P[x] = gp;   // path halving: gp is still an ancestor of x
        x = px;
        px = gp;
    }
    return x;
}

// Root without writes.  The compression pass uses this: a path-halving write
// there could overwrite another thread's final "parent = root" with a mere
// ancestor, and the counting pass relies on every particle pointing at its root.
__device__ __forceinline__ uint32_t find_root_ro(volatile uint32_t *P, uint32_t x)
{
    uint32_t px = P[x];
    while (px != x) {
        x = px;
        px = P[x];
    }
    return x;
}

__device__ __forceinline__ bool unite(volatile uint32_t *P, uint32_t a, uint32_t b)
{
    for (int it = 0; it < kUniteLimit; ++it) {
        a = find_root(P, a);
        b = find_root(P, b);
        if (a == b) return true;
        if (a < b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        const uint32_t old = atomicCAS(const_cast<uint32_t *>(P + a), a, b);
        if (old == a) return true;
        a = old;   // a was linked meanwhile: continue from its new parent
    }
    return false;
}

template <bool SHARED>
__global__ void __launch_bounds__(kDropThreads)
droplet_kernel(SysParams p, DropletOut o, uint32_t *scratch)
{
    extern __shared__ uint32_t dyn_smem[];
    __shared__ uint32_t red[kDropThreads / 32];
    volatile uint32_t *P = SHARED ? dyn_smem : scratch + (size_t)blockIdx.x * (size_t)p.V;
    const int tid = threadIdx.x;
    bool ok = true;
    for (int w = blockIdx.x; w < p.n_walkers; w += gridDim.x) {
        const uint32_t *bits = p.bits + (size_t)w * p.words;
        for (int i = tid; i < p.N; i += kDropThreads) {
            const uint32_t s = particle_site(p, w, i);
            P[s] = s;
        }
        __syncthreads();
        for (int i = tid; i < p.N; i += kDropThreads) {
            const uint32_t s = particle_site(p, w, i);
            for (int k = 0; k < p.d; ++k) {
                const uint32_t t = forward(p, s, k);
                if ((bits[t >> 5] >> (t & 31u)) & 1u) ok &= unite(P, s, t);
            }
        }
        __syncthreads();
        for (int i = tid; i < p.N; i += kDropThreads) {
            const uint32_t s = particle_site(p, w, i);
            P[s] = find_root_ro(P, s);
        }
        __syncthreads();
        for (int i = tid; i < p.N; i += kDropThreads) {
            const uint32_t s = particle_site(p, w, i);
            if (P[s] == s) P[s] = kRootMark;
        }
        __syncthreads();
        for (int i = tid; i < p.N; i += kDropThreads) {
            const uint32_t s = particle_site(p, w, i);
            const uint32_t v = P[s];
            const uint32_t r = (v & kRootMark) ? s : v;
            atomicAdd(const_cast<uint32_t *>(P + r), 1u);
        }
        __syncthreads();
        uint32_t m = 0;
        for (int i = tid; i < p.N; i += kDropThreads) {
            const uint32_t v = P[particle_site(p, w, i)];
            if (v & kRootMark) m = max(m, v & ~kRootMark);
        }
        for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
        if ((tid & 31) == 0) red[tid >> 5] = m;
        __syncthreads();
        if (tid == 0) {
            uint32_t D = 0;
            for (int j = 0; j < kDropThreads / 32; ++j) D = max(D, red[j]);
            o.last[w] = (int32_t)D;
            const int b = p.E[w] - p.e_lo;
            if (b >= 0 && b < p.n_bins) {
                atomicAdd(o.acc + b, 1ull);
                atomicAdd(o.acc + p.n_bins + b, (unsigned long long)D);
                atomicAdd(o.acc + 2 * (size_t)p.n_bins + b, (unsigned long long)D * D);
            } else {
                atomicExch(o.err, 2);
            }
        }
        __syncthreads();   // P and red are reused by the next walker
    }
    if (!ok) atomicExch(o.err, 1);
}

}  // namespace

cudaError_t droplet_plan(const SysParams &p, DropletPlan *plan)
{
    int dev = 0, sms = 0, optin = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t need = (size_t)p.V * sizeof(uint32_t);
    const size_t static_bytes = (kDropThreads / 32) * sizeof(uint32_t);
    plan->shared = need + static_bytes <= (size_t)optin;
    if (plan->shared) {
        plan->smem = need;
        e = cudaFuncSetAttribute(droplet_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)need);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, droplet_kernel<true>,
                                                              kDropThreads, need);
        if (e != cudaSuccess) return e;
        plan->scratch_words = 0;
    } else {
        plan->smem = 0;
        per_sm = 2;
    }
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)sms * per_sm;
    if (!plan->shared) {
        // global parent arrays: at most kDropScratchBytes in total
        const long long fit = (long long)(kDropScratchBytes / need);
        blocks = fit < 1 ? 1 : (fit < blocks ? fit : blocks);
    }
    plan->grid = (int)(p.n_walkers < blocks ? p.n_walkers : blocks);
    if (plan->grid < 1) plan->grid = 1;
    if (!plan->shared) plan->scratch_words = (size_t)plan->grid * (size_t)p.V;
    return cudaSuccess;
}

cudaError_t launch_droplets(const SysParams &p, const DropletOut &o, const DropletPlan &plan,
                            uint32_t *scratch, cudaStream_t stream)
{
    if (plan.shared)
        droplet_kernel<true><<<plan.grid, kDropThreads, plan.smem, stream>>>(p, o, nullptr);
    else
        droplet_kernel<false><<<plan.grid, kDropThreads, 0, stream>>>(p, o, scratch);
    return cudaGetLastError();
}

}  // namespace mucal
