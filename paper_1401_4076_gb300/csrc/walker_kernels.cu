// CUDA kernels of libmucal: initial placement, the walker update of the
// parallel multicanonical method (Sec. 2) for the lattice gas of Eq. 5
// without tunnelling bookkeeping (the device code is in walker_chain.cuh),
// the device-side histogram sum of Eq. 2, the replica exchange of the
// tempering runs and the allocation-free entry point.
//
// Target: sm_103a (GB300).
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda.h>
#include <cuda_runtime.h>

#include "mucal.h"
#include "mucal_internal.h"
#include "walker_chain.cuh"

namespace mucal {
namespace {
// ---------------------------------------------------------------------------
// Initial placement.
// ---------------------------------------------------------------------------
template <typename IdxT>
__global__ void fill_identity(SysParams p)
{
    const size_t total = (size_t)p.n_walkers * (size_t)p.V;
    IdxT *S = reinterpret_cast<IdxT *>(p.S);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x)
        S[i] = (IdxT)(i % (size_t)p.V);
}

// Partial Fisher-Yates from the init stream (counter (j/4 lo, j/4 hi, 0, 1),
// word j%4), then the bitset and a full energy count over the particles,
// looking in the +1 direction of every axis so each bond counts once.
template <int D, typename IdxT>
__device__ void init_one(const SysParams &p, int w)
{
    IdxT *S = walker_S<IdxT>(p, w);
    const uint64_t seed = p.seed_base + (uint64_t)w;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t V = (uint32_t)p.V;
    uint4 r = make_uint4(0, 0, 0, 0);
    for (uint32_t j = 0; j < (uint32_t)p.N; ++j) {
        if ((j & 3u) == 0) r = philox10(make_uint4(j >> 2, 0u, 0u, 1u), k0, k1);
        const uint32_t word = (j & 3u) == 0 ? r.x : (j & 3u) == 1 ? r.y : (j & 3u) == 2 ? r.z : r.w;
        const uint32_t idx = j + __umulhi(word, V - j);
        const IdxT tmp = S[j];
        S[j] = S[idx];
        S[idx] = tmp;
    }
    uint32_t *bits = p.bits + (size_t)w * (size_t)p.words;
    for (uint32_t j = 0; j < (uint32_t)p.N; ++j) {
        const uint32_t s = S[j];
        bits[s >> 5] |= 1u << (s & 31u);
    }
    int pairs = 0;
    for (uint32_t j = 0; j < (uint32_t)p.N; ++j) {
        uint32_t nb[2 * D];
        neighbours<D>(p, (uint32_t)S[j], nb);
#pragma unroll
        for (int k = 0; k < D; ++k) pairs += (int)occupied(bits, nb[2 * k + 1]);
    }
    p.E[w] = -pairs;
}

__global__ void init_walkers_kernel(const SysParams *__restrict__ sys, int s)
{
    const SysParams &p = sys[s];
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= p.n_walkers) return;
    if (p.d == 2) {
        if (p.idx16) init_one<2, uint16_t>(p, w); else init_one<2, uint32_t>(p, w);
    } else {
        if (p.idx16) init_one<3, uint16_t>(p, w); else init_one<3, uint32_t>(p, w);
    }
}

// ---------------------------------------------------------------------------
// H(E) = sum_j H_j(E) (Eq. 2).  Block (x: 256 bins, y: a chunk of walkers);
// each thread sums its bin over the chunk (coalesced across the bins) and
// adds the partial sum to H with one 64-bit atomic.
// ---------------------------------------------------------------------------
constexpr int kReduceWalkers = 64;

__global__ void hist_reduce_kernel(SysParams p)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.n_bins) return;
    const int w0 = blockIdx.y * kReduceWalkers;
    const int w1 = min(w0 + kReduceWalkers, p.hist_rows);
    unsigned long long sum = 0;
    const unsigned long long *h = p.hist + (size_t)w0 * (size_t)p.n_bins + b;
    for (int w = w0; w < w1; ++w, h += p.n_bins) sum += *h;
    if (sum) atomicAdd(p.H + b, sum);
}

// ---------------------------------------------------------------------------
// Replica exchange (parallel tempering): systems k and k+1 (k = parity,
// parity + 2, ...; blockIdx.y picks the pair) are copies of one lattice at
// canonical weights; walker w of the two exchanges configurations with
// probability min(1, exp((beta_k - beta_k+1)(E_k - E_k+1))), decided as
// T == 0xFFFFFFFF || r < T on a per-pair threshold row indexed by
// E_k - E_k+1 + n_bins - 1.  r = word 0 of Philox with walker w's key of
// system k and counter (round, 0, 0, 2).  Thread 0 decides; the block swaps
// bitset words, site lists and energies.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void block_swap_t(T *x, T *y, size_t n)
{
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        const T t = x[i];
        x[i] = y[i];
        y[i] = t;
    }
}

// Swap two byte ranges of even length with the widest accesses their
// alignment allows (16 bytes for the site lists and bitsets of most lattices).
__device__ __forceinline__ void block_swap(void *x, void *y, size_t bytes)
{
    const uintptr_t al = (uintptr_t)x | (uintptr_t)y | (uintptr_t)bytes;
    if ((al & 15) == 0)
        block_swap_t(static_cast<uint4 *>(x), static_cast<uint4 *>(y), bytes / 16);
    else if ((al & 3) == 0)
        block_swap_t(static_cast<uint32_t *>(x), static_cast<uint32_t *>(y), bytes / 4);
    else
        block_swap_t(static_cast<uint16_t *>(x), static_cast<uint16_t *>(y), bytes / 2);
}

__global__ void exchange_kernel(const SysParams *__restrict__ sys, int n_sys, int parity,
                                uint32_t round, const uint32_t *__restrict__ thr, int width,
                                unsigned long long *accepted)
{
    const int k = 2 * (int)blockIdx.y + parity;
    if (k + 1 >= n_sys) return;
    const SysParams &a = sys[k];
    const SysParams &b = sys[k + 1];
    __shared__ int take;
    for (int w = blockIdx.x; w < a.n_walkers; w += gridDim.x) {
        if (threadIdx.x == 0) {
            const uint64_t seed = a.seed_base + (uint64_t)w;
            const uint4 r = philox10(make_uint4(round, 0u, 0u, 2u), (uint32_t)seed, (uint32_t)(seed >> 32));
            const int ea = a.E[w], eb = b.E[w];
            const int idx = ea - eb + (width - 1) / 2;
            const uint32_t T = (idx >= 0 && idx < width) ? thr[(size_t)k * width + idx] : 0u;
            take = (T == 0xFFFFFFFFu || r.x < T) ? 1 : 0;
            if (take) {
                a.E[w] = eb;
                b.E[w] = ea;
                atomicAdd(accepted + k, 1ull);
            }
        }
        __syncthreads();
        if (take) {
            const size_t ib = a.idx16 ? 2 : 4;
            block_swap(a.bits + (size_t)w * a.words, b.bits + (size_t)w * b.words,
                       (size_t)a.words * 4);
            block_swap(static_cast<char *>(a.S) + (size_t)w * a.V * ib,
                       static_cast<char *>(b.S) + (size_t)w * b.V * ib, (size_t)a.V * ib);
        }
        __syncthreads();   // take is rewritten for the next walker
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_exchange(const SysParams *dev_sys, int n_sys, int n_walkers, int parity,
                            uint32_t round, const uint32_t *thr, int width,
                            unsigned long long *accepted, cudaStream_t stream)
{
    const int pairs = (n_sys - parity) / 2;
    if (pairs <= 0) return cudaSuccess;
    dim3 grid((unsigned)(n_walkers < 4096 ? n_walkers : 4096), (unsigned)pairs);
    exchange_kernel<<<grid, 128, 0, stream>>>(dev_sys, n_sys, parity, round, thr, width, accepted);
    return cudaGetLastError();
}

cudaError_t launch_fill_identity(const SysParams *host_sys, const SysParams *dev_sys, int n_sys,
                                 cudaStream_t stream)
{
    (void)dev_sys;
    for (int s = 0; s < n_sys; ++s) {
        const SysParams &p = host_sys[s];
        const size_t total = (size_t)p.n_walkers * (size_t)p.V;
        const int threads = 256;
        size_t blocks = (total + threads - 1) / threads;
        if (blocks > 65536) blocks = 65536;
        if (p.idx16)
            fill_identity<uint16_t><<<(unsigned)blocks, threads, 0, stream>>>(p);
        else
            fill_identity<uint32_t><<<(unsigned)blocks, threads, 0, stream>>>(p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_init_walkers(const SysParams *host_sys, const SysParams *dev_sys, int n_sys,
                                cudaStream_t stream)
{
    for (int s = 0; s < n_sys; ++s) {
        const int threads = 128;
        const int blocks = (host_sys[s].n_walkers + threads - 1) / threads;
        init_walkers_kernel<<<blocks, threads, 0, stream>>>(dev_sys, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t walker_update_max_smem(int *bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const void *fl[4][kWalkerUpdateFns];
    walker_update_fns<false, false>(fl[0]);
    walker_update_tunnel_fns(fl[1]);
    walker_update_persist_fns(fl[2]);
    walker_update_persist_tun_fns(fl[3]);
    const void *fns[4 * kWalkerUpdateFns];
    for (int f = 0; f < 4; ++f)
        for (int i = 0; i < kWalkerUpdateFns; ++i) fns[kWalkerUpdateFns * f + i] = fl[f][i];
    // the dynamic limit leaves room for the largest static shared array (the
    // thread kernel's tunnelling words)
    size_t max_static = 0;
    for (const void *fn : fns) {
        if (!fn) continue;   // flavour without a multi-commit kernel
        cudaFuncAttributes attr{};
        e = cudaFuncGetAttributes(&attr, fn);
        if (e != cudaSuccess) return e;
        max_static = attr.sharedSizeBytes > max_static ? attr.sharedSizeBytes : max_static;
    }
    *bytes -= (int)max_static;
    for (const void *fn : fns) {
        if (!fn) continue;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, *bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

const void *walker_update_fn(const LaunchShape &shape, bool tunnel)
{
    if (shape.persistent)
        return tunnel ? walker_update_fn_persist_tun(shape) : walker_update_fn_persist(shape);
    return tunnel ? walker_update_fn_tunnel(shape) : walker_update_fn_t<false, false>(shape);
}

cudaError_t walker_update_grid(const LaunchShape &shape, bool tunnel, int n_items, int *grid)
{
    *grid = n_items;
    if (!shape.persistent || n_items <= 0) return cudaSuccess;
    const void *fn = walker_update_fn(shape, tunnel);
    if (!fn) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn,
                                                          shape.walkers_per_block * shape.lanes,
                                                          shape.smem_bytes);
    if (e != cudaSuccess) return e;
    const long long resident = (long long)sms * (per_sm > 0 ? per_sm : 1);
    *grid = (int)(resident < n_items ? resident : n_items);
    return cudaSuccess;
}

cudaError_t launch_walker_update(const SysParams *dev_sys, const BlockWork *dev_work, int n_items,
                                 const LaunchShape &shape, uint64_t sweeps, uint32_t iteration,
                                 bool tunnel, int grid, int *next_item, cudaStream_t stream)
{
    if (n_items <= 0) return cudaSuccess;
    const void *fn = walker_update_fn(shape, tunnel);
    if (!fn) return cudaErrorInvalidValue;
    int *counter = shape.persistent ? next_item : nullptr;
    void *args[] = {(void *)&dev_sys, (void *)&dev_work, (void *)&sweeps, (void *)&iteration,
                    (void *)&n_items, (void *)&counter};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3((unsigned)(shape.walkers_per_block * shape.lanes)),
                            args, shape.smem_bytes, stream);
}

size_t thr_smem_words(const SysParams &p) { return thr_words_aligned(p); }

size_t field_smem_bytes(const SysParams &p) { return field_bytes(p); }

size_t thr_window_bytes(const SysParams &p) { return window_bytes(p); }

cudaError_t launch_hist_reduce(const SysParams *host_sys, const SysParams *dev_sys, int n_sys,
                               cudaStream_t stream)
{
    (void)dev_sys;
    for (int s = 0; s < n_sys; ++s) {
        const SysParams &p = host_sys[s];
        dim3 grid((p.n_bins + 255) / 256, (p.hist_rows + kReduceWalkers - 1) / kReduceWalkers);
        hist_reduce_kernel<<<grid, 256, 0, stream>>>(p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mucal

// ===========================================================================
// Allocation-free walker update.
//
// Some callers cannot allocate device memory: code that runs where
// cudaMalloc is not allowed or not wanted (inside a memory pool another
// framework owns, under a strict device-memory budget, or in a process whose
// allocator must not be touched between set-up and teardown).  For them this
// section offers one entry point that runs one iteration's walker update and
// histogram sum for a single system entirely on buffers the caller owns.
// Its scratch (the per-block histogram rows, the per-walker accept counters
// and an input-check flag) lives in the file-scope array below, which every
// GPU that loads this library holds until the process exits.
// ===========================================================================

namespace mucal {
namespace {

// Scratch layout, in 64-bit words: [check flag, padded to 32 words]
// [accept counters: kNoAllocMaxWalkers] [histogram rows: kNoAllocHistWords].
constexpr int kNoAllocMaxWalkers = 1 << 20;
constexpr size_t kNoAllocHistWords = (size_t)1 << 22;
constexpr size_t kNoAllocWords = 32 + (size_t)kNoAllocMaxWalkers + kNoAllocHistWords;
constexpr int kNoAllocLanes = 8;
constexpr int kNoAllocWalkersPerBlock = 32;

}  // namespace

}  // namespace mucal

static __device__ __align__(256) unsigned long long g_noalloc_scratch[mucal::kNoAllocWords];

namespace mucal {
namespace {

// Flags the call as invalid if an energy lies outside the window or a list
// entry outside the lattice; the walker update then does nothing.
__global__ void noalloc_check_kernel(SysParams p, unsigned long long *flag)
{
    const size_t total = (size_t)p.n_walkers * (size_t)p.V;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (size_t i = i0; i < (size_t)p.n_walkers; i += stride) {
        const int bin = p.E[i] - p.e_lo;
        if (bin < 0 || bin >= p.n_bins) atomicOr(flag, 1ull);
    }
    for (size_t i = i0; i < total; i += stride) {
        const uint32_t s = p.idx16 ? (uint32_t)reinterpret_cast<const uint16_t *>(p.S)[i]
                                   : reinterpret_cast<const uint32_t *>(p.S)[i];
        if (s >= (uint32_t)p.V) atomicOr(flag, 2ull);
    }
}

template <bool SB, bool ST>
__global__ void __launch_bounds__(kGroupMaxThreads, 1)
walker_update_noalloc(SysParams p, uint64_t sweeps, uint32_t iter, const unsigned long long *flag)
{
    extern __shared__ __align__(16) uint32_t smem[];
    if (*flag != 0) return;
    BlockWork wk;
    wk.sys = 0;
    wk.walker0 = blockIdx.x * kNoAllocWalkersPerBlock;
    wk.count = min(kNoAllocWalkersPerBlock, p.n_walkers - wk.walker0);
    wk.hist_row = blockIdx.x;
    const BlockSetup bs = block_setup(p, wk, smem, SB ? 1 : 0, ST ? 1 : 0);
    group_body<kNoAllocLanes, SB, ST ? kThrShared : kThrGlobal, false>(p, wk, smem, sweeps, iter);
    block_finish(bs, SB ? 1 : 0);
}

// Per-device set-up: the device address of the scratch array (the array's
// name is only a host-side stand-in in host code) and the shared-memory
// opt-in of the kernel variants.  Both belong to the device's context, so the
// set-up is remembered together with that context's unique id and redone
// when the context has been replaced (after cudaDeviceReset the next call
// finds a new id).
struct NoAllocDevice {
    unsigned long long *scratch = nullptr;
    int max_smem = 0;
    unsigned long long ctx_id = 0;
    bool ready = false;
};

std::mutex g_noalloc_mutex;
NoAllocDevice g_noalloc_dev[64];

// Unique id of the calling thread's current CUDA context, through the driver
// entry points the runtime hands out (the library does not link the driver
// library itself).  False when there is no current context or the entry
// points are unavailable; the set-up then runs again on the next call.
bool current_context_id(unsigned long long *id)
{
    using GetCurrentFn = CUresult (*)(CUcontext *);
    using GetIdFn = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
                cudaSuccess && q1 == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrentFn>(f1);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
                cudaSuccess && q2 == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetIdFn>(f2);
        looked_up = true;
    }
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

cudaError_t noalloc_setup(int dev, NoAllocDevice **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    NoAllocDevice &d = g_noalloc_dev[dev];
    unsigned long long id = 0;
    const bool known = current_context_id(&id);
    if (!d.ready || !known || id != d.ctx_id) {
        d.ready = false;
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int smem = 0;
        e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        const void *fns[] = {(const void *)walker_update_noalloc<true, true>,
                             (const void *)walker_update_noalloc<true, false>,
                             (const void *)walker_update_noalloc<false, true>,
                             (const void *)walker_update_noalloc<false, false>};
        for (const void *fn : fns) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        d.scratch = static_cast<unsigned long long *>(ptr);
        d.max_smem = smem;
        // the symbol lookup has made a context current if none was
        d.ready = current_context_id(&d.ctx_id);
    }
    *out = &d;
    return cudaSuccess;
}

thread_local std::string g_noalloc_error;

int noalloc_fail(int code, const std::string &msg)
{
    g_noalloc_error = msg;
    return code;
}

}  // namespace
}  // namespace mucal

extern "C" const char *mucal_run_walkers_noalloc_error(void)
{
    return mucal::g_noalloc_error.c_str();
}

extern "C" int mucal_run_walkers_noalloc(const mucal_system_desc *sys, int64_t sweeps,
                                         uint32_t iteration, uint32_t *bits, void *S, int32_t *E,
                                         const uint32_t *thr, uint64_t *H, void *cuda_stream)
{
    using namespace mucal;
    if (!sys || !bits || !S || !E || !thr || !H)
        return noalloc_fail(MUCAL_ERR_INVALID_ARG, "a buffer pointer is NULL");
    const mucal_system_desc &d = *sys;
    if ((d.d != 2 && d.d != 3) || d.L < 3 || d.L > 4096)
        return noalloc_fail(MUCAL_ERR_INVALID_ARG, "need d in {2,3} and 3 <= L <= 4096");
    const uint64_t V = d.d == 2 ? (uint64_t)d.L * d.L : (uint64_t)d.L * d.L * d.L;
    if (V > (1u << 24) || V * (uint64_t)d.L >= (1ull << 32))
        return noalloc_fail(MUCAL_ERR_INVALID_ARG, "lattice too large");
    if (d.N <= 0 || (uint64_t)d.N >= V) return noalloc_fail(MUCAL_ERR_INVALID_ARG, "need 0 < N < L^d");
    if (d.n_walkers <= 0 || d.n_walkers > kNoAllocMaxWalkers)
        return noalloc_fail(MUCAL_ERR_INVALID_ARG,
                            "n_walkers must be in [1, 1048576] for the allocation-free call");
    int e_lo = d.e_lo, e_hi = d.e_hi;
    if (e_lo == 0 && e_hi == 0) {
        e_lo = -d.d * d.N;
        e_hi = 0;
    } else if (e_lo < -d.d * d.N || e_hi > 0 || e_lo >= e_hi) {
        return noalloc_fail(MUCAL_ERR_INVALID_ARG, "window must satisfy -dN <= e_lo < e_hi <= 0");
    }
    if (sweeps < 1 || (uint64_t)sweeps * (uint64_t)d.N >= (1ull << 40))
        return noalloc_fail(MUCAL_ERR_INVALID_ARG, "need sweeps >= 1 and sweeps * N < 2^40");
    SysParams p{};
    p.d = d.d;
    p.L = d.L;
    p.N = d.N;
    p.V = (int32_t)V;
    p.L2 = d.L * d.L;
    p.e_lo = e_lo;
    p.n_bins = e_hi - e_lo + 1;
    p.width = 4 * d.d + 1;
    p.tstride = p.width;           // the caller's table has width words per row
    p.words = (int32_t)((V + 31) / 32);
    p.idx16 = V <= 65536 ? 1 : 0;
    p.n_walkers = d.n_walkers;
    p.magL = (uint32_t)(((1ull << 32) + (uint64_t)d.L - 1) / (uint64_t)d.L);
    p.seed_base = d.seed_base;
    p.tun_lo = -1;                 // no tunnelling bookkeeping (tun_state stays NULL)
    p.tun_hi = p.n_bins;
    const int blocks = (d.n_walkers + kNoAllocWalkersPerBlock - 1) / kNoAllocWalkersPerBlock;
    if ((size_t)blocks * (size_t)p.n_bins > kNoAllocHistWords)
        return noalloc_fail(MUCAL_ERR_INVALID_ARG,
                            "ceil(n_walkers / 32) * n_bins exceeds the 4194304 histogram entries "
                            "of the allocation-free scratch");
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    NoAllocDevice *nd = nullptr;
    if (ce == cudaSuccess) ce = noalloc_setup(dev, &nd);
    if (ce != cudaSuccess)
        return noalloc_fail(MUCAL_ERR_CUDA, std::string("set-up failed: ") + cudaGetErrorString(ce));
    unsigned long long *flag = nd->scratch;
    p.accepts = nd->scratch + 32;
    p.hist = nd->scratch + 32 + kNoAllocMaxWalkers;
    p.hist_rows = blocks;
    p.bits = bits;
    p.S = S;
    p.E = E;
    p.thr = thr;
    p.H = reinterpret_cast<unsigned long long *>(H);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t thr_bytes = thr_words_aligned(p) * 4;
    const size_t bits_bytes = (size_t)kNoAllocWalkersPerBlock * (size_t)p.words * 4;
    const bool sb = bits_bytes <= (size_t)nd->max_smem;
    const bool stt = thr_bytes + (sb ? bits_bytes : 0) <= (size_t)nd->max_smem;
    const size_t smem = (sb ? bits_bytes : 0) + (stt ? thr_bytes : 0);
    const int threads = kNoAllocWalkersPerBlock * kNoAllocLanes;
    // scratch keeps the previous call's contents: clear what must start at zero
    ce = cudaMemsetAsync(flag, 0, sizeof(unsigned long long), st);
    if (ce == cudaSuccess)
        ce = cudaMemsetAsync(p.hist, 0, (size_t)blocks * (size_t)p.n_bins * 8, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(p.H, 0, (size_t)p.n_bins * 8, st);
    if (ce == cudaSuccess) {
        noalloc_check_kernel<<<256, 256, 0, st>>>(p, flag);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) {
        if (sb && stt) walker_update_noalloc<true, true><<<blocks, threads, smem, st>>>(p, (uint64_t)sweeps, iteration, flag);
        else if (sb) walker_update_noalloc<true, false><<<blocks, threads, smem, st>>>(p, (uint64_t)sweeps, iteration, flag);
        else if (stt) walker_update_noalloc<false, true><<<blocks, threads, smem, st>>>(p, (uint64_t)sweeps, iteration, flag);
        else walker_update_noalloc<false, false><<<blocks, threads, smem, st>>>(p, (uint64_t)sweeps, iteration, flag);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) {
        dim3 grid((p.n_bins + 255) / 256, (p.hist_rows + kReduceWalkers - 1) / kReduceWalkers);
        hist_reduce_kernel<<<grid, 256, 0, st>>>(p);
        ce = cudaGetLastError();
    }
    unsigned long long bad = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&bad, flag, sizeof bad, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return noalloc_fail(MUCAL_ERR_CUDA, cudaGetErrorString(ce));
    if (bad & 1ull) return noalloc_fail(MUCAL_ERR_INVALID_ARG, "an energy E lies outside the window");
    if (bad & 2ull) return noalloc_fail(MUCAL_ERR_INVALID_ARG, "a list entry of S is not a lattice site");
    return MUCAL_OK;
}
