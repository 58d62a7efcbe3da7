// Device code of the walker update shared by the translation units that
// instantiate it: walker_kernels.cu (plain), walker_kernels_tun.cu (with
// tunnelling bookkeeping), walker_kernels_persist.cu and
// walker_kernels_persist_tun.cu (persistent launches).  Everything here has internal linkage; each unit
// gets its own copy of what it instantiates.
//
// The threshold rows a walker's acceptance test reads come from the table in
// global memory, from the whole table staged in shared memory, or (group and
// field kernels) from a per-walker window of rows in shared memory that bulk
// copies refill as the walker's energy moves (see ThrWindow).
//
// The walker update is integer work with a serial dependency per walker
// (each attempt reads the state the previous accepted attempt wrote), so it
// is bound by latency and issue slots, not by tensor cores or HBM.  Two
// kernels are provided:
//   walker_update_thread: one thread advances one walker;
//   walker_update_group:  a group of G lanes advances one walker.  The lanes
//     evaluate G consecutive attempts against the same state, then commit them
//     in order; after each accepted move the remaining lanes re-evaluate
//     against the updated state, so the chain is exactly the one-thread chain.
// TUN = true adds the tunnelling bookkeeping (Sec. 4): every energy a walker
// takes is compared with the two ends of SysParams::tun_lo/tun_hi.
// PERSIST = true makes the launch persistent (see next_work_item).  Each of
// the four (TUN, PERSIST) flavours is instantiated in a translation unit of
// its own so that they compile in parallel.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "mucal.h"
#include "mucal_internal.h"

namespace mucal {
namespace {

// Largest block of the group kernel: leaves up to 128 registers per thread.
constexpr int kGroupMaxThreads = 512;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// multiply-high/low on words 0 and 2, high halves xor-ed into words 1 and 3
// with the round key, key bumped by the Weyl increments after each round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// ---------------------------------------------------------------------------
// Periodic neighbours of site s on the L^D lattice, s = x + L y (+ L^2 z).
// Only x (and y in 3D) need a division; the outermost axis wraps by comparing
// s itself.  floor(s / L) = umulhi(s, ceil(2^32 / L)) holds since s*L < 2^32.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void neighbours(const SysParams &p, uint32_t s, uint32_t (&nb)[2 * D])
{
    const uint32_t L = (uint32_t)p.L;
    const uint32_t V = (uint32_t)p.V;
    const uint32_t q = __umulhi(s, p.magL);
    const uint32_t x = s - q * L;
    nb[0] = (x == 0) ? s + L - 1 : s - 1;
    nb[1] = (x == L - 1) ? s - (L - 1) : s + 1;
    if constexpr (D == 2) {
        nb[2] = (s < L) ? s + (V - L) : s - L;
        nb[3] = (s >= V - L) ? s - (V - L) : s + L;
    } else {
        const uint32_t L2 = (uint32_t)p.L2;
        const uint32_t q2 = __umulhi(q, p.magL);
        const uint32_t y = q - q2 * L;
        nb[2] = (y == 0) ? s + (L2 - L) : s - L;
        nb[3] = (y == L - 1) ? s - (L2 - L) : s + L;
        nb[4] = (s < L2) ? s + (V - L2) : s - L2;
        nb[5] = (s >= V - L2) ? s - (V - L2) : s + L2;
    }
}

__device__ __forceinline__ uint32_t occupied(const uint32_t *bits, uint32_t s)
{
    return (bits[s >> 5] >> (s & 31u)) & 1u;
}

template <typename IdxT>
__device__ __forceinline__ IdxT *walker_S(const SysParams &p, int w)
{
    return reinterpret_cast<IdxT *>(p.S) + (size_t)w * (size_t)p.V;
}

// Shared-memory words used by the threshold table of system p (rows of
// tstride words, a multiple of 4, so the bitsets behind it stay aligned).
__host__ __device__ __forceinline__ size_t thr_words_aligned(const SysParams &p)
{
    return (((size_t)p.n_bins * (size_t)p.tstride) + 3u) & ~(size_t)3u;
}

// Threshold modes of the group and field kernels: rows read from global
// memory, the whole table staged in shared memory, or a window of rows per
// walker in shared memory.
constexpr int kThrGlobal = 0;
constexpr int kThrShared = 1;
constexpr int kThrWindow = 2;

// Shared-memory bytes of one walker's threshold-row window (kThrWindowRows
// rows of tstride words) and of its 8-byte barrier.
__host__ __device__ __forceinline__ size_t window_bytes(const SysParams &p)
{
    return (size_t)kThrWindowRows * (size_t)p.tstride * 4u + 8u;
}

// Histogram row a walker records into: its own row when per-walker histograms
// are kept, otherwise its block's row.
__device__ __forceinline__ unsigned long long *hist_row(const SysParams &p, int w, int block_row)
{
    const int row = block_row >= 0 ? block_row : w;
    return p.hist + (size_t)row * (size_t)p.n_bins;
}

// Copy n words between global and shared memory, all threads cooperating.
__device__ __forceinline__ void block_copy_words(uint32_t *dst, const uint32_t *src, size_t n)
{
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Shared memory of a walker-update block: [threshold table | bitsets].  The
// block's walkers are contiguous in global memory, so the bitsets move as one
// coalesced copy in and out.
struct BlockSetup {
    const uint32_t *thr;
    uint32_t *gbits;     // first bitset of the block in global memory
    uint32_t *bits0;     // first bitset of the block where the kernel uses it
    size_t block_words;
};

__device__ __forceinline__ BlockSetup block_setup(const SysParams &p, const BlockWork &wk,
                                                  uint32_t *smem, int bits_in_smem,
                                                  int thr_in_smem)
{
    BlockSetup b;
    b.block_words = (size_t)wk.count * (size_t)p.words;
    b.gbits = p.bits + (size_t)wk.walker0 * (size_t)p.words;
    uint32_t *sb = smem;
    if (thr_in_smem) {
        block_copy_words(smem, p.thr, (size_t)p.n_bins * (size_t)p.tstride);
        sb = smem + thr_words_aligned(p);
        b.thr = smem;
    } else {
        b.thr = p.thr;
    }
    if (bits_in_smem) {
        block_copy_words(sb, b.gbits, b.block_words);
        b.bits0 = sb;
    } else {
        b.bits0 = b.gbits;
    }
    if (thr_in_smem || bits_in_smem) __syncthreads();
    return b;
}

__device__ __forceinline__ void block_finish(const BlockSetup &b, int bits_in_smem)
{
    if (bits_in_smem) {
        __syncthreads();
        block_copy_words(b.gbits, b.bits0, b.block_words);
    }
}

// ---------------------------------------------------------------------------
// G lanes per walker (G divides 32).  Lane j of a group owns attempt t0 + j of
// the current batch: it draws its random numbers, reads its particle and
// empty site, and prepares what evaluating them needs once (the words and bit
// positions of their 2*2d neighbours, or their places in a count field).
// Every round the lanes still pending evaluate dE and the acceptance against
// the walker's current state.  The first accepting lane f commits; pending
// lanes before it were rejected by that same state and are recorded at the
// current energy; lanes after it re-evaluate in the next round (their list
// entries are patched in registers when the commit moved the same list
// slot).  The chain is therefore exactly the one-thread chain.  A warp's
// groups step through the rounds in lock-step so no group diverges.
// ---------------------------------------------------------------------------
// Occupation-bit access for the group kernel.  In shared memory a neighbour
// is addressed by its 32-bit shared address, in global memory by a pointer;
// the bit position 32 reads as empty (used for the neighbour of b that is a).
template <bool SHARED>
struct BitAddr;

template <>
struct BitAddr<true> {
    using A = uint32_t;
    uint32_t base;
    __device__ __forceinline__ explicit BitAddr(const uint32_t *bits)
        : base((uint32_t)__cvta_generic_to_shared(bits)) {}
    __device__ __forceinline__ A at(uint32_t site) const { return base + ((site >> 5) << 2); }
    __device__ __forceinline__ static uint32_t load(A a)
    {
        uint32_t v;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
        return v;
    }
};

template <>
struct BitAddr<false> {
    using A = const uint32_t *;
    const uint32_t *base;
    __device__ __forceinline__ explicit BitAddr(const uint32_t *bits) : base(bits) {}
    __device__ __forceinline__ A at(uint32_t site) const { return base + (site >> 5); }
    __device__ __forceinline__ static uint32_t load(A a)
    {
        uint32_t v;
        asm volatile("ld.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
        return v;
    }
};

template <int D, bool SHARED>
struct NbSet {
    typename BitAddr<SHARED>::A addr[2 * D];
    uint32_t shift[2 * D];

    __device__ __forceinline__ void build(const SysParams &p, const BitAddr<SHARED> &ba, uint32_t s,
                                          uint32_t skip)
    {
        uint32_t nb[2 * D];
        neighbours<D>(p, s, nb);
#pragma unroll
        for (int i = 0; i < 2 * D; ++i) {
            addr[i] = ba.at(nb[i]);
            shift[i] = (nb[i] == skip) ? 32u : (nb[i] & 31u);
        }
    }

    __device__ __forceinline__ void load(uint32_t (&w)[2 * D]) const
    {
#pragma unroll
        for (int i = 0; i < 2 * D; ++i) w[i] = BitAddr<SHARED>::load(addr[i]);
    }

    __device__ __forceinline__ int count_from(const uint32_t (&w)[2 * D]) const
    {
        int n = 0;
#pragma unroll
        for (int i = 0; i < 2 * D; ++i) n += (int)(__funnelshift_rc(w[i], 0u, shift[i]) & 1u);
        return n;
    }

    __device__ __forceinline__ int count() const
    {
        uint32_t w[2 * D];
        load(w);
        return count_from(w);
    }
};

template <bool SHARED>
__device__ __forceinline__ uint32_t thr_load(const uint32_t *thr, int idx)
{
    if constexpr (SHARED) {
        uint32_t v;
        const uint32_t a = (uint32_t)__cvta_generic_to_shared(thr + idx);
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
        return v;
    } else {
        return __ldg(thr + idx);
    }
}

// ---------------------------------------------------------------------------
// Threshold-row window (kThrWindow).  A walker's acceptance test reads one
// row of the threshold table per round: the row of its current energy.  When
// the table does not fit in shared memory, every walker keeps the
// kThrWindowRows = 32 rows c - 15 .. c + 16 around a centre c in shared
// memory, as a ring indexed by row mod 32.  When the energy has moved more
// than 3 bins from c, the centre moves to it and the rows that enter the
// window are fetched with asynchronous bulk copies completing on the
// walker's memory barrier.  An energy step is at most 2d bins, so between
// two re-centrings the rounds read rows within 3 of c, which were all in the
// window before the last fetch (the fetched rows lie 7 or more away); the
// fetch of one re-centring is waited for at the next, before any of its rows
// can be read.  Device table rows are tstride = 12 (2D) or 16 (3D) words, so
// every row starts on 16 bytes as the bulk copy requires.  Waits are bounded:
// if one runs out the kernel records it in p.err and carries on.
// ---------------------------------------------------------------------------
constexpr uint32_t kWaitLimit = 1u << 20;

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (bulk-copy) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint32_t a)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t a, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok;
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completing on the barrier at mbar.
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                              uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}

struct ThrWindow {
    uint32_t ring = 0;           // shared byte address of the walker's ring of rows
    uint32_t mbar = 0;           // shared byte address of its barrier
    const uint32_t *table = nullptr;
    int n_rows = 0;
    uint32_t tstride = 0;        // words per row
    int c = 0;                   // centre of the window
    uint32_t phase = 0;          // parity of the barrier phase the next fetch completes
    bool pend = false;           // a fetch is in flight
    bool broken = false;         // a wait ran out: no further fetches or waits

    // Fetch rows [r0, r1] (clipped to the table) into their ring slots; the
    // leader lane issues the copies, every lane of the group records them.
    __device__ __forceinline__ void fetch(int r0, int r1, bool leader)
    {
        if (broken) return;
        r0 = r0 < 0 ? 0 : r0;
        r1 = r1 > n_rows - 1 ? n_rows - 1 : r1;
        if (r0 > r1) return;
        if (leader) {
            constexpr uint32_t NR = (uint32_t)kThrWindowRows;
            const uint32_t rowb = 4u * tstride;
            const uint32_t n = (uint32_t)(r1 - r0 + 1);
            const uint32_t s0 = (uint32_t)r0 & (NR - 1u);
            const uint32_t n1 = n < NR - s0 ? n : NR - s0;
            // earlier reads of the slots being replaced come before the copy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(mbar, n * rowb);
            bulk_copy_g2s(ring + s0 * rowb, table + (size_t)r0 * tstride, n1 * rowb, mbar);
            if (n > n1)
                bulk_copy_g2s(ring, table + (size_t)(r0 + (int)n1) * tstride, (n - n1) * rowb, mbar);
        }
        pend = true;
    }

    // Wait (bounded) for the fetch in flight, if any.  If the wait runs out
    // the failure is recorded in p.err and the window stops fetching (the
    // rounds then read stale rows; the host reports the iteration invalid).
    __device__ __forceinline__ void wait(const SysParams &p)
    {
        if (!pend) return;
        uint32_t ok = 0;
        for (uint32_t i = 0; i < kWaitLimit && !ok; ++i) ok = mbar_try_wait(mbar, phase);
        if (!ok) {
            atomicOr(p.err, 1u);
            broken = true;
            return;             // pend stays set: the end of the chain waits once more
        }
        phase ^= 1u;
        pend = false;
    }
};

// Broadcast a pair of list values from lane src: one shuffle when both fit
// in 16 bits, two otherwise.
template <typename IdxT>
__device__ __forceinline__ void shfl_pair(uint32_t x, uint32_t y, int src, uint32_t &xo, uint32_t &yo)
{
    if constexpr (sizeof(IdxT) == 2) {
        const uint32_t v = __shfl_sync(0xffffffffu, x | (y << 16), src);
        xo = v & 0xFFFFu;
        yo = v >> 16;
    } else {
        xo = __shfl_sync(0xffffffffu, x, src);
        yo = __shfl_sync(0xffffffffu, y, src);
    }
}

// ---------------------------------------------------------------------------
// Views of a walker's occupation for the group rounds.  build() takes the
// attempt (a, b) (a lane without one, valid false, evaluates site 0), load()
// reads the state the round evaluates, d4() + adj4() is 4 dE (adj4() is the
// part that depends on the attempt alone, so it joins the threshold row
// address), commit() applies the lane's move.
// ---------------------------------------------------------------------------

// Through the occupation bitset: dE counts the occupied neighbour bits of a
// and of b (a excluded from b's neighbours), a commit flips the two bits.
template <int D, bool SB>
struct BitView {
    uint32_t *bits;
    BitAddr<SB> ba;
    NbSet<D, SB> na, nb;
    uint32_t *wa_own, *wb_own;   // where this lane's own move would write if it commits
    uint32_t ma_own, mb_own;
    uint32_t wa[2 * D], wb[2 * D];

    __device__ __forceinline__ explicit BitView(uint32_t *b) : bits(b), ba(b) {}

    __device__ __forceinline__ void build(const SysParams &p, uint32_t a, uint32_t b, bool valid)
    {
        na.build(p, ba, valid ? a : 0u, 0xFFFFFFFFu);
        nb.build(p, ba, valid ? b : 0u, valid ? a : 0xFFFFFFFFu);
        wa_own = bits + (a >> 5);
        wb_own = bits + (b >> 5);
        ma_own = 1u << (a & 31u);
        mb_own = 1u << (b & 31u);
    }

    __device__ __forceinline__ void load()
    {
        na.load(wa);
        nb.load(wb);
    }

    __device__ __forceinline__ int d4() const { return 4 * (na.count_from(wa) - nb.count_from(wb)); }
    __device__ __forceinline__ int adj4() const { return 0; }

    __device__ __forceinline__ void commit() const
    {
        if constexpr (SB) {
            atomicAnd(wa_own, ~ma_own);
            atomicOr(wb_own, mb_own);
        } else {
            *wa_own &= ~ma_own;
            *wb_own |= mb_own;
        }
    }
};

// Through a local field (MUCAL_KERNEL_FIELD).  Every walker of the block
// keeps one byte per site in shared memory: c = 4 times the number of
// occupied neighbours of that site (0 .. 8d; times 4 so that a difference of
// counts is a byte offset into a threshold row).  An attempt's energy change
// is then (c[a] - c[b])/4 + [a is a neighbour of b] (a is still occupied when
// b is examined), two byte loads instead of the 2*2d occupation bits, and a
// commit subtracts 4 from the counts of a's neighbours and adds 4 to those
// of b's.  The field is built from the particle list when a block starts and
// the occupation bitset is rebuilt from the list when it ends; the bitset is
// not touched in between.
template <int D>
struct FieldView {
    uint32_t fbase;      // shared byte address of this walker's field
    uint32_t ca, cb;     // shared byte addresses of c[a] and c[b]
    int adj;             // 4 if b is a neighbour of a
    uint32_t ua[4 * D];  // shared word addresses of the 2*2d counts a commit changes
    uint32_t uv[4 * D];  // what the commit adds there: -4 or +4 in the site's byte
    uint32_t va, vb;     // c[a], c[b]

    __device__ __forceinline__ explicit FieldView(uint32_t f) : fbase(f) {}

    __device__ __forceinline__ void build(const SysParams &p, uint32_t a, uint32_t b, bool valid)
    {
        a = valid ? a : 0u;
        b = valid ? b : 0u;
        uint32_t na[2 * D], nb[2 * D];
        neighbours<D>(p, a, na);
        neighbours<D>(p, b, nb);
        ca = fbase + a;
        cb = fbase + b;
        adj = 0;
#pragma unroll
        for (int i = 0; i < 2 * D; ++i) {
            adj |= (na[i] == b) ? 4 : 0;
            ua[i] = fbase + (na[i] & ~3u);
            uv[i] = 0u - (4u << ((na[i] & 3u) << 3));
            ua[2 * D + i] = fbase + (nb[i] & ~3u);
            uv[2 * D + i] = 4u << ((nb[i] & 3u) << 3);
        }
    }

    __device__ __forceinline__ void load()
    {
        asm volatile("ld.shared.u8 %0, [%1];" : "=r"(va) : "r"(ca) : "memory");
        asm volatile("ld.shared.u8 %0, [%1];" : "=r"(vb) : "r"(cb) : "memory");
    }

    __device__ __forceinline__ int d4() const { return (int)va - (int)vb; }
    __device__ __forceinline__ int adj4() const { return adj; }

    // Byte counts stay in [0, 8d]: a decrement meets a count that includes
    // the leaving particle, so no borrow or carry crosses a byte.
    __device__ __forceinline__ void commit() const
    {
#pragma unroll
        for (int i = 0; i < 4 * D; ++i)
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(ua[i]), "r"(uv[i]) : "memory");
    }
};

// The rounds of one walker's chain on G lanes, on a view of its occupation
// (BitView or FieldView).  A later lane whose prefetched list slot a commit
// moved is found by comparing slot indices with the committing lane's (one
// more shuffle) when FIX_BY_SLOT, else by comparing sites; both find the
// same lanes, and which is faster is a matter of the compiled loop.
// TM is the threshold mode: kThrGlobal reads the rows from thr in global
// memory, kThrShared from thr staged in shared memory, kThrWindow from the
// walker's ring of rows at shared address ring_s with its barrier at mbar_s
// (thr then being the global table the ring is filled from).
template <int D, typename IdxT, int G, int TM, bool TUN, bool FIX_BY_SLOT, typename View>
__device__ __forceinline__ void chain_rounds(const SysParams &p, int w, bool active, View v,
                                             const uint32_t *thr, unsigned long long *hist,
                                             uint64_t A, uint32_t iter, uint32_t ring_s = 0u,
                                             uint32_t mbar_s = 0u)
{
    constexpr unsigned FULL = 0xffffffffu;
    constexpr unsigned GMASK = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
    const int lane = threadIdx.x & 31;
    const int j = lane & (G - 1);
    const int gbase = lane - j;
    const unsigned gm = GMASK << gbase;              // this group's lanes in a warp ballot
    const unsigned ltm = gm & ((1u << lane) - 1u);   // ... and those below this lane
    IdxT *S = walker_S<IdxT>(p, w);
    const uint32_t N = (uint32_t)p.N;
    const uint32_t holes = (uint32_t)(p.V - p.N);
    const uint64_t seed = p.seed_base + (uint64_t)w;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    int bin = active ? p.E[w] - p.e_lo : 0;
    // threshold rows as shared byte addresses (or byte offsets into the
    // global table): row of bin b, entry dE = 0, at rbase + row(b) * w4,
    // row(b) = b, or b mod kThrWindowRows in the walker's ring
    const uint32_t thr_s = TM == kThrShared ? (uint32_t)__cvta_generic_to_shared(thr)
                                            : (TM == kThrWindow ? ring_s : 0u);
    const uint32_t rbase = thr_s + 8u * D;
    const uint32_t w4 = 4u * (uint32_t)p.tstride;
    auto row_of = [](int b) -> uint32_t {
        return TM == kThrWindow ? ((uint32_t)b & (uint32_t)(kThrWindowRows - 1)) : (uint32_t)b;
    };
    ThrWindow tw;
    if constexpr (TM == kThrWindow) {
        tw.ring = ring_s;
        tw.mbar = mbar_s;
        tw.table = thr;
        tw.n_rows = p.n_bins;
        tw.tstride = (uint32_t)p.tstride;
        tw.c = bin;
        if (active) {
            if (j == 0) mbar_init(mbar_s, 1u);
            __syncwarp(gm);
            tw.fetch(bin - (kThrWindowRows / 2 - 1), bin + kThrWindowRows / 2, j == 0);
            tw.wait(p);
        }
    }
    // histogram entries are added per run of attempts at one energy: carry
    // holds the run's attempts from earlier batches, rs the warp lane of
    // this batch at which it started
    uint32_t carry = 0;
    uint32_t acc = 0;
    // tunnelling bookkeeping (TUN only), meaningful in lane j == 0: every
    // energy the walker takes is checked against the two ends
    const int tlo = TUN ? p.tun_lo : 0, thi = TUN ? p.tun_hi : 0;
    uint32_t tst = (TUN && active && p.tun_state) ? p.tun_state[w] : 0u;
    uint32_t tcnt = 0;
    auto tunnel = [&](int b_now) {
        if (b_now <= tlo) {
            tcnt += tst == 2u ? 1u : 0u;
            tst = 1u;
        } else if (b_now >= thi) {
            tcnt += tst == 1u ? 1u : 0u;
            tst = 2u;
        }
    };
    if constexpr (TUN) tunnel(bin);
    // the list reads of a batch are issued one batch early, and commits that
    // move a list slot such a read covers patch it.  With PF (G <= 8, where
    // a batch takes few rounds) the random numbers are drawn two batches
    // early and the list entries they select are prefetched into L2 then,
    // since the lists of all walkers can be larger than L2 (measured on
    // GB300: 3D L=32 +11 %, 2D L=64 +3 %; at G = 16 a loss of 6 %).
    constexpr bool PF = G <= 8;
    uint32_t kn = 0, mn = 0, an = 0, bn = 0, r2n = 0;   // the next batch
    uint32_t kq = 0, mq = 0, r2q = 0;                   // the batch after it (PF)
    auto draw = [&](uint64_t t0) {
        const uint64_t t = t0 + (uint64_t)j;
        if (active && t < A) {
            const uint4 r = philox10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), iter, 0u), k0, k1);
            if constexpr (PF) {
                kq = __umulhi(r.x, N);
                mq = __umulhi(r.y, holes);
                r2q = r.z;
                asm volatile("prefetch.L2 [%0];" ::"l"(S + kq));
                asm volatile("prefetch.L2 [%0];" ::"l"(S + N + mq));
            } else {
                kn = __umulhi(r.x, N);
                mn = __umulhi(r.y, holes);
                r2n = r.z;
                an = S[kn];
                bn = S[N + mn];
            }
        }
    };
    auto read = [&](uint64_t t0) {
        const uint64_t t = t0 + (uint64_t)j;
        if (active && t < A) {
            kn = kq;
            mn = mq;
            r2n = r2q;
            an = S[kn];
            bn = S[N + mn];
        }
    };
    draw(0);
    if constexpr (PF) {
        read(0);
        draw(G);
    }
    for (uint64_t t0 = 0; t0 < A; t0 += G) {
        const uint64_t left = A - t0;
        const int n_valid = left < (uint64_t)G ? (int)left : G;
        const bool valid = active && (j < n_valid);
        uint32_t k = kn, m = mn, a = an, b = bn;
        // acceptance T == 2^32 - 1 || r2 < T, as the single compare T >= r2p
        const uint32_t r2p = (r2n == 0xFFFFFFFFu) ? r2n : r2n + 1u;
        if constexpr (PF) {
            read(t0 + G);
            draw(t0 + 2 * G);
        } else {
            draw(t0 + G);
        }
        // lanes without an attempt evaluate site 0 so that every lane can
        // evaluate unconditionally
        v.build(p, a, b, valid);
        // where this lane's own move would write if it commits
        IdxT *pk = S + k;
        IdxT *pm = S + N + m;
        // state of the first round; later rounds load theirs right after the
        // previous commit, ahead of the bookkeeping
        v.load();
        uint32_t radj = rbase + (uint32_t)v.adj4();   // this attempt's adjacency joins the row address
        uint32_t rba = row_of(bin) * w4 + radj;
        bool pend = valid;                      // this lane's attempt is still undecided
        int rs = gbase;
        while (__any_sync(FULL, pend)) {
            const int d4 = v.d4();
            const uint32_t toff = rba + (uint32_t)d4;
            uint32_t T;
            if constexpr (TM != kThrGlobal) {
                asm volatile("ld.shared.u32 %0, [%1];" : "=r"(T) : "r"(toff));
            } else {
                T = __ldg(reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(thr) + toff));
            }
            const int de4 = d4 + v.adj4();   // 4 dE
            const bool accept = pend && T >= r2p;
            // pending lanes are the group's last ones, so the first accepting
            // lane commits, the pending lanes before it were rejected at the
            // current state and those after it (later) evaluate again
            const unsigned bal = __ballot_sync(FULL, accept) & gm;
            const bool commit = bal != 0u;             // the same in every lane of the group
            const bool later = (bal & ltm) != 0u;
            if (accept && !later) {
                v.commit();
                *pk = (IdxT)b;
                *pm = (IdxT)a;
                ++acc;                       // summed over the group's lanes at the end
            }
            // the committing warp lane (any lane when none commits: what the
            // shuffles below bring is then not used)
            const int src = (__ffs(bal) - 1) & 31;
            const int de_f = __shfl_sync(FULL, de4, src) >> 2;
            uint32_t a_f, b_f, k_f = 0, m_f = 0;
            shfl_pair<IdxT>(a, b, src, a_f, b_f);
            if constexpr (FIX_BY_SLOT) shfl_pair<IdxT>(k, m, src, k_f, m_f);
            __syncwarp(FULL);
            // the next round's state, loaded before the (rare) fix below,
            // which reloads it when it moves this lane's sites
            v.load();
            // the commit moved list slots k_f and N + m_f: slot k_f held a_f and
            // slot N + m_f held b_f, and every site sits in exactly one slot,
            // so a lane's slot k is k_f exactly when its (current) a is a_f
            const bool fix_a = later && (FIX_BY_SLOT ? k == k_f : a == a_f);
            const bool fix_b = later && (FIX_BY_SLOT ? m == m_f : b == b_f);
            if (fix_a || fix_b) {            // rare: no warp vote, the lane branches alone
                a = fix_a ? b_f : a;
                b = fix_b ? a_f : b;
                v.build(p, a, b, true);
                v.load();
                radj = rbase + (uint32_t)v.adj4();
            }
            pend = pend && later;
            // a move ends the run at the old energy: attempts rs .. src - 1 of
            // this batch (the committed one is the first at the new energy)
            const bool moved = commit && de_f != 0;
            const uint32_t cnt = carry + (uint32_t)(src - rs);
            if constexpr (TUN) {
                if (moved && j == 0) {
                    if (cnt) atomicAdd(hist + bin, (unsigned long long)cnt);
                    tunnel(bin + de_f);
                }
            } else {
                // (the test of cnt is not needed, but without it the
                // compiled loop is 4 % slower)
                if (moved && j == 0 && cnt) atomicAdd(hist + bin, (unsigned long long)cnt);
            }
            carry = moved ? 0u : carry;
            rs = moved ? src : rs;
            bin += moved ? de_f : 0;
            if constexpr (TM == kThrWindow) {
                // moved is the same in every lane of the group
                if (moved && (bin - tw.c > 3 || tw.c - bin > 3)) {
                    constexpr int LO = kThrWindowRows / 2 - 1, HI = kThrWindowRows / 2;
                    tw.wait(p);        // the previous fetch, before its rows can be read
                    if (bin > tw.c)
                        tw.fetch(max(tw.c + HI + 1, bin - LO), bin + HI, j == 0);
                    else
                        tw.fetch(bin - LO, min(tw.c - LO - 1, bin + HI), j == 0);
                    tw.c = bin;
                }
            }
            rba = row_of(bin) * w4 + radj;
            an = (commit && (FIX_BY_SLOT ? kn == k_f : an == a_f)) ? b_f : an;
            bn = (commit && (FIX_BY_SLOT ? mn == m_f : bn == b_f)) ? a_f : bn;
        }
        // the batch's attempts from rs on are at the final energy
        carry += (uint32_t)(gbase + n_valid - rs);
        if (carry >= 0x40000000u) {
            if (active && j == 0) atomicAdd(hist + bin, (unsigned long long)carry);
            carry = 0;
        }
    }
    if constexpr (TM == kThrWindow) {
        if (active) {
            // no copy may still write into the ring when the block moves on
            if (tw.broken) {
                uint32_t ok = 0;
                for (uint32_t i = 0; i < kWaitLimit && !ok; ++i) ok = mbar_try_wait(mbar_s, tw.phase);
            } else {
                tw.wait(p);
            }
            __syncwarp(gm);
            if (j == 0) mbar_inval(mbar_s);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (active && j == 0) {
        if (carry) atomicAdd(hist + bin, (unsigned long long)carry);
        p.E[w] = bin + p.e_lo;
        p.accepts[w] = acc;
        if (TUN && p.tun_state) {
            p.tun_state[w] = (uint8_t)tst;
            p.tun_count[w] += tcnt;
        }
    }
}

// ---------------------------------------------------------------------------
// Several commits per round (multi-commit rounds).  The rounds above commit
// one accepted move per round and let every later lane evaluate again against
// the new state.  A later lane whose two sites are not next to either site of
// a committed move keeps its energy change; only its threshold changes with
// the energy.  So after the first accepting lane f commits, the round goes on
// through the later lanes in attempt order: each step takes the decisions of
// the still-undecided lanes at the energy reached so far (every lane reads its
// thresholds in the 4d + 1 rows around the round's energy once per round and
// keeps the accept/reject outcomes as a bit mask, so a step reads no memory),
// the first of them that accepts commits next, the undecided lanes
// before it are rejected at that energy, and a lane stops the round (it and
// every later lane evaluate again in the next round) when a committed move
// touched one of its sites' neighbourhoods, moved one of its list slots, or
// took the energy out of the loaded rows.  Every decision is the one the
// serial chain takes, so the chain stays the one-thread chain.  Thresholds
// from global memory or a table staged in shared memory (not the window);
// no tunnelling bookkeeping.  A step issues more instructions than a
// one-commit round (the neighbourhood test alone is 8d compares), so the
// rounds pay off only where a round's loads are long: measured on GB300,
// 3D L = 32 at 4 lanes with thresholds in L2 +10 % (with the list entries
// read through L2 only), the field kernel and 16 lanes slower; the
// autotuner chooses per workload.
// ---------------------------------------------------------------------------
template <int D, typename IdxT, int G, int TM, typename View>
__device__ __forceinline__ void chain_rounds_mc(const SysParams &p, int w, bool active, View v,
                                                const uint32_t *thr, unsigned long long *hist,
                                                uint64_t A, uint32_t iter)
{
    static_assert(TM == kThrGlobal || TM == kThrShared, "multi-commit rounds read rows directly");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr unsigned GMASK = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
    constexpr int O = 2 * D;             // rows bin - O .. bin + O are loaded per round
    constexpr int NT = 2 * O + 1;
    const int lane = threadIdx.x & 31;
    const int j = lane & (G - 1);
    const int gbase = lane - j;
    const unsigned gm = GMASK << gbase;
    const unsigned me = 1u << lane;
    IdxT *S = walker_S<IdxT>(p, w);
    const uint32_t N = (uint32_t)p.N;
    const uint32_t holes = (uint32_t)(p.V - p.N);
    const uint64_t seed = p.seed_base + (uint64_t)w;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int nb = p.n_bins;
    int bin = active ? p.E[w] - p.e_lo : 0;
    const uint32_t thr_s = TM == kThrShared ? (uint32_t)__cvta_generic_to_shared(thr) : 0u;
    const uint32_t rbase = thr_s + 8u * D;
    const uint32_t w4 = 4u * (uint32_t)p.tstride;
    uint32_t carry = 0;
    uint32_t acc = 0;
    constexpr bool PF = G <= 8;
    // list entries are read through L2 only (ld.global.cg): measured on GB300,
    // 3D L = 32 at 4 lanes +7.5 % here (the one-commit rounds lose 2-10 % with it)
    uint32_t kn = 0, mn = 0, an = 0, bn = 0, r2n = 0;
    uint32_t kq = 0, mq = 0, r2q = 0;
    auto draw = [&](uint64_t t0) {
        const uint64_t t = t0 + (uint64_t)j;
        if (active && t < A) {
            const uint4 r = philox10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), iter, 0u), k0, k1);
            if constexpr (PF) {
                kq = __umulhi(r.x, N);
                mq = __umulhi(r.y, holes);
                r2q = r.z;
                asm volatile("prefetch.L2 [%0];" ::"l"(S + kq));
                asm volatile("prefetch.L2 [%0];" ::"l"(S + N + mq));
            } else {
                kn = __umulhi(r.x, N);
                mn = __umulhi(r.y, holes);
                r2n = r.z;
                an = __ldcg(S + kn);
                bn = __ldcg(S + N + mn);
            }
        }
    };
    auto read = [&](uint64_t t0) {
        const uint64_t t = t0 + (uint64_t)j;
        if (active && t < A) {
            kn = kq;
            mn = mq;
            r2n = r2q;
            an = __ldcg(S + kn);
            bn = __ldcg(S + N + mn);
        }
    };
    draw(0);
    if constexpr (PF) {
        read(0);
        draw(G);
    }
    for (uint64_t t0 = 0; t0 < A; t0 += G) {
        const uint64_t left = A - t0;
        const int n_valid = left < (uint64_t)G ? (int)left : G;
        const bool valid = active && (j < n_valid);
        uint32_t k = kn, m = mn, a = an, b = bn;
        const uint32_t r2p = (r2n == 0xFFFFFFFFu) ? r2n : r2n + 1u;
        if constexpr (PF) {
            read(t0 + G);
            draw(t0 + 2 * G);
        } else {
            draw(t0 + G);
        }
        v.build(p, a, b, valid);
        IdxT *pk = S + k;
        IdxT *pm = S + N + m;
        // the sites whose occupation this lane's energy change depends on:
        // the neighbours of a and of b
        uint32_t nbr[4 * D];
        auto neighbourhood = [&]() {
            uint32_t na[2 * D], nbb[2 * D];
            neighbours<D>(p, valid ? a : 0u, na);
            neighbours<D>(p, valid ? b : 0u, nbb);
#pragma unroll
            for (int i = 0; i < 2 * D; ++i) {
                nbr[i] = na[i];
                nbr[2 * D + i] = nbb[i];
            }
        };
        neighbourhood();
        v.load();
        uint32_t radj = rbase + (uint32_t)v.adj4();
        bool pend = valid;
        int rs = gbase;
        while (__any_sync(FULL, pend)) {
            const int d4 = v.d4();
            const int de4 = d4 + v.adj4();
            // bit o: this lane's move is accepted at the energy bin + o - O
            // (rows outside the table are never the walker's energy)
            uint32_t accm = 0u;
#pragma unroll
            for (int o = 0; o < NT; ++o) {
                const int rb = bin + o - O;
                const bool in = rb >= 0 && rb < nb;
                const uint32_t off = (uint32_t)(in ? rb : 0) * w4 + radj + (uint32_t)d4;
                uint32_t t;
                if constexpr (TM == kThrShared) {
                    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(t) : "r"(off));
                } else {
                    t = __ldg(reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(thr) + off));
                }
                accm |= (in && t >= r2p ? 1u : 0u) << o;
            }
            bool clean = pend;       // this lane's evaluation still holds
            bool refresh = false;    // a commit moved one of this lane's list slots
            int off = 0;             // energy change committed in this round
            bool stepping = (__ballot_sync(FULL, pend) & gm) != 0u;
            while (__any_sync(FULL, stepping)) {
                // (a clean lane has |off| <= O)
                const bool acc_now = stepping && pend && clean && ((accm >> ((off + O) & 31)) & 1u);
                const unsigned bal = __ballot_sync(FULL, acc_now) & gm;
                const unsigned unc = __ballot_sync(FULL, stepping && pend && !clean) & gm;
                const unsigned fbit = bal & (0u - bal);
                const unsigned ubit = unc & (0u - unc);
                // an undecided lane before the next acceptance that cannot be
                // decided here stops the round: it and all later lanes go again
                const bool stop = stepping && unc != 0u && (bal == 0u || ubit < fbit);
                // no acceptance among clean undecided lanes: all rejected here
                const bool none = stepping && !stop && bal == 0u;
                const bool step = stepping && !stop && !none;
                if (stop) pend = pend && me >= ubit;
                if (none) pend = false;
                const int f = step ? (__ffs(bal) - 1) : lane;
                if (step && lane == f) {
                    v.commit();
                    *pk = (IdxT)b;
                    *pm = (IdxT)a;
                    ++acc;
                }
                const int de_f = __shfl_sync(FULL, de4, f) >> 2;
                uint32_t a_f, b_f, k_f, m_f;
                shfl_pair<IdxT>(a, b, f, a_f, b_f);
                shfl_pair<IdxT>(k, m, f, k_f, m_f);
                if (step) {
                    // a move ends the run at the energy before it
                    const bool moved = de_f != 0;
                    const uint32_t cnt = carry + (uint32_t)(f - rs);
                    if (moved && j == 0 && cnt) atomicAdd(hist + bin + off, (unsigned long long)cnt);
                    carry = moved ? 0u : carry;
                    rs = moved ? f : rs;
                    off += de_f;
                    pend = pend && lane > f;
                    // list slots the commit moved
                    const bool fa = pend && k == k_f;
                    const bool fb = pend && m == m_f;
                    if (fa || fb) {
                        a = fa ? b_f : a;
                        b = fb ? a_f : b;
                        refresh = true;
                        clean = false;
                    }
                    // occupation the commit changed next to this lane's sites
                    bool hit = false;
#pragma unroll
                    for (int i = 0; i < 4 * D; ++i) hit |= (nbr[i] == a_f) | (nbr[i] == b_f);
                    clean = clean && !hit;
                    // energies beyond the loaded rows are decided next round
                    if (off > O || off < -O) clean = false;
                    // the next batch's list reads see the moved slots
                    an = (kn == k_f) ? b_f : an;
                    bn = (mn == m_f) ? a_f : bn;
                }
                stepping = step;
                __syncwarp(FULL);
            }
            bin += off;
            if (refresh) {
                v.build(p, a, b, true);
                radj = rbase + (uint32_t)v.adj4();
                pk = S + k;
                pm = S + N + m;
                neighbourhood();
            }
            v.load();
        }
        carry += (uint32_t)(gbase + n_valid - rs);
        if (carry >= 0x40000000u) {
            if (active && j == 0) atomicAdd(hist + bin, (unsigned long long)carry);
            carry = 0;
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (active && j == 0) {
        if (carry) atomicAdd(hist + bin, (unsigned long long)carry);
        p.E[w] = bin + p.e_lo;
        p.accepts[w] = acc;
    }
}

// ---------------------------------------------------------------------------
// One thread, one walker: A attempts in order, software-pipelined.  The
// random numbers and list reads of the next PF attempts are in flight in a
// register ring while the current attempt is evaluated (the slot just
// consumed is refilled while its occupation words are being read); a commit patches the
// in-flight list reads it invalidates (same list slot).  The histogram is
// kept as a run length (current bin, count) and added to the histogram row
// only when the energy changes, which records exactly one entry per attempt.
// ---------------------------------------------------------------------------
constexpr int kThreadPipe = 6;

template <int D, typename IdxT, bool SB, bool ST, bool TUN>
__device__ __forceinline__ void chain_thread(const SysParams &p, int w, uint32_t *bits,
                                             const uint32_t *thr, unsigned long long *hist,
                                             uint64_t A, uint32_t iter, uint32_t *s_tun)
{
    constexpr int PF = kThreadPipe;
    IdxT *S = walker_S<IdxT>(p, w);
    const BitAddr<SB> ba(bits);
    const uint32_t N = (uint32_t)p.N;
    const uint32_t holes = (uint32_t)(p.V - p.N);
    const uint64_t seed = p.seed_base + (uint64_t)w;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int width = p.tstride;      // words between threshold rows
    int bin = p.E[w] - p.e_lo;
    int row = bin * width + 2 * D;
    uint32_t run = 0;
    uint32_t acc = 0;
    // tunnelling bookkeeping (TUN only): every energy the walker takes is
    // checked against the two ends.  State in bits 0-1, events in the bits
    // above, kept in this thread's word of the kernel's shared array s_tun
    // (the pipeline ring already fills the registers), touched on moves only.
    if constexpr (TUN) s_tun[threadIdx.x] = p.tun_state ? p.tun_state[w] : 0u;
    auto tunnel = [&](int b_now) {
        if (b_now <= p.tun_lo) {
            const uint32_t tun = s_tun[threadIdx.x];
            s_tun[threadIdx.x] = (tun & ~3u) + ((tun & 3u) == 2u ? 4u : 0u) + 1u;
        } else if (b_now >= p.tun_hi) {
            const uint32_t tun = s_tun[threadIdx.x];
            s_tun[threadIdx.x] = (tun & ~3u) + ((tun & 3u) == 1u ? 4u : 0u) + 2u;
        }
    };
    if constexpr (TUN) tunnel(bin);
    // ra/rb receive the in-flight list reads; a commit that moves a slot an
    // in-flight read covers records the new value in fa/fb instead of
    // touching ra/rb, so that it never waits for the read to land
    constexpr uint32_t NONE = 0xFFFFFFFFu;
    uint32_t rk[PF], rm[PF], rr[PF], ra[PF], rb[PF], fa[PF], fb[PF];
#pragma unroll
    for (int s = 0; s < PF; ++s) {
        rk[s] = NONE;
        rm[s] = NONE;
        fa[s] = NONE;
        fb[s] = NONE;
        rr[s] = ra[s] = rb[s] = 0u;
        const uint64_t t = (uint64_t)s;
        if (t < A) {
            const uint4 r = philox10(make_uint4((uint32_t)t, 0u, iter, 0u), k0, k1);
            rk[s] = __umulhi(r.x, N);
            rm[s] = __umulhi(r.y, holes);
            rr[s] = r.z;
            ra[s] = S[rk[s]];
            rb[s] = S[N + rm[s]];
        }
    }
    for (uint64_t t0 = 0; t0 < A; t0 += PF) {
#pragma unroll
        for (int s = 0; s < PF; ++s) {
            const uint64_t t = t0 + (uint64_t)s;
            if (t < A) {
                const uint32_t a = fa[s] != NONE ? fa[s] : ra[s];
                const uint32_t b = fb[s] != NONE ? fb[s] : rb[s];
                const uint32_t k = rk[s], m = rm[s], r2 = rr[s];
                NbSet<D, SB> na, nb;
                na.build(p, ba, a, 0xFFFFFFFFu);
                nb.build(p, ba, b, a);
                uint32_t wa[2 * D], wb[2 * D];
                na.load(wa);
                nb.load(wb);
                // while the occupation words are in flight, refill this slot
                // with attempt t + PF (its list reads are patched below if this
                // attempt's commit moves the same slot)
                const uint64_t tn = t + PF;
                rk[s] = NONE;
                rm[s] = NONE;
                fa[s] = NONE;
                fb[s] = NONE;
                if (tn < A) {
                    const uint4 r = philox10(make_uint4((uint32_t)tn, (uint32_t)(tn >> 32), iter, 0u),
                                             k0, k1);
                    rk[s] = __umulhi(r.x, N);
                    rm[s] = __umulhi(r.y, holes);
                    rr[s] = r.z;
                    ra[s] = S[rk[s]];
                    rb[s] = S[N + rm[s]];
                }
                const int de = na.count_from(wa) - nb.count_from(wb);
                const uint32_t T = thr_load<ST>(thr, row + de);
                if (T == 0xFFFFFFFFu || r2 < T) {
                    bits[a >> 5] &= ~(1u << (a & 31u));
                    bits[b >> 5] |= 1u << (b & 31u);
                    S[k] = (IdxT)b;
                    S[N + m] = (IdxT)a;
#pragma unroll
                    for (int q = 0; q < PF; ++q) {
                        fa[q] = (rk[q] == k) ? b : fa[q];
                        fb[q] = (rm[q] == m) ? a : fb[q];
                    }
                    ++acc;
                    if (de != 0) {
                        if (run) atomicAdd(hist + bin, (unsigned long long)run);
                        bin += de;
                        row += de * width;
                        run = 0;
                        if constexpr (TUN) tunnel(bin);
                    }
                }
                ++run;
                if (run == 0x80000000u) {
                    atomicAdd(hist + bin, (unsigned long long)run);
                    run = 0;
                }
            }
        }
    }
    if (run) atomicAdd(hist + bin, (unsigned long long)run);
    p.E[w] = bin + p.e_lo;
    p.accepts[w] = acc;
    if (TUN && p.tun_state) {
        const uint32_t tun = s_tun[threadIdx.x];
        p.tun_state[w] = (uint8_t)(tun & 3u);
        p.tun_count[w] += tun >> 2;
    }
}

// Work items of a launch: block b takes item b.  The persistent flavour
// (PERSIST) launches fewer blocks than items; a block that finishes an item
// takes the next one from the counter next_item (which starts at 0).
__device__ __forceinline__ int next_work_item(int *next_item, int *s_item)
{
    __syncthreads();   // the item's shared memory and *s_item are reused
    if (threadIdx.x == 0) *s_item = (int)gridDim.x + atomicAdd(next_item, 1);
    __syncthreads();
    return *s_item;
}

template <bool SB, bool ST, bool TUN, bool PERSIST>
__global__ void __launch_bounds__(kGroupMaxThreads, 1)
walker_update_thread(const SysParams *__restrict__ sys, const BlockWork *__restrict__ work,
                     uint64_t sweeps, uint32_t iter, int n_items, int *next_item)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ uint32_t s_tun[TUN ? kGroupMaxThreads : 1];   // tunnelling words, one per thread
    // one work item per block, or (PERSIST) items pulled from the counter
    auto item_body = [&](const BlockWork &wk) {
        const SysParams &p = sys[wk.sys];
        const BlockSetup bs = block_setup(p, wk, smem, SB ? 1 : 0, ST ? 1 : 0);
        const int lw = threadIdx.x;
        if (lw < wk.count) {
            const int w = wk.walker0 + lw;
            const uint32_t *thr = ST ? smem : p.thr;
            uint32_t *bits0 = SB ? smem + (ST ? thr_words_aligned(p) : 0)
                                 : p.bits + (size_t)wk.walker0 * (size_t)p.words;
            uint32_t *bits = bits0 + (size_t)lw * p.words;
            unsigned long long *hist = hist_row(p, w, wk.hist_row);
            const uint64_t A = sweeps * (uint64_t)p.N;
            if (p.d == 2) {
                if (p.idx16) chain_thread<2, uint16_t, SB, ST, TUN>(p, w, bits, thr, hist, A, iter, s_tun);
                else chain_thread<2, uint32_t, SB, ST, TUN>(p, w, bits, thr, hist, A, iter, s_tun);
            } else {
                if (p.idx16) chain_thread<3, uint16_t, SB, ST, TUN>(p, w, bits, thr, hist, A, iter, s_tun);
                else chain_thread<3, uint32_t, SB, ST, TUN>(p, w, bits, thr, hist, A, iter, s_tun);
            }
        }
        block_finish(bs, SB ? 1 : 0);
    };
    if constexpr (!PERSIST) {
        (void)n_items;
        (void)next_item;
        item_body(work[blockIdx.x]);
    } else {
        __shared__ int s_item;
        for (int item = blockIdx.x; item < n_items;) {
            item_body(work[item]);
            item = next_work_item(next_item, &s_item);
        }
    }
}

// Shared byte addresses of walker lw's threshold-row window and barrier: the
// block's windows start at the first 16-byte boundary at or after `after`
// (behind the bitsets or fields), one per walker of the launch shape, and
// the barriers follow them.
__device__ __forceinline__ void window_addrs(const SysParams &p, uint32_t after, int wpb, int lw,
                                             uint32_t &ring_s, uint32_t &mbar_s)
{
    const uint32_t base = (after + 15u) & ~15u;
    const uint32_t rb = (uint32_t)kThrWindowRows * 4u * (uint32_t)p.tstride;
    ring_s = base + (uint32_t)lw * rb;
    mbar_s = base + (uint32_t)wpb * rb + (uint32_t)lw * 8u;
}

template <int G, bool SB, int TM, bool TUN, bool MC = false>
__device__ __forceinline__ void group_body(const SysParams &p, const BlockWork &wk, uint32_t *smem,
                                           uint64_t sweeps, uint32_t iter)
{
    const int lw = threadIdx.x / G;
    const bool active = lw < wk.count;
    const int w = wk.walker0 + (active ? lw : 0);
    const uint32_t *thr = TM == kThrShared ? smem : p.thr;
    uint32_t *bits0 = SB ? smem + (TM == kThrShared ? thr_words_aligned(p) : 0)
                         : p.bits + (size_t)wk.walker0 * (size_t)p.words;
    uint32_t *bits = bits0 + (size_t)(active ? lw : 0) * p.words;
    unsigned long long *hist = hist_row(p, w, wk.hist_row);
    const uint64_t A = sweeps * (uint64_t)p.N;
    uint32_t ring_s = 0u, mbar_s = 0u;
    if constexpr (TM == kThrWindow) {
        const int wpb = (int)blockDim.x / G;
        const uint32_t after = (uint32_t)__cvta_generic_to_shared(smem) +
                               (SB ? (uint32_t)wpb * (uint32_t)p.words * 4u : 0u);
        window_addrs(p, after, wpb, active ? lw : 0, ring_s, mbar_s);
    }
    // slot compare for G = 4 and 8, site compare otherwise (measured on GB300:
    // 3D L=32 at 4 lanes 1.098e10 -> 1.119e10 with slot compare, which does not
    // wait for the next batch's list reads; the batch at 16 lanes 8.56e9 ->
    // 8.13e9, where the extra shuffle per round costs more)
    constexpr bool kSlot = (G == 4 || G == 8);
    if constexpr (MC) {
        if (p.d == 2) {
            if (p.idx16) chain_rounds_mc<2, uint16_t, G, TM>(p, w, active, BitView<2, SB>(bits), thr, hist, A, iter);
            else chain_rounds_mc<2, uint32_t, G, TM>(p, w, active, BitView<2, SB>(bits), thr, hist, A, iter);
        } else {
            if (p.idx16) chain_rounds_mc<3, uint16_t, G, TM>(p, w, active, BitView<3, SB>(bits), thr, hist, A, iter);
            else chain_rounds_mc<3, uint32_t, G, TM>(p, w, active, BitView<3, SB>(bits), thr, hist, A, iter);
        }
        return;
    }
    if (p.d == 2) {
        if (p.idx16) chain_rounds<2, uint16_t, G, TM, TUN, kSlot>(p, w, active, BitView<2, SB>(bits), thr, hist, A, iter, ring_s, mbar_s);
        else chain_rounds<2, uint32_t, G, TM, TUN, kSlot>(p, w, active, BitView<2, SB>(bits), thr, hist, A, iter, ring_s, mbar_s);
    } else {
        if (p.idx16) chain_rounds<3, uint16_t, G, TM, TUN, kSlot>(p, w, active, BitView<3, SB>(bits), thr, hist, A, iter, ring_s, mbar_s);
        else chain_rounds<3, uint32_t, G, TM, TUN, kSlot>(p, w, active, BitView<3, SB>(bits), thr, hist, A, iter, ring_s, mbar_s);
    }
}

template <int G, bool SB, int TM, bool TUN, bool PERSIST, bool MC = false>
__global__ void __launch_bounds__(kGroupMaxThreads, 1)
walker_update_group(const SysParams *__restrict__ sys, const BlockWork *__restrict__ work,
                    uint64_t sweeps, uint32_t iter, int n_items, int *next_item)
{
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int kTS = TM == kThrShared ? 1 : 0;
    if constexpr (!PERSIST) {
        // one work item per block
        (void)n_items;
        (void)next_item;
        const BlockWork wk = work[blockIdx.x];
        const SysParams &p = sys[wk.sys];
        const BlockSetup bs = block_setup(p, wk, smem, SB ? 1 : 0, kTS);
        group_body<G, SB, TM, TUN, MC>(p, wk, smem, sweeps, iter);
        block_finish(bs, SB ? 1 : 0);
    } else {
        __shared__ int s_item;
        for (int item = blockIdx.x; item < n_items;) {
            const BlockWork wk = work[item];
            const SysParams &p = sys[wk.sys];
            const BlockSetup bs = block_setup(p, wk, smem, SB ? 1 : 0, kTS);
            group_body<G, SB, TM, TUN, MC>(p, wk, smem, sweeps, iter);
            block_finish(bs, SB ? 1 : 0);
            item = next_work_item(next_item, &s_item);
        }
    }
}

// Bytes of one walker's neighbour-count field in shared memory (V rounded up
// to 16, so that every walker's field starts on a 16-byte boundary).
__host__ __device__ __forceinline__ size_t field_bytes(const SysParams &p)
{
    return ((size_t)p.V + 15u) & ~(size_t)15u;
}

// Counts of the block's walkers from their particle lists: zero the fields,
// then add 4 at every neighbour of every particle.
template <int D, typename IdxT>
__device__ __forceinline__ void field_build(const SysParams &p, const BlockWork &wk, uint32_t *fw)
{
    const size_t fwords = field_bytes(p) >> 2;
    const size_t total = (size_t)wk.count * fwords;
    for (size_t i = threadIdx.x; i < total; i += blockDim.x) fw[i] = 0u;
    __syncthreads();
    const uint32_t N = (uint32_t)p.N;
    const uint32_t n_sites = (uint32_t)wk.count * N;
    for (uint32_t i = threadIdx.x; i < n_sites; i += blockDim.x) {
        const uint32_t lw = i / N;
        const uint32_t s = walker_S<IdxT>(p, wk.walker0 + (int)lw)[i - lw * N];
        uint32_t nb[2 * D];
        neighbours<D>(p, s, nb);
        uint32_t *f = fw + (size_t)lw * fwords;
#pragma unroll
        for (int k = 0; k < 2 * D; ++k) atomicAdd(f + (nb[k] >> 2), 4u << ((nb[k] & 3u) << 3));
    }
    __syncthreads();
}

// The block's occupation bitsets from their particle lists, assembled in the
// (now unused) field memory and copied out.
template <typename IdxT>
__device__ __forceinline__ void field_finish(const SysParams &p, const BlockWork &wk, uint32_t *fw)
{
    __syncthreads();   // every chain is done with the fields; the list stores are visible
    const size_t words = (size_t)p.words;
    const size_t total = (size_t)wk.count * words;
    for (size_t i = threadIdx.x; i < total; i += blockDim.x) fw[i] = 0u;
    __syncthreads();
    const uint32_t N = (uint32_t)p.N;
    const uint32_t n_sites = (uint32_t)wk.count * N;
    for (uint32_t i = threadIdx.x; i < n_sites; i += blockDim.x) {
        const uint32_t lw = i / N;
        const uint32_t s = walker_S<IdxT>(p, wk.walker0 + (int)lw)[i - lw * N];
        atomicOr(fw + (size_t)lw * words + (s >> 5), 1u << (s & 31u));
    }
    __syncthreads();
    block_copy_words(p.bits + (size_t)wk.walker0 * words, fw, total);
}

template <int D, typename IdxT, int G, int TM, bool TUN, bool MC = false>
__device__ __forceinline__ void field_item(const SysParams &p, const BlockWork &wk, uint32_t *smem,
                                           uint64_t sweeps, uint32_t iter)
{
    if constexpr (TM == kThrShared) block_copy_words(smem, p.thr, (size_t)p.n_bins * (size_t)p.tstride);
    uint32_t *fw = smem + (TM == kThrShared ? thr_words_aligned(p) : 0);
    field_build<D, IdxT>(p, wk, fw);   // ends with a block barrier, which also covers the table
    const int lw = threadIdx.x / G;
    const bool active = lw < wk.count;
    const int w = wk.walker0 + (active ? lw : 0);
    const uint32_t *thr = TM == kThrShared ? smem : p.thr;
    const uint32_t fbase = (uint32_t)__cvta_generic_to_shared(fw) +
                           (uint32_t)((size_t)(active ? lw : 0) * field_bytes(p));
    unsigned long long *hist = hist_row(p, w, wk.hist_row);
    uint32_t ring_s = 0u, mbar_s = 0u;
    if constexpr (TM == kThrWindow) {
        const int wpb = (int)blockDim.x / G;
        const uint32_t after = (uint32_t)__cvta_generic_to_shared(fw) +
                               (uint32_t)((size_t)wpb * field_bytes(p));
        window_addrs(p, after, wpb, active ? lw : 0, ring_s, mbar_s);
    }
    if constexpr (MC) {
        chain_rounds_mc<D, IdxT, G, TM>(p, w, active, FieldView<D>(fbase), thr, hist,
                                        sweeps * (uint64_t)p.N, iter);
    } else {
        // site compare for moved slots (measured on GB300: the faster one here for every G)
        chain_rounds<D, IdxT, G, TM, TUN, false>(p, w, active, FieldView<D>(fbase), thr, hist,
                                                 sweeps * (uint64_t)p.N, iter, ring_s, mbar_s);
    }
    field_finish<IdxT>(p, wk, fw);
}

template <int G, int TM, bool TUN, bool MC = false>
__device__ __forceinline__ void field_body(const SysParams &p, const BlockWork &wk, uint32_t *smem,
                                           uint64_t sweeps, uint32_t iter)
{
    if (p.d == 2) {
        if (p.idx16) field_item<2, uint16_t, G, TM, TUN, MC>(p, wk, smem, sweeps, iter);
        else field_item<2, uint32_t, G, TM, TUN, MC>(p, wk, smem, sweeps, iter);
    } else {
        if (p.idx16) field_item<3, uint16_t, G, TM, TUN, MC>(p, wk, smem, sweeps, iter);
        else field_item<3, uint32_t, G, TM, TUN, MC>(p, wk, smem, sweeps, iter);
    }
}

template <int G, int TM, bool TUN, bool PERSIST, bool MC = false>
__global__ void __launch_bounds__(kGroupMaxThreads, 1)
walker_update_field(const SysParams *__restrict__ sys, const BlockWork *__restrict__ work,
                    uint64_t sweeps, uint32_t iter, int n_items, int *next_item)
{
    extern __shared__ __align__(16) uint32_t smem[];
    if constexpr (!PERSIST) {
        // one work item per block
        (void)n_items;
        (void)next_item;
        const BlockWork wk = work[blockIdx.x];
        field_body<G, TM, TUN, MC>(sys[wk.sys], wk, smem, sweeps, iter);
    } else {
        __shared__ int s_item;
        for (int item = blockIdx.x; item < n_items;) {
            const BlockWork wk = work[item];
            field_body<G, TM, TUN, MC>(sys[wk.sys], wk, smem, sweeps, iter);
            item = next_work_item(next_item, &s_item);
        }
    }
}

// Threshold mode of a launch shape (group and field kernels).
inline int thr_mode(const LaunchShape &sh)
{
    return sh.thr_in_smem ? kThrShared : (sh.thr_window ? kThrWindow : kThrGlobal);
}

// Multi-commit rounds apply to the group and field kernels at 4 to 32 lanes
// with the thresholds in global memory or a staged table, without the
// tunnelling bookkeeping; other shapes run the one-commit rounds.
template <int G, bool TUN>
constexpr bool kMcFlavour = !TUN && G >= 4;

inline bool use_mc(const LaunchShape &sh)
{
    return sh.multi_commit && thr_mode(sh) != kThrWindow;
}

template <int G, bool TUN, bool PE>
const void *field_fn(const LaunchShape &sh)
{
    if constexpr (kMcFlavour<G, TUN>) {
        if (use_mc(sh))
            return thr_mode(sh) == kThrShared
                       ? (const void *)walker_update_field<G, kThrShared, TUN, PE, true>
                       : (const void *)walker_update_field<G, kThrGlobal, TUN, PE, true>;
    }
    switch (thr_mode(sh)) {
    case kThrShared: return (const void *)walker_update_field<G, kThrShared, TUN, PE>;
    case kThrWindow: return (const void *)walker_update_field<G, kThrWindow, TUN, PE>;
    default: return (const void *)walker_update_field<G, kThrGlobal, TUN, PE>;
    }
}

template <int G, bool SB, bool TUN, bool PE>
const void *group_fn_sb(const LaunchShape &sh)
{
    if constexpr (kMcFlavour<G, TUN>) {
        if (use_mc(sh))
            return thr_mode(sh) == kThrShared
                       ? (const void *)walker_update_group<G, SB, kThrShared, TUN, PE, true>
                       : (const void *)walker_update_group<G, SB, kThrGlobal, TUN, PE, true>;
    }
    switch (thr_mode(sh)) {
    case kThrShared: return (const void *)walker_update_group<G, SB, kThrShared, TUN, PE>;
    case kThrWindow: return (const void *)walker_update_group<G, SB, kThrWindow, TUN, PE>;
    default: return (const void *)walker_update_group<G, SB, kThrGlobal, TUN, PE>;
    }
}

// The walker-update kernel of a launch shape (one TUN flavour).
template <int G, bool TUN, bool PE>
const void *group_fn(const LaunchShape &sh)
{
    return sh.bits_in_smem ? group_fn_sb<G, true, TUN, PE>(sh) : group_fn_sb<G, false, TUN, PE>(sh);
}

// The kernel of a launch shape among the kWalkerUpdateFns of one (TUN, PE) flavour
// (PE: persistent launch); the caller checks that shape.persistent == PE.
template <bool TUN, bool PE>
const void *walker_update_fn_t(const LaunchShape &sh)
{
    if (sh.kernel == 0) {
        if (sh.bits_in_smem && sh.thr_in_smem) return (const void *)walker_update_thread<true, true, TUN, PE>;
        if (sh.bits_in_smem) return (const void *)walker_update_thread<true, false, TUN, PE>;
        if (sh.thr_in_smem) return (const void *)walker_update_thread<false, true, TUN, PE>;
        return (const void *)walker_update_thread<false, false, TUN, PE>;
    }
    if (sh.kernel == 2) {
        switch (sh.lanes) {
        case 2: return field_fn<2, TUN, PE>(sh);
        case 4: return field_fn<4, TUN, PE>(sh);
        case 8: return field_fn<8, TUN, PE>(sh);
        case 16: return field_fn<16, TUN, PE>(sh);
        case 32: return field_fn<32, TUN, PE>(sh);
        default: return nullptr;
        }
    }
    switch (sh.lanes) {
    case 2: return group_fn<2, TUN, PE>(sh);
    case 4: return group_fn<4, TUN, PE>(sh);
    case 8: return group_fn<8, TUN, PE>(sh);
    case 16: return group_fn<16, TUN, PE>(sh);
    case 32: return group_fn<32, TUN, PE>(sh);
    default: return nullptr;
    }
}

// Every walker-update kernel of one (TUN, PE) flavour (for their
// shared-memory attributes).
template <bool TUN, bool PE>
void walker_update_fns(const void *(&fns)[kWalkerUpdateFns])
{
    int i = 0;
    fns[i++] = (const void *)walker_update_thread<true, true, TUN, PE>;
    fns[i++] = (const void *)walker_update_thread<true, false, TUN, PE>;
    fns[i++] = (const void *)walker_update_thread<false, true, TUN, PE>;
    fns[i++] = (const void *)walker_update_thread<false, false, TUN, PE>;
#define MUCAL_GROUP_FNS(G)                                                          \
    fns[i++] = (const void *)walker_update_group<G, true, kThrShared, TUN, PE>;    \
    fns[i++] = (const void *)walker_update_group<G, true, kThrGlobal, TUN, PE>;    \
    fns[i++] = (const void *)walker_update_group<G, true, kThrWindow, TUN, PE>;    \
    fns[i++] = (const void *)walker_update_group<G, false, kThrShared, TUN, PE>;   \
    fns[i++] = (const void *)walker_update_group<G, false, kThrGlobal, TUN, PE>;   \
    fns[i++] = (const void *)walker_update_group<G, false, kThrWindow, TUN, PE>;
    MUCAL_GROUP_FNS(2)
    MUCAL_GROUP_FNS(4)
    MUCAL_GROUP_FNS(8)
    MUCAL_GROUP_FNS(16)
    MUCAL_GROUP_FNS(32)
#undef MUCAL_GROUP_FNS
#define MUCAL_FIELD_FNS(G)                                                     \
    fns[i++] = (const void *)walker_update_field<G, kThrShared, TUN, PE>;     \
    fns[i++] = (const void *)walker_update_field<G, kThrGlobal, TUN, PE>;     \
    fns[i++] = (const void *)walker_update_field<G, kThrWindow, TUN, PE>;
    MUCAL_FIELD_FNS(2)
    MUCAL_FIELD_FNS(4)
    MUCAL_FIELD_FNS(8)
    MUCAL_FIELD_FNS(16)
    MUCAL_FIELD_FNS(32)
#undef MUCAL_FIELD_FNS
    // multi-commit rounds (flavours without tunnelling bookkeeping only)
#define MUCAL_MC_FNS(G)                                                                        \
    if constexpr (kMcFlavour<G, TUN>) {                                                        \
        fns[i++] = (const void *)walker_update_group<G, true, kThrShared, TUN, PE, true>;     \
        fns[i++] = (const void *)walker_update_group<G, true, kThrGlobal, TUN, PE, true>;     \
        fns[i++] = (const void *)walker_update_group<G, false, kThrShared, TUN, PE, true>;    \
        fns[i++] = (const void *)walker_update_group<G, false, kThrGlobal, TUN, PE, true>;    \
        fns[i++] = (const void *)walker_update_field<G, kThrShared, TUN, PE, true>;           \
        fns[i++] = (const void *)walker_update_field<G, kThrGlobal, TUN, PE, true>;           \
    } else {                                                                                   \
        for (int q = 0; q < 6; ++q) fns[i++] = nullptr;                                        \
    }
    MUCAL_MC_FNS(4)
    MUCAL_MC_FNS(8)
    MUCAL_MC_FNS(16)
    MUCAL_MC_FNS(32)
#undef MUCAL_MC_FNS
}

}  // namespace
}  // namespace mucal
