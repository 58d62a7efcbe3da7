// Forward pass of the weight-seeding network with the 128x128 layer on the
// fifth-generation tensor cores (tcgen05): one CTA of four warps per 128 rows.
//
//   1. the CTA stages W2 (bf16, [out][in]) and the layer-1 activations of its
//      128 rows, split into hi = bf16(h1) and lo = bf16(h1 - hi), in shared
//      memory in the K-major, unswizzled core-matrix layout (8 rows x 16 bytes
//      per core matrix; core matrices along K 128 bytes apart, 8-row groups
//      2048 bytes apart);
//   2. warp 0 allocates 128 TMEM columns; thread 0 issues sixteen
//      tcgen05.mma (M = 128, N = 128, K = 16 each; A = hi for k-steps 0-7,
//      then lo) accumulating Z2 = H1 W2^T in fp32 in TMEM, and commits them to
//      an mbarrier;
//   3. after the mbarrier completes, warp q reads TMEM lanes 32q..32q+31 (its
//      rows) with tcgen05.ld, 32 columns at a time, and finishes the row:
//      y = b3 + sum_n W3[n] gelu(Z2[n] + b2[n]).
// The mbarrier wait is bounded; if it runs out the CTA records an error flag,
// frees its TMEM and returns.  Numerics equal the mma.sync path of
// mlp_kernels.cu up to the order of the fp32 sums.
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mucal_internal.h"

namespace mucal {
namespace {

constexpr int TC_H = 128;                      // hidden width
constexpr int TC_ROWS = 128;                   // rows per CTA = TMEM lanes
constexpr int TC_THREADS = 128;
constexpr int TC_OFF_W1 = 0, TC_OFF_B1 = TC_H * 4, TC_OFF_W2 = TC_OFF_B1 + TC_H;
constexpr int TC_OFF_B2 = TC_OFF_W2 + TC_H * TC_H, TC_OFF_W3 = TC_OFF_B2 + TC_H;
constexpr int TC_OFF_B3 = TC_OFF_W3 + TC_H;
constexpr uint32_t TILE_BYTES = TC_ROWS * TC_H * 2;   // one 128x128 bf16 operand
constexpr uint32_t LBO = 128;                  // next core matrix along K
constexpr uint32_t SBO = 2048;                 // next group of 8 rows
constexpr uint32_t SMEM_A_HI = 0, SMEM_A_LO = TILE_BYTES, SMEM_B = 2 * TILE_BYTES;
constexpr uint32_t SMEM_PAR = 3 * TILE_BYTES;  // w1[512], b1, b2, w3, b3 (fp32)
constexpr uint32_t SMEM_BAR = SMEM_PAR + (TC_H * 4 + 3 * TC_H + 4) * 4;
constexpr uint32_t SMEM_TOTAL = SMEM_BAR + 16;
constexpr int WAIT_LIMIT = 1 << 22;

__device__ __forceinline__ uint32_t core_offset(int row, int k)
{
    return (uint32_t)(row >> 3) * SBO + (uint32_t)(k >> 3) * LBO + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// Shared-memory matrix descriptor of the tcgen05 instructions: start address,
// leading and stride byte offsets (all >> 4), descriptor version 1, no
// swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(LBO >> 4) << 16) |
           ((uint64_t)(SBO >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = 128, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_H >> 3) << 17) |
                           ((uint32_t)(TC_ROWS >> 4) << 24);

__device__ __forceinline__ float gelu_tc(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase)
{
    for (int i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
mlp_forward_tc_kernel(const __nv_bfloat16 *__restrict__ wq, const float *__restrict__ X,
                      float *__restrict__ y, int64_t B, int *err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    float *par = reinterpret_cast<float *>(smem + SMEM_PAR);
    float *s_w1 = par, *s_b1 = par + TC_H * 4, *s_b2 = s_b1 + TC_H, *s_w3 = s_b2 + TC_H;
    float *s_b3 = s_w3 + TC_H;
    const uint32_t bar = sbase + SMEM_BAR;
    const uint32_t tmem_slot = sbase + SMEM_BAR + 8;
    uint32_t *tmem_slot_ptr = reinterpret_cast<uint32_t *>(smem + SMEM_BAR + 8);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(tmem_slot), "r"(TC_H));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // small fp32 parameters
    for (int i = tid; i < TC_H * 4; i += TC_THREADS) s_w1[i] = __bfloat162float(wq[TC_OFF_W1 + i]);
    for (int i = tid; i < TC_H; i += TC_THREADS) {
        s_b1[i] = __bfloat162float(wq[TC_OFF_B1 + i]);
        s_b2[i] = __bfloat162float(wq[TC_OFF_B2 + i]);
        s_w3[i] = __bfloat162float(wq[TC_OFF_W3 + i]);
    }
    if (tid == 0) *s_b3 = __bfloat162float(wq[TC_OFF_B3]);
    // W2 -> B operand: 16-byte chunks (row n, 8 consecutive k)
    for (int c = tid; c < TC_H * TC_H / 8; c += TC_THREADS) {
        const int n = c >> 4, kg = c & 15;
        const uint4 v = *reinterpret_cast<const uint4 *>(wq + TC_OFF_W2 + n * TC_H + kg * 8);
        *reinterpret_cast<uint4 *>(smem + SMEM_B + core_offset(n, kg * 8)) = v;
    }
    __syncthreads();
    // layer 1 (K = 4, fp32) of row tid, split into two bf16 terms
    const int64_t row = (int64_t)blockIdx.x * TC_ROWS + tid;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
    if (row < B) {
        x0 = X[row * 4 + 0];
        x1 = X[row * 4 + 1];
        x2 = X[row * 4 + 2];
        x3 = X[row * 4 + 3];
    }
    for (int kg = 0; kg < TC_H / 8; ++kg) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float hv[2], lv[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int n = kg * 8 + 2 * e + u;
                const float z = s_b1[n] + x0 * s_w1[n * 4 + 0] + x1 * s_w1[n * 4 + 1] +
                                x2 * s_w1[n * 4 + 2] + x3 * s_w1[n * 4 + 3];
                const float h = gelu_tc(z);
                hv[u] = __bfloat162float(__float2bfloat16_rn(h));
                lv[u] = h - hv[u];
            }
            hi[e] = pack2(hv[0], hv[1]);
            lo[e] = pack2(lv[0], lv[1]);
        }
        const uint32_t off = core_offset(tid, kg * 8);
        *reinterpret_cast<uint4 *>(smem + SMEM_A_HI + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4 *>(smem + SMEM_A_LO + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    // generic-proxy writes of the operands become visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot_ptr;
    if (tid == 0) {
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            const uint32_t a0 = sbase + (pass == 0 ? SMEM_A_HI : SMEM_A_LO);
#pragma unroll
            for (int ks = 0; ks < TC_H / 16; ++ks) {
                const uint64_t ad = smem_desc(a0 + ks * 2 * LBO);
                const uint64_t bd = smem_desc(sbase + SMEM_B + ks * 2 * LBO);
                const uint32_t acc = (pass > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                    ::"r"(tmem), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                     ::"r"(bar) : "memory");
    }
    const bool ok = mbar_wait(bar, 0);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        float out = *s_b3;
#pragma unroll 1
        for (int cb = 0; cb < TC_H / 32; ++cb) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int n = cb * 32 + i;
                out += s_w3[n] * gelu_tc(v[i] + s_b2[n]);
            }
        }
        const int64_t r = (int64_t)blockIdx.x * TC_ROWS + warp * 32 + lane;
        if (r < B) y[r] = out;
    } else if (lane == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_H));
}

}  // namespace

cudaError_t mlp_forward_tcgen05(const void *wq, const float *X, float *y, int64_t B, int *err,
                                cudaStream_t stream)
{
    static_assert(SMEM_TOTAL <= 227 * 1024, "shared memory");
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TOTAL);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((B + TC_ROWS - 1) / TC_ROWS);
    mlp_forward_tc_kernel<<<blocks, TC_THREADS, SMEM_TOTAL, stream>>>(
        static_cast<const __nv_bfloat16 *>(wq), X, y, B, err);
    return cudaGetLastError();
}

}  // namespace mucal
