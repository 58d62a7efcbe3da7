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
//   3. after the mbarrier completes, warp q reads TMEM lanes 32(q%4) on (its
//      rows) with tcgen05.ld, 32 columns at a time: warps 0-3 the columns
//      0-63, warps 4-7 the columns 64-127; the two halves of
//      y = b3 + sum_n W3[n] gelu(Z2[n] + b2[n]) meet in shared memory.
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
constexpr int TC_THREADS = 256;                // two threads per row: each takes half the columns
constexpr int TC_OFF_W1 = 0, TC_OFF_B1 = TC_H * 4, TC_OFF_W2 = TC_OFF_B1 + TC_H;
constexpr int TC_OFF_B2 = TC_OFF_W2 + TC_H * TC_H, TC_OFF_W3 = TC_OFF_B2 + TC_H;
constexpr int TC_OFF_B3 = TC_OFF_W3 + TC_H;
constexpr uint32_t TILE_BYTES = TC_ROWS * TC_H * 2;   // one 128x128 bf16 operand
constexpr uint32_t LBO = 128;                  // next core matrix along K
constexpr uint32_t SBO = 2048;                 // next group of 8 rows
constexpr uint32_t SMEM_A_HI = 0, SMEM_A_LO = TILE_BYTES, SMEM_B = 2 * TILE_BYTES;
constexpr uint32_t SMEM_PAR = 3 * TILE_BYTES;  // w1[512], b1, b2, w3, b3 (fp32)
constexpr uint32_t SMEM_BAR = SMEM_PAR + (TC_H * 4 + 3 * TC_H + 4) * 4;
constexpr uint32_t SMEM_YP = SMEM_BAR + 16;    // partial outputs of the two column halves
constexpr uint32_t SMEM_TOTAL = SMEM_YP + 2 * TC_ROWS * 4;
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
    // layer 1 (K = 4, fp32) of row r_in, this thread's half of the units,
    // split into two bf16 terms
    const int r_in = tid & (TC_ROWS - 1), half = tid >> 7;
    const int64_t row = (int64_t)blockIdx.x * TC_ROWS + r_in;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
    if (row < B) {
        x0 = X[row * 4 + 0];
        x1 = X[row * 4 + 1];
        x2 = X[row * 4 + 2];
        x3 = X[row * 4 + 3];
    }
    for (int kg = half * 8; kg < half * 8 + 8; ++kg) {
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
        const uint32_t off = core_offset(r_in, kg * 8);
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
    const bool ok = __syncthreads_and(mbar_wait(bar, 0));
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float *yp = reinterpret_cast<float *>(smem + SMEM_YP);
    if (ok) {
        // warp w reads TMEM lanes 32 (w % 4) .. (its rows), columns of its half
        float out = 0.f;
#pragma unroll 1
        for (int cb = half * 2; cb < half * 2 + 2; ++cb) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(cb * 32), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int n = cb * 32 + i;
                out += s_w3[n] * gelu_tc(v[i] + s_b2[n]);
            }
        }
        yp[half * TC_ROWS + r_in] = out;
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (ok && half == 0 && row < B) y[row] = *s_b3 + yp[r_in] + yp[TC_ROWS + r_in];
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_H));
}

__device__ __forceinline__ float gelu_grad_tc(float z)
{
    const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
    return cdf + z * pdf;
}

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Training pass (forward and backward of the mean squared error) of 128 rows
// per CTA, every contraction on tcgen05:
//   Z2 = H1 W2^T            A = H1 (hi, then lo) [row][in],  B = W2   [out][in]
//   dH1 = dZ2 W2            A = dZ2 [row][out],              B = W2^T [in][out]
//   dW2 = dZ2^T H1 (+=)     A = dZ2^T [out][row],            B = H1^T [in][row]
// all K-major in the core-matrix layout; TMEM columns 0-127 hold Z2, 128-255
// dH1 and 256-383 the CTA's share of dW2.  The small gradients (W1, b1, b2,
// W3, b3) and the loss are reduced in fp32 over the CTA's rows, then added to
// grad / loss_out; dW2 is added from TMEM.  Rows past B contribute nothing.
constexpr uint32_t TR_AHI = 0, TR_ALO = TILE_BYTES, TR_W2 = 2 * TILE_BYTES, TR_W2T = 3 * TILE_BYTES;
constexpr uint32_t TR_DZT = 4 * TILE_BYTES, TR_H1T = 5 * TILE_BYTES;
constexpr uint32_t TR_PAR = 6 * TILE_BYTES;                    // w1, b1, b2, w3, b3
constexpr int TR_NPAR = TC_H * 4 + 3 * TC_H + 1;
constexpr uint32_t TR_RED = TR_PAR + ((TR_NPAR * 4 + 15) / 16) * 16;
constexpr int TR_NRED = TC_H * 4 + TC_H + TC_H + TC_H + 2;     // dW1, db1, db2, dW3, db3, loss
constexpr uint32_t TR_BAR = TR_RED + ((TR_NRED * 4 + 15) / 16) * 16;
constexpr uint32_t TR_YP = TR_BAR + 16;        // partial outputs of the two column halves
constexpr uint32_t TR_X = TR_YP + 2 * TC_ROWS * 4;   // x of the CTA's rows, [128][4]
constexpr uint32_t TR_WS = TR_X + TC_ROWS * 4 * 4;   // loss and db3 of warps 0-3
constexpr uint32_t TR_TOTAL = TR_WS + 8 * 4;
// Each CTA writes its gradients (and, last, its loss) as one row of a
// partial buffer; a second kernel sums the rows in CTA order, so that the
// gradients do not depend on the order in which CTAs finish.
constexpr int TC_NPARAM = TC_OFF_B3 + 1;
constexpr int TC_PSTRIDE = ((TC_NPARAM + 1 + 3) / 4) * 4;
constexpr uint32_t TR_COLS = 512;

__global__ void __launch_bounds__(TC_THREADS, 1)
mlp_train_tc_kernel(const __nv_bfloat16 *__restrict__ wq, const float *__restrict__ X,
                    const float *__restrict__ target, int64_t B, float inv_b,
                    float *__restrict__ part, int *err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    float *par = reinterpret_cast<float *>(smem + TR_PAR);
    float *s_w1 = par, *s_b1 = par + TC_H * 4, *s_b2 = s_b1 + TC_H, *s_w3 = s_b2 + TC_H;
    float *s_b3 = s_w3 + TC_H;
    float *red = reinterpret_cast<float *>(smem + TR_RED);
    float *r_w1 = red, *r_b1 = red + TC_H * 4, *r_b2 = r_b1 + TC_H, *r_w3 = r_b2 + TC_H;
    float *ws = reinterpret_cast<float *>(smem + TR_WS);
    const uint32_t bar = sbase + TR_BAR;
    const uint32_t tmem_slot = sbase + TR_BAR + 8;
    uint32_t *tmem_slot_ptr = reinterpret_cast<uint32_t *>(smem + TR_BAR + 8);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(tmem_slot), "r"(TR_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int i = tid; i < TC_H * 4; i += TC_THREADS) s_w1[i] = __bfloat162float(wq[TC_OFF_W1 + i]);
    for (int i = tid; i < TC_H; i += TC_THREADS) {
        s_b1[i] = __bfloat162float(wq[TC_OFF_B1 + i]);
        s_b2[i] = __bfloat162float(wq[TC_OFF_B2 + i]);
        s_w3[i] = __bfloat162float(wq[TC_OFF_W3 + i]);
    }
    if (tid == 0) *s_b3 = __bfloat162float(wq[TC_OFF_B3]);
    for (int i = tid; i < TR_NRED; i += TC_THREADS) red[i] = 0.f;
    if (tid < 8) ws[tid] = 0.f;
    // W2 [out][in] and W2^T [in][out], 16-byte chunks of 8 consecutive k
    for (int c = tid; c < TC_H * TC_H / 8; c += TC_THREADS) {
        const int n = c >> 4, kg = c & 15;
        const uint4 v = *reinterpret_cast<const uint4 *>(wq + TC_OFF_W2 + n * TC_H + kg * 8);
        *reinterpret_cast<uint4 *>(smem + TR_W2 + core_offset(n, kg * 8)) = v;
        // W2^T row n = in, k = out: W2[kg*8 + u][n]
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat16 lo = wq[TC_OFF_W2 + (kg * 8 + 2 * e) * TC_H + n];
            const __nv_bfloat16 hi = wq[TC_OFF_W2 + (kg * 8 + 2 * e + 1) * TC_H + n];
            w[e] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        *reinterpret_cast<uint4 *>(smem + TR_W2T + core_offset(n, kg * 8)) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();
    // layer 1 of row r_in, this thread's half of the units: H1 hi/lo
    // [row][in] and H1^T hi [in][row]
    const int r_in = tid & (TC_ROWS - 1), half = tid >> 7;
    const int64_t row = (int64_t)blockIdx.x * TC_ROWS + r_in;
    const bool live = row < B;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
    if (live) {
        x0 = X[row * 4 + 0];
        x1 = X[row * 4 + 1];
        x2 = X[row * 4 + 2];
        x3 = X[row * 4 + 3];
    }
    for (int kg = half * 8; kg < half * 8 + 8; ++kg) {
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
                const __nv_bfloat16 hb = __float2bfloat16_rn(h);
                hv[u] = __bfloat162float(hb);
                lv[u] = h - hv[u];
                *reinterpret_cast<__nv_bfloat16 *>(smem + TR_H1T + core_offset(n, r_in)) = hb;
            }
            hi[e] = pack2(hv[0], hv[1]);
            lo[e] = pack2(lv[0], lv[1]);
        }
        const uint32_t off = core_offset(r_in, kg * 8);
        *reinterpret_cast<uint4 *>(smem + TR_AHI + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4 *>(smem + TR_ALO + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot_ptr;
    if (tid == 0) {
#pragma unroll
        for (int pass = 0; pass < 2; ++pass)
#pragma unroll
            for (int ks = 0; ks < TC_H / 16; ++ks)
                umma(tmem, smem_desc(sbase + (pass == 0 ? TR_AHI : TR_ALO) + ks * 2 * LBO),
                     smem_desc(sbase + TR_W2 + ks * 2 * LBO), (pass > 0 || ks > 0) ? 1u : 0u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                     ::"r"(bar) : "memory");
    }
    bool ok = __syncthreads_and(mbar_wait(bar, 0));
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // warp w reads TMEM lanes 32 (w % 4) .. (its rows), columns of its half
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    float *yp = reinterpret_cast<float *>(smem + TR_YP);
    if (ok) {
        // pass 1: this half's part of y
        float yh = 0.f;
#pragma unroll 1
        for (int cb = half * 2; cb < half * 2 + 2; ++cb) {
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(cb * 32), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) yh += s_w3[cb * 32 + i] * gelu_tc(v[i] + s_b2[cb * 32 + i]);
        }
        yp[half * TC_ROWS + r_in] = yh;
    }
    __syncthreads();
    float dy_row = 0.f;
    if (ok) {
        const float y = *s_b3 + yp[r_in] + yp[TC_ROWS + r_in];
        const float e = live ? y - target[row] : 0.f;
        const float dy = 2.f * e * inv_b;
        dy_row = dy;
        if (half == 0) {
            const float l = warp_sum(e * e * inv_b), sdy = warp_sum(dy);
            if (lane == 0) {       // warps 0-3; summed in warp order at the end
                ws[warp] = l;
                ws[4 + warp] = sdy;
            }
        }
        // pass 2: dz2 = dy w3 gelu'(z2) in bf16 as dZ2 and dZ2^T for the tensor cores
#pragma unroll 1
        for (int cb = half * 2; cb < half * 2 + 2; ++cb) {
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(cb * 32), v);
#pragma unroll
            for (int g8 = 0; g8 < 4; ++g8) {
                uint32_t pk[4];
#pragma unroll
                for (int e2 = 0; e2 < 4; ++e2) {
                    float dz[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int i = g8 * 8 + 2 * e2 + u;
                        const int n = cb * 32 + i;
                        const float z = v[i] + s_b2[n];
                        dz[u] = dy * s_w3[n] * gelu_grad_tc(z);
                        *reinterpret_cast<__nv_bfloat16 *>(smem + TR_DZT + core_offset(n, r_in)) =
                            __float2bfloat16_rn(dz[u]);
                    }
                    pk[e2] = pack2(dz[0], dz[1]);
                }
                *reinterpret_cast<uint4 *>(smem + TR_ALO + core_offset(r_in, cb * 32 + g8 * 8)) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0 && ok) {
        // dH1 = dZ2 W2 into columns 128..255; dW2 share = dZ2^T H1 into 256..383
#pragma unroll
        for (int ks = 0; ks < TC_H / 16; ++ks)
            umma(tmem + 128, smem_desc(sbase + TR_ALO + ks * 2 * LBO),
                 smem_desc(sbase + TR_W2T + ks * 2 * LBO), ks > 0 ? 1u : 0u);
#pragma unroll
        for (int ks = 0; ks < TC_ROWS / 16; ++ks)
            umma(tmem + 256, smem_desc(sbase + TR_DZT + ks * 2 * LBO),
                 smem_desc(sbase + TR_H1T + ks * 2 * LBO), ks > 0 ? 1u : 0u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                     ::"r"(bar) : "memory");
    }
    ok = __syncthreads_and(ok && mbar_wait(bar, 1));
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // Column sums over the CTA's rows go through shared memory (the operand
    // tiles at offset 0 are free now): each thread writes its row's values of
    // its column half into S[128][128] fp32 (columns XOR-swizzled by the row so
    // that a warp's 32 rows hit 32 banks), then thread t sums column t % 128
    // over the rows of half t / 128.
    float *S = reinterpret_cast<float *>(smem + TR_AHI);
    float *xrow = reinterpret_cast<float *>(smem + TR_X);
    auto s_at = [&](int r, int n) -> float & { return S[r * TC_H + (n ^ (r & 31))]; };
    const int cn = tid & (TC_H - 1), ch = tid >> 7;  // reduction: column, half of the rows
    // (a) db2 += dz2 and (b) dW3 += dy h2, z2 re-read from TMEM
#pragma unroll 1
    for (int q = 0; q < 2 && ok; ++q) {
#pragma unroll 1
        for (int cb = half * 2; cb < half * 2 + 2; ++cb) {
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(cb * 32), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int n = cb * 32 + i;
                const float z = v[i] + s_b2[n];
                s_at(r_in, n) = q == 0 ? dy_row * s_w3[n] * gelu_grad_tc(z) : dy_row * gelu_tc(z);
            }
        }
        __syncthreads();
        float a = 0.f;
        for (int r = ch * 64; r < ch * 64 + 64; ++r) a += s_at(r, cn);
        // two addends (the two row halves) onto zero: the same sum in either order
        atomicAdd((q == 0 ? r_b2 : r_w3) + cn, a);
        __syncthreads();
    }
    if (ok) {
        // (c) dz1 = dh1 gelu'(z1): dW1 += dz1 x, db1 += dz1
#pragma unroll 1
        for (int cb = half * 2; cb < half * 2 + 2; ++cb) {
            float v[32];
            tmem_ld32(tmem + lane_base + 128u + (uint32_t)(cb * 32), v);
#pragma unroll 4
            for (int i = 0; i < 32; ++i) {
                const int n = cb * 32 + i;
                const float z = s_b1[n] + x0 * s_w1[n * 4 + 0] + x1 * s_w1[n * 4 + 1] +
                                x2 * s_w1[n * 4 + 2] + x3 * s_w1[n * 4 + 3];
                s_at(r_in, n) = live ? v[i] * gelu_grad_tc(z) : 0.f;
            }
        }
        if (half == 0) {
            xrow[r_in * 4 + 0] = x0;
            xrow[r_in * 4 + 1] = x1;
            xrow[r_in * 4 + 2] = x2;
            xrow[r_in * 4 + 3] = x3;
        }
    }
    __syncthreads();
    if (ok) {
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f, gb = 0.f;
        for (int r = ch * 64; r < ch * 64 + 64; ++r) {
            const float d = s_at(r, cn);
            g0 += d * xrow[r * 4 + 0];
            g1 += d * xrow[r * 4 + 1];
            g2 += d * xrow[r * 4 + 2];
            g3 += d * xrow[r * 4 + 3];
            gb += d;
        }
        atomicAdd(r_w1 + cn * 4 + 0, g0);
        atomicAdd(r_w1 + cn * 4 + 1, g1);
        atomicAdd(r_w1 + cn * 4 + 2, g2);
        atomicAdd(r_w1 + cn * 4 + 3, g3);
        atomicAdd(r_b1 + cn, gb);
        // this CTA's share of dW2: TMEM lane = out, column = in
        float *prow = part + (size_t)blockIdx.x * TC_PSTRIDE;
#pragma unroll 1
        for (int cb = half * 2; cb < half * 2 + 2; ++cb) {
            float v[32];
            tmem_ld32(tmem + lane_base + 256u + (uint32_t)(cb * 32), v);
            const int out = (warp & 3) * 32 + lane;
            float4 *dst = reinterpret_cast<float4 *>(prow + TC_OFF_W2 + out * TC_H + cb * 32);
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (ok) {
        float *prow = part + (size_t)blockIdx.x * TC_PSTRIDE;
        for (int i = tid; i < TC_H * 4; i += TC_THREADS) prow[TC_OFF_W1 + i] = r_w1[i];
        for (int i = tid; i < TC_H; i += TC_THREADS) {
            prow[TC_OFF_B1 + i] = r_b1[i];
            prow[TC_OFF_B2 + i] = r_b2[i];
            prow[TC_OFF_W3 + i] = r_w3[i];
        }
        if (tid == 0) {
            prow[TC_OFF_B3] = ((ws[4] + ws[5]) + ws[6]) + ws[7];
            prow[TC_NPARAM] = ((ws[0] + ws[1]) + ws[2]) + ws[3];
        }
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TR_COLS));
}

// grad[i] (and, for i = TC_NPARAM, the loss) = the sum of the CTAs' rows in
// CTA order.
__global__ void mlp_tc_grad_reduce_kernel(const float *__restrict__ part, int n_cta,
                                          float *__restrict__ grad, float *__restrict__ loss_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > TC_NPARAM) return;
    float s = 0.f;
    for (int b = 0; b < n_cta; ++b) s += part[(size_t)b * TC_PSTRIDE + i];
    if (i < TC_NPARAM) grad[i] = s;
    else *loss_out = s;
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

namespace mucal {

size_t mlp_train_tcgen05_partial_floats(int64_t B)
{
    return (size_t)((B + TC_ROWS - 1) / TC_ROWS) * TC_PSTRIDE;
}

cudaError_t mlp_train_tcgen05(const void *wq, const float *X, const float *target, int64_t B,
                              float *part, float *grad, float *loss, int *err, cudaStream_t stream)
{
    static_assert(TR_TOTAL <= 227 * 1024, "shared memory");
    cudaError_t e = cudaFuncSetAttribute(mlp_train_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_TOTAL);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((B + TC_ROWS - 1) / TC_ROWS);
    mlp_train_tc_kernel<<<blocks, TC_THREADS, TR_TOTAL, stream>>>(
        static_cast<const __nv_bfloat16 *>(wq), X, target, B, 1.0f / (float)B, part, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mlp_tc_grad_reduce_kernel<<<(TC_NPARAM + 1 + 255) / 256, 256, 0, stream>>>(part, blocks, grad, loss);
    return cudaGetLastError();
}

}  // namespace mucal
