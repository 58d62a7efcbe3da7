// Weight-seeding network of libmucal: a 4-128-128-1 GELU multilayer
// perceptron mapping features of (d, L, rho, E/V) to ln Omega(E)/V, trained
// and evaluated on the GPU.  Not part of the paper: it only proposes starting
// weights W = 1/Omega_pred for the iteration of Sec. 2, which then runs
// unchanged and decides convergence as before.
//
// This file holds the host side, the Adam update and the mma.sync kernels,
// which are the reference path; the default path runs the contractions with
// tcgen05 (mlp_tcgen05.cu).
//
// Numerics: parameters kept in fp32 (master copy, Adam state) and used in
// bf16; the 128x128 contractions run on the tensor cores as bf16 x bf16 with
// fp32 accumulation (here mma.sync m16n8k16); the K=4 input layer, the N=1 output
// layer, GELU and all reductions are fp32.  In the forward pass the layer-1
// activations enter the tensor cores split into two bf16 terms (hi + lo),
// which keeps the network's output smooth in its inputs to about 1e-5
// relative instead of the 4e-3 steps a single bf16 rounding would leave.
//
// Parameter vector (fp32, 17281 entries): W1[128][4], b1[128], W2[128][128]
// (row = output unit), b2[128], W3[128], b3.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mucal.h"
#include "mucal_internal.h"

namespace {

constexpr int H = 128;                         // hidden width
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + H * 4;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + H;
constexpr int NPARAM = OFF_B3 + 1;             // 17281
constexpr int ROWS_PER_WARP = 16;
constexpr int WARPS = 4;
constexpr int ROWS_PER_BLOCK = ROWS_PER_WARP * WARPS;
constexpr int LDS = H + 8;                     // padded bf16 row stride in shared memory
constexpr int NSMALL = H * 4 + H + H + H + 1;  // dW1, db1, db2, dW3, db3 block accumulators

__device__ __forceinline__ float gelu_f(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
    return cdf + z * pdf;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// D += A(16x16, row-major) * B(16x8, column-major), bf16 inputs, fp32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment of a 16x16 tile of a row-major bf16 matrix M (row stride ld):
// rows g and g+8, columns 2t, 2t+1 and 2t+8, 2t+9 (g = lane/4, t = lane%4).
__device__ __forceinline__ void load_a(uint32_t (&a)[4], const __nv_bfloat16 *M, int ld, int k0, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 *p0 = M + (size_t)g * ld + k0 + 2 * t;
    const __nv_bfloat16 *p1 = M + (size_t)(g + 8) * ld + k0 + 2 * t;
    a[0] = *reinterpret_cast<const uint32_t *>(p0);
    a[1] = *reinterpret_cast<const uint32_t *>(p1);
    a[2] = *reinterpret_cast<const uint32_t *>(p0 + 8);
    a[3] = *reinterpret_cast<const uint32_t *>(p1 + 8);
}

// B fragment of the 16x8 tile B(k, n) = Mt[n][k] of a matrix stored with k
// contiguous (row n of Mt, stride ld): k = 2t, 2t+1 and 2t+8, 2t+9, n = g.
__device__ __forceinline__ void load_b(uint32_t (&b)[2], const __nv_bfloat16 *Mt, int ld, int n0, int k0,
                                       int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 *p = Mt + (size_t)(n0 + g) * ld + k0 + 2 * t;
    b[0] = *reinterpret_cast<const uint32_t *>(p);
    b[1] = *reinterpret_cast<const uint32_t *>(p + 8);
}

struct MlpShared {
    __nv_bfloat16 w2[H * LDS];     // W2[out][in]
    __nv_bfloat16 w2t[H * LDS];    // W2^T[in][out]
    __nv_bfloat16 h1[WARPS][ROWS_PER_WARP * LDS];     // bf16(h1)
    __nv_bfloat16 h1lo[WARPS][ROWS_PER_WARP * LDS];   // bf16(h1 - bf16(h1))
    __nv_bfloat16 dz2[WARPS][ROWS_PER_WARP * LDS];
    float w1[H * 4], b1[H], b2[H], w3[H];
    float b3;
    float acc[NSMALL];             // block partial sums of the small gradients
    float loss;
};

// Forward (and, for TRAIN, backward) of ROWS_PER_BLOCK rows per block.
// TRAIN writes h1^T and dz2^T (bf16, [H][ldT]) for the dW2 contraction and adds
// the block's partial gradients of W1, b1, b2, W3, b3 and the loss to grad.
template <bool TRAIN>
__global__ void __launch_bounds__(WARPS * 32)
mlp_rows_kernel(const __nv_bfloat16 *__restrict__ wq, const float *__restrict__ X,
                const float *__restrict__ target, float *__restrict__ y_out, int64_t B,
                float inv_b, __nv_bfloat16 *__restrict__ h1T, __nv_bfloat16 *__restrict__ dz2T,
                int64_t ldT, float *__restrict__ grad, float *__restrict__ loss_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpShared &sm = *reinterpret_cast<MlpShared *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    for (int i = tid; i < H * H; i += blockDim.x) {
        const int o = i / H, n = i % H;
        const __nv_bfloat16 v = wq[OFF_W2 + i];
        sm.w2[o * LDS + n] = v;
        sm.w2t[n * LDS + o] = v;
    }
    for (int i = tid; i < H * 4; i += blockDim.x) sm.w1[i] = __bfloat162float(wq[OFF_W1 + i]);
    for (int i = tid; i < H; i += blockDim.x) {
        sm.b1[i] = __bfloat162float(wq[OFF_B1 + i]);
        sm.b2[i] = __bfloat162float(wq[OFF_B2 + i]);
        sm.w3[i] = __bfloat162float(wq[OFF_W3 + i]);
    }
    if (tid == 0) {
        sm.b3 = __bfloat162float(wq[OFF_B3]);
        sm.loss = 0.f;
    }
    if (TRAIN)
        for (int i = tid; i < NSMALL; i += blockDim.x) sm.acc[i] = 0.f;
    __syncthreads();

    const int64_t r0 = (int64_t)blockIdx.x * ROWS_PER_BLOCK + (int64_t)warp * ROWS_PER_WARP;
    __nv_bfloat16 *h1s = sm.h1[warp];
    __nv_bfloat16 *h1l = sm.h1lo[warp];
    // ---- layer 1 (K = 4, fp32): lane owns units n = lane + 32 q for all 16 rows.
    // h1 enters the tensor cores as the sum of two bf16 numbers (hi + lo), so
    // the activations keep about 16 bits of precision while W2 stays bf16.
    float xr[ROWS_PER_WARP][4];
#pragma unroll
    for (int r = 0; r < ROWS_PER_WARP; ++r) {
        const int64_t row = r0 + r;
#pragma unroll
        for (int c = 0; c < 4; ++c) xr[r][c] = row < B ? X[row * 4 + c] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int n = lane + 32 * q;
        const float w0 = sm.w1[n * 4 + 0], w1 = sm.w1[n * 4 + 1], w2 = sm.w1[n * 4 + 2],
                    w3 = sm.w1[n * 4 + 3], bb = sm.b1[n];
#pragma unroll
        for (int r = 0; r < ROWS_PER_WARP; ++r) {
            const float z = bb + xr[r][0] * w0 + xr[r][1] * w1 + xr[r][2] * w2 + xr[r][3] * w3;
            const float hf = gelu_f(z);
            const __nv_bfloat16 h = __float2bfloat16_rn(hf);
            h1s[r * LDS + n] = h;
            h1l[r * LDS + n] = __float2bfloat16_rn(hf - __bfloat162float(h));
            if (TRAIN) {
                const int64_t row = r0 + r;
                if (row < ldT) h1T[(size_t)n * ldT + row] = h;
            }
        }
    }
    __syncwarp();
    // ---- layer 2 on the tensor cores: Z2[16 x 128] = H1[16 x 128] W2^T
    float acc[H / 8][4];
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
    for (int ks = 0; ks < H / 16; ++ks) {
        uint32_t a[4], al[4];
        load_a(a, h1s, LDS, ks * 16, lane);
        load_a(al, h1l, LDS, ks * 16, lane);
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
            uint32_t b[2];
            load_b(b, sm.w2, LDS, nt * 8, ks * 16, lane);
            mma16816(acc[nt], a, b);
            mma16816(acc[nt], al, b);
        }
    }
    // ---- epilogue: h2 = gelu(z2 + b2), y = h2 . W3 + b3 (rows g and g + 8)
    float ya = 0.f, yb = 0.f;
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int col = nt * 8 + 2 * t + (e & 1);
            const float z = acc[nt][e] + sm.b2[col];
            acc[nt][e] = z;                         // keep z2 for the backward pass
            const float h = gelu_f(z) * sm.w3[col];
            if (e < 2) ya += h; else yb += h;
        }
    }
    ya += __shfl_xor_sync(0xffffffffu, ya, 1);
    ya += __shfl_xor_sync(0xffffffffu, ya, 2);
    yb += __shfl_xor_sync(0xffffffffu, yb, 1);
    yb += __shfl_xor_sync(0xffffffffu, yb, 2);
    ya += sm.b3;
    yb += sm.b3;
    const int64_t rowa = r0 + g, rowb = r0 + g + 8;
    if (t == 0) {
        if (y_out && rowa < B) y_out[rowa] = ya;
        if (y_out && rowb < B) y_out[rowb] = yb;
    }
    if (!TRAIN) return;

    // ---- backward: dL/dy = 2 (y - t) / B
    const float ea = rowa < B ? ya - target[rowa] : 0.f;
    const float eb = rowb < B ? yb - target[rowb] : 0.f;
    const float dya = 2.f * ea * inv_b, dyb = 2.f * eb * inv_b;
    if (t == 0) atomicAdd(&sm.loss, (ea * ea + eb * eb) * inv_b);
    __nv_bfloat16 *dzs = sm.dz2[warp];
    float *acc_w1 = sm.acc, *acc_b1 = sm.acc + H * 4, *acc_b2 = acc_b1 + H, *acc_w3 = acc_b2 + H,
          *acc_b3 = acc_w3 + H;
    {
        // db3: sum of dy over the 16 rows (one value per row, from lanes t == 0)
        float v = (t == 0) ? dya + dyb : 0.f;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(acc_b3, v);
    }
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt) {
        float w3g[2], b2g[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int col = nt * 8 + 2 * t + e;
            const float za = acc[nt][e], zb = acc[nt][e + 2];
            // dW3 += dy * h2
            w3g[e] = dya * gelu_f(za) + dyb * gelu_f(zb);
            const float dza = dya * sm.w3[col] * gelu_grad_f(za);
            const float dzb = dyb * sm.w3[col] * gelu_grad_f(zb);
            b2g[e] = dza + dzb;
            acc[nt][e] = dza;
            acc[nt][e + 2] = dzb;
        }
        // reduce over the 8 row groups (lanes with equal t)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
#pragma unroll
            for (int o = 4; o <= 16; o <<= 1) {
                w3g[e] += __shfl_xor_sync(0xffffffffu, w3g[e], o);
                b2g[e] += __shfl_xor_sync(0xffffffffu, b2g[e], o);
            }
        }
        if (g == 0) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int col = nt * 8 + 2 * t + e;
                atomicAdd(acc_w3 + col, w3g[e]);
                atomicAdd(acc_b2 + col, b2g[e]);
            }
        }
        // dz2 (bf16) to shared memory, row-major, and transposed to global
        const int col = nt * 8 + 2 * t;
        *reinterpret_cast<uint32_t *>(dzs + g * LDS + col) = pack_bf16(acc[nt][0], acc[nt][1]);
        *reinterpret_cast<uint32_t *>(dzs + (g + 8) * LDS + col) = pack_bf16(acc[nt][2], acc[nt][3]);
        if (rowa < ldT) {
            dz2T[(size_t)col * ldT + rowa] = __float2bfloat16_rn(acc[nt][0]);
            dz2T[(size_t)(col + 1) * ldT + rowa] = __float2bfloat16_rn(acc[nt][1]);
        }
        if (rowb < ldT) {
            dz2T[(size_t)col * ldT + rowb] = __float2bfloat16_rn(acc[nt][2]);
            dz2T[(size_t)(col + 1) * ldT + rowb] = __float2bfloat16_rn(acc[nt][3]);
        }
    }
    __syncwarp();
    // ---- dH1[16 x 128] = dZ2[16 x 128] W2 on the tensor cores (B(k=out, n=in) = W2^T[in][out])
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
    for (int ks = 0; ks < H / 16; ++ks) {
        uint32_t a[4];
        load_a(a, dzs, LDS, ks * 16, lane);
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
            uint32_t b[2];
            load_b(b, sm.w2t, LDS, nt * 8, ks * 16, lane);
            mma16816(acc[nt], a, b);
        }
    }
    // ---- dz1 = dh1 * gelu'(z1); dW1 += dz1 x^T, db1 += dz1 (z1 recomputed in fp32)
    float xa[4], xb[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        xa[c] = rowa < B ? X[rowa * 4 + c] : 0.f;
        xb[c] = rowb < B ? X[rowb * 4 + c] : 0.f;
    }
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int n = nt * 8 + 2 * t + e;
            const float w0 = sm.w1[n * 4 + 0], w1 = sm.w1[n * 4 + 1], w2 = sm.w1[n * 4 + 2],
                        w3 = sm.w1[n * 4 + 3], bb = sm.b1[n];
            const float za = bb + xa[0] * w0 + xa[1] * w1 + xa[2] * w2 + xa[3] * w3;
            const float zb = bb + xb[0] * w0 + xb[1] * w1 + xb[2] * w2 + xb[3] * w3;
            const float da = rowa < B ? acc[nt][e] * gelu_grad_f(za) : 0.f;
            const float db = rowb < B ? acc[nt][e + 2] * gelu_grad_f(zb) : 0.f;
            float gw[5] = {da * xa[0] + db * xb[0], da * xa[1] + db * xb[1],
                           da * xa[2] + db * xb[2], da * xa[3] + db * xb[3], da + db};
#pragma unroll
            for (int c = 0; c < 5; ++c)
#pragma unroll
                for (int o = 4; o <= 16; o <<= 1) gw[c] += __shfl_xor_sync(0xffffffffu, gw[c], o);
            if (g == 0) {
#pragma unroll
                for (int c = 0; c < 4; ++c) atomicAdd(acc_w1 + n * 4 + c, gw[c]);
                atomicAdd(acc_b1 + n, gw[4]);
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < NSMALL; i += blockDim.x) {
        int off;
        if (i < H * 4) off = OFF_W1 + i;
        else if (i < H * 5) off = OFF_B1 + (i - H * 4);
        else if (i < H * 6) off = OFF_B2 + (i - H * 5);
        else if (i < H * 7) off = OFF_W3 + (i - H * 6);
        else off = OFF_B3;
        atomicAdd(grad + off, sm.acc[i]);
    }
    if (tid == 0) atomicAdd(loss_out, sm.loss);
}

// dW2[out][in] += sum over rows of dz2T[out][row] h1T[in][row]: a 128x128
// contraction over the batch.  Each block takes a chunk of 256 rows; warp w
// owns output rows 32w .. 32w+31 (two 16-row tiles) and all 128 columns.
constexpr int DW2_ROWS = 256;

__global__ void __launch_bounds__(WARPS * 32)
mlp_dw2_kernel(const __nv_bfloat16 *__restrict__ dz2T, const __nv_bfloat16 *__restrict__ h1T,
               int64_t ldT, float *__restrict__ grad)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t k_begin = (int64_t)blockIdx.x * DW2_ROWS;
    const int64_t k_end = k_begin + DW2_ROWS < ldT ? k_begin + DW2_ROWS : ldT;
    float acc[2][H / 8][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
    for (int64_t k0 = k_begin; k0 < k_end; k0 += 16) {
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
            load_a(a[mt], dz2T + (size_t)(warp * 32 + mt * 16) * ldT, (int)ldT, (int)k0, lane);
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
            uint32_t b[2];
            load_b(b, h1T, (int)ldT, nt * 8, (int)k0, lane);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma16816(acc[mt][nt], a[mt], b);
        }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
            const int o = warp * 32 + mt * 16 + g, n = nt * 8 + 2 * t;
            float *gw = grad + OFF_W2;
            atomicAdd(gw + o * H + n, acc[mt][nt][0]);
            atomicAdd(gw + o * H + n + 1, acc[mt][nt][1]);
            atomicAdd(gw + (o + 8) * H + n, acc[mt][nt][2]);
            atomicAdd(gw + (o + 8) * H + n + 1, acc[mt][nt][3]);
        }
}

// Adam (Kingma and Ba) on the fp32 master parameters, then the bf16 copy.
__global__ void mlp_adam_kernel(float *__restrict__ w, float *__restrict__ grad, float *__restrict__ m1,
                                float *__restrict__ m2, __nv_bfloat16 *__restrict__ wq, int n, float lr,
                                float beta1, float beta2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gr = grad[i];
    const float a = beta1 * m1[i] + (1.f - beta1) * gr;
    const float b = beta2 * m2[i] + (1.f - beta2) * gr * gr;
    m1[i] = a;
    m2[i] = b;
    const float v = w[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    w[i] = v;
    wq[i] = __float2bfloat16_rn(v);
    grad[i] = 0.f;
}

__global__ void mlp_round_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wq, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wq[i] = __float2bfloat16_rn(w[i]);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct Mlp {
    int device = -1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *w = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr, *loss = nullptr;
    __nv_bfloat16 *wq = nullptr;
    int64_t cap = 0;           // rows of the batch buffers (multiple of 256)
    float *X = nullptr, *t = nullptr, *y = nullptr;
    __nv_bfloat16 *h1T = nullptr, *dz2T = nullptr;
    int *d_err = nullptr;      // error flag of the tcgen05 kernels
    float *part = nullptr;     // per-CTA gradient rows of the tcgen05 training kernel
    size_t part_floats = 0;
    bool use_tc = true;        // forward, gradients and training on tcgen05 (else mma.sync)
    int64_t step = 0;
    std::string err;
};

thread_local std::string g_mlp_err;

int mfail(Mlp *m, int code, const std::string &msg)
{
    if (m) m->err = msg; else g_mlp_err = msg;
    return code;
}

#define MLP_TRY(m, call)                                                                        \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return mfail((m), e_ == cudaErrorMemoryAllocation ? MUCAL_ERR_OOM : MUCAL_ERR_CUDA, \
                         std::string(#call ": ") + cudaGetErrorString(e_));                     \
    } while (0)

int ensure_capacity(Mlp *m, int64_t B)
{
    const int64_t need = ((B + 255) / 256) * 256;
    if (need <= m->cap) return MUCAL_OK;
    cudaFree(m->X); cudaFree(m->t); cudaFree(m->y); cudaFree(m->h1T); cudaFree(m->dz2T);
    m->X = m->t = m->y = nullptr;
    m->h1T = m->dz2T = nullptr;
    m->cap = 0;
    MLP_TRY(m, cudaMalloc(&m->X, need * 4 * sizeof(float)));
    MLP_TRY(m, cudaMalloc(&m->t, need * sizeof(float)));
    MLP_TRY(m, cudaMalloc(&m->y, need * sizeof(float)));
    MLP_TRY(m, cudaMalloc(&m->h1T, (size_t)H * need * sizeof(__nv_bfloat16)));
    MLP_TRY(m, cudaMalloc(&m->dz2T, (size_t)H * need * sizeof(__nv_bfloat16)));
    m->cap = need;
    return MUCAL_OK;
}

int upload_batch(Mlp *m, const float *X, const float *t, int64_t B)
{
    int rc = ensure_capacity(m, B);
    if (rc != MUCAL_OK) return rc;
    MLP_TRY(m, cudaMemsetAsync(m->X, 0, m->cap * 4 * sizeof(float), m->stream));
    MLP_TRY(m, cudaMemcpyAsync(m->X, X, B * 4 * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    if (t) {
        MLP_TRY(m, cudaMemsetAsync(m->t, 0, m->cap * sizeof(float), m->stream));
        MLP_TRY(m, cudaMemcpyAsync(m->t, t, B * sizeof(float), cudaMemcpyHostToDevice, m->stream));
        // rows past B contribute nothing: their dz2 is zero
        MLP_TRY(m, cudaMemsetAsync(m->h1T, 0, (size_t)H * m->cap * sizeof(__nv_bfloat16), m->stream));
        MLP_TRY(m, cudaMemsetAsync(m->dz2T, 0, (size_t)H * m->cap * sizeof(__nv_bfloat16), m->stream));
    }
    return MUCAL_OK;
}

size_t rows_smem() { return sizeof(MlpShared); }

int ensure_err(Mlp *m)
{
    if (!m->d_err) {
        MLP_TRY(m, cudaMalloc(&m->d_err, sizeof(int)));
        MLP_TRY(m, cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream));
    }
    return MUCAL_OK;
}

// Read and clear the tcgen05 error flag (waits for the stream).
int check_tc(Mlp *m)
{
    if (!m->d_err) return MUCAL_OK;
    int flag = 0;
    MLP_TRY(m, cudaMemcpyAsync(&flag, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    if (flag) {
        MLP_TRY(m, cudaMemset(m->d_err, 0, sizeof(int)));
        return mfail(m, MUCAL_ERR_STATE, "tcgen05 kernel: a tensor-core wait ran out");
    }
    return MUCAL_OK;
}

int enqueue_grad(Mlp *m, int64_t B)
{
    const int blocks = (int)((B + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
    MLP_TRY(m, cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream));
    if (m->use_tc) {
        int rc = ensure_err(m);
        if (rc != MUCAL_OK) return rc;
        const size_t need = mucal::mlp_train_tcgen05_partial_floats(B);
        if (need > m->part_floats) {
            MLP_TRY(m, cudaStreamSynchronize(m->stream));
            cudaFree(m->part);
            m->part = nullptr;
            m->part_floats = 0;
            MLP_TRY(m, cudaMalloc(&m->part, need * sizeof(float)));
            m->part_floats = need;
        }
        MLP_TRY(m, mucal::mlp_train_tcgen05(m->wq, m->X, m->t, B, m->part, m->grad, m->loss,
                                            m->d_err, m->stream));
        return MUCAL_OK;
    }
    mlp_rows_kernel<true><<<blocks, WARPS * 32, rows_smem(), m->stream>>>(
        m->wq, m->X, m->t, m->y, B, 1.0f / (float)B, m->h1T, m->dz2T, m->cap, m->grad, m->loss);
    MLP_TRY(m, cudaGetLastError());
    const int kblocks = (int)(m->cap / DW2_ROWS);
    mlp_dw2_kernel<<<kblocks, WARPS * 32, 0, m->stream>>>(m->dz2T, m->h1T, m->cap, m->grad);
    MLP_TRY(m, cudaGetLastError());
    return MUCAL_OK;
}

}  // namespace

extern "C" {

int mucal_mlp_param_count(void) { return NPARAM; }

const char *mucal_mlp_last_error(void *mlp)
{
    Mlp *m = static_cast<Mlp *>(mlp);
    return m ? m->err.c_str() : g_mlp_err.c_str();
}

int mucal_mlp_create(void **out, const float *params, int64_t n, void *cuda_stream)
{
    if (!out) return mfail(nullptr, MUCAL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!params || n != NPARAM) return mfail(nullptr, MUCAL_ERR_INVALID_ARG, "need 17281 parameters");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        return mfail(nullptr, MUCAL_ERR_NO_DEVICE, "no CUDA device available");
    }
    Mlp *m = new Mlp();
    auto bail = [&](int code) {
        g_mlp_err = m->err;
        cudaFree(m->w); cudaFree(m->grad); cudaFree(m->m1); cudaFree(m->m2); cudaFree(m->wq);
        cudaFree(m->loss);
        if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
        delete m;
        return code;
    };
    cudaGetDevice(&m->device);
    if (cuda_stream) {
        m->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(mfail(m, MUCAL_ERR_CUDA, "stream creation failed"));
        m->own_stream = true;
    }
    if (cudaMalloc(&m->w, NPARAM * 4) != cudaSuccess || cudaMalloc(&m->grad, NPARAM * 4) != cudaSuccess ||
        cudaMalloc(&m->m1, NPARAM * 4) != cudaSuccess || cudaMalloc(&m->m2, NPARAM * 4) != cudaSuccess ||
        cudaMalloc(&m->wq, NPARAM * 2) != cudaSuccess || cudaMalloc(&m->loss, 4) != cudaSuccess)
        return bail(mfail(m, MUCAL_ERR_OOM, "cudaMalloc failed"));
    if (cudaFuncSetAttribute(mlp_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rows_smem()) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_rows_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rows_smem()) != cudaSuccess)
        return bail(mfail(m, MUCAL_ERR_CUDA, "shared-memory opt-in failed"));
    if (cudaMemcpyAsync(m->w, params, NPARAM * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->grad, 0, NPARAM * 4, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->m1, 0, NPARAM * 4, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->m2, 0, NPARAM * 4, m->stream) != cudaSuccess)
        return bail(mfail(m, MUCAL_ERR_CUDA, "parameter upload failed"));
    mlp_round_kernel<<<(NPARAM + 255) / 256, 256, 0, m->stream>>>(m->w, m->wq, NPARAM);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess)
        return bail(mfail(m, MUCAL_ERR_CUDA, "parameter rounding failed"));
    *out = m;
    return MUCAL_OK;
}

void mucal_mlp_destroy(void *mlp)
{
    Mlp *m = static_cast<Mlp *>(mlp);
    if (!m) return;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    cudaFree(m->w); cudaFree(m->grad); cudaFree(m->m1); cudaFree(m->m2); cudaFree(m->wq);
    cudaFree(m->loss); cudaFree(m->X); cudaFree(m->t); cudaFree(m->y); cudaFree(m->h1T);
    cudaFree(m->dz2T); cudaFree(m->part);
    cudaFree(m->d_err);
    if (m->own_stream) cudaStreamDestroy(m->stream);
    delete m;
}

int mucal_mlp_get_params(void *mlp, float *params, int64_t n, int32_t rounded)
{
    Mlp *m = static_cast<Mlp *>(mlp);
    if (!m || !params || n != NPARAM) return mfail(m, MUCAL_ERR_INVALID_ARG, "need 17281 parameters");
    MLP_TRY(m, cudaSetDevice(m->device));
    if (!rounded) {
        MLP_TRY(m, cudaMemcpyAsync(params, m->w, NPARAM * 4, cudaMemcpyDeviceToHost, m->stream));
        MLP_TRY(m, cudaStreamSynchronize(m->stream));
        return MUCAL_OK;
    }
    std::vector<__nv_bfloat16> q(NPARAM);
    MLP_TRY(m, cudaMemcpyAsync(q.data(), m->wq, NPARAM * 2, cudaMemcpyDeviceToHost, m->stream));
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    for (int i = 0; i < NPARAM; ++i) {
        uint16_t bits;
        std::memcpy(&bits, &q[i], 2);
        const uint32_t f = (uint32_t)bits << 16;
        std::memcpy(&params[i], &f, 4);
    }
    return MUCAL_OK;
}

int mucal_mlp_use_tcgen05(void *mlp, int32_t enable)
{
    Mlp *m = static_cast<Mlp *>(mlp);
    if (!m) return mfail(m, MUCAL_ERR_INVALID_ARG, "mlp is NULL");
    m->use_tc = enable != 0;
    return MUCAL_OK;
}

int mucal_mlp_forward(void *mlp, const float *X, int64_t B, float *y)
{
    Mlp *m = static_cast<Mlp *>(mlp);
    if (m && m->use_tc) return mucal_mlp_forward_tcgen05(mlp, X, B, y);
    if (!m || !X || !y || B <= 0) return mfail(m, MUCAL_ERR_INVALID_ARG, "bad forward arguments");
    MLP_TRY(m, cudaSetDevice(m->device));
    int rc = upload_batch(m, X, nullptr, B);
    if (rc != MUCAL_OK) return rc;
    const int blocks = (int)((B + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
    mlp_rows_kernel<false><<<blocks, WARPS * 32, rows_smem(), m->stream>>>(
        m->wq, m->X, nullptr, m->y, B, 0.f, nullptr, nullptr, 0, nullptr, nullptr);
    MLP_TRY(m, cudaGetLastError());
    MLP_TRY(m, cudaMemcpyAsync(y, m->y, B * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    return MUCAL_OK;
}

int mucal_mlp_forward_tcgen05(void *mlp, const float *X, int64_t B, float *y)
{
    Mlp *m = static_cast<Mlp *>(mlp);
    if (!m || !X || !y || B <= 0) return mfail(m, MUCAL_ERR_INVALID_ARG, "bad forward arguments");
    MLP_TRY(m, cudaSetDevice(m->device));
    int rc = upload_batch(m, X, nullptr, B);
    if (rc != MUCAL_OK) return rc;
    rc = ensure_err(m);
    if (rc != MUCAL_OK) return rc;
    MLP_TRY(m, mucal::mlp_forward_tcgen05(m->wq, m->X, m->y, B, m->d_err, m->stream));
    MLP_TRY(m, cudaMemcpyAsync(y, m->y, B * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    return check_tc(m);
}

int mucal_mlp_gradients(void *mlp, const float *X, const float *t, int64_t B, float *loss, float *grad)
{
    Mlp *m = static_cast<Mlp *>(mlp);
    if (!m || !X || !t || B <= 0) return mfail(m, MUCAL_ERR_INVALID_ARG, "bad gradient arguments");
    MLP_TRY(m, cudaSetDevice(m->device));
    int rc = upload_batch(m, X, t, B);
    if (rc != MUCAL_OK) return rc;
    MLP_TRY(m, cudaMemsetAsync(m->grad, 0, NPARAM * 4, m->stream));
    rc = enqueue_grad(m, B);
    if (rc != MUCAL_OK) return rc;
    if (grad) MLP_TRY(m, cudaMemcpyAsync(grad, m->grad, NPARAM * 4, cudaMemcpyDeviceToHost, m->stream));
    if (loss) MLP_TRY(m, cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream));
    MLP_TRY(m, cudaMemsetAsync(m->grad, 0, NPARAM * 4, m->stream));
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    return check_tc(m);
}

int mucal_mlp_train(void *mlp, const float *X, const float *t, int64_t B, int32_t steps, float lr,
                    float *loss_out)
{
    Mlp *m = static_cast<Mlp *>(mlp);
    if (!m || !X || !t || B <= 0 || steps <= 0 || !(lr > 0.f))
        return mfail(m, MUCAL_ERR_INVALID_ARG, "bad training arguments");
    MLP_TRY(m, cudaSetDevice(m->device));
    int rc = upload_batch(m, X, t, B);
    if (rc != MUCAL_OK) return rc;
    MLP_TRY(m, cudaMemsetAsync(m->grad, 0, NPARAM * 4, m->stream));
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    for (int s = 0; s < steps; ++s) {
        rc = enqueue_grad(m, B);
        if (rc != MUCAL_OK) return rc;
        m->step += 1;
        const float c1 = 1.f - std::pow(beta1, (float)m->step);
        const float c2 = 1.f - std::pow(beta2, (float)m->step);
        mlp_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, m->stream>>>(
            m->w, m->grad, m->m1, m->m2, m->wq, NPARAM, lr, beta1, beta2, eps, c1, c2);
        MLP_TRY(m, cudaGetLastError());
    }
    if (loss_out) MLP_TRY(m, cudaMemcpyAsync(loss_out, m->loss, 4, cudaMemcpyDeviceToHost, m->stream));
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    return check_tc(m);
}

}  // extern "C"
