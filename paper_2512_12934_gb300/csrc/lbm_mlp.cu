// Surrogate MLP ensemble (4 -> 128 -> 128 -> 128 -> 2, GELU), FP32, with
// fused forward, backward and Adam kernels, and an inference kernel that
// runs the two hidden layers on the tcgen05 tensor cores (FP32-accurate
// split products; the default inference path).
//
// One CTA owns TILE samples of one ensemble member.  Forward: the four layers
// run back to back on activations held in shared memory; each 128x128 weight
// matrix is staged transposed so a thread's 4x4 output block reads its four
// weights as one conflict-free float4.  Backward: the whole chain rule for the
// tile (output error, dZ3, dW3, dA2, dZ2, dW2, dA1, dZ1, dW1 and the biases)
// stays on chip; the tile writes its gradient partial with plain stores.  Adam
// sums the tiles' partials in a fixed order (deterministic) and updates.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int I = 4, H = 128, O = 2;
constexpr int TILE = 32;        // samples per CTA
constexpr int NTH = 256;        // threads per CTA
constexpr int oW1 = 0, ob1 = oW1 + H * I, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + H * H;
constexpr int oW4 = ob3 + H, ob4 = oW4 + O * H, P = ob4 + O;
// Device stride of one member's parameters: P rounded up to 32 floats so that
// every member (and every weight matrix in it) starts 128-byte aligned.
constexpr int PS = (P + 31) & ~31;
constexpr size_t SMEM_BYTES = (size_t)(H * H + 2 * TILE * H) * sizeof(float);

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// Stage W [H][H] (row = output neuron) transposed into smem Wt[k][j].
__device__ __forceinline__ void stage_transposed(float* Wt, const float* __restrict__ W) {
    for (int idx = threadIdx.x; idx < H * H; idx += NTH) {
        const int k = idx / H, j = idx % H;  // consecutive threads: consecutive j -> conflict-free store
        Wt[k * H + j] = __ldg(W + j * H + k);
    }
}

// Stage W [H][H] as is into smem (used when the contraction runs over the row index).
__device__ __forceinline__ void stage_plain(float* Ws, const float* __restrict__ W) {
    for (int idx = threadIdx.x; idx < H * H / 4; idx += NTH)
        reinterpret_cast<float4*>(Ws)[idx] = __ldg(reinterpret_cast<const float4*>(W) + idx);
}

// out[s][j] = bias[j] + sum_k in[s][k] * M[k][j] for the tile; M in smem laid out
// [k][j].  Thread: samples 4*sg..+3, columns 4*ng..+3.
__device__ __forceinline__ void tile_gemm(const float* in, const float* M, const float* bias, float (&acc)[4][4]) {
    const int sg = threadIdx.x / 32, ng = threadIdx.x % 32;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = bias ? __ldg(bias + 4 * ng + c) : 0.0f;
#pragma unroll 4
    for (int k = 0; k < H; ++k) {
        const float4 w = reinterpret_cast<const float4*>(M + k * H)[ng];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float a = in[(4 * sg + r) * H + k];
            acc[r][0] = fmaf(a, w.x, acc[r][0]);
            acc[r][1] = fmaf(a, w.y, acc[r][1]);
            acc[r][2] = fmaf(a, w.z, acc[r][2]);
            acc[r][3] = fmaf(a, w.w, acc[r][3]);
        }
    }
}

// Forward pass of TILE samples for one member.  idx (optional) selects rows of X.
// TRAIN: pre-activations Z1..Z3 [E][B][H] are kept for the backward pass.
template <bool TRAIN>
__global__ void __launch_bounds__(NTH) mlp_forward_kernel(const float* __restrict__ params, const float* __restrict__ X,
                                                          const int* __restrict__ idx, int B, float* __restrict__ Y,
                                                          float* __restrict__ Z) {
    extern __shared__ __align__(16) float smem[];
    float* Wt = smem;               // [H][H]
    float* actA = smem + H * H;     // [TILE][H]
    float* actB = actA + TILE * H;  // [TILE][H]
    const int e = blockIdx.y, s0 = blockIdx.x * TILE;
    const float* p = params + (size_t)e * PS;
    const int sg = threadIdx.x / 32, ng = threadIdx.x % 32;
    // layer 1 (K = 4) straight from global
    for (int q = threadIdx.x; q < TILE * H; q += NTH) {
        const int s = q / H, j = q % H, b = s0 + s;
        float z = __ldg(p + ob1 + j);
        if (b < B) {
            const int row = idx ? idx[b] : b;
#pragma unroll
            for (int k = 0; k < I; ++k) z = fmaf(__ldg(p + oW1 + j * I + k), __ldg(X + (size_t)row * I + k), z);
        }
        if (TRAIN && b < B) Z[((size_t)e * 3 + 0) * B * H + (size_t)b * H + j] = z;
        actA[s * H + j] = gelu(z);
    }
    // layers 2 and 3
    const float* in = actA;
    float* out = actB;
#pragma unroll 1
    for (int l = 0; l < 2; ++l) {
        __syncthreads();
        stage_transposed(Wt, p + (l == 0 ? oW2 : oW3));
        __syncthreads();
        float acc[4][4];
        tile_gemm(in, Wt, p + (l == 0 ? ob2 : ob3), acc);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int s = 4 * sg + r, b = s0 + s;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = 4 * ng + c;
                if (TRAIN && b < B) Z[((size_t)e * 3 + 1 + l) * B * H + (size_t)b * H + j] = acc[r][c];
                out[s * H + j] = gelu(acc[r][c]);
            }
        }
        const float* t = in;
        in = out;
        out = const_cast<float*>(t);
    }
    __syncthreads();
    // layer 4 (2 outputs): one warp per group of 4 samples, lanes split k
    {
        const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int s = 4 * w + r, b = s0 + s;
            float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
            for (int q = 0; q < H / 32; ++q) {
                const int k = lane + 32 * q;
                const float a = in[s * H + k];
                y0 = fmaf(a, __ldg(p + oW4 + k), y0);
                y1 = fmaf(a, __ldg(p + oW4 + H + k), y1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                y0 += __shfl_down_sync(0xffffffffu, y0, o);
                y1 += __shfl_down_sync(0xffffffffu, y1, o);
            }
            if (lane == 0 && b < B) {
                Y[((size_t)e * B + b) * O + 0] = y0 + __ldg(p + ob4);
                Y[((size_t)e * B + b) * O + 1] = y1 + __ldg(p + ob4 + 1);
            }
        }
    }
}

// Backward pass of TILE samples of one member; writes this tile's gradient
// partial gp[e][tile][P].  T: targets indexed like X (through idx); the MSE is
// normalised by B * O.
__global__ void __launch_bounds__(NTH) mlp_backward_kernel(const float* __restrict__ params, const float* __restrict__ X,
                                                           const float* __restrict__ T, const int* __restrict__ idx, int B,
                                                           const float* __restrict__ Y, const float* __restrict__ Z,
                                                           float* __restrict__ gp) {
    extern __shared__ __align__(16) float smem[];
    float* Ws = smem;               // [H][H] weights (plain layout)
    float* dZ = smem + H * H;       // [TILE][H]
    float* A = dZ + TILE * H;       // [TILE][H] activations of the layer below
    __shared__ float dY[TILE][O];
    const int e = blockIdx.y, tile = blockIdx.x, s0 = tile * TILE, ntile = gridDim.x;
    const float* p = params + (size_t)e * PS;
    float* g = gp + ((size_t)e * ntile + tile) * P;
    const float* Z1 = Z + ((size_t)e * 3 + 0) * B * H;
    const float* Z2 = Z + ((size_t)e * 3 + 1) * B * H;
    const float* Z3 = Z + ((size_t)e * 3 + 2) * B * H;
    const float scale = 2.0f / (float)(B * O);
    if (threadIdx.x < TILE * O) {
        const int s = threadIdx.x / O, o = threadIdx.x % O, b = s0 + s;
        float d = 0.0f;
        if (b < B) {
            const int row = idx ? idx[b] : b;
            d = scale * (Y[((size_t)e * B + b) * O + o] - __ldg(T + (size_t)row * O + o));
        }
        dY[s][o] = d;
    }
    // A <- A3 = gelu(Z3)
    for (int q = threadIdx.x; q < TILE * H; q += NTH) {
        const int s = q / H, j = q % H, b = s0 + s;
        A[q] = b < B ? gelu(Z3[(size_t)b * H + j]) : 0.0f;
    }
    __syncthreads();
    // output layer: dW4, db4 and dZ3 = (dY W4) * gelu'(Z3)
    for (int q = threadIdx.x; q < O * H; q += NTH) {
        const int o = q / H, k = q % H;
        float acc = 0.0f;
        for (int s = 0; s < TILE; ++s) acc = fmaf(dY[s][o], A[s * H + k], acc);
        g[oW4 + q] = acc;
    }
    if (threadIdx.x < O) {
        float acc = 0.0f;
        for (int s = 0; s < TILE; ++s) acc += dY[s][threadIdx.x];
        g[ob4 + threadIdx.x] = acc;
    }
    for (int q = threadIdx.x; q < TILE * H; q += NTH) {
        const int s = q / H, k = q % H, b = s0 + s;
        const float da = dY[s][0] * __ldg(p + oW4 + k) + dY[s][1] * __ldg(p + oW4 + H + k);
        dZ[q] = b < B ? da * gelu_grad(Z3[(size_t)b * H + k]) : 0.0f;
    }
    __syncthreads();
    // hidden layers 3 and 2: dW = dZ^T A (A = gelu of the layer below), db,
    // then dZ_below = (dZ W) * gelu'(Z_below)
#pragma unroll 1
    for (int l = 0; l < 2; ++l) {
        const int oW = l == 0 ? oW3 : oW2, ob = l == 0 ? ob3 : ob2;
        const float* Zb = l == 0 ? Z2 : Z1;
        for (int q = threadIdx.x; q < TILE * H; q += NTH) {
            const int s = q / H, j = q % H, b = s0 + s;
            A[q] = b < B ? gelu(Zb[(size_t)b * H + j]) : 0.0f;
        }
        stage_plain(Ws, p + oW);
        __syncthreads();
        {
            // dW[j][k] = sum_s dZ[s][j] A[s][k]: thread -> 8 j x 8 k
            const int jg = threadIdx.x / 16, kg = threadIdx.x % 16;
            float acc[8][8];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[a][c] = 0.0f;
            for (int s = 0; s < TILE; ++s) {
                const float4 z0 = reinterpret_cast<const float4*>(dZ + s * H + 8 * jg)[0];
                const float4 z1 = reinterpret_cast<const float4*>(dZ + s * H + 8 * jg)[1];
                const float4 a0 = reinterpret_cast<const float4*>(A + s * H + 8 * kg)[0];
                const float4 a1 = reinterpret_cast<const float4*>(A + s * H + 8 * kg)[1];
                const float zz[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
                const float aa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(zz[a], aa[c], acc[a][c]);
            }
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = 0; c < 8; ++c) g[oW + (8 * jg + a) * H + 8 * kg + c] = acc[a][c];
        }
        if (threadIdx.x < H) {
            float acc = 0.0f;
            for (int s = 0; s < TILE; ++s) acc += dZ[s * H + threadIdx.x];
            g[ob + threadIdx.x] = acc;
        }
        // dA[s][k] = sum_j dZ[s][j] W[j][k]  (W plain: row j contiguous over k)
        float acc[4][4];
        tile_gemm(dZ, Ws, nullptr, acc);
        __syncthreads();  // everyone is done reading dZ
        {
            const int sg = threadIdx.x / 32, ng = threadIdx.x % 32;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int s = 4 * sg + r, b = s0 + s;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int k = 4 * ng + c;
                    dZ[s * H + k] = b < B ? acc[r][c] * gelu_grad(Zb[(size_t)b * H + k]) : 0.0f;
                }
            }
        }
        __syncthreads();
    }
    // first layer: dW1[j][i] = sum_s dZ1[s][j] x[s][i], db1
    for (int q = threadIdx.x; q < H * I; q += NTH) {
        const int j = q / I, i = q % I;
        float acc = 0.0f;
        for (int s = 0; s < TILE; ++s) {
            const int b = s0 + s;
            if (b < B) acc = fmaf(dZ[s * H + j], __ldg(X + (size_t)(idx ? idx[b] : b) * I + i), acc);
        }
        g[oW1 + q] = acc;
    }
    if (threadIdx.x < H) {
        float acc = 0.0f;
        for (int s = 0; s < TILE; ++s) acc += dZ[s * H + threadIdx.x];
        g[ob1 + threadIdx.x] = acc;
    }
}

// Sum of the tiles' partials in tile order -> gradient (and optional Adam).
__global__ void __launch_bounds__(256) mlp_adam_kernel(float* __restrict__ params, float* __restrict__ m,
                                                       float* __restrict__ v, const float* __restrict__ gp, int ntile,
                                                       float lr, float b1, float b2, float c1, float c2, float eps,
                                                       int adam, float* __restrict__ grad_out) {
    const int e = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    float g = 0.0f;
    for (int t = 0; t < ntile; ++t) g += gp[((size_t)e * ntile + t) * P + q];
    const size_t n = (size_t)e * PS + q;
    if (grad_out) grad_out[(size_t)e * P + q] = g;
    if (!adam) return;
    const float mm = b1 * m[n] + (1.0f - b1) * g;
    const float vv = b2 * v[n] + (1.0f - b2) * g * g;
    m[n] = mm;
    v[n] = vv;
    params[n] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// ---- inference kernel: 128 samples per CTA, 8x8 register tiles -----------
// Activations live feature-major in shared memory (act[k][s]); the hidden
// weights are staged from a k-major copy (Wt[k][j]) with 16-byte loads, so a
// thread's inner step reads two float4 of weights and two float4 of inputs
// for 64 FMAs.
constexpr int TB = 128;   // samples per CTA
constexpr int NTB = 256;  // threads: 16 neuron groups x 16 sample groups of 8
constexpr size_t SMEM_BIG = (size_t)(H * H + 2 * H * TB) * sizeof(float);

// Wt[e][l][k][j] = W_{l+2}[j][k] for the two hidden 128x128 layers.
__global__ void mlp_transpose_kernel(const float* __restrict__ params, float* __restrict__ wt) {
    const int e = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;  // over 2 * H * H
    if (q >= 2 * H * H) return;
    const int l = q / (H * H), r = q % (H * H), k = r / H, j = r % H;
    wt[(size_t)e * 2 * H * H + q] = params[(size_t)e * PS + (l ? oW3 : oW2) + j * H + k];
}

__global__ void __launch_bounds__(NTB) mlp_infer_kernel(const float* __restrict__ params,
                                                         const float* __restrict__ wt, const float* __restrict__ X,
                                                         int B, float* __restrict__ Y) {
    extern __shared__ __align__(16) float smem[];
    float* Wt = smem;              // [H][H]
    float* actA = smem + H * H;    // [H][TB]
    float* actB = actA + H * TB;   // [H][TB]
    const int e = blockIdx.y, s0 = blockIdx.x * TB;
    const float* p = params + (size_t)e * PS;
    // layer 1 (K = 4): consecutive threads take consecutive samples
    for (int q = threadIdx.x; q < TB * H; q += NTB) {
        const int j = q / TB, sl = q % TB, b = s0 + sl;
        float z = __ldg(p + ob1 + j);
        if (b < B) {
#pragma unroll
            for (int k = 0; k < I; ++k) z = fmaf(__ldg(p + oW1 + j * I + k), __ldg(X + (size_t)b * I + k), z);
        }
        actA[j * TB + sl] = gelu(z);
    }
    const int ng = threadIdx.x % 16, sg = threadIdx.x / 16;
    float* in = actA;
    float* out = actB;
#pragma unroll 1
    for (int l = 0; l < 2; ++l) {
        __syncthreads();  // the previous layer's outputs and reads of Wt are complete
        const float4* src = reinterpret_cast<const float4*>(wt + ((size_t)e * 2 + l) * H * H);
        for (int q = threadIdx.x; q < H * H / 4; q += NTB) reinterpret_cast<float4*>(Wt)[q] = __ldg(src + q);
        __syncthreads();
        const float* bias = p + (l ? ob3 : ob2);
        // acc[r][c2] holds outputs (8 ng + 2 c2, 8 ng + 2 c2 + 1) of sample
        // 8 sg + r: one packed FP32x2 FMA updates both (each lane rounds as
        // fmaf does)
        float2 acc[8][4];
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) {
            const float2 bc = make_float2(__ldg(bias + 8 * ng + 2 * c2), __ldg(bias + 8 * ng + 2 * c2 + 1));
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r][c2] = bc;
        }
#pragma unroll 2
        for (int k = 0; k < H; ++k) {
            const float4 w0 = reinterpret_cast<const float4*>(Wt + k * H + 8 * ng)[0];
            const float4 w1 = reinterpret_cast<const float4*>(Wt + k * H + 8 * ng)[1];
            const float4 a0 = reinterpret_cast<const float4*>(in + k * TB + 8 * sg)[0];
            const float4 a1 = reinterpret_cast<const float4*>(in + k * TB + 8 * sg)[1];
            const float2 w[4] = {make_float2(w0.x, w0.y), make_float2(w0.z, w0.w), make_float2(w1.x, w1.y),
                                 make_float2(w1.z, w1.w)};
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float2 ar = make_float2(a[r], a[r]);
#pragma unroll
                for (int c2 = 0; c2 < 4; ++c2) acc[r][c2] = __ffma2_rn(ar, w[c2], acc[r][c2]);
            }
        }
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) {
            float4* o0 = reinterpret_cast<float4*>(out + (8 * ng + 2 * c2) * TB + 8 * sg);
            float4* o1 = reinterpret_cast<float4*>(out + (8 * ng + 2 * c2 + 1) * TB + 8 * sg);
            o0[0] = make_float4(gelu(acc[0][c2].x), gelu(acc[1][c2].x), gelu(acc[2][c2].x), gelu(acc[3][c2].x));
            o0[1] = make_float4(gelu(acc[4][c2].x), gelu(acc[5][c2].x), gelu(acc[6][c2].x), gelu(acc[7][c2].x));
            o1[0] = make_float4(gelu(acc[0][c2].y), gelu(acc[1][c2].y), gelu(acc[2][c2].y), gelu(acc[3][c2].y));
            o1[1] = make_float4(gelu(acc[4][c2].y), gelu(acc[5][c2].y), gelu(acc[6][c2].y), gelu(acc[7][c2].y));
        }
        float* t = in;
        in = out;
        out = t;
    }
    __syncthreads();
    // layer 4: one thread per (sample, output)
    {
        const int sl = threadIdx.x % TB, o = threadIdx.x / TB, b = s0 + sl;
        const float* w4 = p + oW4 + o * H;
        float y = __ldg(p + ob4 + o);
#pragma unroll 8
        for (int k = 0; k < H; ++k) y = fmaf(in[k * TB + sl], __ldg(w4 + k), y);
        if (b < B) Y[((size_t)e * B + b) * O + o] = y;
    }
}

// ---- inference on the tensor cores (tcgen05) ------------------------------
// The two hidden layers are D = A . W^T on 128-sample tiles (M = 128 samples,
// N = 128 neurons, K = 128), with A the previous layer's activations and W
// the layer's weight matrix [neuron][input].  FP32 accuracy from three
// products accumulated into one FP32 D in tensor memory:
//   A . W^T  ~  Ah . Wh^T + Al . Wh^T + Ab . Wl^T
// with Ah = tf32(A), Al = A - Ah, Wh = tf32(W) (the first two on kind::tf32,
// where Al is truncated to TF32 by the unit), Wl = bf16(W - Wh) and
// Ab = bf16(A) (kind::f16 with bf16 operands).  The dropped Al . Wl term and
// the roundings of the third product are below 2^-20 of |A||W|.
// Activations go to tensor memory (tcgen05.st, the MMA's A operand); the
// weights of both layers of the CTA's member sit in shared memory in the
// no-swizzle K-major layout (8-row x 16-byte core matrices, the next core
// matrix along K 128 bytes on, the next 8 rows (K * bytes / 16) * 128 bytes
// on), copied in by one bulk copy of the member's prepared image.  Layers 1
// (K = 4) and 4 (N = 2), the biases and GELU run on the FP32 pipes in the
// epilogues; thread (w, l) owns sample 32 (w % 4) + l (its TMEM lane) and
// the 32 neurons of column quarter w / 4.
constexpr int TCT = 512;
constexpr int TC_WH = H * H * 4, TC_WL = H * H * 2, TC_LAYER = TC_WH + TC_WL, TC_IMG = 2 * TC_LAYER;
constexpr size_t TC_SMEM = (size_t)TC_IMG + 128;
constexpr unsigned MLP_TC_TIMEOUT = 1u;

__host__ __device__ inline int tc_canon(int r, int k, int esize) {
    const int E = 16 / esize;
    return (r / 8) * ((H / E) * 128) + (k / E) * 128 + (r % 8) * 16 + (k % E) * esize;
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// img[e][l] = { Wh (TF32 values in FP32 containers), Wl (bf16) } of hidden
// layer l + 2, both in the shared-memory layout above.
__global__ void mlp_tc_prep_kernel(const float* __restrict__ params, unsigned char* __restrict__ img) {
    const int e = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;  // over 2 * H * H
    if (q >= 2 * H * H) return;
    const int l = q / (H * H), r = q % (H * H), j = r / H, k = r % H;
    const float w = params[(size_t)e * PS + (l ? oW3 : oW2) + j * H + k];
    const float wh = tf32_rna(w);
    unsigned char* base = img + (size_t)e * TC_IMG + (size_t)l * TC_LAYER;
    *reinterpret_cast<float*>(base + tc_canon(j, k, 4)) = wh;
    *reinterpret_cast<__nv_bfloat16*>(base + TC_WH + tc_canon(j, k, 2)) = __float2bfloat16_rn(w - wh);
}

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t sbo) {
    // start >> 4, leading byte offset 128 >> 4, stride byte offset >> 4,
    // descriptor version 1 (bit 46), no swizzle
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor of kind::tf32 (fmt 2) / kind::f16 with bf16 (fmt 1):
// FP32 D, K-major A and B, N = 128, M = 128
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(H >> 3) << 17) | ((uint32_t)(TB >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(bool tf32, uint32_t d, uint32_t a, uint64_t b, uint32_t id, int acc) {
    if (tf32)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
                     :: "r"(d), "r"(a), "l"(b), "r"(id), "r"(acc) : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
                     :: "r"(d), "r"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ void tc_st16(uint32_t t, const uint32_t (&v)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
                 :: "r"(t), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
                    "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]) : "memory");
}
__device__ __forceinline__ void tc_st8(uint32_t t, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "r"(t), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]) : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t t, uint32_t (&v)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(t) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Bounded wait on phase `parity` of an mbarrier; false (and the status bit)
// if it did not complete within `limit` SM clock cycles.
constexpr long long TC_WAIT_LIMIT = 2000000000LL;  // about a second at 2 GHz
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, unsigned* status, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        // test_wait does not suspend: the limit counts from the first probe
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(tc_smem(bar)), "r"(parity) : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) {
            atomicOr(status, MLP_TC_TIMEOUT);
            return false;
        }
        __nanosleep(20);
    }
}

__device__ __forceinline__ void tc_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// The activations a[16] of neurons j0..j0+15 (j0 even) of this thread's
// sample as the next MMA's A operand: Ah, Al (one column each) and Ab (two
// per column, the even neuron in the low half).
__device__ __forceinline__ void tc_put_act(uint32_t tAh, uint32_t tAl, uint32_t tAb, int j0, const float (&a)[16]) {
    uint32_t h[16], lo[16], b2[8];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float ah = tf32_rna(a[i]);
        h[i] = __float_as_uint(ah);
        lo[i] = __float_as_uint(a[i] - ah);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_bfloat162 pr = __floats2bfloat162_rn(a[2 * i], a[2 * i + 1]);  // .x = low half
        b2[i] = *reinterpret_cast<const uint32_t*>(&pr);
    }
    tc_st16(tAh + j0, h);
    tc_st16(tAl + j0, lo);
    tc_st8(tAb + j0 / 2, b2);
}

// Persistent per member: CTA (x, e) loads member e's weights once and runs
// tiles x, x + gridDim.x, ... of that member.
__global__ void __launch_bounds__(TCT, 1) mlp_infer_tc_kernel(const float* __restrict__ params,
                                                              const unsigned char* __restrict__ img,
                                                              const float* __restrict__ X, int B,
                                                              float* __restrict__ Y, unsigned* status,
                                                              long long limit) {
    extern __shared__ __align__(128) unsigned char tc_raw[];
    unsigned char* sw = tc_raw + ((128u - (tc_smem(tc_raw) & 127u)) & 127u);
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[2];  // [0] weights landed, [1] MMAs of a layer done
    __shared__ float s_w1[H * I], s_b[3][H], s_w4[O * H], s_b4[O];
    __shared__ float s_part[4][O][TB];
    __shared__ int s_ok, s_mma_pending;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = warp & 3, qc = warp >> 2;
    const int row = 32 * g + lane, j0 = 32 * qc;
    const int e = blockIdx.y, ntiles = (B + TB - 1) / TB;
    const float* p = params + (size_t)e * PS;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_smem(&s_bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_smem(&s_bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
        s_mma_pending = -1;
    }
    __syncthreads();
    bool weights = false;  // thread 0: the weight image has landed
    if (tid == 0) {
        // the member's weight image: four bulk copies onto one transaction count
        const unsigned char* src = img + (size_t)e * TC_IMG;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(tc_smem(&s_bar[0])), "r"(TC_IMG) : "memory");
#pragma unroll
        for (int c = 0; c < 4; ++c)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(tc_smem(sw + c * (TC_IMG / 4))), "l"(src + c * (TC_IMG / 4)), "r"(TC_IMG / 4),
                            "r"(tc_smem(&s_bar[0])) : "memory");
        // the other threads stage the small parameters and run layer 1 meanwhile
        weights = tc_wait(&s_bar[0], 0, status, limit);
        if (!weights) s_ok = 0;
    }
    for (int i = tid; i < H * I; i += TCT) s_w1[i] = p[oW1 + i];
    for (int i = tid; i < H; i += TCT) {
        s_b[0][i] = p[ob1 + i];
        s_b[1][i] = p[ob2 + i];
        s_b[2][i] = p[ob3 + i];
    }
    for (int i = tid; i < O * H; i += TCT) s_w4[i] = p[oW4 + i];
    if (tid < O) s_b4[tid] = p[ob4 + tid];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(tc_smem(&s_tmem)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_sync();
    const uint32_t lane_off = (uint32_t)(32 * g) << 16;
    const uint32_t tD = s_tmem + lane_off, tAh = tD + 128, tAl = tD + 256, tAb = tD + 384;
#pragma unroll 1
    for (int t = blockIdx.x; t < ntiles && s_ok; t += gridDim.x) {
        const int b = t * TB + row;
        // ---- layer 1 (K = 4) on the FP32 pipes, GELU, A of layer 2 ----
        {
            float x[I] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (b < B)
#pragma unroll
                for (int k = 0; k < I; ++k) x[k] = __ldg(X + (size_t)b * I + k);
#pragma unroll
            for (int c = 0; c < 32; c += 16) {
                float a[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int j = j0 + c + i;
                    float z = s_b[0][j];
#pragma unroll
                    for (int k = 0; k < I; ++k) z = fmaf(s_w1[j * I + k], x[k], z);
                    a[i] = gelu(z);
                }
                tc_put_act(tAh, tAl, tAb, j0 + c, a);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
#pragma unroll 1
        for (int l = 0; l < 2; ++l) {
            tc_sync();
            if (tid == 0) {
                // 40 MMAs of the layer from one thread; a K step moves the
                // descriptor's start address by 256 bytes (+16 in its field)
                const uint32_t wh = tc_smem(sw + l * TC_LAYER), wl = wh + TC_WH;
                const uint32_t it = tc_idesc(2), ib = tc_idesc(1);
                const uint32_t d = s_tmem, ah = s_tmem + 128, al = s_tmem + 256, ab = s_tmem + 384;
                const uint64_t dh = tc_desc(wh, (H / 4) * 128), dl = tc_desc(wl, (H / 8) * 128);
#pragma unroll
                for (int s = 0; s < H / 8; ++s) tc_mma(true, d, ah + 8 * s, dh + 16 * s, it, s > 0);
#pragma unroll
                for (int s = 0; s < H / 8; ++s) tc_mma(true, d, al + 8 * s, dh + 16 * s, it, 1);
#pragma unroll
                for (int s = 0; s < H / 16; ++s) tc_mma(false, d, ab + 8 * s, dl + 16 * s, ib, 1);
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(tc_smem(&s_bar[1])) : "memory");
                s_mma_pending = l;
            }
            __syncthreads();
            // two commits per tile: phase parity = layer
            // one decision for the whole CTA: every thread saw the phase complete
            const int ok_before = s_ok;
            if (!__syncthreads_and(ok_before && tc_wait(&s_bar[1], (uint32_t)l, status, limit))) {
                if (tid == 0) s_ok = 0;
                break;
            }
            if (tid == 0) s_mma_pending = -1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (l == 0) {
                // ---- epilogue of layer 2: bias, GELU, A of layer 3 ----
#pragma unroll
                for (int c = 0; c < 32; c += 16) {
                    uint32_t v[16];
                    tc_ld16(tD + j0 + c, v);
                    float a[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) a[i] = gelu(__uint_as_float(v[i]) + s_b[1][j0 + c + i]);
                    tc_put_act(tAh, tAl, tAb, j0 + c, a);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            } else {
                // ---- epilogue of layer 3 and layer 4 (N = 2): partial sums over this quarter ----
                float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
                for (int c = 0; c < 32; c += 16) {
                    uint32_t v[16];
                    tc_ld16(tD + j0 + c, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int j = j0 + c + i;
                        const float a = gelu(__uint_as_float(v[i]) + s_b[2][j]);
                        y0 = fmaf(a, s_w4[j], y0);
                        y1 = fmaf(a, s_w4[H + j], y1);
                    }
                }
                s_part[qc][0][row] = y0;
                s_part[qc][1][row] = y1;
            }
        }
        tc_sync();
        if (s_ok && tid < O * TB) {
            const int r = tid % TB, o = tid / TB, bb = t * TB + r;
            const float y = s_b4[o] + ((s_part[0][o][r] + s_part[1][o][r]) + (s_part[2][o][r] + s_part[3][o][r]));
            if (bb < B) Y[((size_t)e * B + bb) * O + o] = y;
        }
    }
    // a weight copy or MMAs still in flight (their wait ran out) complete
    // before the CTA frees its tensor memory and leaves
    tc_sync();
    if (tid == 0) {
        if (!weights) tc_wait(&s_bar[0], 0, status, TC_WAIT_LIMIT);
        if (s_mma_pending >= 0) tc_wait(&s_bar[1], (uint32_t)s_mma_pending, status, TC_WAIT_LIMIT);
    }
    tc_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(s_tmem), "r"(512) : "memory");
}

// Ensemble mean and relative spread (max over outputs of the population std
// over members / |mean|), two passes over the members.
__global__ void mlp_reduce_kernel(const float* __restrict__ Y, int E, int B, float* __restrict__ mean,
                                  float* __restrict__ spread) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float sp = 0.0f;
#pragma unroll
    for (int o = 0; o < O; ++o) {
        float s = 0.0f;
        for (int e = 0; e < E; ++e) s += Y[((size_t)e * B + b) * O + o];
        const float mu = s / (float)E;
        float s2 = 0.0f;
        for (int e = 0; e < E; ++e) {
            const float d = Y[((size_t)e * B + b) * O + o] - mu;
            s2 = fmaf(d, d, s2);
        }
        mean[(size_t)b * O + o] = mu;
        sp = fmaxf(sp, sqrtf(s2 / (float)E) / fmaxf(fabsf(mu), 1e-30f));
    }
    spread[b] = sp;
}

// splitmix64: deterministic host generator for initial weights and shuffles.
uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

struct lbm_mlp {
    int E = 0;
    cudaStream_t stream = nullptr;
    float* params = nullptr;  // [E][P]
    float* m = nullptr;
    float* v = nullptr;
    int64_t t = 0;            // Adam steps taken
    uint64_t seed = 0;
    float* wt = nullptr;      // [E][2][H][H] k-major copy of the hidden weights (inference)
    unsigned char* tcimg = nullptr;  // [E][TC_IMG] tensor-core images of the hidden weights
    unsigned* status = nullptr;      // device status word of the tensor-core inference
    int infer_path = LBM_MLP_INFER_TENSOR;
    int sms = 1;  // SMs of the device (persistent tensor-core grid)
    long long wait_limit = TC_WAIT_LIMIT;  // SM cycles a tensor-core wait may take
    void* ws = nullptr;       // grow-only device workspace of the per-call buffers
    size_t ws_bytes = 0;
    std::string err;
};

namespace {

lbm_status mfail(lbm_mlp* m, lbm_status st, const std::string& msg) {
    if (m) m->err = msg;
    else lbm::set_thread_error(msg.c_str());
    return st;
}

#define MCK(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) return mfail(mm, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

std::once_flag g_attr_once;
cudaError_t g_attr_err = cudaSuccess;

cudaError_t set_smem_attrs() {
    std::call_once(g_attr_once, [] {
        g_attr_err = cudaFuncSetAttribute(mlp_forward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)SMEM_BYTES);
        if (g_attr_err == cudaSuccess)
            g_attr_err = cudaFuncSetAttribute(mlp_forward_kernel<false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (g_attr_err == cudaSuccess)
            g_attr_err = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)SMEM_BIG);
        if (g_attr_err == cudaSuccess)
            g_attr_err = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)SMEM_BYTES);
        if (g_attr_err == cudaSuccess)
            g_attr_err = cudaFuncSetAttribute(mlp_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)TC_SMEM);
    });
    return g_attr_err;
}

// Per-call device buffers, carved out of the ensemble's workspace (grown, never
// shrunk; reallocated only after the stream has drained).
struct Scratch {
    float *X = nullptr, *T = nullptr, *Y = nullptr, *Z = nullptr, *gp = nullptr, *grad = nullptr;
    int* idx = nullptr;
};

// Element counts of X, T, Y, Z, gp, grad (floats) and idx (ints).
lbm_status carve(lbm_mlp* mm, Scratch& s, size_t nX, size_t nT, size_t nY, size_t nZ, size_t ngp, size_t ngrad,
                 size_t nidx) {
    const size_t cnt[7] = {nX, nT, nY, nZ, ngp, ngrad, nidx};
    size_t off[7], total = 0;
    for (int k = 0; k < 7; ++k) {
        off[k] = total;
        total += (cnt[k] * 4 + 255) / 256 * 256;
    }
    if (total > mm->ws_bytes) {
        MCK(cudaStreamSynchronize(mm->stream));
        if (mm->ws) cudaFree(mm->ws);
        mm->ws = nullptr;
        mm->ws_bytes = 0;
        const size_t want = total + total / 4;
        cudaError_t e = cudaMalloc(&mm->ws, want);
        if (e != cudaSuccess) {
            mm->ws = nullptr;
            return mfail(mm, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                         std::string("mlp workspace: ") + cudaGetErrorString(e));
        }
        mm->ws_bytes = want;
    }
    char* b = static_cast<char*>(mm->ws);
    float** fp[6] = {&s.X, &s.T, &s.Y, &s.Z, &s.gp, &s.grad};
    for (int k = 0; k < 6; ++k) *fp[k] = cnt[k] ? reinterpret_cast<float*>(b + off[k]) : nullptr;
    s.idx = cnt[6] ? reinterpret_cast<int*>(b + off[6]) : nullptr;
    return LBM_OK;
}

#define CARVE(...)                                   \
    do {                                             \
        lbm_status cs_ = carve(mm, s, __VA_ARGS__);  \
        if (cs_ != LBM_OK) return cs_;               \
    } while (0)

// One training (or gradient-only) step on rows idx[0..B) of the device data.
lbm_status run_step(lbm_mlp* mm, Scratch& s, int B, const int* idx, bool adam, double lr, float* grad_out) {
    const int ntile = (B + TILE - 1) / TILE;
    const dim3 grid(ntile, mm->E);
    mlp_forward_kernel<true><<<grid, NTH, SMEM_BYTES, mm->stream>>>(mm->params, s.X, idx, B, s.Y, s.Z);
    MCK(cudaGetLastError());
    mlp_backward_kernel<<<grid, NTH, SMEM_BYTES, mm->stream>>>(mm->params, s.X, s.T, idx, B, s.Y, s.Z, s.gp);
    MCK(cudaGetLastError());
    float c1 = 1.0f, c2 = 1.0f;
    if (adam) {
        mm->t += 1;
        c1 = (float)(1.0 - std::pow(0.9, (double)mm->t));
        c2 = (float)(1.0 - std::pow(0.999, (double)mm->t));
    }
    mlp_adam_kernel<<<dim3((P + 255) / 256, mm->E), 256, 0, mm->stream>>>(
        mm->params, mm->m, mm->v, s.gp, ntile, (float)lr, 0.9f, 0.999f, c1, c2, 1e-8f, adam ? 1 : 0, grad_out);
    MCK(cudaGetLastError());
    return LBM_OK;
}

// Refresh the k-major copy of the hidden weights after any parameter change.
lbm_status refresh_wt(lbm_mlp* mm) {
    mlp_transpose_kernel<<<dim3((2 * H * H + 255) / 256, mm->E), 256, 0, mm->stream>>>(mm->params, mm->wt);
    MCK(cudaGetLastError());
    mlp_tc_prep_kernel<<<dim3((2 * H * H + 255) / 256, mm->E), 256, 0, mm->stream>>>(mm->params, mm->tcimg);
    MCK(cudaGetLastError());
    return LBM_OK;
}

lbm_status launch_infer(lbm_mlp* mm, const float* dX, int n, float* dY) {
    if (mm->infer_path == LBM_MLP_INFER_TENSOR) {
        // persistent per member: about one CTA per SM over all members
        const int ntiles = (n + TB - 1) / TB;
        const int per = std::max(1, std::min(ntiles, mm->sms / mm->E));
        mlp_infer_tc_kernel<<<dim3(per, mm->E), TCT, TC_SMEM, mm->stream>>>(mm->params, mm->tcimg, dX, n, dY,
                                                                             mm->status, mm->wait_limit);
    } else {
        mlp_infer_kernel<<<dim3((n + TB - 1) / TB, mm->E), NTB, SMEM_BIG, mm->stream>>>(mm->params, mm->wt, dX, n,
                                                                                          dY);
    }
    MCK(cudaGetLastError());
    return LBM_OK;
}

// After the stream has drained: a tensor-core wait that ran out is an error
// (the outputs of that call are undefined); the word is cleared for the next.
lbm_status check_infer(lbm_mlp* mm) {
    unsigned st = 0;
    MCK(cudaMemcpy(&st, mm->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st) {
        MCK(cudaMemset(mm->status, 0, sizeof(unsigned)));
        return mfail(mm, LBM_ERR_TIMEOUT, "a tensor-core wait of the inference kernel ran out; outputs undefined");
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

int64_t lbm_mlp_num_params(void) { return P; }

lbm_status lbm_mlp_create(int members, uint64_t seed, void* cuda_stream, lbm_mlp** out) {
    if (!out) return mfail(nullptr, LBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (members < 1 || members > 64) return mfail(nullptr, LBM_ERR_INVALID_ARG, "members must be in [1, 64]");
    lbm_mlp* mm = new (std::nothrow) lbm_mlp();
    if (!mm) return mfail(nullptr, LBM_ERR_OOM, "host allocation failed");
    mm->E = members;
    mm->stream = static_cast<cudaStream_t>(cuda_stream);
    mm->seed = seed;
    cudaError_t e = set_smem_attrs();
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mm->sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t bytes = (size_t)members * PS * sizeof(float);
    if (e == cudaSuccess) e = cudaMalloc((void**)&mm->params, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&mm->m, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&mm->v, bytes);
    if (e == cudaSuccess) e = cudaMemset(mm->m, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(mm->v, 0, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&mm->wt, (size_t)members * 2 * H * H * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&mm->tcimg, (size_t)members * TC_IMG);
    if (e == cudaSuccess) e = cudaMalloc((void**)&mm->status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(mm->status, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        const std::string msg = std::string("mlp allocation: ") + cudaGetErrorString(e);
        lbm_mlp_destroy(mm);
        return mfail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, msg);
    }
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases; member e
    // draws from seed + e
    std::vector<float> h((size_t)members * P, 0.0f);
    for (int m = 0; m < members; ++m) {
        uint64_t st = seed + (uint64_t)m * 0x632BE59BD9B4E019ull;
        float* p = h.data() + (size_t)m * P;
        auto fill = [&](int off, int n, int fan_in) {
            const double bound = 1.0 / std::sqrt((double)fan_in);
            for (int i = 0; i < n; ++i) p[off + i] = (float)((2.0 * uniform01(st) - 1.0) * bound);
        };
        fill(oW1, H * I, I);
        fill(oW2, H * H, H);
        fill(oW3, H * H, H);
        fill(oW4, O * H, H);
    }
    e = cudaMemcpy2D(mm->params, PS * sizeof(float), h.data(), P * sizeof(float), P * sizeof(float), members,
                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        const std::string msg = std::string("mlp upload: ") + cudaGetErrorString(e);
        lbm_mlp_destroy(mm);
        return mfail(nullptr, LBM_ERR_CUDA, msg);
    }
    if (refresh_wt(mm) != LBM_OK) {
        const std::string msg = mm->err;
        lbm_mlp_destroy(mm);
        return mfail(nullptr, LBM_ERR_CUDA, msg);
    }
    *out = mm;
    return LBM_OK;
}

lbm_status lbm_mlp_set_params(lbm_mlp* mm, const float* params) {
    if (!mm || !params) return mfail(mm, LBM_ERR_INVALID_ARG, "NULL argument");
    MCK(cudaStreamSynchronize(mm->stream));
    MCK(cudaMemcpy2D(mm->params, PS * sizeof(float), params, P * sizeof(float), P * sizeof(float), mm->E,
                     cudaMemcpyHostToDevice));
    MCK(cudaMemset(mm->m, 0, (size_t)mm->E * PS * sizeof(float)));
    MCK(cudaMemset(mm->v, 0, (size_t)mm->E * PS * sizeof(float)));
    mm->t = 0;
    return refresh_wt(mm);
}

lbm_status lbm_mlp_get_params(lbm_mlp* mm, float* params) {
    if (!mm || !params) return mfail(mm, LBM_ERR_INVALID_ARG, "NULL argument");
    MCK(cudaStreamSynchronize(mm->stream));
    MCK(cudaMemcpy2D(params, P * sizeof(float), mm->params, PS * sizeof(float), P * sizeof(float), mm->E,
                     cudaMemcpyDeviceToHost));
    return LBM_OK;
}

lbm_status lbm_mlp_forward(lbm_mlp* mm, const float* X, int n, float* Y) {
    if (!mm || !X || !Y || n < 1) return mfail(mm, LBM_ERR_INVALID_ARG, "bad forward request");
    Scratch s;
    CARVE((size_t)n * I, 0, (size_t)mm->E * n * O, 0, 0, 0, 0);
    MCK(cudaMemcpyAsync(s.X, X, (size_t)n * I * sizeof(float), cudaMemcpyHostToDevice, mm->stream));
    lbm_status st = launch_infer(mm, s.X, n, s.Y);
    if (st != LBM_OK) return st;
    MCK(cudaMemcpyAsync(Y, s.Y, (size_t)mm->E * n * O * sizeof(float), cudaMemcpyDeviceToHost, mm->stream));
    MCK(cudaStreamSynchronize(mm->stream));
    return check_infer(mm);
}

lbm_status lbm_mlp_gradient(lbm_mlp* mm, const float* X, const float* T, int n, float* grad) {
    if (!mm || !X || !T || !grad || n < 1) return mfail(mm, LBM_ERR_INVALID_ARG, "bad gradient request");
    Scratch s;
    const int ntile = (n + TILE - 1) / TILE;
    CARVE((size_t)n * I, (size_t)n * O, (size_t)mm->E * n * O, (size_t)mm->E * 3 * n * H,
          (size_t)mm->E * ntile * P, (size_t)mm->E * P, 0);
    MCK(cudaMemcpyAsync(s.X, X, (size_t)n * I * sizeof(float), cudaMemcpyHostToDevice, mm->stream));
    MCK(cudaMemcpyAsync(s.T, T, (size_t)n * O * sizeof(float), cudaMemcpyHostToDevice, mm->stream));
    lbm_status st = run_step(mm, s, n, nullptr, false, 0.0, s.grad);
    if (st != LBM_OK) return st;
    MCK(cudaMemcpyAsync(grad, s.grad, (size_t)mm->E * P * sizeof(float), cudaMemcpyDeviceToHost, mm->stream));
    MCK(cudaStreamSynchronize(mm->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_train(lbm_mlp* mm, const float* X, const float* T, int n, int epochs, int batch, double lr,
                         uint64_t shuffle_seed) {
    if (!mm || !X || !T || n < 1 || epochs < 0 || batch < 1 || !(lr > 0.0))
        return mfail(mm, LBM_ERR_INVALID_ARG, "bad training request");
    batch = std::min(batch, n);
    Scratch s;
    const int ntile = (batch + TILE - 1) / TILE;
    CARVE((size_t)n * I, (size_t)n * O, (size_t)mm->E * batch * O, (size_t)mm->E * 3 * batch * H,
          (size_t)mm->E * ntile * P, 0, (size_t)n);
    MCK(cudaMemcpyAsync(s.X, X, (size_t)n * I * sizeof(float), cudaMemcpyHostToDevice, mm->stream));
    MCK(cudaMemcpyAsync(s.T, T, (size_t)n * O * sizeof(float), cudaMemcpyHostToDevice, mm->stream));
    std::vector<int> perm(n);
    uint64_t rs = shuffle_seed;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = n - 1; i > 0; --i) {  // Fisher-Yates with splitmix64
            const int j = (int)(splitmix64(rs) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        MCK(cudaStreamSynchronize(mm->stream));  // the previous epoch's kernels read s.idx
        MCK(cudaMemcpy(s.idx, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice));
        for (int b0 = 0; b0 + batch <= n; b0 += batch) {
            lbm_status st = run_step(mm, s, batch, s.idx + b0, true, lr, nullptr);
            if (st != LBM_OK) return st;
        }
    }
    lbm_status st = refresh_wt(mm);
    if (st != LBM_OK) return st;
    MCK(cudaStreamSynchronize(mm->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_predict(lbm_mlp* mm, const float* X, int n, float* mean, float* spread, int dst_is_device) {
    if (!mm || !X || !mean || !spread || n < 1) return mfail(mm, LBM_ERR_INVALID_ARG, "bad predict request");
    Scratch s;
    const size_t hn = dst_is_device ? 0 : (size_t)n;
    CARVE(hn * I, hn * O, (size_t)mm->E * n * O, 0, 0, hn, 0);
    const float* dX = X;
    float *dm = mean, *ds = spread;
    if (!dst_is_device) {
        MCK(cudaMemcpyAsync(s.X, X, (size_t)n * I * sizeof(float), cudaMemcpyHostToDevice, mm->stream));
        dX = s.X;
        dm = s.T;
        ds = s.grad;
    }
    lbm_status st = launch_infer(mm, dX, n, s.Y);
    if (st != LBM_OK) return st;
    mlp_reduce_kernel<<<(n + 255) / 256, 256, 0, mm->stream>>>(s.Y, mm->E, n, dm, ds);
    MCK(cudaGetLastError());
    if (!dst_is_device) {
        MCK(cudaMemcpyAsync(mean, dm, (size_t)n * O * sizeof(float), cudaMemcpyDeviceToHost, mm->stream));
        MCK(cudaMemcpyAsync(spread, ds, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, mm->stream));
    }
    MCK(cudaStreamSynchronize(mm->stream));
    return check_infer(mm);
}

lbm_status lbm_mlp_set_wait_limit(lbm_mlp* mm, long long cycles) {
    if (!mm) return mfail(nullptr, LBM_ERR_INVALID_ARG, "mlp is NULL");
    if (cycles < 0) return mfail(mm, LBM_ERR_INVALID_ARG, "cycles must be >= 0");
    MCK(cudaStreamSynchronize(mm->stream));
    mm->wait_limit = cycles ? cycles : TC_WAIT_LIMIT;
    return LBM_OK;
}

lbm_status lbm_mlp_set_infer_path(lbm_mlp* mm, int path) {
    if (!mm) return mfail(nullptr, LBM_ERR_INVALID_ARG, "mlp is NULL");
    if (path != LBM_MLP_INFER_TENSOR && path != LBM_MLP_INFER_SIMT)
        return mfail(mm, LBM_ERR_INVALID_ARG, "unknown inference path");
    MCK(cudaStreamSynchronize(mm->stream));
    mm->infer_path = path;
    return LBM_OK;
}

void lbm_mlp_destroy(lbm_mlp* mm) {
    if (!mm) return;
    if (mm->stream) cudaStreamSynchronize(mm->stream);
    void* p[] = {mm->params, mm->m, mm->v, mm->wt, mm->tcimg, mm->status, mm->ws};
    for (void* q : p)
        if (q) cudaFree(q);
    delete mm;
}

const char* lbm_mlp_last_error(const lbm_mlp* mm) { return mm ? mm->err.c_str() : lbm_last_error(nullptr); }

}  // extern "C"
