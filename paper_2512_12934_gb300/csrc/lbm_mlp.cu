// Surrogate MLP ensemble (4 -> 128 -> 128 -> 128 -> 2, GELU), FP32, with
// fused forward, backward and Adam kernels.
//
// One CTA owns TILE samples of one ensemble member.  Forward: the four layers
// run back to back on activations held in shared memory; each 128x128 weight
// matrix is staged transposed so a thread's 4x4 output block reads its four
// weights as one conflict-free float4.  Backward: the whole chain rule for the
// tile (output error, dZ3, dW3, dA2, dZ2, dW2, dA1, dZ1, dW1 and the biases)
// stays on chip; the tile writes its gradient partial with plain stores.  Adam
// sums the tiles' partials in a fixed order (deterministic) and updates.
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
    return LBM_OK;
}

lbm_status launch_infer(lbm_mlp* mm, const float* dX, int n, float* dY) {
    mlp_infer_kernel<<<dim3((n + TB - 1) / TB, mm->E), NTB, SMEM_BIG, mm->stream>>>(mm->params, mm->wt, dX, n, dY);
    MCK(cudaGetLastError());
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
    const size_t bytes = (size_t)members * PS * sizeof(float);
    if (e == cudaSuccess) e = cudaMalloc((void**)&mm->params, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&mm->m, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&mm->v, bytes);
    if (e == cudaSuccess) e = cudaMemset(mm->m, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(mm->v, 0, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&mm->wt, (size_t)members * 2 * H * H * sizeof(float));
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
    return LBM_OK;
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
    return LBM_OK;
}

void lbm_mlp_destroy(lbm_mlp* mm) {
    if (!mm) return;
    if (mm->stream) cudaStreamSynchronize(mm->stream);
    void* p[] = {mm->params, mm->m, mm->v, mm->wt, mm->ws};
    for (void* q : p)
        if (q) cudaFree(q);
    delete mm;
}

const char* lbm_mlp_last_error(const lbm_mlp* mm) { return mm ? mm->err.c_str() : lbm_last_error(nullptr); }

}  // extern "C"
