// Fused D2Q9 two-component MRT pseudopotential step for sm_103a.
//
// One launch = one time step.  A CTA owns a TX x TY tile of nodes and
// stages the densities (pseudopotentials psi_k = rho_k) of the tile plus a
// two-node halo in shared memory, so the 24-point interaction stencil of
// Eq. 10 reads on-chip data only.  Populations are stored structure-of-
// arrays f[k][i][y][x] (x fastest, pitched rows), read once by the pull
// stream and written once after collision.  Stage order inside the kernel:
//   pull stream (Eq. 2) + halfway bounce-back (Eq. B1) + periodic wrap
//   (Eq. B2) -> inlet NEQ extrapolation (Eqs. 13, 14) + alpha correction
//   (Eqs. 15-19) -> convective outlet (Eqs. 20, 21) -> rho_k, psi_k with
//   ghost mirrors (Eqs. 24, 25) -> F_f (Eq. 10) + F_ads (Eq. 11) -> common
//   velocity (Eqs. 7, 8), outlet rescaled by chi (Eq. 22) -> MRT collision
//   with forcing in moment space (Eqs. 1, 3-6, 9) -> store -> FP64 flux
//   reductions that set lambda and chi for the next step (Eqs. 21, 23).
#include "d2q9_tile.cuh"

namespace lbm {
namespace {

// Fast tiles in FP32 fit in 64 registers; holding them there keeps four
// 256-thread CTAs (eight of 128) resident per SM.
template <typename R, int TX, int TY>
__host__ __device__ constexpr int fast_min_blocks() {
    return sizeof(R) == 4 ? 65536 / (TX * TY * 64) : 1;
}

// Single-instance step: one tile of the launch's list per CTA.
template <typename S, typename R, int TX, int TY, bool GEN>
__global__ void __launch_bounds__(TX * TY, (fast_min_blocks<R, TX, TY>())) d2q9_step_kernel(const __grid_constant__ D2Args<S, R> a) {
    static_assert(!GEN, "general tiles run d2q9_general_kernel");
    grid_dep_wait();
    const int li = a.list_off + blockIdx.x;
    step_tile<S, R, TX, TY, false>(a, a.blocks[li], a.block_flags[li], 0u, -1);
}

template <typename S, typename R, int TX, int TY, bool ROLES>
__global__ void __maxnreg__((gen_maxreg<R, TX, TY, ROLES>())) d2q9_general_kernel(const __grid_constant__ D2Args<S, R> a) {
    grid_dep_wait();
    const int li = a.list_off + blockIdx.x;
    step_tile<S, R, TX, TY, true, ROLES>(a, a.blocks[li], a.block_flags[li], a.block_strips[li], a.block_slot[li]);
}

// Batched step: the list interleaves the tiles of many instances; each CTA
// copies its instance's arguments into shared memory and runs the same tile
// code, so a batch step equals stepping every member on its own.
template <typename S, typename R, int TX, int TY, bool GEN, bool ROLES = true>
__device__ __forceinline__ void batch_tile(const BatchArgs<S, R>& b) {
    __shared__ D2Args<S, R> sa;
    grid_dep_wait();
    const int li = b.off + blockIdx.x;
    const int m = b.member[li];
    {
        static_assert(sizeof(D2Args<S, R>) % 4 == 0, "argument block must be word-sized");
        const int* src = reinterpret_cast<const int*>(b.args + m);
        int* dst = reinterpret_cast<int*>(&sa);
        for (int i = threadIdx.x; i < (int)(sizeof(D2Args<S, R>) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    step_tile<S, R, TX, TY, GEN, ROLES>(sa, b.blocks[li], b.flags[li], b.strips[li], b.slot[li]);
}

template <typename S, typename R, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, (fast_min_blocks<R, TX, TY>())) d2q9_batch_kernel(const __grid_constant__ BatchArgs<S, R> b) {
    batch_tile<S, R, TX, TY, false>(b);
}

template <typename S, typename R, int TX, int TY, bool ROLES>
__global__ void __maxnreg__((gen_maxreg<R, TX, TY, ROLES>())) d2q9_batch_general_kernel(const __grid_constant__ BatchArgs<S, R> b) {
    batch_tile<S, R, TX, TY, true, ROLES>(b);
}

// Same-step chi (Eq. 23 at t + dt).  Runs after the general tiles of the
// step, which left the outlet nodes' post-stream state in a.oc_save and this
// step's FP64 flux partials in a.part_out.  Warp 0 folds the partials in the
// fixed order of the lagged fold; then every outlet node gets its normal
// velocity chi * u_n(x_{N-1}) (Eq. 22), is collided (Eq. 1) and stored.
template <typename S, typename R>
__global__ void __launch_bounds__(256) d2q9_outlet_chi_kernel(const __grid_constant__ D2Args<S, R> a) {
    __shared__ R s_chi;
    grid_dep_wait();
    if (threadIdx.x < 32) {
        LamFold L;
        fold_begin(a, L, a.part_out, a.scal_out);
        double lam, chi;
        fold_finish(a, L, lam, chi, a.part_out, a.scal_out);
        if (threadIdx.x == 0) s_chi = R(chi);
    }
    __syncthreads();
    const R chi = s_chi;
    const FaceDev& F = a.face[a.out_face];
    const int len = F.hi - F.lo + 1;
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        const R* q = a.oc_save + (size_t)(F.base + t) * OC_STRIDE;
        if (q[26] == R(0)) continue;  // a solid node of the face: never written
        const int x = F.side == 0 ? 0 : (F.side == 1 ? a.nx - 1 : F.lo + t);
        const int y = F.side == 2 ? 0 : (F.side == 3 ? a.ny - 1 : F.lo + t);
        const int n = y * a.pitch + x;
        R f[2][9];
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int i = 0; i < 9; ++i) f[k][i] = q[k * 9 + i];
        const R rho0 = q[18], rho1 = q[19];
        const R un = chi * q[25], ut = q[24];
        const R ux = F.side <= 1 ? un : ut, uy = F.side <= 1 ? ut : un;
        if (a.macro) {
            a.macro[n] = rho0;
            a.macro[a.plane + n] = rho1;
            a.macro[2 * a.plane + n] = ux;
            a.macro[3 * a.plane + n] = uy;
        }
        const R uu3 = R(3) * (ux * ux + uy * uy);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            R o[9];
            collide_scalar<R>(a.s[k], k == 0 ? rho0 : rho1, q[20 + 2 * k], q[21 + 2 * k], ux, uy, uu3, f[k], o);
#pragma unroll
            for (int i = 0; i < 9; ++i) Pop<S, R>::st(a.fout, (k * 9 + i) * a.plane + n, o[i], R(0));
        }
        if (!isfinite(rho0 + rho1 + ux + uy)) atomicOr(a.status, 1u);
    }
}

// FP64 mass / speed reduction for diagnostics.
template <typename S, typename R>
__global__ void __launch_bounds__(256) d2q9_diag_kernel(const S* __restrict__ f, const R* __restrict__ macro,
                                                        const uint16_t* __restrict__ info,
                                                        const void* __restrict__ rref, int nx, int ny, int px,
                                                        int py, int pitch, long long plane, double* partials) {
    double m0 = 0.0, m1 = 0.0, umax = 0.0;
    const long long total = (long long)nx * ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % nx), y = (int)(t / nx);
        const long long n = (long long)y * pitch + x;
        const unsigned inf = info[n];
        if (inf & INFO_SOLID) continue;
        double a0 = 0.0, a1 = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            R r0 = R(0), r1 = R(0);
            if constexpr (is_half_<S>()) {
                // reference of the node that pulls direction i next (the node itself on bounce-back)
                long long d = n;
                if (!((inf >> opp_(i)) & 1u)) {
                    int dx = x + ex_(i), dy = y + ey_(i);
                    if (dx < 0) dx += nx; else if (dx >= nx) dx -= nx;
                    if (dy < 0) dy += ny; else if (dy >= ny) dy -= ny;
                    d = (long long)dy * pitch + dx;
                }
                const __half* rr = static_cast<const __half*>(rref);
                r0 = __half2float(rr[d]);
                r1 = __half2float(rr[plane + d]);
            }
            a0 += (double)Pop<S, R>::ld(f, (int)(i * plane + n), w_<R>(i) * r0);
            a1 += (double)Pop<S, R>::ld(f, (int)((9 + i) * plane + n), w_<R>(i) * r1);
        }
        m0 += a0;
        m1 += a1;
        const double ux = (double)macro[2 * plane + n], uy = (double)macro[3 * plane + n];
        umax = fmax(umax, ux * ux + uy * uy);
    }
    (void)px;
    (void)py;
    __shared__ double red[3][8];
    for (int o = 16; o > 0; o >>= 1) {
        m0 += __shfl_down_sync(0xffffffffu, m0, o);
        m1 += __shfl_down_sync(0xffffffffu, m1, o);
        umax = fmax(umax, __shfl_down_sync(0xffffffffu, umax, o));
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][wid] = m0;
        red[1][wid] = m1;
        red[2][wid] = umax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < 8; ++w) {
            a0 += red[0][w];
            a1 += red[1][w];
            a2 = fmax(a2, red[2][w]);
        }
        partials[blockIdx.x * 3 + 0] = a0;
        partials[blockIdx.x * 3 + 1] = a1;
        partials[blockIdx.x * 3 + 2] = a2;
    }
}

}  // namespace

struct TileShape { int tx, ty; };
static const TileShape kVariants[] = {{32, 8}, {32, 4}, {64, 4}, {32, 16}, {32, 8}};

void d2q9_variant_tile(int variant, int* tx, int* ty) {
    *tx = kVariants[variant].tx;
    *ty = kVariants[variant].ty;
}
int d2q9_num_variants() { return (int)(sizeof(kVariants) / sizeof(kVariants[0])); }

// A general list of at most two CTAs per SM is latency-bound: its tiles stage
// with the extra GenRoles warps.  Longer lists (batched ensembles) fill the
// GPU by themselves and stage serially on the node threads.
static bool general_roles(int nblocks) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || sms <= 0)
            sms = 152;
    }
    return nblocks <= 2 * sms;
}

// (Serial staging is built for FP32 storage only, to bound compile time;
// the other precisions always stage with GenRoles.)
template <typename S, typename R, int TX, int TY>
static void launch_tile(const D2Args<S, R>& a, bool general, int nblocks, cudaStream_t st) {
    if (!general) {
        d2q9_step_kernel<S, R, TX, TY, false><<<nblocks, TX * TY, 0, st>>>(a);
        return;
    }
    if constexpr (std::is_same<S, float>::value) {
        if (!general_roles(nblocks)) {
            d2q9_general_kernel<S, R, TX, TY, false><<<nblocks, TX * TY, 0, st>>>(a);
            return;
        }
    }
    d2q9_general_kernel<S, R, TX, TY, true><<<nblocks, GenRoles<TX, TY>::THREADS, 0, st>>>(a);
}

template <typename S, typename R, int TX, int TY>
static void launch_batch_tile(const BatchArgs<S, R>& b, bool general, int nblocks, cudaStream_t st) {
    if (!general) {
        d2q9_batch_kernel<S, R, TX, TY><<<nblocks, TX * TY, 0, st>>>(b);
        return;
    }
    if constexpr (std::is_same<S, float>::value) {
        if (!general_roles(nblocks)) {
            d2q9_batch_general_kernel<S, R, TX, TY, false><<<nblocks, TX * TY, 0, st>>>(b);
            return;
        }
    }
    d2q9_batch_general_kernel<S, R, TX, TY, true><<<nblocks, GenRoles<TX, TY>::THREADS, 0, st>>>(b);
}

template <typename S, typename R>
cudaError_t launch_d2q9_batch(const BatchArgs<S, R>& b, int variant, bool general, int nblocks, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    switch (d2q9_tile_kernel_variant(variant)) {
    case 0: launch_batch_tile<S, R, 32, 8>(b, general, nblocks, st); break;
    case 1: launch_batch_tile<S, R, 32, 4>(b, general, nblocks, st); break;
    case 2: launch_batch_tile<S, R, 64, 4>(b, general, nblocks, st); break;
    case 3: launch_batch_tile<S, R, 32, 16>(b, general, nblocks, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_d2q9_step(const D2Args<S, R>& a, int variant, bool general, int nblocks, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    switch (d2q9_tile_kernel_variant(variant)) {
    case 0: launch_tile<S, R, 32, 8>(a, general, nblocks, st); break;
    case 1: launch_tile<S, R, 32, 4>(a, general, nblocks, st); break;
    case 2: launch_tile<S, R, 64, 4>(a, general, nblocks, st); break;
    case 3: launch_tile<S, R, 32, 16>(a, general, nblocks, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_d2q9_outlet_chi(const D2Args<S, R>& a, cudaStream_t st) {
    if constexpr (std::is_same<S, __half>::value) {
        return cudaErrorNotSupported;
    } else {
        d2q9_outlet_chi_kernel<S, R><<<1, 256, 0, st>>>(a);
        return cudaGetLastError();
    }
}

template <typename S, typename R>
cudaError_t launch_d2q9_diag(const S* f, const R* macro, const uint16_t* info, const void* rref, int nx,
                             int ny, int px, int py, int pitch, long long plane, double* partials, int nblocks,
                             cudaStream_t st) {
    d2q9_diag_kernel<S, R><<<nblocks, 256, 0, st>>>(f, macro, info, rref, nx, ny, px, py, pitch, plane, partials);
    return cudaGetLastError();
}

template cudaError_t launch_d2q9_batch<float, float>(const BatchArgs<float, float>&, int, bool, int, cudaStream_t);
template cudaError_t launch_d2q9_batch<double, double>(const BatchArgs<double, double>&, int, bool, int, cudaStream_t);
template cudaError_t launch_d2q9_batch<__half, float>(const BatchArgs<__half, float>&, int, bool, int, cudaStream_t);
template cudaError_t launch_d2q9_step<float, float>(const D2Args<float, float>&, int, bool, int, cudaStream_t);
template cudaError_t launch_d2q9_step<double, double>(const D2Args<double, double>&, int, bool, int, cudaStream_t);
template cudaError_t launch_d2q9_step<__half, float>(const D2Args<__half, float>&, int, bool, int, cudaStream_t);
template cudaError_t launch_d2q9_outlet_chi<float, float>(const D2Args<float, float>&, cudaStream_t);
template cudaError_t launch_d2q9_outlet_chi<double, double>(const D2Args<double, double>&, cudaStream_t);
template cudaError_t launch_d2q9_outlet_chi<__half, float>(const D2Args<__half, float>&, cudaStream_t);
template cudaError_t launch_d2q9_diag<float, float>(const float*, const float*, const uint16_t*, const void*, int,
                                                    int, int, int, int, long long, double*, int, cudaStream_t);
template cudaError_t launch_d2q9_diag<double, double>(const double*, const double*, const uint16_t*, const void*,
                                                      int, int, int, int, int, long long, double*, int,
                                                      cudaStream_t);
template cudaError_t launch_d2q9_diag<__half, float>(const __half*, const float*, const uint16_t*, const void*, int,
                                                     int, int, int, int, long long, double*, int, cudaStream_t);

}  // namespace lbm
