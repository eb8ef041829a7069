// Persistent multi-step D2Q9 kernel for batched ensembles.
//
// One cooperative launch advances every member of a batch by many time
// steps.  The grid (at most as many CTAs as fit on the GPU at once, checked
// by the occupancy calculator and guaranteed co-resident by the cooperative
// launch) walks the batch's concatenated tile list, fast tiles first, with
// each CTA taking tiles blockIdx.x, blockIdx.x + gridDim.x, ...; between
// time steps a grid-wide barrier makes one step's populations, open-boundary
// state and flux partials visible to the next.  Every wait of that barrier
// is bounded by a clock64 budget: a CTA whose wait runs out sets a timeout
// bit in the batch status word and leaves the kernel, and CTAs still waiting
// see the bit and leave too, so a barrier that can never complete ends the
// launch with an error status instead of hanging the GPU.
//
// The tile code is the one the launch-per-step kernels run (d2q9_tile.cuh);
// general tiles stage serially on the tile's node threads, so one block
// shape serves both kinds of tile.  Loads of data written during the launch
// go through L2 (LBM_COHERENT_LOADS), since L1 and the read-only path are
// not coherent across SMs within a kernel.
#define LBM_COHERENT_LOADS 1
#include "d2q9_tile.cuh"

namespace lbm {
namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier number `target / gridDim.x` (the arrival counter is
// zeroed before each launch and only grows).  Returns false, with the
// timeout bit set, if the wait ran out or another CTA gave up.
template <typename S, typename R>
__device__ __forceinline__ bool grid_barrier(const PersistArgs<S, R>& p, unsigned target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's writes of the step, ordered before its arrival
        atomicAdd(p.bar, 1u);
        const long long t0 = clock64();
        int ok = 1;
        while (ld_acquire_u32(p.bar) < target) {
            if (ld_acquire_u32(p.pstatus) != 0u || clock64() - t0 > p.spin_limit) {
                ok = 0;
                atomicOr(p.pstatus, PERSIST_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename S, typename R, int TX, int TY>
__global__ void __maxnreg__((gen_maxreg<R, TX, TY, false>()))
    d2q9_persist_kernel(const __grid_constant__ PersistArgs<S, R> p) {
    __shared__ D2Args<S, R> sa;
    static_assert(sizeof(D2Args<S, R>) % 4 == 0, "argument block must be word-sized");
    for (int s = 0; s < p.nsteps; ++s) {
        const int par = s & 1;
        const D2Args<S, R>* av = (s == p.nsteps - 1) ? p.args_last[par] : p.args[par];
        for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
            const int m = p.member[t];
            __syncthreads();  // the previous tile is done with sa and the tile's shared memory
            {
                const int* src = reinterpret_cast<const int*>(av + m);
                int* dst = reinterpret_cast<int*>(&sa);
                for (int i = threadIdx.x; i < (int)(sizeof(D2Args<S, R>) / 4); i += blockDim.x) dst[i] = src[i];
            }
            __syncthreads();
            if (t < p.nfast) step_tile<S, R, TX, TY, false>(sa, p.blocks[t], p.flags[t], 0u, -1);
            else step_tile<S, R, TX, TY, true, false>(sa, p.blocks[t], p.flags[t], p.strips[t], p.slot[t]);
        }
        if (s + 1 < p.nsteps && !grid_barrier(p, (unsigned)(s + 1) * gridDim.x + (unsigned)p.bar_skew)) return;
    }
}

template <typename S, typename R, int TX, int TY>
cudaError_t persist_launch_tile(const PersistArgs<S, R>& p, cudaStream_t st, int* grid_out) {
    static int per_sm = -1, sms = 0;
    auto kern = d2q9_persist_kernel<S, R, TX, TY>;
    if (per_sm < 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, 0);
        if (e != cudaSuccess) {
            per_sm = -1;
            return e;
        }
    }
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    const int grid = p.ntiles < per_sm * sms ? p.ntiles : per_sm * sms;
    if (grid_out) *grid_out = grid;
    if (grid <= 0) return cudaSuccess;
    void* args[] = {const_cast<PersistArgs<S, R>*>(&p)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid), dim3(TX * TY), args, 0, st);
}

}  // namespace

template <typename S, typename R>
cudaError_t launch_d2q9_persist(const PersistArgs<S, R>& p, int variant, cudaStream_t st, int* grid_out) {
    if (p.ntiles <= 0 || p.nsteps <= 0) return cudaSuccess;
    switch (d2q9_tile_kernel_variant(variant)) {
    case 0: return persist_launch_tile<S, R, 32, 8>(p, st, grid_out);
    case 1: return persist_launch_tile<S, R, 32, 4>(p, st, grid_out);
    case 2: return persist_launch_tile<S, R, 64, 4>(p, st, grid_out);
    case 3: return persist_launch_tile<S, R, 32, 16>(p, st, grid_out);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_d2q9_persist<float, float>(const PersistArgs<float, float>&, int, cudaStream_t, int*);

}  // namespace lbm
