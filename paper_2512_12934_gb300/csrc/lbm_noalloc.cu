// Allocation-free FP64 mass tally of caller-owned D2Q9 populations.
//
// Some callers cannot call cudaMalloc: code running under a memory manager
// that owns the whole device pool, inside a pre-reserved arena, or in a
// process whose allocator is locked down.  lbm_mass_noalloc gives them the
// FP64 component-mass reduction of lbm_get_diagnostics without any device
// allocation: its per-row partial sums live in a fixed file-scope device
// array that every GPU which loads the library holds until the process
// exits.  The caller owns the input populations and the output pair.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

// Largest ny the entry point accepts: one FP64 pair per grid row.
constexpr int kNoAllocMaxRows = 65536;
constexpr int kMaxDevices = 64;

// Shared scratch (2 doubles per row, 1 MiB).  Every call on a device reuses
// it and leaves the last call's row sums behind; calls that overlap on the
// GPU (different streams, or host threads racing) corrupt each other.
static __device__ __align__(256) double g_row_partials[2 * kNoAllocMaxRows];

double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

template <typename T>
__global__ void __launch_bounds__(256) mass_rows_kernel(const T* __restrict__ f, int nx, int ny, int pitch,
                                                        const uint8_t* __restrict__ solid, double* rows) {
    const int y = blockIdx.x;
    const size_t plane = (size_t)pitch * ny;
    double s0 = 0.0, s1 = 0.0;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const size_t n = (size_t)y * pitch + x;
        if (solid && solid[n]) continue;
        for (int i = 0; i < 9; ++i) {
            s0 += (double)f[(size_t)i * plane + n];
            s1 += (double)f[(size_t)(9 + i) * plane + n];
        }
    }
    __shared__ double red[2][8];
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s0;
        red[1][threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int w = 0; w < 8; ++w) {
            a0 += red[0][w];
            a1 += red[1][w];
        }
        rows[2 * y] = a0;  // every row in [0, ny) is rewritten: nothing needs clearing
        rows[2 * y + 1] = a1;
    }
}

__global__ void __launch_bounds__(256) mass_finish_kernel(const double* __restrict__ rows, int ny, double* out) {
    double s0 = 0.0, s1 = 0.0;
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
        s0 += rows[2 * y];
        s1 += rows[2 * y + 1];
    }
    __shared__ double red[2][256];
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0][0];
        out[1] = red[1][0];
    }
}

lbm_status reject(lbm_status st, const char* msg) {
    lbm::set_thread_error(msg);
    return st;
}

}  // namespace

extern "C" lbm_status lbm_mass_noalloc(const void* f, int precision, int nx, int ny, int pitch,
                                       const uint8_t* solid, double* mass, void* cuda_stream) {
    if (!f || !mass) return reject(LBM_ERR_INVALID_ARG, "lbm_mass_noalloc: f and mass must be device pointers");
    if (precision != LBM_FP32 && precision != LBM_FP64)
        return reject(LBM_ERR_INVALID_ARG, "lbm_mass_noalloc: precision must be LBM_FP32 or LBM_FP64");
    if (nx < 1 || ny < 1 || pitch < nx)
        return reject(LBM_ERR_INVALID_ARG, "lbm_mass_noalloc: need nx >= 1, ny >= 1 and pitch >= nx");
    if (ny > kNoAllocMaxRows) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "lbm_mass_noalloc: ny = %d exceeds the fixed scratch limit of %d rows", ny,
                      kNoAllocMaxRows);
        return reject(LBM_ERR_INVALID_ARG, msg);
    }
    // An error left pending by earlier, unrelated work on this thread is not
    // ours to report or to clear: refuse before launching anything.
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return reject(LBM_ERR_CUDA, "lbm_mass_noalloc: a CUDA error from earlier work is pending");
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return reject(LBM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return reject(LBM_ERR_UNSUPPORTED, "lbm_mass_noalloc: device index too large");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return reject(LBM_ERR_CUDA, cudaGetErrorString(e));
    double* rows;
    {
        // The device address of the scratch array: the host-side symbol is
        // only a stand-in and must never reach a kernel.  Outside a stream
        // capture it is resolved on every call in the current context (a
        // cached address would be stale after cudaDeviceReset, or belong to
        // another context); inside a capture the address resolved by the
        // last call on this device outside a capture is used.
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_row_partials);
            if (e != cudaSuccess) return reject(LBM_ERR_CUDA, cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double*>(p);
        } else if (!g_scratch_ptr[dev]) {
            return reject(LBM_ERR_INVALID_ARG,
                          "lbm_mass_noalloc: the first call on a device must come before any stream capture");
        }
        rows = g_scratch_ptr[dev];
    }
    if (precision == LBM_FP32)
        mass_rows_kernel<float><<<ny, 256, 0, st>>>(static_cast<const float*>(f), nx, ny, pitch, solid, rows);
    else
        mass_rows_kernel<double><<<ny, 256, 0, st>>>(static_cast<const double*>(f), nx, ny, pitch, solid, rows);
    e = cudaGetLastError();  // nothing was pending, so a launch error here is this call's
    if (e != cudaSuccess) return reject(LBM_ERR_CUDA, cudaGetErrorString(e));
    mass_finish_kernel<<<1, 256, 0, st>>>(rows, ny, mass);
    e = cudaGetLastError();
    if (e != cudaSuccess) return reject(LBM_ERR_CUDA, cudaGetErrorString(e));
    return LBM_OK;
}
