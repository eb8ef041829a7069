// Column-marching D2Q9 step for large grids (FP32 storage).
//
// A CTA owns a run of consecutive interior tiles of one tile column (32
// columns wide, a multiple of 8 rows long) and marches up the run 8 rows at
// a time, one warp per row.  For every block of 8 rows a single TMA load
// (cp.async.bulk.tensor, 3D box over [18 planes][10 rows][44 columns])
// brings the post-collision populations of all 18 planes that the block's
// pulls read into shared memory; three buffers keep the copies of the next
// two blocks in flight while a block is processed.  Each warp pulls its row
// once (Eq. 2 with halfway bounce-back, Eq. B1, from shared memory), puts
// the densities into a rolling window of 18 rows x 36 columns (own columns
// plus the two-node halo of Eq. 10's stencil) and keeps the populations in
// registers; it collides that row one block later, when the window holds
// the two rows above it.  Forces (Eqs. 10, 11), velocities (Eqs. 7, 8) and
// the MRT collision with forcing (Eq. 1) are those of the tile kernels (the
// same inline functions).  Compared with a tile kernel, each population is
// read from L2/HBM by one bulk copy instead of one 4-byte load per node and
// direction, the loads of later blocks overlap the arithmetic of the
// current one, and the halo rows above and below a tile are not pulled
// again.
//
// Interior tiles only (the tile's pulls and psi halo stay inside the grid,
// no open face within reach): edge and general tiles keep the tile kernels.
#include <cuda.h>

#include "d2q9_tile.cuh"

namespace lbm {
namespace {

constexpr int MTX = 32;          // columns per CTA (a warp per row)
constexpr int MRB = 8;           // rows per block (warps per CTA)
constexpr int MBW = MTX + 12;    // box columns [xs, xs + MBW), xs = (x0 - 3) rounded down to a multiple of 4
constexpr int MBH = MRB + 2;     // box rows: the sources of one block of pulls
constexpr int MNB = 3;           // box buffers: the copy of block j + 2 is in flight while block j is processed
constexpr int MWR = 2 * MRB + 2; // density window rows: a pulled block, the block being collided, two halo rows
constexpr int MWC = MTX + 4;     // density window columns
constexpr unsigned MBOX_BYTES = 18u * MBH * MBW * 4u;

// One TMA destination: bulk tensor copies need a 128-byte aligned shared
// address, so each buffer is padded to a multiple of 128 bytes.
struct alignas(128) MarchBox {
    float v[18][MBH][MBW];
};
static_assert(sizeof(MarchBox) % 128 == 0, "TMA buffers must stay 128-byte aligned");

struct MarchSmem {
    MarchBox box[MNB];            // at offset 0 of a 128-byte aligned base
    float2 rr[MWR][MWC];          // (rho_1, rho_2) of grid row y in window row (y - ys + 2) mod MWR
    unsigned char sol[MWR][MWC];
    unsigned long long bar[MNB];
    int ok;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Wait for the phase of the given parity to complete, for at most `limit`
// clock64 cycles; false if the wait ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit) {
    const unsigned a = smem_u32(bar);
    const long long t0 = clock64();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tma_load_box(float* dst, const CUtensorMap* map, int x, int y,
                                             unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

// Pull (Eq. 2 with Eq. B1) of node (x, y) from the box in buffer b whose
// first row is row0: f_i(x) = f*_i(x - e_i), or f*_opp(i)(x) when bit i of
// info is set.
__device__ __forceinline__ void pull_box(const MarchSmem& sm, int b, int row0, int xs, int x, int y, unsigned info,
                                         float (&f)[2][9]) {
    const float(*v)[MBH][MBW] = sm.box[b].v;
    if ((info & 0x1ffu) == 0u) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int k = 0; k < 2; ++k) f[k][i] = v[k * 9 + i][y - ey_(i) - row0][x - ex_(i) - xs];
        return;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const bool bb = (info >> i) & 1u;
        const int dir = bb ? opp_(i) : i;
        const int sy = (bb ? y : y - ey_(i)) - row0;
        const int sx = (bb ? x : x - ex_(i)) - xs;
#pragma unroll
        for (int k = 0; k < 2; ++k) f[k][i] = v[k * 9 + dir][sy][sx];
    }
}

__device__ __forceinline__ int wrow_of(int y, int ys) { return (y - ys + 2 + MWR) % MWR; }

// Density pair and solid flag of node (x, y) into window column c; the
// pulled populations are left in f.
__device__ __forceinline__ void density_node(MarchSmem& sm, const D2Args<float, float>& a, int b, int row0, int xs,
                                             int ys, int x, int y, int c, float (&f)[2][9]) {
    const unsigned info = __ldg(a.info + y * a.pitch + x);
    float r0 = 0.f, r1 = 0.f;
    unsigned char sol = 1;
    if (!(info & INFO_SOLID)) {
        pull_box(sm, b, row0, xs, x, y, info, f);
        r0 = rho_of(f[0]);
        r1 = rho_of(f[1]);
        sol = 0;
    }
    const int wr = wrow_of(y, ys);
    sm.rr[wr][c] = make_float2(r0, r1);
    sm.sol[wr][c] = sol;
}

// Halo columns x0 - 2, x0 - 1, x0 + 32, x0 + 33 of `nrows` rows from
// y_first, all taken by warp hw in one pass (4 x nrows <= 32 nodes).
__device__ __forceinline__ void halo_columns(MarchSmem& sm, const D2Args<float, float>& a, int b, int row0, int xs,
                                             int x0, int ys, int y_first, int nrows, int hw) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w == hw && lane < 4 * nrows) {
        const int c4 = lane & 3, y = y_first + (lane >> 2);
        const int c = c4 < 2 ? c4 : MTX + c4;
        float f[2][9];
        density_node(sm, a, b, row0, xs, ys, x0 - 2 + c, y, c, f);
    }
}

// Forces, velocity, collision and store of node (x0 + lane, y) whose
// post-stream populations are f.
__device__ __forceinline__ void collide_node(const MarchSmem& sm, const D2Args<float, float>& a, int x0, int ys,
                                             int y, bool solid_near, const float (&f)[2][9]) {
    const int lane = threadIdx.x & 31;
    const int x = x0 + lane;
    const int n = y * a.pitch + x;
    int wrow[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) wrow[d] = wrow_of(y - 2 + d, ys);  // window rows of y - 2 ... y + 2
    const bool fluid = sm.sol[wrow[2]][lane + 2] == 0;
    const float2 own = sm.rr[wrow[2]][lane + 2];
    const float rho0 = own.x, rho1 = own.y;
    float ux = 0.f, uy = 0.f;
    if (fluid) {
        float g0x, g0y, g1x, g1y;
        psi_gradient<float>([&](int dy, int dx) { return sm.rr[wrow[dy + 2]][lane + 2 + dx]; }, g0x, g0y, g1x, g1y);
        float ax = 0.f, ay = 0.f;
        if (solid_near)
            adhesion_sum<float>([&](int dy, int dx) { return sm.sol[wrow[dy + 2]][lane + 2 + dx]; }, ax, ay);
        const float rt = rho0 + rho1;
        const float inv_rt = 1.f / rt;
        float gw0, gw1;
        adhesion_coeffs(a, rho0, rho1, gw0, gw1);
        const float Fx0 = -a.G12 * rho0 * g1x - gw0 * rho0 * ax + a.body[0] * rho0 * inv_rt;
        const float Fy0 = -a.G12 * rho0 * g1y - gw0 * rho0 * ay + a.body[1] * rho0 * inv_rt;
        const float Fx1 = -a.G12 * rho1 * g0x - gw1 * rho1 * ax + a.body[0] * rho1 * inv_rt;
        const float Fy1 = -a.G12 * rho1 * g0y - gw1 * rho1 * ay + a.body[1] * rho1 * inv_rt;
        const float jx = (jx_of(f[0]) + 0.5f * Fx0) + (jx_of(f[1]) + 0.5f * Fx1);
        const float jy = (jy_of(f[0]) + 0.5f * Fy0) + (jy_of(f[1]) + 0.5f * Fy1);
        ux = jx * inv_rt;
        uy = jy * inv_rt;
        if (a.macro) {
            a.macro[n] = rho0;
            a.macro[a.plane + n] = rho1;
            a.macro[2 * a.plane + n] = ux;
            a.macro[3 * a.plane + n] = uy;
        }
        const float uu3 = 3.f * (ux * ux + uy * uy);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            float o[9];
            collide_scalar<float>(a.s[k], k == 0 ? rho0 : rho1, k == 0 ? Fx0 : Fx1, k == 0 ? Fy0 : Fy1, ux, uy, uu3,
                                  f[k], o);
#pragma unroll
            for (int i = 0; i < 9; ++i) a.fout[(k * 9 + i) * a.plane + n] = o[i];
        }
    }
    const bool bad = fluid && !isfinite(rho0 + rho1 + ux + uy);
    if (__ballot_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, 1u);
}

// Budget of one wait for a bulk copy: ~0.5 s of SM clock (a copy takes
// microseconds); a wait that runs out marks the status word and the CTA
// leaves after a second bounded wait for its copies in flight.
constexpr long long kCopyWaitLimit = 1000000000LL;

// Bulk copies of a run, in issue order: copy 0 holds the sources of the two
// halo rows below the run (rows ys - 2, ys - 1), copy j + 1 those of block j
// (rows ys + 8j ... ys + 8j + 7; block K, past the run, only its first two
// rows, the halo above).  Copy m goes to buffer m % MNB.
__global__ void __launch_bounds__(MTX * MRB, 2)
    d2q9_march_kernel(const __grid_constant__ D2Args<float, float> a, const __grid_constant__ CUtensorMap tmap,
                      const int4* __restrict__ runs, const uint8_t* __restrict__ run_flags) {
    extern __shared__ __align__(128) unsigned char smraw[];
    grid_dep_wait();
    // the launch asks for 128 bytes more than the layout: start it on a 128-byte boundary
    MarchSmem& sm = *reinterpret_cast<MarchSmem*>(smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 run = runs[blockIdx.x];  // {bx | by0 << 16, tiles, first flag, 0}
    const int x0 = (run.x & 0xffff) * MTX - a.xoff;
    const int ys = (run.x >> 16) * MRB - a.yoff;
    const int K = run.y;
    const int xs = (x0 - 3) & ~3;  // x0 >= 3 for interior tiles: a 16-byte aligned box start
    // self-check before any copy: every destination 128-byte aligned, else
    // mark the status word and leave without issuing anything
    unsigned mis = 0u;
#pragma unroll
    for (int q = 0; q < MNB; ++q) mis |= smem_u32(&sm.box[q]) & 127u;
    if (mis) {
        if (threadIdx.x == 0) atomicOr(a.status, 4u);
        return;
    }
    // thread 0 alone issues the copies and waits for them on behalf of the CTA
    int issued = 0, waited = 0;
    auto issue = [&](int m) {  // copy m: the sources of rows [first pulled row - 1, + MBH)
        const int row0 = m == 0 ? ys - 3 : ys + MRB * (m - 1) - 1;
        const int b = m % MNB;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the buffer first
        mbar_expect_tx(&sm.bar[b], MBOX_BYTES);
        tma_load_box(&sm.box[b].v[0][0][0], &tmap, xs, row0, &sm.bar[b]);
        issued = m + 1;
    };
    auto wait_copy = [&](int m) -> bool {  // copies complete in issue order per buffer: use m / MNB of buffer m % MNB
        if (threadIdx.x == 0) {
            int ok = mbar_wait(&sm.bar[m % MNB], (unsigned)((m / MNB) & 1), kCopyWaitLimit) ? 1 : 0;
            waited = m + 1;
            if (!ok) {
                atomicOr(a.status, 2u);
                for (int q = m; q < issued; ++q)  // copies still in flight end before the CTA does
                    mbar_wait(&sm.bar[q % MNB], (unsigned)((q / MNB) & 1), kCopyWaitLimit);
            }
            sm.ok = ok;
        }
        __syncthreads();
        return sm.ok != 0;
    };
    if (threadIdx.x == 0) {
        for (int q = 0; q < MNB; ++q) mbar_init(&sm.bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue(0);
        issue(1);
        if (K >= 1) issue(2);
    }
    __syncthreads();
    (void)waited;
    // halo rows below the run (warps 0, 1), their halo columns (warp 2)
    if (!wait_copy(0)) return;
    if (w < 2) {
        float f[2][9];
        density_node(sm, a, 0, ys - 3, xs, ys, x0 + lane, ys - 2 + w, lane + 2, f);
    }
    halo_columns(sm, a, 0, ys - 3, xs, x0, ys, ys - 2, 2, 2);
    __syncthreads();  // buffer 0 is free again
    // block j: pull rows ys + 8j + w (densities now, collision at block j + 1,
    // once the window holds the two rows above them); collide block j - 1
    float fa[2][9], fb[2][9];
    auto block = [&](int j, float (&fnew)[2][9], float (&fold)[2][9]) -> bool {
        if (threadIdx.x == 0 && j + 2 <= K) issue(j + 3);  // buffer (j + 3) % 3 last served copy j
        if (!wait_copy(j + 1)) return false;
        const int b = (j + 1) % MNB;
        const int row0 = ys + MRB * j - 1;
        const int Y = ys + MRB * j;
        if (j < K) {
            density_node(sm, a, b, row0, xs, ys, x0 + lane, Y + w, lane + 2, fnew);
            halo_columns(sm, a, b, row0, xs, x0, ys, Y, MRB, j & (MRB - 1));
        } else {
            if (w < 2) density_node(sm, a, b, row0, xs, ys, x0 + lane, Y + w, lane + 2, fnew);
            halo_columns(sm, a, b, row0, xs, x0, ys, Y, 2, 2);
        }
        __syncthreads();
        if (j >= 1) {
            const int y = Y - MRB + w;
            collide_node(sm, a, x0, ys, y, (run_flags[run.z + j - 1] & BLOCK_SOLID) != 0, fold);
        }
        __syncthreads();  // window rows and the box buffer are free for the next block
        return true;
    };
    for (int j = 0; j <= K; j += 2) {
        if (!block(j, fa, fb)) return;
        if (j + 1 <= K && !block(j + 1, fb, fa)) return;
    }
}

}  // namespace

size_t d2q9_march_smem_bytes() { return sizeof(MarchSmem) + 128; }

cudaError_t launch_d2q9_march(const D2Args<float, float>& a, const void* tmap, const int4* runs,
                              const uint8_t* run_flags, int nruns, cudaStream_t st) {
    if (nruns <= 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(d2q9_march_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)d2q9_march_smem_bytes());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    d2q9_march_kernel<<<nruns, MTX * MRB, d2q9_march_smem_bytes(), st>>>(a, *static_cast<const CUtensorMap*>(tmap), runs,
                                                                    run_flags);
    return cudaGetLastError();
}

}  // namespace lbm
