// Internal declarations shared by the host runtime (lbm_api.cu) and the
// D2Q9 kernels (lbm_d2q9.cu).  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

// Per-node descriptor word (uint16, same pitched layout as one population
// plane):
//   bits 0..8   direction i's pull source x - e_i is solid or outside a
//               non-periodic edge -> halfway bounce-back (Eq. B1); open-face
//               unknowns also carry the bit and are then rebuilt
//   bit  9      the node itself is solid
//   bits 10..12 face id + 1 when the node lies on an open face
//   bits 13..15 face id + 1 when the node is that face's inward neighbour
//               (x2 of an inlet, x_{N-1} of the outlet)
constexpr unsigned INFO_SOLID = 1u << 9;
constexpr int INFO_FACE_SHIFT = 10;
constexpr int INFO_NBR_SHIFT = 13;
constexpr int MAX_FACES = 4;

// Per-tile flags.  Tiles are split into two launch lists: the fast list
// (deep-interior and edge tiles) and the general list (tiles whose psi halo
// holds an open-face node or crosses an open side, which need the inlet /
// outlet reconstruction and the ghost mirror).
constexpr unsigned BLOCK_EDGE = 1u;     // pull or psi halo crosses a grid edge: wrap / closed-edge logic
constexpr unsigned BLOCK_SOLID = 2u;    // a solid site lies within the tile's psi halo: adhesion
constexpr unsigned BLOCK_GENERAL = 4u;  // general list
constexpr unsigned BLOCK_LAMBDA = 8u;   // general tile that needs lambda / chi (sees outlet face nodes)

constexpr int OC_STRIDE = 28;  // saved outlet-node state: f[18], rho[2], F[4], u_t, u_n(x_{N-1}), written flag

constexpr int FACE_INLET = 1;
constexpr int FACE_OUTLET = 2;

// One open face as the kernels see it.
struct FaceDev {
    int kind;       // FACE_INLET / FACE_OUTLET
    int side;       // 0: x=0, 1: x=nx-1, 2: y=0, 3: y=ny-1
    int lo, hi;     // inclusive extent along the face
    int ox, oy;     // outward normal
    int base;       // first slot of this face in the per-face-node arrays
    int alpha;      // inlet: alpha correction on
    int chi;        // outlet: chi correction on
    double rho_in[2];
    double sxx, syy;  // sum over the unknown set U of w_i e_ix^2 and w_i e_iy^2
};

// Kernel arguments of one D2Q9 step.  S is the population storage type,
// R the arithmetic type.
template <typename S, typename R>
struct D2Args {
    int nx, ny, pitch;
    int plane;              // elements per population plane (pitch * ny); 18 * plane < 2^31
    int px, py;             // periodic axes
    int open_side[4];       // 1 if an open face lies on that side (ghost mirror)
    int xoff, yoff;         // tile-grid origin shift (keeps x_{N-1} with x_N)
    const S* __restrict__ fin;
    S* __restrict__ fout;
    const uint16_t* __restrict__ info;
    const int* __restrict__ blocks;           // tile list: bx | by << 16
    const uint8_t* __restrict__ block_flags;  // per list entry: BLOCK_* flags
    const int* __restrict__ block_slot;       // per list entry: flux-reduction slot or -1
    const unsigned* __restrict__ block_strips;  // per list entry: (side0 + 1) | (side1 + 1) << 8, 0 = none
    int list_off;                             // first list entry of this launch
    int nfaces;
    FaceDev face[MAX_FACES];
    int out_face;           // index of the outlet face or -1
    int have_inlet;
    const R* __restrict__ uin;      // [slot] inward normal speed
    const R* __restrict__ Fp_in;    // [slot][2 nodes][2 comps][2 dims]
    R* __restrict__ Fp_out;
    const R* __restrict__ fo_in;    // [slot][9][2] outlet populations of the last step
    R* __restrict__ fo_out;
    const double* __restrict__ scal_in;   // [0] initial lambda, [1] initial chi, [5] partials valid
    double* __restrict__ scal_out;
    const double* __restrict__ part_in;   // [slot][4] FP64 flux partials of the previous step
    double* __restrict__ part_out;        // [slot][4] partials of this step: Qin, Qout, sum u_n, count
    int nslots;
    R* __restrict__ macro;                // optional [4][plane]: rho1, rho2, ux, uy
    const void* __restrict__ rref_in;     // FP16 storage: [2][plane] half reference densities (decode)
    void* __restrict__ rref_out;          // FP16 storage: reference densities written by this step
    unsigned int* status;
    // same-step chi (Eq. 23 at t + dt): per outlet slot, the state of the
    // outlet node saved for d2q9_outlet_chi_kernel (OC_STRIDE values); NULL
    // for the lagged chi
    R* __restrict__ oc_save;
    // moving walls beyond the closed edges y = 0 (index 0) and y = ny - 1
    // (index 1): x-velocity; wall_on = 0 when both are at rest
    int wall_on;
    R wall_ux[2];
    // Eq. 12: wet_interp = 1 gives both components one adhesion coefficient
    // G_w(rho^e), rho^e = (rho_1 - rho_2)/(rho_1 + rho_2) (piecewise linear
    // within wet_delta of the interface); 0: constant Gw[k] per component
    int wet_interp;
    R wet_delta;
    R G12;
    R Gw[2];
    R s[2][9];
    R body[2];
};

// Batched step: tile list entries of many instances; member[] names the
// instance whose arguments (args[member]) a tile uses.
template <typename S, typename R>
struct BatchArgs {
    const D2Args<S, R>* args;
    const int* blocks;
    const uint8_t* flags;
    const int* slot;
    const unsigned* strips;
    const int* member;
    int off;
};

template <typename S, typename R>
cudaError_t launch_d2q9_batch(const BatchArgs<S, R>& b, int variant, bool general, int nblocks, cudaStream_t st);

// Persistent multi-step launch over a batch's tile list (lbm_d2q9_persist.cu).
// Step s of the launch uses the argument blocks args[s & 1] (args_last[s & 1]
// for its last step, which writes the macroscopic fields); between steps the
// grid waits at a barrier whose every wait is bounded by spin_limit clock64
// cycles.  bar must be zero at launch; pstatus gets PERSIST_TIMEOUT when a
// wait runs out.  bar_skew is added to every barrier target: 0 in normal
// runs, > 0 only to test the timeout path (the barrier can then never
// complete).
constexpr unsigned PERSIST_TIMEOUT = 1u;

template <typename S, typename R>
struct PersistArgs {
    const D2Args<S, R>* args[2];
    const D2Args<S, R>* args_last[2];
    const int* blocks;
    const uint8_t* flags;
    const int* slot;
    const unsigned* strips;
    const int* member;
    int ntiles, nfast, nsteps;
    unsigned* bar;
    unsigned* pstatus;
    long long spin_limit;
    int bar_skew;
};

// grid_out (may be NULL): the number of CTAs launched.
template <typename S, typename R>
cudaError_t launch_d2q9_persist(const PersistArgs<S, R>& p, int variant, cudaStream_t st, int* grid_out);

// Launch one list of tiles of one step: general = false -> fast kernel,
// true -> general kernel; nblocks list entries starting at a.list_off.
template <typename S, typename R>
cudaError_t launch_d2q9_step(const D2Args<S, R>& a, int variant, bool general, int nblocks, cudaStream_t st);

// Same-step chi: after the general tiles of a step, fold that step's flux
// partials into chi (Eq. 23 at t + dt), set the outlet nodes' normal
// velocity (Eq. 22), collide them and store their populations (FP32 and
// FP64 storage).
template <typename S, typename R>
cudaError_t launch_d2q9_outlet_chi(const D2Args<S, R>& a, cudaStream_t st);

// Tile shape of a kernel variant.  Variants 0-3 are tile kernels (32x8,
// 32x4, 64x4, 32x16); variant 4 tiles like variant 0 and runs the interior
// tiles of FP32 contexts through the column-marching kernel.
void d2q9_variant_tile(int variant, int* tx, int* ty);
int d2q9_num_variants();
constexpr int D2Q9_MARCH_VARIANT = 4;
// The tile-kernel variant that serves `variant` (4 -> 0).
inline int d2q9_tile_kernel_variant(int variant) { return variant == D2Q9_MARCH_VARIANT ? 0 : variant; }

// Column-marching step over runs of interior tiles (lbm_d2q9_march.cu).
// runs[r] = {bx | by0 << 16, tiles, first entry in run_flags, 0}; tmap is a
// CUtensorMap over a.fin viewed as [18][ny][pitch] floats with a
// 44 x 10 x 18 box.  Status bit 2 is set if a bulk-copy wait runs out.
size_t d2q9_march_smem_bytes();
cudaError_t launch_d2q9_march(const D2Args<float, float>& a, const void* tmap, const int4* runs,
                              const uint8_t* run_flags, int nruns, cudaStream_t st);
constexpr int D2Q9_MARCH_BOX_W = 44, D2Q9_MARCH_BOX_H = 10;

// FP64 diagnostics over the current populations and macro buffer:
// per-block partials [nblocks][3] = mass1, mass2, max |u|^2.
// (FP16 storage decodes each population with its destination's reference
// density rref [2][plane]; px, py are the periodic flags.)
template <typename S, typename R>
cudaError_t launch_d2q9_diag(const S* f, const R* macro, const uint16_t* info, const void* rref, int nx,
                             int ny, int px, int py, int pitch, long long plane, double* partials, int nblocks,
                             cudaStream_t st);

// Record the calling thread's last error (fixed buffer, no allocation).
void set_thread_error(const char* msg);

}  // namespace lbm
