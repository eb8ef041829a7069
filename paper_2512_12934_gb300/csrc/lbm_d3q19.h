// D3Q19 kernels: argument block, face descriptors and launchers.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lbm3 {

constexpr int Q = 19;

// Per-node info word: bits 0-18 pull source of direction i blocked
// (halfway bounce-back or open-face unknown); bit 19 solid; bits 20-22 face
// id + 1 of an open-face node; bits 23-25 face id + 1 of the face whose
// inward neighbour this node is; bit 26 a solid site lies within the
// interaction stencil (adhesion, Eq. 11, is non-zero).
constexpr uint32_t INFO3_SOLID = 1u << 19;
constexpr int INFO3_FACE_SHIFT = 20;
constexpr int INFO3_NBR_SHIFT = 23;
constexpr uint32_t INFO3_NEAR_SOLID = 1u << 26;
// bit 27: a pull source lies across a periodic edge (the plain index offset
// of a direction does not apply)
constexpr uint32_t INFO3_WRAP = 1u << 27;

enum { FACE3_INLET = 1, FACE3_OUTLET = 2 };
// status word bits of a D3Q19 step: non-finite result; a bounded wait on a
// tensor copy that ran out
constexpr unsigned STATUS3_DIVERGED = 1u, STATUS3_TIMEOUT = 2u;
// density box of one FP32 collide tile (32 x 4 x 4 nodes) and its 2-node halo,
// the tensor-copy box of the density field
constexpr int RHO_BOX3_X = 36, RHO_BOX3_Y = 8, RHO_BOX3_Z = 8;
// device scalars of the open boundaries (ping-pong per step)
enum { SC3_LAMBDA = 0, SC3_CHI = 1, SC3_QIN = 2, SC3_QOUT = 3, SC3_UMEAN = 4, SC3_N = 8 };

struct FaceDev3 {
    int kind, side, axis;  // axis = side / 2
    int o[3];              // outward unit normal
    int a0, a1;            // tangential axes (ascending)
    int lo0, lo1, len0, len1;
    int base, count;       // slot range [base, base + count)
    int alpha, chi;
    double sa[3];          // sum over the unknowns of e_a^2 w (Eq. 19)
};

// Slot of face position (t0, t1) = the node's tangential coordinates.
__host__ __device__ inline int face_slot(const FaceDev3& F, int x, int y, int z) {
    const int c[3] = {x, y, z};
    return F.base + (c[F.a1] - F.lo1) * F.len0 + (c[F.a0] - F.lo0);
}

// Arithmetic type of a storage type: FP16 storage computes in float.
template <typename S>
struct Real {
    using type = S;
};
template <>
struct Real<__half> {
    using type = float;
};

// Kernel arguments.  S is the population storage type; densities,
// velocities and every per-face-slot array are kept in R = Real<S>::type.
template <typename S>
struct D3Args {
    using R = typename Real<S>::type;
    int nx, ny, nz, pitch;
    long long plane;
    int periodic[3];
    int open_side[6];
    const S* fin;
    S* fout;
    const uint32_t* info;
    R* rho;   // [plane][2] (rho_1, rho_2) of each node for the step, (0, 0) at solids (psi = 0)
    R* umac;  // [3][plane] u^eq of the step (may be null)
    // FP16 storage only: [2][plane] half-rounded density of each node, the
    // reference its pulled populations are decoded with (in: this step's
    // populations, out: the ones this step writes)
    const __half* rref_in;
    __half* rref_out;
    int nfaces;
    FaceDev3 face[6];
    int nface_slots, have_inlet, out_count;
    const double* face_speed;  // [slots] inward normal speed
    const double* face_rho;    // [2][slots] inlet composition
    const uint8_t* face_fluid; // [slots]
    R* FpF;                    // [slots][2][3] force at the face node (previous step)
    R* FpN;                    // [slots][2][3] force at its inward neighbour
    R* fo;                     // [slots][2][19] outlet post-boundary populations of the previous step
    R* fface;                  // [slots][2][19] post-boundary populations of this step
    R* unbr;                   // [slots][3] u^eq of the outlet's inward neighbours (Eq. 22)
    const R* adv;              // [3][plane] sum_e w s(x+e) e of Eq. 11 (near-solid nodes)
    double* flux;              // [slots][2] flux terms of this step
    const double* scal_in;
    double* scal_out;
    unsigned int* status;
    R G[3];  // G12, G_w,1, G_w,2
    R body[3];
    R s[2][Q];
};

// rho_map: tensor map of the density field as 8-byte (rho_1, rho_2) pairs
// (FP32 contexts; NULL: the collide kernel stages every density box with
// loads)
template <typename S>
cudaError_t launch_step(const D3Args<S>& a, const CUtensorMap* rho_map, cudaStream_t st,
                        cudaEvent_t mid_a = nullptr, cudaEvent_t mid_b = nullptr);

// FP64 sums over fluid nodes of each component's populations and the
// largest |u|^2: partial [nblocks][3].  FP16 storage decodes every
// population with the reference density of the node that reads it (rref).
template <typename S>
cudaError_t launch_mass(const S* f, const uint32_t* info, const typename Real<S>::type* umac, const __half* rref,
                        int nx, int ny, int nz, int pitch, long long plane, double* partial, int nblocks,
                        cudaStream_t st);

}  // namespace lbm3
