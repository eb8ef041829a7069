// Tile code of the fused D2Q9 two-component MRT pseudopotential step,
// shared by the launch-per-step kernels (lbm_d2q9.cu) and the persistent
// multi-step kernel (lbm_d2q9_persist.cu).
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
//
// Load policy.  A launch-per-step kernel reads populations through the
// read-only path (ld.global.nc) and the open-boundary and reduction state
// of the previous step with plain loads: everything it reads was written
// before it started.  A persistent kernel reads, in one launch, buffers that
// other SMs wrote during that launch; there L1 and the read-only path may
// hold stale lines, so the including file defines LBM_COHERENT_LOADS to 1
// and those loads go to L2 (ld.global.cg).  Each including file gets its
// own copy of everything below (anonymous namespace).
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "lbm_internal.h"

#ifndef LBM_COHERENT_LOADS
#define LBM_COHERENT_LOADS 0
#endif

namespace lbm {
namespace {

// Population loads (pull streaming) and loads of state written by the
// previous step (inlet forces, outlet populations, flux partials, scalars).
template <typename T>
__device__ __forceinline__ T ld_pop(const T* p) {
    if constexpr (LBM_COHERENT_LOADS) return __ldcg(p);
    else return __ldg(p);
}
template <typename T>
__device__ __forceinline__ T ld_mut(const T* p) {
    if constexpr (LBM_COHERENT_LOADS) return __ldcg(p);
    else return *p;
}


// Early-launch graphs (programmatic dependent launch): a step's kernels may
// be launched while the previous step's grids still run, as soon as all of
// their CTAs have started.  Every kernel a step graph holds therefore waits
// here, before it touches any buffer, until the grids it depends on have
// completed and their memory is visible.  A kernel launched without such a
// dependency returns from the wait at once.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- D2Q9 lattice (velocity order fixed by Eqs. 13, 14, 20 and B2) -------
__host__ __device__ constexpr int ex_(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey_(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp_(int i) {
    return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5);
}
template <typename R>
__host__ __device__ constexpr R w_(int i) {
    return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : R(1) / R(36));
}

// 8th-order isotropic interaction weights by |e|^2 (text after Eq. 12).
template <typename R>
__host__ __device__ constexpr R w8_(int dx, int dy) {
    return (dx * dx + dy * dy == 1) ? R(4) / R(21)
         : (dx * dx + dy * dy == 2) ? R(4) / R(45)
         : (dx * dx + dy * dy == 4) ? R(1) / R(60)
         : (dx * dx + dy * dy == 5) ? R(2) / R(315)
         : (dx * dx + dy * dy == 8) ? R(1) / R(5040)
                                    : R(0);
}

// ---- population storage ------------------------------------------------
// FP32 / FP64 store f itself.  FP16 storage keeps half(f_i - w_i rho_ref),
// where rho_ref is the half-rounded density of component k at the node that
// pulls the value in the next step (the writing node itself when the value
// bounces back).  Every node also stores its own rho_ref, so a reader decodes
// all nine pulled values with one reference pair: deviations stay small for
// the major and the minor phase alike.
template <typename S, typename R>
struct Pop {
    static __device__ __forceinline__ R ld(const S* __restrict__ p, int j, R /*wr*/) {
        return static_cast<R>(ld_pop(p + j));
    }
    static __device__ __forceinline__ void st(S* __restrict__ p, int j, R v, R /*wr*/) {
        p[j] = static_cast<S>(v);
    }
};
template <>
struct Pop<__half, float> {
    static __device__ __forceinline__ float ld(const __half* __restrict__ p, int j, float wr) {
        return __half2float(ld_pop(p + j)) + wr;
    }
    static __device__ __forceinline__ void st(__half* __restrict__ p, int j, float v, float wr) {
        p[j] = __float2half_rn(v - wr);
    }
};

template <typename S>
__host__ __device__ constexpr bool is_half_() { return std::is_same<S, __half>::value; }

// Reference densities of node n for decoding its pulled populations.
template <typename S, typename R>
__device__ __forceinline__ void node_ref(const D2Args<S, R>& a, int n, R (&ref)[2]) {
    if constexpr (is_half_<S>()) {
        const __half* rr = static_cast<const __half*>(a.rref_in);
        ref[0] = __half2float(ld_mut(rr + n));
        ref[1] = __half2float(ld_mut(rr + a.plane + n));
    } else {
        ref[0] = R(0);
        ref[1] = R(0);
    }
}

template <typename R>
__device__ __forceinline__ R half_round(R v) {
    return R(__half2float(__float2half_rn(float(v))));
}

template <typename R>
__device__ __forceinline__ R feq_(int i, R rho, R ux, R uy) {
    const R eu = R(ex_(i)) * ux + R(ey_(i)) * uy;
    const R uu = ux * ux + uy * uy;
    return w_<R>(i) * rho * (R(1) + R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu);
}

// ---- pulls -----------------------------------------------------------------
// Node index n = y * pitch + x (32-bit: the host rejects grids whose 18
// population planes exceed 2^31 elements).  Pull stream (Eq. 2): f_i(x) =
// f*_i(x - e_i); a set bit i in `info` means that source is solid or outside
// a closed edge, and halfway bounce-back (Eq. B1) takes f*_opp(i)(x).

// Interior pull: every source lies inside the grid, no wrap needed.
template <typename S, typename R>
__device__ __forceinline__ void pull_interior(const D2Args<S, R>& a, int n, unsigned info, R (&f)[2][9]) {
    R ref[2];
    node_ref(a, n, ref);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const bool bb = (info >> i) & 1u;
        const int src = bb ? n : n - ex_(i) - ey_(i) * a.pitch;
        const int dir = bb ? opp_(i) : i;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            f[k][i] = Pop<S, R>::ld(a.fin, (k * 9 + dir) * a.plane + src, w_<R>(i) * ref[k]);
    }
}

// General pull: sources wrap on periodic axes.
template <typename S, typename R>
__device__ __forceinline__ void pull_wrap(const D2Args<S, R>& a, int x, int y, unsigned info, R (&f)[2][9]) {
    const int n = y * a.pitch + x;
    R ref[2];
    node_ref(a, n, ref);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int src, dir;
        if ((info >> i) & 1u) {
            src = n;
            dir = opp_(i);
        } else {
            int sx = x - ex_(i), sy = y - ey_(i);
            if (sx < 0) sx += a.nx; else if (sx >= a.nx) sx -= a.nx;
            if (sy < 0) sy += a.ny; else if (sy >= a.ny) sy -= a.ny;
            src = sy * a.pitch + sx;
            dir = i;
        }
#pragma unroll
        for (int k = 0; k < 2; ++k)
            f[k][i] = Pop<S, R>::ld(a.fin, (k * 9 + dir) * a.plane + src, w_<R>(i) * ref[k]);
    }
    // Moving wall beyond a closed y edge (halfway bounce-back carrying the
    // wall's momentum): a population reflected there gains
    // 2 w_i rho_k (e_i . u_w) / c_s^2, rho_k the node's own density (the sum
    // of its post-collision populations).  FP32 / FP64 storage.
    if constexpr (!is_half_<S>()) {
        const int side = y == 0 ? 0 : (y == a.ny - 1 ? 1 : -1);
        if (a.wall_on && !a.py && side >= 0 && a.wall_ux[side] != R(0)) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                R rk = R(0);
#pragma unroll
                for (int j = 0; j < 9; ++j) rk += Pop<S, R>::ld(a.fin, (k * 9 + j) * a.plane + n, R(0));
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (((info >> i) & 1u) && (side == 0 ? ey_(i) > 0 : ey_(i) < 0))
                        f[k][i] += R(6) * w_<R>(i) * rk * (R(ex_(i)) * a.wall_ux[side]);
            }
        }
    }
}

// rho_k = sum_i f_i (Eq. 8) in a fixed pairwise order.
template <typename R>
__device__ __forceinline__ R rho_of(const R (&g)[9]) {
    return g[0] + (((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8])));
}
template <typename R>
__device__ __forceinline__ R jx_of(const R (&g)[9]) {
    return (g[1] - g[3]) + ((g[5] - g[7]) + (g[8] - g[6]));
}
template <typename R>
__device__ __forceinline__ R jy_of(const R (&g)[9]) {
    return (g[2] - g[4]) + ((g[5] - g[7]) + (g[6] - g[8]));
}

// Outward normal of a grid side (0: x=0, 1: x=nx-1, 2: y=0, 3: y=ny-1).
__host__ __device__ constexpr int side_ox(int side) { return side == 0 ? -1 : (side == 1 ? 1 : 0); }
__host__ __device__ constexpr int side_oy(int side) { return side == 2 ? -1 : (side == 3 ? 1 : 0); }
// Direction i is unknown at a node of that side when it points into the domain.
__host__ __device__ constexpr bool unknown_(int side, int i) {
    return ex_(i) * side_ox(side) + ey_(i) * side_oy(side) < 0;
}

// Open-face reconstruction of the unknown populations of a face node on side
// SIDE: inlet Eq. 13/14 + alpha (Eqs. 15-19), outlet Eq. 20 with lambda.
// g holds the pulled populations of the inward neighbour x - n.
template <int SIDE, typename S, typename R>
__device__ __forceinline__ void face_fix_with(const D2Args<S, R>& a, const FaceDev& F, int x, int y, R lam,
                                              const R (&g)[2][9], R (&f)[2][9]) {
    constexpr int OX = side_ox(SIDE), OY = side_oy(SIDE);
    const int slot = F.base + ((SIDE <= 1) ? y : x) - F.lo;
    if (F.kind == FACE_INLET) {
        const R* Fp = a.Fp_in + slot * 8;  // [node x1/x2][k][d]
        const R r20 = rho_of(g[0]), r21 = rho_of(g[1]);
        const R jx = (jx_of(g[0]) + R(0.5) * ld_mut(Fp + 4)) + (jx_of(g[1]) + R(0.5) * ld_mut(Fp + 6));
        const R jy = (jy_of(g[0]) + R(0.5) * ld_mut(Fp + 5)) + (jy_of(g[1]) + R(0.5) * ld_mut(Fp + 7));
        const R inv2 = R(1) / (r20 + r21);
        const R u2x = jx * inv2, u2y = jy * inv2;
        const R sp = a.uin[slot];
        const R uix = R(-OX) * sp, uiy = R(-OY) * sp;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const R rin = R(F.rho_in[k]);
            const R r2 = k == 0 ? r20 : r21;
#pragma unroll
            for (int i = 0; i < 9; ++i)
                if (unknown_(SIDE, i))
                    f[k][i] = feq_<R>(i, rin, uix, uiy) + (g[k][i] - feq_<R>(i, r2, u2x, u2y));
            if (F.alpha) {
                const R mx = jx_of(f[k]) + R(0.5) * ld_mut(Fp + k * 2 + 0);
                const R my = jy_of(f[k]) + R(0.5) * ld_mut(Fp + k * 2 + 1);
                // sum over the unknown set of w e_x^2 and w e_y^2 (1/6 normal, 1/18 tangential)
                constexpr R SXX = OX != 0 ? R(1) / R(6) : R(1) / R(18);
                constexpr R SYY = OY != 0 ? R(1) / R(6) : R(1) / R(18);
                const R cx = (rin * uix - mx) / SXX, cy = (rin * uiy - my) / SYY;
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (unknown_(SIDE, i)) f[k][i] += w_<R>(i) * (R(ex_(i)) * cx + R(ey_(i)) * cy);
            }
        }
    } else {
        const R inv = R(1) / (R(1) + lam);
        const R* fo = a.fo_in + slot * 18;
#pragma unroll
        for (int i = 0; i < 9; ++i)
            if (unknown_(SIDE, i))
#pragma unroll
                for (int k = 0; k < 2; ++k) f[k][i] = (ld_mut(fo + i * 2 + k) + lam * g[k][i]) * inv;
    }
}

template <int SIDE, typename S, typename R>
__device__ __forceinline__ void face_fix_side(const D2Args<S, R>& a, const FaceDev& F, int x, int y, R lam,
                                              R (&f)[2][9]) {
    const int x2 = x - side_ox(SIDE), y2 = y - side_oy(SIDE);  // inward neighbour
    const unsigned info2 = a.info[y2 * a.pitch + x2];
    R g[2][9];
    pull_wrap(a, x2, y2, info2, g);
    face_fix_with<SIDE>(a, F, x, y, lam, g, f);
}

template <typename S, typename R>
__device__ __forceinline__ void face_fix(const D2Args<S, R>& a, int x, int y, int fid, R lam, R (&f)[2][9]) {
    const FaceDev& F = a.face[fid];
    switch (F.side) {
    case 0: face_fix_side<0>(a, F, x, y, lam, f); break;
    case 1: face_fix_side<1>(a, F, x, y, lam, f); break;
    case 2: face_fix_side<2>(a, F, x, y, lam, f); break;
    default: face_fix_side<3>(a, F, x, y, lam, f); break;
    }
}

template <typename S, typename R>
__device__ __forceinline__ void pull_general(const D2Args<S, R>& a, int x, int y, unsigned info, R lam,
                                             R (&f)[2][9]) {
    pull_wrap(a, x, y, info, f);
    const int fid = (int)((info >> INFO_FACE_SHIFT) & 7u);
    if (fid) face_fix(a, x, y, fid - 1, lam, f);
}

// Virtual site of the psi stencil: periodic wrap, ghost mirror across an open
// side (Eqs. 24, 25), or solid outside a closed edge.  Returns true if solid.
template <typename S, typename R>
__device__ __forceinline__ bool resolve_site(const D2Args<S, R>& a, int& gx, int& gy) {
    if (gx < 0 || gx >= a.nx) {
        if (a.px) {
            gx %= a.nx;
            if (gx < 0) gx += a.nx;
        } else if (a.open_side[gx < 0 ? 0 : 1]) {
            gx = gx < 0 ? -1 - gx : 2 * a.nx - 1 - gx;
            gx = min(max(gx, 0), a.nx - 1);
        } else {
            return true;
        }
    }
    if (gy < 0 || gy >= a.ny) {
        if (a.py) {
            gy %= a.ny;
            if (gy < 0) gy += a.ny;
        } else if (a.open_side[gy < 0 ? 2 : 3]) {
            gy = gy < 0 ? -1 - gy : 2 * a.ny - 1 - gy;
            gy = min(max(gy, 0), a.ny - 1);
        } else {
            return true;
        }
    }
    return false;
}

// Site of the psi stencil on a tile without open sides: periodic wrap or solid
// outside a closed edge.  Returns true if solid.
template <typename S, typename R>
__device__ __forceinline__ bool resolve_closed(const D2Args<S, R>& a, int& gx, int& gy) {
    if (gx < 0 || gx >= a.nx) {
        if (!a.px) return true;
        gx += gx < 0 ? a.nx : -a.nx;
    }
    if (gy < 0 || gy >= a.ny) {
        if (!a.py) return true;
        gy += gy < 0 ? a.ny : -a.ny;
    }
    return false;
}

// Tile modes: 0 deep interior, 1 edge (wrap / closed edges), 2 general.
// Density pair of a halo site (no populations kept).  Returns false if solid.
template <typename S, typename R, int MODE>
__device__ __forceinline__ bool site_rho(const D2Args<S, R>& a, int gx, int gy, R& r0, R& r1, R lam = R(0)) {
    if (MODE == 2) {
        if (resolve_site(a, gx, gy)) return false;
        const unsigned inf = a.info[gy * a.pitch + gx];
        if (inf & INFO_SOLID) return false;
        R g[2][9];
        pull_general(a, gx, gy, inf, lam, g);
        r0 = rho_of(g[0]);
        r1 = rho_of(g[1]);
    } else if (MODE == 1) {
        if (resolve_closed(a, gx, gy)) return false;
        const unsigned inf = a.info[gy * a.pitch + gx];
        if (inf & INFO_SOLID) return false;
        R g[2][9];
        pull_wrap(a, gx, gy, inf, g);
        r0 = rho_of(g[0]);
        r1 = rho_of(g[1]);
    } else {
        const int n = gy * a.pitch + gx;
        const unsigned inf = a.info[n];
        if (inf & INFO_SOLID) return false;
        R g[2][9];
        pull_interior(a, n, inf, g);
        r0 = rho_of(g[0]);
        r1 = rho_of(g[1]);
    }
    return true;
}

// (rho_1, rho_2) of one site, kept together so that a stencil tap is one
// shared load and, in FP32, both components share packed FP32x2 FMAs.
template <typename R>
struct RhoPair;
template <>
struct RhoPair<float> {
    using type = float2;
};
template <>
struct RhoPair<double> {
    using type = double2;
};
template <typename R>
__device__ __forceinline__ typename RhoPair<R>::type rpair(R a, R b) {
    typename RhoPair<R>::type v;
    v.x = a;
    v.y = b;
    return v;
}

template <typename S, typename R, int TX, int TY>
struct TileSmem {
    typename RhoPair<R>::type rr[TY + 4][TX + 4];
    unsigned char sol[TY + 4][TX + 4];
    R un[TX > TY ? TX : TY];
    R lam, chi;  // outlet coefficients of this step (general tiles that see the outlet)
};

// General tiles also keep up to two face strips: the face nodes of one grid
// side along the tile's halo range, each reconstructed once per tile.
template <typename S, typename R, int TX, int TY>
struct TileSmemGen : TileSmem<S, R, TX, TY> {
    static constexpr int SL = (TX > TY ? TX : TY) + 4;  // strip entries (halo range)
    static constexpr int SO = (TX > TY ? TX : TY);      // own entries
    // The strips are dead once staging has passed its barrier; the FP64 flux
    // terms of the nodes that contribute to Eqs. 21 and 23 (packed per warp in
    // lane order, with their count per warp) are written after it and reuse
    // the space.  Measured on GB300: with separate storage (12 KB per FP32
    // 32x4 tile instead of 7.9 KB) the general list stopped overlapping the
    // fast list inside a step and the step took a third longer.
    union {
        struct {
            R fs_rho[2][SL][2];
            R fs_f[2][SO][18];
        };
        struct {
            double fl[TX * TY / 32][32][4];
            int fcnt[TX * TY / 32];
        };
    };
};

// Stage the tile's densities (own node + two-node halo) in shared memory;
// the own node's post-stream populations stay in registers.
template <typename S, typename R, int TX, int TY, int MODE>
__device__ __forceinline__ void stage_tile(const D2Args<S, R>& a, TileSmem<S, R, TX, TY>& sm, int x0, int y0,
                                           int tx, int ty, R (&f)[2][9], unsigned& info, bool& fluid) {
    constexpr int RX = TX + 4, RY = TY + 4, NT = TX * TY;
    auto stage_own = [&]() {
        const int x = x0 + tx, y = y0 + ty;
        R r0 = R(0), r1 = R(0);
        unsigned char sol = 1;
        if (MODE != 0) {
            const bool inb = (x >= 0 && x < a.nx && y >= 0 && y < a.ny);
            info = INFO_SOLID;
            fluid = false;
            if (inb) {
                info = a.info[y * a.pitch + x];
                fluid = !(info & INFO_SOLID);
                if (fluid) {
                    if (MODE == 2) pull_general(a, x, y, info, R(0), f);
                    else pull_wrap(a, x, y, info, f);
                    r0 = rho_of(f[0]);
                    r1 = rho_of(f[1]);
                    sol = 0;
                }
            } else if (site_rho<S, R, MODE>(a, x, y, r0, r1)) {
                sol = 0;
            }
        } else {
            const int n = y * a.pitch + x;
            info = a.info[n];
            fluid = !(info & INFO_SOLID);
            if (fluid) {
                pull_interior(a, n, info, f);
                r0 = rho_of(f[0]);
                r1 = rho_of(f[1]);
                sol = 0;
            }
        }
        sm.rr[ty + 2][tx + 2] = rpair<R>(r0, r1);
        sm.sol[ty + 2][tx + 2] = sol;
    };
    // halo ring: densities only
    constexpr int RING = RX * RY - TX * TY;
    auto ring_site = [&](int p) {
        int rx, ry;
        if (p < 2 * RX) {                // two rows above
            ry = p / RX;
            rx = p % RX;
        } else if (p < 4 * RX) {         // two rows below
            ry = TY + 2 + (p - 2 * RX) / RX;
            rx = (p - 2 * RX) % RX;
        } else {                          // two columns on each side
            const int q = p - 4 * RX;
            ry = 2 + q / 4;
            const int c = q % 4;
            rx = c < 2 ? c : TX + c;
        }
        R h0 = R(0), h1 = R(0);
        const bool ok = site_rho<S, R, MODE>(a, x0 - 2 + rx, y0 - 2 + ry, h0, h1);
        sm.rr[ry][rx] = rpair<R>(h0, h1);
        sm.sol[ry][rx] = ok ? 0 : 1;
    };
    // When one pass of the node threads covers the ring, its pulls are
    // issued first and the own node's independent loads go out under their
    // latency (measured on GB300: 3 % faster per HBM-resident step with
    // 32x8 tiles, 1 % slower with 32x4 tiles, whose ring takes two passes).
    if constexpr (RING <= NT) {
        if ((int)threadIdx.x < RING) ring_site(threadIdx.x);
        stage_own();
    } else {
        stage_own();
        for (int p = threadIdx.x; p < RING; p += NT) ring_site(p);
    }
}

// Strip geometry: entry e of a strip on side `side` is node (sx, sy).
template <int TX, int TY>
__device__ __forceinline__ void strip_node(int side, int e, int x0, int y0, int nx, int ny, int& sx, int& sy) {
    if (side <= 1) {
        sx = side == 0 ? 0 : nx - 1;
        sy = y0 - 2 + e;
    } else {
        sx = x0 - 2 + e;
        sy = side == 2 ? 0 : ny - 1;
    }
}

// Strip slot of an in-grid site on a face side of this tile, or -1.
template <int TX, int TY>
__device__ __forceinline__ int strip_entry(int side, int gx, int gy, int x0, int y0, int nx, int ny) {
    const int SL = side <= 1 ? TY + 4 : TX + 4;
    int e = -1;
    if (side == 0 && gx == 0) e = gy - (y0 - 2);
    else if (side == 1 && gx == nx - 1) e = gy - (y0 - 2);
    else if (side == 2 && gy == 0) e = gx - (x0 - 2);
    else if (side == 3 && gy == ny - 1) e = gx - (x0 - 2);
    return (e >= 0 && e < SL) ? e : -1;
}

// General-tile staging.  Threads without halo-ring work reconstruct the face
// nodes of the tile's strips (inlet Eqs. 13-19 / outlet Eq. 20) once each;
// own nodes and halo sites that are such face nodes read the result from
// shared memory instead of repeating the reconstruction.
// Barrier over the NT node threads of a tile.  General tiles launch extra
// staging warps that leave after staging, so their later barriers name the
// node threads only (barrier 1); fast tiles are exactly NT threads.
template <bool GEN, int NT>
__device__ __forceinline__ void tile_sync() {
    if constexpr (GEN) asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    else __syncthreads();
}

// Thread roles of a general tile.  Threads [0, NT) own the tile's nodes;
// [NT, NT + RING) each pull one halo-ring node; the warps from SB on
// reconstruct the face strips (and fold lambda and chi, which only face
// reconstruction needs).  The three groups pull concurrently, so a general
// tile's staging latency is one chain of dependent loads instead of three.
template <int TX, int TY>
struct GenRoles {
    static constexpr int NT = TX * TY;
    static constexpr int RX = TX + 4, RY = TY + 4;
    static constexpr int RING = RX * RY - NT;
    static constexpr int SB = (NT + RING + 31) / 32 * 32;
    static constexpr int SL = (TX > TY ? TX : TY) + 4;
    static constexpr int THREADS = SB + (2 * SL + 31) / 32 * 32;
    static_assert(THREADS <= 1024, "general tile exceeds a CTA");
};

// Halo-ring entry p as tile-local coordinates (two rows above, two below,
// two columns on each side).
template <int TX, int TY>
__device__ __forceinline__ void ring_coords(int p, int& rx, int& ry) {
    constexpr int RX = TX + 4;
    if (p < 2 * RX) {
        ry = p / RX;
        rx = p % RX;
    } else if (p < 4 * RX) {
        ry = TY + 2 + (p - 2 * RX) / RX;
        rx = (p - 2 * RX) % RX;
    } else {
        const int q = p - 4 * RX;
        ry = 2 + q / 4;
        const int c = q % 4;
        rx = c < 2 ? c : TX + c;
    }
}

// lambda (Eq. 21) and chi (Eq. 23) from the previous step's FP64 flux
// partials (four terms per slot), summed by one warp in a fixed order so that
// every tile gets the same bits: lane 8j + c sums term j over slots c, c + 8,
// c + 16, ... in order, then the eight chains of a term are added in a
// three-level tree.  GB300's FP64 pipe is narrow, so the FP64 instruction
// count (11 adds per lane) sets this fold's latency.  The loads are issued
// first (begin) and summed later (finish), so that the caller can put its
// own independent loads in between.
struct LamFold {
    double p[8];
    double valid;
};

// part / scal: the partials and scalar block to fold (those of the previous
// step, a.part_in / a.scal_in, for the lagged lambda and chi).
template <typename S, typename R>
__device__ __forceinline__ void fold_begin(const D2Args<S, R>& a, LamFold& L, const double* part,
                                           const double* scal) {
    const int lane = threadIdx.x & 31, j = lane >> 3, c = lane & 7;
    L.valid = ld_mut(scal + 5);
#pragma unroll
    for (int k = 0; k < 8; ++k) L.p[k] = c + 8 * k < a.nslots ? ld_mut(part + (c + 8 * k) * 4 + j) : 0.0;
}
template <typename S, typename R>
__device__ __forceinline__ void fold_begin(const D2Args<S, R>& a, LamFold& L) {
    fold_begin(a, L, a.part_in, a.scal_in);
}

template <typename S, typename R>
__device__ __forceinline__ void fold_finish(const D2Args<S, R>& a, const LamFold& L, double& lam, double& chi,
                                            const double* part, const double* scal) {
    const int lane = threadIdx.x & 31, j = lane >> 3, c = lane & 7;
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (c + 8 * k < a.nslots) t += L.p[k];
    for (int sl = c + 64; sl < a.nslots; sl += 8) t += ld_mut(part + sl * 4 + j);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    double T[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) T[q] = __shfl_sync(0xffffffffu, t, 8 * q);
    // the quotients are taken in the tile's arithmetic precision R, which
    // is where lambda and chi are used
    lam = ld_mut(scal + 0);
    chi = ld_mut(scal + 1);
    if (L.valid != 0.0 && a.out_face >= 0 && T[3] > 0.0) {
        const R um = R(T[2]) / R(T[3]);
        lam = um > R(0) ? double(um) : 0.0;
        chi = (!a.have_inlet || fabs(T[1]) < 1e-14) ? 1.0 : double(R(T[0]) / R(T[1]));
    }
}
template <typename S, typename R>
__device__ __forceinline__ void fold_finish(const D2Args<S, R>& a, const LamFold& L, double& lam, double& chi) {
    fold_finish(a, L, lam, chi, a.part_in, a.scal_in);
}

template <typename S, typename R, int TX, int TY>
__device__ __forceinline__ void stage_tile_general(const D2Args<S, R>& a, TileSmemGen<S, R, TX, TY>& sm, int x0,
                                                   int y0, unsigned strips, unsigned bflags, R (&f)[2][9],
                                                   unsigned& info, bool& fluid) {
    using G = GenRoles<TX, TY>;
    constexpr int NT = G::NT, RING = G::RING;
    const int tid = threadIdx.x;
    const int side0 = (int)(strips & 0xffu) - 1, side1 = (int)((strips >> 8) & 0xffu) - 1;
    const int len0 = side0 < 0 ? 0 : (side0 <= 1 ? G::RY : G::RX);
    const int len1 = side1 < 0 ? 0 : (side1 <= 1 ? G::RY : G::RX);
    auto strip_of = [&](int side) { return side == side0 ? 0 : (side == side1 ? 1 : -1); };

    info = INFO_SOLID;
    fluid = false;
    int own_strip = -1, own_idx = 0;
    int def_j = -1, def_e = 0, def_rx = 0, def_ry = 0;
    // a node whose pull needs lambda but lies outside the strips (a face node
    // beyond two sides, a mirrored ghost site) waits for the second pass
    bool pending = false;
    int pend_x = 0, pend_y = 0, pend_rx = 0, pend_ry = 0;
    unsigned pend_info = 0;

    if (tid < NT) {
        // ---- own node ----
        const int tx = tid % TX, ty = tid / TX;
        const int x = x0 + tx, y = y0 + ty;
        R r0 = R(0), r1 = R(0);
        unsigned char sol = 1;
        if (x >= 0 && x < a.nx && y >= 0 && y < a.ny) {
            info = a.info[y * a.pitch + x];
            fluid = !(info & INFO_SOLID);
            if (fluid) {
                sol = 0;
                const int fid = (int)((info >> INFO_FACE_SHIFT) & 7u);
                if (fid) {
                    const int side = a.face[fid - 1].side;
                    own_strip = strip_of(side);
                    own_idx = side <= 1 ? ty : tx;
                    if (own_strip < 0) pending = true;
                } else {
                    pull_general(a, x, y, info, R(0), f);
                    r0 = rho_of(f[0]);
                    r1 = rho_of(f[1]);
                }
            }
        } else {
            pending = true;
        }
        pend_x = x;
        pend_y = y;
        pend_rx = tx + 2;
        pend_ry = ty + 2;
        sm.rr[ty + 2][tx + 2] = rpair<R>(r0, r1);
        sm.sol[ty + 2][tx + 2] = sol;
    } else if (tid < NT + RING) {
        // ---- halo ring: densities only ----
        int rx, ry;
        ring_coords<TX, TY>(tid - NT, rx, ry);
        int gx = x0 - 2 + rx, gy = y0 - 2 + ry;
        R h0 = R(0), h1 = R(0);
        unsigned char hs = 1;
        if (!resolve_site(a, gx, gy)) {
            const unsigned inf = a.info[gy * a.pitch + gx];
            if (!(inf & INFO_SOLID)) {
                hs = 0;
                const int fid = (int)((inf >> INFO_FACE_SHIFT) & 7u);
                if (fid) {
                    const int side = a.face[fid - 1].side;
                    const int j = strip_of(side);
                    const int e = j >= 0 ? strip_entry<TX, TY>(side, gx, gy, x0, y0, a.nx, a.ny) : -1;
                    if (j >= 0 && e >= 0) {
                        def_j = j;  // filled from the strip after the barrier
                        def_e = e;
                        def_rx = rx;
                        def_ry = ry;
                    } else {
                        pending = true;
                        pend_x = gx;
                        pend_y = gy;
                        pend_rx = rx;
                        pend_ry = ry;
                        pend_info = inf;
                    }
                } else {
                    R g[2][9];
                    pull_general(a, gx, gy, inf, R(0), g);
                    h0 = rho_of(g[0]);
                    h1 = rho_of(g[1]);
                }
            }
        }
        sm.rr[ry][rx] = rpair<R>(h0, h1);
        sm.sol[ry][rx] = hs;
    } else if (tid >= G::SB) {
        // ---- face strips (and lambda, chi) ----
        // warp-uniform: the fold is a warp collective
        const int t = tid - G::SB;
        const bool lam_on = (bflags & BLOCK_LAMBDA) != 0;
        LamFold L;
        if (lam_on && t < 32) fold_begin(a, L);
        const bool has = t < len0 + len1;
        const int j = t < len0 ? 0 : 1;
        const int e = j == 0 ? t : t - len0;
        const int side = j == 0 ? side0 : side1;
        int sx = -1, sy = -1;
        unsigned inf = INFO_SOLID, inf2 = INFO_SOLID;
        if (has) {
            strip_node<TX, TY>(side, e, x0, y0, a.nx, a.ny, sx, sy);
            if (sx >= 0 && sx < a.nx && sy >= 0 && sy < a.ny) {
                inf = a.info[sy * a.pitch + sx];
                // the inward neighbour along this strip's normal, read with
                // the node's own word (a corner node may belong to the face of
                // the other side; it is re-read below then)
                const int x2 = sx - side_ox(side), y2 = sy - side_oy(side);
                if (x2 >= 0 && x2 < a.nx && y2 >= 0 && y2 < a.ny) inf2 = a.info[y2 * a.pitch + x2];
            }
        }
        // both pulls in flight before lambda is folded; only the blend of
        // Eqs. 13-20 waits for it
        const bool face = !(inf & INFO_SOLID) && ((inf >> INFO_FACE_SHIFT) & 7u);
        const int fid = (int)((inf >> INFO_FACE_SHIFT) & 7u) - 1;
        const int fside = face ? a.face[fid].side : 0;
        R g[2][9], gn[2][9];
        if (face) {
            const int x2 = sx - side_ox(fside), y2 = sy - side_oy(fside);
            if (fside != side) inf2 = a.info[y2 * a.pitch + x2];
            pull_wrap(a, sx, sy, inf, g);
            pull_wrap(a, x2, y2, inf2, gn);
        }
        R lam = R(0);
        if (lam_on) {
            // the first strip warp folds; the others read its result (the
            // block flags are tile-uniform, so every strip warp gets here)
            if (t < 32) {
                double dl, dc;
                fold_finish(a, L, dl, dc);
                if (t == 0) {
                    sm.lam = R(dl);
                    sm.chi = R(dc);
                }
            }
            asm volatile("bar.sync 2, %0;" ::"n"(G::THREADS - G::SB) : "memory");
            lam = sm.lam;
        }
        if (face) {
            const FaceDev& F = a.face[fid];
            switch (fside) {
            case 0: face_fix_with<0>(a, F, sx, sy, lam, gn, g); break;
            case 1: face_fix_with<1>(a, F, sx, sy, lam, gn, g); break;
            case 2: face_fix_with<2>(a, F, sx, sy, lam, gn, g); break;
            default: face_fix_with<3>(a, F, sx, sy, lam, gn, g); break;
            }
        }
        if (has && face) {
            sm.fs_rho[j][e][0] = rho_of(g[0]);
            sm.fs_rho[j][e][1] = rho_of(g[1]);
            const int o = side <= 1 ? sy - y0 : sx - x0;
            const bool own = sx >= x0 && sx < x0 + TX && sy >= y0 && sy < y0 + TY;
            if (own)
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int i = 0; i < 9; ++i) sm.fs_f[j][o][k * 9 + i] = g[k][i];
        }
    }
    // ---- second pass: pulls that need lambda outside the strips ----
    if (__syncthreads_or(pending)) {
        if (pending) {
            const R lam = (bflags & BLOCK_LAMBDA) ? sm.lam : R(0);
            R r0 = R(0), r1 = R(0);
            unsigned char sol = 1;
            if (tid < NT) {
                if (fluid) {
                    pull_general(a, pend_x, pend_y, info, lam, f);
                    r0 = rho_of(f[0]);
                    r1 = rho_of(f[1]);
                    sol = 0;
                } else if (site_rho<S, R, 2>(a, pend_x, pend_y, r0, r1, lam)) {
                    sol = 0;
                }
            } else {
                R g[2][9];
                pull_general(a, pend_x, pend_y, pend_info, lam, g);
                r0 = rho_of(g[0]);
                r1 = rho_of(g[1]);
                sol = 0;
            }
            sm.rr[pend_ry][pend_rx] = rpair<R>(r0, r1);
            sm.sol[pend_ry][pend_rx] = sol;
        }
        __syncthreads();
    }
    if (own_strip >= 0) {
        const int tx = tid % TX, ty = tid / TX;
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int i = 0; i < 9; ++i) f[k][i] = sm.fs_f[own_strip][own_idx][k * 9 + i];
        sm.rr[ty + 2][tx + 2] = rpair<R>(rho_of(f[0]), rho_of(f[1]));
    }
    if (def_j >= 0) {
        sm.rr[def_ry][def_rx] = rpair<R>(sm.fs_rho[def_j][def_e][0], sm.fs_rho[def_j][def_e][1]);
    }
}

// Serial staging of a general tile by its NT node threads (strips, own
// node, halo ring in turn).  Used when the general list is long enough to
// fill the GPU by itself (batched ensembles): there the extra staging warps
// of GenRoles cost more SM room than their latency saving is worth.
template <typename S, typename R, int TX, int TY>
__device__ __forceinline__ void stage_tile_compact(const D2Args<S, R>& a, TileSmemGen<S, R, TX, TY>& sm, int x0,
                                                   int y0, int tx, int ty, unsigned strips, unsigned bflags,
                                                   R (&f)[2][9], unsigned& info, bool& fluid) {
    constexpr int RX = TX + 4, RY = TY + 4, NT = TX * TY;
    constexpr int RING = RX * RY - TX * TY;
    const int tid = threadIdx.x;
    // ---- lambda (Eq. 21) and chi (Eq. 23): the last warp folds the previous
    // step's partials (same order, same bits as the staging-role tiles)
    if (bflags & BLOCK_LAMBDA) {
        if (tid >= NT - 32) {
            LamFold L;
            fold_begin(a, L);
            double dl, dc;
            fold_finish(a, L, dl, dc);
            if (tid == NT - 32) {
                sm.lam = R(dl);
                sm.chi = R(dc);
            }
        }
        __syncthreads();
    }
    const R lam = (bflags & BLOCK_LAMBDA) ? sm.lam : R(0);
    const int side0 = (int)(strips & 0xffu) - 1, side1 = (int)((strips >> 8) & 0xffu) - 1;
    const int len0 = side0 < 0 ? 0 : (side0 <= 1 ? RY : RX);
    const int len1 = side1 < 0 ? 0 : (side1 <= 1 ? RY : RX);
    auto strip_of = [&](int side) { return side == side0 ? 0 : (side == side1 ? 1 : -1); };

    // ---- phase 0: face strips ----
    {
        const int base = RING <= NT ? RING : 0;
        for (int t = tid - base; t >= 0 && t < len0 + len1; t += NT) {
            const int j = t < len0 ? 0 : 1;
            const int e = j == 0 ? t : t - len0;
            const int side = j == 0 ? side0 : side1;
            int sx, sy;
            strip_node<TX, TY>(side, e, x0, y0, a.nx, a.ny, sx, sy);
            if (sx < 0 || sx >= a.nx || sy < 0 || sy >= a.ny) continue;
            const unsigned inf = a.info[sy * a.pitch + sx];
            if ((inf & INFO_SOLID) || !((inf >> INFO_FACE_SHIFT) & 7u)) continue;
            R g[2][9];
            pull_general(a, sx, sy, inf, lam, g);
            sm.fs_rho[j][e][0] = rho_of(g[0]);
            sm.fs_rho[j][e][1] = rho_of(g[1]);
            const int o = side <= 1 ? sy - y0 : sx - x0;
            const bool own = sx >= x0 && sx < x0 + TX && sy >= y0 && sy < y0 + TY;
            if (own)
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int i = 0; i < 9; ++i) sm.fs_f[j][o][k * 9 + i] = g[k][i];
        }
    }

    // ---- own node ----
    const int x = x0 + tx, y = y0 + ty;
    const bool inb = (x >= 0 && x < a.nx && y >= 0 && y < a.ny);
    info = INFO_SOLID;
    fluid = false;
    int own_strip = -1, own_idx = 0;
    R r0 = R(0), r1 = R(0);
    unsigned char sol = 1;
    if (inb) {
        info = a.info[y * a.pitch + x];
        fluid = !(info & INFO_SOLID);
        if (fluid) {
            const int fid = (int)((info >> INFO_FACE_SHIFT) & 7u);
            if (fid) {
                const int side = a.face[fid - 1].side;
                own_strip = strip_of(side);
                own_idx = side <= 1 ? ty : tx;
            }
            if (own_strip < 0) {
                pull_general(a, x, y, info, lam, f);
                r0 = rho_of(f[0]);
                r1 = rho_of(f[1]);
            }
            sol = 0;
        }
    } else if (site_rho<S, R, 2>(a, x, y, r0, r1, lam)) {
        sol = 0;
    }
    sm.rr[ty + 2][tx + 2] = rpair<R>(r0, r1);
    sm.sol[ty + 2][tx + 2] = sol;

    // ---- halo ring ----
    int def_j = -1, def_e = 0, def_rx = 0, def_ry = 0;
    for (int p = tid; p < RING; p += NT) {
        int rx, ry;
        if (p < 2 * RX) {
            ry = p / RX;
            rx = p % RX;
        } else if (p < 4 * RX) {
            ry = TY + 2 + (p - 2 * RX) / RX;
            rx = (p - 2 * RX) % RX;
        } else {
            const int q = p - 4 * RX;
            ry = 2 + q / 4;
            const int c = q % 4;
            rx = c < 2 ? c : TX + c;
        }
        int gx = x0 - 2 + rx, gy = y0 - 2 + ry;
        R h0 = R(0), h1 = R(0);
        unsigned char hs = 1;
        if (!resolve_site(a, gx, gy)) {
            const unsigned inf = a.info[gy * a.pitch + gx];
            if (!(inf & INFO_SOLID)) {
                hs = 0;
                const int fid = (int)((inf >> INFO_FACE_SHIFT) & 7u);
                int j = -1, e = -1;
                if (fid) {
                    const int side = a.face[fid - 1].side;
                    j = strip_of(side);
                    if (j >= 0) e = strip_entry<TX, TY>(side, gx, gy, x0, y0, a.nx, a.ny);
                }
                if (j >= 0 && e >= 0 && RING <= NT) {
                    def_j = j;  // filled from the strip after the barrier
                    def_e = e;
                    def_rx = rx;
                    def_ry = ry;
                } else {
                    R g[2][9];
                    pull_general(a, gx, gy, inf, lam, g);
                    h0 = rho_of(g[0]);
                    h1 = rho_of(g[1]);
                }
            }
        }
        sm.rr[ry][rx] = rpair<R>(h0, h1);
        sm.sol[ry][rx] = hs;
    }
    __syncthreads();
    if (own_strip >= 0) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int i = 0; i < 9; ++i) f[k][i] = sm.fs_f[own_strip][own_idx][k * 9 + i];
        sm.rr[ty + 2][tx + 2] = rpair<R>(rho_of(f[0]), rho_of(f[1]));
    }
    if (def_j >= 0) {
        sm.rr[def_ry][def_rx] = rpair<R>(sm.fs_rho[def_j][def_e][0], sm.fs_rho[def_j][def_e][1]);
    }
}

// Eq. 1 for both components of one node in moment space (T of Eq. 3, S of
// Eq. 4), delta form: post-collision moment increments -s (m - m_eq) +
// (1 - s/2) F_m, back-transformed with T^-1 = T^T diag(1/9, 1/36, 1/36, 1/6,
// 1/12, 1/6, 1/12, 1/4, 1/4), with both components of an FP32 node in the
// two lanes of each packed FP32x2 instruction (each lane rounds as the
// scalar operation does).
template <typename V>
struct Lanes;
template <>
struct Lanes<float2> {
    static __device__ __forceinline__ float2 c(float v) { return make_float2(v, v); }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, c(-1.f), a); }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 d) { return __ffma2_rn(a, b, d); }
};
// g: populations, r: density, fx, fy: force, s[1..8]: rates; ux, uy common.
template <typename V>
__device__ __forceinline__ void collide_lanes(const V (&g)[9], V r, V fx, V fy, const V (&s)[9], V ux, V uy, V uu3,
                                              V (&o)[9]) {
    using L = Lanes<V>;
    const V d13 = L::sub(g[1], g[3]), d24 = L::sub(g[2], g[4]), d57 = L::sub(g[5], g[7]), d86 = L::sub(g[8], g[6]);
    const V a13 = L::add(g[1], g[3]), a24 = L::add(g[2], g[4]), a57 = L::add(g[5], g[7]), a68 = L::add(g[6], g[8]);
    const V sa = L::add(a13, a24), sd = L::add(a57, a68);
    const V me = L::fma(L::c(-4), g[0], L::sub(L::mul(L::c(2), sd), sa));
    const V mp = L::fma(L::c(4), g[0], L::fma(L::c(-2), sa, sd));
    const V dpn = L::add(d57, d86), dmn = L::sub(d57, d86);
    const V mjx = L::add(d13, dpn), mqx = L::fma(L::c(-2), d13, dpn);
    const V mjy = L::add(d24, dmn), mqy = L::fma(L::c(-2), d24, dmn);
    const V mxx = L::sub(a13, a24), mxy = L::sub(a57, a68);
    const V uF = L::fma(ux, fx, L::mul(uy, fy));
    V h[9], ns[9];
#pragma unroll
    for (int j = 1; j < 9; ++j) {
        h[j] = L::fma(L::c(-0.5), s[j], L::c(1));
        ns[j] = L::mul(L::c(-1), s[j]);
    }
    const V de = L::fma(ns[1], L::sub(me, L::mul(r, L::sub(uu3, L::c(2)))), L::mul(h[1], L::mul(L::c(6), uF)));
    const V dp = L::fma(ns[2], L::sub(mp, L::mul(r, L::sub(L::c(1), uu3))), L::mul(h[2], L::mul(L::c(-6), uF)));
    const V djx = L::fma(ns[3], L::sub(mjx, L::mul(r, ux)), L::mul(h[3], fx));
    const V dqx = L::fma(ns[4], L::add(mqx, L::mul(r, ux)), L::mul(L::mul(L::c(-1), h[4]), fx));
    const V djy = L::fma(ns[5], L::sub(mjy, L::mul(r, uy)), L::mul(h[5], fy));
    const V dqy = L::fma(ns[6], L::add(mqy, L::mul(r, uy)), L::mul(L::mul(L::c(-1), h[6]), fy));
    const V dxx = L::fma(ns[7], L::sub(mxx, L::mul(r, L::sub(L::mul(ux, ux), L::mul(uy, uy)))),
                         L::mul(h[7], L::mul(L::c(2), L::sub(L::mul(ux, fx), L::mul(uy, fy)))));
    const V dxy = L::fma(ns[8], L::sub(mxy, L::mul(L::mul(r, ux), uy)), L::mul(h[8], L::fma(ux, fy, L::mul(uy, fx))));
    const V ce = L::mul(de, L::c(1.0 / 36.0)), cp = L::mul(dp, L::c(1.0 / 36.0));
    const V cjx = L::mul(djx, L::c(1.0 / 6.0)), cqx = L::mul(dqx, L::c(1.0 / 12.0));
    const V cjy = L::mul(djy, L::c(1.0 / 6.0)), cqy = L::mul(dqy, L::c(1.0 / 12.0));
    const V cxx = L::mul(dxx, L::c(0.25)), cxy = L::mul(dxy, L::c(0.25));
    const V ax_ = L::fma(L::c(-2), cp, L::mul(L::c(-1), ce)), dg = L::fma(L::c(2), ce, cp);
    const V bx = L::fma(L::c(-2), cqx, cjx), by = L::fma(L::c(-2), cqy, cjy);
    const V px = L::add(cjx, cqx), py = L::add(cjy, cqy);
    o[0] = L::fma(L::c(4), L::sub(cp, ce), g[0]);
    o[1] = L::add(g[1], L::add(L::add(ax_, bx), cxx));
    o[2] = L::add(g[2], L::sub(L::add(ax_, by), cxx));
    o[3] = L::add(g[3], L::add(L::sub(ax_, bx), cxx));
    o[4] = L::add(g[4], L::sub(L::sub(ax_, by), cxx));
    o[5] = L::add(g[5], L::add(L::add(L::add(dg, px), py), cxy));
    o[6] = L::add(g[6], L::sub(L::add(L::sub(dg, px), py), cxy));
    o[7] = L::add(g[7], L::add(L::sub(L::sub(dg, px), py), cxy));
    o[8] = L::add(g[8], L::sub(L::sub(L::add(dg, px), py), cxy));
}

template <typename A>
__device__ __forceinline__ void collide_pair(const A& a, const float (&f)[2][9], float rho0, float rho1, float ux,
                                             float uy, float Fx0, float Fy0, float Fx1, float Fy1,
                                             float (&o)[2][9]) {
    const float uu3 = 3.f * (ux * ux + uy * uy);
    float2 g[9], s[9], out[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        g[i] = make_float2(f[0][i], f[1][i]);
        s[i] = make_float2(a.s[0][i], a.s[1][i]);
    }
    collide_lanes<float2>(g, make_float2(rho0, rho1), make_float2(Fx0, Fx1), make_float2(Fy0, Fy1), s,
                          make_float2(ux, ux), make_float2(uy, uy), make_float2(uu3, uu3), out);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        o[0][i] = out[i].x;
        o[1][i] = out[i].y;
    }
}

// Eq. 10's sum over the 24 taps, both components: g_k = sum_e w(|e|^2) e
// psi_k(x + e), with rr(dy, dx) the (rho_1, rho_2) pair at offset (dx, dy).
// Opposite taps share the weight, so the sum runs over the half-plane
// before the centre of w e (psi(x + e) - psi(x - e)); in FP32 both
// components share packed FP32x2 FMAs.
template <typename R, typename RR>
__device__ __forceinline__ void psi_gradient(RR rr, R& g0x, R& g0y, R& g1x, R& g1y) {
    if constexpr (std::is_same<R, float>::value) {
        float2 gx = make_float2(0.f, 0.f), gy = make_float2(0.f, 0.f);
#pragma unroll
        for (int dy = -2; dy <= 0; ++dy)
#pragma unroll
            for (int dx = -2; dx <= 2; ++dx) {
                if (dx * dx + dy * dy == 0 || dx * dx + dy * dy > 8 || (dy == 0 && dx > 0)) continue;
                const float w = w8_<float>(dx, dy);
                const float2 d = __ffma2_rn(rr(-dy, -dx), make_float2(-1.f, -1.f), rr(dy, dx));
                if (dx != 0) gx = __ffma2_rn(make_float2(w * dx, w * dx), d, gx);
                if (dy != 0) gy = __ffma2_rn(make_float2(w * dy, w * dy), d, gy);
            }
        g0x = gx.x;
        g1x = gx.y;
        g0y = gy.x;
        g1y = gy.y;
    } else {
        g0x = g0y = g1x = g1y = R(0);
#pragma unroll
        for (int dy = -2; dy <= 0; ++dy)
#pragma unroll
            for (int dx = -2; dx <= 2; ++dx) {
                if (dx * dx + dy * dy == 0 || dx * dx + dy * dy > 8 || (dy == 0 && dx > 0)) continue;
                const R w = w8_<R>(dx, dy);
                const auto pp = rr(dy, dx), mm = rr(-dy, -dx);
                const R d0 = pp.x - mm.x, d1 = pp.y - mm.y;
                if (dx != 0) {
                    g0x += (w * R(dx)) * d0;
                    g1x += (w * R(dx)) * d1;
                }
                if (dy != 0) {
                    g0y += (w * R(dy)) * d0;
                    g1y += (w * R(dy)) * d1;
                }
            }
    }
}

// Adhesion coefficients of Eq. 11 for the two components at a node with
// densities rho0, rho1.  Eq. 12 (wet_interp): one coefficient for both,
// G_w,1 where rho^e = (rho0 - rho1)/(rho0 + rho1) > delta, G_w,2 where
// rho^e < -delta, and the linear pieces G_w,1 rho^e/delta on (0, delta],
// -G_w,2 rho^e/delta on (-delta, 0] between them.
template <typename S, typename R>
__device__ __forceinline__ void adhesion_coeffs(const D2Args<S, R>& a, R rho0, R rho1, R& gw0, R& gw1) {
    gw0 = a.Gw[0];
    gw1 = a.Gw[1];
    if (a.wet_interp) {
        const R re = (rho0 - rho1) / (rho0 + rho1), d = a.wet_delta;
        const R g = re > d ? a.Gw[0] : (re > R(0) ? a.Gw[0] * re / d : (re > -d ? -a.Gw[1] * re / d : a.Gw[1]));
        gw0 = g;
        gw1 = g;
    }
}

// Eq. 11's sum sum_e w(|e|^2) e s(x + e), with sol(dy, dx) the solid
// indicator (1 solid, 0 fluid) at offset (dx, dy).
template <typename R, typename SOL>
__device__ __forceinline__ void adhesion_sum(SOL sol, R& ax, R& ay) {
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
        for (int dx = -2; dx <= 2; ++dx) {
            if (dx * dx + dy * dy == 0 || dx * dx + dy * dy > 8) continue;
            const R sv = R(sol(dy, dx));
            if (dx != 0) ax += (w8_<R>(dx, dy) * R(dx)) * sv;
            if (dy != 0) ay += (w8_<R>(dx, dy) * R(dy)) * sv;
        }
}

// Eq. 1 for one component of one node in moment space (T of Eq. 3, S of
// Eq. 4), delta form: post-collision moment increments -s (m - m_eq) +
// (1 - s/2) F_m with the analytic equilibrium and forcing moments, then the
// back-transform T^-1 = T^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4,
// 1/4) added to the populations.  uu3 = 3 |u|^2.
template <typename R>
__device__ __forceinline__ void collide_scalar(const R* s, R r, R fx, R fy, R ux, R uy, R uu3, const R (&g)[9],
                                               R (&o)[9]) {
    const R d13 = g[1] - g[3], d24 = g[2] - g[4], d57 = g[5] - g[7], d86 = g[8] - g[6];
    const R a13 = g[1] + g[3], a24 = g[2] + g[4], a57 = g[5] + g[7], a68 = g[6] + g[8];
    const R sa = a13 + a24, sd = a57 + a68;
    const R me = (R(2) * sd - sa) - R(4) * g[0];
    const R mp = (sd - R(2) * sa) + R(4) * g[0];
    const R mjx = d13 + (d57 + d86), mqx = (d57 + d86) - R(2) * d13;
    const R mjy = d24 + (d57 - d86), mqy = (d57 - d86) - R(2) * d24;
    const R mxx = a13 - a24, mxy = a57 - a68;
    const R uF = ux * fx + uy * fy;
    const R de = -s[1] * (me - r * (uu3 - R(2))) + (R(1) - R(0.5) * s[1]) * (R(6) * uF);
    const R dp = -s[2] * (mp - r * (R(1) - uu3)) + (R(1) - R(0.5) * s[2]) * (R(-6) * uF);
    const R djx = -s[3] * (mjx - r * ux) + (R(1) - R(0.5) * s[3]) * fx;
    const R dqx = -s[4] * (mqx + r * ux) - (R(1) - R(0.5) * s[4]) * fx;
    const R djy = -s[5] * (mjy - r * uy) + (R(1) - R(0.5) * s[5]) * fy;
    const R dqy = -s[6] * (mqy + r * uy) - (R(1) - R(0.5) * s[6]) * fy;
    const R dxx = -s[7] * (mxx - r * (ux * ux - uy * uy)) + (R(1) - R(0.5) * s[7]) * (R(2) * (ux * fx - uy * fy));
    const R dxy = -s[8] * (mxy - r * ux * uy) + (R(1) - R(0.5) * s[8]) * (ux * fy + uy * fx);
    const R ce = de * R(1.0 / 36.0), cp = dp * R(1.0 / 36.0);
    const R cjx = djx * R(1.0 / 6.0), cqx = dqx * R(1.0 / 12.0);
    const R cjy = djy * R(1.0 / 6.0), cqy = dqy * R(1.0 / 12.0);
    const R cxx = dxx * R(0.25), cxy = dxy * R(0.25);
    const R ax_ = -ce - R(2) * cp, dg = R(2) * ce + cp;
    const R bx = cjx - R(2) * cqx, by = cjy - R(2) * cqy;
    const R px = cjx + cqx, py = cjy + cqy;
    o[0] = g[0] + (R(4) * (cp - ce));
    o[1] = g[1] + (ax_ + bx + cxx);
    o[2] = g[2] + (ax_ + by - cxx);
    o[3] = g[3] + (ax_ - bx + cxx);
    o[4] = g[4] + (ax_ - by - cxx);
    o[5] = g[5] + (dg + px + py + cxy);
    o[6] = g[6] + (dg - px + py - cxy);
    o[7] = g[7] + (dg - px - py + cxy);
    o[8] = g[8] + (dg + px - py - cxy);
}

// One tile of one step.  bxy = bx | by << 16; bflags = BLOCK_* flags; strips
// and slot are used by general tiles only.
template <typename S, typename R, int TX, int TY, bool GEN, bool ROLES = true>
__device__ __forceinline__ void step_tile(const D2Args<S, R>& a, int bxy, unsigned bflags, unsigned strips,
                                          int slot) {
    constexpr int NT = TX * TY, NW = NT / 32;
    using SmemT = typename std::conditional<GEN, TileSmemGen<S, R, TX, TY>, TileSmem<S, R, TX, TY>>::type;
    __shared__ SmemT smx;
    TileSmem<S, R, TX, TY>& sm = smx;

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = (bxy & 0xffff) * TX - a.xoff, y0 = (bxy >> 16) * TY - a.yoff;
    const int x = x0 + tx, y = y0 + ty;

    R f[2][9];
    unsigned info;
    bool fluid;
    if constexpr (GEN && ROLES)
        stage_tile_general<S, R, TX, TY>(a, smx, x0, y0, strips, bflags, f, info, fluid);
    else if constexpr (GEN)
        stage_tile_compact<S, R, TX, TY>(a, smx, x0, y0, tx, ty, strips, bflags, f, info, fluid);
    else if (bflags & BLOCK_EDGE) stage_tile<S, R, TX, TY, 1>(a, sm, x0, y0, tx, ty, f, info, fluid);
    else stage_tile<S, R, TX, TY, 0>(a, sm, x0, y0, tx, ty, f, info, fluid);
    __syncthreads();
    // general tiles: the ring and strip warps are done once the tile is staged
    if (GEN && tid >= NT) return;

    const R rho0 = sm.rr[ty + 2][tx + 2].x, rho1 = sm.rr[ty + 2][tx + 2].y;
    R Fx0 = R(0), Fy0 = R(0), Fx1 = R(0), Fy1 = R(0);
    R ux = R(0), uy = R(0);
    const int own_face = (int)((info >> INFO_FACE_SHIFT) & 7u) - 1;
    const int nbr_face = (int)((info >> INFO_NBR_SHIFT) & 7u) - 1;
    if (fluid) {
        // ---- Eq. 10: 24-point 8th-order gradient of the other component ----
        R g0x, g0y, g1x, g1y;
        psi_gradient<R>([&](int dy, int dx) { return sm.rr[ty + 2 + dy][tx + 2 + dx]; }, g0x, g0y, g1x, g1y);
        // ---- Eq. 11: adhesion, only in tiles that see a solid site ----
        R ax = R(0), ay = R(0);
        if (bflags & BLOCK_SOLID)
            adhesion_sum<R>([&](int dy, int dx) { return sm.sol[ty + 2 + dy][tx + 2 + dx]; }, ax, ay);
        const R rt = rho0 + rho1;
        const R inv_rt = R(1) / rt;
        R gw0, gw1;
        adhesion_coeffs(a, rho0, rho1, gw0, gw1);
        Fx0 = -a.G12 * rho0 * g1x - gw0 * rho0 * ax + a.body[0] * rho0 * inv_rt;
        Fy0 = -a.G12 * rho0 * g1y - gw0 * rho0 * ay + a.body[1] * rho0 * inv_rt;
        Fx1 = -a.G12 * rho1 * g0x - gw1 * rho1 * ax + a.body[0] * rho1 * inv_rt;
        Fy1 = -a.G12 * rho1 * g0y - gw1 * rho1 * ay + a.body[1] * rho1 * inv_rt;
        // ---- Eqs. 7, 8: common velocity ----
        const R jx = (jx_of(f[0]) + R(0.5) * Fx0) + (jx_of(f[1]) + R(0.5) * Fx1);
        const R jy = (jy_of(f[0]) + R(0.5) * Fy0) + (jy_of(f[1]) + R(0.5) * Fy1);
        ux = jx * inv_rt;
        uy = jy * inv_rt;
    }

    // ---- Eq. 22: outlet normal velocity = chi * u_n(x_{N-1}), same row ----
    R un_nbr = R(0);  // normal velocity of x_{N-1}, same row (outlet nodes)
    if (GEN && a.out_face >= 0) {
        const FaceDev& OF = a.face[a.out_face];
        bool covers;
        if (OF.side == 0) covers = (x0 <= 0);
        else if (OF.side == 1) covers = (x0 + TX > a.nx - 1);
        else if (OF.side == 2) covers = (y0 <= 0);
        else covers = (y0 + TY > a.ny - 1);
        if (covers && OF.chi) {
            const int along = (OF.side <= 1) ? ty : tx;
            if (fluid && nbr_face == a.out_face) sm.un[along] = (OF.side <= 1) ? ux : uy;
            tile_sync<GEN, NT>();
            if (fluid && own_face == a.out_face) {
                const R chi = sm.chi;
                un_nbr = sm.un[along];
                if (OF.side <= 1) ux = chi * un_nbr;
                else uy = chi * un_nbr;
            }
        }
    }

    if (fluid) {
        const int n = y * a.pitch + x;
        // open-boundary state for the next step (inlet forces, outlet populations)
        if (GEN && own_face >= 0) {
            const FaceDev& F = a.face[own_face];
            const int slot = F.base + ((F.side <= 1) ? y : x) - F.lo;
            if (F.kind == FACE_INLET) {
                R* Fp = a.Fp_out + slot * 8;
                Fp[0] = Fx0; Fp[1] = Fy0; Fp[2] = Fx1; Fp[3] = Fy1;
            } else {
                // outlet: keep all nine pairs (only the unknown set is read back)
                R* fo = a.fo_out + slot * 18;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    fo[i * 2 + 0] = f[0][i];
                    fo[i * 2 + 1] = f[1][i];
                }
            }
        }
        if (nbr_face >= 0 && a.face[nbr_face].kind == FACE_INLET) {
            const FaceDev& F = a.face[nbr_face];
            R* Fp = a.Fp_out + (F.base + ((F.side <= 1) ? y : x) - F.lo) * 8 + 4;
            Fp[0] = Fx0; Fp[1] = Fy0; Fp[2] = Fx1; Fp[3] = Fy1;
        }
        bool defer = false;
        if constexpr (GEN) {
            if (a.oc_save && own_face >= 0 && own_face == a.out_face && a.face[own_face].chi) {
                // chi from this step's flux sums (Eq. 23 at t + dt): the outlet
                // node's collision waits for them in d2q9_outlet_chi_kernel
                const FaceDev& F = a.face[own_face];
                R* q = a.oc_save + (size_t)(F.base + ((F.side <= 1) ? y : x) - F.lo) * OC_STRIDE;
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int i = 0; i < 9; ++i) q[k * 9 + i] = f[k][i];
                q[18] = rho0;
                q[19] = rho1;
                q[20] = Fx0;
                q[21] = Fy0;
                q[22] = Fx1;
                q[23] = Fy1;
                q[24] = (F.side <= 1) ? uy : ux;  // tangential velocity
                q[25] = un_nbr;
                q[26] = R(1);                     // written this step
                defer = true;
            }
        }
        if (a.macro && !defer) {
            a.macro[n] = rho0;
            a.macro[a.plane + n] = rho1;
            a.macro[2 * a.plane + n] = ux;
            a.macro[3 * a.plane + n] = uy;
        }
        // ---- Eq. 1 in moment space (T of Eq. 3, S of Eq. 4), delta form ----
        // General tiles (latency-bound) run both components through packed
        // FP32x2 operations; fast tiles (issue- and HBM-bound) measured faster
        // with the scalar form.
        if (defer) {
            // collided by d2q9_outlet_chi_kernel
        } else if constexpr (GEN && std::is_same<R, float>::value) {
            R o2[2][9];
            collide_pair(a, f, rho0, rho1, ux, uy, Fx0, Fy0, Fx1, Fy1, o2);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const R r = k == 0 ? rho0 : rho1;
                if constexpr (is_half_<S>()) {
                    // encode with the reference density of the node that pulls each value
                    const R own = half_round(r);
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const R dref = ((info >> opp_(i)) & 1u) ? own
                                                               : half_round(k ? sm.rr[ty + 2 + ey_(i)][tx + 2 + ex_(i)].y : sm.rr[ty + 2 + ey_(i)][tx + 2 + ex_(i)].x);
                        Pop<S, R>::st(a.fout, (k * 9 + i) * a.plane + n, o2[k][i], w_<R>(i) * dref);
                    }
                    static_cast<__half*>(a.rref_out)[k * a.plane + n] = __float2half_rn(float(r));
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) Pop<S, R>::st(a.fout, (k * 9 + i) * a.plane + n, o2[k][i], R(0));
                }
            }
        } else {
            const R uu3 = R(3) * (ux * ux + uy * uy);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const R* s = a.s[k];
                const R r = k == 0 ? rho0 : rho1;
                const R fx = k == 0 ? Fx0 : Fx1, fy = k == 0 ? Fy0 : Fy1;
                R o[9];
                collide_scalar<R>(s, r, fx, fy, ux, uy, uu3, f[k], o);
                if constexpr (is_half_<S>()) {
                    // encode with the reference density of the node that pulls each value
                    const R own = half_round(r);
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const R dref = ((info >> opp_(i)) & 1u) ? own
                                                               : half_round(k ? sm.rr[ty + 2 + ey_(i)][tx + 2 + ex_(i)].y : sm.rr[ty + 2 + ey_(i)][tx + 2 + ex_(i)].x);
                        Pop<S, R>::st(a.fout, (k * 9 + i) * a.plane + n, o[i], w_<R>(i) * dref);
                    }
                    static_cast<__half*>(a.rref_out)[k * a.plane + n] = __float2half_rn(float(r));
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) Pop<S, R>::st(a.fout, (k * 9 + i) * a.plane + n, o[i], R(0));
                }
            }
        }
    }

    // ---- divergence flag: one atomic per warp at most ----
    {
        const bool bad = fluid && !isfinite(rho0 + rho1 + ux + uy);
        const unsigned m = __ballot_sync(0xffffffffu, bad);
        if (m && (tid & 31) == 0) atomicOr(a.status, 1u);
    }

    // ---- FP64 flux reductions for lambda (Eq. 21) and chi (Eq. 23) ----
    // Few nodes of a tile contribute (its inlet nodes and the outlet's inward
    // neighbours): each writes its FP64 terms to a slot ranked by lane within
    // its warp, then four threads sum one term each over warps and slots in a
    // fixed order (deterministic, no FP64 shuffle tree).
    if constexpr (GEN) {
        if (a.nslots > 0 && slot >= 0) {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            bool has = false;
            if (fluid && own_face >= 0 && a.face[own_face].kind == FACE_INLET) {
                const FaceDev& F = a.face[own_face];
                v[0] = (double)(rho0 + rho1) * (double)(-(R(F.ox) * ux + R(F.oy) * uy));
                has = true;
            }
            if (fluid && nbr_face >= 0 && nbr_face == a.out_face) {
                const FaceDev& F = a.face[nbr_face];
                const double un = (double)(R(F.ox) * ux + R(F.oy) * uy);
                v[1] = (double)(rho0 + rho1) * un;
                v[2] = un;
                v[3] = 1.0;
                has = true;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, has);
            const int lane = tid & 31, wq = tid >> 5;
            if (has) {
                const int rk = __popc(bal & ((1u << lane) - 1u));
#pragma unroll
                for (int j = 0; j < 4; ++j) smx.fl[wq][rk][j] = v[j];
            }
            if (lane == 0) smx.fcnt[wq] = __popc(bal);
            tile_sync<GEN, NT>();
            if (tid < 4) {
                // plain stores: the next step's outlet tiles read them after the
                // kernel boundary, so no fence or atomic is needed
                double acc = 0.0;
                for (int wgrp = 0; wgrp < NW; ++wgrp)
                    for (int r = 0; r < smx.fcnt[wgrp]; ++r) acc += smx.fl[wgrp][r][tid];
                a.part_out[slot * 4 + tid] = acc;
                if (tid == 0) a.scal_out[5] = 1.0;
            }
        }
    }
}

// Register cap of a general tile, within the 64 K register file for every
// variant.  FP32 keeps 80 (measured on GB300: a 64-register cap spilled
// ~0.5 KB per thread and made the step 20 % slower, although it would leave
// room for a fifth fast tile on the SM).
template <int TX, int TY, bool ROLES>
__host__ __device__ constexpr int gen_threads() {
    return ROLES ? GenRoles<TX, TY>::THREADS : TX * TY;
}

// The warps of a CTA are spread over the SM's four sub-partitions, each with
// 16 K registers, so the cap must let ceil(warps / 4) warps fit in 16 K (a
// cap checked against the whole 64 K file alone can leave a block that does
// not launch: 17 warps at 120 registers need 19,200 in one sub-partition).
template <typename R, int TX, int TY, bool ROLES>
__host__ __device__ constexpr int gen_maxreg() {
    constexpr int warps = (gen_threads<TX, TY, ROLES>() + 31) / 32;
    constexpr int fit = 16384 / (((warps + 3) / 4) * 32) / 8 * 8;
    constexpr int want = sizeof(R) == 4 ? 80 : 128;
    return want < fit ? want : fit;
}

}  // namespace
}  // namespace lbm
