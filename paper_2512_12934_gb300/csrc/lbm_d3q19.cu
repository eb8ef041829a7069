// D3Q19 two-component MRT pseudopotential step with the corrected open faces
// (the three-dimensional counterpart of lbm_d2q9.cu).
//
// One time step is three launches on the context's stream:
//   A  d3q_pull_kernel    pull streaming (Eq. 2) with halfway bounce-back
//                         (Eq. B1) and periodic wrap (Eq. B2); inlet
//                         reconstruction (Eq. 13 over the 5 unknowns, alpha
//                         correction Eqs. 15-19); convective outlet (Eq. 20);
//                         component densities rho_k (= psi_k) to a field.
//   B  d3q_collide_kernel rho and the solid indicator of a 32x4x2 tile plus a
//                         2-node halo (ghost mirrors of Eqs. 24-25) staged in
//                         shared memory; forces of Eqs. 10-11 on the 92-vector
//                         8th-order isotropic stencil; common velocity
//                         (Eqs. 7-8) with the outlet rescaled by chi (Eq. 22);
//                         MRT collision with forcing (Eqs. 1, 3-6, 9) with the
//                         19x19 transforms unrolled over compile-time
//                         constants; per-face-node FP64 flux terms.
//   C  d3q_reduce_kernel  fixed-order FP64 sums of the flux terms: lambda
//                         (Eq. 21) and chi (Eq. 23) for the next step.
// Face nodes carry their post-boundary populations from A to B, the outlet's
// previous post-boundary populations (Eq. 20) and the forces the inlet needs
// one step later in small slot-indexed arrays.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm_d3q19.h"

namespace lbm3 {

// ---- lattice (velocity order: rest, +-x, +-y, +-z, the xy, xz, yz edges) ----
__host__ __device__ constexpr int ex_(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                 : 0;
}
__host__ __device__ constexpr int ey_(int i) {
    return (i == 3 || i == 7 || i == 8 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 9 || i == 10 || i == 16 || i == 18) ? -1
                                                                 : 0;
}
__host__ __device__ constexpr int ez_(int i) {
    return (i == 5 || i == 11 || i == 12 || i == 15 || i == 16) ? 1
           : (i == 6 || i == 13 || i == 14 || i == 17 || i == 18) ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int e2_(int i) { return ex_(i) * ex_(i) + ey_(i) * ey_(i) + ez_(i) * ez_(i); }
__host__ __device__ constexpr int opp_(int i) {
    for (int j = 0; j < Q; ++j)
        if (ex_(j) == -ex_(i) && ey_(j) == -ey_(i) && ez_(j) == -ez_(i)) return j;
    return 0;
}
// weights times 36
__host__ __device__ constexpr int w36_(int i) { return e2_(i) == 0 ? 12 : (e2_(i) == 1 ? 2 : 1); }

// Orthogonal moment basis: rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx,
// 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z.
__host__ __device__ constexpr int T_(int r, int i) {
    const int x = ex_(i), y = ey_(i), z = ez_(i), e2 = e2_(i);
    switch (r) {
    case 0: return 1;
    case 1: return 19 * e2 - 30;
    case 2: return (21 * e2 * e2 - 53 * e2 + 24) / 2;
    case 3: return x;
    case 4: return (5 * e2 - 9) * x;
    case 5: return y;
    case 6: return (5 * e2 - 9) * y;
    case 7: return z;
    case 8: return (5 * e2 - 9) * z;
    case 9: return 3 * x * x - e2;
    case 10: return (3 * e2 - 5) * (3 * x * x - e2);
    case 11: return y * y - z * z;
    case 12: return (3 * e2 - 5) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
    }
}
__host__ __device__ constexpr int Tnorm_(int r) {
    int s = 0;
    for (int i = 0; i < Q; ++i) s += T_(r, i) * T_(r, i);
    return s;
}

// 8th-order isotropic stencil weights (second moment 1) by |e|^2, times 5040
__host__ __device__ constexpr int sw5040_(int r2) {
    return r2 == 1 ? 448 : r2 == 2 ? 240 : r2 == 3 ? 96 : r2 == 4 ? 50 : r2 == 5 ? 16 : r2 == 6 ? 8 : r2 == 8 ? 1 : 0;
}

// ---- tiles of the collide kernel -----------------------------------------
constexpr int TX = 32, TY = 4, TZ = 2;
constexpr int HX = TX + 4, HY = TY + 4, HZ = TZ + 4;
constexpr int HN = HX * HY * HZ;

template <typename S>
struct Store;
template <>
struct Store<float> {
    using R = float;
};
template <>
struct Store<double> {
    using R = double;
};

// Wrap a pull source on periodic axes (blocked sources never reach here).
__device__ __forceinline__ int wrap(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

template <typename S>
__device__ __forceinline__ long long node_index(const D3Args<S>& a, int x, int y, int z) {
    return ((long long)z * a.ny + y) * a.pitch + x;
}

// Pull the 19 populations of component k at (x, y, z) (Eq. 2, Eq. B1, Eq. B2).
template <typename S, typename R>
__device__ __forceinline__ void pull(const D3Args<S>& a, int k, int x, int y, int z, uint32_t info, R (&f)[Q]) {
    const S* __restrict__ fin = a.fin + (size_t)k * Q * a.plane;
    const long long n = node_index(a, x, y, z);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (info & (1u << i)) {
            f[i] = (R)fin[(size_t)opp_(i) * a.plane + n];
        } else {
            const int xs = wrap(x - ex_(i), a.nx), ys = wrap(y - ey_(i), a.ny), zs = wrap(z - ez_(i), a.nz);
            f[i] = (R)fin[(size_t)i * a.plane + node_index(a, xs, ys, zs)];
        }
    }
}

template <typename R>
__device__ __forceinline__ void feq(R rho, R ux, R uy, R uz, R (&out)[Q]) {
    const R uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R eu = (R)ex_(i) * ux + (R)ey_(i) * uy + (R)ez_(i) * uz;
        out[i] = rho * ((R)w36_(i) / (R)36) * ((R)1 + (R)3 * eu + (R)4.5 * eu * eu - (R)1.5 * uu);
    }
}

// Density as the rest population plus the sums of opposite pairs.
template <typename R>
__device__ __forceinline__ R sum19(const R (&f)[Q]) {
    R s = f[0];
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (opp_(i) > i) s += f[i] + f[opp_(i)];
    return s;
}

// Momentum as sums of opposite-pair differences (each difference of two
// nearby populations is exact or nearly so, which keeps FP32 j accurate).
template <typename R>
__device__ __forceinline__ void moments_j(const R (&f)[Q], R& jx, R& jy, R& jz) {
    R x = 0, y = 0, z = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int o = opp_(i);
        if (o < i) continue;
        const R d = f[i] - f[o];
        if (ex_(i)) x += (R)ex_(i) * d;
        if (ey_(i)) y += (R)ey_(i) * d;
        if (ez_(i)) z += (R)ez_(i) * d;
    }
    jx = x;
    jy = y;
    jz = z;
}

// Eq. 1 for one component: f <- f - T^-1 S T (f - feq) + T^-1 (I - S/2) T Fbar
template <typename R>
__device__ __forceinline__ void collide(R (&f)[Q], R rho, R ux, R uy, R uz, R Fx, R Fy, R Fz, const R* s) {
    R d[Q], fb[Q];
    feq(rho, ux, uy, uz, d);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        d[i] = f[i] - d[i];
        const R ex = (R)ex_(i), ey = (R)ey_(i), ez = (R)ez_(i);
        const R eu = ex * ux + ey * uy + ez * uz;
        const R ax = (R)3 * (ex - ux) + (R)9 * eu * ex;
        const R ay = (R)3 * (ey - uy) + (R)9 * eu * ey;
        const R az = (R)3 * (ez - uz) + (R)9 * eu * ez;
        fb[i] = ((R)w36_(i) / (R)36) * (ax * Fx + ay * Fy + az * Fz);
    }
    R g[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) {
        R m = 0, mf = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int t = T_(r, i);
            if (t != 0) {
                m += (R)t * d[i];
                mf += (R)t * fb[i];
            }
        }
        g[r] = (-s[r] * m + ((R)1 - (R)0.5 * s[r]) * mf) / (R)Tnorm_(r);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        R acc = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            const int t = T_(r, i);
            if (t != 0) acc += (R)t * g[r];
        }
        f[i] += acc;
    }
}

// ---- kernel A: pull, open faces, densities --------------------------------
template <typename S>
__device__ void face_reconstruct(const D3Args<S>& a, int fid, int x, int y, int z, uint32_t info,
                                 typename Store<S>::R (&f)[2][Q]) {
    using R = typename Store<S>::R;
    const FaceDev3& F = a.face[fid];
    const int ox = F.o[0], oy = F.o[1], oz = F.o[2];
    const int slot = face_slot(F, x, y, z);
    const int x2 = x - ox, y2 = y - oy, z2 = z - oz;
    const uint32_t info2 = a.info[node_index(a, x2, y2, z2)];
    if (F.kind == FACE3_INLET) {
        R f2[2][Q];
        pull<S, R>(a, 0, x2, y2, z2, info2, f2[0]);
        pull<S, R>(a, 1, x2, y2, z2, info2, f2[1]);
        const R* Fp2 = a.FpN + (size_t)slot * 6;
        const R* Fp1 = a.FpF + (size_t)slot * 6;
        R r2[2], jx = 0, jy = 0, jz = 0;
        #pragma unroll
        for (int k = 0; k < 2; ++k) {
            r2[k] = sum19(f2[k]);
            R x_, y_, z_;
            moments_j(f2[k], x_, y_, z_);
            jx += x_ + (R)0.5 * Fp2[k * 3 + 0];
            jy += y_ + (R)0.5 * Fp2[k * 3 + 1];
            jz += z_ + (R)0.5 * Fp2[k * 3 + 2];
        }
        const R rt2 = r2[0] + r2[1];
        const R u2x = jx / rt2, u2y = jy / rt2, u2z = jz / rt2;
        const R speed = (R)a.face_speed[slot];
        const R uin[3] = {-(R)ox * speed, -(R)oy * speed, -(R)oz * speed};
        #pragma unroll
        for (int k = 0; k < 2; ++k) {
            const R rin = (R)a.face_rho[(size_t)k * a.nface_slots + slot];
            R e1[Q], e2[Q];
            feq(rin, uin[0], uin[1], uin[2], e1);
            feq(r2[k], u2x, u2y, u2z, e2);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (ex_(i) * ox + ey_(i) * oy + ez_(i) * oz < 0) f[k][i] = e1[i] + (f2[k][i] - e2[i]);
            if (F.alpha) {
                R mx, my, mz;
                moments_j(f[k], mx, my, mz);
                const R dx = rin * uin[0] - (mx + (R)0.5 * Fp1[k * 3 + 0]);
                const R dy = rin * uin[1] - (my + (R)0.5 * Fp1[k * 3 + 1]);
                const R dz = rin * uin[2] - (mz + (R)0.5 * Fp1[k * 3 + 2]);
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if (ex_(i) * ox + ey_(i) * oy + ez_(i) * oz < 0)
                        f[k][i] += ((R)w36_(i) / (R)36) *
                                   ((R)ex_(i) * dx / (R)F.sa[0] + (R)ey_(i) * dy / (R)F.sa[1] +
                                    (R)ez_(i) * dz / (R)F.sa[2]);
            }
        }
    } else {
        // convective outlet (Eq. 20) with lambda of the previous step
        R fN1[2][Q];
        pull<S, R>(a, 0, x2, y2, z2, info2, fN1[0]);
        pull<S, R>(a, 1, x2, y2, z2, info2, fN1[1]);
        const R lam = (R)a.scal_in[SC3_LAMBDA];
        R* fo = a.fo + (size_t)slot * 2 * Q;
        #pragma unroll
        for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (ex_(i) * ox + ey_(i) * oy + ez_(i) * oz < 0)
                    f[k][i] = (fo[k * Q + i] + lam * fN1[k][i]) / ((R)1 + lam);
        }
        #pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int i = 0; i < Q; ++i) fo[k * Q + i] = f[k][i];
    }
    R* ff = a.fface + (size_t)slot * 2 * Q;
    #pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int i = 0; i < Q; ++i) ff[k * Q + i] = f[k][i];
}

template <typename S>
__global__ void __launch_bounds__(256) d3q_pull_kernel(D3Args<S> a) {
    using R = typename Store<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= a.nx || y >= a.ny || z >= a.nz) return;
    const long long n = node_index(a, x, y, z);
    const uint32_t info = a.info[n];
    if (info & INFO3_SOLID) {
        a.rho[n] = (R)0;
        a.rho[a.plane + n] = (R)0;
        return;
    }
    if ((info >> INFO3_FACE_SHIFT) & 7u) return;  // open-face nodes: d3q_face_pull_kernel
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        R f[Q];
        pull<S, R>(a, k, x, y, z, info, f);
        a.rho[(size_t)k * a.plane + n] = sum19(f);
    }
}

// Face slot -> face index and node coordinates; false for solid positions.
template <typename S>
__device__ __forceinline__ bool slot_node(const D3Args<S>& a, int slot, int& fid, int (&c)[3]) {
    if (slot >= a.nface_slots || !a.face_fluid[slot]) return false;
    fid = 0;
    while (fid + 1 < a.nfaces && slot >= a.face[fid + 1].base) ++fid;
    const FaceDev3& F = a.face[fid];
    const int q = slot - F.base;
    const int ext[3] = {a.nx, a.ny, a.nz};
    c[F.axis] = (F.side & 1) ? ext[F.axis] - 1 : 0;
    c[F.a0] = F.lo0 + q % F.len0;
    c[F.a1] = F.lo1 + q / F.len0;
    return true;
}

// One thread per face slot: pull, open-face reconstruction, densities.
template <typename S>
__global__ void __launch_bounds__(128) d3q_face_pull_kernel(D3Args<S> a) {
    using R = typename Store<S>::R;
    int fid, c[3];
    if (!slot_node(a, blockIdx.x * blockDim.x + threadIdx.x, fid, c)) return;
    const long long n = node_index(a, c[0], c[1], c[2]);
    const uint32_t info = a.info[n];
    R f[2][Q];
    pull<S, R>(a, 0, c[0], c[1], c[2], info, f[0]);
    pull<S, R>(a, 1, c[0], c[1], c[2], info, f[1]);
    face_reconstruct<S>(a, fid, c[0], c[1], c[2], info, f);
    a.rho[n] = sum19(f[0]);
    a.rho[a.plane + n] = sum19(f[1]);
}

// ---- kernel B: forces, velocity, collision --------------------------------
// Resolve a psi / indicator site (Eqs. 10, 11, 24, 25): -1 = solid.
template <typename S>
__device__ __forceinline__ long long psi_site(const D3Args<S>& a, int x, int y, int z) {
    int c[3] = {x, y, z};
    const int ext[3] = {a.nx, a.ny, a.nz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (c[ax] >= 0 && c[ax] < ext[ax]) continue;
        if (a.periodic[ax]) c[ax] = c[ax] < 0 ? c[ax] + ext[ax] : c[ax] - ext[ax];
        else if (c[ax] < 0 && a.open_side[2 * ax]) c[ax] = -1 - c[ax];
        else if (c[ax] >= ext[ax] && a.open_side[2 * ax + 1]) c[ax] = 2 * ext[ax] - 1 - c[ax];
        else return -1;
    }
    const long long n = node_index(a, c[0], c[1], c[2]);
    return (a.info[n] & INFO3_SOLID) ? -1 : n;
}

// Interaction sums over the 92-vector stencil: g_k = sum w psi_k(x+e) e,
// ad = sum w s(x+e) e.  `site(dx, dy, dz, r1, r2, sol)` supplies a site.
template <typename R, typename Site>
__device__ __forceinline__ void stencil_sums(Site site, bool adhesion, R (&g1)[3], R (&g2)[3], R (&ad)[3]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) g1[q] = g2[q] = ad[q] = (R)0;
#pragma unroll
    for (int dz = -2; dz <= 2; ++dz)
#pragma unroll
        for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
            for (int dx = -2; dx <= 2; ++dx) {
                const int r2 = dx * dx + dy * dy + dz * dz;
                const int wq = sw5040_(r2);
                if (r2 == 0 || wq == 0) continue;
                const R w = (R)wq / (R)5040;
                R r1, rr2, sol;
                site(dx, dy, dz, r1, rr2, sol);
                if (dx) {
                    g1[0] += (w * (R)dx) * r1;
                    g2[0] += (w * (R)dx) * rr2;
                }
                if (dy) {
                    g1[1] += (w * (R)dy) * r1;
                    g2[1] += (w * (R)dy) * rr2;
                }
                if (dz) {
                    g1[2] += (w * (R)dz) * r1;
                    g2[2] += (w * (R)dz) * rr2;
                }
                if (adhesion) {
                    if (dx) ad[0] += (w * (R)dx) * sol;
                    if (dy) ad[1] += (w * (R)dy) * sol;
                    if (dz) ad[2] += (w * (R)dz) * sol;
                }
            }
}

template <typename R>
__device__ __forceinline__ void forces(const R* G, R r1, R r2, const R (&g1)[3], const R (&g2)[3], const R (&ad)[3],
                                       const R* body, R (&F1)[3], R (&F2)[3]) {
    // G = {G12, Gw1, Gw2}
    const R rt = r1 + r2;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        F1[q] = -G[0] * r1 * g2[q] - G[1] * r1 * ad[q] + body[q] * r1 / rt;
        F2[q] = -G[0] * r2 * g1[q] - G[2] * r2 * ad[q] + body[q] * r2 / rt;
    }
}

// Force and common velocity of a node from the global density field (used
// by outlet nodes for the chi rescaling, Eq. 22).
template <typename S>
__device__ void node_u_global(const D3Args<S>& a, int x, int y, int z, typename Store<S>::R (&u)[3],
                              typename Store<S>::R& rt_out) {
    using R = typename Store<S>::R;
    const long long n = node_index(a, x, y, z);
    const uint32_t info = a.info[n];
    auto site = [&](int dx, int dy, int dz, R& r1, R& r2, R& sol) {
        const long long m = psi_site(a, x + dx, y + dy, z + dz);
        if (m < 0) {
            r1 = r2 = (R)0;
            sol = (R)1;
        } else {
            r1 = a.rho[m];
            r2 = a.rho[a.plane + m];
            sol = (R)0;
        }
    };
    R g1[3], g2[3], ad[3];
    stencil_sums<R>(site, (info & INFO3_NEAR_SOLID) != 0, g1, g2, ad);
    const R r1 = a.rho[n], r2 = a.rho[a.plane + n];
    R F1[3], F2[3];
    forces<R>(a.G, r1, r2, g1, g2, ad, a.body, F1, F2);
    R f[Q], j[3] = {0, 0, 0};
    #pragma unroll
    for (int k = 0; k < 2; ++k) {
        pull<S, R>(a, k, x, y, z, info, f);
        R jx, jy, jz;
        moments_j(f, jx, jy, jz);
        j[0] += jx;
        j[1] += jy;
        j[2] += jz;
    }
    const R rt = r1 + r2;
    u[0] = (j[0] + (R)0.5 * (F1[0] + F2[0])) / rt;
    u[1] = (j[1] + (R)0.5 * (F1[1] + F2[1])) / rt;
    u[2] = (j[2] + (R)0.5 * (F1[2] + F2[2])) / rt;
    rt_out = rt;
}

// Velocity, collision and store of one node whose populations f and forces
// are known (shared by the interior and the face kernels).
template <typename S>
__device__ __forceinline__ void finish_node(const D3Args<S>& a, long long n, typename Store<S>::R (&f)[2][Q],
                                            typename Store<S>::R r1, typename Store<S>::R r2,
                                            const typename Store<S>::R (&F1)[3], const typename Store<S>::R (&F2)[3],
                                            typename Store<S>::R (&u)[3]) {
    using R = typename Store<S>::R;
    if (!(isfinite((double)(r1 + r2)) && isfinite((double)u[0]) && isfinite((double)u[1]) &&
          isfinite((double)u[2])))
        atomicOr(a.status, 1u);
    if (a.umac) {
        a.umac[n] = u[0];
        a.umac[a.plane + n] = u[1];
        a.umac[2 * a.plane + n] = u[2];
    }
    collide<R>(f[0], r1, u[0], u[1], u[2], F1[0], F1[1], F1[2], a.s[0]);
#pragma unroll
    for (int i = 0; i < Q; ++i) a.fout[(size_t)i * a.plane + n] = (S)f[0][i];
    collide<R>(f[1], r2, u[0], u[1], u[2], F2[0], F2[1], F2[2], a.s[1]);
#pragma unroll
    for (int i = 0; i < Q; ++i) a.fout[(size_t)(Q + i) * a.plane + n] = (S)f[1][i];
}

template <typename R>
__device__ __forceinline__ void common_u(const R (&f)[2][Q], R r1, R r2, const R (&F1)[3], const R (&F2)[3],
                                         R (&u)[3]) {
    R j[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        R jx, jy, jz;
        moments_j(f[k], jx, jy, jz);
        j[0] += jx;
        j[1] += jy;
        j[2] += jz;
    }
    const R rt = r1 + r2;
#pragma unroll
    for (int q = 0; q < 3; ++q) u[q] = (j[q] + (R)0.5 * (F1[q] + F2[q])) / rt;
}

template <typename S>
__global__ void __launch_bounds__(256) d3q_collide_kernel(D3Args<S> a) {
    using R = typename Store<S>::R;
    __shared__ R s_r1[HN];
    __shared__ R s_r2[HN];
    __shared__ unsigned char s_sol[HN];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
    for (int q = tid; q < HN; q += TX * TY * TZ) {
        const int hx = q % HX, hy = (q / HX) % HY, hz = q / (HX * HY);
        const long long m = psi_site(a, x0 - 2 + hx, y0 - 2 + hy, z0 - 2 + hz);
        if (m < 0) {
            s_r1[q] = (R)0;
            s_r2[q] = (R)0;
            s_sol[q] = 1;
        } else {
            s_r1[q] = a.rho[m];
            s_r2[q] = a.rho[a.plane + m];
            s_sol[q] = 0;
        }
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    if (x >= a.nx || y >= a.ny || z >= a.nz) return;
    const long long n = node_index(a, x, y, z);
    const uint32_t info = a.info[n];
    if (info & INFO3_SOLID) return;
    if ((info >> INFO3_FACE_SHIFT) & 7u) return;  // open-face nodes: d3q_face_collide_kernel
    const int hc = (threadIdx.x + 2) + HX * ((threadIdx.y + 2) + HY * (threadIdx.z + 2));
    auto site = [&](int dx, int dy, int dz, R& r1, R& r2, R& sol) {
        const int h = hc + dx + HX * (dy + HY * dz);
        r1 = s_r1[h];
        r2 = s_r2[h];
        sol = (R)s_sol[h];
    };
    R g1[3], g2[3], ad[3];
    stencil_sums<R>(site, (info & INFO3_NEAR_SOLID) != 0, g1, g2, ad);
    const R r1 = s_r1[hc], r2 = s_r2[hc];
    R F1[3], F2[3];
    forces<R>(a.G, r1, r2, g1, g2, ad, a.body, F1, F2);
    const int nid = (int)((info >> INFO3_NBR_SHIFT) & 7u);
    if (nid != 0) {  // force the inlet reconstruction of the next step uses (Eq. 13)
        const FaceDev3& Fc = a.face[nid - 1];
        R* Fp = a.FpN + (size_t)face_slot(Fc, x + Fc.o[0], y + Fc.o[1], z + Fc.o[2]) * 6;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            Fp[q] = F1[q];
            Fp[3 + q] = F2[q];
        }
    }
    R f[2][Q];
    pull<S, R>(a, 0, x, y, z, info, f[0]);
    pull<S, R>(a, 1, x, y, z, info, f[1]);
    R u[3];
    common_u(f, r1, r2, F1, F2, u);
    finish_node<S>(a, n, f, r1, r2, F1, F2, u);
}

// One thread per face slot: forces from the global density field, chi at the
// outlet (Eq. 22), flux terms, the collision.
template <typename S>
__global__ void __launch_bounds__(128) d3q_face_collide_kernel(D3Args<S> a) {
    using R = typename Store<S>::R;
    int fid, c[3];
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (!slot_node(a, slot, fid, c)) return;
    const FaceDev3& Fc = a.face[fid];
    const int x = c[0], y = c[1], z = c[2];
    const long long n = node_index(a, x, y, z);
    const uint32_t info = a.info[n];
    auto site = [&](int dx, int dy, int dz, R& r1, R& r2, R& sol) {
        const long long m = psi_site(a, x + dx, y + dy, z + dz);
        if (m < 0) {
            r1 = r2 = (R)0;
            sol = (R)1;
        } else {
            r1 = a.rho[m];
            r2 = a.rho[a.plane + m];
            sol = (R)0;
        }
    };
    R g1[3], g2[3], ad[3];
    stencil_sums<R>(site, (info & INFO3_NEAR_SOLID) != 0, g1, g2, ad);
    const R r1 = a.rho[n], r2 = a.rho[a.plane + n];
    R F1[3], F2[3];
    forces<R>(a.G, r1, r2, g1, g2, ad, a.body, F1, F2);
    R f[2][Q];
    const R* ff = a.fface + (size_t)slot * 2 * Q;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        f[0][i] = ff[i];
        f[1][i] = ff[Q + i];
    }
    R u[3];
    common_u(f, r1, r2, F1, F2, u);
    const int ax = Fc.axis;
    const double sgn = (double)(Fc.o[0] + Fc.o[1] + Fc.o[2]);  // +1 on a far side, -1 on a near side
    if (Fc.kind == FACE3_OUTLET) {
        R un[3], rtn;
        node_u_global<S>(a, x - Fc.o[0], y - Fc.o[1], z - Fc.o[2], un, rtn);
        a.flux[(size_t)slot * 2 + 0] = (double)rtn * sgn * (double)un[ax];
        a.flux[(size_t)slot * 2 + 1] = sgn * (double)un[ax];
        if (Fc.chi) u[ax] = (R)a.scal_in[SC3_CHI] * un[ax];
    } else {
        a.flux[(size_t)slot * 2 + 0] = (double)(r1 + r2) * (-sgn) * (double)u[ax];
        a.flux[(size_t)slot * 2 + 1] = 0.0;
    }
    R* Fp = a.FpF + (size_t)slot * 6;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        Fp[q] = F1[q];
        Fp[3 + q] = F2[q];
    }
    finish_node<S>(a, n, f, r1, r2, F1, F2, u);
}

// ---- kernel C: lambda and chi from the face flux terms (fixed order) -------
template <typename S>
__global__ void __launch_bounds__(256) d3q_reduce_kernel(D3Args<S> a) {
    __shared__ double s_in[256], s_out[256], s_u[256];
    double qin = 0.0, qout = 0.0, us = 0.0;
    for (int f = 0; f < a.nfaces; ++f) {
        const FaceDev3& F = a.face[f];
        for (int q = threadIdx.x; q < F.count; q += 256) {
            const int slot = F.base + q;
            if (!a.face_fluid[slot]) continue;
            if (F.kind == FACE3_INLET) qin += a.flux[(size_t)slot * 2];
            else {
                qout += a.flux[(size_t)slot * 2];
                us += a.flux[(size_t)slot * 2 + 1];
            }
        }
    }
    s_in[threadIdx.x] = qin;
    s_out[threadIdx.x] = qout;
    s_u[threadIdx.x] = us;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s_in[threadIdx.x] += s_in[threadIdx.x + w];
            s_out[threadIdx.x] += s_out[threadIdx.x + w];
            s_u[threadIdx.x] += s_u[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* sc = a.scal_out;
        const double Qi = s_in[0], Qo = s_out[0];
        sc[SC3_QIN] = Qi;
        sc[SC3_QOUT] = Qo;
        if (a.out_count > 0) {
            const double lam = s_u[0] / (double)a.out_count;
            sc[SC3_UMEAN] = lam;
            sc[SC3_LAMBDA] = lam > 0.0 ? lam : 0.0;
            sc[SC3_CHI] = (!a.have_inlet || fabs(Qo) < 1e-14) ? 1.0 : Qi / Qo;
        } else {
            sc[SC3_UMEAN] = a.scal_in[SC3_UMEAN];
            sc[SC3_LAMBDA] = a.scal_in[SC3_LAMBDA];
            sc[SC3_CHI] = a.scal_in[SC3_CHI];
        }
    }
}

// ---- diagnostics: FP64 masses over fluid nodes and the largest |u|^2 ------
template <typename S>
__global__ void __launch_bounds__(256) d3q_mass_kernel(const S* __restrict__ f, const uint32_t* __restrict__ info,
                                                       const S* __restrict__ umac, int nx, int ny, int nz,
                                                       int pitch, long long plane, double* __restrict__ partial) {
    __shared__ double s0[256], s1[256], s2[256];
    double m0 = 0.0, m1 = 0.0, u2 = 0.0;
    const long long total = (long long)nx * ny * nz;
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < total; q += (long long)gridDim.x * 256) {
        const int x = (int)(q % nx);
        const long long yz = q / nx;
        const long long n = yz * pitch + x;
        if (info[n] & INFO3_SOLID) continue;
        for (int i = 0; i < Q; ++i) {
            m0 += (double)f[(size_t)i * plane + n];
            m1 += (double)f[(size_t)(Q + i) * plane + n];
        }
        const double ux = (double)umac[n], uy = (double)umac[plane + n], uz = (double)umac[2 * plane + n];
        u2 = fmax(u2, ux * ux + uy * uy + uz * uz);
    }
    s0[threadIdx.x] = m0;
    s1[threadIdx.x] = m1;
    s2[threadIdx.x] = u2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s0[threadIdx.x] += s0[threadIdx.x + w];
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[blockIdx.x * 3] = s0[0];
        partial[blockIdx.x * 3 + 1] = s1[0];
        partial[blockIdx.x * 3 + 2] = s2[0];
    }
}

template <typename S>
cudaError_t launch_step(const D3Args<S>& a, cudaStream_t st, cudaEvent_t mid_a, cudaEvent_t mid_b) {
    const dim3 blkA(32, 4, 2);
    const dim3 grdA((a.nx + 31) / 32, (a.ny + 3) / 4, (a.nz + 1) / 2);
    const int fblocks = (a.nface_slots + 127) / 128;
    d3q_pull_kernel<S><<<grdA, blkA, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.nface_slots > 0) {
        d3q_face_pull_kernel<S><<<fblocks, 128, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (mid_a) cudaEventRecord(mid_a, st);
    const dim3 blkB(TX, TY, TZ);
    const dim3 grdB((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + TZ - 1) / TZ);
    d3q_collide_kernel<S><<<grdB, blkB, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (mid_b) cudaEventRecord(mid_b, st);
    if (a.nface_slots > 0) {
        d3q_face_collide_kernel<S><<<fblocks, 128, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        d3q_reduce_kernel<S><<<1, 256, 0, st>>>(a);
        e = cudaGetLastError();
    }
    return e;
}

template <typename S>
cudaError_t launch_mass(const S* f, const uint32_t* info, const S* umac, int nx, int ny, int nz, int pitch,
                        long long plane, double* partial, int nblocks, cudaStream_t st) {
    d3q_mass_kernel<S><<<nblocks, 256, 0, st>>>(f, info, umac, nx, ny, nz, pitch, plane, partial);
    return cudaGetLastError();
}

template cudaError_t launch_step<float>(const D3Args<float>&, cudaStream_t, cudaEvent_t, cudaEvent_t);
template cudaError_t launch_step<double>(const D3Args<double>&, cudaStream_t, cudaEvent_t, cudaEvent_t);
template cudaError_t launch_mass<float>(const float*, const uint32_t*, const float*, int, int, int, int, long long,
                                        double*, int, cudaStream_t);
template cudaError_t launch_mass<double>(const double*, const uint32_t*, const double*, int, int, int, int,
                                         long long, double*, int, cudaStream_t);

}  // namespace lbm3
