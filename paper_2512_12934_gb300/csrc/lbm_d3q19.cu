// D3Q19 two-component MRT pseudopotential step with the corrected open faces
// (the three-dimensional counterpart of lbm_d2q9.cu).
//
// One time step is five launches on the context's stream:
//   A  d3q_pull_kernel      pull streaming (Eq. 2) with halfway bounce-back
//                           (Eq. B1) and periodic wrap (Eq. B2) of interior
//                           nodes; component densities rho_k (= psi_k) to a
//                           field.
//   A' d3q_face_pull_kernel one thread per open-face slot: the same pull,
//                           then inlet reconstruction (Eq. 13 over the 5
//                           unknowns, alpha correction Eqs. 15-19) or the
//                           convective outlet (Eq. 20); densities.
//   B  d3q_collide_kernel   rho and the solid indicator of a 32x4xTZ tile plus
//                           a 2-node halo (ghost mirrors of Eqs. 24-25) staged
//                           in shared memory; forces of Eqs. 10-11 on the
//                           92-vector 8th-order isotropic stencil; common
//                           velocity (Eqs. 7-8); MRT collision with forcing
//                           (Eqs. 1, 3-6, 9) with the 19x19 transforms
//                           unrolled over compile-time constants; per-face-node
//                           FP64 flux terms.
//   B' d3q_outlet_kernel    outlet nodes: normal velocity chi times that of the
//                           inward neighbour (Eq. 22), collision.
//   C  d3q_reduce_kernel    fixed-order FP64 sums of the flux terms: lambda
//                           (Eq. 21) and chi (Eq. 23) for the next step.
// Face nodes carry their post-boundary populations from A' to B, the outlet's
// previous post-boundary populations (Eq. 20) and the forces the inlet needs
// one step later in small slot-indexed arrays.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

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

// Compile-time loop: f(std::integral_constant<int, i>) for i in [B, E), so
// every lattice constant below is a template constant (no runtime tables).
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// acc += c * v with the integer c folded at compile time (0: nothing).
template <int c, typename R>
__device__ __forceinline__ void acc_c(R& acc, R v) {
    if constexpr (c == 1) acc += v;
    else if constexpr (c == -1) acc -= v;
    else if constexpr (c != 0) acc += (R)c * v;
}

// ---- tiles of the collide kernel -----------------------------------------
// Tiles are TX x TY x TZ nodes; FP32 storage takes TZ = 4 (512 threads, two
// CTAs per SM: a staged halo of 4.5 sites per node instead of 6.75), the
// others TZ = 2 (FP64 needs 140 registers a thread, FP16 storage 80).
constexpr int TX = 32, TY = 4;
constexpr int HX = TX + 4, HY = TY + 4;
template <typename S>
struct Tile3 {
    static constexpr int TZ = std::is_same<S, float>::value ? 4 : 2;
    static constexpr int HZ = TZ + 4;
    static constexpr int HN = HX * HY * HZ;
    static constexpr int NT = TX * TY * TZ;
    static constexpr int MIN_BLOCKS = sizeof(S) == 8 ? 1 : (sizeof(S) == 4 ? 2 : 3);
};
static_assert(HX == RHO_BOX3_X && HY == RHO_BOX3_Y && Tile3<float>::HZ == RHO_BOX3_Z,
              "the density tensor-copy box must be the FP32 collide tile plus its halo");

template <typename R>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
};
template <>
struct Pair<double> {
    using type = double2;
};

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
template <>
struct Store<__half> {
    using R = float;
};

template <typename S>
__device__ __forceinline__ constexpr bool is_half() {
    return std::is_same<S, __half>::value;
}

// A stored population as a real number (FP16 storage: the deviation only).
template <typename S>
__device__ __forceinline__ typename Store<S>::R ld_pop(S v) {
    if constexpr (is_half<S>()) return __half2float(v);
    else return v;
}

// Density rounded to the half-precision reference of FP16 storage.
__device__ __forceinline__ float half_round(float r) { return __half2float(__float2half_rn(r)); }

// Wrap a pull source on periodic axes (blocked sources never reach here).
__device__ __forceinline__ int wrap(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

template <typename S>
__device__ __forceinline__ long long node_index(const D3Args<S>& a, int x, int y, int z) {
    return ((long long)z * a.ny + y) * a.pitch + x;
}

// Pull the 19 populations of component k at (x, y, z) (Eq. 2, Eq. B1, Eq. B2).
// Away from periodic edges the source of direction i is n minus a fixed
// offset (e_x + e_y pitch + e_z ny pitch); across an edge it is wrapped.
template <typename S, typename R, bool FAST = true>
__device__ __forceinline__ void pull(const D3Args<S>& a, int k, int x, int y, int z, uint32_t info, R (&f)[Q]) {
    const S* __restrict__ fin = a.fin + (size_t)k * Q * a.plane;
    const long long n = node_index(a, x, y, z);
    const long long sy = a.pitch, sz = (long long)a.ny * a.pitch;
    const bool wrapped = (info & INFO3_WRAP) != 0;
    // FP16 storage: every value this node pulls was encoded against its
    // reference density (the writer used the same half-rounded density)
    R ref = 0;
    if constexpr (is_half<S>()) ref = __half2float(a.rref_in[(size_t)k * a.plane + n]);
    if (FAST && !wrapped && (info & 0x7FFFFu) == 0u) {
        // no blocked direction, no wrap (most fluid nodes): straight neighbour loads
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            long long src = n;
            if constexpr (ex_(i) != 0) src -= ex_(i);
            if constexpr (ey_(i) == 1) src -= sy;
            if constexpr (ey_(i) == -1) src += sy;
            if constexpr (ez_(i) == 1) src -= sz;
            if constexpr (ez_(i) == -1) src += sz;
            f[i] = (R)ld_pop(fin[(size_t)i * a.plane + src]);
            if constexpr (is_half<S>()) f[i] += ((R)w36_(i) / (R)36) * ref;
        });
        return;
    }
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (info & (1u << i)) {
            f[i] = (R)ld_pop(fin[(size_t)opp_(i) * a.plane + n]);
        } else if (!wrapped) {
            long long src = n;
            if constexpr (ex_(i) != 0) src -= ex_(i);
            if constexpr (ey_(i) == 1) src -= sy;
            if constexpr (ey_(i) == -1) src += sy;
            if constexpr (ez_(i) == 1) src -= sz;
            if constexpr (ez_(i) == -1) src += sz;
            f[i] = (R)ld_pop(fin[(size_t)i * a.plane + src]);
        } else {
            const int xs = ex_(i) ? wrap(x - ex_(i), a.nx) : x;
            const int ys = ey_(i) ? wrap(y - ey_(i), a.ny) : y;
            const int zs = ez_(i) ? wrap(z - ez_(i), a.nz) : z;
            f[i] = (R)ld_pop(fin[(size_t)i * a.plane + node_index(a, xs, ys, zs)]);
        }
        if constexpr (is_half<S>()) f[i] += ((R)w36_(i) / (R)36) * ref;
    });
}

template <typename R>
__device__ __forceinline__ void feq(R rho, R ux, R uy, R uz, R (&out)[Q]) {
    const R uu = ux * ux + uy * uy + uz * uz;
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        R eu = 0;
        acc_c<ex_(i)>(eu, ux);
        acc_c<ey_(i)>(eu, uy);
        acc_c<ez_(i)>(eu, uz);
        out[i] = rho * ((R)w36_(i) / (R)36) * ((R)1 + (R)3 * eu + (R)4.5 * eu * eu - (R)1.5 * uu);
    });
}

// Density as the rest population plus the sums of opposite pairs.
template <typename R>
__device__ __forceinline__ R sum19(const R (&f)[Q]) {
    R s = f[0];
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if constexpr (opp_(i) > i) s += f[i] + f[opp_(i)];
    });
    return s;
}

// Momentum as sums of opposite-pair differences (each difference of two
// nearby populations is exact or nearly so, which keeps FP32 j accurate).
template <typename R>
__device__ __forceinline__ void moments_j(const R (&f)[Q], R& jx, R& jy, R& jz) {
    R x = 0, y = 0, z = 0;
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if constexpr (opp_(i) > i) {
            const R d = f[i] - f[opp_(i)];
            acc_c<ex_(i)>(x, d);
            acc_c<ey_(i)>(y, d);
            acc_c<ez_(i)>(z, d);
        }
    });
    jx = x;
    jy = y;
    jz = z;
}

// Eq. 1 for one component: f <- f - T^-1 S (T f - m^eq) + T^-1 (I - S/2) F_m,
// T^-1 = T^T diag(1/|row|^2) (orthogonal rows).  m^eq = T f^eq and F_m =
// T Fbar (Eqs. 6, 9) are written out as the polynomials they reduce to for
// this basis (rho; e: rho(19u^2 - 11); eps: rho(6 - 11u^2)/2; j: rho u;
// q: -2 rho u/3; 3p_xx: rho(3u_x^2 - u^2); 3pi_xx: -3p_xx/2; p_ww:
// rho(u_y^2 - u_z^2); pi_ww: -p_ww/2; p_ab: rho u_a u_b; m: 0 -- and for
// F_m the same moments of the Guo term: 0, 38 u.F, -11 u.F, F, -2F/3,
// 2(3u_xF_x - u.F), -(3u_xF_x - u.F), 2(u_yF_y - u_zF_z), -(u_yF_y - u_zF_z),
// u_aF_b + u_bF_a, 0).  All entries of T are template constants.
// Moments through opposite pairs: the even rows of T (rho, e, eps, p, pi)
// weigh f_i and f_ibar alike, the odd rows (j, q, m) with opposite signs, so
// T f needs only the pair sums P_i = f_i + f_ibar and differences
// D_i = f_i - f_ibar (i over one member of each pair), and the back
// transform splits the same way.
template <int r>
__host__ __device__ constexpr bool odd_row() {
    return r == 3 || r == 4 || r == 5 || r == 6 || r == 7 || r == 8 || r == 16 || r == 17 || r == 18;
}

template <typename R>
__device__ __forceinline__ void collide(R (&f)[Q], R rho, R ux, R uy, R uz, R Fx, R Fy, R Fz, const R* s) {
    R P[Q], D[Q];  // only the entries of the first member of each pair are used
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if constexpr (opp_(i) > i) {
            P[i] = f[i] + f[opp_(i)];
            D[i] = f[i] - f[opp_(i)];
        }
    });
    R m[Q];
    static_for<0, Q>([&](auto Rr) {
        constexpr int r = decltype(Rr)::value;
        R acc = 0;
        if constexpr (!odd_row<r>()) acc_c<T_(r, 0)>(acc, f[0]);
        static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if constexpr (opp_(i) > i) {
                if constexpr (odd_row<r>()) acc_c<T_(r, i)>(acc, D[i]);
                else acc_c<T_(r, i)>(acc, P[i]);
            }
        });
        m[r] = acc;
    });
    const R uu = ux * ux + uy * uy + uz * uz;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    const R pxx = (R)2 * ux * ux - uy * uy - uz * uz, fxx = (R)2 * ((R)2 * ux * Fx - uy * Fy - uz * Fz);
    const R pww = uy * uy - uz * uz, fww = (R)2 * (uy * Fy - uz * Fz);
    const R meq[Q] = {rho, rho * ((R)19 * uu - (R)11), rho * ((R)6 - (R)11 * uu) * (R)0.5, rho * ux,
                      -(R)2 / (R)3 * rho * ux, rho * uy, -(R)2 / (R)3 * rho * uy, rho * uz, -(R)2 / (R)3 * rho * uz,
                      rho * pxx, -(R)0.5 * rho * pxx, rho * pww, -(R)0.5 * rho * pww, rho * ux * uy, rho * uy * uz,
                      rho * ux * uz, 0, 0, 0};
    const R mF[Q] = {0, (R)38 * uF, -(R)11 * uF, Fx, -(R)2 / (R)3 * Fx, Fy, -(R)2 / (R)3 * Fy, Fz,
                     -(R)2 / (R)3 * Fz, fxx, -(R)0.5 * fxx, fww, -(R)0.5 * fww, ux * Fy + uy * Fx, uy * Fz + uz * Fy,
                     ux * Fz + uz * Fx, 0, 0, 0};
    R g[Q];
    static_for<0, Q>([&](auto Rr) {
        constexpr int r = decltype(Rr)::value;
        // the density row drops out: m_rho = m^eq_rho by definition and the
        // forcing term has no density moment
        if constexpr (r == 0) g[r] = (R)0;
        else g[r] = (-s[r] * (m[r] - meq[r]) + ((R)1 - (R)0.5 * s[r]) * mF[r]) * ((R)1 / (R)Tnorm_(r));
    });
    {
        R acc = 0;
        static_for<0, Q>([&](auto Rr) {
            constexpr int r = decltype(Rr)::value;
            acc_c<T_(r, 0)>(acc, g[r]);
        });
        f[0] += acc;
    }
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if constexpr (opp_(i) > i) {
            R ev = 0, od = 0;
            static_for<0, Q>([&](auto Rr) {
                constexpr int r = decltype(Rr)::value;
                if constexpr (odd_row<r>()) acc_c<T_(r, i)>(od, g[r]);
                else acc_c<T_(r, i)>(ev, g[r]);
            });
            f[i] += ev + od;
            f[opp_(i)] += ev - od;
        }
    });
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
__global__ void __launch_bounds__(256, 4) d3q_pull_kernel(D3Args<S> a) {
    using R = typename Store<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= a.nx || y >= a.ny || z >= a.nz) return;
    const long long n = node_index(a, x, y, z);
    const uint32_t info = a.info[n];
    if (info & INFO3_SOLID) {  // psi = 0 at solid sites of the force stencil
        reinterpret_cast<typename Pair<R>::type*>(a.rho)[n] = typename Pair<R>::type{(R)0, (R)0};
        return;
    }
    if ((info >> INFO3_FACE_SHIFT) & 7u) return;  // open-face nodes: d3q_face_pull_kernel
    if constexpr (is_half<S>()) {
        // sum w_i = 1: rho_k = rho_ref + the sum of the stored deviations
        const long long sy = a.pitch, sz = (long long)a.ny * a.pitch;
        const bool wrapped = (info & INFO3_WRAP) != 0;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const S* __restrict__ fin = a.fin + (size_t)k * Q * a.plane;
            float acc = 0.0f;
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                long long src;
                int ii = i;
                if (info & (1u << i)) {
                    src = n;
                    ii = opp_(i);
                } else if (!wrapped) {
                    src = n - ex_(i) - (long long)ey_(i) * sy - (long long)ez_(i) * sz;
                } else {
                    src = node_index(a, ex_(i) ? wrap(x - ex_(i), a.nx) : x, ey_(i) ? wrap(y - ey_(i), a.ny) : y,
                                     ez_(i) ? wrap(z - ez_(i), a.nz) : z);
                }
                acc += __half2float(fin[(size_t)ii * a.plane + src]);
            });
            a.rho[2 * n + k] = __half2float(a.rref_in[(size_t)k * a.plane + n]) + acc;
        }
    } else {
        R r[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            R f[Q];
            pull<S, R, false>(a, k, x, y, z, info, f);
            r[k] = sum19(f);
        }
        reinterpret_cast<typename Pair<R>::type*>(a.rho)[n] = typename Pair<R>::type{r[0], r[1]};
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
    reinterpret_cast<typename Pair<R>::type*>(a.rho)[n] = typename Pair<R>::type{sum19(f[0]), sum19(f[1])};
}

// ---- kernel B: forces, velocity, collision --------------------------------
// Resolve a psi / indicator site (Eqs. 10, 11, 24, 25) to a node index:
// periodic wrap, ghost mirror across open sides, -1 outside a closed side
// (a solid wall).  Solid nodes inside the grid carry (0, 0) in the density
// field: psi = 0 there, as at closed sides.
template <typename S>
__device__ __forceinline__ long long site_index(const D3Args<S>& a, int x, int y, int z) {
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
    return node_index(a, c[0], c[1], c[2]);
}

// Interaction sums over the 92-vector stencil: g_k = sum w psi_k(x+e) e,
// `site(dx, dy, dz)` returns the (psi_1, psi_2) pair of a site (0 at solids).
// Pairs (e, -e) share the weight: g += w e (psi(x+e) - psi(x-e)); c runs over
// the half of the 5x5x5 cube before its centre (index 62), -e is site 124 - c.
// In FP32 both components go through one packed FP32x2 operation per term
// (each lane rounds as the scalar FMA does).
template <typename R, typename Site>
__device__ __forceinline__ void stencil_sums(Site site, R (&g1)[3], R (&g2)[3]) {
    if constexpr (std::is_same<R, float>::value) {
        float2 g[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) g[q] = make_float2(0.f, 0.f);
        static_for<0, 62>([&](auto C) {
            constexpr int c = decltype(C)::value;
            constexpr int dx = c % 5 - 2, dy = (c / 5) % 5 - 2, dz = c / 25 - 2;
            constexpr int r2 = dx * dx + dy * dy + dz * dz;
            constexpr int wq = sw5040_(r2);
            if constexpr (wq != 0) {
                constexpr float w = (float)wq / 5040.f;
                const float2 d = __ffma2_rn(site(-dx, -dy, -dz), make_float2(-1.f, -1.f), site(dx, dy, dz));
                if constexpr (dx != 0) g[0] = __ffma2_rn(make_float2(w * dx, w * dx), d, g[0]);
                if constexpr (dy != 0) g[1] = __ffma2_rn(make_float2(w * dy, w * dy), d, g[1]);
                if constexpr (dz != 0) g[2] = __ffma2_rn(make_float2(w * dz, w * dz), d, g[2]);
            }
        });
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            g1[q] = g[q].x;
            g2[q] = g[q].y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) g1[q] = g2[q] = (R)0;
        static_for<0, 62>([&](auto C) {
            constexpr int c = decltype(C)::value;
            constexpr int dx = c % 5 - 2, dy = (c / 5) % 5 - 2, dz = c / 25 - 2;
            constexpr int r2 = dx * dx + dy * dy + dz * dz;
            constexpr int wq = sw5040_(r2);
            if constexpr (wq != 0) {
                const R w = (R)wq / (R)5040;
                const auto p = site(dx, dy, dz), m = site(-dx, -dy, -dz);
                const R d1 = p.x - m.x, d2 = p.y - m.y;
                if constexpr (dx != 0) {
                    g1[0] += (w * (R)dx) * d1;
                    g2[0] += (w * (R)dx) * d2;
                }
                if constexpr (dy != 0) {
                    g1[1] += (w * (R)dy) * d1;
                    g2[1] += (w * (R)dy) * d2;
                }
                if constexpr (dz != 0) {
                    g1[2] += (w * (R)dz) * d1;
                    g2[2] += (w * (R)dz) * d2;
                }
            }
        });
    }
}

// sum_e w s(x+e) e of Eq. 11 (geometry only; precomputed per near-solid node)
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Wait for phase `parity` of an mbarrier for at most about a second of SM
// clock; false if the wait ran out.
__device__ __forceinline__ bool bar_wait(unsigned long long* bar, unsigned parity) {
    const long long t0 = clock64();
    for (;;) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(smem_addr(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
        if (clock64() - t0 > 2000000000LL) return false;
    }
}

template <typename S>
__device__ __forceinline__ void adhesion_vector(const D3Args<S>& a, long long n, uint32_t info,
                                                typename Store<S>::R (&ad)[3]) {
    using R = typename Store<S>::R;
    if (info & INFO3_NEAR_SOLID) {
        ad[0] = (R)a.adv[n];
        ad[1] = (R)a.adv[a.plane + n];
        ad[2] = (R)a.adv[2 * a.plane + n];
    } else {
        ad[0] = ad[1] = ad[2] = (R)0;
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

template <typename R>
__device__ __forceinline__ void add_j(const R (&f)[Q], R (&j)[3]) {
    R jx, jy, jz;
    moments_j(f, jx, jy, jz);
    j[0] += jx;
    j[1] += jy;
    j[2] += jz;
}

// Store the post-collision populations of component k at node n.  FP16
// storage writes half(f*_i - w_i rho_ref), rho_ref being the half-rounded
// density of component k at the node that pulls f*_i next step: x + e_i, or
// x itself when that neighbour is solid or outside (halfway bounce-back).
// dest_ref(I, k) returns that reference (already half-rounded).
template <typename S, typename DestRho>
__device__ __forceinline__ void store_pop(const D3Args<S>& a, int k, long long n, const typename Store<S>::R (&f)[Q],
                                          DestRho dest_ref) {
    using R = typename Store<S>::R;
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if constexpr (is_half<S>()) {
            const R ref = dest_ref(I, k);
            a.fout[(size_t)(k * Q + i) * a.plane + n] = __float2half_rn(f[i] - ((R)w36_(i) / (R)36) * ref);
        } else {
            a.fout[(size_t)(k * Q + i) * a.plane + n] = (S)f[i];
        }
    });
}

template <typename S>
__device__ __forceinline__ void check_store_u(const D3Args<S>& a, long long n, typename Store<S>::R rt,
                                              const typename Store<S>::R (&u)[3]) {
    if (!(isfinite((float)rt) && isfinite((float)u[0]) && isfinite((float)u[1]) && isfinite((float)u[2])))
        atomicOr(a.status, STATUS3_DIVERGED);
    if (a.umac) {
        a.umac[n] = u[0];
        a.umac[a.plane + n] = u[1];
        a.umac[2 * a.plane + n] = u[2];
    }
}

// Every fluid node of a 32x4xTZ tile: forces from the staged densities (the
// halo resolves periodic wraps and the ghost mirrors of Eqs. 24-25), the
// common velocity, the collision.  Open-face nodes take their post-boundary
// populations from the face kernel; outlet nodes stop after the force (their
// normal velocity waits for the inward neighbour's, Eq. 22), and the inward
// neighbours of the outlet hand theirs over with the flux terms of Eqs. 21, 23.
// Residency: FP32 runs 2 CTAs of 512 per SM (64 registers, a few spilled
// words), FP16 storage 3 of 256 (its decode needs more live values), FP64 1
// of 256.  Tiles without a fluid node leave before staging.
template <typename S>
__global__ void __launch_bounds__(Tile3<S>::NT, Tile3<S>::MIN_BLOCKS)
    d3q_collide_kernel(D3Args<S> a, const __grid_constant__ CUtensorMap rho_map, int use_tma) {
    using R = typename Store<S>::R;
    constexpr int TZ = Tile3<S>::TZ, HN = Tile3<S>::HN, NT = Tile3<S>::NT;
    // (rho_1, rho_2) of the tile and its halo, psi = 0 at solids; 128-byte
    // aligned: an interior FP32 tile receives it as one tensor copy
    __shared__ __align__(128) typename Pair<R>::type s_rr[HN];
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ __half2 s_ref[is_half<S>() ? HN : 1];  // FP16 storage: the same densities rounded to half
    __shared__ R s_rate[2][Q];  // relaxation rates of both components (indexed by component below)
    // component 0's pulled populations, kept for its collision after
    // component 1's (FP32 arithmetic; FP64 pulls them again, its tile would
    // exceed the static shared-memory limit)
    constexpr bool STASH = sizeof(R) == 4;
    __shared__ R s_f0[STASH ? Q : 1][STASH ? NT : 1];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    const bool in_grid = x < a.nx && y < a.ny && z < a.nz;
    const long long n = in_grid ? node_index(a, x, y, z) : 0;
    const uint32_t info = in_grid ? a.info[n] : (uint32_t)INFO3_SOLID;
    // a tile without fluid nodes has nothing to stage or collide
    if (!__syncthreads_or(!(info & INFO3_SOLID))) return;
    if (tid < 2 * Q) s_rate[tid / Q][tid % Q] = a.s[tid / Q][tid % Q];
    // tiles whose halo lies inside the grid need no wrap / mirror / wall resolution
    const bool inner = x0 >= 2 && y0 >= 2 && z0 >= 2 && x0 + TX + 2 <= a.nx && y0 + TY + 2 <= a.ny &&
                       z0 + TZ + 2 <= a.nz;
    bool staged = false;
    if constexpr (std::is_same<S, float>::value) {
        // interior FP32 tile: the (TX+4) x (TY+4) x (TZ+4) box of density
        // pairs as one TMA copy (x0 - 2 is even: an 8-byte element start on a
        // 16-byte boundary); the block-uniform test keeps a misaligned
        // destination on the load path
        if (use_tma && inner && (smem_addr(s_rr) & 127u) == 0u) {
            if (tid == 0) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bar)) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&s_bar)),
                             "r"((unsigned)(HN * sizeof(typename Pair<R>::type)))
                             : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], "
                    "[%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(s_rr)),
                    "l"(&rho_map), "r"(x0 - 2), "r"(y0 - 2), "r"(z0 - 2), "r"(smem_addr(&s_bar))
                    : "memory");
            }
            __syncthreads();  // the barrier exists before anyone waits on it; s_rate is written
            if (!bar_wait(&s_bar, 0u) && tid == 0) atomicOr(a.status, STATUS3_TIMEOUT);
            staged = true;
        }
    }
    if (!staged) {
        const auto* rp = reinterpret_cast<const typename Pair<R>::type*>(a.rho);
        for (int q = tid; q < HN; q += NT) {
            const int hx = q % HX, hy = (q / HX) % HY, hz = q / (HX * HY);
            const long long m = inner ? node_index(a, x0 - 2 + hx, y0 - 2 + hy, z0 - 2 + hz)
                                      : site_index(a, x0 - 2 + hx, y0 - 2 + hy, z0 - 2 + hz);
            const typename Pair<R>::type v = m < 0 ? typename Pair<R>::type{(R)0, (R)0} : rp[m];
            s_rr[q] = v;
            if constexpr (is_half<S>()) s_ref[q] = __floats2half2_rn((float)v.x, (float)v.y);
        }
        __syncthreads();
    }
    if (info & INFO3_SOLID) return;  // solid, or outside the grid
    const int hc = (threadIdx.x + 2) + HX * ((threadIdx.y + 2) + HY * (threadIdx.z + 2));
    auto site = [&](int dx, int dy, int dz) { return s_rr[hc + dx + HX * (dy + HY * dz)]; };
    const int fid = (int)((info >> INFO3_FACE_SHIFT) & 7u);
    const int nid = (int)((info >> INFO3_NBR_SHIFT) & 7u);
    R f[Q];
    R j[3] = {0, 0, 0};
    int slot = -1;
    if (fid == 0) pull<S, R>(a, 0, x, y, z, info, f);  // loads overlap the stencil below
    R g1[3], g2[3], ad[3];
    stencil_sums<R>(site, g1, g2);
    adhesion_vector<S>(a, n, info, ad);
    const R r1 = s_rr[hc].x, r2 = s_rr[hc].y;
    R F1[3], F2[3];
    forces<R>(a.G, r1, r2, g1, g2, ad, a.body, F1, F2);
    const R rt = r1 + r2;
    if (fid == 0) {
        add_j(f, j);
        if constexpr (STASH)
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                s_f0[i][tid] = f[i];
            });
        pull<S, R>(a, 1, x, y, z, info, f);
        add_j(f, j);
    } else {
        const FaceDev3& Fc = a.face[fid - 1];
        slot = face_slot(Fc, x, y, z);
        R* Fp = a.FpF + (size_t)slot * 6;  // this step's force: next step's inlet, this step's outlet
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            Fp[q] = F1[q];
            Fp[3 + q] = F2[q];
        }
        if (Fc.kind == FACE3_OUTLET) return;  // finished by d3q_outlet_kernel
        const R* ff = a.fface + (size_t)slot * 2 * Q;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                f[i] = ff[k * Q + i];
            });
            add_j(f, j);
        }
    }
    R u[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) u[q] = (j[q] + (R)0.5 * (F1[q] + F2[q])) / rt;
    if (nid != 0) {
        const FaceDev3& Fc = a.face[nid - 1];
        const int ns = face_slot(Fc, x + Fc.o[0], y + Fc.o[1], z + Fc.o[2]);
        R* Fp = a.FpN + (size_t)ns * 6;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            Fp[q] = F1[q];
            Fp[3 + q] = F2[q];
        }
        if (Fc.kind == FACE3_OUTLET) {
            const double sg = (double)(Fc.o[0] + Fc.o[1] + Fc.o[2]);
            R* un = a.unbr + (size_t)ns * 3;
            un[0] = u[0];
            un[1] = u[1];
            un[2] = u[2];
            a.flux[(size_t)ns * 2 + 0] = (double)rt * sg * (double)u[Fc.axis];
            a.flux[(size_t)ns * 2 + 1] = sg * (double)u[Fc.axis];
        }
    }
    if (fid != 0) {  // inlet node: flux term of Q_in
        const FaceDev3& Fc = a.face[fid - 1];
        const double sg = (double)(Fc.o[0] + Fc.o[1] + Fc.o[2]);
        a.flux[(size_t)slot * 2 + 0] = (double)rt * (-sg) * (double)u[Fc.axis];
        a.flux[(size_t)slot * 2 + 1] = 0.0;
    }
    check_store_u<S>(a, n, rt, u);
    // reader densities for FP16 storage: the staged tile (periodic wraps
    // resolved) or this node when the direction is blocked
    auto dest_rho = [&](auto I, int k) -> R {
        constexpr int i = decltype(I)::value;
        const int h = (info & (1u << opp_(i))) ? hc : hc + ex_(i) + HX * (ey_(i) + HY * ez_(i));
        const __half2 r = s_ref[h];
        return k ? __high2float(r) : __low2float(r);
    };
    if constexpr (is_half<S>()) {
        a.rref_out[n] = __float2half_rn(r1);
        a.rref_out[a.plane + n] = __float2half_rn(r2);
    }
    // collide component 1 (still in registers), then component 0 (from the
    // shared-memory copy in FP32, pulled again in FP64): one loop body, so
    // the unrolled collision is in the instruction stream once
#pragma unroll 1
    for (int k = 1; k >= 0; --k) {
        if (k == 0) {
            if (fid == 0) {
                if constexpr (STASH)
                    static_for<0, Q>([&](auto I) {
                        constexpr int i = decltype(I)::value;
                        f[i] = s_f0[i][tid];
                    });
                else pull<S, R>(a, 0, x, y, z, info, f);
            } else {
                const R* ff = a.fface + (size_t)slot * 2 * Q;
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    f[i] = ff[i];
                });
            }
        }
        const R rk = k ? r2 : r1;
        const R fx = k ? F2[0] : F1[0], fy = k ? F2[1] : F1[1], fz = k ? F2[2] : F1[2];
        collide<R>(f, rk, u[0], u[1], u[2], fx, fy, fz, s_rate[k]);
        store_pop<S>(a, k, n, f, dest_rho);
    }
}

// One thread per outlet slot: the outlet node's velocity with the normal
// component chi times that of its inward neighbour (Eq. 22), the collision.
template <typename S>
__global__ void __launch_bounds__(128) d3q_outlet_kernel(D3Args<S> a) {
    using R = typename Store<S>::R;
    int fid, c[3];
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (!slot_node(a, slot, fid, c)) return;
    const FaceDev3& Fc = a.face[fid];
    if (Fc.kind != FACE3_OUTLET) return;
    const long long n = node_index(a, c[0], c[1], c[2]);
    const R r1 = a.rho[2 * n], r2 = a.rho[2 * n + 1], rt = r1 + r2;
    const R* Fp = a.FpF + (size_t)slot * 6;
    const R F1[3] = {Fp[0], Fp[1], Fp[2]}, F2[3] = {Fp[3], Fp[4], Fp[5]};
    const R* ff = a.fface + (size_t)slot * 2 * Q;
    R f[Q], j[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            f[i] = ff[k * Q + i];
        });
        add_j(f, j);
    }
    R u[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) u[q] = (j[q] + (R)0.5 * (F1[q] + F2[q])) / rt;
    if (Fc.chi) u[Fc.axis] = (R)a.scal_in[SC3_CHI] * a.unbr[(size_t)slot * 3 + Fc.axis];
    check_store_u<S>(a, n, rt, u);
    const uint32_t info = a.info[n];
    auto dest_rho = [&](auto I, int k) -> R {
        constexpr int i = decltype(I)::value;
        long long m = n;
        if (!(info & (1u << opp_(i)))) m = site_index(a, c[0] + ex_(i), c[1] + ey_(i), c[2] + ez_(i));
        return half_round(a.rho[2 * m + k]);
    };
    if constexpr (is_half<S>()) {
        a.rref_out[n] = __float2half_rn(r1);
        a.rref_out[a.plane + n] = __float2half_rn(r2);
    }
    collide<R>(f, r2, u[0], u[1], u[2], F2[0], F2[1], F2[2], a.s[1]);
    store_pop<S>(a, 1, n, f, dest_rho);
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        f[i] = ff[i];
    });
    collide<R>(f, r1, u[0], u[1], u[2], F1[0], F1[1], F1[2], a.s[0]);
    store_pop<S>(a, 0, n, f, dest_rho);
}

// ---- kernel C: lambda and chi from the face flux terms (fixed order) -------
// One block of 1024 threads; each thread owns a fixed set of slots and the
// tree below has a fixed shape, so the sums are deterministic.  Slots of
// solid face positions hold the zeros they were created with.
constexpr int RED = 1024;
template <typename S>
__global__ void __launch_bounds__(RED) d3q_reduce_kernel(D3Args<S> a) {
    __shared__ double s_in[RED], s_out[RED], s_u[RED];
    double qin = 0.0, qout = 0.0, us = 0.0;
    const double2* fl = reinterpret_cast<const double2*>(a.flux);
    for (int f = 0; f < a.nfaces; ++f) {
        const FaceDev3& F = a.face[f];
        const bool inlet = F.kind == FACE3_INLET;
#pragma unroll 4
        for (int q = threadIdx.x; q < F.count; q += RED) {
            const double2 v = fl[F.base + q];
            if (inlet) qin += v.x;
            else {
                qout += v.x;
                us += v.y;
            }
        }
    }
    s_in[threadIdx.x] = qin;
    s_out[threadIdx.x] = qout;
    s_u[threadIdx.x] = us;
    __syncthreads();
    for (int w = RED / 2; w > 0; w >>= 1) {
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
                                                       const typename Store<S>::R* __restrict__ umac,
                                                       const __half* __restrict__ rref, int nx, int ny, int nz,
                                                       int pitch, long long plane, double* __restrict__ partial) {
    __shared__ double s0[256], s1[256], s2[256];
    double m0 = 0.0, m1 = 0.0, u2 = 0.0;
    const long long total = (long long)nx * ny * nz;
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < total; q += (long long)gridDim.x * 256) {
        const int x = (int)(q % nx);
        const long long yz = q / nx;
        const int y = (int)(yz % ny), z = (int)(yz / ny);
        const long long n = yz * pitch + x;
        const uint32_t inf = info[n];
        if (inf & INFO3_SOLID) continue;
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            double v0 = (double)ld_pop(f[(size_t)i * plane + n]);
            double v1 = (double)ld_pop(f[(size_t)(Q + i) * plane + n]);
            if constexpr (is_half<S>()) {
                // decode with the reference of the node that will pull the value
                long long m = n;
                if (!(inf & (1u << opp_(i)))) {
                    const int xs = ex_(i) ? wrap(x + ex_(i), nx) : x;
                    const int ys = ey_(i) ? wrap(y + ey_(i), ny) : y;
                    const int zs = ez_(i) ? wrap(z + ez_(i), nz) : z;
                    m = ((long long)zs * ny + ys) * pitch + xs;
                }
                const double w = (double)w36_(i) / 36.0;
                v0 += w * (double)__half2float(rref[m]);
                v1 += w * (double)__half2float(rref[plane + m]);
            }
            m0 += v0;
            m1 += v1;
        });
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
cudaError_t launch_step(const D3Args<S>& a, const CUtensorMap* rho_map, cudaStream_t st, cudaEvent_t mid_a,
                        cudaEvent_t mid_b) {
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
    constexpr int TZ = Tile3<S>::TZ;
    const dim3 blkB(TX, TY, TZ);
    const dim3 grdB((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + TZ - 1) / TZ);
    static const CUtensorMap kNoMap{};
    d3q_collide_kernel<S><<<grdB, blkB, 0, st>>>(a, rho_map ? *rho_map : kNoMap, rho_map ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (mid_b) cudaEventRecord(mid_b, st);
    if (a.nface_slots > 0) {
        d3q_outlet_kernel<S><<<fblocks, 128, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        d3q_reduce_kernel<S><<<1, RED, 0, st>>>(a);
        e = cudaGetLastError();
    }
    return e;
}

template <typename S>
cudaError_t launch_mass(const S* f, const uint32_t* info, const typename Real<S>::type* umac, const __half* rref,
                        int nx, int ny, int nz, int pitch, long long plane, double* partial, int nblocks,
                        cudaStream_t st) {
    d3q_mass_kernel<S><<<nblocks, 256, 0, st>>>(f, info, umac, rref, nx, ny, nz, pitch, plane, partial);
    return cudaGetLastError();
}

template cudaError_t launch_step<float>(const D3Args<float>&, const CUtensorMap*, cudaStream_t, cudaEvent_t,
                                          cudaEvent_t);
template cudaError_t launch_step<double>(const D3Args<double>&, const CUtensorMap*, cudaStream_t, cudaEvent_t,
                                          cudaEvent_t);
template cudaError_t launch_step<__half>(const D3Args<__half>&, const CUtensorMap*, cudaStream_t, cudaEvent_t,
                                          cudaEvent_t);
template cudaError_t launch_mass<float>(const float*, const uint32_t*, const float*, const __half*, int, int, int,
                                        int, long long, double*, int, cudaStream_t);
template cudaError_t launch_mass<double>(const double*, const uint32_t*, const double*, const __half*, int, int, int,
                                         int, long long, double*, int, cudaStream_t);
template cudaError_t launch_mass<__half>(const __half*, const uint32_t*, const float*, const __half*, int, int, int,
                                         int, long long, double*, int, cudaStream_t);

}  // namespace lbm3
