// Host runtime of the D3Q19 path: validation, geometry classification,
// device state, stepping and the read-back entry points.  lbm_api.cu
// dispatches every lbm_* call on a D3Q19 context here.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_d3q19.h"
#include "lbm_d3q19_host.h"

namespace lbm3 {

namespace {

// host copy of the lattice (same order as the kernels)
const int HX_[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
const int HY_[Q] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
const int HZ_[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};

double hw(int i) {
    const int e2 = HX_[i] * HX_[i] + HY_[i] * HY_[i] + HZ_[i] * HZ_[i];
    return e2 == 0 ? 1.0 / 3.0 : (e2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

double host_feq(int i, double rho, double ux, double uy, double uz) {
    const double eu = HX_[i] * ux + HY_[i] * uy + HZ_[i] * uz;
    const double uu = ux * ux + uy * uy + uz * uz;
    return rho * hw(i) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

int hopp(int i) {
    for (int j = 0; j < Q; ++j)
        if (HX_[j] == -HX_[i] && HY_[j] == -HY_[i] && HZ_[j] == -HZ_[i]) return j;
    return 0;
}

// stored value <-> real value (FP16 storage: deviation from wr = w_i rho_ref)
template <typename S>
S enc(double v, double wr) {
    return (S)v;
}
template <>
__half enc<__half>(double v, double wr) {
    return __float2half_rn((float)(v - wr));
}
template <typename S>
double dec(S v, double wr) {
    return (double)v;
}
template <>
double dec<__half>(__half v, double wr) {
    return (double)__half2float(v) + wr;
}

}  // namespace

struct Ctx3 {
    int nx = 0, ny = 0, nz = 0, pitch = 0;
    long long plane = 0;
    int precision = LBM_FP32;
    size_t sb = 4;  // bytes per stored population
    size_t rb = 4;  // bytes per real value (densities, velocities, face state)
    cudaStream_t stream = nullptr;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    uint32_t* info = nullptr;
    void* rho = nullptr;
    void* umac = nullptr;
    int nfaces = 0;
    FaceDev3 face[6];
    int nslots = 0, have_inlet = 0, out_count = 0;
    int open_side[6] = {0, 0, 0, 0, 0, 0};
    int periodic[3] = {0, 0, 0};
    double* face_speed = nullptr;
    double* face_rho = nullptr;
    uint8_t* face_fluid = nullptr;
    void* FpF = nullptr;
    void* FpN = nullptr;
    void* fo = nullptr;
    void* fface = nullptr;
    void* unbr = nullptr;
    void* adv = nullptr;
    __half* rref[2] = {nullptr, nullptr};  // FP16 storage: [2][plane] reference densities per parity
    double* flux = nullptr;
    double* scal[2] = {nullptr, nullptr};
    unsigned int* status = nullptr;
    // FP32: tensor map of the density field as 8-byte (rho_1, rho_2) pairs,
    // box (36, 8, 8) = one collide tile and its halo
    CUtensorMap rho_map{};
    int have_rho_map = 0;
    double* mass_partial = nullptr;
    int mass_blocks = 0;
    double G[3] = {0, 0, 0}, body[3] = {0, 0, 0}, s[2][Q];
    int64_t step = 0, launches = 0;
    std::vector<uint8_t> solid;     // [nz][ny][nx]
    std::vector<uint32_t> hinfo;    // [nz][ny][pitch]
    std::vector<double> hadv;       // [3][nz][ny][pitch] adhesion vectors
    std::vector<double> face_speed_h, face_rho_h;
    // kernel timing
    int time_every = 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    double t_pull = 0.0, t_collide = 0.0;
    int64_t t_samples = 0;
    std::string err;
};

namespace {

lbm_status fail3(Ctx3* c, std::string* err, lbm_status st, const std::string& msg) {
    if (c) c->err = msg;
    if (err) *err = msg;
    return st;
}

#define CK3(call)                                                                                      \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail3(c, nullptr, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,     \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                          \
    } while (0)

size_t nbytes_f(const Ctx3* c) { return (size_t)2 * Q * c->plane * c->sb; }

void tangential(int side, int& a0, int& a1) {
    const int ax = side / 2;
    a0 = ax == 0 ? 1 : 0;
    a1 = ax == 2 ? 1 : 2;
}

long long hidx(const Ctx3* c, int x, int y, int z) { return ((long long)z * c->ny + y) * c->nx + x; }
long long didx(const Ctx3* c, int x, int y, int z) { return ((long long)z * c->ny + y) * c->pitch + x; }

// psi-site resolution on the host (ghost mirrors across open sides, periodic
// wrap, solid outside closed sides): -1 = solid
long long host_site(const Ctx3* c, int x, int y, int z) {
    int p[3] = {x, y, z};
    const int ext[3] = {c->nx, c->ny, c->nz};
    for (int a = 0; a < 3; ++a) {
        if (p[a] >= 0 && p[a] < ext[a]) continue;
        if (c->periodic[a]) p[a] = ((p[a] % ext[a]) + ext[a]) % ext[a];
        else if (p[a] < 0 && c->open_side[2 * a]) p[a] = -1 - p[a];
        else if (p[a] >= ext[a] && c->open_side[2 * a + 1]) p[a] = 2 * ext[a] - 1 - p[a];
        else return -1;
    }
    const long long h = hidx(c, p[0], p[1], p[2]);
    return c->solid[h] ? -1 : h;
}

// Node (pitched index) that pulls population i of node (x, y, z) next step:
// the neighbour x + e_i (periodic wrap), or the node itself when its pull of
// the opposite direction is blocked (bounce-back / open-face unknown).
long long reader_of(const Ctx3* c, int x, int y, int z, int i) {
    const long long d = didx(c, x, y, z);
    if (c->hinfo[d] & (1u << hopp(i))) return d;
    int p[3] = {x + HX_[i], y + HY_[i], z + HZ_[i]};
    const int ext[3] = {c->nx, c->ny, c->nz};
    for (int a = 0; a < 3; ++a) p[a] = (p[a] + ext[a]) % ext[a];
    return didx(c, p[0], p[1], p[2]);
}

// Upload populations fd [2][19][plane] (real values) into buffer `which`.
// FP16 storage also sets that parity's reference densities to the
// half-rounded sums of each node's populations and encodes every value
// against the reference of the node that pulls it.
template <typename S>
lbm_status put_f(Ctx3* c, const std::vector<double>& fd, int which) {
    std::vector<S> buf((size_t)2 * Q * c->plane, enc<S>(0.0, 0.0));
    std::vector<__half> ref;
    const bool half = std::is_same<S, __half>::value;
    if (half) {
        ref.assign((size_t)2 * c->plane, __float2half_rn(0.0f));
        for (long long d = 0; d < c->plane; ++d) {
            if (c->hinfo[d] & INFO3_SOLID) continue;
            for (int k = 0; k < 2; ++k) {
                double r = 0.0;
                for (int i = 0; i < Q; ++i) r += fd[((size_t)k * Q + i) * c->plane + d];
                ref[(size_t)k * c->plane + d] = __float2half_rn((float)r);
            }
        }
    }
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                const long long d = didx(c, x, y, z);
                if (c->hinfo[d] & INFO3_SOLID) continue;
                for (int k = 0; k < 2; ++k)
                    for (int i = 0; i < Q; ++i) {
                        double wr = 0.0;
                        if (half)
                            wr = hw(i) * (double)__half2float(ref[(size_t)k * c->plane + reader_of(c, x, y, z, i)]);
                        buf[((size_t)k * Q + i) * c->plane + d] = enc<S>(fd[((size_t)k * Q + i) * c->plane + d], wr);
                    }
            }
    CK3(cudaMemcpy(c->f[which], buf.data(), buf.size() * sizeof(S), cudaMemcpyHostToDevice));
    if (half) CK3(cudaMemcpy(c->rref[which], ref.data(), ref.size() * sizeof(__half), cudaMemcpyHostToDevice));
    return LBM_OK;
}

// Download buffer `which` as real values fd [2][19][plane].
template <typename S>
lbm_status get_f(Ctx3* c, std::vector<double>& fd, int which) {
    std::vector<S> buf((size_t)2 * Q * c->plane);
    CK3(cudaMemcpy(buf.data(), c->f[which], buf.size() * sizeof(S), cudaMemcpyDeviceToHost));
    std::vector<__half> ref;
    const bool half = std::is_same<S, __half>::value;
    if (half) {
        ref.resize((size_t)2 * c->plane);
        CK3(cudaMemcpy(ref.data(), c->rref[which], ref.size() * sizeof(__half), cudaMemcpyDeviceToHost));
    }
    fd.assign((size_t)2 * Q * c->plane, 0.0);
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                const long long d = didx(c, x, y, z);
                if (c->hinfo[d] & INFO3_SOLID) continue;
                for (int k = 0; k < 2; ++k)
                    for (int i = 0; i < Q; ++i) {
                        double wr = 0.0;
                        if (half)
                            wr = hw(i) * (double)__half2float(ref[(size_t)k * c->plane + reader_of(c, x, y, z, i)]);
                        fd[((size_t)k * Q + i) * c->plane + d] = dec<S>(buf[((size_t)k * Q + i) * c->plane + d], wr);
                    }
            }
    return LBM_OK;
}

template <typename S>
void fill_args(const Ctx3* c, D3Args<S>& a, bool write_u) {
    using T = typename Real<S>::type;
    std::memset(&a, 0, sizeof(a));
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    a.pitch = c->pitch;
    a.plane = c->plane;
    for (int q = 0; q < 3; ++q) a.periodic[q] = c->periodic[q];
    for (int q = 0; q < 6; ++q) a.open_side[q] = c->open_side[q];
    a.fin = static_cast<const S*>(c->f[c->cur]);
    a.fout = static_cast<S*>(c->f[1 - c->cur]);
    a.rref_in = c->rref[c->cur];
    a.rref_out = c->rref[1 - c->cur];
    a.info = c->info;
    a.rho = static_cast<T*>(c->rho);
    a.umac = write_u ? static_cast<T*>(c->umac) : nullptr;
    a.nfaces = c->nfaces;
    for (int q = 0; q < c->nfaces; ++q) a.face[q] = c->face[q];
    a.nface_slots = c->nslots;
    a.have_inlet = c->have_inlet;
    a.out_count = c->out_count;
    a.face_speed = c->face_speed;
    a.face_rho = c->face_rho;
    a.face_fluid = c->face_fluid;
    a.FpF = static_cast<T*>(c->FpF);
    a.FpN = static_cast<T*>(c->FpN);
    a.fo = static_cast<T*>(c->fo);
    a.fface = static_cast<T*>(c->fface);
    a.unbr = static_cast<T*>(c->unbr);
    a.adv = static_cast<const T*>(c->adv);
    a.flux = c->flux;
    a.scal_in = c->scal[c->step & 1];
    a.scal_out = c->scal[(c->step + 1) & 1];
    a.status = c->status;
    for (int q = 0; q < 3; ++q) {
        a.G[q] = (T)c->G[q];
        a.body[q] = (T)c->body[q];
    }
    for (int k = 0; k < 2; ++k)
        for (int r = 0; r < Q; ++r) a.s[k][r] = (T)c->s[k][r];
}

template <typename S>
lbm_status upload_state(Ctx3* c, const double* rho_init, const double* u_init) {
    using T = typename Real<S>::type;
    const long long N = (long long)c->nx * c->ny * c->nz;
    std::vector<double> fh((size_t)2 * Q * c->plane, 0.0);
    std::vector<T> rh((size_t)2 * c->plane, T(0)), uh((size_t)3 * c->plane, T(0));
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                const long long h = hidx(c, x, y, z), d = didx(c, x, y, z);
                if (c->solid[h]) continue;  // (0, 0) in the density field: psi = 0 there
                double u[3];
                for (int a = 0; a < 3; ++a) u[a] = u_init ? u_init[(size_t)a * N + h] : 0.0;
                for (int k = 0; k < 2; ++k) {
                    const double r = rho_init[(size_t)k * N + h];
                    rh[2 * (size_t)d + k] = (T)r;
                    for (int i = 0; i < Q; ++i) fh[((size_t)k * Q + i) * c->plane + d] = host_feq(i, r, u[0], u[1], u[2]);
                }
                for (int a = 0; a < 3; ++a) uh[(size_t)a * c->plane + d] = (T)u[a];
            }
    c->cur = 0;
    CK3(cudaStreamSynchronize(c->stream));
    lbm_status pst = put_f<S>(c, fh, 0);
    if (pst != LBM_OK) return pst;
    CK3(cudaMemsetAsync(c->f[1], 0, nbytes_f(c), c->stream));
    CK3(cudaMemcpyAsync(c->rho, rh.data(), rh.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    CK3(cudaMemcpyAsync(c->umac, uh.data(), uh.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    // open-face state: outlet "previous" populations = the initial ones,
    // lagged forces 0, lambda 0, chi 1
    if (c->nslots > 0) {
        std::vector<T> fo((size_t)c->nslots * 2 * Q, T(0));
        for (int fi = 0; fi < c->nfaces; ++fi) {
            const FaceDev3& F = c->face[fi];
            for (int q = 0; q < F.count; ++q) {
                int p[3];
                const int ext[3] = {c->nx, c->ny, c->nz};
                p[F.axis] = (F.side & 1) ? ext[F.axis] - 1 : 0;
                p[F.a0] = F.lo0 + q % F.len0;
                p[F.a1] = F.lo1 + q / F.len0;
                const long long d = didx(c, p[0], p[1], p[2]);
                for (int k = 0; k < 2; ++k)
                    for (int i = 0; i < Q; ++i)
                        fo[((size_t)(F.base + q) * 2 + k) * Q + i] = (T)fh[((size_t)k * Q + i) * c->plane + d];
            }
        }
        CK3(cudaMemcpyAsync(c->fo, fo.data(), fo.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
        CK3(cudaStreamSynchronize(c->stream));
        CK3(cudaMemsetAsync(c->FpF, 0, (size_t)c->nslots * 6 * c->rb, c->stream));
        CK3(cudaMemsetAsync(c->FpN, 0, (size_t)c->nslots * 6 * c->rb, c->stream));
    }
    double sc[SC3_N] = {0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    CK3(cudaMemcpyAsync(c->scal[0], sc, sizeof(sc), cudaMemcpyHostToDevice, c->stream));
    CK3(cudaMemcpyAsync(c->scal[1], sc, sizeof(sc), cudaMemcpyHostToDevice, c->stream));
    CK3(cudaMemsetAsync(c->status, 0, sizeof(unsigned int), c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    c->step = 0;
    return LBM_OK;
}

// FP32 contexts: tensor map of the density field ([plane] pairs of floats as
// 8-byte elements over x, y, z) for the collide kernel's one-copy staging of
// interior tiles.  Without the driver entry point the kernel stages with
// loads instead (same values).
void make_rho_map(Ctx3* c) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    c->have_rho_map = 0;
    if (c->precision != LBM_FP32) return;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)c->pitch, (cuuint64_t)c->ny, (cuuint64_t)c->nz};
    const cuuint64_t strides[2] = {(cuuint64_t)c->pitch * 8, (cuuint64_t)c->pitch * 8 * (cuuint64_t)c->ny};
    const cuuint32_t box[3] = {(cuuint32_t)RHO_BOX3_X, (cuuint32_t)RHO_BOX3_Y, (cuuint32_t)RHO_BOX3_Z};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = reinterpret_cast<Encode>(fn)(&c->rho_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, c->rho, dims,
                                                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    c->have_rho_map = r == CUDA_SUCCESS ? 1 : 0;
}

lbm_status check_status3(Ctx3* c) {
    unsigned int st = 0;
    CK3(cudaMemcpyAsync(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    if (st & STATUS3_TIMEOUT)
        return fail3(c, nullptr, LBM_ERR_TIMEOUT, "a bounded wait on the density-box tensor copy ran out");
    if (st) return fail3(c, nullptr, LBM_ERR_DIVERGED, "non-finite density or velocity produced");
    return LBM_OK;
}

}  // namespace

void destroy(Ctx3* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    void* p[] = {c->f[0], c->f[1], c->info, c->rho, c->umac, c->face_speed, c->face_rho, c->face_fluid, c->FpF,
                 c->FpN, c->fo, c->fface, c->unbr, c->adv, c->flux, c->scal[0], c->scal[1], c->status, c->mass_partial};
    for (void* q : p)
        if (q) cudaFree(q);
    for (__half* q : c->rref)
        if (q) cudaFree(q);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

const char* error(const Ctx3* c) { return c->err.c_str(); }

lbm_status create(const lbm_grid* g, const lbm_params* p, const lbm_open_bc* bcs, int nbc, const uint8_t* solid,
                  const double* rho_init, const double* u_init, void* stream, Ctx3** out, std::string* err) {
    Ctx3* c = nullptr;
    *out = nullptr;
    if (g->nx < 5 || g->ny < 5 || g->nz < 5)
        return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "extent: every D3Q19 axis needs >= 5 nodes");
    if ((long long)g->nx * g->ny * g->nz > (1ll << 31) - 1)
        return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "extent: grid too large");
    if (p->precision != LBM_FP32 && p->precision != LBM_FP64 && p->precision != LBM_FP32_FP16STORE)
        return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "unknown precision");
    if (!(p->nu[0] > 0.0) || !(p->nu[1] > 0.0)) return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "viscosities must be > 0");
    if (nbc < 0 || nbc > 6 || (nbc > 0 && !bcs)) return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "bad face list");
    if (!rho_init) return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "rho_init is NULL");

    c = new (std::nothrow) Ctx3();
    if (!c) return fail3(nullptr, err, LBM_ERR_OOM, "host allocation failed");
    c->nx = g->nx;
    c->ny = g->ny;
    c->nz = g->nz;
    c->pitch = (g->nx + 31) / 32 * 32;
    c->plane = (long long)c->pitch * c->ny * c->nz;
    c->precision = p->precision;
    c->sb = p->precision == LBM_FP64 ? 8 : (p->precision == LBM_FP32_FP16STORE ? 2 : 4);
    c->rb = p->precision == LBM_FP64 ? 8 : 4;
    c->stream = static_cast<cudaStream_t>(stream);
    for (int a = 0; a < 3; ++a) c->periodic[a] = g->periodic[a] ? 1 : 0;
    const long long N = (long long)c->nx * c->ny * c->nz;
    c->solid.assign((size_t)N, 0);
    if (solid)
        for (long long h = 0; h < N; ++h) c->solid[h] = solid[h] ? 1 : 0;

    // relaxation rates: S = diag[1, s_e, s_eps, 1, s_q, 1, s_q, 1, s_q, s_nu,
    // s_pi, s_nu, s_pi, s_nu, s_nu, s_nu, s_m, s_m, s_m], s_pi = s_eps, s_m = s_q
    const double numax = std::max(p->nu[0], p->nu[1]);
    const double sq = p->s_q > 0.0 ? p->s_q : 1.2;
    for (int k = 0; k < 2; ++k) {
        const double snu = 1.0 / (3.0 * p->nu[k] + 0.5);
        const double seps = p->s_eps_mode == LBM_SEPS_MAX_NU ? 1.0 / (3.0 * numax + 0.5) : snu;
        const double se = p->s_e > 0.0 ? p->s_e : snu;
        const double s[Q] = {1.0, se, seps, 1.0, sq, 1.0, sq, 1.0, sq, snu, seps, snu, seps, snu, snu, snu, sq, sq, sq};
        for (int r = 0; r < Q; ++r) {
            if (!(s[r] > 0.0 && s[r] < 2.0)) {
                destroy(c);
                return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "relaxation rate outside (0, 2)");
            }
            c->s[k][r] = s[r];
        }
    }
    c->G[0] = p->G12;
    c->G[1] = p->Gw[0];
    c->G[2] = p->Gw[1];
    for (int a = 0; a < 3; ++a) c->body[a] = p->body_force[a];

    // faces
    const int ext[3] = {c->nx, c->ny, c->nz};
    std::vector<int> faceid((size_t)N, 0), nbrid((size_t)N, 0);
    int nout = 0, slots = 0;
    c->nfaces = nbc;
    for (int f = 0; f < nbc; ++f) {
        const lbm_open_bc& b = bcs[f];
        FaceDev3& F = c->face[f];
        std::memset(&F, 0, sizeof(F));
        if (b.kind != LBM_INLET_VELOCITY && b.kind != LBM_OUTLET_CONVECTIVE) {
            destroy(c);
            return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "face kind");
        }
        if (b.side < 0 || b.side > 5 || c->periodic[b.side / 2]) {
            destroy(c);
            return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "face side (none on a periodic axis)");
        }
        F.kind = b.kind == LBM_INLET_VELOCITY ? FACE3_INLET : FACE3_OUTLET;
        F.side = b.side;
        F.axis = b.side / 2;
        F.o[F.axis] = (b.side & 1) ? 1 : -1;
        tangential(b.side, F.a0, F.a1);
        if (b.lo[0] < 0 || b.hi[0] >= ext[F.a0] || b.lo[0] > b.hi[0] || b.lo[1] < 0 || b.hi[1] >= ext[F.a1] ||
            b.lo[1] > b.hi[1]) {
            destroy(c);
            return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "face extent");
        }
        F.lo0 = b.lo[0];
        F.lo1 = b.lo[1];
        F.len0 = b.hi[0] - b.lo[0] + 1;
        F.len1 = b.hi[1] - b.lo[1] + 1;
        F.base = slots;
        F.count = F.len0 * F.len1;
        slots += F.count;
        F.alpha = b.alpha_correction ? 1 : 0;
        F.chi = b.chi_correction ? 1 : 0;
        for (int i = 0; i < Q; ++i) {
            const int en = HX_[i] * F.o[0] + HY_[i] * F.o[1] + HZ_[i] * F.o[2];
            if (en >= 0) continue;
            F.sa[0] += HX_[i] * HX_[i] * hw(i);
            F.sa[1] += HY_[i] * HY_[i] * hw(i);
            F.sa[2] += HZ_[i] * HZ_[i] * hw(i);
        }
        if (F.kind == FACE3_OUTLET) ++nout;
        else c->have_inlet = 1;
        c->open_side[b.side] = 1;
    }
    if (nout > 1) {
        destroy(c);
        return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "at most one outlet face");
    }
    c->nslots = slots;
    c->face_speed_h.assign((size_t)slots, 0.0);
    c->face_rho_h.assign((size_t)2 * slots, 0.0);
    std::vector<uint8_t> ffl((size_t)std::max(1, slots), 0);
    for (int f = 0; f < nbc; ++f) {
        const lbm_open_bc& b = bcs[f];
        const FaceDev3& F = c->face[f];
        for (int q = 0; q < F.count; ++q) {
            int pp[3];
            pp[F.axis] = (F.side & 1) ? ext[F.axis] - 1 : 0;
            pp[F.a0] = F.lo0 + q % F.len0;
            pp[F.a1] = F.lo1 + q / F.len0;
            const long long h = hidx(c, pp[0], pp[1], pp[2]);
            const int slot = F.base + q;
            c->face_speed_h[slot] = (F.kind == FACE3_INLET && b.u_profile) ? b.u_profile[q] : 0.0;
            for (int k = 0; k < 2; ++k)
                c->face_rho_h[(size_t)k * slots + slot] =
                    b.rho_profile ? b.rho_profile[(size_t)k * F.count + q] : b.rho_in[k];
            if (c->solid[h]) continue;
            if (faceid[h]) {
                destroy(c);
                return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "a node lies on two faces");
            }
            faceid[h] = f + 1;
            ffl[slot] = 1;
            if (F.kind == FACE3_OUTLET) ++c->out_count;
        }
    }
    for (int f = 0; f < nbc; ++f) {
        const FaceDev3& F = c->face[f];
        for (int q = 0; q < F.count; ++q) {
            int pp[3];
            pp[F.axis] = (F.side & 1) ? ext[F.axis] - 1 : 0;
            pp[F.a0] = F.lo0 + q % F.len0;
            pp[F.a1] = F.lo1 + q / F.len0;
            if (c->solid[hidx(c, pp[0], pp[1], pp[2])]) continue;
            const long long h2 = hidx(c, pp[0] - F.o[0], pp[1] - F.o[1], pp[2] - F.o[2]);
            if (c->solid[h2] || faceid[h2]) {
                destroy(c);
                return fail3(nullptr, err, LBM_ERR_INVALID_ARG,
                             "the inward neighbour of a face node must be an ordinary fluid node");
            }
            if (nbrid[h2]) {
                destroy(c);
                return fail3(nullptr, err, LBM_ERR_INVALID_ARG, "a node is the inward neighbour of two faces");
            }
            nbrid[h2] = f + 1;
        }
    }

    // info words
    c->hinfo.assign((size_t)c->plane, INFO3_SOLID);
    c->hadv.assign((size_t)3 * c->plane, 0.0);
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                const long long h = hidx(c, x, y, z);
                uint32_t w = 0;
                if (c->solid[h]) {
                    c->hinfo[didx(c, x, y, z)] = INFO3_SOLID;
                    continue;
                }
                for (int i = 0; i < Q; ++i) {
                    int pp[3] = {x - HX_[i], y - HY_[i], z - HZ_[i]};
                    bool blocked = false;
                    for (int a = 0; a < 3 && !blocked; ++a) {
                        if (pp[a] >= 0 && pp[a] < ext[a]) continue;
                        if (!c->periodic[a]) blocked = true;
                        else {
                            pp[a] = (pp[a] + ext[a]) % ext[a];
                            w |= INFO3_WRAP;
                        }
                    }
                    if (!blocked && c->solid[hidx(c, pp[0], pp[1], pp[2])]) blocked = true;
                    if (blocked) w |= 1u << i;
                }
                w |= (uint32_t)faceid[h] << INFO3_FACE_SHIFT;
                w |= (uint32_t)nbrid[h] << INFO3_NBR_SHIFT;
                // sum_e w s(x+e) e over the 8th-order stencil (Eq. 11)
                static const int W5040[9] = {0, 448, 240, 96, 50, 16, 8, 0, 1};
                double adh[3] = {0.0, 0.0, 0.0};
                bool near = false;
                for (int dz = -2; dz <= 2; ++dz)
                    for (int dy = -2; dy <= 2; ++dy)
                        for (int dx = -2; dx <= 2; ++dx) {
                            const int r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 == 0 || r2 > 8 || W5040[r2] == 0) continue;
                            if (host_site(c, x + dx, y + dy, z + dz) >= 0) continue;
                            near = true;
                            const double wgt = W5040[r2] / 5040.0;
                            adh[0] += wgt * dx;
                            adh[1] += wgt * dy;
                            adh[2] += wgt * dz;
                        }
                if (near) {
                    w |= INFO3_NEAR_SOLID;
                    for (int q = 0; q < 3; ++q) c->hadv[(size_t)q * c->plane + didx(c, x, y, z)] = adh[q];
                }
                c->hinfo[didx(c, x, y, z)] = w;
            }

    // device allocations
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
    };
    alloc(&c->f[0], nbytes_f(c));
    alloc(&c->f[1], nbytes_f(c));
    alloc((void**)&c->info, (size_t)c->plane * sizeof(uint32_t));
    alloc(&c->rho, (size_t)2 * c->plane * c->rb);
    alloc(&c->umac, (size_t)3 * c->plane * c->rb);
    alloc((void**)&c->face_speed, (size_t)slots * sizeof(double));
    alloc((void**)&c->face_rho, (size_t)2 * slots * sizeof(double));
    alloc((void**)&c->face_fluid, (size_t)slots);
    alloc(&c->FpF, (size_t)slots * 6 * c->rb);
    alloc(&c->FpN, (size_t)slots * 6 * c->rb);
    alloc(&c->fo, (size_t)slots * 2 * Q * c->rb);
    alloc(&c->fface, (size_t)slots * 2 * Q * c->rb);
    if (c->precision == LBM_FP32_FP16STORE) {
        alloc((void**)&c->rref[0], (size_t)2 * c->plane * sizeof(__half));
        alloc((void**)&c->rref[1], (size_t)2 * c->plane * sizeof(__half));
    }
    alloc(&c->unbr, (size_t)slots * 3 * c->rb);
    alloc(&c->adv, (size_t)3 * c->plane * c->rb);
    alloc((void**)&c->flux, (size_t)slots * 2 * sizeof(double));
    alloc((void**)&c->scal[0], SC3_N * sizeof(double));
    alloc((void**)&c->scal[1], SC3_N * sizeof(double));
    alloc((void**)&c->status, sizeof(unsigned int));
    c->mass_blocks = 304;
    alloc((void**)&c->mass_partial, (size_t)c->mass_blocks * 3 * sizeof(double));
    if (e != cudaSuccess) {
        const std::string msg = std::string("device allocation: ") + cudaGetErrorString(e);
        const lbm_status st = e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
        destroy(c);
        return fail3(nullptr, err, st, msg);
    }
    e = cudaMemcpy(c->info, c->hinfo.data(), c->hinfo.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (c->rb == 8) {
            e = cudaMemcpy(c->adv, c->hadv.data(), c->hadv.size() * sizeof(double), cudaMemcpyHostToDevice);
        } else {
            std::vector<float> af(c->hadv.begin(), c->hadv.end());
            e = cudaMemcpy(c->adv, af.data(), af.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
    }
    std::vector<double>().swap(c->hadv);
    if (e == cudaSuccess && slots > 0) {
        e = cudaMemcpy(c->face_speed, c->face_speed_h.data(), (size_t)slots * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->face_rho, c->face_rho_h.data(), (size_t)2 * slots * sizeof(double),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->face_fluid, ffl.data(), (size_t)slots, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(c->flux, 0, (size_t)slots * 2 * sizeof(double));
    }
    if (e != cudaSuccess) {
        const std::string msg = std::string("upload: ") + cudaGetErrorString(e);
        destroy(c);
        return fail3(nullptr, err, LBM_ERR_CUDA, msg);
    }
    make_rho_map(c);
    const lbm_status st = c->sb == 8   ? upload_state<double>(c, rho_init, u_init)
                          : c->sb == 2 ? upload_state<__half>(c, rho_init, u_init)
                                       : upload_state<float>(c, rho_init, u_init);
    if (st != LBM_OK) {
        if (err) *err = c->err;
        destroy(c);
        return st;
    }
    *out = c;
    return LBM_OK;
}

lbm_status reset(Ctx3* c, const double* rho_init, const double* u_init) {
    if (!rho_init) return fail3(c, nullptr, LBM_ERR_INVALID_ARG, "rho_init is NULL");
    CK3(cudaStreamSynchronize(c->stream));
    return c->sb == 8   ? upload_state<double>(c, rho_init, u_init)
           : c->sb == 2 ? upload_state<__half>(c, rho_init, u_init)
                        : upload_state<float>(c, rho_init, u_init);
}

lbm_status step(Ctx3* c, int64_t nsteps) {
    if (nsteps < 0) return fail3(c, nullptr, LBM_ERR_INVALID_ARG, "nsteps must be >= 0");
    for (int64_t s = 0; s < nsteps; ++s) {
        const bool timed = c->time_every > 0 && (c->step % c->time_every) == 0;
        cudaError_t e;
        if (timed) cudaEventRecord(c->ev[0], c->stream);
        if (c->sb == 8) {
            D3Args<double> a;
            fill_args(c, a, true);
            e = launch_step<double>(a, nullptr, c->stream, timed ? c->ev[1] : nullptr,
                                 timed ? c->ev[2] : nullptr);
        } else if (c->sb == 2) {
            D3Args<__half> a;
            fill_args(c, a, true);
            e = launch_step<__half>(a, nullptr, c->stream, timed ? c->ev[1] : nullptr,
                                 timed ? c->ev[2] : nullptr);
        } else {
            D3Args<float> a;
            fill_args(c, a, true);
            e = launch_step<float>(a, c->have_rho_map ? &c->rho_map : nullptr, c->stream, timed ? c->ev[1] : nullptr,
                                 timed ? c->ev[2] : nullptr);
        }
        if (e != cudaSuccess) return fail3(c, nullptr, LBM_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
        if (timed) {
            CK3(cudaEventSynchronize(c->ev[2]));
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, c->ev[0], c->ev[1]);
            cudaEventElapsedTime(&b, c->ev[1], c->ev[2]);
            c->t_pull += a;
            c->t_collide += b;
            ++c->t_samples;
        }
        c->launches += c->nslots > 0 ? 5 : 2;
        c->cur = 1 - c->cur;
        ++c->step;
    }
    return LBM_OK;
}

lbm_status sync(Ctx3* c) {
    CK3(cudaStreamSynchronize(c->stream));
    return check_status3(c);
}

lbm_status enable_timing(Ctx3* c, int every) {
    if (every < 0) return fail3(c, nullptr, LBM_ERR_INVALID_ARG, "every must be >= 0");
    for (cudaEvent_t& ev : c->ev)
        if (!ev) CK3(cudaEventCreate(&ev));
    c->time_every = every;
    c->t_pull = c->t_collide = 0.0;
    c->t_samples = 0;
    return LBM_OK;
}

lbm_status kernel_time_split(Ctx3* c, double* pull_ms, double* collide_ms, int64_t* samples) {
    CK3(cudaStreamSynchronize(c->stream));
    const double n = c->t_samples > 0 ? (double)c->t_samples : 1.0;
    if (pull_ms) *pull_ms = c->t_pull / n;
    if (collide_ms) *collide_ms = c->t_collide / n;
    if (samples) *samples = c->t_samples;
    return LBM_OK;
}

template <typename T, typename O>
static lbm_status macros_impl(Ctx3* c, O* rho, O* u, bool dst_dev) {
    const long long N = (long long)c->nx * c->ny * c->nz;
    CK3(cudaStreamSynchronize(c->stream));
    std::vector<T> r((size_t)2 * c->plane), uu((size_t)3 * c->plane);
    CK3(cudaMemcpy(r.data(), c->rho, r.size() * sizeof(T), cudaMemcpyDeviceToHost));
    CK3(cudaMemcpy(uu.data(), c->umac, uu.size() * sizeof(T), cudaMemcpyDeviceToHost));
    std::vector<O> ro((size_t)2 * N), uo((size_t)3 * N);
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                const long long h = hidx(c, x, y, z), d = didx(c, x, y, z);
                const bool s = c->solid[h] != 0;
                for (int k = 0; k < 2; ++k) ro[(size_t)k * N + h] = s ? O(0) : (O)r[2 * (size_t)d + k];
                for (int a = 0; a < 3; ++a) uo[(size_t)a * N + h] = s ? O(0) : (O)uu[(size_t)a * c->plane + d];
            }
    if (dst_dev) {
        CK3(cudaMemcpy(rho, ro.data(), ro.size() * sizeof(O), cudaMemcpyHostToDevice));
        CK3(cudaMemcpy(u, uo.data(), uo.size() * sizeof(O), cudaMemcpyHostToDevice));
    } else {
        std::memcpy(rho, ro.data(), ro.size() * sizeof(O));
        std::memcpy(u, uo.data(), uo.size() * sizeof(O));
    }
    return LBM_OK;
}

lbm_status get_macros(Ctx3* c, float* rho, float* u, int dst_is_device) {
    lbm_status st = check_status3(c);
    if (st != LBM_OK) return st;
    return c->rb == 8 ? macros_impl<double, float>(c, rho, u, dst_is_device != 0)
                      : macros_impl<float, float>(c, rho, u, dst_is_device != 0);
}

lbm_status get_macros_f64(Ctx3* c, double* rho, double* u) {
    lbm_status st = check_status3(c);
    if (st != LBM_OK) return st;
    return c->rb == 8 ? macros_impl<double, double>(c, rho, u, false) : macros_impl<float, double>(c, rho, u, false);
}

template <typename S>
static lbm_status pops_impl(Ctx3* c, double* f, const double* fin) {
    const long long N = (long long)c->nx * c->ny * c->nz;
    CK3(cudaStreamSynchronize(c->stream));
    std::vector<double> fd;
    if (!fin) {
        lbm_status st = get_f<S>(c, fd, c->cur);
        if (st != LBM_OK) return st;
    } else {
        fd.assign((size_t)2 * Q * c->plane, 0.0);
    }
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                const long long h = hidx(c, x, y, z), d = didx(c, x, y, z);
                for (int q = 0; q < 2 * Q; ++q) {
                    if (fin) fd[(size_t)q * c->plane + d] = c->solid[h] ? 0.0 : fin[(size_t)q * N + h];
                    else f[(size_t)q * N + h] = c->solid[h] ? 0.0 : fd[(size_t)q * c->plane + d];
                }
            }
    if (fin) return put_f<S>(c, fd, c->cur);
    return LBM_OK;
}

lbm_status get_populations(Ctx3* c, double* f) {
    return c->sb == 8 ? pops_impl<double>(c, f, nullptr)
                      : (c->sb == 2 ? pops_impl<__half>(c, f, nullptr) : pops_impl<float>(c, f, nullptr));
}

lbm_status set_populations(Ctx3* c, const double* f) {
    return c->sb == 8 ? pops_impl<double>(c, nullptr, f)
                      : (c->sb == 2 ? pops_impl<__half>(c, nullptr, f) : pops_impl<float>(c, nullptr, f));
}

lbm_status diagnostics(Ctx3* c, lbm_diag* d) {
    cudaError_t e;
    if (c->sb == 8)
        e = launch_mass<double>((const double*)c->f[c->cur], c->info, (const double*)c->umac, nullptr, c->nx, c->ny,
                                c->nz, c->pitch, c->plane, c->mass_partial, c->mass_blocks, c->stream);
    else if (c->sb == 2)
        e = launch_mass<__half>((const __half*)c->f[c->cur], c->info, (const float*)c->umac, c->rref[c->cur], c->nx,
                                c->ny, c->nz, c->pitch, c->plane, c->mass_partial, c->mass_blocks, c->stream);
    else
        e = launch_mass<float>((const float*)c->f[c->cur], c->info, (const float*)c->umac, nullptr, c->nx, c->ny,
                               c->nz, c->pitch, c->plane, c->mass_partial, c->mass_blocks, c->stream);
    if (e != cudaSuccess) return fail3(c, nullptr, LBM_ERR_CUDA, std::string("diagnostics: ") + cudaGetErrorString(e));
    ++c->launches;
    std::vector<double> part((size_t)c->mass_blocks * 3);
    double sc[SC3_N];
    unsigned int st = 0;
    CK3(cudaMemcpyAsync(part.data(), c->mass_partial, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaMemcpyAsync(sc, c->scal[c->step & 1], sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaMemcpyAsync(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    double m0 = 0.0, m1 = 0.0, u2 = 0.0;
    for (int b = 0; b < c->mass_blocks; ++b) {
        m0 += part[(size_t)b * 3];
        m1 += part[(size_t)b * 3 + 1];
        u2 = std::max(u2, part[(size_t)b * 3 + 2]);
    }
    d->mass[0] = m0;
    d->mass[1] = m1;
    d->lambda = sc[SC3_LAMBDA];
    d->chi = sc[SC3_CHI];
    d->q_in = sc[SC3_QIN];
    d->q_out = sc[SC3_QOUT];
    d->max_speed = std::sqrt(u2);
    d->step = c->step;
    d->launches = c->launches;
    d->status = st ? LBM_ERR_DIVERGED : LBM_OK;
    return LBM_OK;
}

}  // namespace lbm3
