// Host runtime behind the C ABI of include/lbm.h: parameter validation,
// per-node descriptors, device allocation, the step loop over the fused
// kernel, FP64 diagnostics and checkpoints.
#include <cuda_fp16.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_d3q19_host.h"

using namespace lbm;

namespace {
thread_local char g_thread_err[512] = "";
}  // namespace

void lbm::set_thread_error(const char* msg) {
    std::snprintf(g_thread_err, sizeof g_thread_err, "%s", msg ? msg : "");
}

namespace {

constexpr int kEx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int kEy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
constexpr double kW[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                          1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

double host_feq(int i, double rho, double ux, double uy) {
    const double eu = kEx[i] * ux + kEy[i] * uy;
    const double uu = ux * ux + uy * uy;
    return kW[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

void side_normal(int side, int* ox, int* oy) {
    *ox = side == 0 ? -1 : (side == 1 ? 1 : 0);
    *oy = side == 2 ? -1 : (side == 3 ? 1 : 0);
}

}  // namespace

struct lbm_ctx {
    lbm3::Ctx3* d3 = nullptr;  // non-null: a D3Q19 context (lbm_d3q19_host.cu owns it)
    lbm_grid grid{};
    lbm_params params{};
    int nx = 0, ny = 0, pitch = 0;
    int plane = 0;
    int precision = LBM_FP32;
    size_t sbytes = 4;  // bytes per stored population
    size_t rbytes = 4;  // bytes per arithmetic value (aux + macro buffers)
    cudaStream_t stream = nullptr;
    int device = 0;
    void* f[2] = {nullptr, nullptr};
    uint16_t* info = nullptr;
    int* blocks = nullptr;          // tile list: fast tiles first, then general tiles
    uint8_t* block_flags = nullptr;
    unsigned* block_strips = nullptr;
    int nfast = 0, ngeneral = 0;
    int64_t fast_nodes = 0, general_nodes = 0;  // fluid nodes owned by each tile list
    // column-marching variant: runs of interior tiles, one CTA each
    int4* march_runs = nullptr;
    uint8_t* march_flags = nullptr;
    int nmarch = 0, march_tiles = 0;
    CUtensorMap tmap[2];  // TMA descriptors of f[0], f[1] as [18][ny][pitch] floats
    int have_tmap = 0;
    int64_t tiling_gen = 0;                      // bumped whenever the tile lists are rebuilt
    void* uin = nullptr;
    void* Fp[2] = {nullptr, nullptr};
    void* fo[2] = {nullptr, nullptr};
    double* scal[2] = {nullptr, nullptr};
    double* partials[2] = {nullptr, nullptr};  // FP64 flux partials per tile slot, ping-pong
    int* block_slot = nullptr;
    unsigned int* status = nullptr;
    void* macro = nullptr;
    void* rref[2] = {nullptr, nullptr};  // FP16 storage: per-node half reference densities [2][plane]
    std::vector<uint16_t> h_info;        // host copy of the per-node descriptors
    double* diag_partials = nullptr;
    int diag_blocks = 0;
    int nslots = 0;
    int nfaces = 0;
    FaceDev faces[MAX_FACES]{};
    int out_face = -1, have_inlet = 0;
    int open_side[4] = {0, 0, 0, 0};
    int nface_nodes = 0;
    int xoff = 0, yoff = 0, variant = 0, tx = 32, ty = 8;
    dim3 gdim;
    int cur = 0;
    int64_t step = 0;
    int64_t launches = 0;
    double s[2][9]{};
    // CUDA-graph replay of step runs: one executable graph per starting parity
    int use_graphs = 1;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int gexec_early[2] = {0, 0};  // the graph of that parity launches its steps early
    // sampled per-launch timing
    std::vector<int> h_faceid, h_nbrid;  // per node (unpitched): face id + 1, inward-neighbour face id + 1
    std::vector<uint8_t> host_solid;   // pitched copy of the solid mask
    std::vector<uint8_t> host_solid_in;  // unpitched mask (re-initialisation)
    void* stage = nullptr;             // pinned staging buffer for host transfers
    size_t stage_bytes = 0;
    int timing_every = 0;
    // same-step chi (Eq. 23 at t + dt): outlet-node state between the general
    // tiles and d2q9_outlet_chi_kernel, [slot][OC_STRIDE]
    int chi_same_step = 0;
    void* oc_state = nullptr;
    // moving walls beyond the closed edges y = 0 / y = ny - 1 (x-velocity)
    double wall_ux[2] = {0.0, 0.0};
    double wet_delta = 0.0;  // > 0: Eq. 12's phase-dependent adhesion coefficient
    // persistent schedule of a single context: a batch of one member
    int schedule = LBM_SCHEDULE_GRAPHS;
    lbm_batch* solo = nullptr;
    std::vector<cudaEvent_t> ev_start, ev_mid, ev_stop;
    int n_samples = 0;
    std::string err;
};

namespace {

lbm_status fail(lbm_ctx* c, lbm_status st, const std::string& msg) {
    if (c) c->err = msg;
    else lbm::set_thread_error(msg.c_str());
    return st;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
    return fail(c, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                         \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);           \
    } while (0)

constexpr int kGraphSteps = 32;  // even: a replay leaves the ping-pong parity unchanged

// Early-launch step graphs (LBM_SCHEDULE_GRAPHS_EARLY): every edge between
// two kernel nodes of a captured step graph becomes a programmatic edge that
// fires once all CTAs of the upstream kernel have started.  The downstream
// kernel is then launched while the upstream one still runs, and its CTAs
// wait on the device (griddepcontrol.wait at the top of every step kernel)
// until the upstream grids have completed and their writes are visible:
// the order of all memory accesses is that of the plain graph, only the
// launch latency between steps is hidden.
cudaError_t early_launch_edges(cudaGraph_t g) {
    size_t n = 0;
    cudaError_t e = cudaGraphGetEdges(g, nullptr, nullptr, nullptr, &n);
    if (e != cudaSuccess || n == 0) return e;
    std::vector<cudaGraphNode_t> from(n), to(n);
    std::vector<cudaGraphEdgeData> ed(n);
    e = cudaGraphGetEdges(g, from.data(), to.data(), ed.data(), &n);
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
        cudaGraphNodeType tf, tt;
        e = cudaGraphNodeGetType(from[i], &tf);
        if (e == cudaSuccess) e = cudaGraphNodeGetType(to[i], &tt);
        if (e != cudaSuccess) break;
        if (tf != cudaGraphNodeTypeKernel || tt != cudaGraphNodeTypeKernel ||
            ed[i].type != cudaGraphDependencyTypeDefault || ed[i].from_port != cudaGraphKernelNodePortDefault)
            continue;
        e = cudaGraphRemoveDependencies(g, &from[i], &to[i], &ed[i], 1);
        cudaGraphEdgeData pe{};
        pe.from_port = cudaGraphKernelNodePortLaunchCompletion;
        pe.type = cudaGraphDependencyTypeProgrammatic;
        if (e == cudaSuccess) e = cudaGraphAddDependencies(g, &from[i], &to[i], &pe, 1);
    }
    return e;
}

// Instantiate a captured step graph.  early: first the early-launch form;
// if the driver refuses it, the plain graph (*early_used tells which).
cudaError_t instantiate_step_graph(cudaGraph_t g, bool early, cudaGraphExec_t* out, int* early_used) {
    *early_used = 0;
    if (early) {
        cudaGraph_t eg = nullptr;
        cudaError_t e = cudaGraphClone(&eg, g);
        if (e == cudaSuccess) e = early_launch_edges(eg);
        if (e == cudaSuccess) e = cudaGraphInstantiate(out, eg, 0);
        if (eg) cudaGraphDestroy(eg);
        if (e == cudaSuccess) {
            *early_used = 1;
            return e;
        }
        *out = nullptr;
        cudaGetLastError();
    }
    return cudaGraphInstantiate(out, g, 0);
}
constexpr int kPersistSteps = 1024;  // steps per persistent launch
// clock64 budget of one grid-barrier wait: ~1 s at the 2.07 GHz SM clock,
// several hundred times the longest step of any batch measured
constexpr long long kDefaultSpinLimit = 2000000000LL;
constexpr int kMaxSamples = 4096;

void free_ctx(lbm_ctx* c) {
    if (!c) return;
    if (c->solo) lbm_batch_destroy(c->solo);
    for (int p = 0; p < 2; ++p)
        if (c->gexec[p]) cudaGraphExecDestroy(c->gexec[p]);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (cudaEvent_t e : c->ev_start) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_mid) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_stop) cudaEventDestroy(e);
    void* ptrs[] = {c->oc_state, c->march_runs, c->march_flags, c->f[0], c->f[1], c->info, c->blocks, c->block_flags, c->block_strips, c->uin, c->Fp[0], c->Fp[1], c->fo[0], c->fo[1],
                    c->scal[0], c->scal[1], c->partials[0], c->partials[1], c->block_slot, c->status,
                    c->macro, c->diag_partials, c->rref[0], c->rref[1]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->stage) cudaFreeHost(c->stage);
    delete c;
}

template <typename S, typename R>
D2Args<S, R> make_args_par(lbm_ctx* c, int in, bool write_macros) {
    D2Args<S, R> a{};
    const int out = 1 - in;
    a.nx = c->nx;
    a.ny = c->ny;
    a.pitch = c->pitch;
    a.plane = c->plane;
    a.px = c->grid.periodic[0] ? 1 : 0;
    a.py = c->grid.periodic[1] ? 1 : 0;
    for (int i = 0; i < 4; ++i) a.open_side[i] = c->open_side[i];
    a.xoff = c->xoff;
    a.yoff = c->yoff;
    a.fin = static_cast<const S*>(c->f[in]);
    a.fout = static_cast<S*>(c->f[out]);
    a.info = c->info;
    a.blocks = c->blocks;
    a.block_flags = c->block_flags;
    a.block_slot = c->block_slot;
    a.block_strips = c->block_strips;
    a.list_off = 0;
    a.nfaces = c->nfaces;
    for (int i = 0; i < c->nfaces; ++i) a.face[i] = c->faces[i];
    a.out_face = c->out_face;
    a.have_inlet = c->have_inlet;
    a.uin = static_cast<const R*>(c->uin);
    a.Fp_in = static_cast<const R*>(c->Fp[in]);
    a.Fp_out = static_cast<R*>(c->Fp[out]);
    a.fo_in = static_cast<const R*>(c->fo[in]);
    a.fo_out = static_cast<R*>(c->fo[out]);
    a.scal_in = c->scal[in];
    a.scal_out = c->scal[out];
    a.part_in = c->partials[in];
    a.part_out = c->partials[out];
    a.nslots = c->nslots;
    a.macro = write_macros ? static_cast<R*>(c->macro) : nullptr;
    a.rref_in = c->rref[in];
    a.rref_out = c->rref[out];
    a.status = c->status;
    a.oc_save = (c->chi_same_step && c->oc_state) ? static_cast<R*>(c->oc_state) : nullptr;
    a.wall_on = (c->wall_ux[0] != 0.0 || c->wall_ux[1] != 0.0) ? 1 : 0;
    a.wall_ux[0] = (R)c->wall_ux[0];
    a.wall_ux[1] = (R)c->wall_ux[1];
    a.wet_interp = c->wet_delta > 0.0 ? 1 : 0;
    a.wet_delta = (R)(c->wet_delta > 0.0 ? c->wet_delta : 1.0);
    a.G12 = (R)c->params.G12;
    a.Gw[0] = (R)c->params.Gw[0];
    a.Gw[1] = (R)c->params.Gw[1];
    for (int k = 0; k < 2; ++k)
        for (int r = 0; r < 9; ++r) a.s[k][r] = (R)c->s[k][r];
    a.body[0] = (R)c->params.body_force[0];
    a.body[1] = (R)c->params.body_force[1];
    return a;
}

template <typename S, typename R>
D2Args<S, R> make_args(lbm_ctx* c, bool write_macros) {
    return make_args_par<S, R>(c, c->cur, write_macros);
}

// Both tile lists of one step.  side != nullptr: the general list runs on a
// forked branch (used while capturing graphs).
template <typename S, typename R>
cudaError_t launch_lists(lbm_ctx* c, bool macros, cudaStream_t st, cudaStream_t side,
                         cudaEvent_t mid = nullptr) {
    D2Args<S, R> a = make_args<S, R>(c, macros);
    cudaError_t e = cudaSuccess;
    const bool fork = side && c->nfast > 0 && c->ngeneral > 0;
    if (fork) {
        e = cudaEventRecord(c->ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, c->ev_fork, 0);
    }
    // Forked (graph) steps launch the general list first: its CTAs are few
    // but large (staging warps), and placed before the fast list fills the
    // SMs they start at once instead of waiting for fast CTAs to drain.
    D2Args<S, R> ag = a;
    ag.list_off = c->nfast;
    // same-step chi: the outlet nodes are collided after the general tiles
    // (on their stream), once the step's flux partials exist
    const bool chi_same = a.oc_save != nullptr;
    if (fork && e == cudaSuccess) e = launch_d2q9_step<S, R>(ag, c->variant, true, c->ngeneral, side);
    if (fork && chi_same && e == cudaSuccess) e = launch_d2q9_outlet_chi<S, R>(a, side);
    if constexpr (std::is_same<S, float>::value && std::is_same<R, float>::value) {
        if (e == cudaSuccess && c->nmarch > 0)
            e = launch_d2q9_march(a, &c->tmap[c->cur], c->march_runs, c->march_flags, c->nmarch, st);
    }
    if (e == cudaSuccess) e = launch_d2q9_step<S, R>(a, c->variant, false, c->nfast, st);
    if (e == cudaSuccess && mid) e = cudaEventRecord(mid, st);
    if (!fork && e == cudaSuccess) e = launch_d2q9_step<S, R>(ag, c->variant, true, c->ngeneral, st);
    if (!fork && chi_same && e == cudaSuccess) e = launch_d2q9_outlet_chi<S, R>(a, st);
    if (fork && e == cudaSuccess) {
        e = cudaEventRecord(c->ev_join, side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_join, 0);
    }
    return e;
}

template <typename S, typename R>
lbm_status launch_one(lbm_ctx* c, bool macros, cudaStream_t st, cudaEvent_t mid = nullptr) {
    cudaError_t e = launch_lists<S, R>(c, macros, st, nullptr, mid);
    if (e != cudaSuccess) return cuda_fail(c, e, "d2q9 step launch");
    // the ping-pong slot written by this step becomes current
    c->cur = 1 - c->cur;
    c->step += 1;
    c->launches += (c->nfast > 0) + (c->ngeneral > 0) + (c->nmarch > 0) + (c->chi_same_step ? 1 : 0);
    return LBM_OK;
}

// Capture kGraphSteps consecutive steps that start at ping-pong parity `par`.
template <typename S, typename R>
lbm_status ensure_graph(lbm_ctx* c, int par) {
    if (c->gexec[par]) return LBM_OK;
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    if (!c->side_stream) CK(cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
    if (!c->ev_fork) CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    if (!c->ev_join) CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    const int saved = c->cur;
    c->cur = par;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i) {
        e = launch_lists<S, R>(c, false, c->cap_stream, c->side_stream);
        c->cur = 1 - c->cur;
    }
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    c->cur = saved;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess)
        e = instantiate_step_graph(g, c->schedule == LBM_SCHEDULE_GRAPHS_EARLY, &c->gexec[par], &c->gexec_early[par]);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec[par] = nullptr;
        return cuda_fail(c, e, "step graph capture");
    }
    return LBM_OK;
}

// cnt steps without macro output: graph replays, then single launches.
template <typename S, typename R>
lbm_status run_plain(lbm_ctx* c, int64_t cnt) {
    while (c->use_graphs && cnt >= kGraphSteps) {
        if (ensure_graph<S, R>(c, c->cur) != LBM_OK) {
            c->use_graphs = 0;  // capture unavailable: keep launching the same kernel directly
            cudaGetLastError();
            break;
        }
        cudaError_t e = cudaGraphLaunch(c->gexec[c->cur], c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "step graph launch");
        c->step += kGraphSteps;
        c->launches += (int64_t)kGraphSteps *
                       ((c->nfast > 0) + (c->ngeneral > 0) + (c->nmarch > 0) + (c->chi_same_step ? 1 : 0));
        cnt -= kGraphSteps;
    }
    for (; cnt > 0; --cnt) {
        lbm_status st = launch_one<S, R>(c, false, c->stream);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

template <typename S, typename R>
lbm_status launch_sampled(lbm_ctx* c, bool macros) {
    const int i = c->n_samples;
    if ((int)c->ev_start.size() <= i) {
        cudaEvent_t a, m, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&m));
        CK(cudaEventCreate(&b));
        c->ev_start.push_back(a);
        c->ev_mid.push_back(m);
        c->ev_stop.push_back(b);
    }
    CK(cudaEventRecord(c->ev_start[i], c->stream));
    lbm_status st = launch_one<S, R>(c, macros, c->stream, c->ev_mid[i]);
    if (st != LBM_OK) return st;
    CK(cudaEventRecord(c->ev_stop[i], c->stream));
    c->n_samples += 1;
    return LBM_OK;
}

template <typename S, typename R>
lbm_status run_steps(lbm_ctx* c, int64_t n) {
    auto sampling = [c]() { return c->timing_every > 0 && c->n_samples < kMaxSamples; };
    int64_t remaining = n;
    while (remaining > 1) {
        int64_t chunk = remaining - 1;  // the last step writes the macroscopic fields
        if (sampling()) {
            const int64_t until = (c->timing_every - c->step % c->timing_every) % c->timing_every;
            if (until == 0) {
                lbm_status st = launch_sampled<S, R>(c, false);
                if (st != LBM_OK) return st;
                --remaining;
                continue;
            }
            chunk = std::min(chunk, until);
        }
        lbm_status st = run_plain<S, R>(c, chunk);
        if (st != LBM_OK) return st;
        remaining -= chunk;
    }
    if (sampling() && c->step % c->timing_every == 0) return launch_sampled<S, R>(c, true);
    return launch_one<S, R>(c, true, c->stream);
}

// Store/convert helpers for host <-> device population and aux transfers.
template <typename S>
S to_store(double v, double wr);
template <>
float to_store<float>(double v, double) { return (float)v; }
template <>
double to_store<double>(double v, double) { return v; }
template <>
__half to_store<__half>(double v, double wr) { return __float2half_rn((float)(v - wr)); }

template <typename S>
double from_store(S v, double wr);
template <>
double from_store<float>(float v, double) { return (double)v; }
template <>
double from_store<double>(double v, double) { return v; }
template <>
double from_store<__half>(__half v, double wr) { return (double)__half2float(v) + wr; }

// Destination of direction i leaving node (x, y): the node that pulls it next
// step, or the node itself when the value bounces back (pull bit opp(i) set).
void dest_node(const lbm_ctx* c, int x, int y, int i, int* dx, int* dy) {
    const int opp = (i == 0) ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5);
    const uint16_t inf = c->h_info[(size_t)y * c->pitch + x];
    if ((inf >> opp) & 1u) {
        *dx = x;
        *dy = y;
        return;
    }
    int u = x + kEx[i], v = y + kEy[i];
    if (u < 0) u += c->nx;
    else if (u >= c->nx) u -= c->nx;
    if (v < 0) v += c->ny;
    else if (v >= c->ny) v -= c->ny;
    *dx = u;
    *dy = v;
}

// Upload post-collision populations fh [2][9][ny][nx] (double) into buffer
// `which`.  FP16 storage also sets that parity's reference densities to the
// half-rounded node densities and encodes each value against its destination.
template <typename S>
lbm_status upload_f(lbm_ctx* c, const double* fh, int which) {
    const size_t count = (size_t)18 * c->plane;
    CK(cudaStreamSynchronize(c->stream));  // the staging buffer may still feed an earlier copy
    S* buf = static_cast<S*>(c->stage);
    const size_t N = (size_t)c->nx * c->ny;
    std::vector<__half> ref;
    if (std::is_same<S, __half>::value) {
        ref.assign((size_t)2 * c->plane, __float2half_rn(0.0f));
        for (int k = 0; k < 2; ++k)
            for (int y = 0; y < c->ny; ++y)
                for (int x = 0; x < c->nx; ++x) {
                    double r = 0.0;
                    for (int i = 0; i < 9; ++i) r += fh[((size_t)k * 9 + i) * N + (size_t)y * c->nx + x];
                    ref[(size_t)k * c->plane + (size_t)y * c->pitch + x] = __float2half_rn((float)r);
                }
    }
    std::fill(buf, buf + count, to_store<S>(0.0, 0.0));
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < 9; ++i)
            for (int y = 0; y < c->ny; ++y)
                for (int x = 0; x < c->nx; ++x) {
                    const size_t d = (size_t)y * c->pitch + x;
                    if (c->host_solid[d]) continue;
                    const double v = fh[((size_t)k * 9 + i) * N + (size_t)y * c->nx + x];
                    double wr = 0.0;
                    if (!ref.empty()) {
                        int dx, dy;
                        dest_node(c, x, y, i, &dx, &dy);
                        wr = kW[i] * (double)__half2float(ref[(size_t)k * c->plane + (size_t)dy * c->pitch + dx]);
                    }
                    buf[(size_t)(k * 9 + i) * c->plane + d] = to_store<S>(v, wr);
                }
    CK(cudaMemcpyAsync(c->f[which], buf, count * sizeof(S), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (!ref.empty())
        CK(cudaMemcpy(c->rref[which], ref.data(), ref.size() * sizeof(__half), cudaMemcpyHostToDevice));
    return LBM_OK;
}

template <typename S>
lbm_status download_f(lbm_ctx* c, double* fh) {
    const size_t count = (size_t)18 * c->plane;
    CK(cudaStreamSynchronize(c->stream));
    const S* buf = static_cast<const S*>(c->stage);
    CK(cudaMemcpyAsync(c->stage, c->f[c->cur], count * sizeof(S), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::vector<__half> ref;
    if (std::is_same<S, __half>::value) {
        ref.resize((size_t)2 * c->plane);
        CK(cudaMemcpy(ref.data(), c->rref[c->cur], ref.size() * sizeof(__half), cudaMemcpyDeviceToHost));
    }
    const size_t N = (size_t)c->nx * c->ny;
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < 9; ++i)
            for (int y = 0; y < c->ny; ++y)
                for (int x = 0; x < c->nx; ++x) {
                    const size_t d = (size_t)y * c->pitch + x;
                    double v = 0.0;
                    if (!c->host_solid[d]) {
                        double wr = 0.0;
                        if (!ref.empty()) {
                            int dx, dy;
                            dest_node(c, x, y, i, &dx, &dy);
                            wr = kW[i] * (double)__half2float(ref[(size_t)k * c->plane + (size_t)dy * c->pitch + dx]);
                        }
                        v = from_store<S>(buf[(size_t)(k * 9 + i) * c->plane + d], wr);
                    }
                    fh[((size_t)k * 9 + i) * N + (size_t)y * c->nx + x] = v;
                }
    return LBM_OK;
}

lbm_status check_status(lbm_ctx* c) {
    unsigned int st = 0;
    CK(cudaMemcpyAsync(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st & 4u) return fail(c, LBM_ERR_CUDA, "a bulk-copy destination was not 128-byte aligned; nothing was copied");
    if (st & 2u) return fail(c, LBM_ERR_TIMEOUT, "a bounded wait for a bulk copy ran out");
    if (st) return fail(c, LBM_ERR_DIVERGED, "non-finite density or velocity produced");
    return LBM_OK;
}

template <typename R>
lbm_status copy_macros(lbm_ctx* c, void* rho, void* u, bool to_double, bool dst_dev) {
    const size_t N = (size_t)c->nx * c->ny;
    CK(cudaStreamSynchronize(c->stream));
    const R* buf = static_cast<const R*>(c->stage);
    CK(cudaMemcpyAsync(c->stage, c->macro, (size_t)4 * c->plane * sizeof(R), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::vector<float> fr, fu;
    if (!to_double) {
        fr.resize(2 * N);
        fu.resize(2 * N);
    }
    for (int q = 0; q < 4; ++q)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                const size_t d = (size_t)y * c->pitch + x;
                double v = c->host_solid[d] ? 0.0 : (double)buf[(size_t)q * c->plane + d];
                const size_t h = (size_t)(q & 1) * N + (size_t)y * c->nx + x;
                if (to_double) {
                    (q < 2 ? static_cast<double*>(rho) : static_cast<double*>(u))[h] = v;
                } else {
                    (q < 2 ? fr : fu)[h] = (float)v;
                }
            }
    if (!to_double) {
        if (dst_dev) {
            CK(cudaMemcpyAsync(rho, fr.data(), fr.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(u, fu.data(), fu.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        } else {
            std::memcpy(rho, fr.data(), fr.size() * sizeof(float));
            std::memcpy(u, fu.data(), fu.size() * sizeof(float));
        }
    }
    return LBM_OK;
}

template <typename S, typename R>
lbm_status init_state(lbm_ctx* c, const double* rho_init, const double* u_init, const uint8_t* solid) {
    const int nx = c->nx, ny = c->ny;
    const size_t N = (size_t)nx * ny;
    std::vector<double> fh((size_t)18 * N, 0.0);
    std::vector<R> macro((size_t)4 * c->plane, R(0));
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t h = (size_t)y * nx + x;
            if (solid && solid[h]) continue;
            const double ux = u_init ? u_init[h] : 0.0, uy = u_init ? u_init[N + h] : 0.0;
            for (int k = 0; k < 2; ++k)
                for (int i = 0; i < 9; ++i) fh[((size_t)k * 9 + i) * N + h] = host_feq(i, rho_init[k * N + h], ux, uy);
            const size_t d = (size_t)y * c->pitch + x;
            macro[d] = (R)rho_init[h];
            macro[c->plane + d] = (R)rho_init[N + h];
            macro[2 * c->plane + d] = (R)ux;
            macro[3 * c->plane + d] = (R)uy;
        }
    lbm_status st = upload_f<S>(c, fh.data(), 0);
    if (st != LBM_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    std::memcpy(c->stage, macro.data(), macro.size() * sizeof(R));
    CK(cudaMemcpyAsync(c->macro, c->stage, macro.size() * sizeof(R), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // open-boundary state: outlet populations of the "previous" step are the
    // initial ones; inlet forces start at zero; lambda = 0, chi = 1
    std::vector<R> fo((size_t)std::max(1, c->nface_nodes) * 18, R(0));
    for (int fi = 0; fi < c->nfaces; ++fi) {
        const FaceDev& F = c->faces[fi];
        if (F.kind != FACE_OUTLET) continue;
        for (int t = F.lo; t <= F.hi; ++t) {
            const int x = F.side == 0 ? 0 : (F.side == 1 ? nx - 1 : t);
            const int y = F.side == 2 ? 0 : (F.side == 3 ? ny - 1 : t);
            const size_t h = (size_t)y * nx + x;
            for (int k = 0; k < 2; ++k)
                for (int i = 0; i < 9; ++i)
                    fo[((size_t)(F.base + t - F.lo) * 9 + i) * 2 + k] = (R)fh[((size_t)k * 9 + i) * N + h];
        }
    }
    CK(cudaMemcpy(c->fo[0], fo.data(), fo.size() * sizeof(R), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->fo[1], fo.data(), fo.size() * sizeof(R), cudaMemcpyHostToDevice));
    const size_t nfn = (size_t)std::max(1, c->nface_nodes);
    CK(cudaMemset(c->Fp[0], 0, nfn * 8 * sizeof(R)));
    CK(cudaMemset(c->Fp[1], 0, nfn * 8 * sizeof(R)));
    CK(cudaMemset(c->status, 0, sizeof(unsigned int)));
    // lambda0 = 0, chi0 = 1; [5] = 0: no flux partials yet
    double sc[8] = {0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    CK(cudaMemcpy(c->scal[0], sc, sizeof(sc), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->scal[1], sc, sizeof(sc), cudaMemcpyHostToDevice));
    c->cur = 0;
    c->step = 0;
    return LBM_OK;
}

// lambda / chi the next step would compute from the live partials, written
// into the current scalar block as its initial values (valid flag cleared).
lbm_status fold_partials(lbm_ctx* c) {
    double sc[8];
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(sc, c->scal[c->cur], sizeof(sc), cudaMemcpyDeviceToHost));
    if (sc[5] == 0.0 || c->nslots == 0) return LBM_OK;
    std::vector<double> pp((size_t)c->nslots * 4);
    CK(cudaMemcpy(pp.data(), c->partials[c->cur], pp.size() * 8, cudaMemcpyDeviceToHost));
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int sl = 0; sl < c->nslots; ++sl)
        for (int j = 0; j < 4; ++j) t[j] += pp[(size_t)sl * 4 + j];
    if (c->out_face >= 0 && t[3] > 0.0) {
        const double um = t[2] / t[3];
        sc[0] = um > 0.0 ? um : 0.0;
        sc[1] = (!c->have_inlet || std::fabs(t[1]) < 1e-14) ? 1.0 : t[0] / t[1];
    }
    sc[5] = 0.0;
    CK(cudaMemcpy(c->scal[c->cur], sc, sizeof(sc), cudaMemcpyHostToDevice));
    return LBM_OK;
}

// (Re)build the tile grid and the two tile lists for tile-shape variant v.
// TMA descriptors of both population buffers for the column-marching
// kernel: a float tensor [18][ny][pitch] with a box of 44 x 10 x 18
// (columns x rows x planes).  cuTensorMapEncodeTiled comes from the driver
// through the runtime's entry-point query, so no driver library is linked.
lbm_status make_tensor_maps(lbm_ctx* c) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(c, LBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        encode = reinterpret_cast<Encode>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)c->pitch, (cuuint64_t)c->ny, 18};
    const cuuint64_t strides[2] = {(cuuint64_t)c->pitch * 4, (cuuint64_t)c->plane * 4};
    const cuuint32_t box[3] = {(cuuint32_t)D2Q9_MARCH_BOX_W, (cuuint32_t)D2Q9_MARCH_BOX_H, 18};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int p = 0; p < 2; ++p) {
        CUresult r = encode(&c->tmap[p], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->f[p], dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(c, LBM_ERR_CUDA, "cuTensorMapEncodeTiled rejected the population layout");
    }
    c->have_tmap = 1;
    return LBM_OK;
}

lbm_status build_tiles(lbm_ctx* c, int v, bool sync_first) {
    if (v < 0 || v >= d2q9_num_variants()) return fail(c, LBM_ERR_INVALID_ARG, "unknown tile variant");
    if (sync_first) CK(cudaStreamSynchronize(c->stream));
    const int nx = c->nx, ny = c->ny;
    const lbm_grid* grid = &c->grid;
    const std::vector<int>& faceid = c->h_faceid;
    const std::vector<int>& nbrid = c->h_nbrid;
    const size_t N = (size_t)nx * ny;
    std::vector<uint8_t> sol(N);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) sol[(size_t)y * nx + x] = c->host_solid[(size_t)y * c->pitch + x];
    // the current tiling's flux partials become lambda / chi values in the
    // scalar block (valid flag 0), so a new tiling continues the same run
    if (c->partials[c->cur] && c->scal[c->cur]) {
        lbm_status fs = fold_partials(c);
        if (fs != LBM_OK) return fs;
    }
    c->variant = v;
    c->xoff = c->yoff = 0;
    c->nslots = 0;
    c->tiling_gen += 1;
    // tile grid: keep x_{N-1} and x_N of the outlet in one tile
    d2q9_variant_tile(c->variant, &c->tx, &c->ty);
    if (c->out_face >= 0) {
        const FaceDev& F = c->faces[c->out_face];
        if (F.side == 1 && nx % c->tx == 1) c->xoff = 1;
        if (F.side == 3 && ny % c->ty == 1) c->yoff = 1;
    }
    c->gdim = dim3((unsigned)((nx + c->xoff + c->tx - 1) / c->tx), (unsigned)((ny + c->yoff + c->ty - 1) / c->ty), 1);

    // Tile lists.  A tile whose psi halo holds an open-face node or crosses an
    // open side goes to the general list (inlet/outlet reconstruction, ghost
    // mirror); the rest go to the fast list, flagged EDGE when the pull halo
    // crosses a grid edge (wrap / closed edge) and SOLID when a solid site can
    // enter the adhesion stencil.  Tiles of the general list that own inlet
    // nodes or outlet-neighbour nodes join the flux reduction.
    std::vector<int> list_fast, list_gen;
    std::vector<uint8_t> fl_fast, fl_gen;
    std::vector<unsigned> strips_gen;
    int64_t gen_nodes = 0, fast_nodes_cnt = 0;
    std::vector<int> slots;
    for (unsigned by = 0; by < c->gdim.y; ++by)
        for (unsigned bx = 0; bx < c->gdim.x; ++bx) {
            const int x0 = (int)bx * c->tx - c->xoff, y0 = (int)by * c->ty - c->yoff;
            const bool edge = x0 - 3 < 0 || x0 + c->tx + 3 > nx || y0 - 3 < 0 || y0 + c->ty + 3 > ny;
            bool gen = (x0 - 2 < 0 && c->open_side[0]) || (x0 + c->tx + 2 > nx && c->open_side[1]) ||
                       (y0 - 2 < 0 && c->open_side[2]) || (y0 + c->ty + 2 > ny && c->open_side[3]);
            bool near_solid = false, part = false, closed_edge = false;
            // every site of the psi halo, resolved as the kernel resolves it
            // (periodic wrap, ghost mirror on open sides, solid outside a closed edge)
            for (int yy = y0 - 2; yy < y0 + c->ty + 2; ++yy)
                for (int xx = x0 - 2; xx < x0 + c->tx + 2; ++xx) {
                    int gx = xx, gy = yy;
                    bool outside = false;
                    if (gx < 0 || gx >= nx) {
                        if (grid->periodic[0]) gx = ((gx % nx) + nx) % nx;
                        else if (c->open_side[gx < 0 ? 0 : 1]) gx = std::min(std::max(gx < 0 ? -1 - gx : 2 * nx - 1 - gx, 0), nx - 1);
                        else outside = true;
                    }
                    if (gy < 0 || gy >= ny) {
                        if (grid->periodic[1]) gy = ((gy % ny) + ny) % ny;
                        else if (c->open_side[gy < 0 ? 2 : 3]) gy = std::min(std::max(gy < 0 ? -1 - gy : 2 * ny - 1 - gy, 0), ny - 1);
                        else outside = true;
                    }
                    if (outside) {
                        closed_edge = true;
                        continue;
                    }
                    const size_t h = (size_t)gy * nx + gx;
                    gen = gen || faceid[h] != 0;
                    near_solid = near_solid || sol[h] != 0;
                    const bool own = xx >= x0 && xx < x0 + c->tx && yy >= y0 && yy < y0 + c->ty &&
                                     xx >= 0 && xx < nx && yy >= 0 && yy < ny;
                    if (own && !sol[h] &&
                        ((faceid[h] && c->faces[faceid[h] - 1].kind == FACE_INLET) ||
                         (nbrid[h] && nbrid[h] - 1 == c->out_face)))
                        part = true;
                }
            uint8_t fl = 0;
            if (edge) fl |= BLOCK_EDGE;
            if (near_solid || closed_edge || gen) fl |= BLOCK_SOLID;
            const int packed = (int)bx | ((int)by << 16);
            int64_t own_fluid = 0;
            for (int yy = std::max(0, y0); yy < std::min(ny, y0 + c->ty); ++yy)
                for (int xx = std::max(0, x0); xx < std::min(nx, x0 + c->tx); ++xx)
                    own_fluid += sol[(size_t)yy * nx + xx] ? 0 : 1;
            if (own_fluid == 0) continue;  // nothing to update: the tile is not launched
            (gen ? gen_nodes : fast_nodes_cnt) += own_fluid;
            if (gen) {
                // face sides seen by the tile's psi halo (after the ghost mirror):
                // each gets a strip of face nodes reconstructed once per tile
                int cnt[4] = {0, 0, 0, 0};
                bool sees_outlet = false;
                for (int yy = y0 - 2; yy < y0 + c->ty + 2; ++yy)
                    for (int xx = x0 - 2; xx < x0 + c->tx + 2; ++xx) {
                        int gx = xx, gy = yy;
                        if (gx < 0 || gx >= nx) {
                            if (grid->periodic[0]) gx = ((gx % nx) + nx) % nx;
                            else if (c->open_side[gx < 0 ? 0 : 1]) gx = gx < 0 ? -1 - gx : 2 * nx - 1 - gx;
                            else continue;
                        }
                        if (gy < 0 || gy >= ny) {
                            if (grid->periodic[1]) gy = ((gy % ny) + ny) % ny;
                            else if (c->open_side[gy < 0 ? 2 : 3]) gy = gy < 0 ? -1 - gy : 2 * ny - 1 - gy;
                            else continue;
                        }
                        if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
                        const int fid = faceid[(size_t)gy * nx + gx];
                        if (fid) {
                            cnt[c->faces[fid - 1].side] += 1;
                            if (c->faces[fid - 1].kind == FACE_OUTLET) sees_outlet = true;
                        }
                    }
                unsigned strips = 0;
                int nstrip = 0;
                for (int pass = 0; pass < 2; ++pass) {
                    int best = -1;
                    for (int sd = 0; sd < 4; ++sd)
                        if (cnt[sd] > 0 && (best < 0 || cnt[sd] > cnt[best])) best = sd;
                    if (best < 0) break;
                    strips |= (unsigned)(best + 1) << (8 * nstrip++);
                    cnt[best] = 0;
                }
                strips_gen.push_back(strips);
                list_gen.push_back(packed);
                fl_gen.push_back(fl | BLOCK_GENERAL | (sees_outlet ? BLOCK_LAMBDA : 0u));
                slots.push_back(part ? c->nslots++ : -1);
            } else {
                list_fast.push_back(packed);
                fl_fast.push_back(fl);
            }
        }
    // column-marching variant: interior tiles (neither edge nor general)
    // leave the fast list and form runs along their tile column
    std::vector<int4> runs;
    std::vector<uint8_t> run_fl;
    if (v == D2Q9_MARCH_VARIANT && c->precision == LBM_FP32) {
        std::vector<int> col_flag((size_t)c->gdim.x * c->gdim.y, -1);
        std::vector<int> keep;
        std::vector<uint8_t> keep_fl;
        for (size_t t = 0; t < list_fast.size(); ++t) {
            const int bx = list_fast[t] & 0xffff, by = list_fast[t] >> 16;
            if (fl_fast[t] & BLOCK_EDGE) {
                keep.push_back(list_fast[t]);
                keep_fl.push_back(fl_fast[t]);
            } else {
                col_flag[(size_t)bx * c->gdim.y + by] = fl_fast[t];
            }
        }
        int64_t interior = (int64_t)list_fast.size() - (int64_t)keep.size();
        int sms = 152, dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // segment length: about eight runs per SM (two resident at a time), 2 to 64 tiles
        const int seg = (int)std::min<int64_t>(64, std::max<int64_t>(2, (interior + 8 * sms - 1) / (8 * sms)));
        for (unsigned bx = 0; bx < c->gdim.x; ++bx) {
            unsigned by = 0;
            while (by < c->gdim.y) {
                if (col_flag[(size_t)bx * c->gdim.y + by] < 0) {
                    ++by;
                    continue;
                }
                unsigned end = by;
                while (end < c->gdim.y && col_flag[(size_t)bx * c->gdim.y + end] >= 0 && (int)(end - by) < seg) ++end;
                runs.push_back(make_int4((int)bx | ((int)by << 16), (int)(end - by), (int)run_fl.size(), 0));
                for (unsigned t = by; t < end; ++t) run_fl.push_back((uint8_t)col_flag[(size_t)bx * c->gdim.y + t]);
                by = end;
            }
        }
        list_fast.swap(keep);
        fl_fast.swap(keep_fl);
    }
    c->nmarch = (int)runs.size();
    c->march_tiles = (int)run_fl.size();
    c->nfast = (int)list_fast.size();
    c->ngeneral = (int)list_gen.size();
    c->fast_nodes = fast_nodes_cnt;
    c->general_nodes = gen_nodes;
    std::vector<int> blist(list_fast);
    blist.insert(blist.end(), list_gen.begin(), list_gen.end());
    std::vector<uint8_t> bflags(fl_fast);
    bflags.insert(bflags.end(), fl_gen.begin(), fl_gen.end());
    std::vector<int> slot_all((size_t)c->nfast, -1);
    slot_all.insert(slot_all.end(), slots.begin(), slots.end());
    std::vector<unsigned> strip_all((size_t)c->nfast, 0u);
    strip_all.insert(strip_all.end(), strips_gen.begin(), strips_gen.end());

    void* old[] = {c->blocks, c->block_flags, c->block_slot, c->block_strips, c->partials[0], c->partials[1],
                   c->march_runs, c->march_flags};
    c->march_runs = nullptr;
    c->march_flags = nullptr;
    for (void* p : old)
        if (p) cudaFree(p);
    c->blocks = nullptr;
    c->block_flags = nullptr;
    c->block_slot = nullptr;
    c->block_strips = nullptr;
    c->partials[0] = c->partials[1] = nullptr;
    for (int p = 0; p < 2; ++p)
        if (c->gexec[p]) {
            cudaGraphExecDestroy(c->gexec[p]);
            c->gexec[p] = nullptr;
        }
    CK(cudaMalloc((void**)&c->blocks, blist.size() * sizeof(int) + 4));
    CK(cudaMalloc((void**)&c->block_flags, bflags.size() + 4));
    CK(cudaMalloc((void**)&c->block_slot, slot_all.size() * sizeof(int) + 4));
    CK(cudaMalloc((void**)&c->block_strips, strip_all.size() * sizeof(unsigned) + 4));
    for (int p = 0; p < 2; ++p) {
        CK(cudaMalloc((void**)&c->partials[p], (size_t)std::max(1, c->nslots) * 4 * 8));
        CK(cudaMemset(c->partials[p], 0, (size_t)std::max(1, c->nslots) * 4 * 8));
    }
    CK(cudaMemcpy(c->block_strips, strip_all.data(), strip_all.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->blocks, blist.data(), blist.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->block_flags, bflags.data(), bflags.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->block_slot, slot_all.data(), slot_all.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (c->nmarch > 0) {
        CK(cudaMalloc((void**)&c->march_runs, runs.size() * sizeof(int4)));
        CK(cudaMalloc((void**)&c->march_flags, run_fl.size()));
        CK(cudaMemcpy(c->march_runs, runs.data(), runs.size() * sizeof(int4), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->march_flags, run_fl.data(), run_fl.size(), cudaMemcpyHostToDevice));
        if (!c->have_tmap) {
            lbm_status ts = make_tensor_maps(c);
            if (ts != LBM_OK) return ts;
        }
    }
    // a new tiling renumbers the slots: old partials are void (folded above)
    CK(cudaMemset(c->scal[0] + 5, 0, sizeof(double)));
    CK(cudaMemset(c->scal[1] + 5, 0, sizeof(double)));
    return LBM_OK;
}


// ---- snapshots (autotuning runs trial steps and then puts the state back) ----
struct Snapshot {
    void* f = nullptr;
    void* Fp = nullptr;
    void* fo = nullptr;
    void* rref = nullptr;
    void* macro = nullptr;
    double scal[8];
    int cur = 0;
    int64_t step = 0;
};

size_t fbytes_of(const lbm_ctx* c) { return (size_t)18 * c->plane * c->sbytes; }
size_t nfn_of(const lbm_ctx* c) { return (size_t)std::max(1, c->nface_nodes); }

lbm_status take_snapshot(lbm_ctx* c, Snapshot* s) {
    lbm_status st = fold_partials(c);  // independent of the tiling
    if (st != LBM_OK) return st;
    const size_t nfn = nfn_of(c);
    CK(cudaMalloc(&s->f, fbytes_of(c)));
    CK(cudaMalloc(&s->Fp, nfn * 8 * c->rbytes));
    CK(cudaMalloc(&s->fo, nfn * 18 * c->rbytes));
    CK(cudaMalloc(&s->rref, (size_t)2 * c->plane * 2));
    CK(cudaMalloc(&s->macro, (size_t)4 * c->plane * c->rbytes));
    CK(cudaMemcpy(s->f, c->f[c->cur], fbytes_of(c), cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(s->Fp, c->Fp[c->cur], nfn * 8 * c->rbytes, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(s->fo, c->fo[c->cur], nfn * 18 * c->rbytes, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(s->rref, c->rref[c->cur], (size_t)2 * c->plane * 2, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(s->macro, c->macro, (size_t)4 * c->plane * c->rbytes, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(s->scal, c->scal[c->cur], sizeof(s->scal), cudaMemcpyDeviceToHost));
    s->cur = c->cur;
    s->step = c->step;
    return LBM_OK;
}

lbm_status restore_snapshot(lbm_ctx* c, Snapshot* s) {
    CK(cudaStreamSynchronize(c->stream));
    const size_t nfn = nfn_of(c);
    c->cur = s->cur;
    c->step = s->step;
    CK(cudaMemcpy(c->f[c->cur], s->f, fbytes_of(c), cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(c->Fp[c->cur], s->Fp, nfn * 8 * c->rbytes, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(c->fo[c->cur], s->fo, nfn * 18 * c->rbytes, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(c->rref[c->cur], s->rref, (size_t)2 * c->plane * 2, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(c->macro, s->macro, (size_t)4 * c->plane * c->rbytes, cudaMemcpyDeviceToDevice));
    double sc[8];
    std::memcpy(sc, s->scal, sizeof(sc));
    sc[5] = 0.0;  // lambda / chi come from the folded values, whatever the tiling
    CK(cudaMemcpy(c->scal[c->cur], sc, sizeof(sc), cudaMemcpyHostToDevice));
    CK(cudaMemset(c->scal[1 - c->cur] + 5, 0, sizeof(double)));
    return LBM_OK;
}

void free_snapshot(Snapshot* s) {
    void* p[] = {s->f, s->Fp, s->fo, s->rref, s->macro};
    for (void* q : p)
        if (q) cudaFree(q);
    *s = Snapshot();
}

}  // namespace

// ---- batched ensembles ------------------------------------------------------
struct lbm_batch {
    std::vector<lbm_ctx*> m;
    cudaStream_t stream = nullptr;
    int precision = LBM_FP32;
    int variant = 0;
    int nfast = 0, ngeneral = 0;
    int* blocks = nullptr;
    uint8_t* flags = nullptr;
    int* slot = nullptr;
    unsigned* strips = nullptr;
    int* member = nullptr;
    void* args[4] = {nullptr, nullptr, nullptr, nullptr};  // [bpar + 2 * macros][member]
    std::vector<int> base_cur;   // member parity when the argument arrays were built
    std::vector<int64_t> base_gen;  // member tiling generation when they were built
    int bpar = 0;                // steps taken since, modulo 2
    int use_graphs = 1;
    cudaStream_t cap_stream = nullptr, side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int gexec_early[2] = {0, 0};
    int64_t launches = 0;
    // persistent schedule: one cooperative launch per run of up to
    // kPersistSteps steps, grid barriers with bounded waits between steps
    int schedule = LBM_SCHEDULE_GRAPHS;
    unsigned* pbar = nullptr;     // barrier arrivals (zeroed before each launch)
    unsigned* pstatus = nullptr;  // PERSIST_TIMEOUT once a barrier wait ran out
    long long spin_limit = kDefaultSpinLimit;
    int bar_skew = 0;             // fault injection for tests: extra arrivals every barrier waits for
    int persist_grid = 0;         // CTAs of the last persistent launch
    std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status st, const std::string& msg) {
    if (b) b->err = msg;
    else lbm::set_thread_error(msg.c_str());
    return st;
}

#define BCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void free_batch_lists(lbm_batch* b) {
    void* p[] = {b->blocks, b->flags, b->slot, b->strips, b->member, b->args[0], b->args[1], b->args[2], b->args[3]};
    for (void* q : p)
        if (q) cudaFree(q);
    b->blocks = nullptr;
    b->flags = nullptr;
    b->slot = nullptr;
    b->strips = nullptr;
    b->member = nullptr;
    for (int i = 0; i < 4; ++i) b->args[i] = nullptr;
    for (int p2 = 0; p2 < 2; ++p2)
        if (b->gexec[p2]) {
            cudaGraphExecDestroy(b->gexec[p2]);
            b->gexec[p2] = nullptr;
        }
}

// Concatenate the members' tile lists (fast tiles first, then general tiles)
// and upload the per-member argument blocks for both parities.
template <typename S, typename R>
lbm_status build_batch(lbm_batch* b) {
    // one kernel instantiation serves the whole batch: every member must use
    // the tile shape of the first one (members re-tiled on their own follow)
    const int v = d2q9_tile_kernel_variant(b->m[0]->variant);
    for (lbm_ctx* c : b->m)
        if (c->variant != v) {
            lbm_status st = build_tiles(c, v, true);
            if (st != LBM_OK) return bfail(b, st, c->err);
        }
    b->variant = v;
    free_batch_lists(b);
    b->nfast = 0;
    b->ngeneral = 0;
    std::vector<int> blk, mem, slt;
    std::vector<uint8_t> flg;
    std::vector<unsigned> stp;
    for (int pass = 0; pass < 2; ++pass)
        for (size_t mi = 0; mi < b->m.size(); ++mi) {
            lbm_ctx* c = b->m[mi];
            const int n = pass == 0 ? c->nfast : c->ngeneral;
            const int off = pass == 0 ? 0 : c->nfast;
            if (n == 0) continue;
            std::vector<int> cb(n), cs(n);
            std::vector<uint8_t> cf(n);
            std::vector<unsigned> cst(n);
            BCK(cudaMemcpy(cb.data(), c->blocks + off, n * sizeof(int), cudaMemcpyDeviceToHost));
            BCK(cudaMemcpy(cf.data(), c->block_flags + off, n, cudaMemcpyDeviceToHost));
            BCK(cudaMemcpy(cs.data(), c->block_slot + off, n * sizeof(int), cudaMemcpyDeviceToHost));
            BCK(cudaMemcpy(cst.data(), c->block_strips + off, n * sizeof(unsigned), cudaMemcpyDeviceToHost));
            blk.insert(blk.end(), cb.begin(), cb.end());
            flg.insert(flg.end(), cf.begin(), cf.end());
            slt.insert(slt.end(), cs.begin(), cs.end());
            stp.insert(stp.end(), cst.begin(), cst.end());
            mem.insert(mem.end(), (size_t)n, (int)mi);
            (pass == 0 ? b->nfast : b->ngeneral) += n;
        }
    if ((size_t)b->nfast + (size_t)b->ngeneral != blk.size() || mem.size() != blk.size())
        return bfail(b, LBM_ERR_INVALID_ARG, "inconsistent batch tile lists");
    const size_t nt = blk.size() + 1;
    BCK(cudaMalloc((void**)&b->blocks, nt * sizeof(int)));
    BCK(cudaMalloc((void**)&b->flags, nt));
    BCK(cudaMalloc((void**)&b->slot, nt * sizeof(int)));
    BCK(cudaMalloc((void**)&b->strips, nt * sizeof(unsigned)));
    BCK(cudaMalloc((void**)&b->member, nt * sizeof(int)));
    BCK(cudaMemcpy(b->blocks, blk.data(), blk.size() * sizeof(int), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->flags, flg.data(), flg.size(), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->slot, slt.data(), slt.size() * sizeof(int), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->strips, stp.data(), stp.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->member, mem.data(), mem.size() * sizeof(int), cudaMemcpyHostToDevice));
    b->base_cur.resize(b->m.size());
    b->base_gen.resize(b->m.size());
    for (size_t mi = 0; mi < b->m.size(); ++mi) b->base_gen[mi] = b->m[mi]->tiling_gen;
    for (int q = 0; q < 4; ++q) {
        std::vector<D2Args<S, R>> av(b->m.size());
        for (size_t mi = 0; mi < b->m.size(); ++mi) {
            b->base_cur[mi] = b->m[mi]->cur;
            av[mi] = make_args_par<S, R>(b->m[mi], b->m[mi]->cur ^ (q & 1), q >= 2);
        }
        BCK(cudaMalloc(&b->args[q], av.size() * sizeof(D2Args<S, R>)));
        BCK(cudaMemcpy(b->args[q], av.data(), av.size() * sizeof(D2Args<S, R>), cudaMemcpyHostToDevice));
    }
    b->bpar = 0;
    return LBM_OK;
}

template <typename S, typename R>
cudaError_t batch_launch(lbm_batch* b, bool macros, cudaStream_t st, cudaStream_t side) {
    BatchArgs<S, R> a{};
    a.args = static_cast<const D2Args<S, R>*>(b->args[b->bpar + (macros ? 2 : 0)]);
    a.blocks = b->blocks;
    a.flags = b->flags;
    a.slot = b->slot;
    a.strips = b->strips;
    a.member = b->member;
    a.off = 0;
    cudaError_t e = cudaSuccess;
    const bool fork = side && b->nfast > 0 && b->ngeneral > 0;
    if (fork) {
        e = cudaEventRecord(b->ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, b->ev_fork, 0);
    }
    // general list first when forked (see launch_lists)
    BatchArgs<S, R> ag = a;
    ag.off = b->nfast;
    if (fork && e == cudaSuccess) e = launch_d2q9_batch<S, R>(ag, b->variant, true, b->ngeneral, side);
    if (e == cudaSuccess) e = launch_d2q9_batch<S, R>(a, b->variant, false, b->nfast, st);
    if (!fork && e == cudaSuccess) e = launch_d2q9_batch<S, R>(ag, b->variant, true, b->ngeneral, st);
    if (fork && e == cudaSuccess) {
        e = cudaEventRecord(b->ev_join, side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_join, 0);
    }
    return e;
}

void batch_advance(lbm_batch* b, int64_t n, int64_t launches = -1) {
    for (lbm_ctx* c : b->m) {
        if (n & 1) c->cur = 1 - c->cur;
        c->step += n;
    }
    if (n & 1) b->bpar ^= 1;
    b->launches += launches >= 0 ? launches : n * ((b->nfast > 0) + (b->ngeneral > 0));
}

// n steps of every member as persistent launches (FP32 storage only).
template <typename S, typename R>
lbm_status batch_run_persistent(lbm_batch* b, int64_t n) {
    if constexpr (!std::is_same<S, float>::value || !std::is_same<R, float>::value) {
        (void)n;
        return bfail(b, LBM_ERR_UNSUPPORTED, "the persistent schedule is built for FP32 storage only");
    } else {
        if (!b->pbar) {
            BCK(cudaMalloc((void**)&b->pbar, sizeof(unsigned)));
            BCK(cudaMalloc((void**)&b->pstatus, sizeof(unsigned)));
            BCK(cudaMemsetAsync(b->pstatus, 0, sizeof(unsigned), b->stream));
        }
        const D2Args<S, R>* const* av = reinterpret_cast<const D2Args<S, R>* const*>(b->args);
        int64_t rem = n;
        while (rem > 0) {
            const int chunk = (int)std::min<int64_t>(rem, kPersistSteps);
            const bool last = chunk == rem;  // the call's last step writes the macroscopic fields
            PersistArgs<S, R> p{};
            p.args[0] = av[b->bpar];
            p.args[1] = av[b->bpar ^ 1];
            p.args_last[0] = last ? av[b->bpar + 2] : p.args[0];
            p.args_last[1] = last ? av[(b->bpar ^ 1) + 2] : p.args[1];
            p.blocks = b->blocks;
            p.flags = b->flags;
            p.slot = b->slot;
            p.strips = b->strips;
            p.member = b->member;
            p.ntiles = b->nfast + b->ngeneral;
            p.nfast = b->nfast;
            p.nsteps = chunk;
            p.bar = b->pbar;
            p.pstatus = b->pstatus;
            p.spin_limit = b->spin_limit;
            p.bar_skew = b->bar_skew;
            BCK(cudaMemsetAsync(b->pbar, 0, sizeof(unsigned), b->stream));
            BCK((launch_d2q9_persist<S, R>(p, b->variant, b->stream, &b->persist_grid)));
            batch_advance(b, chunk, 1);
            rem -= chunk;
        }
        return LBM_OK;
    }
}

template <typename S, typename R>
lbm_status batch_graph(lbm_batch* b, int par) {
    if (b->gexec[par]) return LBM_OK;
    if (!b->cap_stream) BCK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    if (!b->side_stream) BCK(cudaStreamCreateWithFlags(&b->side_stream, cudaStreamNonBlocking));
    if (!b->ev_fork) BCK(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    if (!b->ev_join) BCK(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
    const int saved = b->bpar;
    b->bpar = par;
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i) {
        e = batch_launch<S, R>(b, false, b->cap_stream, b->side_stream);
        b->bpar ^= 1;
    }
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    b->bpar = saved;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess)
        e = instantiate_step_graph(g, b->schedule == LBM_SCHEDULE_GRAPHS_EARLY, &b->gexec[par], &b->gexec_early[par]);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->gexec[par] = nullptr;
        return bfail(b, LBM_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
}

template <typename S, typename R>
lbm_status batch_run(lbm_batch* b, int64_t n) {
    // a member stepped or re-tiled on its own since the arrays were built:
    // rebuild them (its buffers or parity changed)
    for (size_t mi = 0; mi < b->m.size(); ++mi)
        if ((b->m[mi]->cur ^ b->base_cur[mi]) != b->bpar || b->m[mi]->tiling_gen != b->base_gen[mi]) {
            BCK(cudaStreamSynchronize(b->stream));
            lbm_status st = build_batch<S, R>(b);
            if (st != LBM_OK) return st;
            break;
        }
    if (b->schedule == LBM_SCHEDULE_PERSISTENT) return batch_run_persistent<S, R>(b, n);
    int64_t rem = n;
    while (rem > 1) {
        if (b->use_graphs && rem - 1 >= kGraphSteps) {
            if (batch_graph<S, R>(b, b->bpar) != LBM_OK) {
                b->use_graphs = 0;
                cudaGetLastError();
                continue;
            }
            BCK(cudaGraphLaunch(b->gexec[b->bpar], b->stream));
            batch_advance(b, kGraphSteps);  // even: bpar unchanged
            rem -= kGraphSteps;
            continue;
        }
        BCK((batch_launch<S, R>(b, false, b->stream, nullptr)));
        batch_advance(b, 1);
        --rem;
    }
    if (rem == 1) {
        BCK((batch_launch<S, R>(b, true, b->stream, nullptr)));
        batch_advance(b, 1);
    }
    return LBM_OK;
}

template <typename S, typename R>
lbm_status batch_dispatch_build(lbm_batch* b) { return build_batch<S, R>(b); }

lbm_status batch_build_any(lbm_batch* b) {
    if (b->precision == LBM_FP64) return batch_dispatch_build<double, double>(b);
    if (b->precision == LBM_FP32) return batch_dispatch_build<float, float>(b);
    return batch_dispatch_build<__half, float>(b);
}

lbm_status batch_run_any(lbm_batch* b, int64_t n) {
    if (b->precision == LBM_FP64) return batch_run<double, double>(b, n);
    if (b->precision == LBM_FP32) return batch_run<float, float>(b, n);
    return batch_run<__half, float>(b, n);
}

// Time `steps` steps of every tile variant from the same starting state and
// keep the fastest (members' states are restored afterwards).
lbm_status batch_autotune(lbm_batch* b, int steps, int* chosen, double* best_ms) {
    BCK(cudaStreamSynchronize(b->stream));
    std::vector<Snapshot> snaps(b->m.size());
    for (size_t i = 0; i < b->m.size(); ++i) {
        lbm_status st = take_snapshot(b->m[i], &snaps[i]);
        if (st != LBM_OK) return bfail(b, st, b->m[i]->err);
    }
    cudaEvent_t t0, t1;
    BCK(cudaEventCreate(&t0));
    BCK(cudaEventCreate(&t1));
    int best = -1;
    double bestms = 1e300;
    lbm_status st = LBM_OK;
    for (int v = 0; v < D2Q9_MARCH_VARIANT && st == LBM_OK; ++v) {
        for (size_t i = 0; i < b->m.size() && st == LBM_OK; ++i) {
            st = restore_snapshot(b->m[i], &snaps[i]);
            if (st == LBM_OK) st = build_tiles(b->m[i], v, true);
        }
        if (st != LBM_OK) break;
        b->variant = v;
        st = batch_build_any(b);
        if (st != LBM_OK) break;
        st = batch_run_any(b, std::max(2, steps / 4));  // warm-up (also captures the graphs)
        if (st != LBM_OK) break;
        BCK(cudaEventRecord(t0, b->stream));
        st = batch_run_any(b, steps);
        BCK(cudaEventRecord(t1, b->stream));
        BCK(cudaEventSynchronize(t1));
        float ms = 0.0f;
        BCK(cudaEventElapsedTime(&ms, t0, t1));
        if (ms < bestms) {
            bestms = ms;
            best = v;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    for (size_t i = 0; i < b->m.size(); ++i) {
        lbm_status s2 = restore_snapshot(b->m[i], &snaps[i]);
        if (s2 == LBM_OK && best >= 0) s2 = build_tiles(b->m[i], best, true);
        free_snapshot(&snaps[i]);
        if (st == LBM_OK) st = s2;
    }
    if (st != LBM_OK) return st;
    b->variant = best;
    st = batch_build_any(b);
    *chosen = best;
    if (best_ms) *best_ms = bestms / steps;
    return st;
}

// Time `steps` steps of the column-marching variant on the context itself
// from its current state (restored afterwards) and keep it if it beats
// best_ms per step; otherwise the context keeps the tile variant *variant.
lbm_status autotune_march(lbm_ctx* c, int steps, int* variant, double* best_ms) {
    Snapshot snap;
    lbm_status st = take_snapshot(c, &snap);
    if (st != LBM_OK) return st;
    const int best = *variant;
    st = build_tiles(c, D2Q9_MARCH_VARIANT, true);
    double ms = 1e300;
    if (st == LBM_OK && c->nmarch > 0) {
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        CK(cudaEventCreate(&t0));
        CK(cudaEventCreate(&t1));
        st = run_steps<float, float>(c, std::max(2, steps / 4));  // warm-up (also captures the graphs)
        if (st == LBM_OK) {
            CK(cudaEventRecord(t0, c->stream));
            st = run_steps<float, float>(c, steps);
            CK(cudaEventRecord(t1, c->stream));
            CK(cudaEventSynchronize(t1));
            float el = 0.0f;
            CK(cudaEventElapsedTime(&el, t0, t1));
            ms = el / steps;
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
    }
    lbm_status s2 = restore_snapshot(c, &snap);
    const bool take = st == LBM_OK && ms < *best_ms;
    if (s2 == LBM_OK) s2 = build_tiles(c, take ? D2Q9_MARCH_VARIANT : best, true);
    free_snapshot(&snap);
    if (st != LBM_OK) return st;
    if (s2 != LBM_OK) return s2;
    if (take) {
        *variant = D2Q9_MARCH_VARIANT;
        *best_ms = ms;
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_version(void) { return "paper_2512_12934_gb300 lbm 0.1 (sm_103a)"; }

const char* lbm_last_error(const lbm_ctx* ctx) {
    if (ctx && ctx->d3) return lbm3::error(ctx->d3);
    if (ctx) return ctx->err.c_str();
    return g_thread_err;
}

lbm_status lbm_create(const lbm_grid* grid, const lbm_params* params, const lbm_open_bc* bcs, int nbc,
                      const uint8_t* solid, const double* rho_init, const double* u_init,
                      void* cuda_stream, lbm_ctx** out) {
    lbm_ctx* c = nullptr;
    if (!out) return fail(nullptr, LBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !params || !rho_init) return fail(nullptr, LBM_ERR_INVALID_ARG, "grid, params and rho_init are required");
    if (grid->lattice == LBM_D3Q19) {
        std::string err;
        lbm3::Ctx3* c3 = nullptr;
        lbm_status st = lbm3::create(grid, params, bcs, nbc, solid, rho_init, u_init, cuda_stream, &c3, &err);
        if (st != LBM_OK) return fail(nullptr, st, err);
        c = new (std::nothrow) lbm_ctx();
        if (!c) {
            lbm3::destroy(c3);
            return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
        }
        c->d3 = c3;
        *out = c;
        return LBM_OK;
    }
    if (grid->lattice != LBM_D2Q9) return fail(nullptr, LBM_ERR_UNSUPPORTED, "unknown lattice");
    for (int f = 0; f < nbc; ++f)
        if (bcs && bcs[f].rho_profile)
            return fail(nullptr, LBM_ERR_UNSUPPORTED, "rho_profile is implemented for D3Q19 faces only");
    if (grid->nz != 1) return fail(nullptr, LBM_ERR_INVALID_ARG, "D2Q9 needs nz == 1");
    if (grid->nx < 5 || grid->ny < 5) return fail(nullptr, LBM_ERR_INVALID_ARG, "every extent must be >= 5");
    if (18LL * ((grid->nx + 31) / 32 * 32) * grid->ny >= (1LL << 31))
        return fail(nullptr, LBM_ERR_INVALID_ARG, "grid too large: 18 population planes must stay below 2^31 elements");
    if (params->precision != LBM_FP32 && params->precision != LBM_FP64 &&
        params->precision != LBM_FP32_FP16STORE)
        return fail(nullptr, LBM_ERR_INVALID_ARG, "unknown precision");
    if (nbc < 0 || nbc > MAX_FACES || (nbc > 0 && !bcs))
        return fail(nullptr, LBM_ERR_INVALID_ARG, "nbc must be in [0, 4] with a bcs array");
    for (int k = 0; k < 2; ++k)
        if (!(params->nu[k] > 0.0) || !std::isfinite(params->nu[k]))
            return fail(nullptr, LBM_ERR_INVALID_ARG, "viscosities must be positive");

    c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    c->grid = *grid;
    c->params = *params;
    if (c->params.s_q <= 0.0) c->params.s_q = 1.2;
    c->nx = grid->nx;
    c->ny = grid->ny;
    c->pitch = (grid->nx + 31) / 32 * 32;
    c->plane = c->pitch * grid->ny;
    c->precision = params->precision;
    c->sbytes = params->precision == LBM_FP64 ? 8 : (params->precision == LBM_FP32_FP16STORE ? 2 : 4);
    c->rbytes = params->precision == LBM_FP64 ? 8 : 4;
    c->stream = static_cast<cudaStream_t>(cuda_stream);

    // relaxation rates (Eqs. 4, 5; s_eps from the most viscous phase, Sec. III A)
    const double numax = std::max(params->nu[0], params->nu[1]);
    for (int k = 0; k < 2; ++k) {
        const double snu = 1.0 / (3.0 * params->nu[k] + 0.5);
        const double seps = params->s_eps_mode == LBM_SEPS_MAX_NU ? 1.0 / (3.0 * numax + 0.5) : snu;
        const double se = params->s_e > 0.0 ? params->s_e : snu;
        const double s[9] = {1.0, se, seps, 1.0, c->params.s_q, 1.0, c->params.s_q, snu, snu};
        for (int r = 0; r < 9; ++r) {
            if (!(s[r] > 0.0 && s[r] < 2.0)) {
                free_ctx(c);
                return fail(nullptr, LBM_ERR_INVALID_ARG, "a relaxation rate falls outside (0, 2)");
            }
            c->s[k][r] = s[r];
        }
    }

    const int nx = c->nx, ny = c->ny;
    const size_t N = (size_t)nx * ny;
    std::vector<uint8_t> sol(N, 0);
    if (solid)
        for (size_t i = 0; i < N; ++i) sol[i] = solid[i] ? 1 : 0;

    // open faces
    std::vector<int> faceid(N, 0), nbrid(N, 0);
    std::vector<double> uin_h;
    c->nfaces = nbc;
    int noutlet = 0;
    for (int fi = 0; fi < nbc; ++fi) {
        const lbm_open_bc& b = bcs[fi];
        FaceDev& F = c->faces[fi];
        if ((b.kind != LBM_INLET_VELOCITY && b.kind != LBM_OUTLET_CONVECTIVE) || b.side < 0 || b.side > 3) {
            free_ctx(c);
            return fail(nullptr, LBM_ERR_INVALID_ARG, "bad face kind or side");
        }
        const int along = b.side <= 1 ? ny : nx;
        if (b.lo[0] < 0 || b.hi[0] >= along || b.lo[0] > b.hi[0]) {
            free_ctx(c);
            return fail(nullptr, LBM_ERR_INVALID_ARG, "face extent out of range");
        }
        if ((b.side <= 1 && grid->periodic[0]) || (b.side >= 2 && grid->periodic[1])) {
            free_ctx(c);
            return fail(nullptr, LBM_ERR_INVALID_ARG, "open face on a periodic axis");
        }
        F.kind = b.kind == LBM_INLET_VELOCITY ? FACE_INLET : FACE_OUTLET;
        F.side = b.side;
        F.lo = b.lo[0];
        F.hi = b.hi[0];
        side_normal(b.side, &F.ox, &F.oy);
        F.base = c->nface_nodes;
        F.alpha = b.alpha_correction ? 1 : 0;
        F.chi = b.chi_correction ? 1 : 0;
        F.rho_in[0] = b.rho_in[0];
        F.rho_in[1] = b.rho_in[1];
        F.sxx = F.syy = 0.0;
        for (int i = 0; i < 9; ++i)
            if (kEx[i] * F.ox + kEy[i] * F.oy < 0) {
                F.sxx += kW[i] * kEx[i] * kEx[i];
                F.syy += kW[i] * kEy[i] * kEy[i];
            }
        if (F.kind == FACE_OUTLET) {
            ++noutlet;
            c->out_face = fi;
        } else {
            c->have_inlet = 1;
        }
        c->open_side[b.side] = 1;
        const int len = F.hi - F.lo + 1;
        c->nface_nodes += len;
        for (int t = 0; t < len; ++t)
            uin_h.push_back((F.kind == FACE_INLET && b.u_profile) ? b.u_profile[t] : 0.0);
        for (int t = F.lo; t <= F.hi; ++t) {
            const int x = b.side == 0 ? 0 : (b.side == 1 ? nx - 1 : t);
            const int y = b.side == 2 ? 0 : (b.side == 3 ? ny - 1 : t);
            const size_t h = (size_t)y * nx + x;
            if (sol[h]) continue;
            if (faceid[h]) {
                free_ctx(c);
                return fail(nullptr, LBM_ERR_INVALID_ARG, "a node lies on two open faces");
            }
            faceid[h] = fi + 1;
        }
    }
    if (noutlet > 1) {
        free_ctx(c);
        return fail(nullptr, LBM_ERR_INVALID_ARG, "at most one outlet face");
    }
    for (int fi = 0; fi < nbc; ++fi) {
        const FaceDev& F = c->faces[fi];
        for (int t = F.lo; t <= F.hi; ++t) {
            const int x = F.side == 0 ? 0 : (F.side == 1 ? nx - 1 : t);
            const int y = F.side == 2 ? 0 : (F.side == 3 ? ny - 1 : t);
            if (sol[(size_t)y * nx + x]) continue;
            const size_t h2 = (size_t)(y - F.oy) * nx + (x - F.ox);
            if (sol[h2] || faceid[h2] || nbrid[h2]) {
                free_ctx(c);
                return fail(nullptr, LBM_ERR_INVALID_ARG, "the inward neighbour of a face node must be plain fluid");
            }
            nbrid[h2] = fi + 1;
        }
    }

    // per-node descriptors
    std::vector<uint16_t> info((size_t)c->plane, (uint16_t)INFO_SOLID);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t h = (size_t)y * nx + x;
            unsigned v = 0;
            if (sol[h]) {
                v = INFO_SOLID;
            } else {
                for (int i = 0; i < 9; ++i) {
                    int sx = x - kEx[i], sy = y - kEy[i];
                    bool blocked = false;
                    if (sx < 0 || sx >= nx) {
                        if (grid->periodic[0]) sx = (sx + nx) % nx;
                        else blocked = true;
                    }
                    if (sy < 0 || sy >= ny) {
                        if (grid->periodic[1]) sy = (sy + ny) % ny;
                        else blocked = true;
                    }
                    if (!blocked && sol[(size_t)sy * nx + sx]) blocked = true;
                    if (blocked) v |= 1u << i;
                }
                v |= (unsigned)faceid[h] << INFO_FACE_SHIFT;
                v |= (unsigned)nbrid[h] << INFO_NBR_SHIFT;
            }
            info[(size_t)y * c->pitch + x] = (uint16_t)v;
        }

    // device allocation
    const size_t fbytes = (size_t)18 * c->plane * c->sbytes;
    const int nfn = std::max(1, c->nface_nodes);
    c->diag_blocks = 152 * 4;
    cudaError_t e = cudaGetDevice(&c->device);
    void** allocs[] = {&c->f[0], &c->f[1], (void**)&c->info, &c->uin, &c->Fp[0], &c->Fp[1], &c->fo[0], &c->fo[1],
                       (void**)&c->scal[0], (void**)&c->scal[1], (void**)&c->status, &c->macro, (void**)&c->diag_partials,
                       &c->rref[0], &c->rref[1]};
    const size_t sizes[] = {fbytes, fbytes, (size_t)c->plane * 2, (size_t)nfn * c->rbytes,
                            (size_t)nfn * 8 * c->rbytes, (size_t)nfn * 8 * c->rbytes,
                            (size_t)nfn * 18 * c->rbytes, (size_t)nfn * 18 * c->rbytes, 64, 64,
                            16,
                            (size_t)4 * c->plane * c->rbytes, (size_t)c->diag_blocks * 3 * 8,
                            (size_t)2 * c->plane * 2, (size_t)2 * c->plane * 2};
    for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]) && e == cudaSuccess; ++i) {
        e = cudaMalloc(allocs[i], sizes[i]);
        if (e == cudaSuccess) e = cudaMemset(*allocs[i], 0, sizes[i]);
    }
    if (e != cudaSuccess) {
        const lbm_status st = e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
        const std::string msg = std::string("device allocation: ") + cudaGetErrorString(e);
        free_ctx(c);
        return fail(nullptr, st, msg);
    }
    e = cudaMemcpy(c->info, info.data(), info.size() * 2, cudaMemcpyHostToDevice);
    c->h_info = info;

    if (e == cudaSuccess && c->nface_nodes > 0) {
        if (c->rbytes == 8) {
            e = cudaMemcpy(c->uin, uin_h.data(), uin_h.size() * 8, cudaMemcpyHostToDevice);
        } else {
            std::vector<float> uf(uin_h.begin(), uin_h.end());
            e = cudaMemcpy(c->uin, uf.data(), uf.size() * 4, cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        const std::string msg = std::string("upload: ") + cudaGetErrorString(e);
        free_ctx(c);
        return fail(nullptr, LBM_ERR_CUDA, msg);
    }
    c->host_solid.assign((size_t)c->plane, 1);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) c->host_solid[(size_t)y * c->pitch + x] = sol[(size_t)y * nx + x];
    c->stage_bytes = std::max((size_t)18 * c->plane * c->sbytes, (size_t)4 * c->plane * c->rbytes);
    e = cudaMallocHost(&c->stage, c->stage_bytes);
    if (e != cudaSuccess) {
        c->stage = nullptr;
        const std::string msg = std::string("pinned staging allocation: ") + cudaGetErrorString(e);
        free_ctx(c);
        return fail(nullptr, LBM_ERR_OOM, msg);
    }
    c->host_solid_in.assign(sol.begin(), sol.end());
    c->h_faceid = faceid;
    c->h_nbrid = nbrid;
    // default tile shape: narrow tiles (more CTAs, shorter chains) for small
    // grids, 32x8 for large ones (measured on GB300; lbm_set_tile_variant
    // overrides)
    lbm_status st = build_tiles(c, (long long)nx * ny < (1LL << 22) ? 1 : 0, false);
    if (st != LBM_OK) {
        const std::string msg = c->err;
        free_ctx(c);
        return fail(nullptr, st, msg);
    }
    if (c->precision == LBM_FP64) st = init_state<double, double>(c, rho_init, u_init, solid ? sol.data() : nullptr);
    else if (c->precision == LBM_FP32) st = init_state<float, float>(c, rho_init, u_init, solid ? sol.data() : nullptr);
    else st = init_state<__half, float>(c, rho_init, u_init, solid ? sol.data() : nullptr);
    if (st != LBM_OK) {
        const std::string msg = c->err;
        free_ctx(c);
        return fail(nullptr, st, msg);
    }
    *out = c;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int64_t nsteps) {
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (c->d3) return lbm3::step(c->d3, nsteps);
    if (nsteps < 0) return fail(c, LBM_ERR_INVALID_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return LBM_OK;
    if (c->schedule == LBM_SCHEDULE_PERSISTENT) {
        if (!c->solo) {
            lbm_ctx* one[1] = {c};
            lbm_status st = lbm_batch_create(one, 1, c->stream, &c->solo);
            if (st == LBM_OK) st = lbm_batch_set_schedule(c->solo, LBM_SCHEDULE_PERSISTENT);
            if (st != LBM_OK) {
                const std::string msg = c->solo ? c->solo->err : lbm_last_error(nullptr);
                lbm_batch_destroy(c->solo);
                c->solo = nullptr;
                return fail(c, st, msg);
            }
        }
        lbm_status st = batch_run_any(c->solo, nsteps);
        if (st != LBM_OK) return fail(c, st, c->solo->err);
        return LBM_OK;
    }
    if (c->precision == LBM_FP64) return run_steps<double, double>(c, nsteps);
    if (c->precision == LBM_FP32) return run_steps<float, float>(c, nsteps);
    return run_steps<__half, float>(c, nsteps);
}

lbm_status lbm_reset(lbm_ctx* c, const double* rho_init, const double* u_init) {
    if (!c || !rho_init) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    if (c->d3) return lbm3::reset(c->d3, rho_init, u_init);
    const uint8_t* sol = c->host_solid_in.data();
    if (c->precision == LBM_FP64) return init_state<double, double>(c, rho_init, u_init, sol);
    if (c->precision == LBM_FP32) return init_state<float, float>(c, rho_init, u_init, sol);
    return init_state<__half, float>(c, rho_init, u_init, sol);
}

lbm_status lbm_sync(lbm_ctx* c) {
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (c->d3) return lbm3::sync(c->d3);
    if (c->solo) {
        lbm_status st = lbm_batch_sync(c->solo);
        if (st != LBM_OK) return fail(c, st, c->solo->err);
    }
    return check_status(c);
}

lbm_status lbm_set_schedule(lbm_ctx* c, int schedule) {
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (c->d3) return fail(c, LBM_ERR_UNSUPPORTED, "not implemented for D3Q19 contexts");
    if (schedule != LBM_SCHEDULE_GRAPHS && schedule != LBM_SCHEDULE_PERSISTENT &&
        schedule != LBM_SCHEDULE_GRAPHS_EARLY)
        return fail(c, LBM_ERR_INVALID_ARG, "unknown schedule");
    if (schedule == LBM_SCHEDULE_PERSISTENT && c->precision != LBM_FP32)
        return fail(c, LBM_ERR_UNSUPPORTED, "the persistent schedule is built for FP32 storage only");
    if (schedule == LBM_SCHEDULE_PERSISTENT && c->chi_same_step)
        return fail(c, LBM_ERR_UNSUPPORTED, "the persistent schedule runs the lagged chi only");
    CK(cudaStreamSynchronize(c->stream));
    if ((schedule == LBM_SCHEDULE_GRAPHS_EARLY) != (c->schedule == LBM_SCHEDULE_GRAPHS_EARLY))
        for (int p = 0; p < 2; ++p)  // graphs of the other form
            if (c->gexec[p]) {
                cudaGraphExecDestroy(c->gexec[p]);
                c->gexec[p] = nullptr;
                c->gexec_early[p] = 0;
            }
    c->schedule = schedule;
    return LBM_OK;
}

lbm_status lbm_get_schedule(lbm_ctx* c, int* schedule, int* early_in_use) {
    if (!c || !schedule || !early_in_use) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    *schedule = c->d3 ? LBM_SCHEDULE_GRAPHS : c->schedule;
    *early_in_use = c->d3 ? 0 : ((c->gexec[0] && c->gexec_early[0]) || (c->gexec[1] && c->gexec_early[1]));
    return LBM_OK;
}

lbm_status lbm_set_wall_velocity(lbm_ctx* c, int side, double ux) {
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (c->d3) return fail(c, LBM_ERR_UNSUPPORTED, "not implemented for D3Q19 contexts");
    if (side != LBM_YMIN && side != LBM_YMAX) return fail(c, LBM_ERR_INVALID_ARG, "side must be LBM_YMIN or LBM_YMAX");
    if (c->grid.periodic[1] || c->open_side[side])
        return fail(c, LBM_ERR_INVALID_ARG, "a moving wall needs a closed (non-periodic, not open) y edge");
    if (!std::isfinite(ux) || std::fabs(ux) > 0.2) return fail(c, LBM_ERR_INVALID_ARG, "wall speed must be finite and |u| <= 0.2");
    if (ux != 0.0 && c->precision == LBM_FP32_FP16STORE)
        return fail(c, LBM_ERR_UNSUPPORTED, "moving walls are built for FP32 and FP64 storage");
    CK(cudaStreamSynchronize(c->stream));
    c->wall_ux[side == LBM_YMIN ? 0 : 1] = ux;
    for (int p = 0; p < 2; ++p)  // captured steps carry the old arguments
        if (c->gexec[p]) {
            cudaGraphExecDestroy(c->gexec[p]);
            c->gexec[p] = nullptr;
        }
    return LBM_OK;
}

lbm_status lbm_set_wetting(lbm_ctx* c, double delta) {
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (c->d3) return fail(c, LBM_ERR_UNSUPPORTED, "not implemented for D3Q19 contexts");
    if (!std::isfinite(delta) || delta > 1.0) return fail(c, LBM_ERR_INVALID_ARG, "delta must be in (0, 1], or <= 0 to switch off");
    CK(cudaStreamSynchronize(c->stream));
    c->wet_delta = delta > 0.0 ? delta : 0.0;
    for (int p = 0; p < 2; ++p)  // captured steps carry the old arguments
        if (c->gexec[p]) {
            cudaGraphExecDestroy(c->gexec[p]);
            c->gexec[p] = nullptr;
        }
    return LBM_OK;
}

lbm_status lbm_set_chi_timing(lbm_ctx* c, int same_step) {
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (c->d3) return fail(c, LBM_ERR_UNSUPPORTED, "not implemented for D3Q19 contexts");
    if (same_step && c->precision == LBM_FP32_FP16STORE)
        return fail(c, LBM_ERR_UNSUPPORTED, "same-step chi is built for FP32 and FP64 storage");
    if (same_step && c->schedule == LBM_SCHEDULE_PERSISTENT)
        return fail(c, LBM_ERR_UNSUPPORTED, "the persistent schedule runs the lagged chi only");
    CK(cudaStreamSynchronize(c->stream));
    const bool on = same_step && c->out_face >= 0 && c->faces[c->out_face].chi;
    if (on && !c->oc_state) {
        const size_t bytes = (size_t)std::max(1, c->nface_nodes) * OC_STRIDE * c->rbytes;
        CK(cudaMalloc(&c->oc_state, bytes));
        CK(cudaMemset(c->oc_state, 0, bytes));
    }
    c->chi_same_step = on ? 1 : 0;
    for (int p = 0; p < 2; ++p)  // captured steps carry the old launch sequence
        if (c->gexec[p]) {
            cudaGraphExecDestroy(c->gexec[p]);
            c->gexec[p] = nullptr;
        }
    return LBM_OK;
}

lbm_status lbm_get_macros(lbm_ctx* c, float* rho, float* u, int dst_is_device) {
    if (!c || !rho || !u) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    if (c->d3) return lbm3::get_macros(c->d3, rho, u, dst_is_device);
    lbm_status st = check_status(c);
    if (st != LBM_OK) return st;
    if (c->rbytes == 8) return copy_macros<double>(c, rho, u, false, dst_is_device != 0);
    return copy_macros<float>(c, rho, u, false, dst_is_device != 0);
}

lbm_status lbm_get_macros_f64(lbm_ctx* c, double* rho, double* u) {
    if (!c || !rho || !u) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    if (c->d3) return lbm3::get_macros_f64(c->d3, rho, u);
    lbm_status st = check_status(c);
    if (st != LBM_OK) return st;
    if (c->rbytes == 8) return copy_macros<double>(c, rho, u, true, false);
    return copy_macros<float>(c, rho, u, true, false);
}

lbm_status lbm_get_populations(lbm_ctx* c, double* f) {
    if (!c || !f) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    if (c->d3) return lbm3::get_populations(c->d3, f);
    if (c->precision == LBM_FP64) return download_f<double>(c, f);
    if (c->precision == LBM_FP32) return download_f<float>(c, f);
    return download_f<__half>(c, f);
}

lbm_status lbm_set_populations(lbm_ctx* c, const double* f) {
    if (!c || !f) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    if (c->d3) return lbm3::set_populations(c->d3, f);
    if (c->precision == LBM_FP64) return upload_f<double>(c, f, c->cur);
    if (c->precision == LBM_FP32) return upload_f<float>(c, f, c->cur);
    return upload_f<__half>(c, f, c->cur);
}

lbm_status lbm_get_diagnostics(lbm_ctx* c, lbm_diag* out) {
    if (!c || !out) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    if (c->d3) return lbm3::diagnostics(c->d3, out);
    cudaError_t e;
    const int px = c->grid.periodic[0] ? 1 : 0, py = c->grid.periodic[1] ? 1 : 0;
    const void* rr = c->rref[c->cur];
    if (c->precision == LBM_FP64)
        e = launch_d2q9_diag<double, double>((const double*)c->f[c->cur], (const double*)c->macro, c->info, rr,
                                             c->nx, c->ny, px, py, c->pitch, c->plane, c->diag_partials,
                                             c->diag_blocks, c->stream);
    else if (c->precision == LBM_FP32)
        e = launch_d2q9_diag<float, float>((const float*)c->f[c->cur], (const float*)c->macro, c->info, rr, c->nx,
                                           c->ny, px, py, c->pitch, c->plane, c->diag_partials, c->diag_blocks,
                                           c->stream);
    else
        e = launch_d2q9_diag<__half, float>((const __half*)c->f[c->cur], (const float*)c->macro, c->info, rr,
                                            c->nx, c->ny, px, py, c->pitch, c->plane, c->diag_partials,
                                            c->diag_blocks, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "diag launch");
    c->launches += 1;
    std::vector<double> part((size_t)c->diag_blocks * 3);
    double sc[8];
    unsigned int stw = 0;
    CK(cudaMemcpyAsync(part.data(), c->diag_partials, part.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(sc, c->scal[c->cur], sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&stw, c->status, sizeof(stw), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double m0 = 0.0, m1 = 0.0, u2 = 0.0;
    for (int b = 0; b < c->diag_blocks; ++b) {
        m0 += part[(size_t)b * 3];
        m1 += part[(size_t)b * 3 + 1];
        u2 = std::max(u2, part[(size_t)b * 3 + 2]);
    }
    out->mass[0] = m0;
    out->mass[1] = m1;
    // lambda / chi the next step will use: the same sums the outlet tiles form
    out->lambda = sc[0];
    out->chi = sc[1];
    out->q_in = 0.0;
    out->q_out = 0.0;
    if (sc[5] != 0.0 && c->nslots > 0) {
        std::vector<double> pp((size_t)c->nslots * 4);
        CK(cudaMemcpy(pp.data(), c->partials[c->cur], pp.size() * 8, cudaMemcpyDeviceToHost));
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int sl = 0; sl < c->nslots; ++sl)
            for (int j = 0; j < 4; ++j) t[j] += pp[(size_t)sl * 4 + j];
        out->q_in = t[0];
        out->q_out = t[1];
        if (c->out_face >= 0 && t[3] > 0.0) {
            const double um = t[2] / t[3];
            out->lambda = um > 0.0 ? um : 0.0;
            out->chi = (!c->have_inlet || std::fabs(t[1]) < 1e-14) ? 1.0 : t[0] / t[1];
        }
    }
    out->max_speed = std::sqrt(u2);
    out->step = c->step;
    out->launches = c->launches;
    out->status = stw ? LBM_ERR_DIVERGED : LBM_OK;
    return LBM_OK;
}

lbm_status lbm_save(lbm_ctx* c, const char* path) {
    if (!c || !path) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    if (c->d3) return fail(c, LBM_ERR_UNSUPPORTED, "not implemented for D3Q19 contexts");
    CK(cudaStreamSynchronize(c->stream));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(c, LBM_ERR_IO, std::string("cannot open ") + path);
    const size_t fbytes = (size_t)18 * c->plane * c->sbytes;
    const size_t nfn = (size_t)std::max(1, c->nface_nodes);
    const size_t mbytes = (size_t)4 * c->plane * c->rbytes;
    const size_t pbytes = (size_t)std::max(1, c->nslots) * 4 * 8;
    const size_t rbytes_ref = (size_t)2 * c->plane * 2;
    std::vector<char> buf(fbytes + nfn * 8 * c->rbytes + nfn * 18 * c->rbytes + 64 + mbytes + pbytes + rbytes_ref);
    char* p = buf.data();
    CK(cudaMemcpy(p, c->f[c->cur], fbytes, cudaMemcpyDeviceToHost));
    p += fbytes;
    CK(cudaMemcpy(p, c->Fp[c->cur], nfn * 8 * c->rbytes, cudaMemcpyDeviceToHost));
    p += nfn * 8 * c->rbytes;
    CK(cudaMemcpy(p, c->fo[c->cur], nfn * 18 * c->rbytes, cudaMemcpyDeviceToHost));
    p += nfn * 18 * c->rbytes;
    CK(cudaMemcpy(p, c->scal[c->cur], 64, cudaMemcpyDeviceToHost));
    p += 64;
    CK(cudaMemcpy(p, c->macro, mbytes, cudaMemcpyDeviceToHost));
    p += mbytes;
    CK(cudaMemcpy(p, c->partials[c->cur], pbytes, cudaMemcpyDeviceToHost));
    p += pbytes;
    CK(cudaMemcpy(p, c->rref[c->cur], rbytes_ref, cudaMemcpyDeviceToHost));
    const char magic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '3'};
    const int64_t hdr[6] = {c->nx, c->ny, c->precision, c->nface_nodes, c->step, (int64_t)buf.size()};
    bool ok = std::fwrite(magic, 1, 8, fp) == 8 && std::fwrite(hdr, sizeof(hdr), 1, fp) == 1 &&
              std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(c, LBM_ERR_IO, std::string("write failed: ") + path);
    return LBM_OK;
}

lbm_status lbm_load(lbm_ctx* c, const char* path) {
    if (!c || !path) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    if (c->d3) return fail(c, LBM_ERR_UNSUPPORTED, "not implemented for D3Q19 contexts");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(c, LBM_ERR_IO, std::string("cannot open ") + path);
    char magic[8];
    int64_t hdr[6];
    const size_t fbytes = (size_t)18 * c->plane * c->sbytes;
    const size_t nfn = (size_t)std::max(1, c->nface_nodes);
    const size_t mbytes = (size_t)4 * c->plane * c->rbytes;
    const size_t pbytes = (size_t)std::max(1, c->nslots) * 4 * 8;
    const size_t rbytes_ref = (size_t)2 * c->plane * 2;
    const size_t total = fbytes + nfn * 8 * c->rbytes + nfn * 18 * c->rbytes + 64 + mbytes + pbytes + rbytes_ref;
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "LBMCKPT3", 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, fp) == 1 && hdr[0] == c->nx && hdr[1] == c->ny &&
              hdr[2] == c->precision && hdr[3] == c->nface_nodes && hdr[5] == (int64_t)total;
    std::vector<char> buf(total);
    ok = ok && std::fread(buf.data(), 1, total, fp) == total;
    std::fclose(fp);
    if (!ok) return fail(c, LBM_ERR_IO, std::string("not a matching checkpoint: ") + path);
    CK(cudaStreamSynchronize(c->stream));
    const char* p = buf.data();
    CK(cudaMemcpy(c->f[c->cur], p, fbytes, cudaMemcpyHostToDevice));
    p += fbytes;
    CK(cudaMemcpy(c->Fp[c->cur], p, nfn * 8 * c->rbytes, cudaMemcpyHostToDevice));
    p += nfn * 8 * c->rbytes;
    CK(cudaMemcpy(c->fo[c->cur], p, nfn * 18 * c->rbytes, cudaMemcpyHostToDevice));
    p += nfn * 18 * c->rbytes;
    CK(cudaMemcpy(c->scal[c->cur], p, 64, cudaMemcpyHostToDevice));
    p += 64;
    CK(cudaMemcpy(c->macro, p, mbytes, cudaMemcpyHostToDevice));
    p += mbytes;
    CK(cudaMemcpy(c->partials[c->cur], p, pbytes, cudaMemcpyHostToDevice));
    p += pbytes;
    CK(cudaMemcpy(c->rref[c->cur], p, rbytes_ref, cudaMemcpyHostToDevice));
    c->step = hdr[4];
    return LBM_OK;
}

lbm_status lbm_enable_kernel_timing(lbm_ctx* c, int every) {
    if (!c || every < 0) return fail(c, LBM_ERR_INVALID_ARG, "bad timing request");
    if (c->d3) return lbm3::enable_timing(c->d3, every);
    CK(cudaStreamSynchronize(c->stream));
    c->timing_every = every;
    c->n_samples = 0;
    return LBM_OK;
}

lbm_status lbm_kernel_time(lbm_ctx* c, double* mean_ms, int64_t* samples) {
    double fast = 0.0, gen = 0.0;
    lbm_status st = lbm_kernel_time_split(c, &fast, &gen, samples);
    if (st != LBM_OK) return st;
    *mean_ms = fast + gen;
    return LBM_OK;
}

lbm_status lbm_kernel_time_split(lbm_ctx* c, double* fast_ms, double* general_ms, int64_t* samples) {
    if (!c || !fast_ms || !general_ms || !samples) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    if (c->d3) return lbm3::kernel_time_split(c->d3, fast_ms, general_ms, samples);
    CK(cudaStreamSynchronize(c->stream));
    double tf = 0.0, tg = 0.0;
    for (int i = 0; i < c->n_samples; ++i) {
        float a = 0.0f, b = 0.0f;
        CK(cudaEventElapsedTime(&a, c->ev_start[i], c->ev_mid[i]));
        CK(cudaEventElapsedTime(&b, c->ev_mid[i], c->ev_stop[i]));
        tf += a;
        tg += b;
    }
    *samples = c->n_samples;
    *fast_ms = c->n_samples ? tf / c->n_samples : 0.0;
    *general_ms = c->n_samples ? tg / c->n_samples : 0.0;
    return LBM_OK;
}

lbm_status lbm_set_tile_variant(lbm_ctx* c, int variant) {
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (c->d3) return fail(c, LBM_ERR_UNSUPPORTED, "not implemented for D3Q19 contexts");
    return build_tiles(c, variant, true);
}

int lbm_num_tile_variants(void) { return d2q9_num_variants(); }

lbm_status lbm_tile_stats(lbm_ctx* c, int* variant, int* fast_tiles, int* general_tiles, int64_t* fast_nodes,
                          int64_t* general_nodes) {
    if (!c || !variant || !fast_tiles || !general_tiles || !fast_nodes || !general_nodes)
        return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    if (c->d3) return fail(c, LBM_ERR_UNSUPPORTED, "not implemented for D3Q19 contexts");
    *variant = c->variant;
    *fast_tiles = c->nfast + c->march_tiles;
    *general_tiles = c->ngeneral;
    *fast_nodes = c->fast_nodes;
    *general_nodes = c->general_nodes;
    return LBM_OK;
}

lbm_status lbm_set_graph_mode(lbm_ctx* c, int use_graphs) {
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (c->d3) return LBM_OK;  // D3Q19 steps are plain launches
    c->use_graphs = use_graphs ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_batch_create(lbm_ctx* const* members, int n, void* cuda_stream, lbm_batch** out) {
    if (!out) return bfail(nullptr, LBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!members || n < 1) return bfail(nullptr, LBM_ERR_INVALID_ARG, "need at least one member");
    for (int i = 0; i < n; ++i)
        if (members[i] && members[i]->d3)
            return bfail(nullptr, LBM_ERR_UNSUPPORTED, "batches of D3Q19 contexts are not implemented");
    for (int i = 0; i < n; ++i) {
        if (!members[i]) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL member");
        if (members[i]->precision != members[0]->precision)
            return bfail(nullptr, LBM_ERR_INVALID_ARG, "members must share one precision");
        if (members[i]->chi_same_step)
            return bfail(nullptr, LBM_ERR_UNSUPPORTED, "batches run the lagged chi only (lbm_set_chi_timing)");
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return bfail(nullptr, LBM_ERR_INVALID_ARG, "a member appears twice");
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ERR_OOM, "host allocation failed");
    b->m.assign(members, members + n);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->precision = members[0]->precision;
    b->variant = members[0]->variant;
    lbm_status st = LBM_OK;
    for (lbm_ctx* c : b->m)
        if (st == LBM_OK && c->variant != b->variant) st = build_tiles(c, b->variant, true);
    if (st == LBM_OK) st = batch_build_any(b);
    if (st != LBM_OK) {
        const std::string msg = b->err;
        free_batch_lists(b);
        delete b;
        return bfail(nullptr, st, msg);
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps) {
    if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "batch is NULL");
    if (nsteps < 0) return bfail(b, LBM_ERR_INVALID_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return LBM_OK;
    return batch_run_any(b, nsteps);
}

lbm_status lbm_batch_sync(lbm_batch* b) {
    if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "batch is NULL");
    BCK(cudaStreamSynchronize(b->stream));
    if (b->pstatus) {
        unsigned ps = 0;
        BCK(cudaMemcpy(&ps, b->pstatus, sizeof(ps), cudaMemcpyDeviceToHost));
        if (ps & PERSIST_TIMEOUT) {
            BCK(cudaMemset(b->pstatus, 0, sizeof(unsigned)));  // reported once; reset the members to go on
            return bfail(b, LBM_ERR_TIMEOUT,
                         "a grid barrier of the persistent schedule timed out; the members' states are undefined");
        }
    }
    for (lbm_ctx* c : b->m) {
        lbm_status st = check_status(c);
        if (st != LBM_OK) return bfail(b, st, c->err);
    }
    return LBM_OK;
}

lbm_status lbm_batch_set_tile_variant(lbm_batch* b, int variant) {
    if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "batch is NULL");
    if (variant < 0 || variant >= d2q9_num_variants()) return bfail(b, LBM_ERR_INVALID_ARG, "unknown tile variant");
    BCK(cudaStreamSynchronize(b->stream));
    for (lbm_ctx* c : b->m) BCK(cudaStreamSynchronize(c->stream));
    for (lbm_ctx* c : b->m) {
        lbm_status st = build_tiles(c, variant, true);
        if (st != LBM_OK) return bfail(b, st, c->err);
    }
    b->variant = variant;
    return batch_build_any(b);
}

lbm_status lbm_batch_autotune(lbm_batch* b, int steps, int* variant, double* ms_per_step) {
    if (!b || !variant || steps < 1) return bfail(b, LBM_ERR_INVALID_ARG, "bad autotune request");
    return batch_autotune(b, steps, variant, ms_per_step);
}

lbm_status lbm_autotune(lbm_ctx* c, int steps, int* variant, double* ms_per_step) {
    if (!c || !variant || steps < 1) return fail(c, LBM_ERR_INVALID_ARG, "bad autotune request");
    if (c->d3) return fail(c, LBM_ERR_UNSUPPORTED, "not implemented for D3Q19 contexts");
    lbm_batch* b = nullptr;
    lbm_ctx* one[1] = {c};
    lbm_status st = lbm_batch_create(one, 1, c->stream, &b);
    if (st != LBM_OK) return fail(c, st, lbm_last_error(nullptr));
    double best_ms = 0.0;
    st = batch_autotune(b, steps, variant, &best_ms);
    if (st != LBM_OK) fail(c, st, b->err);
    lbm_batch_destroy(b);
    if (st == LBM_OK && c->precision == LBM_FP32) st = autotune_march(c, steps, variant, &best_ms);
    if (st == LBM_OK && ms_per_step) *ms_per_step = best_ms;
    return st;
}

lbm_status lbm_batch_info(lbm_batch* b, int* variant, int* fast_tiles, int* general_tiles, int64_t* launches) {
    if (!b || !variant || !fast_tiles || !general_tiles || !launches)
        return bfail(b, LBM_ERR_INVALID_ARG, "NULL argument");
    *variant = b->variant;
    *fast_tiles = b->nfast;
    *general_tiles = b->ngeneral;
    *launches = b->launches;
    return LBM_OK;
}

lbm_status lbm_batch_set_graph_mode(lbm_batch* b, int use_graphs) {
    if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "batch is NULL");
    b->use_graphs = use_graphs ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_batch_set_schedule(lbm_batch* b, int schedule) {
    if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "batch is NULL");
    if (schedule != LBM_SCHEDULE_GRAPHS && schedule != LBM_SCHEDULE_PERSISTENT &&
        schedule != LBM_SCHEDULE_GRAPHS_EARLY)
        return bfail(b, LBM_ERR_INVALID_ARG, "unknown schedule");
    if (schedule == LBM_SCHEDULE_PERSISTENT && b->precision != LBM_FP32)
        return bfail(b, LBM_ERR_UNSUPPORTED, "the persistent schedule is built for FP32 storage only");
    if ((schedule == LBM_SCHEDULE_GRAPHS_EARLY) != (b->schedule == LBM_SCHEDULE_GRAPHS_EARLY)) {
        BCK(cudaStreamSynchronize(b->stream));
        for (int p = 0; p < 2; ++p)
            if (b->gexec[p]) {
                cudaGraphExecDestroy(b->gexec[p]);
                b->gexec[p] = nullptr;
                b->gexec_early[p] = 0;
            }
    }
    b->schedule = schedule;
    return LBM_OK;
}

lbm_status lbm_batch_get_schedule(lbm_batch* b, int* schedule, int* early_in_use) {
    if (!b || !schedule || !early_in_use) return bfail(b, LBM_ERR_INVALID_ARG, "NULL argument");
    *schedule = b->schedule;
    *early_in_use = (b->gexec[0] && b->gexec_early[0]) || (b->gexec[1] && b->gexec_early[1]);
    return LBM_OK;
}

lbm_status lbm_batch_persistent_grid(lbm_batch* b, int* ctas) {
    if (!b || !ctas) return bfail(b, LBM_ERR_INVALID_ARG, "NULL argument");
    *ctas = b->persist_grid;
    return LBM_OK;
}

lbm_status lbm_batch_inject_barrier_fault(lbm_batch* b, int extra_arrivals, int64_t spin_limit_cycles) {
    if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "batch is NULL");
    if (extra_arrivals < 0) return bfail(b, LBM_ERR_INVALID_ARG, "extra_arrivals must be >= 0");
    BCK(cudaStreamSynchronize(b->stream));
    b->bar_skew = extra_arrivals;
    b->spin_limit = spin_limit_cycles > 0 ? (long long)spin_limit_cycles : kDefaultSpinLimit;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_batch_lists(b);
    if (b->pbar) cudaFree(b->pbar);
    if (b->pstatus) cudaFree(b->pstatus);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->side_stream) cudaStreamDestroy(b->side_stream);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : lbm_last_error(nullptr); }

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    if (c->d3) {
        lbm3::destroy(c->d3);
        delete c;
        return;
    }
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_ctx(c);
}

}  // extern "C"
