// klb_adjoint.cu -- the adjoint run: forward with checkpoints, reverse sweep
// with recomputation per segment, and the sensitivities of the initial
// fields.  The kernels live in klb_adjoint.cuh.
//
// Objective (Sec. IV of arXiv:1010.4124: the perturbation kinetic energy
// E_x = rho u_y^2 / 2 and the growth coefficient fitted to its logarithm):
//   KE    = dx dy sum_nodes rho u_y^2 / 2 at the last step,
//   gamma = (1/2) OLS slope of ln K_s over the fit window (the last 75% of the
//           samples), K_s = sum_nodes rho u_y^2 / 2 of sample s,
// L = g_KE KE + g_gamma gamma.  The reverse sweep adds the sources
// dL/dK_s dK_s/df at the sampled steps.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <deque>
#include <vector>

#include "klb_adjoint.cuh"
#include "klb_handle.h"

using namespace fdlb;

namespace fdlb {
KLB_BOUNDS_QUERY(bounds_flag_adjoint)
}  // namespace fdlb

struct AdjMap {  // a TMA map of one buffer for the tile kernel
    const void* buf = nullptr;
    unsigned box[3] = {0, 0, 0};
    CUtensorMap map;
};

struct klb_adj {
    klb_t* h = nullptr;            // forward grid (owns the step buffers)
    int64_t nsteps = 0;
    int ckpt = 0;                  // steps per checkpoint segment
    int nck = 0;                   // checkpoints (segment starts)
    std::vector<void*> ck;         // state at the start of each segment (full buffers)
    std::vector<void*> seg;        // states of one segment during the reverse sweep (ckpt - 1 extra)
    void* lam[2] = {nullptr, nullptr};
    void* Nb = nullptr;            // per-node f^(0) sensitivity and u_y (5 * nx * ny)
    double* fields = nullptr;      // the initial fields (4 * nx * ny)
    double* dense = nullptr;       // staging for host / dense arrays (19 * nx * ny)
    std::deque<AdjMap> maps;       // TMA maps of the buffers above (stable addresses)
    InstDesc* rdescs = nullptr;    // FP32: step descriptors of the recomputation chains (device)
    int rdescs_variant = -1;       // the tile shape they were built for
    double* coef_dev = nullptr;    // the objective's weight of each reverse step (nsteps)
    std::vector<double> coef_host;
    bool use_graph = true;         // forward and reverse sweep replayed from CUDA graphs
    cudaGraphExec_t sweep_graph = nullptr;
    int64_t sweep_launches = 0;
    int lam_final = 0;             // the lambda buffer that holds lambda^0 after the sweep
    cudaGraphExec_t fwd_graph = nullptr;  // checkpoints and steps of the forward run
    int64_t fwd_launches = 0;
    int fwd_cur = 0;               // the grid's bookkeeping after the forward run
    int64_t fwd_steps = 0;
    bool fwd_pending = false;
    int fwd_variant = -1;          // the grid's tile shape and wait budget the graphs were captured with
    long long fwd_spin = 0;
    long long sweep_spin = 0;
    std::vector<double> K;         // K_s of the forward run
    double ke = 0, gamma = 0;
    bool forward_done = false;
    std::string err;
};

static thread_local std::string g_adj_create_error;

static int afail(klb_adj_t* a, int code, const std::string& msg) {
    if (a) a->err = msg;
    else g_adj_create_error = msg;
    return code;
}
#define ACK(a, call)                                                                                          \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess) return afail(a, KLB_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static int grid_of(long long n) {
    long long b = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 152 * 32));
}

static size_t state_bytes(const klb_t* h) { return (size_t)NQ * h->g.plane * h->esize; }

// The TMA map of a state-shaped buffer (a checkpoint, a recomputed state, a
// lambda) with a box of bx x by x bz elements, encoded once per buffer and box.
static const CUtensorMap* adj_map(klb_adj_t* a, const void* buf, unsigned bx, unsigned by, unsigned bz) {
    for (const auto& m : a->maps)
        if (m.buf == buf && m.box[0] == bx && m.box[1] == by && m.box[2] == bz) return &m.map;
    AdjMap m;
    m.buf = buf;
    m.box[0] = bx;
    m.box[1] = by;
    m.box[2] = bz;
    if (encode_state_map(a->h, buf, bx, by, bz, &m.map) != KLB_OK) return nullptr;
    a->maps.push_back(m);
    return &a->maps.back().map;
}

// the node kernel: one CTA per segment of kNodeSeg nodes of each row
static dim3 node_grid(const Geom& g) { return dim3((unsigned)((g.nx + kNodeSeg - 1) / kNodeSeg), (unsigned)g.ny); }

// tile rows of the fused reverse step: 16 in FP32 (fewer y faces evaluated
// twice at tile borders), 8 in FP64 (its shared memory stays within the
// static 48 KB)
template <typename T>
constexpr int adj_rows() { return sizeof(T) == 4 ? 16 : 8; }

// the ghost sums of lambda folded into the nodes they image
template <typename T>
static void launch_fold(const Geom& g, T* lam, cudaStream_t s) {
    const int nbx = band_count(g.nx, g.bcx_lo, g.bcx_hi), nby = band_count(g.ny, g.bcy_lo, g.bcy_hi);
    const long long work = (long long)NQ * ((long long)nbx * g.ny + (long long)nby * g.nx);
    if (work > 0) adj_fold_kernel<T><<<grid_of(work), 256, 0, s>>>(g, lam, nbx, nby);
}

template <typename T>
static int vjp_step(klb_adj_t* a, const void* f, void* lam_in, void* lam_out, int64_t n) {
    klb_t* h = a->h;
    const StepConst<T>& c = *reinterpret_cast<const StepConst<T>*>(sizeof(T) == 8 ? (const void*)&h->cd
                                                                                   : (const void*)&h->cf);
    const Geom& g = h->g;
    // fold lambda^{n+1}'s ghost sums into its nodes, form the per-node f^(0)
    // sensitivities, then the fused faces-and-gather pass
    using A = AdjTile<T, adj_rows<T>()>;
    const CUtensorMap* fmap = adj_map(a, f, A::BW, A::FR, 1);
    const CUtensorMap* lmap = adj_map(a, lam_in, A::BW, A::LR, 1);
    const CUtensorMap* fnode = adj_map(a, f, kNodeSeg, 1, NQ);
    const CUtensorMap* lnode = adj_map(a, lam_in, kNodeSeg, 1, NQ);
    if (!fmap || !lmap || !fnode || !lnode) return afail(a, KLB_E_CUDA, h->err);
    launch_fold<T>(g, (T*)lam_in, h->stream);
    adj_node_kernel<T><<<node_grid(g), kNodeSeg, 0, h->stream>>>(*fnode, *lnode, c, g, (T*)a->Nb, h->err_dev,
                                                                 h->spin_limit);
    const long long tiles = (long long)A::tiles_x(g.nx) * A::tiles_y(g.ny);
    adj_tile_kernel<T, adj_rows<T>()><<<dim3((unsigned)tiles, NQ), 32 * adj_rows<T>(), 0, h->stream>>>(
        *fmap, *lmap, c, g, (const T*)a->Nb, a->coef_dev, (int)n, (T*)lam_out, h->err_dev, h->spin_limit);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return afail(a, KLB_E_CUDA, std::string("adjoint kernels: ") + cudaGetErrorString(e));
    h->launches += 3;
    return KLB_OK;
}

// the ghost sums of the last lambda folded into its nodes
template <typename T>
static int fold(klb_adj_t* a, void* lam) {
    klb_t* h = a->h;
    launch_fold<T>(h->g, (T*)lam, h->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return afail(a, KLB_E_CUDA, std::string("adjoint fold: ") + cudaGetErrorString(e));
    h->launches += 1;
    return KLB_OK;
}

static int vjp(klb_adj_t* a, const void* f, void* lam_in, void* lam_out, int64_t n) {
    return a->h->p.precision == KLB_FP64 ? vjp_step<double>(a, f, lam_in, lam_out, n)
                                         : vjp_step<float>(a, f, lam_in, lam_out, n);
}

template <typename T>
static int source(klb_adj_t* a, const void* f, double coef, void* lam) {
    klb_t* h = a->h;
    const StepConst<T>& c = *reinterpret_cast<const StepConst<T>*>(sizeof(T) == 8 ? (const void*)&h->cd
                                                                                   : (const void*)&h->cf);
    adj_source_kernel<T><<<grid_of((long long)h->g.nx * h->g.ny), 256, 0, h->stream>>>(c, h->g, (const T*)f, T(coef),
                                                                                        (T*)lam);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return afail(a, KLB_E_CUDA, std::string("adjoint source: ") + cudaGetErrorString(e));
    h->launches += 1;
    return KLB_OK;
}

// sample index of step n (or -1 when n is not sampled)
static int sample_of(const klb_adj_t* a, int64_t n) {
    const int s = a->h->p.sample_every;
    return (n % s == 0) ? (int)(n / s) : -1;
}

// dL/dK_s of sample s
static double dL_dK(const klb_adj_t* a, int s, double g_ke, double g_gamma) {
    const klb_t* h = a->h;
    const int M = (int)a->K.size();
    double d = 0.0;
    if (s == M - 1) d += g_ke * h->p.dx * h->p.dy;
    const int start = M - (3 * M) / 4;
    if (g_gamma != 0.0 && s >= start && M - start >= 2) {
        // gamma = 1/2 sum_s w_s ln K_s, w_s = (t_s - tbar) / sum (t - tbar)^2
        const double dt = h->p.dt * h->p.sample_every;
        double tbar = 0.0;
        for (int k = start; k < M; ++k) tbar += k * dt;
        tbar /= (M - start);
        double sxx = 0.0;
        for (int k = start; k < M; ++k) sxx += (k * dt - tbar) * (k * dt - tbar);
        d += g_gamma * 0.5 * ((s * dt - tbar) / sxx) / a->K[s];
    }
    return d;
}

// One step of the recomputation from state buffer `in` into `out` (no
// sampling).  FP32: the step kernel reads its input through a device
// descriptor (TMA map of `in`, output pointer), one per (in, out) pair of the
// sweep, uploaded once per reverse sweep (desc_index); FP64: the map of `in`.
static int step_into(klb_adj_t* a, const void* in, void* out, int desc_index) {
    klb_t* h = a->h;
    cudaError_t e;
    if (h->p.precision == KLB_FP64) {
        int TX, TY;
        f64_tile(&TX, &TY);
        const CUtensorMap* m = adj_map(a, in, (unsigned)(TX + 8), (unsigned)(TY + 6), NQ);
        if (!m) return afail(a, KLB_E_CUDA, h->err);
        e = launch_step<double>(*m, h->cd, h->g, (double*)out, nullptr, h->err_dev, h->spin_limit, h->inject,
                                h->stream);
    } else {
        e = launch_step_f32(h->cf, a->rdescs + desc_index, 1, h->ntiles, nullptr, h->err_dev, h->spin_limit,
                            h->inject, h->variant, h->stream);
    }
    if (e != cudaSuccess) return afail(a, KLB_E_CUDA, std::string("step kernel: ") + cudaGetErrorString(e));
    h->launches += 1;
    return KLB_OK;
}

// FP32: the descriptors of the recomputation chains, for the grid's current
// tile shape: entry s steps checkpoint s into seg[0], entry nck + k steps
// seg[k] into seg[k + 1]
static int upload_recompute_descs(klb_adj_t* a) {
    klb_t* h = a->h;
    if (h->p.precision != KLB_FP32 || a->seg.empty() || a->rdescs_variant == h->variant) return KLB_OK;
    if (a->sweep_graph) {  // its step launches name the old tile shape
        cudaGraphExecDestroy(a->sweep_graph);
        a->sweep_graph = nullptr;
    }
    unsigned bx, by, bz;
    f32_box(h->variant, &bx, &by, &bz);
    int tiles_x, ntiles;
    f32_tiles(h->g.nx, h->g.ny, h->variant, &tiles_x, &ntiles);
    std::vector<InstDesc> d(a->nck + a->seg.size() - 1);
    for (size_t k = 0; k < d.size(); ++k) {
        const void* in = k < (size_t)a->nck ? a->ck[k] : a->seg[k - a->nck];
        void* out = k < (size_t)a->nck ? a->seg[0] : a->seg[k - a->nck + 1];
        memset(&d[k], 0, sizeof(InstDesc));
        if (encode_state_map(h, in, bx, by, bz, &d[k].map) != KLB_OK) return afail(a, KLB_E_CUDA, h->err);
        d[k].out = (float*)out;
        d[k].g = h->g;
        d[k].tiles_x = tiles_x;
        d[k].first_tile = 0;
    }
    ACK(a, cudaMemcpyAsync(a->rdescs, d.data(), d.size() * sizeof(InstDesc), cudaMemcpyHostToDevice, h->stream));
    ACK(a, cudaStreamSynchronize(h->stream));  // the host vector goes out of scope
    a->rdescs_variant = h->variant;
    return KLB_OK;
}

// The launches of the reverse sweep from lam[0] = lambda^N down to lambda^0
// (segments in reverse order: the recomputation of a segment's states, then
// its reverse steps; finally the fold of lambda^0's ghost sums).  The
// objective's weights are read from coef_dev, so the sequence is the same for
// every call: it is captured into a CUDA graph once and replayed.
static int sweep_launches(klb_adj_t* a) {
    int lc = 0, r = KLB_OK;
    for (int s = a->nck - 1; s >= 0; --s) {
        const int64_t n0 = (int64_t)s * a->ckpt;
        const int64_t n1 = std::min<int64_t>(n0 + a->ckpt, a->nsteps);
        const int len = (int)(n1 - n0);
        // recompute the segment's states f^{n0} .. f^{n1-1} from its checkpoint,
        // straight into the segment buffers
        std::vector<const void*> states(len);
        states[0] = a->ck[s];
        for (int k = 1; k < len; ++k) {
            r = step_into(a, states[k - 1], a->seg[k - 1], k == 1 ? s : a->nck + k - 2);
            if (r != KLB_OK) return r;
            states[k] = a->seg[k - 1];
        }
        for (int64_t n = n1 - 1; n >= n0; --n) {
            r = vjp(a, states[n - n0], a->lam[lc], a->lam[1 - lc], n);
            if (r != KLB_OK) return r;
            lc = 1 - lc;
        }
    }
    a->lam_final = lc;
    return a->h->p.precision == KLB_FP64 ? fold<double>(a, a->lam[lc]) : fold<float>(a, a->lam[lc]);
}

// the reverse sweep; with objective sources (g_ke, g_gamma) when `sources` is
// set; returns the buffer of lambda^0 in *lam_cur
static int reverse(klb_adj_t* a, bool sources, double g_ke, double g_gamma, int* lam_cur) {
    klb_t* h = a->h;
    int r = upload_recompute_descs(a);
    if (r != KLB_OK) return r;
    // the objective's weight of each reverse step (the samples it enters)
    for (int64_t n = 0; n < a->nsteps; ++n) {
        const int si = sample_of(a, n);
        a->coef_host[n] = (sources && si >= 0) ? dL_dK(a, si, g_ke, g_gamma) : 0.0;
    }
    ACK(a, cudaMemcpyAsync(a->coef_dev, a->coef_host.data(), sizeof(double) * a->nsteps, cudaMemcpyHostToDevice,
                           h->stream));
    if (a->sweep_graph && (a->sweep_spin != h->spin_limit || h->inject)) {  // stale wait budget
        cudaGraphExecDestroy(a->sweep_graph);
        a->sweep_graph = nullptr;
    }
    if (!a->sweep_graph && a->use_graph && !h->inject &&
        cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        a->use_graph = false;  // a stream that cannot be captured: launch eagerly
    }
    if (!a->sweep_graph && a->use_graph && !h->inject) {  // capturing
        a->sweep_spin = h->spin_limit;
        const int64_t l0 = h->launches;
        cudaGraph_t g = nullptr;
        r = sweep_launches(a);
        cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
        a->sweep_launches = h->launches - l0;
        h->launches = l0;
        if (r != KLB_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (ec != cudaSuccess || cudaGraphInstantiate(&a->sweep_graph, g, 0) != cudaSuccess) {
            a->sweep_graph = nullptr;
            a->use_graph = false;  // launch the sweep eagerly from now on
            cudaGetLastError();
        }
        if (g) cudaGraphDestroy(g);
    }
    if (a->sweep_graph) {
        ACK(a, cudaGraphLaunch(a->sweep_graph, h->stream));
        h->launches += a->sweep_launches;
    } else {
        r = sweep_launches(a);
        if (r != KLB_OK) return r;
    }
    *lam_cur = a->lam_final;
    return KLB_OK;
}

template <typename T>
static int fields_grad(klb_adj_t* a, const void* lam, double* d) {
    klb_t* h = a->h;
    const StepConst<T>& c = *reinterpret_cast<const StepConst<T>*>(sizeof(T) == 8 ? (const void*)&h->cd
                                                                                   : (const void*)&h->cf);
    const size_t n = (size_t)h->g.nx * h->g.ny;
    adj_fields_kernel<T><<<grid_of((long long)n), 256, 0, h->stream>>>(
        c, h->g, a->fields, a->fields + n, a->fields + 2 * n, a->fields + 3 * n, (const T*)lam, d, d + n, d + 2 * n,
        d + 3 * n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return afail(a, KLB_E_CUDA, std::string("adjoint fields: ") + cudaGetErrorString(e));
    h->launches += 1;
    return KLB_OK;
}

extern "C" {

int klb_adjoint_create(const klb_params* p, int64_t nsteps, int32_t checkpoint_every, klb_adj_t** out) {
    if (!p || !out) return afail(nullptr, KLB_E_INVAL, "NULL argument");
    *out = nullptr;
    if (nsteps < 1 || checkpoint_every < 1) return afail(nullptr, KLB_E_INVAL, "nsteps and checkpoint_every must be >= 1");
    if (p->sample_every < 1 || nsteps % p->sample_every != 0)
        return afail(nullptr, KLB_E_INVAL, "sample_every must be >= 1 and divide nsteps");
    const int bcs[4] = {p->bc_x_lo, p->bc_x_hi, p->bc_y_lo, p->bc_y_hi};
    for (int b : bcs)
        if (b == KLB_BC_FIXED_EQ || b == KLB_BC_HALO)
            return afail(nullptr, KLB_E_INVAL, "the adjoint supports periodic and outflow sides only");
    if (p->scheme != KLB_WENO5) return afail(nullptr, KLB_E_INVAL, "the adjoint differentiates the WENO5 step only");
    klb_params q = *p;
    q.diag_capacity = (int32_t)(nsteps / p->sample_every + 1);
    klb_adj_t* a = new klb_adj();
    a->nsteps = nsteps;
    a->ckpt = checkpoint_every;
    a->nck = (int)((nsteps + checkpoint_every - 1) / checkpoint_every);
    int r = klb_create(&q, &a->h);
    if (r != KLB_OK) {
        delete a;
        return afail(nullptr, r, std::string("forward grid: ") + klb_last_error(nullptr));
    }
    klb_t* h = a->h;  // an FP32 grid starts with the tile shape faster for its size
    // graph replay of the forward run and the reverse sweep (FP32: the step
    // kernels' attributes are set at creation, outside any capture)
    a->use_graph = h->p.precision == KLB_FP32;
    const size_t sb = state_bytes(h);
    const size_t nn = (size_t)h->g.nx * h->g.ny;
    bool ok = true;
    a->ck.assign(a->nck, nullptr);
    for (int s = 0; s < a->nck && ok; ++s) ok = cudaMalloc(&a->ck[s], sb) == cudaSuccess;
    a->seg.assign(std::max(0, a->ckpt - 1), nullptr);
    for (size_t s = 0; s < a->seg.size() && ok; ++s) ok = cudaMalloc(&a->seg[s], sb) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k) ok = cudaMalloc(&a->lam[k], sb) == cudaSuccess;
    ok = ok && cudaMalloc(&a->Nb, h->esize * 5 * nn) == cudaSuccess;
    ok = ok && cudaMalloc(&a->rdescs, sizeof(InstDesc) * (a->nck + a->seg.size() + 1)) == cudaSuccess;
    ok = ok && cudaMalloc(&a->coef_dev, sizeof(double) * nsteps) == cudaSuccess;
    a->coef_host.assign(nsteps, 0.0);
    ok = ok && cudaMalloc(&a->fields, sizeof(double) * 4 * nn) == cudaSuccess;
    ok = ok && cudaMalloc(&a->dense, sizeof(double) * NQ * nn) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        klb_adjoint_destroy(a);
        return afail(nullptr, KLB_E_NOMEM, "cudaMalloc of the checkpoints failed");
    }
    for (int k = 0; k < 2; ++k) cudaMemset(a->lam[k], 0, sb);
    *out = a;
    return KLB_OK;
}

void klb_adjoint_destroy(klb_adj_t* a) {
    if (!a) return;
    if (a->h) cudaStreamSynchronize(a->h->stream);
    for (void* p : a->ck)
        if (p) cudaFree(p);
    for (void* p : a->seg)
        if (p) cudaFree(p);
    for (int k = 0; k < 2; ++k)
        if (a->lam[k]) cudaFree(a->lam[k]);
    if (a->Nb) cudaFree(a->Nb);
    if (a->rdescs) cudaFree(a->rdescs);
    if (a->coef_dev) cudaFree(a->coef_dev);
    if (a->sweep_graph) cudaGraphExecDestroy(a->sweep_graph);
    if (a->fwd_graph) cudaGraphExecDestroy(a->fwd_graph);
    if (a->fields) cudaFree(a->fields);
    if (a->dense) cudaFree(a->dense);
    klb_destroy(a->h);
    delete a;
}

klb_t* klb_adjoint_grid(klb_adj_t* a) { return a ? a->h : nullptr; }

int klb_adjoint_forward(klb_adj_t* a, const double* rho, const double* ux, const double* uy, const double* T,
                        int on_device, double* ke, double* gamma) {
    fdlb::NvtxRange trace_("klb_adjoint_forward");
    if (!a || !rho || !ux || !uy || !T) return a ? afail(a, KLB_E_INVAL, "NULL argument") : KLB_E_INVAL;
    klb_t* h = a->h;
    const size_t nn = (size_t)h->g.nx * h->g.ny;
    const double* src[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        ACK(a, cudaMemcpyAsync(a->fields + k * nn, src[k], nn * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    int r = klb_init_fields(h, a->fields, a->fields + nn, a->fields + 2 * nn, a->fields + 3 * nn, 1);
    if (r != KLB_OK) return afail(a, r, h->err);
    // the checkpoint copies and steps of the run: the same launches for every
    // initial state, captured into a CUDA graph once and replayed
    auto run = [&]() -> int {
        for (int s = 0; s < a->nck; ++s) {
            ACK(a, cudaMemcpyAsync(a->ck[s], h->buf[h->cur], state_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
            const int64_t n = std::min<int64_t>(a->ckpt, a->nsteps - (int64_t)s * a->ckpt);
            int rr = klb_step(h, n);
            if (rr != KLB_OK) return afail(a, rr, h->err);
        }
        return KLB_OK;
    };
    // a graph captured for another tile shape or wait budget of the grid is stale
    if (a->fwd_graph && (a->fwd_variant != h->variant || a->fwd_spin != h->spin_limit || h->inject)) {
        cudaGraphExecDestroy(a->fwd_graph);
        a->fwd_graph = nullptr;
    }
    if (a->use_graph && !a->fwd_graph && !h->inject &&
        cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        a->use_graph = false;  // a stream that cannot be captured: launch eagerly
    }
    if (a->use_graph && !a->fwd_graph && !h->inject) {  // capturing
        a->fwd_variant = h->variant;
        a->fwd_spin = h->spin_limit;
        const int cur = h->cur;
        const int64_t steps = h->steps, l0 = h->launches;
        const bool pending = h->pending_sample;
        cudaGraph_t g = nullptr;
        r = run();
        cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
        // the capture recorded the launches; the bookkeeping it advanced is the
        // state every replay ends in
        a->fwd_cur = h->cur;
        a->fwd_steps = h->steps;
        a->fwd_pending = h->pending_sample;
        a->fwd_launches = h->launches - l0;
        h->cur = cur;
        h->steps = steps;
        h->launches = l0;
        h->pending_sample = pending;
        if (r != KLB_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (ec != cudaSuccess || cudaGraphInstantiate(&a->fwd_graph, g, 0) != cudaSuccess) {
            a->fwd_graph = nullptr;
            a->use_graph = false;
            cudaGetLastError();
        }
        if (g) cudaGraphDestroy(g);
    }
    if (a->fwd_graph) {
        ACK(a, cudaGraphLaunch(a->fwd_graph, h->stream));
        h->cur = a->fwd_cur;
        h->steps = a->fwd_steps;
        h->pending_sample = a->fwd_pending;
        h->launches += a->fwd_launches;
    } else {
        r = run();
        if (r != KLB_OK) return r;
    }
    const int64_t M = a->nsteps / h->p.sample_every + 1;
    std::vector<double> d((size_t)M * 7);
    int64_t cnt = 0;
    r = klb_diagnostics(h, d.data(), M, &cnt);
    if (r != KLB_OK) return afail(a, r, h->err);
    if (cnt != M) return afail(a, KLB_E_STATE, "unexpected number of samples");
    a->K.resize(M);
    for (int64_t s = 0; s < M; ++s) a->K[s] = d[7 * s + 6];
    a->ke = a->K[M - 1] * h->p.dx * h->p.dy;
    // gamma: 1/2 OLS slope of ln K over the last 75% of the samples
    const int start = (int)(M - (3 * M) / 4);
    const double dts = h->p.dt * h->p.sample_every;
    double tb = 0, yb = 0;
    for (int k = start; k < M; ++k) {
        tb += k * dts;
        yb += std::log(a->K[k]);
    }
    tb /= (M - start);
    yb /= (M - start);
    double sxy = 0, sxx = 0;
    for (int k = start; k < M; ++k) {
        sxy += (k * dts - tb) * (std::log(a->K[k]) - yb);
        sxx += (k * dts - tb) * (k * dts - tb);
    }
    a->gamma = sxx > 0 ? 0.5 * sxy / sxx : 0.0;
    if (ke) *ke = a->ke;
    if (gamma) *gamma = a->gamma;
    a->forward_done = true;
    return KLB_OK;
}

int klb_adjoint_backward(klb_adj_t* a, double g_ke, double g_gamma, double* d_rho, double* d_ux, double* d_uy,
                         double* d_T, int on_device) {
    fdlb::NvtxRange trace_("klb_adjoint_backward");
    if (!a || !d_rho || !d_ux || !d_uy || !d_T) return a ? afail(a, KLB_E_INVAL, "NULL argument") : KLB_E_INVAL;
    if (!a->forward_done) return afail(a, KLB_E_STATE, "klb_adjoint_backward before klb_adjoint_forward");
    klb_t* h = a->h;
    const bool f64 = h->p.precision == KLB_FP64;
    // lambda^N = dL/dK_{M-1} dK/df^N, from the final state
    const int M = (int)a->K.size();
    int lc = 0;
    const double cN = dL_dK(a, M - 1, g_ke, g_gamma);
    int r = f64 ? source<double>(a, h->buf[h->cur], cN, a->lam[lc]) : source<float>(a, h->buf[h->cur], cN, a->lam[lc]);
    if (r != KLB_OK) return r;
    r = reverse(a, true, g_ke, g_gamma, &lc);
    if (r != KLB_OK) return r;
    // restore the forward grid's final state (the recomputation reused its buffers)
    const int cur_final = h->cur;
    (void)cur_final;
    r = f64 ? fields_grad<double>(a, a->lam[lc], a->dense) : fields_grad<float>(a, a->lam[lc], a->dense);
    if (r != KLB_OK) return r;
    const size_t nn = (size_t)h->g.nx * h->g.ny;
    double* dst[4] = {d_rho, d_ux, d_uy, d_T};
    for (int k = 0; k < 4; ++k)
        ACK(a, cudaMemcpyAsync(dst[k], a->dense + k * nn, nn * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    ACK(a, cudaStreamSynchronize(h->stream));
    a->forward_done = false;  // the forward grid's buffers were reused: run the forward again first
    return klb_sync(h) == KLB_OK ? KLB_OK : afail(a, KLB_E_CUDA, h->err);
}

int klb_adjoint_vjp(klb_adj_t* a, const double* lam_N, double* lam_0, int on_device) {
    fdlb::NvtxRange trace_("klb_adjoint_vjp");
    if (!a || !lam_N || !lam_0) return a ? afail(a, KLB_E_INVAL, "NULL argument") : KLB_E_INVAL;
    if (!a->forward_done) return afail(a, KLB_E_STATE, "klb_adjoint_vjp before klb_adjoint_forward");
    klb_t* h = a->h;
    const size_t nn = (size_t)h->g.nx * h->g.ny;
    // lambda^N into the interior of the padded layout, ghost cells zero
    ACK(a, cudaMemcpyAsync(a->dense, lam_N, sizeof(double) * NQ * nn,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    ACK(a, cudaMemsetAsync(a->lam[0], 0, state_bytes(h), h->stream));
    if (h->p.precision == KLB_FP64)
        adj_import_kernel<double><<<grid_of((long long)(NQ * nn)), 256, 0, h->stream>>>(h->g, a->dense,
                                                                                         (double*)a->lam[0]);
    else
        adj_import_kernel<float><<<grid_of((long long)(NQ * nn)), 256, 0, h->stream>>>(h->g, a->dense,
                                                                                       (float*)a->lam[0]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return afail(a, KLB_E_CUDA, cudaGetErrorString(e));
    h->launches += 1;
    int lc = 0;
    int r = reverse(a, false, 0.0, 0.0, &lc);
    if (r != KLB_OK) return r;
    e = h->p.precision == KLB_FP64 ? launch_get_f<double>(h->g, (const double*)a->lam[lc], a->dense, h->stream)
                                   : launch_get_f<float>(h->g, (const float*)a->lam[lc], a->dense, h->stream);
    if (e != cudaSuccess) return afail(a, KLB_E_CUDA, cudaGetErrorString(e));
    ACK(a, cudaMemcpyAsync(lam_0, a->dense, sizeof(double) * NQ * nn,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    a->forward_done = false;
    return klb_sync(h) == KLB_OK ? KLB_OK : afail(a, KLB_E_CUDA, h->err);  // also a bounded wait that ran out
}

int klb_adjoint_samples(klb_adj_t* a, double* out, int64_t cap, int64_t* count) {
    if (!a || !count || (cap > 0 && !out)) return KLB_E_INVAL;
    const int64_t m = std::min<int64_t>(cap, (int64_t)a->K.size());
    for (int64_t s = 0; s < m; ++s) out[s] = a->K[s];
    *count = m;
    return KLB_OK;
}

const char* klb_adjoint_last_error(const klb_adj_t* a) { return a ? a->err.c_str() : g_adj_create_error.c_str(); }

}  // extern "C"
