// klb_batch.cu -- batched engine: many FP32 grids of uneven size stepped by
// one launch of the persistent step kernel per time step, the step loop
// replayed from a CUDA graph, and an autotuner over the kernel's tile shapes.
//
// Used for the paper's parameter sweeps (Sec. IV: Kelvin-Helmholtz runs over
// the widths D_v and D_rho of the velocity and density transition layers):
// every instance is a full grid with its own fields, boundaries and
// diagnostics series; the instances share the step constants (dx, dy, dt,
// tau, ring speeds, epsilon).
#include <limits.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "klb_handle.h"

using namespace fdlb;

struct klb_batch {
    std::vector<klb_t*> m;         // member grids (owned)
    cudaStream_t stream = nullptr; // shared by all members
    bool own_stream = false;
    InstDesc* descs_dev = nullptr; // [2][n]: all members with their state in buf[p]
    int ntiles = 0;                // tiles of one launch
    int variant = 0;
    int* err_dev = nullptr;        // error word of the batched step kernel
    DiagJob* jobs_dev = nullptr;   // [2][n]: every member's sample of the state in buf[p]
    int diag_ctas = 0;             // CTAs of one batched sample (all members)
    bool use_graph = true;
    int period = 0;                // steps per sampling period (graph unit)
    int graph_steps = 0;           // steps captured in one graph
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // by starting parity
    int64_t graph_launches = 0;    // kernel launches inside one graph
    int64_t launches = 0;
    std::string err;
};

static thread_local std::string g_batch_create_error;

static int bfail(klb_batch_t* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    else g_batch_create_error = msg;
    return code;
}
#define BCK(b, call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return bfail(b, KLB_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static void drop_graphs(klb_batch_t* b) {
    for (int p = 0; p < 2; ++p)
        if (b->graph[p]) {
            cudaGraphExecDestroy(b->graph[p]);
            b->graph[p] = nullptr;
        }
}

// descriptors of every member for both parities; the members' tiles are laid
// end to end in the launch's tile index space
static int upload(klb_batch_t* b) {
    const int n = (int)b->m.size();
    std::vector<InstDesc> d(2 * (size_t)n);
    int first = 0;
    for (int i = 0; i < n; ++i) {
        klb_t* h = b->m[i];
        int tiles_x, nt;
        f32_tiles(h->g.nx, h->g.ny, b->variant, &tiles_x, &nt);
        // per member below 2^24 tiles (the float quotient estimate of the tile
        // map is exact there), and the batch's tile index space within int
        if (nt >= (1 << 24) || first > INT_MAX - nt) return bfail(b, KLB_E_INVAL, "batch too large for the FP32 tile index");
        for (int p = 0; p < 2; ++p) {
            InstDesc& e = d[(size_t)p * n + i];
            memset(&e, 0, sizeof(InstDesc));
            e.map = h->map[p];
            e.out = (float*)h->buf[1 - p];
            e.g = h->g;
            e.tiles_x = tiles_x;
            e.first_tile = first;
        }
        first += nt;
    }
    BCK(b, cudaMemcpy(b->descs_dev, d.data(), d.size() * sizeof(InstDesc), cudaMemcpyHostToDevice));
    b->ntiles = first;
    // the members' stand-alone diagnostics, their CTAs laid end to end
    std::vector<DiagJob> jb(2 * (size_t)n);
    int cta = 0;
    for (int i = 0; i < n; ++i) {
        klb_t* h = b->m[i];
        int tiles_x, nt;
        f32_tiles(h->g.nx, h->g.ny, b->variant, &tiles_x, &nt);
        const int grid = f32_grid(h->g.nx, h->g.ny, b->variant);
        for (int p = 0; p < 2; ++p) {
            DiagJob& j = jb[(size_t)p * n + i];
            j.f = (const float*)h->buf[p];
            j.g = h->g;
            j.tiles_x = tiles_x;
            j.ntiles = nt;
            j.grid = grid;
            j.first_cta = cta;
            j.partials = h->diag_partials;
            j.ring = h->diag_ring;
            j.cap = h->cap;
            j.counter = h->nsamp_dev;
            j.err = h->err_dev;
        }
        cta += grid;
    }
    BCK(b, cudaMemcpy(b->jobs_dev, jb.data(), jb.size() * sizeof(DiagJob), cudaMemcpyHostToDevice));
    b->diag_ctas = cta;
    drop_graphs(b);
    return KLB_OK;
}

static int same_state(klb_batch_t* b) {
    for (klb_t* h : b->m) {
        if (!h->initialized) return bfail(b, KLB_E_STATE, "a member has no initial state (klb_init_fields)");
        if (h->broken) return bfail(b, KLB_E_STATE, "a member's tile shape could not be restored (klb_set_variant)");
        if (h->cur != b->m[0]->cur || h->steps != b->m[0]->steps)
            return bfail(b, KLB_E_STATE, "members are not at the same step (re-initialise them together)");
    }
    return KLB_OK;
}

// the samples due on the members' current state: the records of every due
// member in one launch, their folds in a second (each member's records and
// fold are those of its own stand-alone diagnostics, hence the same bits)
static int batch_sample(klb_batch_t* b) {
    DueMask due;
    memset(&due, 0, sizeof(due));
    bool any = false;
    for (size_t i = 0; i < b->m.size(); ++i)
        if (b->m[i]->pending_sample) {
            due.w[i >> 5] |= 1u << (i & 31);
            any = true;
        }
    if (!any) return KLB_OK;
    const int p = b->m[0]->cur;
    const int n = (int)b->m.size();
    const DiagJob* jobs = b->jobs_dev + (size_t)p * n;
    cudaError_t e = launch_diag_f32_batch(b->m[0]->cf, jobs, n, b->diag_ctas, b->variant, due, b->stream);
    if (e == cudaSuccess) e = launch_diag_finalize_batch(jobs, n, due, b->stream);
    if (e != cudaSuccess) return bfail(b, KLB_E_CUDA, std::string("batched diagnostics: ") + cudaGetErrorString(e));
    b->launches += 2;
    for (klb_t* h : b->m) h->pending_sample = false;
    return KLB_OK;
}

// one batched step: the samples that are due before it (the initial state),
// the step of every member in one launch, then the samples due after it
static int batch_step_once(klb_batch_t* b) {
    int r = batch_sample(b);
    if (r != KLB_OK) return r;
    const int p = b->m[0]->cur;
    const int n = (int)b->m.size();
    klb_t* h0 = b->m[0];
    cudaError_t e = launch_step_f32(h0->cf, b->descs_dev + (size_t)p * n, n, b->ntiles, nullptr, b->err_dev,
                                    h0->spin_limit, h0->inject, b->variant, b->stream);
    if (e != cudaSuccess) return bfail(b, KLB_E_CUDA, std::string("batched step kernel: ") + cudaGetErrorString(e));
    b->launches += 1;
    for (klb_t* h : b->m) handle_after_step(h);
    return batch_sample(b);
}

// capture graph_steps batched steps starting from parity p and a step count
// that is a multiple of the sampling period
static int build_graph(klb_batch_t* b, int p) {
    std::vector<int> cur(b->m.size());
    std::vector<int64_t> steps(b->m.size()), launches(b->m.size());
    std::vector<bool> pending(b->m.size());
    for (size_t i = 0; i < b->m.size(); ++i) {
        cur[i] = b->m[i]->cur;
        steps[i] = b->m[i]->steps;
        launches[i] = b->m[i]->launches;
        pending[i] = b->m[i]->pending_sample;
        b->m[i]->pending_sample = false;
    }
    const int64_t l0 = b->launches;
    cudaGraph_t g = nullptr;
    BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int r = KLB_OK;
    for (int s = 0; s < b->graph_steps && r == KLB_OK; ++s) r = batch_step_once(b);
    cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
    // the capture only recorded the launches: restore the members' bookkeeping
    for (size_t i = 0; i < b->m.size(); ++i) {
        b->m[i]->cur = cur[i];
        b->m[i]->steps = steps[i];
        b->m[i]->launches = launches[i];
        b->m[i]->pending_sample = pending[i];
    }
    b->graph_launches = b->launches - l0;
    b->launches = l0;
    if (r != KLB_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (ec != cudaSuccess) return bfail(b, KLB_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    cudaError_t ei = cudaGraphInstantiate(&b->graph[p], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        b->graph[p] = nullptr;
        return bfail(b, KLB_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    }
    return KLB_OK;
}

static int64_t gcd64(int64_t a, int64_t b) { return b == 0 ? a : gcd64(b, a % b); }

extern "C" {

int klb_batch_create(const klb_params* ps, int n, klb_batch_t** out) {
    if (!ps || !out || n < 1) return bfail(nullptr, KLB_E_INVAL, "NULL argument or n < 1");
    if (n > kMaxInstances) return bfail(nullptr, KLB_E_INVAL, "too many instances in one batch");
    *out = nullptr;
    const klb_params& p0 = ps[0];
    for (int i = 0; i < n; ++i) {
        const klb_params& p = ps[i];
        if (p.precision != KLB_FP32) return bfail(nullptr, KLB_E_INVAL, "batches step FP32 grids");
        if (p.dx != p0.dx || p.dy != p0.dy || p.dt != p0.dt || p.tau != p0.tau || p.v[0] != p0.v[0] ||
            p.v[1] != p0.v[1] || p.v[2] != p0.v[2] || p.eps != p0.eps || p.scheme != p0.scheme)
            return bfail(nullptr, KLB_E_INVAL, "instances of a batch must share dx, dy, dt, tau, v, eps and scheme");
    }
    klb_batch_t* b = new klb_batch();
    auto cleanup = [&](int code, const std::string& msg) {
        klb_batch_destroy(b);
        return bfail(nullptr, code, msg);
    };
    if (p0.stream) {
        b->stream = (cudaStream_t)p0.stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return bfail(nullptr, KLB_E_CUDA, "cudaStreamCreate failed");
    } else {
        b->own_stream = true;
    }
    if (prepare_f32_kernels() != cudaSuccess) {  // kernel attributes set outside any graph capture
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return bfail(nullptr, KLB_E_CUDA, "cannot configure the step kernels");
    }
    int64_t period = 2;
    for (int i = 0; i < n; ++i) {
        klb_params p = ps[i];
        p.stream = b->stream;
        klb_t* h = nullptr;
        int r = klb_create(&p, &h);
        if (r != KLB_OK) return cleanup(r, std::string("member ") + std::to_string(i) + ": " + klb_last_error(nullptr));
        b->m.push_back(h);
        // one launch steps all members: their tensor maps must have the batch's tile shape
        if (h->variant != b->variant && klb_set_variant(h, b->variant) != KLB_OK)
            return cleanup(KLB_E_CUDA, std::string("member ") + std::to_string(i) + ": " + h->err);
        if (p.sample_every > 0) period = period / gcd64(period, p.sample_every) * p.sample_every;
    }
    b->period = (int)std::min<int64_t>(period, 1 << 20);
    b->graph_steps = b->period * (int)std::max<int64_t>(1, (64 + b->period - 1) / b->period);
    if (b->period > 512) b->use_graph = false;  // sampling periods that do not fit one graph
    if (cudaMalloc(&b->descs_dev, 2 * sizeof(InstDesc) * n) != cudaSuccess ||
        cudaMalloc(&b->jobs_dev, 2 * sizeof(DiagJob) * n) != cudaSuccess ||
        cudaMalloc(&b->err_dev, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(KLB_E_NOMEM, "cudaMalloc of the batch descriptors failed");
    }
    if (cudaMemset(b->err_dev, 0, sizeof(int)) != cudaSuccess) return cleanup(KLB_E_CUDA, "cudaMemset failed");
    if (upload(b) != KLB_OK) return cleanup(KLB_E_CUDA, b->err);
    *out = b;
    return KLB_OK;
}

void klb_batch_destroy(klb_batch_t* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (klb_t* h : b->m) {
        h->own_stream = false;  // the batch owns the stream
        klb_destroy(h);
    }
    if (b->descs_dev) cudaFree(b->descs_dev);
    if (b->err_dev) cudaFree(b->err_dev);
    if (b->jobs_dev) cudaFree(b->jobs_dev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int klb_batch_size(const klb_batch_t* b) { return b ? (int)b->m.size() : -1; }

klb_t* klb_batch_member(klb_batch_t* b, int i) {
    if (!b || i < 0 || i >= (int)b->m.size()) return nullptr;
    return b->m[i];
}

int klb_batch_step(klb_batch_t* b, int64_t n) {
    fdlb::NvtxRange trace_("klb_batch_step");
    if (!b) return KLB_E_INVAL;
    if (n < 0) return bfail(b, KLB_E_INVAL, "negative step count");
    int r = same_state(b);
    if (r != KLB_OK) return r;
    while (n > 0) {
        klb_t* h0 = b->m[0];
        const bool aligned = h0->steps % b->period == 0;
        if (b->use_graph && aligned && n >= b->graph_steps) {
            // samples due before the period (the initial state) are taken eagerly
            r = batch_sample(b);
            if (r != KLB_OK) return r;
            const int p = h0->cur;
            if (!b->graph[p]) {
                r = build_graph(b, p);
                if (r != KLB_OK) return r;
            }
            BCK(b, cudaGraphLaunch(b->graph[p], b->stream));
            b->launches += b->graph_launches;
            for (klb_t* h : b->m) {  // graph_steps is even: the parity is back where it started
                h->steps += b->graph_steps;
                h->pending_sample = false;  // the period's last sample was taken inside the graph
            }
            n -= b->graph_steps;
        } else {
            r = batch_step_once(b);
            if (r != KLB_OK) return r;
            n -= 1;
        }
    }
    return KLB_OK;
}

int klb_batch_sync(klb_batch_t* b) {
    if (!b) return KLB_E_INVAL;
    BCK(b, cudaStreamSynchronize(b->stream));
    int v = 0;
    BCK(b, cudaMemcpy(&v, b->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) {
        BCK(b, cudaMemset(b->err_dev, 0, sizeof(int)));
        if (v & ERR_TIMEOUT) return bfail(b, KLB_E_DEVICE_TIMEOUT, "a bounded device-side wait ran out");
    }
    for (klb_t* h : b->m) {
        int r = klb_sync(h);
        if (r != KLB_OK) return bfail(b, r, h->err);
    }
    return KLB_OK;
}

int klb_batch_set_variant(klb_batch_t* b, int variant) {
    if (!b) return KLB_E_INVAL;
    if (variant < 0 || variant > 1) return bfail(b, KLB_E_INVAL, "unknown kernel variant");
    BCK(b, cudaStreamSynchronize(b->stream));
    for (klb_t* h : b->m) {
        int r = klb_set_variant(h, variant);
        if (r != KLB_OK) return bfail(b, r, h->err);
    }
    b->variant = variant;
    return upload(b);
}

int klb_batch_get_variant(const klb_batch_t* b) { return b ? b->variant : -1; }

int klb_batch_use_graph(klb_batch_t* b, int on) {
    if (!b) return KLB_E_INVAL;
    b->use_graph = on != 0 && b->period <= 512;
    return KLB_OK;
}

int klb_batch_autotune(klb_batch_t* b, int steps, int* variant) {
    fdlb::NvtxRange trace_("klb_batch_autotune");
    if (!b || steps < 1) return b ? bfail(b, KLB_E_INVAL, "steps must be >= 1") : KLB_E_INVAL;
    int r = same_state(b);
    if (r != KLB_OK) return r;
    BCK(b, cudaStreamSynchronize(b->stream));
    // snapshot of every member's current buffer: the trials must leave no trace
    std::vector<void*> snap(b->m.size(), nullptr);
    auto release = [&]() {
        for (void* s : snap)
            if (s) cudaFree(s);
    };
    for (size_t i = 0; i < b->m.size(); ++i) {
        klb_t* h = b->m[i];
        const size_t bytes = (size_t)NQ * h->g.plane * h->esize;
        if (cudaMalloc(&snap[i], bytes) != cudaSuccess) {
            cudaGetLastError();
            release();
            return bfail(b, KLB_E_NOMEM, "no room for the autotuning snapshot");
        }
        BCK(b, cudaMemcpyAsync(snap[i], h->buf[h->cur], bytes, cudaMemcpyDeviceToDevice, b->stream));
    }
    const int p0 = b->m[0]->cur;
    const int n = (int)b->m.size();
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    float best_ms = -1.f;
    int best = 0;
    for (int v = 0; v <= 1; ++v) {
        r = klb_batch_set_variant(b, v);
        if (r != KLB_OK) break;
        klb_t* h0 = b->m[0];
        int p = p0;
        for (int s = 0; s < steps + 2; ++s) {  // two untimed launches, then `steps` timed ones
            if (s == 2) cudaEventRecord(e0, b->stream);
            cudaError_t e = launch_step_f32(h0->cf, b->descs_dev + (size_t)p * n, n, b->ntiles, nullptr, b->err_dev,
                                            h0->spin_limit, 0, v, b->stream);
            if (e != cudaSuccess) {
                r = bfail(b, KLB_E_CUDA, std::string("autotune launch: ") + cudaGetErrorString(e));
                break;
            }
            p = 1 - p;
        }
        float ms = 0.f;
        cudaError_t et = cudaEventRecord(e1, b->stream);
        if (et == cudaSuccess) et = cudaEventSynchronize(e1);
        if (et == cudaSuccess) et = cudaEventElapsedTime(&ms, e0, e1);
        if (et != cudaSuccess && r == KLB_OK)
            r = bfail(b, KLB_E_CUDA, std::string("autotune timing: ") + cudaGetErrorString(et));
        if (r == KLB_OK && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best = v;
        }
        // restore the state for the next trial (and for the run after the last one)
        for (size_t i = 0; i < b->m.size(); ++i) {
            klb_t* h = b->m[i];
            cudaError_t ec = cudaMemcpyAsync(h->buf[p0], snap[i], (size_t)NQ * h->g.plane * h->esize,
                                             cudaMemcpyDeviceToDevice, b->stream);
            if (ec != cudaSuccess && r == KLB_OK)
                r = bfail(b, KLB_E_CUDA, std::string("autotune restore: ") + cudaGetErrorString(ec));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t es = cudaStreamSynchronize(b->stream);
    release();
    if (es != cudaSuccess && r == KLB_OK) r = bfail(b, KLB_E_CUDA, std::string("autotune: ") + cudaGetErrorString(es));
    if (r != KLB_OK) return r;
    r = klb_batch_set_variant(b, best);
    if (r == KLB_OK && variant) *variant = best;
    return r;
}

int64_t klb_batch_launch_count(const klb_batch_t* b) { return b ? b->launches : -1; }

int64_t klb_batch_tiles(const klb_batch_t* b) { return b ? b->ntiles : -1; }

const char* klb_batch_last_error(const klb_batch_t* b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

}  // extern "C"
