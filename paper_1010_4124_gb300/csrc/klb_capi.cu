// klb_capi.cu -- implementation of the C ABI declared in include/klb.h.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "klb_handle.h"

using namespace fdlb;


static thread_local std::string g_create_error;

static int fail(klb_t* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}
int fdlb::handle_fail(klb_t* h, int code, const std::string& msg) { return fail(h, code, msg); }

int fdlb::bounds_flags() {
#ifdef KLB_CHECK_BOUNDS
    return bounds_flag_aux_f32() | bounds_flag_aux_f64() | bounds_flag_step_f32() | bounds_flag_step_f32_lo() |
           bounds_flag_step_f64() | bounds_flag_adjoint() | bounds_flag_slabs();
#else
    return 0;
#endif
}

static int cuda_fail(klb_t* h, cudaError_t e, const char* where) {
    return fail(h, KLB_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(h, call)                                            \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// constants of the step from the problem statement
// ---------------------------------------------------------------------------
template <typename T>
static void fill_const(const klb_params& p, StepConst<T>& c) {
    c.scheme = p.scheme;
    const double h = 0.5 * std::sqrt(3.0);
    const double cs[6] = {0.5, -0.5, -1.0, -0.5, 0.5, 1.0};  // cos(60 i deg), i = 1..6
    const double sn[6] = {h, h, 0.0, -h, -h, 0.0};            // sin(60 i deg)
    const double eps = p.eps > 0 ? p.eps : 1e-6;
    for (int q = 0; q < NQ; ++q) {
        double vx = 0, vy = 0;
        if (q > 0) {
            const int k = (q - 1) / 6, i = (q - 1) % 6;
            vx = p.v[k] * cs[i];
            vy = p.v[k] * sn[i];
        }
        c.vx[q] = T(vx);
        c.vy[q] = T(vy);
        c.v2[q] = T(vx * vx + vy * vy);
        c.cx[q] = T(p.dt * vx / p.dx);
        c.cy[q] = T(p.dt * vy / p.dy);
        // FP32 weno() works with sigma scaled by 3/4, hence eps too; the FP64 path uses eps itself
        c.ex[q] = vx != 0 ? T(0.75 * eps / (vx * vx)) : T(0);
        c.ey[q] = vy != 0 ? T(0.75 * eps / (vy * vy)) : T(0);
    }
    for (int q = 0; q < NQ; ++q) {
        c.epair[q][0] = c.ex[q];
        c.epair[q][1] = c.ey[q];
    }
    for (int m = 0; m < 3; ++m) {
        c.epair[19 + m][0] = c.ex[6 * m + 3];
        c.epair[19 + m][1] = c.ex[6 * m + 6];
    }
    {
        int ys[12], n = 0;  // the velocities with v_y != 0 in slot order
        for (int q = 1; q < NQ; ++q)
            if ((q - 1) % 3 != 2) ys[n++] = q;
        for (int k = 0; k < 6; ++k) {
            c.epair[22 + k][0] = c.ey[ys[2 * k]];
            c.epair[22 + k][1] = c.ey[ys[2 * k + 1]];
        }
    }
    // F_k(T) = T [a_{k+1} a_{k+2} - 4 (a_{k+1} + a_{k+2}) T + 24 T^2] / [3 a_k (a_k - a_{k+1})(a_k - a_{k+2})]
    for (int k = 0; k < 3; ++k) {
        const double ak = p.v[k] * p.v[k];
        const double a1 = p.v[(k + 1) % 3] * p.v[(k + 1) % 3];
        const double a2 = p.v[(k + 2) % 3] * p.v[(k + 2) % 3];
        const double den = 3.0 * ak * (ak - a1) * (ak - a2);
        c.fk[k][0] = T(a1 * a2 / den);
        c.fk[k][1] = T(-4.0 * (a1 + a2) / den);
        c.fk[k][2] = T(24.0 / den);
        c.a4[k] = T(4.0 * (a1 + a2));
        c.pk[k] = T(a1 * a2);
        c.den[k] = T(den);
    }
    // inverse of the Gram matrix G_ab = sum_q B_aq B_bq, B = (1, v_x, v_y, |v|^2)
    double B[4][NQ], G[4][8];
    for (int q = 0; q < NQ; ++q) {
        const double vx = double(c.vx[q]), vy = double(c.vy[q]);
        B[0][q] = 1.0;
        B[1][q] = vx;
        B[2][q] = vy;
        B[3][q] = vx * vx + vy * vy;
    }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 8; ++b) {
            G[a][b] = 0.0;
            if (b < 4)
                for (int q = 0; q < NQ; ++q) G[a][b] += B[a][q] * B[b][q];
            else
                G[a][b] = (b - 4 == a) ? 1.0 : 0.0;
        }
    for (int col = 0; col < 4; ++col) {  // Gauss-Jordan with partial pivoting
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (std::fabs(G[r][col]) > std::fabs(G[piv][col])) piv = r;
        for (int b = 0; b < 8; ++b) std::swap(G[col][b], G[piv][b]);
        const double d = G[col][col];
        for (int b = 0; b < 8; ++b) G[col][b] /= d;
        for (int r = 0; r < 4; ++r)
            if (r != col) {
                const double m = G[r][col];
                for (int b = 0; b < 8; ++b) G[r][b] -= m * G[col][b];
            }
    }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) c.ginv[a][b] = T(G[a][b + 4]);
    c.dt = T(p.dt);
    c.dx = T(p.dx);
    c.dy = T(p.dy);
    c.eps = T(eps);
    c.relax = T(p.dt / p.tau);
}
void fdlb::step_constants(const klb_params& p, StepConst<float>& c) { fill_const(p, c); }
void fdlb::step_constants(const klb_params& p, StepConst<double>& c) { fill_const(p, c); }

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

// 3-D map over (x: pitch, y: ny + 6 rows, z: 19 planes) of a state buffer of
// the handle's layout, with the given box (x extent a 16-byte multiple).
int fdlb::encode_state_map(klb_t* h, const void* base, unsigned bx, unsigned by, unsigned bz, CUtensorMap* map) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(h, KLB_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const Geom& g = h->g;
    cuuint64_t dims[3] = {(cuuint64_t)g.px, (cuuint64_t)(g.ny + 2 * GY), (cuuint64_t)NQ};
    cuuint64_t strides[2] = {(cuuint64_t)g.px * h->esize, (cuuint64_t)g.plane * h->esize};
    cuuint32_t box[3] = {bx, by, bz};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, h->p.precision == KLB_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, KLB_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return KLB_OK;
}

// the map of a state buffer with the step kernel's box
static int make_map(klb_t* h, void* base, CUtensorMap* map) {
    if (h->p.precision == KLB_FP64) {  // one tile of TX x TY nodes plus halo
        int TX, TY;
        f64_tile(&TX, &TY);
        return fdlb::encode_state_map(h, base, (unsigned)(TX + 8), (unsigned)(TY + 6), (unsigned)NQ, map);
    }
    unsigned bx, by, bz;  // one tile of the persistent FP32 kernel
    f32_box(h->variant, &bx, &by, &bz);
    return fdlb::encode_state_map(h, base, bx, by, bz, map);
}

extern "C" {

void klb_params_default(klb_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->v[0] = 1.0;
    p->v[1] = 2.0;
    p->v[2] = 3.0;
    p->bc_x_lo = p->bc_x_hi = p->bc_y_lo = p->bc_y_hi = KLB_BC_PERIODIC;
    p->precision = KLB_FP32;
    p->eps = 1e-6;
    p->scheme = KLB_WENO5;
}

int klb_create(const klb_params* pin, klb_t** out) {
    if (!pin || !out) return fail(nullptr, KLB_E_INVAL, "NULL argument");
    *out = nullptr;
    const klb_params& p = *pin;
    if (p.nx < 1 || p.ny < 1) return fail(nullptr, KLB_E_INVAL, "nx and ny must be >= 1");
    if ((long long)p.nx + 16 > (1ll << 31) / 2) return fail(nullptr, KLB_E_INVAL, "nx too large");
    if (!(p.dx > 0) || !(p.dy > 0) || !(p.dt > 0) || !(p.tau > 0))
        return fail(nullptr, KLB_E_INVAL, "dx, dy, dt and tau must be > 0");
    for (int k = 0; k < 3; ++k)
        if (!(p.v[k] > 0)) return fail(nullptr, KLB_E_INVAL, "ring speeds must be > 0");
    if (p.v[0] == p.v[1] || p.v[1] == p.v[2] || p.v[0] == p.v[2])
        return fail(nullptr, KLB_E_INVAL, "ring speeds must be distinct");
    const int bcs[4] = {p.bc_x_lo, p.bc_x_hi, p.bc_y_lo, p.bc_y_hi};
    for (int b : bcs)
        if (b < 0 || b > 3) return fail(nullptr, KLB_E_INVAL, "unknown boundary kind");
    if (p.bc_x_lo == KLB_BC_HALO || p.bc_x_hi == KLB_BC_HALO)
        return fail(nullptr, KLB_E_INVAL, "halo sides are y sides (slabs cut the grid in y)");
    if ((p.bc_x_lo == KLB_BC_PERIODIC) != (p.bc_x_hi == KLB_BC_PERIODIC) ||
        (p.bc_y_lo == KLB_BC_PERIODIC) != (p.bc_y_hi == KLB_BC_PERIODIC))
        return fail(nullptr, KLB_E_INVAL, "a periodic side must pair with a periodic side");
    if (p.precision != KLB_FP32 && p.precision != KLB_FP64) return fail(nullptr, KLB_E_INVAL, "unknown precision");
    if (p.sample_every < 0 || p.diag_capacity < 0) return fail(nullptr, KLB_E_INVAL, "negative diagnostics setting");
    if (p.eps < 0) return fail(nullptr, KLB_E_INVAL, "eps must be >= 0");
    if (p.scheme < KLB_WENO5 || p.scheme > KLB_TVD2) return fail(nullptr, KLB_E_INVAL, "unknown convection scheme");

    const double vmax = std::max(p.v[0], std::max(p.v[1], p.v[2]));
    // FP32 WENO5 squares the reciprocals of its smoothness indicators, each at
    // least 3/4 eps / v_a^2 for the velocity component v_a of its plane (the
    // largest |v_a| is vmax): those squares and the weights' sum must stay
    // normal FP32 numbers
    if (p.precision == KLB_FP32 && p.scheme == KLB_WENO5 && p.eps > 0 && 0.75 * p.eps / (vmax * vmax) < 2e-19)
        return fail(nullptr, KLB_E_INVAL, "eps too small for the FP32 WENO5 weights (3/4 eps / max(v)^2 < 2e-19)");
    const double cfl = vmax * p.dt / std::min(p.dx, p.dy);
    if (p.dt / p.tau > 2.0)
        fprintf(stderr, "klb: warning: dt/tau = %g > 2 (the BGK factor 1 - dt/tau exceeds -1)\n", p.dt / p.tau);
    if (cfl > 0.03 * (1 + 1e-9))
        fprintf(stderr, "klb: warning: CFL max(v) dt/min(dx,dy) = %g > 0.03; forward Euler + WENO5 may grow\n", cfl);

    klb_t* h = new klb();
    h->p = p;
    if (h->p.eps == 0) h->p.eps = 1e-6;
    h->esize = p.precision == KLB_FP64 ? 8 : 4;
    Geom& g = h->g;
    g.nx = p.nx;
    g.ny = p.ny;
    g.px = ((p.nx + GX + 3) + 31) / 32 * 32;
    g.plane = (long long)g.px * (p.ny + 2 * GY);
    g.bcx_lo = p.bc_x_lo;
    g.bcx_hi = p.bc_x_hi;
    g.bcy_lo = p.bc_y_lo;
    g.bcy_hi = p.bc_y_hi;
    fill_const(h->p, h->cf);
    fill_const(h->p, h->cd);
    if (p.precision == KLB_FP64) {
        int TX, TY;
        f64_tile(&TX, &TY);
        h->nparts = ((p.nx + TX - 1) / TX) * ((p.ny + TY - 1) / TY);
    } else {
        // room for the partial records of either tile shape
        h->nparts = std::max(f32_grid(p.nx, p.ny, 0), f32_grid(p.nx, p.ny, 1));
    }
    h->cap = p.diag_capacity > 0 ? p.diag_capacity : 4096;
    h->variant = p.precision == KLB_FP32 ? f32_default_variant(p.nx, p.ny) : 0;

    auto cleanup = [&](int code) {
        klb_destroy(h);
        return code;
    };
    const size_t fbytes = (size_t)NQ * g.plane * h->esize;
    for (int i = 0; i < 2; ++i) {
        if (cudaMalloc(&h->buf[i], fbytes) != cudaSuccess) {
            cudaGetLastError();
            fail(nullptr, KLB_E_NOMEM, "cudaMalloc of the distribution buffers failed");
            return cleanup(KLB_E_NOMEM);
        }
        if (cudaMemset(h->buf[i], 0, fbytes) != cudaSuccess) {
            fail(nullptr, KLB_E_CUDA, "cudaMemset failed");
            return cleanup(KLB_E_CUDA);
        }
    }
    if (cudaMalloc(&h->fields_dev, sizeof(double) * 4 * (size_t)p.nx * p.ny) != cudaSuccess ||
        cudaMalloc(&h->diag_ring, sizeof(double) * 7 * (size_t)h->cap) != cudaSuccess ||
        cudaMalloc(&h->diag_partials, sizeof(double) * 8 * (size_t)h->nparts) != cudaSuccess ||
        cudaMalloc(&h->err_dev, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->nsamp_dev, sizeof(long long)) != cudaSuccess ||
        (p.precision == KLB_FP32 && cudaMalloc(&h->descs_dev, 2 * sizeof(InstDesc)) != cudaSuccess)) {
        cudaGetLastError();
        fail(nullptr, KLB_E_NOMEM, "cudaMalloc of the staging buffers failed");
        return cleanup(KLB_E_NOMEM);
    }
    if (cudaMemset(h->err_dev, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(h->nsamp_dev, 0, sizeof(long long)) != cudaSuccess) {
        fail(nullptr, KLB_E_CUDA, "cudaMemset failed");
        return cleanup(KLB_E_CUDA);
    }
    if (p.stream) {
        h->stream = (cudaStream_t)p.stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            fail(nullptr, KLB_E_CUDA, "cudaStreamCreate failed");
            return cleanup(KLB_E_CUDA);
        }
        h->own_stream = true;
    }
    for (int i = 0; i < 2; ++i) {
        int r = make_map(h, h->buf[i], &h->map[i]);
        if (r != KLB_OK) {
            g_create_error = h->err;
            return cleanup(r);
        }
    }
    if (p.precision == KLB_FP32) {
        int r = fdlb::handle_upload_descs(h);
        if (r != KLB_OK) {
            g_create_error = h->err;
            return cleanup(r);
        }
        // graph replay of the step loop (FP32 WENO5): the kernel attributes are
        // set here, outside any capture; runs of at least 64 steps, a multiple
        // of the sampling period and even (the parity comes back)
        if (p.scheme == KLB_WENO5 && fdlb::prepare_f32_kernels() == cudaSuccess) {
            const int64_t unit = p.sample_every > 0 ? (p.sample_every % 2 == 0 ? p.sample_every : 2ll * p.sample_every)
                                                    : 2;
            if (unit <= 512) h->graph_steps = (int)(unit * ((64 + unit - 1) / unit));
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        fail(nullptr, KLB_E_CUDA, "device synchronisation after allocation failed");
        return cleanup(KLB_E_CUDA);
    }
    *out = h;
    return KLB_OK;
}

void klb_destroy(klb_t* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    fdlb::handle_drop_graphs(h);
    for (int i = 0; i < 2; ++i)
        if (h->buf[i]) cudaFree(h->buf[i]);
    if (h->fields_dev) cudaFree(h->fields_dev);
    if (h->fdense_dev) cudaFree(h->fdense_dev);
    if (h->diag_ring) cudaFree(h->diag_ring);
    if (h->diag_partials) cudaFree(h->diag_partials);
    if (h->err_dev) cudaFree(h->err_dev);
    if (h->nsamp_dev) cudaFree(h->nsamp_dev);
    if (h->descs_dev) cudaFree(h->descs_dev);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// The device's view of a host array: the array itself when it is pinned
// (page-locked and mapped, as cudaHostAlloc / cudaHostRegister make it; the
// kernels then read or write it across the host link directly, with no
// staging copy), else NULL.
static void* device_view(const void* host) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

static int stage_fields(klb_t* h, const double* rho, const double* ux, const double* uy, const double* T,
                        int on_device, const double** d) {
    const size_t n = (size_t)h->g.nx * h->g.ny;
    const double* src[4] = {rho, ux, uy, T};
    for (int i = 0; i < 4; ++i) {
        if (!src[i]) return fail(h, KLB_E_INVAL, "NULL field pointer");
        if (on_device) {
            d[i] = src[i];
        } else if (const void* v = device_view(src[i])) {
            d[i] = (const double*)v;
        } else {
            CK(h, cudaMemcpyAsync(h->fields_dev + i * n, src[i], n * sizeof(double), cudaMemcpyHostToDevice,
                                  h->stream));
            d[i] = h->fields_dev + i * n;
        }
    }
    return KLB_OK;
}

int klb_init_fields(klb_t* h, const double* rho, const double* ux, const double* uy, const double* T,
                    int on_device) {
    fdlb::NvtxRange trace_("klb_init_fields");
    if (!h) return KLB_E_INVAL;
    const double* d[4];
    int r = stage_fields(h, rho, ux, uy, T, on_device, d);
    if (r != KLB_OK) return r;
    cudaError_t e;
    // the state goes to buffer 0 only: the first step writes every node and
    // ghost image of buffer 1 (the fixed-equilibrium ghosts, which steps never
    // write, go to both)
    if (h->p.precision == KLB_FP64) {
        e = launch_init_feq<double>(h->cd, h->g, d[0], d[1], d[2], d[3], (double*)h->buf[0], nullptr, h->stream);
        if (e == cudaSuccess)
            e = launch_fixed_ghosts<double>(h->cd, h->g, d[0], d[1], d[2], d[3], (double*)h->buf[0],
                                            (double*)h->buf[1], h->stream);
    } else {
        e = launch_init_feq<float>(h->cf, h->g, d[0], d[1], d[2], d[3], (float*)h->buf[0], nullptr, h->stream);
        if (e == cudaSuccess)
            e = launch_fixed_ghosts<float>(h->cf, h->g, d[0], d[1], d[2], d[3], (float*)h->buf[0],
                                           (float*)h->buf[1], h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "init kernels");
    CK(h, cudaMemsetAsync(h->nsamp_dev, 0, sizeof(long long), h->stream));
    h->launches += 2;
    h->cur = 0;
    h->steps = 0;
    h->pending_sample = h->p.sample_every > 0;
    h->initialized = true;
    return KLB_OK;
}

static int ensure_dense(klb_t* h) {
    if (!h->fdense_dev) {
        if (cudaMalloc(&h->fdense_dev, sizeof(double) * NQ * (size_t)h->g.nx * h->g.ny) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, KLB_E_NOMEM, "cudaMalloc of the distribution staging buffer failed");
        }
    }
    return KLB_OK;
}

int klb_set_f(klb_t* h, const double* f, int on_device) {
    if (!h || !f) return h ? fail(h, KLB_E_INVAL, "NULL f") : KLB_E_INVAL;
    if (!h->initialized) return fail(h, KLB_E_STATE, "klb_set_f before klb_init_fields");
    const double* src = f;
    if (!on_device) {
        int r = ensure_dense(h);
        if (r != KLB_OK) return r;
        CK(h, cudaMemcpyAsync(h->fdense_dev, f, sizeof(double) * NQ * (size_t)h->g.nx * h->g.ny,
                              cudaMemcpyHostToDevice, h->stream));
        src = h->fdense_dev;
    }
    cudaError_t e = h->p.precision == KLB_FP64
                        ? launch_set_f<double>(h->g, src, (double*)h->buf[h->cur], h->stream)
                        : launch_set_f<float>(h->g, src, (float*)h->buf[h->cur], h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_f kernel");
    h->launches += 1;
    return KLB_OK;
}

static int check_err(klb_t* h) {
    int v = 0;
    CK(h, cudaMemcpyAsync(&v, h->err_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (fdlb::bounds_flags() != 0)
        return fail(h, KLB_E_BOUNDS, "bounds-checked build: a kernel formed an index outside its buffer");
    if (v) {
        CK(h, cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        if (v & ERR_TIMEOUT) return fail(h, KLB_E_DEVICE_TIMEOUT, "a bounded device-side wait ran out");
        if (v & ERR_NONFINITE) return fail(h, KLB_E_NONFINITE, "a sampled state had rho or T non-finite or <= 0");
    }
    return KLB_OK;
}

int klb_sync(klb_t* h) {
    if (!h) return KLB_E_INVAL;
    CK(h, cudaStreamSynchronize(h->stream));
    return check_err(h);
}

int klb_get_f(klb_t* h, double* f, int on_device) {
    if (!h || !f) return h ? fail(h, KLB_E_INVAL, "NULL f") : KLB_E_INVAL;
    if (!h->initialized) return fail(h, KLB_E_STATE, "klb_get_f before klb_init_fields");
    double* dst = f;
    if (!on_device) {
        int r = ensure_dense(h);
        if (r != KLB_OK) return r;
        dst = h->fdense_dev;
    }
    cudaError_t e = h->p.precision == KLB_FP64
                        ? launch_get_f<double>(h->g, (const double*)h->buf[h->cur], dst, h->stream)
                        : launch_get_f<float>(h->g, (const float*)h->buf[h->cur], dst, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_f kernel");
    h->launches += 1;
    if (!on_device)
        CK(h, cudaMemcpyAsync(f, h->fdense_dev, sizeof(double) * NQ * (size_t)h->g.nx * h->g.ny,
                              cudaMemcpyDeviceToHost, h->stream));
    return klb_sync(h);
}

}  // extern "C"

// partial diagnostics records written by one launch of the current kernel
static int records(const klb_t* h) {
    if (h->p.precision == KLB_FP64) return h->nparts;
    return f32_grid(h->g.nx, h->g.ny, h->variant);
}

int fdlb::handle_upload_descs(klb_t* h) {
    if (h->p.precision != KLB_FP32) return KLB_OK;
    int tiles_x, ntiles;
    f32_tiles(h->g.nx, h->g.ny, h->variant, &tiles_x, &ntiles);
    // the kernels split a tile index into (row, column) by a float quotient
    // estimate that is exact below 2^24 tiles
    if (ntiles >= (1 << 24)) return fail(h, KLB_E_INVAL, "grid too large for the FP32 tile index (2^24 tiles)");
    InstDesc d[2];
    for (int p = 0; p < 2; ++p) {  // descriptor p: the state is in buf[p], the next one goes to buf[1 - p]
        memset(&d[p], 0, sizeof(InstDesc));
        d[p].map = h->map[p];
        d[p].out = (float*)h->buf[1 - p];
        d[p].g = h->g;
        d[p].tiles_x = tiles_x;
        d[p].first_tile = 0;
    }
    CK(h, cudaMemcpy(h->descs_dev, d, sizeof(d), cudaMemcpyHostToDevice));
    h->ntiles = ntiles;
    return KLB_OK;
}

void fdlb::handle_after_step(klb_t* h) {
    h->cur = 1 - h->cur;
    h->steps += 1;
    if (h->p.sample_every > 0 && h->steps % h->p.sample_every == 0) h->pending_sample = true;
}

// one step: optional fused diagnostics of the input state, then ping-pong
static int one_step(klb_t* h) {
    double* parts = nullptr;
    if (h->pending_sample) parts = h->diag_partials;
    cudaError_t e;
    const int src = h->cur, dst = 1 - h->cur;
    if (h->p.precision == KLB_FP64)
        e = launch_step<double>(h->map[src], h->cd, h->g, (double*)h->buf[dst], parts, h->err_dev, h->spin_limit,
                                h->inject, h->stream);
    else
        e = launch_step_f32(h->cf, h->descs_dev + src, 1, h->ntiles, parts, h->err_dev, h->spin_limit, h->inject,
                            h->variant, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
    h->launches += 1;
    if (parts) {
        e = launch_diag_finalize(parts, records(h), h->diag_ring, h->cap, h->nsamp_dev, h->err_dev, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics finalize");
        h->launches += 1;
        h->pending_sample = false;
    }
    fdlb::handle_after_step(h);
    return KLB_OK;
}

void fdlb::handle_drop_graphs(klb_t* h) {
    for (int p = 0; p < 2; ++p)
        for (int d = 0; d < 2; ++d)
            if (h->graph[p][d]) {
                cudaGraphExecDestroy(h->graph[p][d]);
                h->graph[p][d] = nullptr;
            }
}

// capture graph_steps steps from the handle's present parity and sampling
// state (a step count that is a multiple of the sampling period): the
// capture records the launches only, so the bookkeeping is restored after it
static int build_step_graph(klb_t* h) {
    const int p = h->cur, d = h->pending_sample ? 1 : 0;
    const int cur = h->cur;
    const int64_t steps = h->steps, launches = h->launches;
    const bool pending = h->pending_sample;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        h->use_graph = false;  // a stream that cannot be captured: one launch per step
        return KLB_OK;
    }
    int r = KLB_OK;
    for (int s = 0; s < h->graph_steps && r == KLB_OK; ++s) r = one_step(h);
    cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
    h->graph_launches[p][d] = h->launches - launches;
    h->cur = cur;
    h->steps = steps;
    h->launches = launches;
    h->pending_sample = pending;
    if (r != KLB_OK || ec != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        h->use_graph = false;  // step one launch at a time from now on
        cudaGetLastError();
        return r != KLB_OK ? r : KLB_OK;
    }
    cudaError_t ei = cudaGraphInstantiate(&h->graph[p][d], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        h->graph[p][d] = nullptr;
        h->use_graph = false;
        cudaGetLastError();
    }
    return KLB_OK;
}

extern "C" {

int klb_step(klb_t* h, int64_t n) {
    fdlb::NvtxRange trace_("klb_step");
    if (!h) return KLB_E_INVAL;
    if (n < 0) return fail(h, KLB_E_INVAL, "negative step count");
    if (!h->initialized) return fail(h, KLB_E_STATE, "klb_step before klb_init_fields");
    if (h->broken) return fail(h, KLB_E_STATE, "the handle's tile shape could not be restored (klb_set_variant)");
    const int se = h->p.sample_every;
    while (n > 0) {
        // FP32 WENO5 runs of graph_steps steps, starting at a sampling point,
        // are replayed from a CUDA graph (small grids are bound by launch
        // latency); the graph's steps leave the parity where it was and the
        // next sample due, exactly as stepping one launch at a time would
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const bool graphable = h->use_graph && h->graph_steps > 0 && n >= h->graph_steps && h->inject == 0 &&
                               (se == 0 || h->steps % se == 0) &&
                               cudaStreamIsCapturing(h->stream, &cs) == cudaSuccess &&
                               cs == cudaStreamCaptureStatusNone;
        if (graphable) {
            const int p = h->cur, d = h->pending_sample ? 1 : 0;
            if (!h->graph[p][d]) {
                int r = build_step_graph(h);
                if (r != KLB_OK) return r;
            }
            if (h->graph[p][d]) {
                CK(h, cudaGraphLaunch(h->graph[p][d], h->stream));
                h->launches += h->graph_launches[p][d];
                h->steps += h->graph_steps;
                h->pending_sample = se > 0;  // graph_steps is a multiple of the sampling period
                n -= h->graph_steps;
                continue;
            }
        }
        int r = one_step(h);
        if (r != KLB_OK) return r;
        n -= 1;
    }
    return KLB_OK;
}

}  // extern "C"

// take the sample of the current state if it is due and no step has taken it
static int flush_sample(klb_t* h) {
    if (!h->pending_sample) return KLB_OK;
    cudaError_t e = h->p.precision == KLB_FP64
                        ? launch_diag_partials<double>(h->cd, h->g, (const double*)h->buf[h->cur],
                                                       h->diag_partials, h->stream)
                        : launch_diag_f32(h->cf, h->g, (const float*)h->buf[h->cur], h->diag_partials,
                                          h->variant, h->stream);
    if (e == cudaSuccess)
        e = launch_diag_finalize(h->diag_partials, records(h), h->diag_ring, h->cap, h->nsamp_dev, h->err_dev,
                                 h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics kernels");
    h->launches += 2;
    h->pending_sample = false;
    return KLB_OK;
}

static int read_nsamples(klb_t* h, long long* n) {
    CK(h, cudaMemcpyAsync(n, h->nsamp_dev, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return KLB_OK;
}

extern "C" {

int klb_moments(klb_t* h, double* rho, double* ux, double* uy, double* T, int on_device) {
    fdlb::NvtxRange trace_("klb_moments");
    if (!h) return KLB_E_INVAL;
    if (!h->initialized) return fail(h, KLB_E_STATE, "klb_moments before klb_init_fields");
    const size_t n = (size_t)h->g.nx * h->g.ny;
    double* dst[4] = {rho, ux, uy, T};
    double* d[4];
    bool direct[4];  // host outputs the kernel writes directly (pinned, mapped)
    for (int i = 0; i < 4; ++i) {
        void* v = (!on_device && dst[i]) ? device_view(dst[i]) : nullptr;
        direct[i] = v != nullptr;
        d[i] = on_device ? dst[i] : (v ? (double*)v : (dst[i] ? h->fields_dev + i * n : nullptr));
    }
    cudaError_t e = h->p.precision == KLB_FP64
                        ? launch_fields<double>(h->cd, h->g, (const double*)h->buf[h->cur], d[0], d[1], d[2], d[3],
                                                h->stream)
                        : launch_fields<float>(h->cf, h->g, (const float*)h->buf[h->cur], d[0], d[1], d[2], d[3],
                                               h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "fields kernel");
    h->launches += 1;
    if (!on_device)
        for (int i = 0; i < 4; ++i)
            if (dst[i] && !direct[i])
                CK(h, cudaMemcpyAsync(dst[i], d[i], n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return klb_sync(h);
}

int klb_mean_density(klb_t* h, double* out, int on_device) {
    if (!h) return KLB_E_INVAL;
    if (!out) return fail(h, KLB_E_INVAL, "NULL argument");
    if (!h->initialized) return fail(h, KLB_E_STATE, "klb_mean_density before klb_init_fields");
    double* d = on_device ? out : h->fields_dev;  // staging: fields_dev holds 4 nx ny >= ny doubles
    cudaError_t e = h->p.precision == KLB_FP64
                        ? launch_mean_density<double>(h->g, (const double*)h->buf[h->cur], d, h->stream)
                        : launch_mean_density<float>(h->g, (const float*)h->buf[h->cur], d, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "mean density kernel");
    h->launches += 1;
    if (!on_device) CK(h, cudaMemcpyAsync(out, d, h->g.ny * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return klb_sync(h);
}

int klb_diagnostics(klb_t* h, double* out, int64_t cap, int64_t* count) {
    fdlb::NvtxRange trace_("klb_diagnostics");
    if (!h || !count || (cap > 0 && !out)) return h ? fail(h, KLB_E_INVAL, "NULL argument") : KLB_E_INVAL;
    if (!h->initialized) return fail(h, KLB_E_STATE, "klb_diagnostics before klb_init_fields");
    int r = flush_sample(h);
    if (r != KLB_OK) return r;
    long long ns = 0;
    r = read_nsamples(h, &ns);
    if (r != KLB_OK) return r;
    const int64_t avail = std::min<int64_t>(ns, h->cap);
    const int64_t m = std::min<int64_t>(avail, cap);
    const int64_t first = ns - avail;  // oldest retained sample
    // the retained samples in ring order: at most two contiguous runs of slots
    for (int64_t i = 0; i < m;) {
        const int64_t slot = (first + i) % h->cap;
        const int64_t run = std::min<int64_t>(m - i, h->cap - slot);
        CK(h, cudaMemcpyAsync(out + 7 * i, h->diag_ring + 7 * slot, 7 * run * sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
        i += run;
    }
    *count = m;
    return klb_sync(h);
}

int64_t klb_step_count(const klb_t* h) { return h ? h->steps : -1; }

int64_t klb_launch_count(const klb_t* h) { return h ? h->launches : -1; }

int klb_debug_inject_wait_timeout(klb_t* h, int64_t polls) {
    if (!h || polls < 0) return KLB_E_INVAL;
    h->inject = polls > 0 ? 1 : 0;
    h->spin_limit = polls > 0 ? polls : kDefaultSpin;
    fdlb::handle_drop_graphs(h);  // the wait budget is a launch parameter
    return KLB_OK;
}

int klb_debug_bounds_probe(klb_t* h) {
    if (!h) return KLB_E_INVAL;
#ifdef KLB_CHECK_BOUNDS
    if (h->p.precision != KLB_FP32) return fail(h, KLB_E_INVAL, "the probe writes past an FP32 state buffer");
    cudaError_t e = launch_bounds_probe((float*)h->buf[h->cur], (long long)NQ * h->g.plane, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "bounds probe");
    return KLB_OK;
#else
    return fail(h, KLB_E_INVAL, "the bounds probe exists in the bounds-checked build (libklb_checked.so) only");
#endif
}

int klb_set_variant(klb_t* h, int variant) {
    if (!h) return KLB_E_INVAL;
    if (variant < 0 || variant > 1) return fail(h, KLB_E_INVAL, "unknown kernel variant");
    if (h->p.precision == KLB_FP64) {
        if (variant != 0) return fail(h, KLB_E_INVAL, "the FP64 step has one variant");
        return KLB_OK;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    const int old = h->variant;
    // put the old tile shape back (maps and descriptors); a rollback that
    // fails leaves the handle unusable rather than silently inconsistent
    auto rollback = [&](int code) {
        const std::string msg = h->err;
        h->variant = old;
        bool ok = true;
        for (int j = 0; j < 2; ++j) ok = make_map(h, h->buf[j], &h->map[j]) == KLB_OK && ok;
        ok = ok && fdlb::handle_upload_descs(h) == KLB_OK;
        if (!ok) {
            h->broken = true;
            return fail(h, KLB_E_STATE, msg + "; restoring the previous tile shape failed too (" + h->err +
                                            "): the handle refuses further steps");
        }
        h->err = msg;
        return code;
    };
    fdlb::handle_drop_graphs(h);  // their launches name the old tile shape
    h->variant = variant;
    for (int i = 0; i < 2; ++i) {
        int r = make_map(h, h->buf[i], &h->map[i]);
        if (r != KLB_OK) return rollback(r);
    }
    int r = fdlb::handle_upload_descs(h);
    if (r != KLB_OK) return rollback(r);  // keep the handle as it was
    return KLB_OK;
}

int klb_get_variant(const klb_t* h) { return h ? h->variant : -1; }

int klb_layout(const klb_t* h, const void** base, int64_t* pitch, int64_t* plane, int32_t* gx, int32_t* gy) {
    if (!h) return KLB_E_INVAL;
    if (base) *base = h->buf[h->cur];
    if (pitch) *pitch = h->g.px;
    if (plane) *plane = h->g.plane;
    if (gx) *gx = GX;
    if (gy) *gy = GY;
    return KLB_OK;
}

const char* klb_last_error(const klb_t* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

// ---------------------------------------------------------------------------
// checkpoint / resume
// ---------------------------------------------------------------------------
struct SaveHeader {
    char magic[8];
    int32_t version, nx, ny, precision;
    int64_t steps, nsamples;
    int32_t cap, pending;
    klb_params p;
};

int klb_save(klb_t* h, const char* path) {
    if (!h || !path) return KLB_E_INVAL;
    if (!h->initialized) return fail(h, KLB_E_STATE, "klb_save before klb_init_fields");
    int r = flush_sample(h);
    if (r != KLB_OK) return r;
    r = klb_sync(h);
    if (r != KLB_OK) return r;
    const size_t fbytes = (size_t)NQ * h->g.plane * h->esize;
    std::string blob(fbytes, '\0');
    std::string ring(sizeof(double) * 7 * h->cap, '\0');
    CK(h, cudaMemcpy(&blob[0], h->buf[h->cur], fbytes, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(&ring[0], h->diag_ring, ring.size(), cudaMemcpyDeviceToHost));
    SaveHeader hd{};
    memcpy(hd.magic, "KLBSAVE1", 8);
    hd.version = 1;
    hd.nx = h->g.nx;
    hd.ny = h->g.ny;
    hd.precision = h->p.precision;
    long long ns = 0;
    r = read_nsamples(h, &ns);
    if (r != KLB_OK) return r;
    hd.steps = h->steps;
    hd.nsamples = ns;
    hd.cap = h->cap;
    hd.pending = h->pending_sample;
    hd.p = h->p;
    hd.p.stream = nullptr;
    FILE* fp = fopen(path, "wb");
    if (!fp) return fail(h, KLB_E_IO, std::string("cannot open ") + path);
    bool ok = fwrite(&hd, sizeof(hd), 1, fp) == 1 && fwrite(ring.data(), 1, ring.size(), fp) == ring.size() &&
              fwrite(blob.data(), 1, blob.size(), fp) == blob.size();
    ok = (fclose(fp) == 0) && ok;
    return ok ? KLB_OK : fail(h, KLB_E_IO, std::string("write failed: ") + path);
}

int klb_load(klb_t* h, const char* path) {
    if (!h || !path) return KLB_E_INVAL;
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(h, KLB_E_IO, std::string("cannot open ") + path);
    SaveHeader hd{};
    if (fread(&hd, sizeof(hd), 1, fp) != 1 || memcmp(hd.magic, "KLBSAVE1", 8) != 0) {
        fclose(fp);
        return fail(h, KLB_E_IO, "not a klb checkpoint");
    }
    if (hd.nx != h->g.nx || hd.ny != h->g.ny || hd.precision != h->p.precision || hd.cap != h->cap) {
        fclose(fp);
        return fail(h, KLB_E_INVAL, "checkpoint does not match the handle (nx, ny, precision, diag capacity)");
    }
    const size_t fbytes = (size_t)NQ * h->g.plane * h->esize;
    std::string blob(fbytes, '\0');
    std::string ring(sizeof(double) * 7 * h->cap, '\0');
    bool ok = fread(&ring[0], 1, ring.size(), fp) == ring.size() && fread(&blob[0], 1, blob.size(), fp) == blob.size();
    fclose(fp);
    if (!ok) return fail(h, KLB_E_IO, "truncated checkpoint");
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(h->buf[0], blob.data(), fbytes, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->buf[1], blob.data(), fbytes, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->diag_ring, ring.data(), ring.size(), cudaMemcpyHostToDevice));
    const long long ns = hd.nsamples;
    CK(h, cudaMemcpy(h->nsamp_dev, &ns, sizeof(long long), cudaMemcpyHostToDevice));
    h->cur = 0;
    h->steps = hd.steps;
    h->pending_sample = hd.pending != 0;
    h->initialized = true;
    return KLB_OK;
}

}  // extern "C"
