// klb_slabs.cu -- the grid cut in y into slabs, each a grid of its own, with
// the ghost rows at every cut copied from the neighbouring slab before each
// step (the domain decomposition of Eq. 47 over the grid of Sec. III.B).
//
// Per step: one launch of halo_copy_kernel (for every cut, the three rows on
// each side into the other slab's ghost rows, 19 planes, interior columns),
// then one step launch per slab, all on one stream.  A node's update reads
// only its stencil, and the ghost rows hold exactly the rows the whole grid
// would hold there, so the slabs reproduce the whole grid bit for bit.
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "klb_handle.h"

using namespace fdlb;

namespace {

// one block of rows to copy: rows [src_row, src_row + 3) of src into rows
// [dst_row, dst_row + 3) of dst (array rows, ghost rows counted), interior
// columns, all 19 planes
struct HaloCopy {
    const void* src;
    void* dst;
    long long src_plane, dst_plane;
    int src_px, dst_px;
    int src_row, dst_row;
};

template <typename T>
__global__ void halo_copy_kernel(const HaloCopy* __restrict__ jobs, int njobs, int nx) {
    const long long per_job = 3ll * NQ * nx;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < njobs * per_job;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / per_job);
        long long r = t - j * per_job;
        const int q = (int)(r / (3ll * nx));
        r -= q * 3ll * nx;
        const int row = (int)(r / nx), i = (int)(r - (long long)row * nx);
        const HaloCopy& J = jobs[j];
        const T* src = (const T*)J.src;
        T* dst = (T*)J.dst;
        const long long s = q * J.src_plane + (long long)(J.src_row + row) * J.src_px + (i + GX);
        const long long d = q * J.dst_plane + (long long)(J.dst_row + row) * J.dst_px + (i + GX);
        KLB_GUARD(d, NQ * J.dst_plane) dst[d] = KLB_LOAD(src, s, NQ * J.src_plane, T(0));
    }
}

}  // namespace

namespace fdlb {
KLB_BOUNDS_QUERY(bounds_flag_slabs)
}  // namespace fdlb

struct klb_slabs {
    klb_params p{};
    int n = 0;
    std::vector<int> row0, rows;
    std::vector<klb_t*> m;
    HaloCopy* jobs_dev[2] = {nullptr, nullptr};  // copies for members at buffer parity 0 and 1
    int njobs = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
};

static thread_local std::string g_slabs_create_error;

static int sfail(klb_slabs_t* s, int code, const std::string& msg) {
    if (s) s->err = msg;
    else g_slabs_create_error = msg;
    return code;
}

extern "C" {

int klb_slab_partition(int32_t ny, int32_t n, int32_t* row0, int32_t* rows) {
    if (n < 1 || !row0 || !rows || ny < 3 * n) return KLB_E_INVAL;
    int r = 0;
    for (int k = 0; k < n; ++k) {
        row0[k] = r;
        rows[k] = ny / n + (k < ny % n ? 1 : 0);
        r += rows[k];
    }
    return KLB_OK;
}

int klb_slab_neighbors(const klb_params* p, int32_t n, int32_t k, int32_t* below, int32_t* above) {
    if (!p || !below || !above || n < 1 || k < 0 || k >= n) return KLB_E_INVAL;
    const bool per = p->bc_y_lo == KLB_BC_PERIODIC;
    *below = k > 0 ? k - 1 : (per ? n - 1 : -1);
    *above = k < n - 1 ? k + 1 : (per ? 0 : -1);
    return KLB_OK;
}

void klb_slabs_destroy(klb_slabs_t* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (klb_t* h : s->m) klb_destroy(h);
    for (int b = 0; b < 2; ++b)
        if (s->jobs_dev[b]) cudaFree(s->jobs_dev[b]);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int klb_slabs_create(const klb_params* p, int32_t n, klb_slabs_t** out) {
    if (!p || !out) return sfail(nullptr, KLB_E_INVAL, "NULL argument");
    *out = nullptr;
    if (n < 1) return sfail(nullptr, KLB_E_INVAL, "at least one slab");
    if (p->bc_y_lo == KLB_BC_HALO || p->bc_y_hi == KLB_BC_HALO)
        return sfail(nullptr, KLB_E_INVAL, "the domain's own y sides cannot be halo sides");
    klb_slabs_t* s = new klb_slabs();
    s->p = *p;
    s->n = n;
    s->row0.resize(n);
    s->rows.resize(n);
    if (klb_slab_partition(p->ny, n, s->row0.data(), s->rows.data()) != KLB_OK) {
        delete s;
        return sfail(nullptr, KLB_E_INVAL, "every slab needs at least 3 rows (ny >= 3 n)");
    }
    if (p->stream) {
        s->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return sfail(nullptr, KLB_E_CUDA, "cudaStreamCreate failed");
        }
        s->own_stream = true;
    }
    const bool per = p->bc_y_lo == KLB_BC_PERIODIC;
    for (int k = 0; k < n; ++k) {
        klb_params q = *p;
        q.ny = s->rows[k];
        q.stream = s->stream;
        if (n > 1) {
            q.bc_y_lo = (k > 0 || per) ? KLB_BC_HALO : p->bc_y_lo;
            q.bc_y_hi = (k < n - 1 || per) ? KLB_BC_HALO : p->bc_y_hi;
        }
        klb_t* h = nullptr;
        int r = klb_create(&q, &h);
        if (r != KLB_OK) {
            const std::string msg = std::string("slab ") + std::to_string(k) + ": " + klb_last_error(nullptr);
            klb_slabs_destroy(s);
            return sfail(nullptr, r, msg);
        }
        s->m.push_back(h);
    }
    if (n > 1) {
        // for every slab and side with a neighbour: its ghost rows from that
        // neighbour's edge rows, in the buffers of each parity
        for (int b = 0; b < 2; ++b) {
            std::vector<HaloCopy> jobs;
            for (int k = 0; k < n; ++k) {
                int below, above;
                klb_slab_neighbors(p, n, k, &below, &above);
                klb_t* d = s->m[k];
                for (int side = 0; side < 2; ++side) {
                    const int nb = side == 0 ? below : above;
                    if (nb < 0) continue;
                    klb_t* src = s->m[nb];
                    HaloCopy J;
                    J.src = src->buf[b];
                    J.dst = d->buf[b];
                    J.src_plane = src->g.plane;
                    J.dst_plane = d->g.plane;
                    J.src_px = src->g.px;
                    J.dst_px = d->g.px;
                    // below: the neighbour's top three rows into rows -3..-1;
                    // above: its bottom three rows into rows ny..ny+2
                    J.src_row = side == 0 ? src->g.ny - 3 + GY : GY;
                    J.dst_row = side == 0 ? 0 : d->g.ny + GY;
                    jobs.push_back(J);
                }
            }
            s->njobs = (int)jobs.size();
            if (cudaMalloc(&s->jobs_dev[b], sizeof(HaloCopy) * jobs.size()) != cudaSuccess ||
                cudaMemcpy(s->jobs_dev[b], jobs.data(), sizeof(HaloCopy) * jobs.size(), cudaMemcpyHostToDevice) !=
                    cudaSuccess) {
                cudaGetLastError();
                klb_slabs_destroy(s);
                return sfail(nullptr, KLB_E_NOMEM, "allocation of the halo copy table failed");
            }
        }
    }
    *out = s;
    return KLB_OK;
}

int klb_slabs_init_fields(klb_slabs_t* s, const double* rho, const double* ux, const double* uy, const double* T,
                          int on_device) {
    if (!s || !rho || !ux || !uy || !T) return s ? sfail(s, KLB_E_INVAL, "NULL argument") : KLB_E_INVAL;
    for (int k = 0; k < s->n; ++k) {
        const size_t off = (size_t)s->row0[k] * s->p.nx;  // rows of a [ny][nx] array are contiguous
        int r = klb_init_fields(s->m[k], rho + off, ux + off, uy + off, T + off, on_device);
        if (r != KLB_OK) return sfail(s, r, s->m[k]->err);
    }
    return KLB_OK;
}

int klb_slabs_step(klb_slabs_t* s, int64_t n) {
    fdlb::NvtxRange trace_("klb_slabs_step");
    if (!s) return KLB_E_INVAL;
    if (n < 0) return sfail(s, KLB_E_INVAL, "negative step count");
    for (klb_t* h : s->m)
        if (!h->initialized) return sfail(s, KLB_E_STATE, "klb_slabs_step before klb_slabs_init_fields");
    const long long work = 3ll * NQ * s->p.nx * s->njobs;
    const int grid = (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, 152ll * 32));
    for (int64_t t = 0; t < n; ++t) {
        if (s->njobs > 0) {
            const int b = s->m[0]->cur;  // the slabs step together: one parity
            if (s->p.precision == KLB_FP64)
                halo_copy_kernel<double><<<grid, 256, 0, s->stream>>>(s->jobs_dev[b], s->njobs, s->p.nx);
            else
                halo_copy_kernel<float><<<grid, 256, 0, s->stream>>>(s->jobs_dev[b], s->njobs, s->p.nx);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return sfail(s, KLB_E_CUDA, std::string("halo copy: ") + cudaGetErrorString(e));
        }
        for (klb_t* h : s->m) {
            int r = klb_step(h, 1);
            if (r != KLB_OK) return sfail(s, r, h->err);
        }
    }
    return KLB_OK;
}

int klb_slabs_get_f(klb_slabs_t* s, double* f, int on_device) {
    if (!s || !f) return s ? sfail(s, KLB_E_INVAL, "NULL argument") : KLB_E_INVAL;
    const size_t nx = (size_t)s->p.nx, ny = (size_t)s->p.ny;
    for (int k = 0; k < s->n; ++k) {
        klb_t* h = s->m[k];
        const size_t rows = (size_t)s->rows[k];
        std::vector<double> host;
        double* tmp = nullptr;  // the slab's [19][rows][nx] distribution
        if (on_device) {
            if (cudaMalloc(&tmp, sizeof(double) * NQ * rows * nx) != cudaSuccess) {
                cudaGetLastError();
                return sfail(s, KLB_E_NOMEM, "staging of a slab's distribution");
            }
        } else {
            host.resize(NQ * rows * nx);
            tmp = host.data();
        }
        int r = klb_get_f(h, tmp, on_device);
        for (int q = 0; q < NQ && r == KLB_OK; ++q) {
            double* dst = f + (q * ny + s->row0[k]) * nx;
            const double* src = tmp + q * rows * nx;
            if (on_device) {
                if (cudaMemcpyAsync(dst, src, sizeof(double) * rows * nx, cudaMemcpyDeviceToDevice, s->stream) !=
                    cudaSuccess)
                    r = KLB_E_CUDA;
            } else {
                memcpy(dst, src, sizeof(double) * rows * nx);
            }
        }
        if (on_device) {
            if (cudaStreamSynchronize(s->stream) != cudaSuccess) r = KLB_E_CUDA;
            cudaFree(tmp);
        }
        if (r != KLB_OK) return sfail(s, r, h->err.empty() ? "copy of a slab's distribution" : h->err);
    }
    return KLB_OK;
}

klb_t* klb_slabs_member(klb_slabs_t* s, int32_t k) { return (s && k >= 0 && k < s->n) ? s->m[k] : nullptr; }

const char* klb_slabs_last_error(const klb_slabs_t* s) { return s ? s->err.c_str() : g_slabs_create_error.c_str(); }

}  // extern "C"
