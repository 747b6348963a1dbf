// klb_noalloc.cu -- diagnostics of a state without any device allocation.
//
// klb_diagnostics_static() runs the same diagnostics reduction as the
// handle-based path (the per-CTA partial records, then one block that folds
// them), but keeps the partial records in a fixed array of this translation
// unit instead of a buffer allocated by cudaMalloc, and takes the state, its
// layout and the output as plain device pointers.  It serves callers that
// cannot allocate device memory while they run: code running under an
// external memory manager that owns every allocation, a caller that must not
// grow the device footprint after start-up, or a latency-bound loop that
// cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
// The first call on each device looks up the scratch's device address; make
// it before any stream capture.
#include <climits>
#include <mutex>

#include "klb_handle.h"

using namespace fdlb;

// Scratch: one partial record (8 doubles) per CTA of the FP32 reduction or
// per 32 x 8 tile of the FP64 reduction, at most kStaticRecords records
// (256 KiB).  Every GPU that loads the library holds this array until the
// process exits.  Every call on a device shares it.
static constexpr int kStaticRecords = 4096;
static __device__ __align__(256) double g_static_partials[8 * kStaticRecords];
static __device__ long long g_static_counter;  // sample counter the fold kernel advances (one slot: unused)
static __device__ int g_static_flag;           // non-finite flag the fold kernel raises

namespace {

struct Scratch {
    double* partials = nullptr;
    long long* counter = nullptr;
    int* flag = nullptr;
    bool ready = false;
};
constexpr int kMaxDevices = 64;
Scratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

// Device addresses of the scratch on the current device.  In host code the
// arrays' names are host-side stand-ins, not device addresses: the addresses
// come from cudaGetSymbolAddress, once per device, with that device current.
int scratch_for_current_device(Scratch* out, std::string* msg) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        *msg = "no current CUDA device (or device index beyond 63)";
        return KLB_E_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    Scratch& s = g_scratch[dev];
    if (!s.ready) {
        cudaError_t e1 = cudaGetSymbolAddress((void**)&s.partials, g_static_partials);
        cudaError_t e2 = cudaGetSymbolAddress((void**)&s.counter, g_static_counter);
        cudaError_t e3 = cudaGetSymbolAddress((void**)&s.flag, g_static_flag);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            *msg = std::string("cudaGetSymbolAddress failed: ") +
                   cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3));
            return KLB_E_CUDA;
        }
        s.ready = true;
    }
    *out = s;
    return KLB_OK;
}

thread_local std::string g_static_error;

}  // namespace

extern "C" {

int klb_diagnostics_static(const void* f, int32_t precision, int32_t nx, int32_t ny, int64_t pitch,
                           int64_t plane, const double v[3], double* out, void* stream) {
    if (!f || !v || !out) {
        g_static_error = "NULL argument";
        return KLB_E_INVAL;
    }
    if (precision != KLB_FP32 && precision != KLB_FP64) {
        g_static_error = "unknown precision";
        return KLB_E_INVAL;
    }
    if (nx < 1 || ny < 1 || pitch < nx + GX + 3 || plane < pitch * (int64_t)(ny + 2 * GY)) {
        g_static_error = "inconsistent grid size, pitch or plane stride";
        return KLB_E_INVAL;
    }
    // the kernels keep the row pitch and the row index (ghost rows included)
    // in int and form element offsets in 64 bits
    if (pitch > INT_MAX || (int64_t)ny + 2 * GY > INT_MAX) {
        g_static_error = "row pitch beyond the int range of the kernels' row arithmetic";
        return KLB_E_INVAL;
    }
    if (precision == KLB_FP32) {
        // the FP32 reduction splits a tile index into (row, column) by a float
        // quotient estimate that is exact below 2^24 tiles
        int tiles_x = 0, ntiles = 0;
        f32_tiles(nx, ny, 0, &tiles_x, &ntiles);
        if (ntiles >= (1 << 24)) {
            g_static_error = "grid too large for the FP32 tile index (2^24 tiles)";
            return KLB_E_INVAL;
        }
    }
    // partial records the reduction writes, against the scratch capacity
    const long long records =
        precision == KLB_FP32 ? (long long)f32_grid(nx, ny, 0) : ((nx + 31) / 32) * (long long)((ny + 7) / 8);
    if (records > kStaticRecords) {
        g_static_error = "the reduction needs " + std::to_string(records) + " partial records; the static scratch holds " +
                         std::to_string(kStaticRecords) + " (FP64 grids up to 4096 tiles of 32 x 8 nodes)";
        return KLB_E_INVAL;
    }
    Scratch s;
    int r = scratch_for_current_device(&s, &g_static_error);
    if (r != KLB_OK) return r;

    klb_params p;
    klb_params_default(&p);
    p.nx = nx;
    p.ny = ny;
    p.dx = p.dy = p.dt = p.tau = 1.0;  // the diagnostics use the velocities only
    p.v[0] = v[0];
    p.v[1] = v[1];
    p.v[2] = v[2];
    Geom g{};
    g.nx = nx;
    g.ny = ny;
    g.px = (int)pitch;
    g.plane = plane;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(s.flag, 0, sizeof(int), st);  // the flag must start at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(s.counter, 0, sizeof(long long), st);
    if (e == cudaSuccess) {
        if (precision == KLB_FP32) {
            StepConst<float> c{};
            step_constants(p, c);
            e = launch_diag_f32(c, g, (const float*)f, s.partials, 0, st);
        } else {
            StepConst<double> c{};
            step_constants(p, c);
            e = launch_diag_partials<double>(c, g, (const double*)f, s.partials, st);
        }
    }
    if (e == cudaSuccess) e = launch_diag_finalize(s.partials, (int)records, out, 1, s.counter, s.flag, st);
    if (e != cudaSuccess) {
        g_static_error = std::string("diagnostics kernels: ") + cudaGetErrorString(e);
        return KLB_E_CUDA;
    }
    return KLB_OK;
}

const char* klb_diagnostics_static_error(void) { return g_static_error.c_str(); }

}  // extern "C"
