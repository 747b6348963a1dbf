// klb_launch.h -- host-side declarations shared by the kernel files and the
// C ABI implementation (not part of the public interface).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "klb_device.cuh"

namespace fdlb {

// Polls granted to the second, draining wait after a bounded wait ran out.
constexpr long long kDrainPolls = 1ll << 22;
// Default poll budget of the tile-load wait.
constexpr long long kDefaultSpin = 1ll << 22;

// One fused step from the state behind `in_map` into `out` (klb_step_f32.cu /
// klb_step_f64.cu).  diag_partials != NULL also reduces the diagnostics of the
// input state; spin_limit bounds the tile-load wait; inject != 0 adds a wait
// on a barrier nothing arrives on (fault injection for tests).
template <typename T>
cudaError_t launch_step(const CUtensorMap& in_map, const StepConst<T>& c, const Geom& g, T* out,
                        double* diag_partials, int* err, long long spin_limit, int inject, cudaStream_t stream);
// FP64 step: TX x TY tiles, one thread per node (klb_step_f64.cu)
void f64_tile(int* tx, int* ty);
// FP32 step (klb_step_f32.cu): persistent CTAs over tiles of 32 columns x
// 16 rows (variant 0) or 8 rows (variant 1); f32_grid = number of CTAs (and
// of diagnostics partial records); f32_box = the TMA box of one tile.
void f32_tiles(int nx, int ny, int variant, int* tiles_x, int* ntiles);
int f32_grid(int nx, int ny, int variant);
int f32_default_variant(int nx, int ny);  // the tile shape a new FP32 handle starts with
void f32_box(int variant, unsigned* bx, unsigned* by, unsigned* bz);
// Descriptor of one grid for the FP32 step: the TMA map of its current state,
// the buffer that receives the next one, its geometry and the index of its
// first tile in the launch's tile index space.  Lives in device memory.
constexpr int kMaxInstances = 256;
struct InstDesc {  // aligned as its CUtensorMap member
    CUtensorMap map;
    float* out;
    Geom g;
    int tiles_x;
    int first_tile;
};
// The diagnostics of one member of a batch, reproduced exactly as its own
// stand-alone reduction would do them (same tiles per CTA, same records).
struct DiagJob {
    const float* f;        // the member's state (buffer of the parity sampled)
    Geom g;
    int tiles_x, ntiles;   // its tiles for the batch's tile shape
    int grid;              // CTAs (records) of its stand-alone reduction, f32_grid
    int first_cta;         // its first CTA in the batched launch
    double* partials;      // its records (grid x 8 doubles)
    double* ring;          // its ring of samples, capacity cap
    int cap;
    long long* counter;    // its sample counter
    int* err;              // its error word
};
// members due for a sample (bit j for member j; kMaxInstances bits)
struct DueMask {
    unsigned w[8];
};
// bit j of the mask, selected with constant indices only (a dynamically
// indexed parameter would be copied to local memory)
#define KLB_DUE_BIT(m, j)                                                                             \
    ((((j) >> 5) == 0 ? (m).w[0] : ((j) >> 5) == 1 ? (m).w[1] : ((j) >> 5) == 2 ? (m).w[2]            \
      : ((j) >> 5) == 3 ? (m).w[3] : ((j) >> 5) == 4 ? (m).w[4] : ((j) >> 5) == 5 ? (m).w[5]          \
      : ((j) >> 5) == 6 ? (m).w[6] : (m).w[7]) >> ((j) & 31) & 1u)
// the records of every due member in one launch of total_ctas CTAs (variant:
// the batch's tile shape), then their folds into their rings in one launch
cudaError_t launch_diag_f32_batch(const StepConst<float>& c, const DiagJob* jobs, int njobs, int total_ctas,
                                  int variant, DueMask due, cudaStream_t s);
cudaError_t launch_diag_finalize_batch(const DiagJob* jobs, int njobs, DueMask due, cudaStream_t s);

// One launch steps every grid of `descs` (ninst entries, ntiles tiles in all).
// diag_partials (ninst == 1 only) also reduces the diagnostics of the input.
cudaError_t launch_step_f32(const StepConst<float>& c, const InstDesc* descs, int ninst, int ntiles,
                            double* diag_partials, int* err, long long spin_limit, int inject, int variant,
                            cudaStream_t stream);
// set the kernels' attributes and query the device once (before any capture)
cudaError_t prepare_f32_kernels();
// the step with a lower-order convection scheme (c.scheme 1..3), rows 8 or 16
cudaError_t launch_step_f32_lo(const StepConst<float>& c, const InstDesc* descs, int ninst, int ntiles,
                               double* diag_partials, int* err, long long spin_limit, int inject, int rows, int grid,
                               cudaStream_t stream);
cudaError_t launch_diag_f32(const StepConst<float>& c, const Geom& g, const float* f, double* partials, int variant,
                            cudaStream_t s);

// f := f^(0)(fields) on the interior, with ghost images (klb_aux.cu).
template <typename T>
cudaError_t launch_init_feq(const StepConst<T>& c, const Geom& g, const double* rho, const double* ux,
                            const double* uy, const double* Tm, T* out_a, T* out_b, cudaStream_t s);
// Fixed-equilibrium ghosts of both buffers from the edge nodes of the fields.
template <typename T>
cudaError_t launch_fixed_ghosts(const StepConst<T>& c, const Geom& g, const double* rho, const double* ux,
                                const double* uy, const double* Tm, T* out_a, T* out_b, cudaStream_t s);
// interior f from / to a dense double array [19][ny][nx]
template <typename T>
cudaError_t launch_set_f(const Geom& g, const double* src, T* dst, cudaStream_t s);
template <typename T>
cudaError_t launch_get_f(const Geom& g, const T* src, double* dst, cudaStream_t s);
// macroscopic fields of the interior
// rho_bar[j] = (1/nx) sum_i rho(i, j) for j < ny (klb_aux.cuh)
template <typename T>
cudaError_t launch_mean_density(const Geom& g, const T* f, double* out, cudaStream_t s);
template <typename T>
cudaError_t launch_fields(const StepConst<T>& c, const Geom& g, const T* f, double* rho, double* ux, double* uy,
                          double* Tm, cudaStream_t s);
// stand-alone diagnostics partials of a state (same tiles and order as the fused path)
template <typename T>
cudaError_t launch_diag_partials(const StepConst<T>& c, const Geom& g, const T* f, double* partials,
                                 cudaStream_t s);
// reduce nparts partial records into ring slot (*counter % cap) of `ring`
// (7 doubles per slot), advance *counter; sets ERR_NONFINITE in *err.  The slot
// is chosen on the device, so the launch can be captured in a CUDA graph.
cudaError_t launch_diag_finalize(const double* partials, int nparts, double* ring, int cap, long long* counter,
                                 int* err, cudaStream_t s);

// Bounds-checked builds: each translation unit's flag of an index out of
// range (read and cleared; always 0 in ordinary builds), and their union.
int bounds_flag_aux_f32();
int bounds_flag_aux_f64();
int bounds_flag_step_f32();
int bounds_flag_step_f32_lo();
int bounds_flag_step_f64();
int bounds_flag_adjoint();
int bounds_flag_slabs();
int bounds_flags();
// bounds-checked builds only: one guarded store past the end of a buffer of
// n floats (skipped and flagged); cudaErrorNotSupported elsewhere
cudaError_t launch_bounds_probe(float* p, long long n, cudaStream_t s);

}  // namespace fdlb
