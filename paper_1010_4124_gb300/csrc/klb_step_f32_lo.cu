// klb_step_f32_lo.cu -- the FP32 step with the lower-order convection schemes
// the paper compares with WENO5 (Sec. III.B, Fig. 2): first-order upwind,
// second-order upwind and second-order TVD, for both tile heights.  A
// translation unit of its own so that it compiles beside the WENO5 one.
// One kernel form serves single grids and batches here (the instance lookup
// costs a single grid little next to the step).
#include "klb_step_f32.cuh"

namespace fdlb {

template <int TY>
static cudaError_t launch_rows(const StepConst<float>& c, const InstDesc* descs, int ninst, int ntiles,
                               double* diag_partials, int* err, long long spin_limit, int inject, int grid,
                               cudaStream_t stream) {
    switch (c.scheme) {
    case 1: return launch_f32_t<TY, 1, true>(c, descs, ninst, ntiles, diag_partials, err, spin_limit, inject, grid, stream);
    case 2: return launch_f32_t<TY, 2, true>(c, descs, ninst, ntiles, diag_partials, err, spin_limit, inject, grid, stream);
    case 3: return launch_f32_t<TY, 3, true>(c, descs, ninst, ntiles, diag_partials, err, spin_limit, inject, grid, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_f32_lo(const StepConst<float>& c, const InstDesc* descs, int ninst, int ntiles,
                               double* diag_partials, int* err, long long spin_limit, int inject, int rows, int grid,
                               cudaStream_t stream) {
    if (rows == 8) return launch_rows<8>(c, descs, ninst, ntiles, diag_partials, err, spin_limit, inject, grid, stream);
    return launch_rows<16>(c, descs, ninst, ntiles, diag_partials, err, spin_limit, inject, grid, stream);
}

KLB_BOUNDS_QUERY(bounds_flag_step_f32_lo)

}  // namespace fdlb
