// klb_step_f32.cu -- FP32 instantiation of the fused step (production path).
#include "klb_step.cuh"

namespace fdlb {
template <>
cudaError_t launch_step<float>(const CUtensorMap& in_map, const StepConst<float>& c, const Geom& g, float* out,
                               double* diag_partials, int* err, long long spin_limit, int inject,
                               cudaStream_t stream) {
    return launch_step_impl<float>(in_map, c, g, out, diag_partials, err, spin_limit, inject, stream);
}
void step_tile_shape(int precision, int* tx, int* ty) {
    if (precision == 1) {
        *tx = StepTile<double>::TX;
        *ty = StepTile<double>::TY;
    } else {
        *tx = StepTile<float>::TX;
        *ty = StepTile<float>::TY;
    }
}
}  // namespace fdlb
