// klb_step_f64.cu -- FP64 instantiation of the fused step (parity path).
// Built with -fmad=false: every multiply and add is rounded separately, as in
// the paper's formulas evaluated term by term.
#include "klb_step.cuh"

namespace fdlb {
template <>
cudaError_t launch_step<double>(const CUtensorMap& in_map, const StepConst<double>& c, const Geom& g, double* out,
                                double* diag_partials, int* err, long long spin_limit, int inject,
                                cudaStream_t stream) {
    return launch_step_impl<double>(in_map, c, g, out, diag_partials, err, spin_limit, inject, stream);
}
void f64_tile(int* tx, int* ty) {
    *tx = StepTile<double>::TX;
    *ty = StepTile<double>::TY;
}
KLB_BOUNDS_QUERY(bounds_flag_step_f64)

}  // namespace fdlb
