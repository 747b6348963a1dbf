// klb_aux_f64.cu -- FP64 instantiations of the auxiliary kernels (parity path;
// built with -fmad=false like the FP64 step).
#include "klb_aux.cuh"

namespace fdlb {

KLB_AUX_INST(double)

// FP64 diagnostics partials over the tiles of the FP64 step kernel (32 x 8)
template <>
cudaError_t launch_diag_partials<double>(const StepConst<double>& c, const Geom& g, const double* f,
                                         double* partials, cudaStream_t s) {
    return launch_diag_partials_tiles<double, 32, 8>(c, g, f, partials, s);
}

KLB_BOUNDS_QUERY(bounds_flag_aux_f64)

}  // namespace fdlb
