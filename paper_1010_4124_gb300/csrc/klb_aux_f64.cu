// klb_aux_f64.cu -- FP64 instantiations of the auxiliary kernels (parity path;
// built with -fmad=false like the FP64 step).
#include "klb_aux.cuh"

namespace fdlb {

KLB_AUX_INST(double, 32, 8)

}  // namespace fdlb
