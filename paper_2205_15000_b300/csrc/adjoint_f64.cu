// FP64 instantiations of the adjoint sweep kernel.
#include "adjoint_kernel.cuh"

namespace scd {

cudaError_t launch_adjoint_sweep_f64(const AdjointLaunch &a, cudaStream_t st) {
    return adjoint_launch_t<double>(a, st);
}

int adjoint_occupancy_f64(int ept, int bs, int stepper) { return adjoint_occupancy_t<double>(ept, bs, stepper); }

SC_BOUNDS_ACCESSOR(bounds_adjoint_f64)

}  // namespace scd
