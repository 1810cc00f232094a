// FP32 instantiations of the adjoint sweep kernel.
#include "adjoint_kernel.cuh"

namespace scd {

cudaError_t launch_adjoint_sweep_f32(const AdjointLaunch &a, cudaStream_t st) {
    return adjoint_launch_t<float>(a, st);
}

int adjoint_occupancy_f32(int ept, int bs, int stepper) { return adjoint_occupancy_t<float>(ept, bs, stepper); }

SC_BOUNDS_ACCESSOR(bounds_adjoint_f32)

}  // namespace scd
