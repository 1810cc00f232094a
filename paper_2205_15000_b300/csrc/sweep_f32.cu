// FP32 (production) instantiations of the sweep kernel.
#include "sweep_kernel.cuh"

namespace scd {

cudaError_t launch_sweep_f32(const SweepLaunch &a, cudaStream_t st) { return sweep_launch_t<float>(a, st); }

int sweep_occupancy_f32(int ept, int bs, int stepper, bool weighted) {
    return sweep_occupancy_t<float>(ept, bs, stepper, weighted);
}

SC_BOUNDS_ACCESSOR(bounds_sweep_f32)

}  // namespace scd
