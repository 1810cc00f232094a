// FP64 (plain) instantiations of the sweep kernel.
#include "sweep_kernel.cuh"

namespace scd {

cudaError_t launch_sweep_f64(const SweepLaunch &a, cudaStream_t st) { return sweep_launch_t<double>(a, st); }

int sweep_occupancy_f64(int ept, int bs, int stepper, bool weighted) {
    return sweep_occupancy_t<double>(ept, bs, stepper, weighted);
}

SC_BOUNDS_ACCESSOR(bounds_sweep_f64)

}  // namespace scd
