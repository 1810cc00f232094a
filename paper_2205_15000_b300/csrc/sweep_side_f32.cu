// FP32 batch sweep kernels that also run lattice transfers of other members as
// work items (a separate unit, so it compiles in parallel with sweep_f32.cu).
#include "sweep_kernel.cuh"

namespace scd {

// FP32 batch sweep with lattice transfers as work items
static cudaError_t sweep_side_launch(const SweepLaunch &a, cudaStream_t st) {
    if (a.retarded || a.blocked || a.n_side < 1) return cudaErrorInvalidValue;
    if (a.stepper == 1)
        return a.weighted ? sweep_dispatch<float, false, 1, true, false, true>(a, st)
                          : sweep_dispatch<float, false, 1, false, false, true>(a, st);
    if (a.stepper != 0) return cudaErrorInvalidValue;
    return a.weighted ? sweep_dispatch<float, false, 0, true, false, true>(a, st)
                      : sweep_dispatch<float, false, 0, false, false, true>(a, st);
}

// blocks per SM of the FP32 batch sweep with transfer items
static int sweep_side_occupancy(int ept, int bs, int stepper, bool weighted) {
    if (stepper == 1)
        return weighted ? occ_dispatch<float, false, 1, true, true>(ept, bs) : occ_dispatch<float, false, 1, false, true>(ept, bs);
    return weighted ? occ_dispatch<float, false, 0, true, true>(ept, bs) : occ_dispatch<float, false, 0, false, true>(ept, bs);
}

cudaError_t launch_sweep_side_f32(const SweepLaunch &a, cudaStream_t st) { return sweep_side_launch(a, st); }

int sweep_side_occupancy_f32(int ept, int bs, int stepper, bool weighted) {
    return sweep_side_occupancy(ept, bs, stepper, weighted);
}

SC_BOUNDS_ACCESSOR(bounds_sweep_side_f32)

}  // namespace scd
