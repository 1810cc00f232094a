// Launch interface of the adjoint sweep (see adjoint.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace scd {

struct AdjointLaunch {
    const GrainSweep *grain;   // the context's sweep descriptor (device)
    const int2 *items;         // (0, group), longest first
    int32_t n_items;
    int32_t *counter;
    void *scratch;             // per warp: [lines][max_ns][2][ne_pad] complex
    int64_t scratch_stride;
    int64_t scratch_elems;     // complex T elements of the whole scratch
    const void *wimg;          // T4 per slot: cotangents of (Re Sf, Im Sf, Sg, SF)
    void *gimg;                // T4 per slot, out (accumulated): cotangents of (Re, Im of Delta eta, a)
    int32_t first_sweep;       // the differentiated sweep started from homogeneous values
    int32_t parity;            // exit buffer the differentiated sweep read
    int32_t energies_per_lane;
    int32_t retarded;          // LDOS mode: wimg holds n_e weights per slot
    int32_t grid_blocks, block_threads;
    int32_t stepper;           // 0 closed-form step, 1 implicit midpoint rule
    int32_t blocked;           // the grain's energies are split into blocks (items carry the block)
    int32_t ckpt;              // forward gamma kept every ckpt samples and recomputed (0: parked at
                               // every sample); FP32 closed-form Matsubara/Ozaki adjoint only
};

cudaError_t launch_adjoint_sweep(bool fp64, const AdjointLaunch &a, cudaStream_t s);
int adjoint_occupancy(bool fp64, int ept, int block_threads, int stepper);
// per-precision instantiations (adjoint_f32.cu, adjoint_f64.cu)
cudaError_t launch_adjoint_sweep_f32(const AdjointLaunch &a, cudaStream_t s);
cudaError_t launch_adjoint_sweep_f64(const AdjointLaunch &a, cudaStream_t s);
int adjoint_occupancy_f32(int ept, int block_threads, int stepper);
int adjoint_occupancy_f64(int ept, int block_threads, int stepper);
cudaError_t launch_adjoint_outputs(const GridDev &grid, const uint8_t *mask, const double *delta,
                                   const double *aind, double t, const CompNorm &normD, double kappa, double n_in,
                                   const double *gdn, const double *gj, const double *gF, double gFtot,
                                   double *gacc, double *gdelta, double *gaind, cudaStream_t s);
cudaError_t launch_adjoint_rotate_back(bool fp64, const PairDev *pairs, int32_t n_pairs, const BackLine *bl,
                                       const GridDev &grid, const uint8_t *mask, const double *gacc, void *wimg,
                                       cudaStream_t s);
cudaError_t launch_adjoint_ldos_back(bool fp64, const PairDev *pairs, int32_t n_pairs, const BackLine *bl,
                                     const GridDev &grid, const uint8_t *mask, const double *gN, int32_t n_e,
                                     void *wimg, cudaStream_t s);
cudaError_t launch_adjoint_rotate(bool fp64, const LineGeo *geo, const int32_t *slot_line, int64_t n_slots,
                                  const PairDev *pairs, const GridDev &grid, const int32_t *ghost,
                                  const void *gimg, double *gdelta, double *gaind, cudaStream_t s);

}  // namespace scd
