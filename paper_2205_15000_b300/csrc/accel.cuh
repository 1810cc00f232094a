// Device side of the self-consistency accelerators (App. E).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace scd {

// x = (Re Delta, Im Delta, kappa^2 A_x, kappa^2 A_y): Delta components over the
// grain points, A components over the whole grid (only when aind != nullptr);
// g = (Delta_new, kappa^2 A_new); d = g - x.
struct AccelArgs {
    int64_t npts;
    int nc;               // order-parameter components: x has 2 nc Delta components (+ 2 for A)
    const uint8_t *mask;
    double *delta;        // x: Delta, [nc][npts] complex interleaved; updated at grain points
    double *aind;         // x: A_ind, 2 per point, or nullptr; updated everywhere
    const double *dnew;   // g: Delta_new
    const double *anew;   // g: A_ind from the sweep's current, or nullptr
    double k2;            // kappa^2
    double *v;            // Polyak velocity, [kAccelComps][npts]
    double *dprev;        // Barzilai-Borwein: the previous d, [kAccelComps][npts]
    double *m;            // CongAcc: moving average of d, [kAccelComps][npts]
};

constexpr int kAccelComps = 10;                    // 2 x 4 Delta components + A_x, A_y
constexpr int kAccelSums = 3 + 3 * kAccelComps;    // reduction slots, see accel.cu

// Deterministic reductions of d against the state buffers; sums[kAccelSums] on
// the device (two launches, fixed order).  partials: [blocks][kAccelSums].
cudaError_t launch_accel_reduce(const AccelArgs &a, double *partials, int blocks, double *sums,
                                cudaStream_t s);
// x <- x + step: kind 0 Picard (x += alpha d), 1 Polyak (v = (1-beta) v + alpha d,
// x += v), 2 Barzilai-Borwein (x += alpha d, dprev = d), 3 CongAcc
// (m_c = w_c m_c + (1-w_c) d_c, x_c += alpha_c m_c); alpha_c, w_c: kAccelComps.
cudaError_t launch_accel_update(const AccelArgs &a, int kind, double alpha, double beta,
                                const double *alpha_c, const double *w_c, cudaStream_t s);
int accel_reduce_blocks(int64_t npts, int sm_count);

}  // namespace scd
