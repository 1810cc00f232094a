// Induced vector potential by zero-padded FFT convolution (App. D).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace scd {

// Largest transform length (one row of complex doubles in 64 KB of shared
// memory); grids whose padded size exceeds it keep the direct sum.
constexpr int kVecpotMaxFft = 4096;

// Device buffers of one context's transform (owned by the context).
struct VecpotFft {
    int px = 0, py = 0, lx = 0, ly = 0;  // padded sizes and their log2
    double2 *tw_x = nullptr, *tw_y = nullptr;  // exp(-2 pi i k / n), k < n/2
    double2 *buf = nullptr;   // py x px work array
    double2 *tbuf = nullptr;  // px x py work array (transposed)
    double2 *ghat = nullptr;  // transform of the wrapped kernel, px x py
};

// log2 of the padded size for a grid extent (power of two >= 2 n)
int vecpot_fft_log2(int n_grid);
// allow the row kernel its shared memory (once per process)
cudaError_t vecpot_fft_attributes();
// transform of the padded, wrapped G table (W x W, G[|dx| W + |dy|])
cudaError_t vecpot_fft_prepare(const VecpotFft &f, const double *G, int W, int nx, int ny, cudaStream_t st);
// A_ind = -(1/kappa^2) G * (j - <j>) on every grid point; jsum holds sum_mask j
cudaError_t vecpot_fft_apply(const VecpotFft &f, const GridDev &grid, const uint8_t *mask, const double *j,
                             const double *jsum, double n_in, double inv_k2, double *aind, cudaStream_t st);

}  // namespace scd
