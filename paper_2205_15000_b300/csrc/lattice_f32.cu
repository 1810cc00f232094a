// FP32 production path of the lattice transfers (Sec. 3.1): the field
// conversion onto the ghost-padded grid and the kernels of the rotation and the
// rotate-back, per grain and over every member of a batch (device code of the
// transfers in lattice_f32.cuh).  The FP64 sweep keeps the plain FP64 kernels in
// kernels.cu.
#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "lattice_f32.cuh"

namespace scd {

// Delta (n_comp components, one after another) and A_ind to FP32 on the padded
// grid (nx+2) x (ny+2): each padded point takes the values of its nearest grain
// point (the ghost map), zero where it has none, so the rotation gathers its
// bilinear stencil directly
__device__ __forceinline__ void fields_f32_point(const GridDev &grid, const int32_t *__restrict__ ghost,
                                                 const double2 *__restrict__ delta, const double2 *__restrict__ aind,
                                                 float4 *__restrict__ pad0, float2 *__restrict__ padc, int64_t b) {
    const int64_t npad = (int64_t)(grid.nx + 2) * (grid.ny + 2);
    const int64_t np = (int64_t)grid.nx * grid.ny;
    const int g = ghost[b];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (g >= 0) {
        const double2 d = delta[g];
        v.x = (float)d.x;
        v.y = (float)d.y;
        if (aind) {
            const double2 a = aind[g];
            v.z = (float)a.x;
            v.w = (float)a.y;
        }
    }
    pad0[b] = v;
    for (int c = 1; c < grid.n_comp; ++c) {
        float2 e = make_float2(0.f, 0.f);
        if (g >= 0) {
            const double2 d = delta[c * np + g];
            e = make_float2((float)d.x, (float)d.y);
        }
        padc[(c - 1) * npad + b] = e;
    }
}

__global__ void fields_f32_kernel(GridDev grid, const int32_t *__restrict__ ghost, const double2 *__restrict__ delta,
                                  const double2 *__restrict__ aind, float4 *__restrict__ pad0,
                                  float2 *__restrict__ padc) {
    const int64_t npad = (int64_t)(grid.nx + 2) * (grid.ny + 2);
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < npad) fields_f32_point(grid, ghost, delta, aind, pad0, padc, b);
}

cudaError_t launch_fields_f32(const GridDev &grid, const int32_t *ghost, const double *delta, const double *aind,
                              float4 *pad0, float2 *padc, cudaStream_t st) {
    const int64_t npad = (int64_t)(grid.nx + 2) * (grid.ny + 2);
    const int bs = 256;
    fields_f32_kernel<<<(unsigned)((npad + bs - 1) / bs), bs, 0, st>>>(
        grid, ghost, (const double2 *)delta, (const double2 *)aind, pad0, padc);
    return cudaGetLastError();
}

template <int GAUGE>
__global__ void __launch_bounds__(128) rotate_f32_kernel(const LineF32 *__restrict__ lines,
                                                         const PairF32 *__restrict__ pairs, GridDev grid,
                                                         const int32_t *__restrict__ ghost,
                                                         const float4 *__restrict__ pad0,
                                                         const float2 *__restrict__ padc, float4 *__restrict__ out) {
    const int64_t L0 = (int64_t)blockIdx.x * 16 + 4 * (threadIdx.x >> 5);  // 16 lines per block
    if (L0 >= grid.n_lines) return;
    rotate_f32_quad<GAUGE>(lines, L0, grid.n_lines, pairs, grid, ghost, pad0, padc, out, threadIdx.x & 31);
}

cudaError_t launch_rotate_f32(const LineF32 *lines, const int32_t *slot_line, int64_t n_slots,
                              const PairF32 *pairs, const GridDev &grid, const int32_t *ghost,
                              const float4 *pad0, const float2 *padc, float4 *image_in,
                              cudaStream_t st) {
    (void)slot_line;
    (void)n_slots;
    const unsigned nb = (unsigned)((grid.n_lines + 15) / 16);  // 16 lines per block, four per warp
    if (nb == 0) return cudaSuccess;
    if (grid.gauge == 2)
        rotate_f32_kernel<2><<<nb, 128, 0, st>>>(lines, pairs, grid, ghost, pad0, padc, image_in);
    else if (grid.gauge == 1)
        rotate_f32_kernel<1><<<nb, 128, 0, st>>>(lines, pairs, grid, ghost, pad0, padc, image_in);
    else
        rotate_f32_kernel<0><<<nb, 128, 0, st>>>(lines, pairs, grid, ghost, pad0, padc, image_in);
    return cudaGetLastError();
}

template <int NC>
__global__ void __launch_bounds__(128) rotate_back_f32_kernel(const PairF32 *__restrict__ pairs, int32_t n_pairs,
                                       const BackLine *__restrict__ bl, GridDev grid,
                                       const uint8_t *__restrict__ mask, const float4 *__restrict__ img,
                                       double *__restrict__ acc) {
    rotate_back_f32_block<NC>(pairs, n_pairs, bl, grid, mask, img, acc, blockIdx.x);
}

cudaError_t launch_rotate_back_f32(const PairF32 *pairs, int32_t n_pairs, const BackLine *bl,
                                   const GridDev &grid, const uint8_t *mask, const float4 *image_out,
                                   double *acc, cudaStream_t st) {
    const int bs = 128;
    const unsigned nb = (unsigned)back_tiles(grid.nx, grid.ny);  // a tile of 8 x 4 points per block of four warps
    switch (grid.n_comp) {
        case 1: rotate_back_f32_kernel<1><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask, image_out, acc); break;
        case 2: rotate_back_f32_kernel<2><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask, image_out, acc); break;
        case 3: rotate_back_f32_kernel<3><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask, image_out, acc); break;
        case 4: rotate_back_f32_kernel<4><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask, image_out, acc); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The same transfers for every member of a batch in one launch: each block
// serves one member (its blocks of 256 padded points, 256 slots, or 32 grid
// points), with the member's table in shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) batch_fields_f32_kernel(const MemberDev *__restrict__ m,
                                                               const int64_t *__restrict__ off, int n) {
    __shared__ MemberDev M;
    const int64_t b = batch_member(m, off, n, M) * blockDim.x + threadIdx.x;
    if (b < M.n_pad) fields_f32_point(M.grid, M.ghost, (const double2 *)M.delta, (const double2 *)M.aind, M.pad0, M.padc, b);
}

__global__ void __launch_bounds__(128) batch_rotate_f32_kernel(const MemberDev *__restrict__ m,
                                                               const int64_t *__restrict__ off, int n) {
    __shared__ MemberDev M;
    const int64_t blk = batch_member(m, off, n, M);  // 16 lines per block, four per warp
    const int64_t L0 = blk * 16 + 4 * (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (L0 >= M.grid.n_lines) return;
    switch (M.grid.gauge) {
        case 2: rotate_f32_quad<2>(M.lines, L0, M.grid.n_lines, M.pairs, M.grid, M.ghost, M.pad0, M.padc, M.image_in, lane); break;
        case 1: rotate_f32_quad<1>(M.lines, L0, M.grid.n_lines, M.pairs, M.grid, M.ghost, M.pad0, M.padc, M.image_in, lane); break;
        default: rotate_f32_quad<0>(M.lines, L0, M.grid.n_lines, M.pairs, M.grid, M.ghost, M.pad0, M.padc, M.image_in, lane);
    }
}

// off: prefix of the members' tiles of 8 x 4 grid points, zero for members with
// another component count than NC
template <int NC>
__global__ void __launch_bounds__(128) batch_rotate_back_f32_kernel(const MemberDev *__restrict__ m,
                                                                    const int64_t *__restrict__ off, int n) {
    __shared__ MemberDev M;
    const int64_t blk = batch_member(m, off, n, M);
    rotate_back_f32_block<NC>(M.pairs, M.n_pairs, M.back, M.grid, M.mask, M.image_out, M.acc, blk);
}

cudaError_t launch_batch_fields_rotate_f32(const MemberDev *members, const int64_t *off_pad, int64_t pad_blocks,
                                           const int64_t *off_slots, int64_t slot_blocks, int n, cudaStream_t st) {
    if (pad_blocks > 0) batch_fields_f32_kernel<<<(unsigned)pad_blocks, 256, 0, st>>>(members, off_pad, n);
    if (slot_blocks > 0) batch_rotate_f32_kernel<<<(unsigned)slot_blocks, 128, 0, st>>>(members, off_slots, n);
    return cudaGetLastError();
}

cudaError_t launch_batch_rotate_back_f32(const MemberDev *members, const int64_t *off_blocks, int64_t n_blocks,
                                         int nc, int n, cudaStream_t st) {
    if (n_blocks < 1) return cudaSuccess;
    const unsigned g = (unsigned)n_blocks;
    switch (nc) {
        case 1: batch_rotate_back_f32_kernel<1><<<g, 128, 0, st>>>(members, off_blocks, n); break;
        case 2: batch_rotate_back_f32_kernel<2><<<g, 128, 0, st>>>(members, off_blocks, n); break;
        case 3: batch_rotate_back_f32_kernel<3><<<g, 128, 0, st>>>(members, off_blocks, n); break;
        case 4: batch_rotate_back_f32_kernel<4><<<g, 128, 0, st>>>(members, off_blocks, n); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

SC_BOUNDS_ACCESSOR(bounds_lattice_f32)

}  // namespace scd
