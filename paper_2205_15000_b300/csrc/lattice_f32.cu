// FP32 production path of the lattice transfers (Sec. 3.1: bilinear
// interpolation from the reference grid to each rotated lattice and back).
//
// Positions on the lattices are kept in 64-bit fixed point with 40 fractional
// bits (grid units), so the cell index is an exact shift and the bilinear
// weight an exact fraction; the interpolation itself runs in FP32 and the
// Fermi-surface sums are accumulated in FP32 over blocks of 16 pairs and then
// in FP64.  The FP64 sweep keeps the plain FP64 kernels in kernels.cu.
#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace scd {

namespace {

__device__ __forceinline__ void split_fixed(int64_t v, int &cell, float &frac) {
    cell = (int)(v >> kFixBits);
    const uint32_t f32 = (uint32_t)((v >> (kFixBits - 32)) & 0xffffffffll);
    frac = (float)f32 * 2.3283064365386963e-10f;  // 2^-32
}

}  // namespace

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

// Bilinear Delta and A_ind at sample q of a line from the ghost-filled padded
// grid, which holds the nearest grain point's values wherever a stencil point
// with a nonzero weight can fall; GAUGE (sc_gauge) selects how A_ext enters: the
// symmetric gauge's per-line constant, or the landau / solenoid potential at the
// sample.  The fourth value of a slot is 0 (the bounds-checked build counts a
// stencil point with a nonzero weight and no grain neighbour as a violation).
template <int GAUGE>
__device__ __forceinline__ float4 rotate_f32_sample(const LineF32 &ln, const PairF32 &pp, const GridDev &grid,
                                                    const int32_t *__restrict__ ghost,
                                                    const float4 *__restrict__ pad0, const float2 *__restrict__ padc,
                                                    int q) {
    const int px = grid.nx + 2;
    const int64_t npad = (int64_t)px * (grid.ny + 2);
    int i0, j0;
    float fx, fy;
    split_fixed(ln.gx0 + (int64_t)q * pp.dx, i0, fx);
    split_fixed(ln.gy0 + (int64_t)q * pp.dy, j0, fy);
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i0 >= -1 && i0 <= grid.nx - 1 && j0 >= -1 && j0 <= grid.ny - 1) {
        const int base = (j0 + 1) * px + (i0 + 1);
        const float4 p00 = pad0[base], p10 = pad0[base + 1], p01 = pad0[base + px], p11 = pad0[base + px + 1];
        const float w00 = (1.f - fx) * (1.f - fy), w10 = fx * (1.f - fy), w01 = (1.f - fx) * fy, w11 = fx * fy;
        const float dr = w00 * p00.x + w10 * p10.x + w01 * p01.x + w11 * p11.x;
        const float di = w00 * p00.y + w10 * p10.y + w01 * p01.y + w11 * p11.y;
        const float ax = w00 * p00.z + w10 * p10.z + w01 * p01.z + w11 * p11.z;
        const float ay = w00 * p00.w + w10 * p10.w + w01 * p01.w + w11 * p11.w;
        o.x = pp.eta * dr;
        o.y = pp.eta * di;
        // Delta(p, sample) = sum_c eta_c(p) Delta_c(sample) (Eq. order_parameter)
        for (int c = 1; c < grid.n_comp; ++c) {
            const float2 *pc = padc + (c - 1) * npad;
            const float2 e00 = pc[base], e10 = pc[base + 1], e01 = pc[base + px], e11 = pc[base + px + 1];
            o.x += pp.eta_c[c] * (w00 * e00.x + w10 * e10.x + w01 * e01.x + w11 * e11.x);
            o.y += pp.eta_c[c] * (w00 * e00.y + w10 * e10.y + w01 * e01.y + w11 * e11.y);
        }
#ifdef SC_DEBUG_BOUNDS
        in_bounds((ghost[base] >= 0 || w00 == 0.f) && (ghost[base + 1] >= 0 || w10 == 0.f) &&
                          (ghost[base + px] >= 0 || w01 == 0.f) && (ghost[base + px + 1] >= 0 || w11 == 0.f)
                      ? 0
                      : -1,
                  1);
#else
        (void)ghost;
#endif
        float az = ln.aext;
        if (GAUGE != 0) {
            // landau and solenoid gauges: A_ext at the sample, from its exact
            // fixed-point offset to the gauge origin
            const float sc = (float)(grid.h / (double)(1ll << kFixBits));  // fixed-point unit times h
            const float xr = (float)(ln.gx0 + (int64_t)q * pp.dx - grid.gfx) * sc;
            const float yr = (float)(ln.gy0 + (int64_t)q * pp.dy - grid.gfy) * sc;
            float axe, aye;
            if (GAUGE == 2) {
                const float c = 0.5f * (float)grid.flux / (xr * xr + yr * yr);
                axe = -c * yr;
                aye = c * xr;
            } else {
                axe = -(float)grid.bfield * yr;
                aye = 0.f;
            }
            az += (float)grid.charge_sign * (pp.ex_f * axe + pp.ey_f * aye);
        }
        o.z = az + (float)grid.charge_sign * (pp.ex_f * ax + pp.ey_f * ay);
    }
    return o;
}

// One warp per four consecutive lines (lines of a pair are neighbours on the
// lattice), eight lanes per line: lane (k, s) takes the sample of line L0 + k at
// lattice index mb + s, so one pass of the warp covers a patch of 8 samples x 4
// lines -- its bilinear stencils lie within about nine grid rows and columns at
// any angle -- and stores 8 consecutive slots (128 bytes) of each line.
template <int GAUGE>
__device__ __forceinline__ void rotate_f32_quad(const LineF32 *__restrict__ lines, int64_t L0, int32_t n_lines,
                                                const PairF32 *__restrict__ pairs, const GridDev &grid,
                                                const int32_t *__restrict__ ghost, const float4 *__restrict__ pad0,
                                                const float2 *__restrict__ padc, float4 *__restrict__ out, int lane) {
    // each quarter-warp (8 lanes, one wavefront of 16-byte loads) takes 2 lines x 4
    // samples: lines k = 0..3, samples s = 0..7 of the patch
    const int k = ((lane >> 2) & 1) + 2 * (lane >> 4), s = (lane & 3) + 4 * ((lane >> 3) & 1);
    const int64_t L = L0 + k;
    LineF32 ln{};
    bool ok = L < n_lines;
    if (ok) ln = lines[L];
    ok = ok && in_bounds(ln.pair, grid.n_pairs);
    const int nsl = ln.ns > 0 ? ln.ns : 1;
    ok = ok && in_bounds(ln.slot0, grid.n_slots) && in_bounds((int64_t)ln.slot0 + nsl - 1, grid.n_slots);
    int lo = ok ? ln.m0 : INT_MAX, hi = ok ? ln.m0 + nsl : INT_MIN;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    const PairF32 &pp = pairs[ok ? ln.pair : 0];
    for (int mb = lo; mb < hi; mb += 8) {
        const int q = mb + s - ln.m0;
        if (ok && q >= 0 && q < nsl) out[ln.slot0 + q] = rotate_f32_sample<GAUGE>(ln, pp, grid, ghost, pad0, padc, q);
    }
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

// Rotate back: for every pair, bilinear gather of the four image slots around the
// grid point's lattice coordinates and the Fermi-surface sum.  A block of four
// warps takes a tile of 8 x 4 grid points (so a warp's gathers of one pair touch
// a patch of about nine lattice lines and samples); warp q sums the 16-pair
// chunks q, q + 4, q + 8, ... of every point (FP32 within a chunk, FP64 across
// chunks), so the lanes of a warp gather neighbouring samples of the same pair;
// warp 0 adds the four partial sums in a fixed order.
template <int NC>
__device__ __forceinline__ void rotate_back_f32_block(const PairF32 *__restrict__ pairs, int32_t n_pairs,
                                                      const BackLine *__restrict__ bl, const GridDev &grid,
                                                      const uint8_t *__restrict__ mask, const float4 *__restrict__ img,
                                                      double *__restrict__ acc, int64_t blk) {
    constexpr int NV = 5 + 2 * NC;
    __shared__ double part[3][NV][32];
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the block's tile of 8 x 4 points (back_tiles), one point per lane
    const int64_t tiles_x = (grid.nx + 7) / 8;
    const int64_t ty = blk / tiles_x, tx = blk - ty * tiles_x;
    // each quarter-warp takes 4 x 2 of the tile's points
    const int64_t i = tx * 8 + (lane & 3) + 4 * ((lane >> 3) & 1), j = ty * 4 + ((lane >> 2) & 1) + 2 * (lane >> 4);
    const bool live = i < grid.nx && j < grid.ny;
    const int64_t idx = live ? j * grid.nx + i : 0;
    double A[NV] = {};  // the point's sums; [5 + 2c], [6 + 2c]: <eta_c Sf> of components c >= 1
    if (live && mask[idx]) {
        for (int p0 = 16 * q; p0 < n_pairs; p0 += 64) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
            float ac[2 * NC] = {};
            const int pe = min(p0 + 16, n_pairs);
            for (int p = p0; p < pe; ++p) {
                // the pair's rotate-back fields as five 16-byte loads
                const longlong2 *pv = (const longlong2 *)(pairs + p);
                const longlong2 q0 = pv[0], q1 = pv[1], q2 = pv[2];  // (ui, uj), (u0, vi), (vj, v0)
                const int4 lr = *(const int4 *)(pv + 3);             // l_lo, l_hi, lat0
                const float4 wt = *(const float4 *)(pv + 4);         // w_eta, w_ex, w_ey, w_sum
                int iu, iv;
                float wu, wv;
                split_fixed(i * q0.x + j * q0.y + q1.x, iu, wu);
                split_fixed(i * q1.y + j * q2.x + q2.y, iv, wv);
                const int la = min(max(iu, lr.x), lr.y), lb = min(max(iu + 1, lr.x), lr.y);
                const BackLine La = back_chord_at(bl, grid.n_back, lr.z + (la - lr.x), iv, wv);
                const BackLine Lb = back_chord_at(bl, grid.n_back, lr.z + (lb - lr.x), iv, wv);
                const int ma0 = min(max(iv, La.m0), La.m0 + La.ns - 1);
                const int ma1 = min(max(iv + 1, La.m0), La.m0 + La.ns - 1);
                const int mb0 = min(max(iv, Lb.m0), Lb.m0 + Lb.ns - 1);
                const int mb1 = min(max(iv + 1, Lb.m0), Lb.m0 + Lb.ns - 1);
                const float4 sa0 = ld_chk(img, (int64_t)La.slot0 + (ma0 - La.m0), grid.n_slots);
                const float4 sa1 = ld_chk(img, (int64_t)La.slot0 + (ma1 - La.m0), grid.n_slots);
                const float4 sb0 = ld_chk(img, (int64_t)Lb.slot0 + (mb0 - Lb.m0), grid.n_slots);
                const float4 sb1 = ld_chk(img, (int64_t)Lb.slot0 + (mb1 - Lb.m0), grid.n_slots);
                const float wa0 = (1.f - wu) * (1.f - wv), wa1 = (1.f - wu) * wv;
                const float wb0 = wu * (1.f - wv), wb1 = wu * wv;
                const float x0 = wa0 * sa0.x + wa1 * sa1.x + wb0 * sb0.x + wb1 * sb1.x;
                const float x1 = wa0 * sa0.y + wa1 * sa1.y + wb0 * sb0.y + wb1 * sb1.y;
                const float x2 = wa0 * sa0.z + wa1 * sa1.z + wb0 * sb0.z + wb1 * sb1.z;
                const float x3 = wa0 * sa0.w + wa1 * sa1.w + wb0 * sb0.w + wb1 * sb1.w;
                // S_f, S_F are equal at phi and phi + pi; S_g and v change sign together
                a0 += wt.x * x0;
                a1 += wt.x * x1;
                a2 += wt.y * x2;
                a3 += wt.z * x2;
                a4 += wt.w * x3;
                if constexpr (NC > 1) {
                    const float4 wc4 = *(const float4 *)(pv + 5);  // w_eta_c
                    const float wc[4] = {wc4.x, wc4.y, wc4.z, wc4.w};
#pragma unroll
                    for (int c = 1; c < NC; ++c) {
                        ac[2 * c] += wc[c] * x0;
                        ac[2 * c + 1] += wc[c] * x1;
                    }
                }
            }
            A[0] += a0;
            A[1] += a1;
            A[2] += a2;
            A[3] += a3;
            A[4] += a4;
#pragma unroll
            for (int c = 2; c < 2 * NC; ++c) A[3 + c] += ac[c];
        }
    }
    if (q > 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) part[q - 1][v][lane] = A[v];
    }
    __syncthreads();
    if (q != 0 || !live) return;
#pragma unroll
    for (int v = 0; v < NV; ++v) A[v] = (A[v] + part[0][v][lane]) + (part[1][v][lane] + part[2][v][lane]);
    acc[idx] = A[0];
    acc[npts + idx] = A[1];
    acc[2 * npts + idx] = A[2];
    acc[3 * npts + idx] = A[3];
    acc[4 * npts + idx] = A[4];
#pragma unroll
    for (int c = 1; c < NC; ++c) {
        acc[(3 + 2 * c) * npts + idx] = A[3 + 2 * c];
        acc[(4 + 2 * c) * npts + idx] = A[4 + 2 * c];
    }
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
