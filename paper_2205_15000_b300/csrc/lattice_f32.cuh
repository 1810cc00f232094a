// Device code of the FP32 lattice transfers (Sec. 3.1: bilinear interpolation
// from the reference grid to each rotated lattice and back), shared by their own
// kernels (lattice_f32.cu) and by the batch sweep launches that run the
// transfers of other members as work items of their own (sweep_side_f32.cu).
//
// Positions on the lattices are kept in 64-bit fixed point with 40 fractional
// bits (grid units), so the cell index is an exact shift and the bilinear
// weight an exact fraction; the interpolation itself runs in FP32 and the
// Fermi-surface sums are accumulated in FP32 over blocks of 16 pairs and then
// in FP64.
#pragma once
#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace scd {

__device__ __forceinline__ void split_fixed(int64_t v, int &cell, float &frac) {
    cell = (int)(v >> kFixBits);
    const uint32_t f32 = (uint32_t)((v >> (kFixBits - 32)) & 0xffffffffll);
    frac = (float)f32 * 2.3283064365386963e-10f;  // 2^-32
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

// Rotate back: for every pair, bilinear gather of the four image slots around the
// grid point's lattice coordinates and the Fermi-surface sum.  The grid is taken
// in tiles of 8 x 4 points, one point per lane (so a warp's gathers of one pair
// touch a patch of about nine lattice lines and samples).  The pairs are summed
// in chunks of 16 (FP32 within a chunk, FP64 across chunks); the chunks q, q + 4,
// q + 8, ... form partial sum S_q, and the point's sums are (S_0 + S_1) + (S_2 +
// S_3), whichever warps computed the partial sums.

// grid point (i, j) of lane `lane` in tile blk: each quarter-warp takes 4 x 2 of
// the tile's points
__device__ __forceinline__ void back_tile_point(const GridDev &grid, int64_t blk, int lane, int64_t &i, int64_t &j) {
    const int64_t tiles_x = (grid.nx + 7) / 8;
    const int64_t ty = blk / tiles_x, tx = blk - ty * tiles_x;
    i = tx * 8 + (lane & 3) + 4 * ((lane >> 3) & 1);
    j = ty * 4 + ((lane >> 2) & 1) + 2 * (lane >> 4);
}

// Partial sum S_q of grid point (i, j): the 16-pair chunks q, q + 4, q + 8, ...
// added into A ([5 + 2c], [6 + 2c]: <eta_c Sf> of components c >= 1).
template <int NC>
__device__ __forceinline__ void back_partial(const PairF32 *__restrict__ pairs, int32_t n_pairs,
                                             const BackLine *__restrict__ bl, const GridDev &grid,
                                             const float4 *__restrict__ img, int64_t i, int64_t j, int q,
                                             double (&A)[5 + 2 * NC]) {
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

// the point's sums into the accumulator planes
template <int NC>
__device__ __forceinline__ void back_store(double *__restrict__ acc, int64_t npts, int64_t idx, const double (&A)[5 + 2 * NC]) {
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

// A block of four warps per tile: warp q computes S_q; warp 0 adds the four.
template <int NC>
__device__ __forceinline__ void rotate_back_f32_block(const PairF32 *__restrict__ pairs, int32_t n_pairs,
                                                      const BackLine *__restrict__ bl, const GridDev &grid,
                                                      const uint8_t *__restrict__ mask, const float4 *__restrict__ img,
                                                      double *__restrict__ acc, int64_t blk) {
    constexpr int NV = 5 + 2 * NC;
    __shared__ double part[3][NV][32];
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t i, j;
    back_tile_point(grid, blk, lane, i, j);
    const bool live = i < grid.nx && j < grid.ny;
    const int64_t idx = live ? j * grid.nx + i : 0;
    double A[NV] = {};
    if (live && mask[idx]) back_partial<NC>(pairs, n_pairs, bl, grid, img, i, j, q, A);
    if (q > 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) part[q - 1][v][lane] = A[v];
    }
    __syncthreads();
    if (q != 0 || !live) return;
#pragma unroll
    for (int v = 0; v < NV; ++v) A[v] = (A[v] + part[0][v][lane]) + (part[1][v][lane] + part[2][v][lane]);
    back_store<NC>(acc, (int64_t)grid.nx * grid.ny, idx, A);
}

// One warp per tile (a work item of a batch sweep launch): S_0 .. S_3 one after
// another, added in the same order as the block's, so both give the same sums.
template <int NC>
__device__ __forceinline__ void rotate_back_f32_warp(const PairF32 *__restrict__ pairs, int32_t n_pairs,
                                                     const BackLine *__restrict__ bl, const GridDev &grid,
                                                     const uint8_t *__restrict__ mask, const float4 *__restrict__ img,
                                                     double *__restrict__ acc, int64_t blk, int lane) {
    constexpr int NV = 5 + 2 * NC;
    int64_t i, j;
    back_tile_point(grid, blk, lane, i, j);
    const bool live = i < grid.nx && j < grid.ny;
    if (!live) return;
    const int64_t idx = j * grid.nx + i;
    double S01[NV] = {}, S23[NV] = {};
    if (mask[idx]) {
        for (int q = 0; q < 4; ++q) {
            double A[NV] = {};
            back_partial<NC>(pairs, n_pairs, bl, grid, img, i, j, q, A);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (q < 2) S01[v] += A[v];
                else S23[v] += A[v];
            }
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) S01[v] = S01[v] + S23[v];
    back_store<NC>(acc, (int64_t)grid.nx * grid.ny, idx, S01);
}

}  // namespace scd
