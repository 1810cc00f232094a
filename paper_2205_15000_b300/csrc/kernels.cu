// CUDA kernels of the Riccati sweep (sm_103a).
//
//  rotate_fields  grid Delta(R), A(R) -> per-slot (Delta eta, sigma v.A) on the
//                 rotated lattices (bilinear, nearest-grain-point fill)      [Sec. 3.1]
//  sweep          per (line, energy): gamma along +e_par (angle p) and gamma along
//                 -e_par (angle p+P, = conj gamma~ of angle p), closed-form steps,
//                 propagator and energy sums fused into the backward pass   [Eqs. riccati,
//                 riccati_tilde, riccati_parameterization, symmetries; App. C]
//  rotate_back    per grid point: bilinear gather of every pair's image and the
//                 Fermi-surface sum                                         [Sec. 3.1]
//  outputs        gap equation, current, free energy, residual norms      [Eqs. gapeq_fixpoint,
//                                                                            current_density, qcLWFE]
//  vector_pot     A_ind = -(1/kappa^2) G * (j - <j>)                        [App. D]
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "riccati_step.cuh"

namespace scd {

#define FULL_MASK 0xffffffffu

// ---------------------------------------------------------------------------
// rotate_fields: one thread per image slot
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool bilinear(const GridDev &g, const int32_t *__restrict__ ghost,
                                         const double *__restrict__ f, double x, double y,
                                         double &o0, double &o1) {
    const double gx = (x - g.x0) / g.h - 0.5, gy = (y - g.y0) / g.h - 0.5;
    const double fi = floor(gx), fj = floor(gy);
    const int i0 = (int)fi, j0 = (int)fj;
    const double fx = gx - fi, fy = gy - fj;
    o0 = o1 = 0.0;
    if (i0 < -1 || i0 > g.nx - 1 || j0 < -1 || j0 > g.ny - 1) return false;
    const int px = g.nx + 2;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const double w = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy);
            const int src = ghost[(j0 + b + 1) * px + (i0 + a + 1)];
            if (src < 0) {
                if (w != 0.0) return false;
                continue;
            }
            o0 += w * f[2 * (int64_t)src];
            o1 += w * f[2 * (int64_t)src + 1];
        }
    return true;
}

template <typename T>
__global__ void rotate_kernel(const LineGeo *__restrict__ geo, const int32_t *__restrict__ slot_line,
                              int64_t n_slots, const PairDev *__restrict__ pairs, GridDev grid,
                              const int32_t *__restrict__ ghost, const double *__restrict__ delta,
                              const double *__restrict__ aind, typename Vec4<T>::type *out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slots) return;
    const int32_t Ls = slot_line[s];
    if (!in_bounds(Ls, grid.n_lines)) return;
    const LineGeo lg = geo[Ls];
    if (!in_bounds(lg.pair, grid.n_pairs)) return;
    const PairDev pp = pairs[lg.pair];
    const double h = grid.h;
    const double sc = lg.ns > 0 ? (double)(lg.m0 + (int)(s - lg.slot0)) * h : lg.smid;
    const double lh = lg.l * h;
    const double x = grid.ox + lh * (-pp.ey) + sc * pp.ex;
    const double y = grid.oy + lh * pp.ex + sc * pp.ey;
    double dr, di, ax = 0.0, ay = 0.0;
    bool ok = bilinear(grid, ghost, delta, x, y, dr, di);
    dr *= pp.eta;
    di *= pp.eta;
    // Delta(p, sample) = sum_c eta_c(p) Delta_c(sample) (Eq. order_parameter)
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    for (int c = 1; c < grid.n_comp; ++c) {
        double er, ei;
        ok = bilinear(grid, ghost, delta + 2 * npts * c, x, y, er, ei) && ok;
        dr += pp.eta_c[c] * er;
        di += pp.eta_c[c] * ei;
    }
    if (aind) ok = bilinear(grid, ghost, aind, x, y, ax, ay) && ok;
    // external vector potential of the gauge about (xg, yg): symmetric
    // B/2 (-(y - yg), x - xg), landau B (-(y - yg), 0), solenoid
    // alpha/(2 r^2) (-(y - yg), x - xg) (Eq. solenoid_gauge)
    const double dxg = x - grid.gx, dyg = y - grid.gy;
    if (grid.gauge == 2) {
        const double c = 0.5 * grid.flux / (dxg * dxg + dyg * dyg);
        ax += -c * dyg;
        ay += c * dxg;
    } else if (grid.gauge == 1) {
        ax += -grid.bfield * dyg;
    } else {
        ax += -0.5 * grid.bfield * dyg;
        ay += 0.5 * grid.bfield * dxg;
    }
    const double a = grid.charge_sign * (pp.ex * ax + pp.ey * ay);
    typename Vec4<T>::type o;
    o.x = (T)dr;
    o.y = (T)di;
    o.z = (T)a;
    o.w = ok ? T(0) : T(1);  // 1 flags a sample whose stencil left the grid
    out[s] = o;
}

__global__ void fp64_math_kernel(const double *__restrict__ x, int64_t n, double *__restrict__ rcp,
                                 double *__restrict__ rsq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    rcp[i] = Mth<double>::rcp(x[i]);
    rsq[i] = Mth<double>::rsqrt(x[i]);
}

// FP32 fused multiply-add rate: eight independent chains per thread, scalar or
// two-wide (fma.rn.f32x2: two lane-operations per instruction)
template <bool PK>
__global__ void __launch_bounds__(256) fma_rate_kernel(float *out, int iters, float a, float b) {
    float s = 0.f;
    if constexpr (PK) {
        float2 x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = make_float2((float)(threadIdx.x + k), (float)(blockIdx.x + k));
        const float2 A = make_float2(a, a), B = make_float2(b, b);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = __ffma2_rn(x[k], A, B);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s += x[k].x + x[k].y;
    } else {
        float x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = (float)(threadIdx.x + k);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s += x[k];
    }
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t measure_fma_rate(bool packed, int sm_count, double *lane_ops_per_s, cudaStream_t st) {
    const int blocks = sm_count * 8, threads = 256, iters = 100000;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the second launch is timed
        e = cudaEventRecord(e0, st);
        if (packed)
            fma_rate_kernel<true><<<blocks, threads, 0, st>>>(out, iters, 0.999999f, 1e-7f);
        else
            fma_rate_kernel<false><<<blocks, threads, 0, st>>>(out, iters, 0.999999f, 1e-7f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e == cudaSuccess)
        *lane_ops_per_s = (double)blocks * threads * 8.0 * iters * (packed ? 2.0 : 1.0) / (ms * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return e;
}

cudaError_t launch_fp64_math(const double *x, int64_t n, double *rcp, double *rsqrt, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int bs = 256;
    fp64_math_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(x, n, rcp, rsqrt);
    return cudaGetLastError();
}

cudaError_t launch_rotate(bool fp64, const LineGeo *geo, const int32_t *slot_line, int64_t n_slots,
                          const PairDev *pairs, const GridDev &grid, const int32_t *ghost,
                          const double *delta, const double *aind, void *image_in,
                          cudaStream_t st) {
    const int bs = 256;
    const unsigned nb = (unsigned)((n_slots + bs - 1) / bs);
    if (fp64)
        rotate_kernel<double><<<nb, bs, 0, st>>>(geo, slot_line, n_slots, pairs, grid, ghost, delta,
                                                 aind, (double4_32a *)image_in);
    else
        rotate_kernel<float><<<nb, bs, 0, st>>>(geo, slot_line, n_slots, pairs, grid, ghost, delta,
                                                aind, (float4 *)image_in);
    return cudaGetLastError();
}

// The sweep kernels are instantiated per precision in sweep_f32.cu / sweep_f64.cu.
cudaError_t launch_sweep(bool fp64, const SweepLaunch &a, cudaStream_t st) {
    return fp64 ? launch_sweep_f64(a, st) : launch_sweep_f32(a, st);
}

int sweep_occupancy(bool fp64, int ept, int bs, int stepper, bool weighted) {
    return fp64 ? sweep_occupancy_f64(ept, bs, stepper, weighted) : sweep_occupancy_f32(ept, bs, stepper, weighted);
}

// ---------------------------------------------------------------------------
// rotate_back: one thread per grid point.  For every pair the point's lattice
// coordinates (u across lines, v along them) select two lines (clamped to the
// pair's range, replaced by the nearest line with samples) and two samples on
// each (clamped to the line); the bilinear mix of the four image slots enters
// the Fermi-surface sums with the weights of both angles of the pair.
// ---------------------------------------------------------------------------
template <typename T, int NC>
__global__ void rotate_back_kernel(const PairDev *__restrict__ pairs, int32_t n_pairs,
                                   const BackLine *__restrict__ bl, GridDev grid,
                                   const uint8_t *__restrict__ mask,
                                   const typename Vec4<T>::type *__restrict__ img,
                                   double *__restrict__ acc) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= npts) return;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    double ac[2 * NC] = {};  // <eta_c Sf> of components c >= 1
    if (mask[idx]) {
        const double fi = (double)(idx % grid.nx), fj = (double)(idx / grid.nx);
        for (int p = 0; p < n_pairs; ++p) {
            const PairDev pp = pairs[p];
            const double u = fma(fi, -pp.ey, fma(fj, pp.ex, pp.u0));
            const double v = fma(fi, pp.ex, fma(fj, pp.ey, pp.v0));
            const double fu = floor(u), fv = floor(v);
            const int iu = (int)fu, iv = (int)fv;
            const double wu = u - fu, wv = v - fv;
            double x0 = 0, x1 = 0, x2 = 0, x3 = 0;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int l = min(max(iu + b, pp.l_lo), pp.l_hi);
                const BackLine L = back_chord_at(bl, grid.n_back, pp.lat0 + (l - pp.l_lo), iv, wv);
                const double wl = b ? wu : 1.0 - wu;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int m = min(max(iv + c, L.m0), L.m0 + L.ns - 1);
                    const typename Vec4<T>::type s = ld_chk(img, (int64_t)L.slot0 + (m - L.m0), grid.n_slots);
                    const double w = wl * (c ? wv : 1.0 - wv);
                    x0 += w * (double)s.x;
                    x1 += w * (double)s.y;
                    x2 += w * (double)s.z;
                    x3 += w * (double)s.w;
                }
            }
            const double ws = pp.wa + pp.wb;
            // S_f and S_F are the same at phi and phi + pi; S_g and v change sign
            a0 += ws * pp.eta * x0;
            a1 += ws * pp.eta * x1;
            a2 += ws * pp.ex * x2;
            a3 += ws * pp.ey * x2;
            a4 += ws * x3;
#pragma unroll
            for (int c = 1; c < NC; ++c) {
                ac[2 * c] += ws * pp.eta_c[c] * x0;
                ac[2 * c + 1] += ws * pp.eta_c[c] * x1;
            }
        }
    }
    acc[idx] = a0;
    acc[npts + idx] = a1;
    acc[2 * npts + idx] = a2;
    acc[3 * npts + idx] = a3;
    acc[4 * npts + idx] = a4;
#pragma unroll
    for (int c = 1; c < NC; ++c) {
        acc[(3 + 2 * c) * npts + idx] = ac[2 * c];
        acc[(4 + 2 * c) * npts + idx] = ac[2 * c + 1];
    }
}

cudaError_t launch_rotate_back(bool fp64, const PairDev *pairs, int32_t n_pairs, const BackLine *bl,
                               const GridDev &grid, const uint8_t *mask, const void *image_out,
                               double *acc, cudaStream_t st) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int bs = 128;
    const unsigned nb = (unsigned)((npts + bs - 1) / bs);
#define SC_RB(NC)                                                                                            \
    case NC:                                                                                                 \
        if (fp64)                                                                                            \
            rotate_back_kernel<double, NC><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask,                \
                                                              (const double4_32a *)image_out, acc);          \
        else                                                                                                 \
            rotate_back_kernel<float, NC><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask,                 \
                                                             (const float4 *)image_out, acc);                \
        break;
    switch (grid.n_comp) {
        SC_RB(1) SC_RB(2) SC_RB(3) SC_RB(4)
        default: return cudaErrorInvalidValue;
    }
#undef SC_RB
    return cudaGetLastError();
}

// LDOS rotate-back: N(R, eps_n) = sum_p [w_{p+P} X_p(n) + w_p X_p(mirror n)]
template <typename T>
__global__ void ldos_back_kernel(const PairDev *__restrict__ pairs, int32_t n_pairs,
                                 const BackLine *__restrict__ bl, GridDev grid,
                                 const uint8_t *__restrict__ mask, const T *__restrict__ img,
                                 int32_t n_e, double *__restrict__ out) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (idx >= npts) return;
    double acc = 0.0;
    if (mask[idx]) {
        const double fi = (double)(idx % grid.nx), fj = (double)(idx / grid.nx);
        const int nm = n_e - 1 - n;
        for (int p = 0; p < n_pairs; ++p) {
            const PairDev pp = pairs[p];
            const double u = fma(fi, -pp.ey, fma(fj, pp.ex, pp.u0));
            const double v = fma(fi, pp.ex, fma(fj, pp.ey, pp.v0));
            const double fu = floor(u), fv = floor(v);
            const int iu = (int)fu, iv = (int)fv;
            const double wu = u - fu, wv = v - fv;
            double xn = 0, xm = 0;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int l = min(max(iu + b, pp.l_lo), pp.l_hi);
                const BackLine L = back_chord_at(bl, grid.n_back, pp.lat0 + (l - pp.l_lo), iv, wv);
                const double wl = b ? wu : 1.0 - wu;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int m = min(max(iv + c, L.m0), L.m0 + L.ns - 1);
                    const int64_t sl = (int64_t)(L.slot0 + (m - L.m0)) * n_e;
                    const double w = wl * (c ? wv : 1.0 - wv);
                    xn += w * (double)ld_chk(img, sl + n, grid.n_slots * n_e);
                    xm += w * (double)ld_chk(img, sl + nm, grid.n_slots * n_e);
                }
            }
            acc += pp.wb * xn + pp.wa * xm;
        }
    }
    out[(int64_t)n * npts + idx] = acc;
}

cudaError_t launch_ldos_back(bool fp64, const PairDev *pairs, int32_t n_pairs, const BackLine *bl,
                             const GridDev &grid, const uint8_t *mask, const void *img, int32_t n_e,
                             double *out, cudaStream_t st) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int bs = 128;
    dim3 nb((unsigned)((npts + bs - 1) / bs), (unsigned)n_e);
    if (fp64)
        ldos_back_kernel<double><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask, (const double *)img,
                                                    n_e, out);
    else
        ldos_back_kernel<float><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask, (const float *)img,
                                                   n_e, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// outputs: Delta_new = (t/2pi) <eta Sf> / D, j = sigma (t/pi) <v Sg>,
// F = |Delta|^2 D - (t/2) <SF> + (kappa^2/2) |curl A_ind|^2; block sums of the
// residual, the norm, F and of non-finite values go to sums[0..3].
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL_MASK, v, off);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;
}

__device__ __forceinline__ void outputs_block(const GridDev &grid, const uint8_t *__restrict__ mask,
                                              const double *__restrict__ acc, const double *__restrict__ delta,
                                              const double *__restrict__ aind, double t, const CompNorm &normD,
                                              double kappa, double *__restrict__ dn, double *__restrict__ jo,
                                              double *__restrict__ F, double *__restrict__ partials, int64_t blk) {
    __shared__ double sh[32];
    const int nx = grid.nx, ny = grid.ny;
    const int64_t npts = (int64_t)nx * ny;
    const int64_t idx = blk * blockDim.x + threadIdx.x;
    double num = 0, den = 0, fs = 0, bad = 0;
    if (idx < npts) {
        if (!mask[idx]) {
            for (int c = 0; c < grid.n_comp; ++c) dn[2 * (c * npts + idx)] = dn[2 * (c * npts + idx) + 1] = 0.0;
            jo[2 * idx] = jo[2 * idx + 1] = 0.0;
            F[idx] = 0.0;
        } else {
            const double cj = grid.charge_sign * t / 3.141592653589793;
            jo[2 * idx] = cj * acc[2 * npts + idx];
            jo[2 * idx + 1] = cj * acc[3 * npts + idx];
            // component c (Eq. gapeq_fixpoint): Delta_c = (t/2pi) <eta_c Sf> / D_c;
            // F gains |Delta_c|^2 D_c per component
            double f = -0.5 * t * acc[4 * npts + idx];
            bool fin = true;
            for (int c = 0; c < grid.n_comp; ++c) {
                const int64_t pr = c == 0 ? 0 : 3 + 2 * c, pim = c == 0 ? 1 : 4 + 2 * c;
                const double k = normD.kD[c];
                const double dr = k * acc[pr * npts + idx], di = k * acc[pim * npts + idx];
                const int64_t o = 2 * (c * npts + idx);
                dn[o] = dr;
                dn[o + 1] = di;
                const double d0r = delta[o], d0i = delta[o + 1];
                const double d2 = d0r * d0r + d0i * d0i;
                f += d2 * normD.D[c];
                const double er = dr - d0r, ei = di - d0i;
                num += er * er + ei * ei;
                den += d2;
                fin = fin && isfinite(dr) && isfinite(di);
            }
            if (aind && kappa > 0.0) {
                const int i = (int)(idx % nx), j = (int)(idx / nx);
                const int ia = i > 0 ? i - 1 : i, ib = i < nx - 1 ? i + 1 : i;
                const int ja = j > 0 ? j - 1 : j, jb = j < ny - 1 ? j + 1 : j;
                const double dAy = (aind[2 * ((int64_t)j * nx + ib) + 1] - aind[2 * ((int64_t)j * nx + ia) + 1]) /
                                   ((ib - ia) * grid.h);
                const double dAx = (aind[2 * ((int64_t)jb * nx + i)] - aind[2 * ((int64_t)ja * nx + i)]) /
                                   ((jb - ja) * grid.h);
                const double B = dAy - dAx;
                f += 0.5 * kappa * kappa * B * B;
            }
            F[idx] = f;
            fs = f;
            bad = (fin && isfinite(f) && isfinite(jo[2 * idx]) && isfinite(jo[2 * idx + 1])) ? 0.0 : 1.0;
        }
    }
    const double s0 = block_sum(num, sh);
    const double s1 = block_sum(den, sh);
    const double s2 = block_sum(fs, sh);
    const double s3 = (double)__syncthreads_count(bad != 0.0);  // points with a non-finite value
    if (threadIdx.x == 0) {  // per-block partials, summed in block order by final_sums_kernel
        double *pb = partials + 4 * blk;
        pb[0] = s0;
        pb[1] = s1;
        pb[2] = s2;
        pb[3] = s3;
    }
}

__global__ void outputs_kernel(GridDev grid, const uint8_t *__restrict__ mask,
                               const double *__restrict__ acc, const double *__restrict__ delta,
                               const double *__restrict__ aind, double t, CompNorm normD, double kappa,
                               double *__restrict__ dn, double *__restrict__ jo,
                               double *__restrict__ F, double *__restrict__ partials) {
    outputs_block(grid, mask, acc, delta, aind, t, normD, kappa, dn, jo, F, partials, blockIdx.x);
}

// Deterministic completion of a block reduction: slot k of out = the sum over
// blocks of partials[b][k], in a fixed order (strided per thread, then a fixed tree).
__device__ __forceinline__ void final_sums_block(const double *__restrict__ partials, int nblocks, int nslots,
                                                 double *__restrict__ out) {
    __shared__ double sh[32];
    for (int k = 0; k < nslots; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(int64_t)b * nslots + k];
        const double tot = block_sum(v, sh);
        if (threadIdx.x == 0) out[k] = tot;
    }
}

__global__ void final_sums_kernel(const double *__restrict__ partials, int nblocks, int nslots,
                                  double *__restrict__ out) {
    final_sums_block(partials, nblocks, nslots, out);
}

// Every batch member's outputs in one launch (blocks of 256 grid points over all
// members, the member found by bisection of the block offsets), then one block
// per member completes its sums in the same fixed order as a single context.
__global__ void batch_outputs_kernel(const MemberDev *__restrict__ m, const int64_t *__restrict__ off, int n) {
    __shared__ MemberDev M;
    const int64_t blk = batch_member(m, off, n, M);
    outputs_block(M.grid, M.mask, M.acc, M.delta, M.aind, M.t, M.norms, M.kappa, M.dnew, M.j, M.F, M.partials, blk);
}

__global__ void batch_final_sums_kernel(const MemberDev *__restrict__ m, const int64_t *__restrict__ off) {
    const MemberDev &M = m[blockIdx.x];
    final_sums_block(M.partials, (int)(off[blockIdx.x + 1] - off[blockIdx.x]), 4, M.sums);
}

// The members' grid points, 256 per block: Delta (all component planes) in, A_ind
// zeroed; or Delta_new, j, F out.  The arrays of all members hold member after member;
// pt_off[g] is where member g starts, in complex values for Delta (the sum of n_comp
// nx ny over the members before it).
__global__ void batch_set_fields_kernel(const MemberDev *__restrict__ m, const int64_t *__restrict__ off, int n,
                                        const int64_t *__restrict__ pt_off, const double *__restrict__ delta_all) {
    __shared__ MemberDev M;
    __shared__ int64_t base_sh;
    const int64_t blk = batch_member(m, off, n, M);
    if (threadIdx.x == 0) {
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= (int64_t)blockIdx.x) lo = mid;
            else hi = mid;
        }
        base_sh = pt_off[lo];
    }
    __syncthreads();
    const int64_t np = (int64_t)M.grid.nx * M.grid.ny;
    const int64_t i = blk * blockDim.x + threadIdx.x;
    if (i >= np) return;
    double *d = (double *)M.delta;  // the member's own buffers
    for (int c = 0; c < M.grid.n_comp; ++c) {
        const int64_t o = 2 * (c * np + i);
        d[o] = delta_all[2 * base_sh + o];
        d[o + 1] = delta_all[2 * base_sh + o + 1];
    }
    double *a = (double *)M.aind;
    a[2 * i] = 0.0;
    a[2 * i + 1] = 0.0;
}

// pt_off here: prefix over the members of n_comp np (Delta_new) and, separately,
// of np (j, F), passed as [2][n + 1]
__global__ void batch_get_outputs_kernel(const MemberDev *__restrict__ m, const int64_t *__restrict__ off, int n,
                                         const int64_t *__restrict__ pt_off, double *__restrict__ dnew_all,
                                         double *__restrict__ j_all, double *__restrict__ F_all) {
    __shared__ MemberDev M;
    __shared__ int64_t bc_sh, bp_sh;
    const int64_t blk = batch_member(m, off, n, M);
    if (threadIdx.x == 0) {
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= (int64_t)blockIdx.x) lo = mid;
            else hi = mid;
        }
        bc_sh = pt_off[lo];
        bp_sh = pt_off[(n + 1) + lo];
    }
    __syncthreads();
    const int64_t np = (int64_t)M.grid.nx * M.grid.ny;
    const int64_t i = blk * blockDim.x + threadIdx.x;
    if (i >= np) return;
    if (dnew_all)
        for (int c = 0; c < M.grid.n_comp; ++c) {
            const int64_t o = 2 * (c * np + i);
            dnew_all[2 * bc_sh + o] = M.dnew[o];
            dnew_all[2 * bc_sh + o + 1] = M.dnew[o + 1];
        }
    if (j_all) {
        j_all[2 * (bp_sh + i)] = M.j[2 * i];
        j_all[2 * (bp_sh + i) + 1] = M.j[2 * i + 1];
    }
    if (F_all) F_all[bp_sh + i] = M.F[i];
}

cudaError_t launch_batch_set_fields(const MemberDev *members, const int64_t *off_blocks, int64_t n_blocks,
                                    const int64_t *pt_off, int n, const double *delta_all, cudaStream_t st) {
    if (n_blocks > 0) batch_set_fields_kernel<<<(unsigned)n_blocks, 256, 0, st>>>(members, off_blocks, n, pt_off, delta_all);
    return cudaGetLastError();
}

cudaError_t launch_batch_get_outputs(const MemberDev *members, const int64_t *off_blocks, int64_t n_blocks,
                                     const int64_t *pt_off, int n, double *dnew_all, double *j_all, double *F_all,
                                     cudaStream_t st) {
    if (n_blocks > 0)
        batch_get_outputs_kernel<<<(unsigned)n_blocks, 256, 0, st>>>(members, off_blocks, n, pt_off, dnew_all, j_all,
                                                                     F_all);
    return cudaGetLastError();
}

cudaError_t launch_batch_outputs(const MemberDev *members, const int64_t *off_blocks, int64_t n_blocks, int n,
                                 cudaStream_t st) {
    batch_outputs_kernel<<<(unsigned)n_blocks, 256, 0, st>>>(members, off_blocks, n);
    batch_final_sums_kernel<<<(unsigned)n, 256, 0, st>>>(members, off_blocks);
    return cudaGetLastError();
}

int reduce_blocks(int64_t npts) { return (int)((npts + 255) / 256); }

cudaError_t launch_outputs(const GridDev &grid, const uint8_t *mask, const double *acc,
                           const double *delta, const double *aind, double t, const CompNorm &normD,
                           double kappa, double *delta_new, double *j, double *F, double *sums,
                           double *partials, cudaStream_t st) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int bs = 256, nb = reduce_blocks(npts);
    outputs_kernel<<<(unsigned)nb, bs, 0, st>>>(grid, mask, acc, delta, aind, t, normD, kappa, delta_new, j, F,
                                                partials);
    final_sums_kernel<<<1, 256, 0, st>>>(partials, nb, 4, sums);
    return cudaGetLastError();
}

__global__ void mean_current_kernel(GridDev grid, const uint8_t *__restrict__ mask,
                                    const double *__restrict__ j, double *partials) {
    __shared__ double sh[32];
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double jx = 0, jy = 0;
    if (idx < npts && mask[idx]) {
        jx = j[2 * idx];
        jy = j[2 * idx + 1];
    }
    const double sx = block_sum(jx, sh);
    const double sy = block_sum(jy, sh);
    if (threadIdx.x == 0) {
        partials[2 * (int64_t)blockIdx.x] = sx;
        partials[2 * (int64_t)blockIdx.x + 1] = sy;
    }
}

cudaError_t launch_mean_current(const GridDev &grid, const uint8_t *mask, const double *j,
                                double *sums, double *partials, cudaStream_t st) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int bs = 256, nb = reduce_blocks(npts);
    mean_current_kernel<<<(unsigned)nb, bs, 0, st>>>(grid, mask, j, partials);
    final_sums_kernel<<<1, 256, 0, st>>>(partials, nb, 2, sums);
    return cudaGetLastError();
}

// A_ind(R) = -(1/kappa^2) sum_R' G(|dx|, |dy|) (j(R') - <j>)   (App. D, full correlation)
// One thread per output point; sources staged through shared memory in tiles.
__global__ void vector_potential_kernel(GridDev grid, const uint8_t *__restrict__ mask,
                                        const double *__restrict__ j, const double *__restrict__ jsum,
                                        double n_in, const double *__restrict__ G, int W,
                                        double inv_k2, double *__restrict__ aind) {
    __shared__ double sx[256], sy[256];
    __shared__ int si[256], sj[256];
    const int nx = grid.nx;
    const int64_t npts = (int64_t)nx * grid.ny;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int xi = (int)(idx % nx), yi = (int)(idx / nx);
    const double mx = jsum[0] / n_in, my = jsum[1] / n_in;
    double ax = 0, ay = 0;
    for (int64_t base = 0; base < npts; base += blockDim.x) {
        const int64_t q = base + threadIdx.x;
        __syncthreads();
        if (q < npts && mask[q]) {
            sx[threadIdx.x] = j[2 * q] - mx;
            sy[threadIdx.x] = j[2 * q + 1] - my;
        } else {
            sx[threadIdx.x] = 0.0;
            sy[threadIdx.x] = 0.0;
        }
        si[threadIdx.x] = (int)(q % nx);
        sj[threadIdx.x] = (int)(q / nx);
        __syncthreads();
        const int cnt = (int)min((int64_t)blockDim.x, npts - base);
        if (idx < npts) {
            for (int k = 0; k < cnt; ++k) {
                const double g = G[abs(si[k] - xi) * W + abs(sj[k] - yi)];
                ax += g * sx[k];
                ay += g * sy[k];
            }
        }
    }
    if (idx < npts) {
        aind[2 * idx] = -inv_k2 * ax;
        aind[2 * idx + 1] = -inv_k2 * ay;
    }
}

cudaError_t launch_vector_potential(const GridDev &grid, const uint8_t *mask, const double *j,
                                    const double *jsum, double n_in, const double *G, int W,
                                    double inv_k2, double *aind, cudaStream_t st) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int bs = 256;
    vector_potential_kernel<<<(unsigned)((npts + bs - 1) / bs), bs, 0, st>>>(grid, mask, j, jsum, n_in,
                                                                             G, W, inv_k2, aind);
    return cudaGetLastError();
}

__global__ void copy_kernel(int64_t n, const double *__restrict__ s, double *__restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = s[i];
}

cudaError_t launch_copy_delta(int64_t n, const double *src, double *dst, cudaStream_t st) {
    const int bs = 256;
    copy_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}

// max |a - b| over n complex values (boundary convergence of the burn-in)
template <typename T>
__global__ void max_diff_kernel(int64_t n, const T *__restrict__ a, const T *__restrict__ b,
                                unsigned long long *out) {
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    for (int64_t i = i0; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double dx = (double)a[2 * i] - (double)b[2 * i];
        const double dy = (double)a[2 * i + 1] - (double)b[2 * i + 1];
        const double d = sqrt(dx * dx + dy * dy);
        m = (d > m || d != d) ? (d != d ? 1e300 : d) : m;
    }
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(FULL_MASK, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

cudaError_t launch_max_diff(int64_t n, const void *a, const void *b, bool fp64, double *out,
                            cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    const int bs = 256;
    int nb = (int)((n + bs - 1) / bs);
    if (nb > 4096) nb = 4096;
    if (nb < 1) nb = 1;
    if (fp64)
        max_diff_kernel<double><<<nb, bs, 0, st>>>(n, (const double *)a, (const double *)b,
                                                   (unsigned long long *)out);
    else
        max_diff_kernel<float><<<nb, bs, 0, st>>>(n, (const float *)a, (const float *)b,
                                                  (unsigned long long *)out);
    return cudaGetLastError();
}

// Blocked sweep images: each slot's four sums added over the energy blocks in
// block order (grid-stride over the slots; one thread per slot and component).
template <typename T>
__global__ void block_sum_kernel(const T *__restrict__ blocks, int nb, int64_t n, T *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T s = blocks[i];
        for (int k = 1; k < nb; ++k) s += blocks[(int64_t)k * n + i];
        out[i] = s;
    }
}

cudaError_t launch_block_sum(bool fp64, const void *blocks, int nb, int64_t n_slots, void *out, cudaStream_t st) {
    const int64_t n = 4 * n_slots;
    const int bs = 256;
    int64_t g = (n + bs - 1) / bs;
    if (g > 65536) g = 65536;
    if (g < 1) g = 1;
    if (fp64)
        block_sum_kernel<double><<<(unsigned)g, bs, 0, st>>>((const double *)blocks, nb, n, (double *)out);
    else
        block_sum_kernel<float><<<(unsigned)g, bs, 0, st>>>((const float *)blocks, nb, n, (float *)out);
    return cudaGetLastError();
}

SC_BOUNDS_ACCESSOR(bounds_kernels)

}  // namespace scd
