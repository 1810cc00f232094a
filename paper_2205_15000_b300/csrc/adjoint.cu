// Adjoint (reverse-mode) sweep: d(loss)/d(Delta(R), A_ind(R)) for losses that
// depend on the sweep's outputs (Delta_new, j, F), with the boundary entry
// values of the differentiated sweep held fixed.
//
// Per line and energy the forward sweep is two chains of closed-form steps,
// gamma_{i+1} = Phi(gamma_i; c_i) along +e_par and beta_{j+1} = Phi(beta_j; c'_j)
// along -e_par, and the energy sums at each sample are functions of
// (gamma, beta, Delta_sample).  Reverse mode needs every gamma and beta in the
// order opposite to the one they were made in, so the adjoint kernel runs
//   pass 1  (+e_par)  gamma chain, gamma parked at every sample;
//   pass 2  (-e_par)  beta chain, and the gamma adjoint lambda in the same
//                     direction (lambda runs against gamma); beta and the
//                     local beta cotangent are parked;
//   pass 3  (+e_par)  the beta adjoint mu.
// Each step's cotangent with respect to its coefficients (Delta_c, a_c) is
// split half-half onto the segment's two samples (the end segments use one
// sample), giving d(loss)/d(sample values); the transpose of the bilinear
// rotation then gives d(loss)/d(Delta(R)) and d(loss)/d(A_ind(R)).
#include <cuda_runtime.h>
#include <stdint.h>

#include "adjoint.cuh"
#include "riccati_step.cuh"

namespace scd {

#define FULLM 0xffffffffu

namespace {

template <typename T>
__device__ __forceinline__ void atomic_add4(typename Vec4<T>::type *p, T a, T b, T c, T d) {
    T *q = (T *)p;
    atomicAdd(q + 0, a);
    atomicAdd(q + 1, b);
    atomicAdd(q + 2, c);
    atomicAdd(q + 3, d);
}

}  // namespace

// cotangents of the outputs -> cotangents of the accumulators (and the direct
// Delta and A_ind terms of the free energy)
__global__ void adjoint_outputs_kernel(GridDev grid, const uint8_t *__restrict__ mask,
                                       const double *__restrict__ delta, const double *__restrict__ aind,
                                       double t, CompNorm normD, double kappa, double n_in,
                                       const double *__restrict__ gdn, const double *__restrict__ gj,
                                       const double *__restrict__ gF, double gFtot, double *__restrict__ gacc,
                                       double *__restrict__ gdelta, double *__restrict__ gaind) {
    const int nx = grid.nx, ny = grid.ny;
    const int64_t npts = (int64_t)nx * ny;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= npts) return;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    double ac[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // components c >= 1: cotangents of <eta_c Sf>
    if (mask[idx]) {
        if (gdn) {
            for (int c = 0; c < grid.n_comp; ++c) {
                const double cd = normD.kD[c];
                ac[2 * c] = cd * gdn[2 * (c * npts + idx)];
                ac[2 * c + 1] = cd * gdn[2 * (c * npts + idx) + 1];
            }
            a0 = ac[0];
            a1 = ac[1];
        }
        if (gj) {
            const double cj = grid.charge_sign * t / 3.141592653589793;
            a2 = cj * gj[2 * idx];
            a3 = cj * gj[2 * idx + 1];
        }
        const double fb = (gF ? gF[idx] : 0.0) + gFtot / n_in;
        a4 = -0.5 * t * fb;
        // F = sum_c |Delta_c|^2 D_c + ...: direct terms
        for (int c = 0; c < grid.n_comp; ++c) {
            const int64_t o = 2 * (c * npts + idx);
            atomicAdd(&gdelta[o], 2.0 * normD.D[c] * fb * delta[o]);
            atomicAdd(&gdelta[o + 1], 2.0 * normD.D[c] * fb * delta[o + 1]);
        }
        if (aind && kappa > 0.0 && fb != 0.0) {
            const int i = (int)(idx % nx), j = (int)(idx / nx);
            const int ia = i > 0 ? i - 1 : i, ib = i < nx - 1 ? i + 1 : i;
            const int ja = j > 0 ? j - 1 : j, jb = j < ny - 1 ? j + 1 : j;
            const double hx = (ib - ia) * grid.h, hy = (jb - ja) * grid.h;
            const double B = (aind[2 * ((int64_t)j * nx + ib) + 1] - aind[2 * ((int64_t)j * nx + ia) + 1]) / hx -
                             (aind[2 * ((int64_t)jb * nx + i)] - aind[2 * ((int64_t)ja * nx + i)]) / hy;
            const double gB = kappa * kappa * B * fb;
            atomicAdd(&gaind[2 * ((int64_t)j * nx + ib) + 1], gB / hx);
            atomicAdd(&gaind[2 * ((int64_t)j * nx + ia) + 1], -gB / hx);
            atomicAdd(&gaind[2 * ((int64_t)jb * nx + i)], -gB / hy);
            atomicAdd(&gaind[2 * ((int64_t)ja * nx + i)], gB / hy);
        }
    }
    gacc[idx] = a0;
    gacc[npts + idx] = a1;
    gacc[2 * npts + idx] = a2;
    gacc[3 * npts + idx] = a3;
    gacc[4 * npts + idx] = a4;
    for (int c = 1; c < grid.n_comp; ++c) {
        gacc[(3 + 2 * c) * npts + idx] = ac[2 * c];
        gacc[(4 + 2 * c) * npts + idx] = ac[2 * c + 1];
    }
}

// transpose of rotate_back: scatter the accumulator cotangents onto the slots
template <typename T>
__global__ void adjoint_rotate_back_kernel(const PairDev *__restrict__ pairs, int32_t n_pairs,
                                           const BackLine *__restrict__ bl, GridDev grid,
                                           const uint8_t *__restrict__ mask, const double *__restrict__ gacc,
                                           typename Vec4<T>::type *__restrict__ wimg) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= npts || !mask[idx]) return;
    const double g0 = gacc[idx], g1 = gacc[npts + idx], g2 = gacc[2 * npts + idx], g3 = gacc[3 * npts + idx],
                 g4 = gacc[4 * npts + idx];
    double gc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = 1; c < grid.n_comp; ++c) {
        gc[2 * c] = gacc[(3 + 2 * c) * npts + idx];
        gc[2 * c + 1] = gacc[(4 + 2 * c) * npts + idx];
    }
    const double fi = (double)(idx % grid.nx), fj = (double)(idx / grid.nx);
    for (int p = 0; p < n_pairs; ++p) {
        const PairDev pp = pairs[p];
        const double ws = pp.wa + pp.wb;
        double wf0 = ws * pp.eta * g0, wf1 = ws * pp.eta * g1;
        for (int c = 1; c < grid.n_comp; ++c) {  // S_f enters every component's plane
            wf0 += ws * pp.eta_c[c] * gc[2 * c];
            wf1 += ws * pp.eta_c[c] * gc[2 * c + 1];
        }
        const double wg = ws * (pp.ex * g2 + pp.ey * g3), wF = ws * g4;
        const double u = fma(fi, -pp.ey, fma(fj, pp.ex, pp.u0));
        const double v = fma(fi, pp.ex, fma(fj, pp.ey, pp.v0));
        const double fu = floor(u), fv = floor(v);
        const int iu = (int)fu, iv = (int)fv;
        const double wu = u - fu, wv = v - fv;
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const int l = min(max(iu + bb, pp.l_lo), pp.l_hi);
            const BackLine Ln = back_chord_at(bl, grid.n_back, pp.lat0 + (l - pp.l_lo), iv, wv);
            const double wl = bb ? wu : 1.0 - wu;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int m = min(max(iv + c, Ln.m0), Ln.m0 + Ln.ns - 1);
                const double w = wl * (c ? wv : 1.0 - wv);
                if (w == 0.0 || !in_bounds((int64_t)Ln.slot0 + (m - Ln.m0), grid.n_slots)) continue;
                atomic_add4<T>(wimg + Ln.slot0 + (m - Ln.m0), (T)(w * wf0), (T)(w * wf1), (T)(w * wg), (T)(w * wF));
            }
        }
    }
}

// transpose of the LDOS rotate-back: N(R, e_n) = sum_p [w_{p+P} X_p(n) + w_p X_p(mirror n)]
template <typename T>
__global__ void adjoint_ldos_back_kernel(const PairDev *__restrict__ pairs, int32_t n_pairs,
                                         const BackLine *__restrict__ bl, GridDev grid,
                                         const uint8_t *__restrict__ mask, const double *__restrict__ gN,
                                         int32_t n_e, T *__restrict__ wimg) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (idx >= npts || !mask[idx]) return;
    const double gn = gN[(int64_t)n * npts + idx], gm = gN[(int64_t)(n_e - 1 - n) * npts + idx];
    if (gn == 0.0 && gm == 0.0) return;
    const double fi = (double)(idx % grid.nx), fj = (double)(idx / grid.nx);
    for (int p = 0; p < n_pairs; ++p) {
        const PairDev pp = pairs[p];
        // slot value n enters N(n) with w_{p+P} and N(mirror n) with w_p
        const double gv = pp.wb * gn + pp.wa * gm;
        const double u = fma(fi, -pp.ey, fma(fj, pp.ex, pp.u0));
        const double v = fma(fi, pp.ex, fma(fj, pp.ey, pp.v0));
        const double fu = floor(u), fv = floor(v);
        const int iu = (int)fu, iv = (int)fv;
        const double wu = u - fu, wv = v - fv;
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const int l = min(max(iu + bb, pp.l_lo), pp.l_hi);
            const BackLine Ln = back_chord_at(bl, grid.n_back, pp.lat0 + (l - pp.l_lo), iv, wv);
            const double wlin = bb ? wu : 1.0 - wu;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int m = min(max(iv + c, Ln.m0), Ln.m0 + Ln.ns - 1);
                const double w = wlin * (c ? wv : 1.0 - wv);
                if (w == 0.0 || !in_bounds((int64_t)Ln.slot0 + (m - Ln.m0), grid.n_slots)) continue;
                atomicAdd(&wimg[(int64_t)(Ln.slot0 + (m - Ln.m0)) * n_e + n], (T)(w * gv));
            }
        }
    }
}

cudaError_t launch_adjoint_ldos_back(bool fp64, const PairDev *pairs, int32_t n_pairs, const BackLine *bl,
                                     const GridDev &grid, const uint8_t *mask, const double *gN, int32_t n_e,
                                     void *wimg, cudaStream_t st) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int bs = 128;
    dim3 nb((unsigned)((npts + bs - 1) / bs), (unsigned)n_e);
    if (fp64)
        adjoint_ldos_back_kernel<double><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask, gN, n_e, (double *)wimg);
    else
        adjoint_ldos_back_kernel<float><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask, gN, n_e, (float *)wimg);
    return cudaGetLastError();
}

// transpose of rotate_fields: scatter the sample-value cotangents onto the grid
template <typename T>
__global__ void adjoint_rotate_kernel(const LineGeo *__restrict__ geo, const int32_t *__restrict__ slot_line,
                                      int64_t n_slots, const PairDev *__restrict__ pairs, GridDev grid,
                                      const int32_t *__restrict__ ghost,
                                      const typename Vec4<T>::type *__restrict__ gimg,
                                      double *__restrict__ gdelta, double *__restrict__ gaind) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slots) return;
    const int32_t Ls = slot_line[s];
    if (!in_bounds(Ls, grid.n_lines)) return;
    const LineGeo lg = geo[Ls];
    if (lg.ns == 0) return;  // no sample, no cotangent
    if (!in_bounds(lg.pair, grid.n_pairs)) return;
    const typename Vec4<T>::type gv = gimg[s];
    const double gdr = (double)gv.x, gdi = (double)gv.y, ga = (double)gv.z;
    if (gdr == 0.0 && gdi == 0.0 && ga == 0.0) return;
    const PairDev pp = pairs[lg.pair];
    const double h = grid.h;
    const double sc = (double)(lg.m0 + (int)(s - lg.slot0)) * h;
    const double lh = lg.l * h;
    const double x = grid.ox + lh * (-pp.ey) + sc * pp.ex;
    const double y = grid.oy + lh * pp.ex + sc * pp.ey;
    const double gx = (x - grid.x0) / h - 0.5, gy = (y - grid.y0) / h - 0.5;
    const double fi = floor(gx), fj = floor(gy);
    const int i0 = (int)fi, j0 = (int)fj;
    const double fx = gx - fi, fy = gy - fj;
    if (i0 < -1 || i0 > grid.nx - 1 || j0 < -1 || j0 > grid.ny - 1) return;
    const int px = grid.nx + 2;
    const double sa = grid.charge_sign * ga;
#pragma unroll
    for (int bq = 0; bq < 2; ++bq)
#pragma unroll
        for (int aq = 0; aq < 2; ++aq) {
            const double w = (aq ? fx : 1.0 - fx) * (bq ? fy : 1.0 - fy);
            const int src = ghost[(j0 + bq + 1) * px + (i0 + aq + 1)];
            if (src < 0 || w == 0.0) continue;
            atomicAdd(&gdelta[2 * (int64_t)src], w * pp.eta * gdr);
            atomicAdd(&gdelta[2 * (int64_t)src + 1], w * pp.eta * gdi);
            // Delta(p, sample) = sum_c eta_c(p) Delta_c(sample)
            const int64_t npts = (int64_t)grid.nx * grid.ny;
            for (int c = 1; c < grid.n_comp; ++c) {
                atomicAdd(&gdelta[2 * (c * npts + src)], w * pp.eta_c[c] * gdr);
                atomicAdd(&gdelta[2 * (c * npts + src) + 1], w * pp.eta_c[c] * gdi);
            }
            if (gaind) {
                atomicAdd(&gaind[2 * (int64_t)src], w * sa * pp.ex);
                atomicAdd(&gaind[2 * (int64_t)src + 1], w * sa * pp.ey);
            }
        }
}

// The adjoint sweep kernel is instantiated per precision in adjoint_f32.cu /
// adjoint_f64.cu.
cudaError_t launch_adjoint_sweep(bool fp64, const AdjointLaunch &a, cudaStream_t st) {
    return fp64 ? launch_adjoint_sweep_f64(a, st) : launch_adjoint_sweep_f32(a, st);
}

int adjoint_occupancy(bool fp64, int ept, int bs, int stepper) {
    return fp64 ? adjoint_occupancy_f64(ept, bs, stepper) : adjoint_occupancy_f32(ept, bs, stepper);
}

cudaError_t launch_adjoint_outputs(const GridDev &grid, const uint8_t *mask, const double *delta,
                                   const double *aind, double t, const CompNorm &normD, double kappa, double n_in,
                                   const double *gdn, const double *gj, const double *gF, double gFtot,
                                   double *gacc, double *gdelta, double *gaind, cudaStream_t st) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int bs = 256;
    adjoint_outputs_kernel<<<(unsigned)((npts + bs - 1) / bs), bs, 0, st>>>(
        grid, mask, delta, aind, t, normD, kappa, n_in, gdn, gj, gF, gFtot, gacc, gdelta, gaind);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_rotate_back(bool fp64, const PairDev *pairs, int32_t n_pairs, const BackLine *bl,
                                       const GridDev &grid, const uint8_t *mask, const double *gacc, void *wimg,
                                       cudaStream_t st) {
    const int64_t npts = (int64_t)grid.nx * grid.ny;
    const int bs = 128;
    const unsigned nb = (unsigned)((npts + bs - 1) / bs);
    if (fp64)
        adjoint_rotate_back_kernel<double><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask, gacc,
                                                              (double4_32a *)wimg);
    else
        adjoint_rotate_back_kernel<float><<<nb, bs, 0, st>>>(pairs, n_pairs, bl, grid, mask, gacc, (float4 *)wimg);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_rotate(bool fp64, const LineGeo *geo, const int32_t *slot_line, int64_t n_slots,
                                  const PairDev *pairs, const GridDev &grid, const int32_t *ghost,
                                  const void *gimg, double *gdelta, double *gaind, cudaStream_t st) {
    const int bs = 256;
    const unsigned nb = (unsigned)((n_slots + bs - 1) / bs);
    if (fp64)
        adjoint_rotate_kernel<double><<<nb, bs, 0, st>>>(geo, slot_line, n_slots, pairs, grid, ghost,
                                                         (const double4_32a *)gimg, gdelta, gaind);
    else
        adjoint_rotate_kernel<float><<<nb, bs, 0, st>>>(geo, slot_line, n_slots, pairs, grid, ghost,
                                                        (const float4 *)gimg, gdelta, gaind);
    return cudaGetLastError();
}

SC_BOUNDS_ACCESSOR(bounds_adjoint_transposes)

}  // namespace scd
