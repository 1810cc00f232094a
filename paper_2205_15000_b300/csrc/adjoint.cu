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

namespace {

#define FULLM 0xffffffffu

template <typename T>
__device__ __forceinline__ Cx<T> cconj(Cx<T> a) {
    return Cx<T>{a.x, -a.y};
}
template <typename T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) {
    return Cx<T>{a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ Cx<T> cscale(Cx<T> a, T s) {
    return Cx<T>{a.x * s, a.y * s};
}
template <typename T>
__device__ __forceinline__ Cx<T> cmuli(Cx<T> a) {  // i a
    return Cx<T>{-a.y, a.x};
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <typename T>
__device__ __forceinline__ T line_sum(T v, int Lw) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        if (off < Lw) v += __shfl_xor_sync(FULLM, v, off);
    return v;
}

template <typename T>
__device__ __forceinline__ void atomic_add4(typename Vec4<T>::type *p, T a, T b, T c, T d) {
    T *q = (T *)p;
    atomicAdd(q + 0, a);
    atomicAdd(q + 1, b);
    atomicAdd(q + 2, c);
    atomicAdd(q + 3, d);
}

}  // namespace

#ifndef SC_ADJOINT_MIN_BLOCKS
#define SC_ADJOINT_MIN_BLOCKS 4  // FP32: 4 blocks of 128 threads per SM (at most 128 registers)
#endif

template <typename T, int EPT, bool RET>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? SC_ADJOINT_MIN_BLOCKS : 1) adjoint_sweep_kernel(AdjointLaunch a) {
    // parked per (sample, energy): 0 = gamma then beta, 1 = local beta cotangent,
    // 2 (retarded) = gamma cotangent handed to the mirror energy's lane
    constexpr int NS = RET ? 3 : 2;
    typedef typename Vec4<T>::type T4;
    typedef Cx<T> C;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    C *const warp_slab = (C *)a.scratch + wid * a.scratch_stride;
    const GrainSweep &gs = *a.grain;
    const int Lw = gs.lanes, G = gs.lines_per_warp;
    const int gi = lane / Lw, r = lane - gi * Lw;
    const T4 *__restrict__ img = (const T4 *)gs.image_in;
    const T4 *__restrict__ wimg = (const T4 *)a.wimg;
    T4 *__restrict__ gimg = (T4 *)a.gimg;
    const C *__restrict__ exit_prev = (const C *)gs.exits[a.parity];
    const T h = (T)gs.h;
    const int n_e = gs.n_e, ne_pad = gs.ne_pad;
    C *slab = warp_slab + (int64_t)gi * gs.max_ns * NS * ne_pad;
    const T pi = T(3.141592653589793);

    T zr0[EPT], zi[EPT];
    int nid[EPT], mir[EPT];
    bool ev[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int n = r + Lw * e;
        ev[e] = n < n_e;
        nid[e] = ev[e] ? n : n_e - 1;
        if (RET) {
            zr0[e] = (T)gs.energies[nid[e]];
            zi[e] = (T)gs.broadening;
            mir[e] = n_e - 1 - nid[e];
        } else {
            zr0[e] = T(0);
            zi[e] = (T)(gs.t * (nid[e] + 0.5));
            mir[e] = nid[e];
        }
    }
    const T *__restrict__ wl = (const T *)a.wimg;  // retarded: n_e weights per slot

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1);
        item = __shfl_sync(FULLM, item, 0);
        if (item >= a.n_items) break;
        const int2 it = a.items[item];
        const int L = gs.groups[(int64_t)it.y * G + gi];
        const bool lv = L >= 0;
        const LineDev &ln = gs.lines[lv ? L : 0];
        const int ns = lv ? ln.ns : 0;  // lines without samples do not enter the loss
        const int nsl = ns > 0 ? ns : 1;
        const int nsteps = ns > 0 ? ns + 1 : 0;
        int nmax = nsteps;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nmax = max(nmax, __shfl_xor_sync(FULLM, nmax, off));
        if (nmax == 0) continue;
        const T lead = (T)ln.lead, tail = (T)ln.tail;
        const int slot0 = ln.slot0;
        const T4 *li = img + slot0;
        auto park = [&](int i, int k, int e) -> C & { return slab[((int64_t)i * NS + k) * ne_pad + r + Lw * e]; };
        auto parkn = [&](int i, int k, int n) -> C & { return slab[((int64_t)i * NS + k) * ne_pad + n]; };

        // ---------------- pass 1: gamma along +e_par ----------------
        C g[EPT], g0[EPT];
        T4 sp = li[0];
        if (a.first_sweep) {
            const T d2 = sp.x * sp.x + sp.y * sp.y;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                StepCoef<T> c;
                step_coef<T>(sp.x, sp.y, d2, zr0[e] + sp.z, zi[e], lead, c);
                g[e] = c.gh;
            }
        } else {
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                T gx = 0, gy = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const C v = exit_prev[(int64_t)ln.tap_f[q] * n_e + nid[e]];
                    gx += (T)ln.w_f[q] * v.x;
                    gy += (T)ln.w_f[q] * v.y;
                }
                g[e] = C{gx, gy};
            }
        }
#pragma unroll
        for (int e = 0; e < EPT; ++e) g0[e] = g[e];
        {
            T4 sq = sp;
            for (int i = 0; i < nsteps; ++i) {
                const T dr = T(0.5) * (sp.x + sq.x), di = T(0.5) * (sp.y + sq.y), av = T(0.5) * (sp.z + sq.z);
                const T ell = (i == 0) ? lead : (i == ns ? tail : h);
                const T d2 = dr * dr + di * di;
#pragma unroll
                for (int e = 0; e < EPT; ++e) {
                    StepCoef<T> c;
                    step_coef<T>(dr, di, d2, zr0[e] + av, zi[e], ell, c);
                    step_apply<T>(c, g[e]);
                }
                if (i < ns) {
#pragma unroll
                    for (int e = 0; e < EPT; ++e) park(i, 0, e) = g[e];
                }
                sp = sq;
                sq = li[min(i + 1, nsl - 1)];
            }
        }
        __syncwarp();

        // ---------------- pass 2: beta along -e_par, gamma adjoint ----------------
        C b[EPT], b0[EPT], lam[EPT];
        T4 sh = li[nsl - 1];
        if (a.first_sweep) {
            const T d2 = sh.x * sh.x + sh.y * sh.y;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                StepCoef<T> c;
                step_coef<T>(sh.x, sh.y, d2, zr0[e] - sh.z, zi[e], tail, c);
                b[e] = c.gh;
            }
        } else {
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                T gx = 0, gy = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const C v = exit_prev[(int64_t)ln.tap_b[q] * n_e + nid[e]];
                    gx += (T)ln.w_b[q] * v.x;
                    gy += (T)ln.w_b[q] * v.y;
                }
                b[e] = C{gx, gy};
            }
        }
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            b0[e] = b[e];
            lam[e] = C{T(0), T(0)};
        }
        {
            T4 slo = sh;
            for (int j = 0; j < nmax; ++j) {
                const bool act = j < nsteps;
                const int q = nsl - 1 - j;  // sample reached (j < ns)
                const bool at_sample = act && j < ns;
                // the next step's parked gammas (written long ago) are fetched into L2
                if (j + 1 < ns) {
#pragma unroll
                    for (int e = 0; e < EPT; ++e) prefetch_l2(&park(q - 1, 0, e));
                }
                T cdr = 0, cdi = 0, ca = 0, sdr = 0, sdi = 0;
                if (act) {
                    const T dr = T(0.5) * (sh.x + slo.x), di = T(0.5) * (sh.y + slo.y), av = T(0.5) * (sh.z + slo.z);
                    const T ell = (j == 0) ? tail : (j == ns ? lead : h);
                    const T d2 = dr * dr + di * di;
                    T4 W = {};
                    if (!RET && at_sample) W = wimg[slot0 + q];
                    const C Wf{W.x, W.y};
#pragma unroll
                    for (int e = 0; e < EPT; ++e) {
                        // the forward segment with the same samples, and the beta step
                        // across it (angle p + P: a -> -a); for Matsubara energies the
                        // two share Omega, E and c2 up to complex conjugation
                        MobCoef<T> cf, cb;
                        mob_coef<T>(dr, di, d2, zr0[e] + av, zi[e], ell, cf);
                        if (RET)
                            mob_coef<T>(dr, di, d2, zr0[e] - av, zi[e], ell, cb);
                        else
                            mob_coef_mirror<T>(cf, dr, di, -av, zi[e], cb);
                        b[e] = mob_apply<T>(cb, b[e]);
                        // forward segment differentiated at its start
                        const C start = at_sample ? park(q, 0, e) : g0[e];
                        StepGrad<T> Gd;
                        mob_grad<T>(cf, dr, di, zr0[e] + av, zi[e], ell, start, Gd);
                        if (ev[e]) {
                            const C l = lam[e];
                            const C t1 = cmul(cconj(Gd.dR), l), t2 = cmul(Gd.dP, cconj(l));
                            cdr += t1.x + t2.x;
                            cdi += t1.y + t2.y;
                            ca += cmul(cconj(Gd.dQ), l).x;
                        }
                        C lnew = cmul(cconj(Gd.dg), lam[e]);
                        if (!RET && at_sample && ev[e]) {
                            const C gf = start, bt = b[e];
                            // D = 1 + gamma conj(beta)
                            const C Dd{T(1) + gf.x * bt.x + gf.y * bt.y, gf.y * bt.x - gf.x * bt.y};
                            const C iD = crcp(Dd);
                            const C iD2 = cmul(iD, iD), iDc2 = cconj(iD2);
                            const C Wc = cconj(Wf);
                            const C Ds{slo.x, slo.y};
                            // local cotangents of the sample's energy sums
                            const C ga = cmul(cmuli(cscale(iDc2, T(2) * pi)), cadd(Wf, cmul(cmul(bt, bt), Wc)));
                            const C gb2 = cmul(cmuli(cscale(iDc2, T(-4) * pi * W.z)), bt);
                            const C gcF = cmuli(cscale(Ds, T(2) * W.w));
                            const C gbar = cadd(cadd(ga, gb2), gcF);
                            const C ba = cmul(cmuli(cscale(iD2, T(2) * pi)), cadd(Wf, cmul(cmul(gf, gf), Wc)));
                            const C bb2 = cmul(cmuli(cscale(iD2, T(4) * pi * W.z)), gf);
                            const C bbar = cadd(cadd(ba, bb2), gcF);
                            lnew = cadd(lnew, gbar);
                            // direct dependence of S_F on the sample value: -2 i wF (gamma + beta)
                            const C sF = cmuli(cscale(cadd(gf, bt), T(-2) * W.w));
                            sdr += sF.x;
                            sdi += sF.y;
                            park(q, 1, e) = bbar;
                        } else if (!RET && at_sample) {
                            park(q, 1, e) = C{T(0), T(0)};
                        }
                        lam[e] = lnew;
                    }
                    if (RET && at_sample) {
                        // LDOS value of this lane's energy n: 2 Re(1/D) - 1 with
                        // D = 1 + gamma_f(mirror n) conj(beta_n); the gamma cotangent
                        // belongs to the forward chain of the mirror energy
#pragma unroll
                        for (int e = 0; e < EPT; ++e) {
                            C gbar{T(0), T(0)}, bbar{T(0), T(0)};
                            if (ev[e]) {
                                const T Wv = wl[(int64_t)(slot0 + q) * n_e + nid[e]];
                                const C gf = parkn(q, 0, mir[e]), bt = b[e];
                                const C Dd{T(1) + gf.x * bt.x + gf.y * bt.y, gf.y * bt.x - gf.x * bt.y};
                                const C iD = crcp(Dd);
                                const C iD2 = cmul(iD, iD);
                                gbar = cscale(cmul(cconj(iD2), bt), T(-2) * Wv);
                                bbar = cscale(cmul(iD2, gf), T(-2) * Wv);
                            }
                            if (ev[e]) parkn(q, 2, mir[e]) = gbar;  // each valid energy has one partner
                            park(q, 1, e) = bbar;
                        }
                    }
                }
                if (RET) {
                    __syncwarp();
                    if (at_sample) {
#pragma unroll
                        for (int e = 0; e < EPT; ++e) {
                            if (ev[e]) lam[e] = cadd(lam[e], park(q, 2, e));
                        }
                    }
                    __syncwarp();
                }
                if (at_sample) {
#pragma unroll
                    for (int e = 0; e < EPT; ++e) park(q, 0, e) = b[e];
                }
                cdr = line_sum(cdr, Lw);
                cdi = line_sum(cdi, Lw);
                ca = line_sum(ca, Lw);
                sdr = line_sum(sdr, Lw);
                sdi = line_sum(sdi, Lw);
                if (act && r == 0) {
                    const int hi = min(ns - j, ns - 1), lo = max(ns - 1 - j, 0);
                    T4 *ph = gimg + slot0 + hi;
                    T4 *pl = gimg + slot0 + lo;
                    atomicAdd(&ph->x, T(0.5) * cdr);
                    atomicAdd(&ph->y, T(0.5) * cdi);
                    atomicAdd(&ph->z, T(0.5) * ca);
                    atomicAdd(&pl->x, T(0.5) * cdr + (at_sample ? sdr : T(0)));
                    atomicAdd(&pl->y, T(0.5) * cdi + (at_sample ? sdi : T(0)));
                    atomicAdd(&pl->z, T(0.5) * ca);
                }
                if (act) {
                    sh = slo;
                    slo = li[max(nsl - 2 - j, 0)];
                }
            }
        }
        __syncwarp();

        // ---------------- pass 3: beta adjoint along +e_par ----------------
        C mu[EPT];
        {
            T4 sa = li[0], sb = li[0];
            for (int i = 0; i < nmax; ++i) {
                const bool act = i < nsteps;
                T cdr = 0, cdi = 0, ca = 0;
                // the next step's parked beta and beta cotangent are fetched into L2
                if (i + 1 < ns) {
#pragma unroll
                    for (int e = 0; e < EPT; ++e) {
                        prefetch_l2(&park(i + 1, 0, e));
                        prefetch_l2(&park(i + 1, 1, e));
                    }
                }
                if (act) {
                    if (i == 0) {
#pragma unroll
                        for (int e = 0; e < EPT; ++e) mu[e] = park(0, 1, e);
                    } else {
                        const T dr = T(0.5) * (sa.x + sb.x), di = T(0.5) * (sa.y + sb.y), av = T(0.5) * (sa.z + sb.z);
                        const T ell = (i == ns) ? tail : h;
                        const T d2 = dr * dr + di * di;
#pragma unroll
                        for (int e = 0; e < EPT; ++e) {
                            const C start = i < ns ? park(i, 0, e) : b0[e];
                            MobCoef<T> cb;
                            mob_coef<T>(dr, di, d2, zr0[e] - av, zi[e], ell, cb);
                            StepGrad<T> Gd;
                            mob_grad<T>(cb, dr, di, zr0[e] - av, zi[e], ell, start, Gd);
                            if (ev[e]) {
                                const C m = mu[e];
                                const C t1 = cmul(cconj(Gd.dR), m), t2 = cmul(Gd.dP, cconj(m));
                                cdr += t1.x + t2.x;
                                cdi += t1.y + t2.y;
                                ca -= cmul(cconj(Gd.dQ), m).x;  // Q = z - a
                            }
                            C mnew = cmul(cconj(Gd.dg), mu[e]);
                            if (i < ns) mnew = cadd(mnew, park(i, 1, e));
                            mu[e] = mnew;
                        }
                    }
                }
                cdr = line_sum(cdr, Lw);
                cdi = line_sum(cdi, Lw);
                ca = line_sum(ca, Lw);
                if (act && i > 0 && r == 0) {
                    const int s0 = max(i - 1, 0), s1 = min(i, ns - 1);
                    T4 *p0 = gimg + slot0 + s0;
                    T4 *p1 = gimg + slot0 + s1;
                    atomicAdd(&p0->x, T(0.5) * cdr);
                    atomicAdd(&p0->y, T(0.5) * cdi);
                    atomicAdd(&p0->z, T(0.5) * ca);
                    atomicAdd(&p1->x, T(0.5) * cdr);
                    atomicAdd(&p1->y, T(0.5) * cdi);
                    atomicAdd(&p1->z, T(0.5) * ca);
                }
                if (act) {
                    sa = sb;
                    sb = li[min(i + 1, nsl - 1)];
                }
            }
        }
        __syncwarp();
    }
}

// cotangents of the outputs -> cotangents of the accumulators (and the direct
// Delta and A_ind terms of the free energy)
__global__ void adjoint_outputs_kernel(GridDev grid, const uint8_t *__restrict__ mask,
                                       const double *__restrict__ delta, const double *__restrict__ aind,
                                       double t, double normD, double kappa, double n_in,
                                       const double *__restrict__ gdn, const double *__restrict__ gj,
                                       const double *__restrict__ gF, double gFtot, double *__restrict__ gacc,
                                       double *__restrict__ gdelta, double *__restrict__ gaind) {
    const int nx = grid.nx, ny = grid.ny;
    const int64_t npts = (int64_t)nx * ny;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= npts) return;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    if (mask[idx]) {
        const double cd = t / (2.0 * 3.141592653589793) / normD;
        if (gdn) {
            a0 = cd * gdn[2 * idx];
            a1 = cd * gdn[2 * idx + 1];
        }
        if (gj) {
            const double cj = grid.charge_sign * t / 3.141592653589793;
            a2 = cj * gj[2 * idx];
            a3 = cj * gj[2 * idx + 1];
        }
        const double fb = (gF ? gF[idx] : 0.0) + gFtot / n_in;
        a4 = -0.5 * t * fb;
        // F = |Delta|^2 D + ...: direct term
        atomicAdd(&gdelta[2 * idx], 2.0 * normD * fb * delta[2 * idx]);
        atomicAdd(&gdelta[2 * idx + 1], 2.0 * normD * fb * delta[2 * idx + 1]);
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
    const double fi = (double)(idx % grid.nx), fj = (double)(idx / grid.nx);
    for (int p = 0; p < n_pairs; ++p) {
        const PairDev pp = pairs[p];
        const double ws = pp.wa + pp.wb;
        const double wf0 = ws * pp.eta * g0, wf1 = ws * pp.eta * g1;
        const double wg = ws * (pp.ex * g2 + pp.ey * g3), wF = ws * g4;
        const double u = fma(fi, -pp.ey, fma(fj, pp.ex, pp.u0));
        const double v = fma(fi, pp.ex, fma(fj, pp.ey, pp.v0));
        const double fu = floor(u), fv = floor(v);
        const int iu = (int)fu, iv = (int)fv;
        const double wu = u - fu, wv = v - fv;
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const int l = min(max(iu + bb, pp.l_lo), pp.l_hi);
            const BackLine Ln = bl[pp.line0 + (l - pp.l_lo)];
            const double wl = bb ? wu : 1.0 - wu;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int m = min(max(iv + c, Ln.m0), Ln.m0 + Ln.ns - 1);
                const double w = wl * (c ? wv : 1.0 - wv);
                if (w == 0.0) continue;
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
            const BackLine Ln = bl[pp.line0 + (l - pp.l_lo)];
            const double wlin = bb ? wu : 1.0 - wu;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int m = min(max(iv + c, Ln.m0), Ln.m0 + Ln.ns - 1);
                const double w = wlin * (c ? wv : 1.0 - wv);
                if (w == 0.0) continue;
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
    const LineGeo lg = geo[slot_line[s]];
    if (lg.ns == 0) return;  // no sample, no cotangent
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
            if (gaind) {
                atomicAdd(&gaind[2 * (int64_t)src], w * sa * pp.ex);
                atomicAdd(&gaind[2 * (int64_t)src + 1], w * sa * pp.ey);
            }
        }
}

template <typename T, bool RET>
static cudaError_t adjoint_dispatch(const AdjointLaunch &a, cudaStream_t st) {
    dim3 grid(a.grid_blocks), block(a.block_threads);
    switch (a.energies_per_lane) {
#define SC_CASE(E) \
    case E: adjoint_sweep_kernel<T, E, RET><<<grid, block, 0, st>>>(a); break;
        SC_CASE(1) SC_CASE(2) SC_CASE(3) SC_CASE(4) SC_CASE(5) SC_CASE(6) SC_CASE(7) SC_CASE(8)
#undef SC_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_sweep(bool fp64, const AdjointLaunch &a, cudaStream_t st) {
    if (a.retarded) return fp64 ? adjoint_dispatch<double, true>(a, st) : adjoint_dispatch<float, true>(a, st);
    return fp64 ? adjoint_dispatch<double, false>(a, st) : adjoint_dispatch<float, false>(a, st);
}

int adjoint_occupancy(bool fp64, int ept, int bs) {
    int n = 0;
    switch (ept) {
#define SC_CASE(E)                                                                                        \
    case E:                                                                                               \
        if (fp64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adjoint_sweep_kernel<double, E, true>, bs, 0); \
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adjoint_sweep_kernel<float, E, true>, bs, 0);       \
        break;
        SC_CASE(1) SC_CASE(2) SC_CASE(3) SC_CASE(4) SC_CASE(5) SC_CASE(6) SC_CASE(7) SC_CASE(8)
#undef SC_CASE
        default: n = 0;
    }
    return n;
}

cudaError_t launch_adjoint_outputs(const GridDev &grid, const uint8_t *mask, const double *delta,
                                   const double *aind, double t, double normD, double kappa, double n_in,
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

}  // namespace scd
