// The adjoint sweep kernel (sm_103a), included by the per-precision units
// adjoint_f32.cu and adjoint_f64.cu, which instantiate it and define the
// launchers.  The method is described in adjoint.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "adjoint.cuh"
#include "adjoint_x2.cuh"
#include "bounds.cuh"
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


}  // namespace

#ifndef SC_ADJOINT_MIN_BLOCKS
#define SC_ADJOINT_MIN_BLOCKS 4  // FP32: 4 blocks of 128 threads per SM (at most 128 registers)
#endif

// BLK: the grain's energies are split into blocks; each item carries its block and
// the lane's energies are set up per item (once per launch otherwise).
template <typename T, int EPT, bool RET, int STEP, bool BLK = false, bool CK = false>
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
    const T *__restrict__ wl = (const T *)a.wimg;  // retarded: n_e weights per slot
    const int nb = BLK ? gs.n_blocks : 1;
    // the lane's energies from energy e0 on
    auto energies = [&](int e0) {
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int n = e0 + r + Lw * e;
            ev[e] = n < n_e;
            nid[e] = ev[e] ? n : n_e - 1;
            if (RET) {
                zr0[e] = (T)gs.energies[nid[e]];
                zi[e] = (T)gs.broadening;
                mir[e] = n_e - 1 - nid[e];
            } else {
                zr0[e] = T(0);
                zi[e] = gs.mats_eps ? (T)gs.mats_eps[nid[e]] : (T)(gs.t * (nid[e] + 0.5));
                mir[e] = nid[e];
            }
        }
    };
    if constexpr (!BLK) energies(0);

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1);
        item = __shfl_sync(FULLM, item, 0);
        if (item >= a.n_items) break;
        const int2 it = a.items[item];
        if constexpr (sizeof(T) == 4 && !RET && STEP == 0) {
            // FP32 closed-form Matsubara/Ozaki adjoint: packed energy pairs
            adjoint_item_x2<EPT, BLK, CK>(a, it, gs, (Cx<float> *)warp_slab, lane);
            continue;
        }
        // line group and energy block of this item (one block unless the energies
        // exceed one lane layout)
        const int grp = BLK ? it.y / nb : it.y;
        if constexpr (BLK) energies((it.y - grp * nb) * ne_pad);
        const int64_t gq = (int64_t)grp * G + gi;
        int L = in_bounds(gq, (int64_t)gs.n_groups * G) ? gs.groups[gq] : -1;
        if (L >= 0 && !in_bounds(L, gs.n_lines)) L = -1;
        const LineDev &ln = gs.lines[L >= 0 ? L : 0];
        const bool lv = L >= 0 && line_tables_ok(ln, gs.n_slots, gs.n_lines, !a.first_sweep,
                                                 (int64_t)(slab - (C *)a.scratch), NS * ne_pad, a.scratch_elems);
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
                if constexpr (STEP == 0) {
                    const T d2 = dr * dr + di * di;
#pragma unroll
                    for (int e = 0; e < EPT; ++e) {
                        StepCoef<T> c;
                        step_coef<T>(dr, di, d2, zr0[e] + av, zi[e], ell, c);
                        step_apply<T>(c, g[e]);
                    }
                } else {
                    const MidSeg<T> ms = mid_seg<T>(dr, di, ell);
#pragma unroll
                    for (int e = 0; e < EPT; ++e) g[e] = midpoint_step<T>(ms, zr0[e] + av, zi[e], g[e]);
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
                        const C start = at_sample ? park(q, 0, e) : g0[e];
                        StepGrad<T> Gd;
                        if constexpr (STEP == 0) {
                            MobCoef<T> cf, cb;
                            mob_coef<T>(dr, di, d2, zr0[e] + av, zi[e], ell, cf);
                            if (RET)
                                mob_coef<T>(dr, di, d2, zr0[e] - av, zi[e], ell, cb);
                            else
                                mob_coef_mirror<T>(cf, dr, di, -av, zi[e], cb);
                            b[e] = mob_apply<T>(cb, b[e]);
                            // forward segment differentiated at its start
                            mob_grad<T>(cf, dr, di, zr0[e] + av, zi[e], ell, start, Gd);
                        } else {
                            const MidSeg<T> ms = mid_seg<T>(dr, di, ell);
                            b[e] = midpoint_step<T>(ms, zr0[e] - av, zi[e], b[e]);
                            midpoint_grad<T>(ms, dr, di, zr0[e] + av, zi[e], start, Gd);
                        }
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
                            C bbar = cadd(cadd(ba, bb2), gcF);
                            // weighted energy sums (Ozaki's poles): every term of energy n
                            // carries its weight
                            const T wn = gs.mats_w ? (T)gs.mats_w[nid[e]] : T(1);
                            lnew = cadd(lnew, cscale(gbar, wn));
                            bbar = cscale(bbar, wn);
                            // direct dependence of S_F on the sample value: -2 i wF (gamma + beta)
                            const C sF = cmuli(cscale(cadd(gf, bt), T(-2) * W.w * wn));
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
                            StepGrad<T> Gd;
                            if constexpr (STEP == 0) {
                                MobCoef<T> cb;
                                mob_coef<T>(dr, di, d2, zr0[e] - av, zi[e], ell, cb);
                                mob_grad<T>(cb, dr, di, zr0[e] - av, zi[e], ell, start, Gd);
                            } else {
                                midpoint_grad<T>(mid_seg<T>(dr, di, ell), dr, di, zr0[e] - av, zi[e], start, Gd);
                            }
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

template <typename T, bool RET, int STEP, bool BLK = false, bool CK = false>
static cudaError_t adjoint_dispatch(const AdjointLaunch &a, cudaStream_t st) {
    dim3 grid(a.grid_blocks), block(a.block_threads);
    switch (a.energies_per_lane) {
#define SC_CASE(E) \
    case E: adjoint_sweep_kernel<T, E, RET, STEP, BLK, CK><<<grid, block, 0, st>>>(a); break;
        SC_CASE(1) SC_CASE(2) SC_CASE(3) SC_CASE(4) SC_CASE(5) SC_CASE(6) SC_CASE(7) SC_CASE(8)
#undef SC_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t adjoint_launch_t(const AdjointLaunch &a, cudaStream_t st) {
    if (a.retarded && a.blocked) return cudaErrorInvalidValue;  // the LDOS keeps one energy block
    if (a.stepper == 1) {
        if (a.retarded) return adjoint_dispatch<T, true, 1>(a, st);
        return a.blocked ? adjoint_dispatch<T, false, 1, true>(a, st) : adjoint_dispatch<T, false, 1>(a, st);
    }
    if (a.stepper != 0) return cudaErrorInvalidValue;
    if (a.ckpt > 0) {  // kept-and-recomputed forward gammas: FP32 Matsubara/Ozaki adjoint only
        if constexpr (sizeof(T) == 4) {
            if (a.retarded) return cudaErrorInvalidValue;
            return a.blocked ? adjoint_dispatch<T, false, 0, true, true>(a, st)
                             : adjoint_dispatch<T, false, 0, false, true>(a, st);
        }
        return cudaErrorInvalidValue;
    }
    if (a.retarded) return adjoint_dispatch<T, true, 0>(a, st);
    return a.blocked ? adjoint_dispatch<T, false, 0, true>(a, st) : adjoint_dispatch<T, false, 0>(a, st);
}

// blocks per SM of the retarded instantiation (the larger one) bound both
template <typename T>
static int adjoint_occupancy_t(int ept, int bs, int stepper) {
    int n = 0;
    switch (ept) {
#define SC_CASE(E)                                                                                  \
    case E:                                                                                         \
        if (stepper == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adjoint_sweep_kernel<T, E, true, 1>, bs, 0); \
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adjoint_sweep_kernel<T, E, true, 0>, bs, 0);              \
        break;
        SC_CASE(1) SC_CASE(2) SC_CASE(3) SC_CASE(4) SC_CASE(5) SC_CASE(6) SC_CASE(7) SC_CASE(8)
#undef SC_CASE
        default: n = 0;
    }
    return n;
}

}  // namespace scd
