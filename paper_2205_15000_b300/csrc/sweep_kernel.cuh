// The Riccati sweep kernel (sm_103a), included by the per-precision units
// sweep_f32.cu and sweep_f64.cu, which instantiate it and define the launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "lattice_f32.cuh"
#include "riccati_step.cuh"
#include "sweep_x2.cuh"

namespace scd {

#ifndef FULL_MASK
#define FULL_MASK 0xffffffffu
#endif

// ---------------------------------------------------------------------------
// The sweep.  A warp owns G = 32 / Lw lines of one work item; each line gets Lw
// lanes and each lane EPT energies (n = lane_in_line + Lw * e).  Persistent:
// warps take items (longest lines first) from an atomic counter.
//
// Forward pass: gamma of angle p from smin to smax; gamma at every sample is
// parked in the warp's scratch slab ([line][sample][energy]).
// Backward pass: gamma of angle p + P from smax to smin; at each sample the
// parked gamma and the new one give the propagator of both angles
// (gamma~(p) = conj gamma(p + P), Eq. symmetries), summed over the lane's
// energies and then over the line's lanes by shuffles.
// ---------------------------------------------------------------------------
#ifndef SC_SWEEP_MIN_BLOCKS
#define SC_SWEEP_MIN_BLOCKS 5  // FP32: 5 blocks of 128 threads per SM (at most 102 registers)
#endif
#ifndef SC_SWEEP_MIN_BLOCKS_MID
#define SC_SWEEP_MIN_BLOCKS_MID 5  // FP32 implicit-midpoint instantiations
#endif

// One work item: the G lines of group it.y of grain gs, EPT energies per lane;
// STEP 0 = closed-form step, 1 = implicit midpoint rule; WGT: weighted energy
// sums (Ozaki's poles) in the Matsubara mode; BLK: the launch holds a grain whose
// energies are split into blocks (item y of a grain is line group y / n_blocks
// with energy block y % n_blocks, whose sample sums go to that block's own image;
// a grain of one block is swept as without BLK).
template <typename T, int EPT, bool RET, int STEP, bool WGT, bool BLK>
__device__ __forceinline__ void sweep_item(const SweepLaunch &a, const int2 it, const GrainSweep &gs,
                                           Cx<T> *const warp_slab, const int lane) {
    typedef typename Vec4<T>::type T4;
    typedef Cx<T> C;
    {
        const int Lw = gs.lanes, G = gs.lines_per_warp;
        const int gi = lane / Lw, r = lane - gi * Lw;
        const T4 *__restrict__ img = (const T4 *)gs.image_in;
        const C *__restrict__ exit_prev = (const C *)gs.exits[a.parity];
        C *__restrict__ exit_cur = (C *)gs.exits[a.parity ^ 1];
        C *slab = warp_slab + (int64_t)gi * gs.max_ns * gs.ne_pad;
        const T h = (T)gs.h;
        const int n_e = gs.n_e;
        const int ne_pad = gs.ne_pad;
        // energy block of this item (several when the energies exceed one lane layout)
        const int nb = BLK ? gs.n_blocks : 1;
        const int grp = BLK ? it.y / nb : it.y;
        // this item's energies: the grain's part [e_first, e_end), its block of ne_pad
        const int e_end = gs.e_count > 0 ? gs.e_first + gs.e_count : n_e;
        const int e0 = gs.e_first + (BLK ? (it.y - grp * nb) * ne_pad : 0);

        // the lane's energies: z = zr0 + i zi (+ a along the line)
        T zr0[EPT], zi[EPT];
        T wv[WGT ? EPT : 1];  // weights of the lane's energies (WGT)
        int nid[EPT], mir[EPT];
        bool ev[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int n = e0 + r + Lw * e;
            ev[e] = n < e_end;
            const int nn = ev[e] ? n : e_end - 1;
            nid[e] = nn;
            if (RET) {
                zr0[e] = (T)gs.energies[nn];
                zi[e] = (T)gs.broadening;
                mir[e] = n_e - 1 - nn;
            } else {
                zr0[e] = T(0);
                // Ozaki's poles (WGT) come with their energies; Matsubara energies are t (n + 1/2)
                zi[e] = WGT ? (T)gs.mats_eps[nn] : (T)(gs.t * (nn + 0.5));
                mir[e] = nn;
                if constexpr (WGT) wv[e] = ev[e] ? (T)gs.mats_w[nn] : T(0);
            }
        }
        const int64_t gq = (int64_t)grp * G + gi;
        int L = in_bounds(gq, (int64_t)gs.n_groups * G) ? gs.groups[gq] : -1;
        if (L >= 0 && !in_bounds(L, gs.n_lines)) L = -1;
        const LineDev &ln = gs.lines[L >= 0 ? L : 0];
        const bool lv = L >= 0 && line_tables_ok(ln, gs.n_slots, gs.n_lines, !a.first_sweep,
                                                 (int64_t)(slab - (C *)a.scratch), ne_pad, a.scratch_elems);
        const int ns = lv ? ln.ns : 0;
        const int nsl = ns > 0 ? ns : 1;
        const int nsteps = lv ? ns + 1 : 0;
        int nmax = nsteps;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nmax = max(nmax, __shfl_xor_sync(FULL_MASK, nmax, off));
        const T lead = (T)ln.lead, tail = (T)ln.tail;
        const int slot0 = ln.slot0;
        const T4 *li = img + slot0;

        // ---------------- forward: angle p, along +e_par ----------------
        C g[EPT];
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
                    const T w = (T)ln.w_f[q];
                    gx += w * v.x;
                    gy += w * v.y;
                }
                g[e].x = gx;
                g[e].y = gy;
            }
        }
        // segment i joins samples max(i-1, 0) and min(i, nsl-1); the end segments
        // (i = 0 and i = ns) see a single sample
        T4 sq = sp;                      // s[min(i, nsl-1)]
        T4 sn = li[min(1, nsl - 1)];     // s[min(i+1, nsl-1)], prefetched
        for (int i = 0; i < nsteps; ++i) {
            const T dr = T(0.5) * (sp.x + sq.x), di = T(0.5) * (sp.y + sq.y);
            const T av = T(0.5) * (sp.z + sq.z);
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
                C *dst = slab + (int64_t)i * ne_pad + r;
#pragma unroll
                for (int e = 0; e < EPT; ++e) dst[Lw * e] = g[e];
            }
            sp = sq;
            sq = sn;
            sn = li[min(i + 2, nsl - 1)];
        }
        if (lv) {
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (ev[e]) exit_cur[(int64_t)ln.exit_f * n_e + nid[e]] = g[e];
        }

        __syncwarp();  // parked gammas of other lanes are read in retarded mode

        // ---------------- backward: angle p + P, along -e_par ----------------
        // (a -> -a; samples visited nsl-1 ... 0)
        T4 sh = li[nsl - 1];
        if (a.first_sweep) {
            const T d2 = sh.x * sh.x + sh.y * sh.y;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                StepCoef<T> c;
                step_coef<T>(sh.x, sh.y, d2, zr0[e] - sh.z, zi[e], tail, c);
                g[e] = c.gh;
            }
        } else {
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                T gx = 0, gy = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const C v = exit_prev[(int64_t)ln.tap_b[q] * n_e + nid[e]];
                    const T w = (T)ln.w_b[q];
                    gx += w * v.x;
                    gy += w * v.y;
                }
                g[e].x = gx;
                g[e].y = gy;
            }
        }
        // backward segment j joins samples min(nsl-j, nsl-1) and max(nsl-1-j, 0)
        T4 slo = sh;                     // s[max(nsl-1-j, 0)] = sample reached (j < ns)
        T4 snb = li[max(nsl - 2, 0)];    // prefetched s[max(nsl-2-j, 0)]
        for (int j = 0; j < nmax; ++j) {
            const bool act = j < nsteps;
            const int qs = nsl - 1 - j;          // sample reached after this step
            const bool comb = act && j < ns;     // a sample to combine at
            C gf[EPT];
            if (comb) {
                const C *src = slab + (int64_t)qs * ne_pad;
#pragma unroll
                for (int e = 0; e < EPT; ++e) gf[e] = src[RET ? mir[e] : (r + Lw * e)];
            }
            if (act) {
                const T dr = T(0.5) * (sh.x + slo.x), di = T(0.5) * (sh.y + slo.y);
                const T av = T(0.5) * (sh.z + slo.z);
                const T ell = (j == 0) ? tail : (j == ns ? lead : h);
                if constexpr (STEP == 0) {
                    const T d2 = dr * dr + di * di;
#pragma unroll
                    for (int e = 0; e < EPT; ++e) {
                        StepCoef<T> c;
                        step_coef<T>(dr, di, d2, zr0[e] - av, zi[e], ell, c);
                        step_apply<T>(c, g[e]);
                    }
                } else {
                    const MidSeg<T> ms = mid_seg<T>(dr, di, ell);
#pragma unroll
                    for (int e = 0; e < EPT; ++e) g[e] = midpoint_step<T>(ms, zr0[e] - av, zi[e], g[e]);
                }
            }
            if (!RET) {
                // propagator of angle p from gamma = gf, gamma~ = conj(g):
                //   D = 1 + gf conj(g);  f + conj f~ = -2 i pi (gf/D + g/conj D)
                //   2 Re g = 4 pi Im(1/D);  2 Re I = 2 Im(conj(Delta)(gf + g))
                T sfr = 0, sfi = 0, sg = 0, sFr = 0, sFi = 0;
                if (comb) {
#pragma unroll
                    for (int e = 0; e < EPT; ++e) {
                        if (!ev[e]) continue;
                        const C gb = g[e], ga = gf[e];
                        const T pr = ga.x * gb.x + ga.y * gb.y;   // ga * conj(gb)
                        const T pi_ = ga.y * gb.x - ga.x * gb.y;
                        const T Dr = T(1) + pr, Di = pi_;
                        const T rD = Mth<T>::rcp(Dr * Dr + Di * Di);
                        const T ir = Dr * rD, ii = -Di * rD;      // 1/D
                        // ga/D + gb conj(1/D)
                        if constexpr (WGT) {
                            const T w = wv[e];
                            sg += w * ii;
                            sfr += w * ((ga.x * ir - ga.y * ii) + (gb.x * ir + gb.y * ii));
                            sfi += w * ((ga.x * ii + ga.y * ir) + (gb.y * ir - gb.x * ii));
                            sFr += w * (ga.x + gb.x);
                            sFi += w * (ga.y + gb.y);
                        } else {
                            sg += ii;
                            sfr += (ga.x * ir - ga.y * ii) + (gb.x * ir + gb.y * ii);
                            sfi += (ga.x * ii + ga.y * ir) + (gb.y * ir - gb.x * ii);
                            sFr += ga.x + gb.x;
                            sFi += ga.y + gb.y;
                        }
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    if (off >= Lw) continue;
                    sfr += __shfl_xor_sync(FULL_MASK, sfr, off);
                    sfi += __shfl_xor_sync(FULL_MASK, sfi, off);
                    sg += __shfl_xor_sync(FULL_MASK, sg, off);
                    sFr += __shfl_xor_sync(FULL_MASK, sFr, off);
                    sFi += __shfl_xor_sync(FULL_MASK, sFi, off);
                }
                if (comb && r == 0) {
                    const T twopi = T(6.283185307179586), fourpi = T(12.566370614359172);
                    T4 o;
                    o.x = twopi * sfi;                          // Re Sf
                    o.y = -twopi * sfr;                         // Im Sf
                    o.z = fourpi * sg;                          // Sg
                    o.w = T(2) * (slo.x * sFi - slo.y * sFr);   // SF
                    // a blocked sweep writes each energy block's sums into the block's own image
                    T4 *po = (T4 *)gs.image_out + (BLK ? (int64_t)(it.y - grp * nb) * gs.n_slots : 0) + slot0 + qs;
                    *po = o;
                }
            } else if (comb) {
                // LDOS: -Im g / pi = Re[(1 - p)/(1 + p)] = 2 Re(1/D) - 1
                T *outl = (T *)gs.image_out + (int64_t)(slot0 + qs) * n_e;
#pragma unroll
                for (int e = 0; e < EPT; ++e) {
                    if (!ev[e]) continue;
                    const C gb = g[e], ga = gf[e];
                    const T pr = ga.x * gb.x + ga.y * gb.y;
                    const T pi_ = ga.y * gb.x - ga.x * gb.y;
                    const T Dr = T(1) + pr, Di = pi_;
                    const T rD = Mth<T>::rcp(Dr * Dr + Di * Di);
                    outl[nid[e]] = T(2) * Dr * rD - T(1);
                }
            }
            if (act) {
                sh = slo;
                slo = snb;
                snb = li[max(nsl - 3 - j, 0)];
            }
        }
        if (lv) {
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (ev[e]) exit_cur[(int64_t)ln.exit_b * n_e + nid[e]] = g[e];
        }
        __syncwarp();  // the slab is rewritten by the next item
    }
}

// 9 or 10 energies per lane (FP32 Matsubara/Ozaki sweep on 16 or 32 lanes per
// line): 4 blocks per SM, 128 registers
#ifndef SC_SWEEP_MIN_BLOCKS_WIDE
#define SC_SWEEP_MIN_BLOCKS_WIDE 4
#endif

// A lattice transfer of another batch member as a work item of a sweep launch:
// the rotation of four of its lines, or the rotate-back of one of its tiles (the
// same arithmetic as the transfer kernels, so the same values).  A call, not
// inlined, so that the sweep's register allocation is its own.
static __device__ __noinline__ void side_item(const SweepLaunch &a, int64_t s, const int lane) {
    const int2 v = a.side[s];
    const int m = v.x >> 1;
    if (!in_bounds(m, a.n_side_members)) return;
    const MemberDev &M = a.side_members[m];
    if ((v.x & 1) == 0) {
        const int64_t L0 = 4 * (int64_t)v.y;
        if (L0 >= M.grid.n_lines) return;
        switch (M.grid.gauge) {
            case 2: rotate_f32_quad<2>(M.lines, L0, M.grid.n_lines, M.pairs, M.grid, M.ghost, M.pad0, M.padc, M.image_in, lane); break;
            case 1: rotate_f32_quad<1>(M.lines, L0, M.grid.n_lines, M.pairs, M.grid, M.ghost, M.pad0, M.padc, M.image_in, lane); break;
            default: rotate_f32_quad<0>(M.lines, L0, M.grid.n_lines, M.pairs, M.grid, M.ghost, M.pad0, M.padc, M.image_in, lane);
        }
    } else {
        rotate_back_f32_warp<1>(M.pairs, M.n_pairs, M.back, M.grid, M.mask, M.image_out, M.acc, v.y, lane);
    }
}

// SIDE: the launch also carries a.n_side lattice transfers (FP32 batch sweeps):
// counter value c is transfer s(c) when s(c + 1) > s(c), s(c) = floor(c n_side /
// (n_items + n_side)), else sweep item c - s(c), so the transfers are spread
// evenly over the sweep items, which keep their longest-first order.
template <typename T, int EPT, bool RET, int STEP, bool WGT, bool BLK = false, bool SIDE = false>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? (EPT > 8 ? SC_SWEEP_MIN_BLOCKS_WIDE
                                                                 : (STEP ? SC_SWEEP_MIN_BLOCKS_MID : SC_SWEEP_MIN_BLOCKS))
                                                      : 1)
    sweep_kernel(SweepLaunch a) {
    static_assert(!SIDE || (sizeof(T) == 4 && !RET && !BLK), "transfer items run in FP32 batch sweeps only");
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    Cx<T> *const warp_slab = (Cx<T> *)a.scratch + wid * a.scratch_stride;
    const int64_t n_side = SIDE ? (int64_t)a.n_side : 0;
    const int64_t total = (int64_t)a.n_items + n_side;
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(a.counter, 1);
        c = __shfl_sync(FULL_MASK, c, 0);
        if (c >= total) break;
        int item = c;
        if constexpr (SIDE) {
            const int64_t s0 = (int64_t)c * n_side / total, s1 = ((int64_t)c + 1) * n_side / total;
            if (s1 > s0) {
                side_item(a, s0, lane);
                continue;
            }
            item = c - (int)s0;
        }
        const int2 it = a.items[item];
        if (!in_bounds(it.x, a.n_grains)) continue;
        if constexpr (sizeof(T) == 4)  // FP32: packed energy pairs
            sweep_item_x2<EPT, RET, STEP, WGT, BLK>(a, it, a.grains[it.x], (Cx<float> *)warp_slab, lane);
        else
            sweep_item<T, EPT, RET, STEP, WGT, BLK>(a, it, a.grains[it.x], warp_slab, lane);
    }
}

template <typename T, bool RET, int STEP, bool WGT, bool BLK = false, bool SIDE = false>
static cudaError_t sweep_dispatch(const SweepLaunch &a, cudaStream_t st) {
    dim3 grid(a.grid_blocks), block(a.block_threads);
    switch (a.energies_per_lane) {
#define SC_CASE(E) \
    case E: sweep_kernel<T, E, RET, STEP, WGT, BLK, SIDE><<<grid, block, 0, st>>>(a); break;
        SC_CASE(1) SC_CASE(2) SC_CASE(3) SC_CASE(4) SC_CASE(5) SC_CASE(6) SC_CASE(7) SC_CASE(8)
        case 9:
        case 10:
            // the wide layouts exist for the FP32 sweep without energy blocks only
            if constexpr (sizeof(T) == 4 && !RET && !BLK) {
                if (a.energies_per_lane == 9) sweep_kernel<T, 9, RET, STEP, WGT, BLK, SIDE><<<grid, block, 0, st>>>(a);
                else sweep_kernel<T, 10, RET, STEP, WGT, BLK, SIDE><<<grid, block, 0, st>>>(a);
                break;
            } else {
                return cudaErrorInvalidValue;
            }
#undef SC_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T, int STEP>
static cudaError_t sweep_launch_s(const SweepLaunch &a, cudaStream_t st) {
    if (a.retarded) return sweep_dispatch<T, true, STEP, false>(a, st);
    if (a.blocked)
        return a.weighted ? sweep_dispatch<T, false, STEP, true, true>(a, st)
                          : sweep_dispatch<T, false, STEP, false, true>(a, st);
    return a.weighted ? sweep_dispatch<T, false, STEP, true>(a, st) : sweep_dispatch<T, false, STEP, false>(a, st);
}

template <typename T>
static cudaError_t sweep_launch_t(const SweepLaunch &a, cudaStream_t st) {
    if (a.stepper == 1) return sweep_launch_s<T, 1>(a, st);
    if (a.stepper != 0) return cudaErrorInvalidValue;
    return sweep_launch_s<T, 0>(a, st);
}

template <typename T, bool RET, int STEP, bool WGT, bool SIDE = false>
static int occ_dispatch(int ept, int bs) {
    int n = 0;
    switch (ept) {
#define SC_CASE(E) \
    case E: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, E, RET, STEP, WGT, false, SIDE>, bs, 0); break;
        SC_CASE(1) SC_CASE(2) SC_CASE(3) SC_CASE(4) SC_CASE(5) SC_CASE(6) SC_CASE(7) SC_CASE(8)
#undef SC_CASE
        case 9:
        case 10:
            if constexpr (sizeof(T) == 4 && !RET) {
                if (ept == 9) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, 9, RET, STEP, WGT, false, SIDE>, bs, 0);
                else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, 10, RET, STEP, WGT, false, SIDE>, bs, 0);
            } else {
                n = 0;
            }
            break;
        default: n = 0;
    }
    return n;
}

// blocks per SM: the smaller of the context's Matsubara instantiation (plain
// or weighted) and the retarded one (both launch with the same plan)
template <typename T>
static int sweep_occupancy_t(int ept, int bs, int stepper, bool weighted) {
    int a, b;
    if (ept > 8)  // the wide layouts have no retarded instantiation (the LDOS keeps at most 8)
        return stepper == 1 ? (weighted ? occ_dispatch<T, false, 1, true>(ept, bs) : occ_dispatch<T, false, 1, false>(ept, bs))
                            : (weighted ? occ_dispatch<T, false, 0, true>(ept, bs) : occ_dispatch<T, false, 0, false>(ept, bs));
    if (stepper == 1) {
        a = weighted ? occ_dispatch<T, false, 1, true>(ept, bs) : occ_dispatch<T, false, 1, false>(ept, bs);
        b = occ_dispatch<T, true, 1, false>(ept, bs);
    } else {
        a = weighted ? occ_dispatch<T, false, 0, true>(ept, bs) : occ_dispatch<T, false, 0, false>(ept, bs);
        b = occ_dispatch<T, true, 0, false>(ept, bs);
    }
    return a < b ? a : b;
}

}  // namespace scd
