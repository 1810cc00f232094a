// The FP32 closed-form Matsubara sweep on packed pairs of energies.  Every lane
// applies the same arithmetic to its EPT energies, so energies (2k, 2k+1) of a
// lane travel as one float2 through the step and the propagator sums with
// sm_100's two-wide FP32 instructions (fma/mul/add .f32x2): one issue slot per
// two lane-operations, which is what bounds the scalar kernel.  The transcendental
// unit instructions stay per energy; an odd EPT runs its last energy through the
// same formulation on single values.
//
// Arithmetic is that of step_coef / step_apply (App. C closed-form step) and of
// the propagator sums of the scalar sweep, rearranged for the packed form:
//   * for Matsubara energies z = zr + i eps with zr = +-a shared by the lane's
//     energies, Re Omega^2 = (|Delta|^2 - zr^2) + eps^2 and Im Omega^2 = -2 zr eps;
//   * u = |Omega^2| + |Re Omega^2| = 2 s^2 and one rsqrt of u give sqrt(2) s and
//     sqrt(2) y/(2s); the 1/sqrt(2) is folded into the per-segment constants;
//   * signs are carried (-Re K, E - 1, -Im 1/D) so that most complex products are
//     one multiply and one fused multiply-add.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bounds.cuh"
#include "kernels.cuh"
#include "riccati_step.cuh"

namespace scd {

#ifndef FULL_MASK
#define FULL_MASK 0xffffffffu
#endif

typedef float2 f2;

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ f2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ f2 pk2(float lo, float hi) { return make_float2(lo, hi); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 neg2(f2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ f2 rsqrt2(f2 v) { return make_float2(Mth<float>::rsqrt(v.x), Mth<float>::rsqrt(v.y)); }
__device__ __forceinline__ f2 rcp2(f2 v) { return make_float2(Mth<float>::rcp(v.x), Mth<float>::rcp(v.y)); }

// The same operations on one value: the odd last energy of a lane runs the same
// formulation as the pairs (templates below on V = f2 or float).
__device__ __forceinline__ float add2(float a, float b) { return a + b; }
__device__ __forceinline__ float sub2(float a, float b) { return a - b; }
__device__ __forceinline__ float mul2(float a, float b) { return a * b; }
__device__ __forceinline__ float fma2(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float neg2(float a) { return -a; }
__device__ __forceinline__ float rsqrt2(float v) { return Mth<float>::rsqrt(v); }
__device__ __forceinline__ float rcp2(float v) { return Mth<float>::rcp(v); }

template <typename V>
__device__ __forceinline__ V bcv(float v);
template <>
__device__ __forceinline__ f2 bcv<f2>(float v) { return bc2(v); }
template <>
__device__ __forceinline__ float bcv<float>(float v) { return v; }

__device__ __forceinline__ f2 absv(f2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float absv(float a) { return fabsf(a); }
__device__ __forceinline__ f2 ex2v(f2 a) { return make_float2(ex2_approx(a.x), ex2_approx(a.y)); }
__device__ __forceinline__ float ex2v(float a) { return ex2_approx(a); }
__device__ __forceinline__ void sincosv(float t, float &s, float &c) { Mth<float>::sincos_(t, &s, &c); }
__device__ __forceinline__ void sincosv(f2 t, f2 &s, f2 &c) {
    sincosv(t.x, s.x, c.x);
    sincosv(t.y, s.y, c.y);
}
// sqrt(2) times the principal square root (Re >= 0) of x + i y, from sq = sqrt(2) s
// and yq = sqrt(2) y/(2 s), s = sqrt((|x + i y| + |x|)/2)
__device__ __forceinline__ void principal(float x, float y, float sq, float yq, float &re, float &im) {
    re = x >= 0.f ? sq : fabsf(yq);
    im = x >= 0.f ? yq : copysignf(sq, y);
}
__device__ __forceinline__ void principal(f2 x, f2 y, f2 sq, f2 yq, f2 &re, f2 &im) {
    principal(x.x, y.x, sq.x, yq.x, re.x, im.x);
    principal(x.y, y.y, sq.y, yq.y, re.y, im.y);
}

// fetch the line of global memory holding p into L2 (a hint; no register result)
__device__ __forceinline__ void l2_hint(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

constexpr float kRs2 = 0.70710678118654752f;  // 1/sqrt(2)
constexpr float kLog2e = 1.4426950408889634f;

// Per-segment constants shared by the lane's energies: Delta = dr + i di, the
// segment length ell, and the part of z = zr + i zi that all energies share --
// the Doppler shift zr = +-a for Matsubara energies (zi = eps_n per energy), the
// broadening zi for the retarded sweep (zr = E_n +- a per energy).
template <typename V>
struct SegT {
    V c0;    // Matsubara: |Delta|^2 - zr^2; retarded: |Delta|^2 + zi^2
    V m2;    // Matsubara: -2 zr; retarded: -2 zi
    V zs;    // Matsubara: zr; retarded: zi
    V sh;    // retarded: the Doppler shift added to each energy
    V dr, di, ndr, ndi;
    V el;   // -2 ell log2(e) / sqrt(2): sqrt(2) Re Omega -> log2 |E|
    V ntl;  // -2 ell / sqrt(2): sqrt(2) Im Omega -> arg E
};
typedef SegT<f2> Seg2;

template <bool RET, typename V = f2>
__device__ __forceinline__ SegT<V> seg2(float dr, float di, float shift, float broad, float ell) {
    SegT<V> s;
    const float d2 = dr * dr + di * di;
    const float zs = RET ? broad : shift;
    s.c0 = bcv<V>(RET ? d2 + zs * zs : d2 - zs * zs);
    s.m2 = bcv<V>(-2.f * zs);
    s.zs = bcv<V>(zs);
    s.sh = bcv<V>(shift);
    s.dr = bcv<V>(dr);
    s.di = bcv<V>(di);
    s.ndr = bcv<V>(-dr);
    s.ndi = bcv<V>(-di);
    s.el = bcv<V>(-2.f * kLog2e * kRs2 * ell);
    s.ntl = bcv<V>(-2.f * kRs2 * ell);
    return s;
}

// gamma_h, E and K of the closed-form step for two energies (packed) or one;
// stored as (gh, E, -Re K, Im K).
template <typename V>
struct CoefT {
    V ghx, ghy, ex, ey, nkx, ky;
};
typedef CoefT<f2> Coef2;

// from Omega^2 = x + i y and z = zr + i zi
template <typename V>
__device__ __forceinline__ void coef2_core(const SegT<V> &s, const V x, const V y, const V zr, const V zi,
                                           CoefT<V> &c) {
    const V n2 = fma2(x, x, mul2(y, y));     // |Omega|^4
    const V rn = rsqrt2(n2);                 // 1/|Omega|^2
    const V r = mul2(n2, rn);                // |Omega|^2
    const V u = add2(r, absv(x));            // 2 s^2
    const V ru = rsqrt2(u);
    const V sq = mul2(u, ru);                // sqrt(2) s
    const V yq = mul2(y, ru);                // sqrt(2) y / (2 s)
    // sqrt(2) Omega on the principal branch (Re Omega >= 0)
    V orr, oi;
    principal(x, y, sq, yq, orr, oi);
    // w = z + i Omega and 1/w = iwr - i iwn
    const V wr = fma2(oi, bcv<V>(-kRs2), zr);
    const V wi = fma2(orr, bcv<V>(kRs2), zi);
    const V rw = rcp2(fma2(wr, wr, mul2(wi, wi)));
    const V iwr = mul2(wr, rw), iwn = mul2(wi, rw);
    // 1/(2 Omega) = conj(Omega) / (2 |Omega|^2) = i2r - i i2n
    const V t = mul2(rn, bcv<V>(0.5f * kRs2));
    const V i2r = mul2(orr, t), i2n = mul2(oi, t);
    // gamma_h = -Delta / w
    c.ghx = fma2(s.ndr, iwr, mul2(s.ndi, iwn));
    c.ghy = fma2(s.dr, iwn, mul2(s.ndi, iwr));
    // E = exp(-2 ell Omega) = eu (cos th + i sin th), th = -2 ell Im Omega
    const V la = mul2(orr, s.el), th = mul2(oi, s.ntl);
    const V eu = ex2v(la);
    V sn, cs;
    sincosv(th, sn, cs);
    c.ex = mul2(eu, cs);
    c.ey = mul2(eu, sn);
    // (1 - E)/(2 Omega) = ccr + i cci with E - 1 = nomr + i ey
    const V nomr = fma2(eu, cs, bcv<V>(-1.f));
    const V nccr = fma2(nomr, i2r, mul2(c.ey, i2n));      // -ccr
    const V cci = fma2(nomr, i2n, mul2(neg2(c.ey), i2r));
    // K = i conj(Delta) (1 - E)/(2 Omega)
    c.nkx = fma2(s.di, nccr, mul2(s.dr, cci));             // -Re K
    c.ky = fma2(s.ndr, nccr, mul2(s.di, cci));             // Im K
}

// q: the energies' own part of z (Matsubara: eps_n; retarded: E_n)
template <bool RET, typename V>
__device__ __forceinline__ void coef2(const SegT<V> &s, const V q, CoefT<V> &c) {
    if constexpr (RET) {
        const V zr = add2(q, s.sh);
        coef2_core(s, fma2(neg2(zr), zr, s.c0), mul2(zr, s.m2), zr, s.zs, c);
    } else {
        coef2_core(s, fma2(q, q, s.c0), mul2(q, s.m2), s.zs, q, c);
    }
}

// gamma' = gamma_h + (gamma - gamma_h) E / (1 - K (gamma - gamma_h))
template <typename V>
__device__ __forceinline__ void apply2(const CoefT<V> &c, V &gx, V &gy) {
    const V dx = sub2(gx, c.ghx), dy = sub2(gy, c.ghy);
    const V nr = fma2(dx, c.ex, mul2(neg2(dy), c.ey));
    const V ni = fma2(dx, c.ey, mul2(dy, c.ex));
    const V dnr = fma2(c.nkx, dx, fma2(c.ky, dy, bcv<V>(1.f)));
    const V dni = fma2(c.nkx, dy, mul2(neg2(c.ky), dx));
    const V rd = rcp2(fma2(dnr, dnr, mul2(dni, dni)));
    gx = fma2(fma2(nr, dnr, mul2(ni, dni)), rd, c.ghx);
    gy = fma2(fma2(ni, dnr, mul2(neg2(nr), dni)), rd, c.ghy);
}

// Propagator of angle p at one sample for two energies, from gamma = ga (parked,
// forward) and gamma~ = conj(gb) (backward), added with weights m into the
// packed sums: sfr, sfi (Re/Im of sum f + conj f~ up to -2 i pi), nsg (minus the
// sum of Im 1/D), sFr, sFi (sum of ga + gb).
struct Sums2 {
    f2 sfr, sfi, nsg, sFr, sFi;
};

__device__ __forceinline__ void prop2(const f2 gax, const f2 gay, const f2 gbx, const f2 gby, const f2 m,
                                      Sums2 &S) {
    const f2 Dr = fma2(gax, gbx, fma2(gay, gby, bc2(1.f)));   // 1 + ga conj(gb)
    const f2 Di = fma2(gay, gbx, mul2(neg2(gax), gby));
    const f2 rD = rcp2(fma2(Dr, Dr, mul2(Di, Di)));
    const f2 ir = mul2(Dr, rD), nii = mul2(Di, rD);           // 1/D = ir - i nii
    const f2 Sx = add2(gax, gbx), Sy = add2(gay, gby);
    const f2 Qy = sub2(gay, gby), Px = sub2(gbx, gax);
    S.sfr = fma2(m, fma2(Sx, ir, mul2(Qy, nii)), S.sfr);
    S.sfi = fma2(m, fma2(Sy, ir, mul2(Px, nii)), S.sfi);
    S.nsg = fma2(m, nii, S.nsg);
    S.sFr = fma2(m, Sx, S.sFr);
    S.sFi = fma2(m, Sy, S.sFi);
}

// Implicit midpoint rule (App. C) for two energies: the root g1 of
// c2 g1^2 + c1 g1 + c0 = 0 continuous in Delta, g1 = 2 c0 / (sqrt(c1^2 - 4 c2 c0) - c1),
// with c2 = i ell Delta*/4, c1 = 2 c2 g0 + i ell z - 1, c0 = (c2 g0 + i ell z + 1) g0
// + i ell Delta (the arithmetic of midpoint_step, packed).
template <typename V>
struct MidT {
    V c2x, c2y, ildx, ildy, ell, nell;
};
typedef MidT<f2> Mid2;

template <typename V = f2>
__device__ __forceinline__ MidT<V> mid2(float dr, float di, float ell) {
    const float q = 0.25f * ell;
    MidT<V> m;
    m.c2x = bcv<V>(q * di);
    m.c2y = bcv<V>(q * dr);
    m.ildx = bcv<V>(-ell * di);
    m.ildy = bcv<V>(ell * dr);
    m.ell = bcv<V>(ell);
    m.nell = bcv<V>(-ell);
    return m;
}

template <typename V>
__device__ __forceinline__ void midpoint2(const MidT<V> &m, const V zr, const V zi, V &gx, V &gy) {
    const V c2gx = fma2(m.c2x, gx, mul2(neg2(m.c2y), gy));
    const V c2gy = fma2(m.c2x, gy, mul2(m.c2y, gx));
    const V lzr = mul2(m.ell, zr);
    const V c1x = fma2(bcv<V>(2.f), c2gx, fma2(m.nell, zi, bcv<V>(-1.f)));
    const V c1y = fma2(bcv<V>(2.f), c2gy, lzr);
    const V ux = add2(c2gx, fma2(m.nell, zi, bcv<V>(1.f)));
    const V uy = add2(c2gy, lzr);
    const V c0x = fma2(ux, gx, fma2(neg2(uy), gy, m.ildx));
    const V c0y = fma2(ux, gy, fma2(uy, gx, m.ildy));
    const V ccx = fma2(m.c2x, c0x, mul2(neg2(m.c2y), c0y));
    const V ccy = fma2(m.c2x, c0y, mul2(m.c2y, c0x));
    const V dx = fma2(c1x, c1x, fma2(neg2(c1y), c1y, mul2(bcv<V>(-4.f), ccx)));
    const V dy = fma2(add2(c1x, c1x), c1y, mul2(bcv<V>(-4.f), ccy));
    // sqrt(2) times the principal square root of dx + i dy
    const V n2 = fma2(dx, dx, mul2(dy, dy));
    const V r = mul2(n2, rsqrt2(n2));
    const V u = add2(r, absv(dx));
    const V ru = rsqrt2(u);
    const V sq = mul2(u, ru), yq = mul2(dy, ru);
    V sr, si;
    principal(dx, dy, sq, yq, sr, si);
    // g1 = 2 c0 / den, den = sqrt - c1; 2/den = idx - i idn
    const V denx = fma2(sr, bcv<V>(kRs2), neg2(c1x)), deny = fma2(si, bcv<V>(kRs2), neg2(c1y));
    const V rd = rcp2(mul2(bcv<V>(0.5f), fma2(denx, denx, mul2(deny, deny))));
    const V idx = mul2(denx, rd), idn = mul2(deny, rd);
    gx = fma2(c0x, idx, mul2(c0y, idn));
    gy = fma2(c0y, idx, mul2(neg2(c0x), idn));
}

// One work item of the packed sweep (see sweep_item for the layout of lines,
// lanes and items).  The warp's slab holds, per sample, the NP parked pairs of
// every lane as float4 (gx of the pair, gy of the pair) at [k][lane], then the
// scalar tail energy of every lane.  STEP 0 = closed-form step, 1 = implicit
// midpoint rule; RET: retarded sweep (LDOS) whose backward pass combines each
// energy with the parked gamma of the mirror energy.
template <int EPT, bool RET, int STEP, bool WGT, bool BLK>
__device__ __forceinline__ void sweep_item_x2(const SweepLaunch &a, const int2 it, const GrainSweep &gs,
                                              Cx<float> *const warp_slab, const int lane) {
    typedef Cx<float> C;
    constexpr int NP = EPT / 2;
    constexpr int NPA = NP > 0 ? NP : 1;
    constexpr bool TAIL = (EPT & 1) != 0;
    const int Lw = gs.lanes, G = gs.lines_per_warp;
    const int gi = lane / Lw, r = lane - gi * Lw;
    const float4 *__restrict__ img = (const float4 *)gs.image_in;
    const C *__restrict__ exit_prev = (const C *)gs.exits[a.parity];
    C *__restrict__ exit_cur = (C *)gs.exits[a.parity ^ 1];
    C *slab = warp_slab + (int64_t)gi * gs.max_ns * gs.ne_pad;
    const float h = (float)gs.h;
    const int n_e = gs.n_e;
    const int ne_pad = gs.ne_pad;
    const int nb = BLK ? gs.n_blocks : 1;
    const int grp = BLK ? it.y / nb : it.y;
    // this item's energies: the grain's part [e_first, e_end), its block of ne_pad
    const int e_end = gs.e_count > 0 ? gs.e_first + gs.e_count : n_e;
    const int e0 = gs.e_first + (BLK ? (it.y - grp * nb) * ne_pad : 0);
    const float broad = RET ? (float)gs.broadening : 0.f;

    // the lane's energies: Matsubara t (n + 1/2) or Ozaki's poles with the weights
    // of their sums (0 for padded lane slots); retarded: the real energies E_n and,
    // per energy, the float offset of the mirror energy's parked gamma in a slab row
    float zq[EPT], wv[EPT];
    int nid[EPT];
    bool ev[EPT];
    int mo[RET ? EPT : 1];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int n = e0 + r + Lw * e;
        ev[e] = n < e_end;
        const int nn = ev[e] ? n : e_end - 1;
        nid[e] = nn;
        if constexpr (RET) {
            zq[e] = (float)gs.energies[nn];
            wv[e] = 0.f;
            const int nm = n_e - 1 - nn, em = nm / Lw, rm = nm - em * Lw;
            mo[e] = em < 2 * NP ? 4 * ((em >> 1) * Lw + rm) + (em & 1) : 2 * (2 * NP * Lw + rm);
        } else {
            zq[e] = WGT ? (float)gs.mats_eps[nn] : (float)(gs.t * (nn + 0.5));
            wv[e] = ev[e] ? (WGT ? (float)gs.mats_w[nn] : 1.f) : 0.f;
        }
    }
    f2 Q[NPA], M[NPA];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        Q[k] = pk2(zq[2 * k], zq[2 * k + 1]);
        M[k] = pk2(wv[2 * k], wv[2 * k + 1]);
    }
    // z of energy e on a segment with Doppler shift sh
    auto zr_of = [&](int e, float sh) { return RET ? zq[e] + sh : sh; };
    auto zi_of = [&](int e) { return RET ? broad : zq[e]; };

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
    const float lead = (float)ln.lead, tail = (float)ln.tail;
    const int slot0 = ln.slot0;
    const float4 *li = img + slot0;
    const int tail_off = 2 * NP * Lw + r;  // the tail energy's place in a sample's slab row

    f2 GX[NPA], GY[NPA];
    C gt{0.f, 0.f};
    // one step of every energy over a segment (Delta = dr + i di, shift sh, length ell)
    auto step = [&](float dr, float di, float sh, float ell) {
        if constexpr (STEP == 0) {
            const Seg2 s = seg2<RET>(dr, di, sh, broad, ell);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                Coef2 c;
                coef2<RET>(s, Q[k], c);
                apply2(c, GX[k], GY[k]);
            }
            if constexpr (TAIL) {
                const SegT<float> s1 = seg2<RET, float>(dr, di, sh, broad, ell);
                CoefT<float> c;
                coef2<RET>(s1, zq[EPT - 1], c);
                apply2(c, gt.x, gt.y);
            }
        } else {
            const Mid2 m = mid2(dr, di, ell);
#pragma unroll
            for (int k = 0; k < NP; ++k)
                midpoint2(m, RET ? add2(Q[k], bc2(sh)) : bc2(sh), RET ? bc2(broad) : Q[k], GX[k], GY[k]);
            if constexpr (TAIL) midpoint2(mid2<float>(dr, di, ell), zr_of(EPT - 1, sh), zi_of(EPT - 1), gt.x, gt.y);
        }
    };
    // entry values: the previous sweep's exits (4 taps) or gamma_h at the first sample
    auto entry = [&](const int *taps, const double *w, float dr, float di, float sh, float ell) {
        if (a.first_sweep) {
            const Seg2 s = seg2<RET>(dr, di, sh, broad, ell);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                Coef2 c;
                coef2<RET>(s, Q[k], c);
                GX[k] = c.ghx;
                GY[k] = c.ghy;
            }
            if constexpr (TAIL) {
                const SegT<float> s1 = seg2<RET, float>(dr, di, sh, broad, ell);
                CoefT<float> c;
                coef2<RET>(s1, zq[EPT - 1], c);
                gt = C{c.ghx, c.ghy};
            }
        } else {
            float gx[EPT], gy[EPT];
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                float sx = 0.f, sy = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const C v = exit_prev[(int64_t)taps[q] * n_e + nid[e]];
                    const float wq = (float)w[q];
                    sx += wq * v.x;
                    sy += wq * v.y;
                }
                gx[e] = sx;
                gy[e] = sy;
            }
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                GX[k] = pk2(gx[2 * k], gx[2 * k + 1]);
                GY[k] = pk2(gy[2 * k], gy[2 * k + 1]);
            }
            if constexpr (TAIL) gt = C{gx[EPT - 1], gy[EPT - 1]};
        }
    };
    auto exits = [&](int line) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            if (ev[2 * k]) exit_cur[(int64_t)line * n_e + nid[2 * k]] = C{GX[k].x, GY[k].x};
            if (ev[2 * k + 1]) exit_cur[(int64_t)line * n_e + nid[2 * k + 1]] = C{GX[k].y, GY[k].y};
        }
        if constexpr (TAIL)
            if (ev[EPT - 1]) exit_cur[(int64_t)line * n_e + nid[EPT - 1]] = gt;
    };

    // ---------------- forward: angle p, along +e_par ----------------
    float4 sp = li[0];
    entry(ln.tap_f, ln.w_f, sp.x, sp.y, sp.z, lead);
    float4 sq = sp;
    float4 sn = li[min(1, nsl - 1)];
    for (int i = 0; i < nsteps; ++i) {
        const float dr = 0.5f * (sp.x + sq.x), di = 0.5f * (sp.y + sq.y);
        const float av = 0.5f * (sp.z + sq.z);
        const float ell = (i == 0) ? lead : (i == ns ? tail : h);
        step(dr, di, av, ell);
        if (i < ns) {
            C *row = slab + (int64_t)i * ne_pad;
            float4 *row4 = (float4 *)row;
#pragma unroll
            for (int k = 0; k < NP; ++k) row4[k * Lw + r] = make_float4(GX[k].x, GX[k].y, GY[k].x, GY[k].y);
            if constexpr (TAIL) row[tail_off] = gt;
        }
        sp = sq;
        sq = sn;
        sn = li[min(i + 2, nsl - 1)];
    }
    if (lv) exits(ln.exit_f);

    __syncwarp();  // the retarded pass reads gammas parked by other lanes

    // ---------------- backward: angle p + P, along -e_par ----------------
    float4 sh = li[nsl - 1];
    entry(ln.tap_b, ln.w_b, sh.x, sh.y, -sh.z, tail);
    float4 slo = sh;
    float4 snb = li[max(nsl - 2, 0)];
    for (int j = 0; j < nmax; ++j) {
        const bool act = j < nsteps;
        const int qs = nsl - 1 - j;
        const bool comb = act && j < ns;
        // parked gammas of the sample reached by this step (angle p): the lane's own
        // energies, or (retarded) the mirror energies
        f2 PX[NPA], PY[NPA];
        C gft{0.f, 0.f};
        if (comb) {
            const C *row = slab + (int64_t)qs * ne_pad;
            if constexpr (RET) {
                const float *rowf = (const float *)row;
                float px[EPT], py[EPT];
#pragma unroll
                for (int e = 0; e < EPT; ++e) {
                    px[e] = rowf[mo[e]];
                    py[e] = rowf[mo[e] + (mo[e] >= 4 * NP * Lw ? 1 : 2)];
                }
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    PX[k] = pk2(px[2 * k], px[2 * k + 1]);
                    PY[k] = pk2(py[2 * k], py[2 * k + 1]);
                }
                if constexpr (TAIL) gft = C{px[EPT - 1], py[EPT - 1]};
            } else {
                const float4 *row4 = (const float4 *)row;
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const float4 v = row4[k * Lw + r];
                    PX[k] = make_float2(v.x, v.y);
                    PY[k] = make_float2(v.z, v.w);
                }
                if constexpr (TAIL) gft = row[tail_off];
            }
        }
        if (act) {
            const float dr = 0.5f * (sh.x + slo.x), di = 0.5f * (sh.y + slo.y);
            const float av = 0.5f * (sh.z + slo.z);
            const float ell = (j == 0) ? tail : (j == ns ? lead : h);
            step(dr, di, -av, ell);
        }
        if constexpr (!RET) {
            float sfr = 0.f, sfi = 0.f, sg = 0.f, sFr = 0.f, sFi = 0.f;
            if (comb) {
                Sums2 S{bc2(0.f), bc2(0.f), bc2(0.f), bc2(0.f), bc2(0.f)};
#pragma unroll
                for (int k = 0; k < NP; ++k) prop2(PX[k], PY[k], GX[k], GY[k], M[k], S);
                sfr = S.sfr.x + S.sfr.y;
                sfi = S.sfi.x + S.sfi.y;
                sg = -(S.nsg.x + S.nsg.y);
                sFr = S.sFr.x + S.sFr.y;
                sFi = S.sFi.x + S.sFi.y;
                if constexpr (TAIL) {
                    const C gb = gt, ga = gft;
                    const float w = wv[EPT - 1];
                    const float Dr = 1.f + (ga.x * gb.x + ga.y * gb.y);
                    const float Di = ga.y * gb.x - ga.x * gb.y;
                    const float rD = Mth<float>::rcp(Dr * Dr + Di * Di);
                    const float ir = Dr * rD, ii = -Di * rD;
                    sg += w * ii;
                    sfr += w * ((ga.x + gb.x) * ir + (gb.y - ga.y) * ii);
                    sfi += w * ((ga.y + gb.y) * ir + (ga.x - gb.x) * ii);
                    sFr += w * (ga.x + gb.x);
                    sFi += w * (ga.y + gb.y);
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
                const float twopi = 6.283185307179586f, fourpi = 12.566370614359172f;
                float4 o;
                o.x = twopi * sfi;                          // Re Sf
                o.y = -twopi * sfr;                         // Im Sf
                o.z = fourpi * sg;                          // Sg
                o.w = 2.f * (slo.x * sFi - slo.y * sFr);    // SF
                // a blocked sweep writes each energy block's sums into the block's own image
                float4 *po = (float4 *)gs.image_out + (BLK ? (int64_t)(it.y - grp * nb) * gs.n_slots : 0) + slot0 + qs;
                *po = o;
            }
        } else if (comb) {
            // LDOS: -Im g / pi = 2 Re(1/D) - 1 with D = 1 + ga conj(gb)
            float *outl = (float *)gs.image_out + (int64_t)(slot0 + qs) * n_e;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const f2 Dr = fma2(PX[k], GX[k], fma2(PY[k], GY[k], bc2(1.f)));
                const f2 Di = fma2(PY[k], GX[k], mul2(neg2(PX[k]), GY[k]));
                const f2 v = fma2(mul2(Dr, rcp2(fma2(Dr, Dr, mul2(Di, Di)))), bc2(2.f), bc2(-1.f));
                if (ev[2 * k]) outl[nid[2 * k]] = v.x;
                if (ev[2 * k + 1]) outl[nid[2 * k + 1]] = v.y;
            }
            if constexpr (TAIL) {
                const C gb = gt, ga = gft;
                const float Dr = 1.f + (ga.x * gb.x + ga.y * gb.y);
                const float Di = ga.y * gb.x - ga.x * gb.y;
                const float rD = Mth<float>::rcp(Dr * Dr + Di * Di);
                if (ev[EPT - 1]) outl[nid[EPT - 1]] = 2.f * Dr * rD - 1.f;
            }
        }
        if (act) {
            sh = slo;
            slo = snb;
            snb = li[max(nsl - 3 - j, 0)];
        }
    }
    if (lv) exits(ln.exit_b);
    __syncwarp();
}

}  // namespace scd
