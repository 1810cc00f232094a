// The FP32 adjoint sweep (closed-form step, Matsubara or Ozaki energies) on
// packed pairs of energies: the lane's energies (2k, 2k+1) travel as float2
// through the three passes with sm_100's two-wide FP32 instructions, as in the
// forward sweep of sweep_x2.cuh; an odd last energy runs the same formulation
// on single values.  The arithmetic is that of the scalar adjoint kernel
// (adjoint_kernel.cuh): the Moebius form of the step (mob_coef, mob_apply,
// mob_grad of riccati_step.cuh) and the cotangents of the propagator sums,
// with complex numbers carried as (real parts, imaginary parts) of the pair.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "adjoint.cuh"
#include "bounds.cuh"
#include "sweep_x2.cuh"

namespace scd {

// complex value(s) with packed parts: V = f2 (two energies) or float (one)
template <typename V>
struct CV {
    V x, y;
};

template <typename V>
__device__ __forceinline__ CV<V> cmulv(const CV<V> a, const CV<V> b) {
    return CV<V>{fma2(a.x, b.x, mul2(neg2(a.y), b.y)), fma2(a.x, b.y, mul2(a.y, b.x))};
}
// conj(a) b
template <typename V>
__device__ __forceinline__ CV<V> cmulcv(const CV<V> a, const CV<V> b) {
    return CV<V>{fma2(a.x, b.x, mul2(a.y, b.y)), fma2(a.x, b.y, mul2(neg2(a.y), b.x))};
}
template <typename V>
__device__ __forceinline__ CV<V> caddv(const CV<V> a, const CV<V> b) {
    return CV<V>{add2(a.x, b.x), add2(a.y, b.y)};
}
template <typename V>
__device__ __forceinline__ CV<V> cscalev(const CV<V> a, const V s) {
    return CV<V>{mul2(a.x, s), mul2(a.y, s)};
}
template <typename V>
__device__ __forceinline__ CV<V> cmuliv(const CV<V> a) {  // i a
    return CV<V>{neg2(a.y), a.x};
}
template <typename V>
__device__ __forceinline__ CV<V> cconjv(const CV<V> a) {
    return CV<V>{a.x, neg2(a.y)};
}
template <typename V>
__device__ __forceinline__ CV<V> crcpv(const CV<V> a) {
    const V r = rcp2(fma2(a.x, a.x, mul2(a.y, a.y)));
    return CV<V>{mul2(a.x, r), neg2(mul2(a.y, r))};
}

// Moebius coefficients of one step for the energies q (z = zr + i q, zr shared),
// gamma' = (a gamma + b)/(c gamma + d), with E = exp(-2 Omega ell),
// c2 = (1 - E)/Omega and iO = 1/Omega (the quantities of mob_coef).
template <typename V>
struct MobV {
    CV<V> a, b, c, d, E, c2, iO;
};

template <typename V>
__device__ __forceinline__ void mob_assemble_v(float dr, float di, float zr, const V zi, MobV<V> &m) {
    const V tr = fma2(bcv<V>(zr), m.c2.x, mul2(neg2(zi), m.c2.y));  // z c2
    const V ti = fma2(bcv<V>(zr), m.c2.y, mul2(zi, m.c2.x));
    const V ur = fma2(bcv<V>(dr), m.c2.x, mul2(bcv<V>(-di), m.c2.y));  // Delta c2
    const V ui = fma2(bcv<V>(dr), m.c2.y, mul2(bcv<V>(di), m.c2.x));
    const V vr = fma2(bcv<V>(dr), m.c2.x, mul2(bcv<V>(di), m.c2.y));   // Delta* c2
    const V vi = fma2(bcv<V>(dr), m.c2.y, mul2(bcv<V>(-di), m.c2.x));
    const V ope = add2(bcv<V>(1.f), m.E.x);
    m.a = CV<V>{sub2(ope, ti), add2(m.E.y, tr)};
    m.d = CV<V>{add2(ope, ti), sub2(m.E.y, tr)};
    m.b = CV<V>{neg2(ui), ur};
    m.c = CV<V>{vi, neg2(vr)};
}

template <typename V>
__device__ __forceinline__ void mob_coef_v(float dr, float di, float d2, float zr, const V zi, float ell,
                                           MobV<V> &m) {
    const V x = fma2(zi, zi, bcv<V>(d2 - zr * zr));  // Re Omega^2
    const V y = mul2(bcv<V>(-2.f * zr), zi);          // Im Omega^2
    const V n2 = fma2(x, x, mul2(y, y));
    const V rn = rsqrt2(n2);                          // 1/|Omega|^2
    const V r = mul2(n2, rn);                         // |Omega^2|
    const V hs = mul2(bcv<V>(0.5f), add2(r, absv(x)));
    const V q = rsqrt2(hs);
    const V s = mul2(hs, q);
    const V yq = mul2(mul2(bcv<V>(0.5f), y), q);
    V orr, oi;
    // principal square root: Re Omega >= 0 (the helper works on the sqrt(2)-scaled
    // pair (sqrt(2) s, sqrt(2) y/(2 s)); here s and y/(2 s) themselves)
    principal(x, y, s, yq, orr, oi);
    const V ro = rcp2(fma2(orr, orr, mul2(oi, oi)));
    m.iO = CV<V>{mul2(orr, ro), neg2(mul2(oi, ro))};
    const V eu = ex2v(mul2(orr, bcv<V>(-2.f * ell * kLog2e)));
    V sn, cs;
    sincosv(mul2(oi, bcv<V>(2.f * ell)), sn, cs);
    m.E = CV<V>{mul2(eu, cs), neg2(mul2(eu, sn))};
    const CV<V> om{sub2(bcv<V>(1.f), m.E.x), neg2(m.E.y)};
    m.c2 = cmulv(om, m.iO);
    mob_assemble_v(dr, di, zr, zi, m);
}

// the same segment for z' = -conj(z) (the other direction of a Matsubara pair)
template <typename V>
__device__ __forceinline__ void mob_mirror_v(const MobV<V> &f, float dr, float di, float zr, const V zi,
                                             MobV<V> &m) {
    m.E = cconjv(f.E);
    m.c2 = cconjv(f.c2);
    m.iO = cconjv(f.iO);
    mob_assemble_v(dr, di, zr, zi, m);
}

template <typename V>
__device__ __forceinline__ CV<V> mob_apply_v(const MobV<V> &m, const CV<V> g) {
    const CV<V> n = caddv(cmulv(m.a, g), m.b);
    const CV<V> u = crcpv(caddv(cmulv(m.c, g), m.d));
    return cmulv(n, u);
}

template <typename V>
struct GradV {
    CV<V> dg, dP, dQ, dR;
};

// derivatives of the step at its start value g (see mob_grad)
template <typename V>
__device__ __forceinline__ void mob_grad_v(const MobV<V> &m, float dr, float di, float zr, const V zi, float ell,
                                           const CV<V> g, GradV<V> &G) {
    const CV<V> u = crcpv(caddv(cmulv(m.c, g), m.d));
    const CV<V> gp = cmulv(caddv(cmulv(m.a, g), m.b), u);
    const CV<V> Ab = cmulv(g, u);
    const CV<V> gpu = cmulv(gp, u);
    const CV<V> Db{neg2(gpu.x), neg2(gpu.y)};
    const CV<V> Cb = cmulv(g, Db);
    const CV<V> Eu2 = cmulv(m.E, cmulv(u, u));
    G.dg = cscalev(Eu2, bcv<V>(4.f));
    const V l2 = bcv<V>(2.f * ell);
    const CV<V> kap = cmulv(CV<V>{fma2(l2, m.E.x, neg2(m.c2.x)), fma2(l2, m.E.y, neg2(m.c2.y))}, m.iO);
    const CV<V> apd = caddv(Ab, Db);
    const CV<V> amd{sub2(Ab.x, Db.x), sub2(Ab.y, Db.y)};
    const CV<V> t1 = cmulv(m.E, apd);
    const CV<V> z{bcv<V>(zr), zi};
    const CV<V> w1 = cmulv(amd, z);
    const CV<V> w2 = cmulv(u, CV<V>{bcv<V>(dr), bcv<V>(di)});
    const CV<V> w3 = cmulv(Cb, CV<V>{bcv<V>(dr), bcv<V>(-di)});
    const CV<V> w{sub2(add2(w1.x, w2.x), w3.x), sub2(add2(w1.y, w2.y), w3.y)};
    const CV<V> kw = cmulv(kap, w);
    const V m2l = bcv<V>(-2.f * ell);
    const CV<V> S{fma2(m2l, t1.x, neg2(kw.y)), fma2(m2l, t1.y, kw.x)};  // -2 ell E (Ab + Db) + i kappa w
    const CV<V> SO = cmulv(S, m.iO);                                     // S / Omega
    const CV<V> sR = cmulv(SO, CV<V>{bcv<V>(0.5f * dr), bcv<V>(-0.5f * di)});
    const CV<V> sP = cmulv(SO, CV<V>{bcv<V>(0.5f * dr), bcv<V>(0.5f * di)});
    const CV<V> sQ = cmulv(SO, z);
    const CV<V> cB = cmulv(m.c2, u), cC = cmulv(m.c2, Cb), cA = cmulv(m.c2, amd);
    G.dR = CV<V>{sub2(sR.x, cB.y), add2(sR.y, cB.x)};
    G.dP = CV<V>{add2(sP.x, cC.y), sub2(sP.y, cC.x)};
    G.dQ = CV<V>{sub2(neg2(sQ.x), cA.y), add2(neg2(sQ.y), cA.x)};
}

// One work item of the packed FP32 adjoint (Matsubara or Ozaki energies, the
// closed-form step).  Slab rows per sample: [0] gamma then beta, [1] the local
// beta cotangent, each as NP float4 pairs per lane ([k][lane]) and the scalar
// tail energy of every lane; after them (and the kept rows) one row each for the
// entry values of gamma and beta.  CK: pass 1 keeps gamma only at the samples
// 0, k, 2k, ... (k = a.ckpt) in rows after the 2 max_ns sample rows, and pass 2
// recomputes the samples of each stretch [ck, ck + k) from its kept value (the
// same steps as pass 1, so the same values) when it enters the stretch.
template <int EPT, bool BLK, bool CK>
__device__ __forceinline__ void adjoint_item_x2(const AdjointLaunch &a, const int2 it, const GrainSweep &gs,
                                                Cx<float> *const warp_slab, const int lane) {
    typedef Cx<float> C;
    typedef CV<f2> P2;
    typedef CV<float> P1;
    constexpr int NP = EPT / 2;
    constexpr int NPA = NP > 0 ? NP : 1;
    constexpr bool TAIL = (EPT & 1) != 0;
    const int Lw = gs.lanes, G = gs.lines_per_warp;
    const int gi = lane / Lw, r = lane - gi * Lw;
    const float4 *__restrict__ img = (const float4 *)gs.image_in;
    const float4 *__restrict__ wimg = (const float4 *)a.wimg;
    float4 *__restrict__ gimg = (float4 *)a.gimg;
    const C *__restrict__ exit_prev = (const C *)gs.exits[a.parity];
    const float h = (float)gs.h;
    const int n_e = gs.n_e, ne_pad = gs.ne_pad;
    const int ck = CK ? a.ckpt : 1;
    const int64_t nkept = CK ? (gs.max_ns + ck - 1) / ck : 0;
    // rows per line: two per sample, the kept gammas, and the entry values of gamma and beta
    const int64_t lrows = 2 * (int64_t)gs.max_ns + nkept + 2;
    C *slab = warp_slab + (int64_t)gi * lrows * ne_pad;
    const float pi = 3.141592653589793f;
    const int nb = BLK ? gs.n_blocks : 1;
    const int grp = BLK ? it.y / nb : it.y;
    const int e0 = BLK ? (it.y - grp * nb) * ne_pad : 0;

    // the lane's energies and the weights of their sums (0 for padded slots)
    float zq[EPT], wv[EPT];
    int nid[EPT];
    bool ev[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int n = e0 + r + Lw * e;
        ev[e] = n < n_e;
        nid[e] = ev[e] ? n : n_e - 1;
        zq[e] = gs.mats_eps ? (float)gs.mats_eps[nid[e]] : (float)(gs.t * (nid[e] + 0.5));
        wv[e] = ev[e] ? (gs.mats_w ? (float)gs.mats_w[nid[e]] : 1.f) : 0.f;
    }
    f2 Q[NPA], M[NPA], EVM[NPA];  // energies, sum weights, 1/0 for valid energies
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        Q[k] = pk2(zq[2 * k], zq[2 * k + 1]);
        M[k] = pk2(wv[2 * k], wv[2 * k + 1]);
        EVM[k] = pk2(ev[2 * k] ? 1.f : 0.f, ev[2 * k + 1] ? 1.f : 0.f);
    }
    const float evt = TAIL && ev[EPT - 1] ? 1.f : 0.f;

    const int64_t gq = (int64_t)grp * G + gi;
    int L = in_bounds(gq, (int64_t)gs.n_groups * G) ? gs.groups[gq] : -1;
    if (L >= 0 && !in_bounds(L, gs.n_lines)) L = -1;
    const LineDev &ln = gs.lines[L >= 0 ? L : 0];
    const bool lv = L >= 0 && line_tables_ok(ln, gs.n_slots, gs.n_lines, !a.first_sweep,
                                             (int64_t)(slab - (C *)a.scratch), 2 * ne_pad, a.scratch_elems) &&
                    in_bounds((int64_t)(slab - (C *)a.scratch) + lrows * ne_pad - 1, a.scratch_elems);
    const int ns = lv ? ln.ns : 0;  // lines without samples do not enter the loss
    const int nsl = ns > 0 ? ns : 1;
    const int nsteps = ns > 0 ? ns + 1 : 0;
    int nmax = nsteps;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nmax = max(nmax, __shfl_xor_sync(FULL_MASK, nmax, off));
    if (nmax == 0) return;
    const float lead = (float)ln.lead, tail = (float)ln.tail;
    const int slot0 = ln.slot0;
    const float4 *li = img + slot0;
    const int tail_off = 2 * NP * Lw + r;
    auto row = [&](int i, int k) -> C * { return slab + ((int64_t)i * 2 + k) * ne_pad; };
    auto ld2 = [&](int i, int k, int p) -> P2 {
        const float4 v = ((const float4 *)row(i, k))[p * Lw + r];
        return P2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
    };
    auto st2 = [&](int i, int k, int p, const P2 v) {
        ((float4 *)row(i, k))[p * Lw + r] = make_float4(v.x.x, v.x.y, v.y.x, v.y.y);
    };
    auto ld1 = [&](int i, int k) -> P1 {
        const C v = row(i, k)[tail_off];
        return P1{v.x, v.y};
    };
    auto st1 = [&](int i, int k, const P1 v) { row(i, k)[tail_off] = C{v.x, v.y}; };
    // kept gamma c (CK): the row after the sample rows
    auto krow = [&](int c) -> C * { return slab + (2 * (int64_t)gs.max_ns + c) * ne_pad; };
    // entry values of gamma (k = 0) and beta (k = 1), parked rather than held in registers
    C *const erow[2] = {slab + (2 * (int64_t)gs.max_ns + nkept) * ne_pad,
                        slab + (2 * (int64_t)gs.max_ns + nkept + 1) * ne_pad};
    auto est2 = [&](int k, int p, const P2 v) {
        ((float4 *)erow[k])[p * Lw + r] = make_float4(v.x.x, v.x.y, v.y.x, v.y.y);
    };
    auto eld2 = [&](int k, int p) -> P2 {
        const float4 v = ((const float4 *)erow[k])[p * Lw + r];
        return P2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
    };
    auto est1 = [&](int k, const P1 v) { erow[k][tail_off] = C{v.x, v.y}; };
    auto eld1 = [&](int k) -> P1 { return P1{erow[k][tail_off].x, erow[k][tail_off].y}; };
    // entry values: the previous sweep's exits (4 taps) or gamma_h of the first segment
    auto entry = [&](const int *taps, const double *w, const float4 s, float zr, float ell, P2 *gp, P1 &gt) {
        if (a.first_sweep) {
            const Seg2 sg = seg2<false>(s.x, s.y, zr, 0.f, ell);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                Coef2 c;
                coef2<false>(sg, Q[k], c);
                gp[k] = P2{c.ghx, c.ghy};
            }
            if constexpr (TAIL) {
                const SegT<float> s1 = seg2<false, float>(s.x, s.y, zr, 0.f, ell);
                CoefT<float> c;
                coef2<false>(s1, zq[EPT - 1], c);
                gt = P1{c.ghx, c.ghy};
            }
        } else {
            float gx[EPT], gy[EPT];
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                float sx = 0.f, sy = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const C v = exit_prev[(int64_t)taps[q] * n_e + nid[e]];
                    sx += (float)w[q] * v.x;
                    sy += (float)w[q] * v.y;
                }
                gx[e] = sx;
                gy[e] = sy;
            }
#pragma unroll
            for (int k = 0; k < NP; ++k) gp[k] = P2{pk2(gx[2 * k], gx[2 * k + 1]), pk2(gy[2 * k], gy[2 * k + 1])};
            if constexpr (TAIL) gt = P1{gx[EPT - 1], gy[EPT - 1]};
        }
    };

    // ---------------- pass 1: gamma along +e_par (the forward sweep's steps) ----------------
    P2 g[NPA];
    P1 gt{0.f, 0.f};
    float4 sp = li[0];
    entry(ln.tap_f, ln.w_f, sp, sp.z, lead, g, gt);
#pragma unroll
    for (int k = 0; k < NP; ++k) est2(0, k, g[k]);
    if constexpr (TAIL) est1(0, gt);
    {
        float4 sq = sp;
        for (int i = 0; i < nsteps; ++i) {
            const float dr = 0.5f * (sp.x + sq.x), di = 0.5f * (sp.y + sq.y), av = 0.5f * (sp.z + sq.z);
            const float ell = (i == 0) ? lead : (i == ns ? tail : h);
            const Seg2 sg = seg2<false>(dr, di, av, 0.f, ell);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                Coef2 c;
                coef2<false>(sg, Q[k], c);
                apply2(c, g[k].x, g[k].y);
            }
            if constexpr (TAIL) {
                const SegT<float> s1 = seg2<false, float>(dr, di, av, 0.f, ell);
                CoefT<float> c;
                coef2<false>(s1, zq[EPT - 1], c);
                apply2(c, gt.x, gt.y);
            }
            if (i < ns) {
                if constexpr (CK) {
                    if (i % ck == 0) {
                        C *kr = krow(i / ck);
#pragma unroll
                        for (int k = 0; k < NP; ++k)
                            ((float4 *)kr)[k * Lw + r] = make_float4(g[k].x.x, g[k].x.y, g[k].y.x, g[k].y.y);
                        if constexpr (TAIL) kr[tail_off] = C{gt.x, gt.y};
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < NP; ++k) st2(i, 0, k, g[k]);
                    if constexpr (TAIL) st1(i, 0, gt);
                }
            }
            sp = sq;
            sq = li[min(i + 1, nsl - 1)];
        }
    }
    __syncwarp();

    // ---------------- pass 2: beta along -e_par, gamma adjoint ----------------
    P2 b[NPA], lam[NPA];
    P1 bt{0.f, 0.f}, lat{0.f, 0.f};
    float4 sh = li[nsl - 1];
    entry(ln.tap_b, ln.w_b, sh, -sh.z, tail, b, bt);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        est2(1, k, b[k]);
        lam[k] = P2{bc2(0.f), bc2(0.f)};
    }
    if constexpr (TAIL) est1(1, bt);
    {
        float4 slo = sh;
        for (int j = 0; j < nmax; ++j) {
            const bool act = j < nsteps;
            const int q = nsl - 1 - j;  // sample reached (j < ns)
            const bool at_sample = act && j < ns;
            // the next step's parked gammas (written long ago) are fetched into L2
            if (!CK && j + 1 < ns) {
#pragma unroll
                for (int k = 0; k < NP; ++k) l2_hint((const float4 *)row(q - 1, 0) + k * Lw + r);
                if constexpr (TAIL) l2_hint(row(q - 1, 0) + tail_off);
            }
            float cdr = 0.f, cdi = 0.f, ca = 0.f, sdr = 0.f, sdi = 0.f;
            if (act) {
                const float dr = 0.5f * (sh.x + slo.x), di = 0.5f * (sh.y + slo.y), av = 0.5f * (sh.z + slo.z);
                const float ell = (j == 0) ? tail : (j == ns ? lead : h);
                const float d2 = dr * dr + di * di;
                float4 W = make_float4(0.f, 0.f, 0.f, 0.f);
                if (at_sample) W = wimg[slot0 + q];
                // cotangent weights of the sample's energy sums (see the scalar kernel)
                const float kga = 2.f * pi, kgb = -4.f * pi * W.z, kF = 2.f * W.w;
                f2 Cdr = bc2(0.f), Cdi = bc2(0.f), Ca = bc2(0.f), Sdr = bc2(0.f), Sdi = bc2(0.f);
                auto one = [&](auto &bb, auto &la, const auto gstart, auto zi, auto wn, auto evm,
                               auto &cdr_, auto &cdi_, auto &ca_, auto &sdr_, auto &sdi_, auto &bbar_out) {
                    using Vv = std::decay_t<decltype(zi)>;
                    MobV<Vv> cf, cb;
                    mob_coef_v<Vv>(dr, di, d2, av, zi, ell, cf);
                    mob_mirror_v<Vv>(cf, dr, di, -av, zi, cb);
                    bb = mob_apply_v(cb, bb);
                    GradV<Vv> Gd;
                    mob_grad_v<Vv>(cf, dr, di, av, zi, ell, gstart, Gd);
                    // coefficient cotangents: conj(dR) lam + dP conj(lam), Re(conj(dQ) lam)
                    const CV<Vv> t1 = cmulcv(Gd.dR, la);
                    const CV<Vv> t2 = cmulv(Gd.dP, cconjv(la));
                    cdr_ = fma2(evm, add2(t1.x, t2.x), cdr_);
                    cdi_ = fma2(evm, add2(t1.y, t2.y), cdi_);
                    ca_ = fma2(evm, cmulcv(Gd.dQ, la).x, ca_);
                    CV<Vv> lnew = cmulcv(Gd.dg, la);
                    if (at_sample) {
                        const CV<Vv> gf = gstart, btv = bb;
                        // D = 1 + gamma conj(beta)
                        const CV<Vv> Dd{add2(bcv<Vv>(1.f), fma2(gf.x, btv.x, mul2(gf.y, btv.y))),
                                        fma2(gf.y, btv.x, mul2(neg2(gf.x), btv.y))};
                        const CV<Vv> iD = crcpv(Dd);
                        const CV<Vv> iD2 = cmulv(iD, iD), iDc2 = cconjv(iD2);
                        const CV<Vv> Wf{bcv<Vv>(W.x), bcv<Vv>(W.y)};
                        const CV<Vv> Wc{bcv<Vv>(W.x), bcv<Vv>(-W.y)};
                        const CV<Vv> Ds{bcv<Vv>(slo.x), bcv<Vv>(slo.y)};
                        const CV<Vv> ga = cmulv(cmuliv(cscalev(iDc2, bcv<Vv>(kga))), caddv(Wf, cmulv(cmulv(btv, btv), Wc)));
                        const CV<Vv> gb2 = cmulv(cmuliv(cscalev(iDc2, bcv<Vv>(kgb))), btv);
                        const CV<Vv> gcF = cmuliv(cscalev(Ds, bcv<Vv>(kF)));
                        const CV<Vv> gbar = caddv(caddv(ga, gb2), gcF);
                        const CV<Vv> ba = cmulv(cmuliv(cscalev(iD2, bcv<Vv>(kga))), caddv(Wf, cmulv(cmulv(gf, gf), Wc)));
                        const CV<Vv> bb2 = cmulv(cmuliv(cscalev(iD2, bcv<Vv>(-kgb))), gf);
                        const CV<Vv> bbar = caddv(caddv(ba, bb2), gcF);
                        // every term of energy n carries its weight (0 for padded slots)
                        lnew = caddv(lnew, cscalev(gbar, wn));
                        bbar_out = cscalev(bbar, wn);
                        // direct dependence of S_F on the sample value: -2 i wF (gamma + beta)
                        const CV<Vv> sF = cmuliv(cscalev(caddv(gf, btv), mul2(bcv<Vv>(-2.f * W.w), wn)));
                        sdr_ = add2(sdr_, sF.x);
                        sdi_ = add2(sdi_, sF.y);
                    }
                    la = lnew;
                };
                if constexpr (CK) {
                    // entering the stretch [q0, q0 + k) from above: its gammas again
                    if (at_sample && (q == ns - 1 || (q + 1) % ck == 0)) {
                        const int q0 = q - q % ck;
                        const C *kr = krow(q0 / ck);
                        P2 gg[NPA];
                        P1 ggt{0.f, 0.f};
#pragma unroll
                        for (int k = 0; k < NP; ++k) {
                            const float4 v = ((const float4 *)kr)[k * Lw + r];
                            gg[k] = P2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
                            st2(q0, 0, k, gg[k]);
                        }
                        if constexpr (TAIL) {
                            ggt = P1{kr[tail_off].x, kr[tail_off].y};
                            st1(q0, 0, ggt);
                        }
                        float4 s0 = li[q0];
                        for (int i = q0 + 1; i <= q; ++i) {
                            const float4 s1 = li[i];
                            const float rdr = 0.5f * (s0.x + s1.x), rdi = 0.5f * (s0.y + s1.y);
                            const float rav = 0.5f * (s0.z + s1.z);
                            const Seg2 sg = seg2<false>(rdr, rdi, rav, 0.f, h);
#pragma unroll
                            for (int k = 0; k < NP; ++k) {
                                Coef2 c;
                                coef2<false>(sg, Q[k], c);
                                apply2(c, gg[k].x, gg[k].y);
                                st2(i, 0, k, gg[k]);
                            }
                            if constexpr (TAIL) {
                                const SegT<float> s1t = seg2<false, float>(rdr, rdi, rav, 0.f, h);
                                CoefT<float> c;
                                coef2<false>(s1t, zq[EPT - 1], c);
                                apply2(c, ggt.x, ggt.y);
                                st1(i, 0, ggt);
                            }
                            s0 = s1;
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const P2 start = at_sample ? ld2(q, 0, k) : eld2(0, k);
                    P2 bbar{bc2(0.f), bc2(0.f)};
                    one(b[k], lam[k], start, Q[k], M[k], EVM[k], Cdr, Cdi, Ca, Sdr, Sdi, bbar);
                    if (at_sample) st2(q, 1, k, bbar);
                }
                cdr = Cdr.x + Cdr.y;
                cdi = Cdi.x + Cdi.y;
                ca = Ca.x + Ca.y;
                sdr = Sdr.x + Sdr.y;
                sdi = Sdi.x + Sdi.y;
                if constexpr (TAIL) {
                    const P1 start = at_sample ? ld1(q, 0) : eld1(0);
                    P1 bbar{0.f, 0.f};
                    one(bt, lat, start, zq[EPT - 1], wv[EPT - 1], evt, cdr, cdi, ca, sdr, sdi, bbar);
                    if (at_sample) st1(q, 1, bbar);
                }
            }
            if (at_sample) {
#pragma unroll
                for (int k = 0; k < NP; ++k) st2(q, 0, k, b[k]);
                if constexpr (TAIL) st1(q, 0, bt);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                if (off >= Lw) continue;
                cdr += __shfl_xor_sync(FULL_MASK, cdr, off);
                cdi += __shfl_xor_sync(FULL_MASK, cdi, off);
                ca += __shfl_xor_sync(FULL_MASK, ca, off);
                sdr += __shfl_xor_sync(FULL_MASK, sdr, off);
                sdi += __shfl_xor_sync(FULL_MASK, sdi, off);
            }
            if (act && r == 0) {
                const int hi = min(ns - j, ns - 1), lo = max(ns - 1 - j, 0);
                float4 *ph = gimg + slot0 + hi;
                float4 *pl = gimg + slot0 + lo;
                atomicAdd(&ph->x, 0.5f * cdr);
                atomicAdd(&ph->y, 0.5f * cdi);
                atomicAdd(&ph->z, 0.5f * ca);
                atomicAdd(&pl->x, 0.5f * cdr + (at_sample ? sdr : 0.f));
                atomicAdd(&pl->y, 0.5f * cdi + (at_sample ? sdi : 0.f));
                atomicAdd(&pl->z, 0.5f * ca);
            }
            if (act) {
                sh = slo;
                slo = li[max(nsl - 2 - j, 0)];
            }
        }
    }
    __syncwarp();

    // ---------------- pass 3: beta adjoint along +e_par ----------------
    P2 mu[NPA];
    P1 mut{0.f, 0.f};
    {
        float4 sa = li[0], sb = li[0];
        for (int i = 0; i < nmax; ++i) {
            const bool act = i < nsteps;
            // the next step's parked beta and beta cotangent are fetched into L2
            if (i + 1 < ns) {
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    l2_hint((const float4 *)row(i + 1, 0) + k * Lw + r);
                    l2_hint((const float4 *)row(i + 1, 1) + k * Lw + r);
                }
                if constexpr (TAIL) {
                    l2_hint(row(i + 1, 0) + tail_off);
                    l2_hint(row(i + 1, 1) + tail_off);
                }
            }
            float cdr = 0.f, cdi = 0.f, ca = 0.f;
            if (act) {
                if (i == 0) {
#pragma unroll
                    for (int k = 0; k < NP; ++k) mu[k] = ld2(0, 1, k);
                    if constexpr (TAIL) mut = ld1(0, 1);
                } else {
                    const float dr = 0.5f * (sa.x + sb.x), di = 0.5f * (sa.y + sb.y), av = 0.5f * (sa.z + sb.z);
                    const float ell = (i == ns) ? tail : h;
                    const float d2 = dr * dr + di * di;
                    f2 Cdr = bc2(0.f), Cdi = bc2(0.f), Ca = bc2(0.f);
                    auto one = [&](auto &m_, const auto bstart, auto zi, auto evm, auto &cdr_, auto &cdi_,
                                   auto &ca_, const auto cot) {
                        using Vv = std::decay_t<decltype(zi)>;
                        MobV<Vv> cb;
                        mob_coef_v<Vv>(dr, di, d2, -av, zi, ell, cb);
                        GradV<Vv> Gd;
                        mob_grad_v<Vv>(cb, dr, di, -av, zi, ell, bstart, Gd);
                        const CV<Vv> t1 = cmulcv(Gd.dR, m_);
                        const CV<Vv> t2 = cmulv(Gd.dP, cconjv(m_));
                        cdr_ = fma2(evm, add2(t1.x, t2.x), cdr_);
                        cdi_ = fma2(evm, add2(t1.y, t2.y), cdi_);
                        ca_ = fma2(neg2(evm), cmulcv(Gd.dQ, m_).x, ca_);  // Q = z - a
                        m_ = caddv(cmulcv(Gd.dg, m_), cot);
                    };
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const P2 start = i < ns ? ld2(i, 0, k) : eld2(1, k);
                        const P2 cot = i < ns ? ld2(i, 1, k) : P2{bc2(0.f), bc2(0.f)};
                        one(mu[k], start, Q[k], EVM[k], Cdr, Cdi, Ca, cot);
                    }
                    cdr = Cdr.x + Cdr.y;
                    cdi = Cdi.x + Cdi.y;
                    ca = Ca.x + Ca.y;
                    if constexpr (TAIL) {
                        const P1 start = i < ns ? ld1(i, 0) : eld1(1);
                        const P1 cot = i < ns ? ld1(i, 1) : P1{0.f, 0.f};
                        one(mut, start, zq[EPT - 1], evt, cdr, cdi, ca, cot);
                    }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                if (off >= Lw) continue;
                cdr += __shfl_xor_sync(FULL_MASK, cdr, off);
                cdi += __shfl_xor_sync(FULL_MASK, cdi, off);
                ca += __shfl_xor_sync(FULL_MASK, ca, off);
            }
            if (act && i > 0 && r == 0) {
                const int s0 = max(i - 1, 0), s1 = min(i, ns - 1);
                float4 *p0 = gimg + slot0 + s0;
                float4 *p1 = gimg + slot0 + s1;
                atomicAdd(&p0->x, 0.5f * cdr);
                atomicAdd(&p0->y, 0.5f * cdi);
                atomicAdd(&p0->z, 0.5f * ca);
                atomicAdd(&p1->x, 0.5f * cdr);
                atomicAdd(&p1->y, 0.5f * cdi);
                atomicAdd(&p1->z, 0.5f * ca);
            }
            if (act) {
                sa = sb;
                sb = li[min(i + 1, nsl - 1)];
            }
        }
    }
    __syncwarp();
}

}  // namespace scd
