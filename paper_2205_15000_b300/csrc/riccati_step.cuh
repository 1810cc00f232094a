// Device math of one closed-form Riccati step, shared by the sweep kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace scd {

// ---------------------------------------------------------------------------
// Precision traits: FP32 uses the approximate PTX unit instructions, FP64 the
// IEEE-accurate library functions (the plain FP64 sweep).
// ---------------------------------------------------------------------------
template <typename T>
struct Mth;

template <>
struct Mth<float> {
    static __device__ __forceinline__ float rcp(float v) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
        return r;
    }
    static __device__ __forceinline__ float rsqrt(float v) {
        float r;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
        return r;
    }
    static __device__ __forceinline__ float sqrt(float v) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
        return r;
    }
    static __device__ __forceinline__ float expneg(float u) {  // exp(-u) = 2^(-u log2 e)
        float r;
        const float x = -u * 1.4426950408889634f;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ void sincos_(float x, float *s, float *c) {
        asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*s) : "f"(x));
        asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*c) : "f"(x));
    }
};

// FP64 on the device: reciprocal and reciprocal square root by Newton-Raphson
// iteration from the FP32 unit approximations (relative error below 2^-22):
//   1/v:       r <- r + r (1 - v r)
//   1/sqrt(v): y <- y + y (1/2 - (v/2) y^2)
// each step squares the relative error, so two steps pass double precision
// (about 1 ulp, not the correctly rounded IEEE result).  Arguments whose FP32
// approximation is zero, infinite or NaN (outside the float range) take the IEEE
// operation.  sin and cos share one argument reduction (sincos).  The host keeps
// the IEEE forms.
template <>
struct Mth<double> {
    static __host__ __device__ __forceinline__ double rcp(double v) {
#ifdef __CUDA_ARCH__
        const float s = Mth<float>::rcp((float)v);
        if (!(fabsf(s) < 3.0e38f) || s == 0.f) return 1.0 / v;
        double r = (double)s;
        r = fma(r, fma(-v, r, 1.0), r);
        r = fma(r, fma(-v, r, 1.0), r);
        return r;
#else
        return 1.0 / v;
#endif
    }
    static __host__ __device__ __forceinline__ double rsqrt(double v) {
#ifdef __CUDA_ARCH__
        const float s = Mth<float>::rsqrt((float)v);
        if (!(s < 3.0e38f) || !(s > 0.f)) return 1.0 / ::sqrt(v);
        double y = (double)s;
        const double hv = 0.5 * v;
        y = fma(y, fma(-hv * y, y, 0.5), y);
        y = fma(y, fma(-hv * y, y, 0.5), y);
        return y;
#else
        return 1.0 / ::sqrt(v);
#endif
    }
    static __host__ __device__ __forceinline__ double sqrt(double v) { return ::sqrt(v); }
    static __host__ __device__ __forceinline__ double expneg(double u) { return ::exp(-u); }
    static __host__ __device__ __forceinline__ void sincos_(double x, double *s, double *c) {
#ifdef __CUDA_ARCH__
        ::sincos(x, s, c);
#else
        *s = ::sin(x);
        *c = ::cos(x);
#endif
    }
};

template <typename T>
struct Cx {
    T x, y;
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    typedef float4 type;
};
template <>
struct Vec4<double> {
    typedef double4_32a type;
};

// Coefficients of one closed-form step over a segment with constant Delta and
// z (stepping method, App. C).  For d gamma/ds = i (Delta* g^2 + 2 z g + Delta):
//   Omega   = sqrt(|Delta|^2 - z^2)          principal branch, Re Omega >= 0
//   gamma_h = -Delta / (z + i Omega)          fixed point that is stable along s
//   E = exp(-2 Omega ell),  K = i Delta* (1 - E) / (2 Omega)
//   gamma'  = gamma_h + (gamma - gamma_h) E / (1 - K (gamma - gamma_h))
// (gamma - gamma_h obeys a Bernoulli equation whose solution is this Moebius map.)
template <typename T>
struct StepCoef {
    Cx<T> gh, E, K;
};

template <typename T>
__host__ __device__ __forceinline__ void step_coef(T dr, T di, T d2, T zr, T zi, T ell, StepCoef<T> &c) {
    typedef Mth<T> M;
    const T x = d2 - zr * zr + zi * zi;  // Re Omega^2
    const T y = T(-2) * zr * zi;         // Im Omega^2
    using ::fabs;
    using ::copysign;
    // |Omega|^2 = |Omega^2|: one reciprocal square root gives both r and the
    // 1/(2 Omega) factor below
    const T n2 = x * x + y * y;
    const T rn = M::rsqrt(n2);           // 1/|Omega|^2
    const T r = n2 * rn;                 // |Omega^2|
    const T hs = T(0.5) * (r + fabs(x));
    const T q = M::rsqrt(hs);            // 1/s
    const T s = hs * q;                  // s = sqrt((r + |x|)/2)
    const T yq = T(0.5) * y * q;         // y / (2 s)
    T Or, Oi;
    if (x >= T(0)) {
        Or = s;
        Oi = yq;
    } else {
        Or = fabs(yq);
        Oi = copysign(s, y);
    }
    const T wr = zr - Oi, wi = zi + Or;  // w = z + i Omega
    // 1/w from the reciprocal of its squared modulus; 1/(2 Omega) = conj(Omega)/(2 |Omega|^2)
    const T rw = M::rcp(wr * wr + wi * wi);
    const T iwr = wr * rw, iwi = -wi * rw;                    // 1/w
    const T ro = T(0.5) * rn;
    const T i2r = Or * ro, i2i = -Oi * ro;                    // 1/(2 Omega)
    c.gh.x = -(dr * iwr - di * iwi);
    c.gh.y = -(dr * iwi + di * iwr);
    const T eu = M::expneg(T(2) * ell * Or);
    T sn, cs;
    M::sincos_(T(2) * ell * Oi, &sn, &cs);
    c.E.x = eu * cs;
    c.E.y = -eu * sn;
    const T omr = T(1) - c.E.x, omi = -c.E.y;  // 1 - E
    const T ccr = omr * i2r - omi * i2i, cci = omr * i2i + omi * i2r;
    c.K.x = -(dr * cci - di * ccr);  // K = i conj(Delta) (1 - E)/(2 Omega)
    c.K.y = dr * ccr + di * cci;
}

template <typename T>
__host__ __device__ __forceinline__ void step_apply(const StepCoef<T> &c, Cx<T> &g) {
    const T dx = g.x - c.gh.x, dy = g.y - c.gh.y;
    const T nr = dx * c.E.x - dy * c.E.y, ni = dx * c.E.y + dy * c.E.x;
    const T dnr = T(1) - (c.K.x * dx - c.K.y * dy), dni = -(c.K.x * dy + c.K.y * dx);
    const T rd = Mth<T>::rcp(dnr * dnr + dni * dni);
    g.x = c.gh.x + (nr * dnr + ni * dni) * rd;
    g.y = c.gh.y + (ni * dnr - nr * dni) * rd;
}

// ---------------------------------------------------------------------------
// Derivatives of one closed-form step, for the adjoint sweep.  The step
// gamma' = Phi(gamma; P, Q, R) is analytic in gamma and, separately, in the
// coefficients P = Delta*, Q = z, R = Delta (Delta and Delta* treated as
// independent variables).  With Omega^2 = P R - Q^2, w = Q + i Omega,
// gamma_h = -R/w, E = exp(-2 Omega ell), c = (1 - E)/(2 Omega), K = i P c,
// delta = gamma - gamma_h, N = 1 - K delta:
//   dPhi/dgamma = E / N^2
//   dOmega/dP = R/(2 Omega), dOmega/dR = P/(2 Omega), dOmega/dQ = -Q/Omega
//   dgamma_h/dP = i gamma_h^2/(2 Omega), dgamma_h/dQ = i gamma_h/Omega,
//   dgamma_h/dR = i/(2 Omega)
//   dE/dX = -2 ell E dOmega/dX,  dc/dX = (ell E - c)/Omega dOmega/dX
//   dPhi/dX = dgamma_h/dX (1 - E/N^2) + (delta/N) dE/dX + (delta^2 E/N^2) dK/dX
// ---------------------------------------------------------------------------
template <typename T>
struct StepGrad {
    Cx<T> dg, dP, dQ, dR;  // dPhi/dgamma, dPhi/dP, dPhi/dQ, dPhi/dR
};

template <typename T>
__host__ __device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
    return Cx<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

template <typename T>
__host__ __device__ __forceinline__ Cx<T> crcp(Cx<T> a) {
    const T r = Mth<T>::rcp(a.x * a.x + a.y * a.y);
    return Cx<T>{a.x * r, -a.y * r};
}

// One step from g over a segment with Delta = (dr, di), z = (zr, zi), length ell:
// returns gamma' in g_out and the derivatives in G.
template <typename T>
__host__ __device__ __forceinline__ void step_grad(T dr, T di, T zr, T zi, T ell, Cx<T> g, Cx<T> &g_out,
                                                   StepGrad<T> &G) {
    typedef Mth<T> M;
    typedef Cx<T> C;
    using ::copysign;
    using ::fabs;
    const T d2 = dr * dr + di * di;
    const T x = d2 - zr * zr + zi * zi;
    const T y = T(-2) * zr * zi;
    // |Omega|^2 = |Omega^2|: one reciprocal square root gives both r and the
    // 1/(2 Omega) factor below
    const T n2 = x * x + y * y;
    const T rn = M::rsqrt(n2);           // 1/|Omega|^2
    const T r = n2 * rn;                 // |Omega^2|
    const T hs = T(0.5) * (r + fabs(x));
    const T q = M::rsqrt(hs);
    const T s = hs * q;
    const T yq = T(0.5) * y * q;
    C Om;
    if (x >= T(0)) {
        Om.x = s;
        Om.y = yq;
    } else {
        Om.x = fabs(yq);
        Om.y = copysign(s, y);
    }
    const C z{zr, zi}, D{dr, di}, Dc{dr, -di};
    const C w{zr - Om.y, zi + Om.x};
    const C iw = crcp(w);
    const C i2O = crcp(C{T(2) * Om.x, T(2) * Om.y});  // 1/(2 Omega)
    const C gh = cmul(C{-dr, -di}, iw);
    const T eu = M::expneg(T(2) * ell * Om.x);
    T sn, cs;
    M::sincos_(T(2) * ell * Om.y, &sn, &cs);
    const C E{eu * cs, -eu * sn};
    const C c = cmul(C{T(1) - E.x, -E.y}, i2O);
    const C iDc_c = cmul(Dc, c);
    const C K{-iDc_c.y, iDc_c.x};  // i Delta* c
    const C del{g.x - gh.x, g.y - gh.y};
    const C Kd = cmul(K, del);
    const C N{T(1) - Kd.x, -Kd.y};
    const C iN = crcp(N);
    const C A2 = cmul(del, iN);                 // delta / N
    const C u = cmul(A2, E);
    g_out = C{gh.x + u.x, gh.y + u.y};
    const C EN2 = cmul(E, cmul(iN, iN));        // E / N^2
    G.dg = EN2;
    const C A1{T(1) - EN2.x, -EN2.y};
    const C A3 = cmul(cmul(del, del), EN2);      // delta^2 E / N^2
    // dOmega/dX
    const C OmP = cmul(D, i2O), OmR = cmul(Dc, i2O);
    const C OmQ = cmul(C{T(-2) * z.x, T(-2) * z.y}, i2O);
    // dgamma_h/dX
    const C gh2 = cmul(gh, gh);
    const C t1 = cmul(gh2, i2O);
    const C ghP{-t1.y, t1.x};
    const C t2 = cmul(gh, i2O);
    const C ghQ{T(-2) * t2.y, T(2) * t2.x};
    const C ghR{-i2O.y, i2O.x};
    // E_X = eX OmX, c_X = cX OmX
    const C eX{T(-2) * ell * E.x, T(-2) * ell * E.y};
    const C cX = cmul(C{T(2) * (ell * E.x - c.x), T(2) * (ell * E.y - c.y)}, i2O);
    const C iDcX = cmul(Dc, cX);
    const C Bk{-iDcX.y, iDcX.x};                 // i Delta* cX
    const C B1 = cmul(A2, eX), B2 = cmul(A3, Bk);
    const C B{B1.x + B2.x, B1.y + B2.y};
    const C ic{-c.y, c.x};
    const C p1 = cmul(ghP, A1), p2 = cmul(OmP, B), p3 = cmul(A3, ic);
    G.dP = C{p1.x + p2.x + p3.x, p1.y + p2.y + p3.y};
    const C q1 = cmul(ghQ, A1), q2 = cmul(OmQ, B);
    G.dQ = C{q1.x + q2.x, q1.y + q2.y};
    const C r1 = cmul(ghR, A1), r2 = cmul(OmR, B);
    G.dR = C{r1.x + r2.x, r1.y + r2.y};
}

// ---------------------------------------------------------------------------
// The same step as a Moebius map, for the adjoint sweep.  The Riccati equation
// d gamma/ds = i (Delta* gamma^2 + 2 z gamma + Delta) is the projective image of
// (u, v)' = M (u, v) with M = [[i z, i Delta], [-i Delta*, -i z]] (gamma = u/v),
// whose eigenvalues are +-Omega.  exp(M ell) = cosh(Omega ell) + sinh(Omega ell)
// M/Omega; scaled by 2 exp(-Omega ell), with E = exp(-2 Omega ell) and
// c2 = (1 - E)/Omega, its entries are
//   a = 1 + E + i z c2,  b = i Delta c2,  c = -i Delta* c2,  d = 1 + E - i z c2,
// and gamma' = (a gamma + b)/(c gamma + d), with ad - bc = 4E.
// ---------------------------------------------------------------------------
template <typename T>
struct MobCoef {
    Cx<T> a, b, c, d;  // gamma' = (a gamma + b)/(c gamma + d)
    Cx<T> E, c2, iO;   // exp(-2 Omega ell), (1 - E)/Omega, 1/Omega
};

template <typename T>
__host__ __device__ __forceinline__ void mob_assemble(T dr, T di, T zr, T zi, MobCoef<T> &m) {
    const T tr = zr * m.c2.x - zi * m.c2.y, ti = zr * m.c2.y + zi * m.c2.x;             // z c2
    const T ur = dr * m.c2.x - di * m.c2.y, ui = dr * m.c2.y + di * m.c2.x;             // Delta c2
    const T vr = dr * m.c2.x + di * m.c2.y, vi = dr * m.c2.y - di * m.c2.x;             // Delta* c2
    const T ope = T(1) + m.E.x;
    m.a = Cx<T>{ope - ti, m.E.y + tr};
    m.d = Cx<T>{ope + ti, m.E.y - tr};
    m.b = Cx<T>{-ui, ur};
    m.c = Cx<T>{vi, -vr};
}

template <typename T>
__host__ __device__ __forceinline__ void mob_coef(T dr, T di, T d2, T zr, T zi, T ell, MobCoef<T> &m) {
    typedef Mth<T> M;
    using ::copysign;
    using ::fabs;
    const T x = d2 - zr * zr + zi * zi;  // Re Omega^2
    const T y = T(-2) * zr * zi;         // Im Omega^2
    // |Omega|^2 = |Omega^2|: one reciprocal square root gives both r and the
    // 1/(2 Omega) factor below
    const T n2 = x * x + y * y;
    const T rn = M::rsqrt(n2);           // 1/|Omega|^2
    const T r = n2 * rn;                 // |Omega^2|
    const T hs = T(0.5) * (r + fabs(x));
    const T q = M::rsqrt(hs);
    const T s = hs * q;
    const T yq = T(0.5) * y * q;
    T Or, Oi;
    if (x >= T(0)) {
        Or = s;
        Oi = yq;
    } else {
        Or = fabs(yq);
        Oi = copysign(s, y);
    }
    const T ro = M::rcp(Or * Or + Oi * Oi);
    m.iO = Cx<T>{Or * ro, -Oi * ro};
    const T eu = M::expneg(T(2) * ell * Or);
    T sn, cs;
    M::sincos_(T(2) * ell * Oi, &sn, &cs);
    m.E = Cx<T>{eu * cs, -eu * sn};
    const T omr = T(1) - m.E.x, omi = -m.E.y;
    m.c2 = Cx<T>{omr * m.iO.x - omi * m.iO.y, omr * m.iO.y + omi * m.iO.x};
    mob_assemble<T>(dr, di, zr, zi, m);
}

// Coefficients of the same segment for z' = -conj(z) (the opposite direction of
// a Matsubara pair: z = a + i eps_n, z' = -a + i eps_n).  Omega^2 is conjugated,
// and so are Omega, E and c2.
template <typename T>
__host__ __device__ __forceinline__ void mob_coef_mirror(const MobCoef<T> &f, T dr, T di, T zr, T zi,
                                                         MobCoef<T> &m) {
    m.E = Cx<T>{f.E.x, -f.E.y};
    m.c2 = Cx<T>{f.c2.x, -f.c2.y};
    m.iO = Cx<T>{f.iO.x, -f.iO.y};
    mob_assemble<T>(dr, di, zr, zi, m);
}

template <typename T>
__host__ __device__ __forceinline__ Cx<T> mob_apply(const MobCoef<T> &m, Cx<T> g) {
    const Cx<T> n{m.a.x * g.x - m.a.y * g.y + m.b.x, m.a.x * g.y + m.a.y * g.x + m.b.y};
    const Cx<T> u = crcp(Cx<T>{m.c.x * g.x - m.c.y * g.y + m.d.x, m.c.x * g.y + m.c.y * g.x + m.d.y});
    return cmul(n, u);
}

// Derivatives of gamma' = Phi(gamma; P = Delta*, Q = z, R = Delta) in the
// Moebius form.  With u = 1/(c gamma + d) and Ab = gamma u, Bb = u,
// Cb = -gamma' gamma u, Db = -gamma' u (the partials of gamma' by a, b, c, d):
//   dPhi/dgamma = 4 E u^2
//   dPhi/dX = Omega_X S + i c2 (Ab dQ + Bb dR - Cb dP - Db dQ)     (X in P, Q, R)
//   S = -2 ell E (Ab + Db) + i kappa ((Ab - Db) z + Bb Delta - Cb Delta*)
//   kappa = dc2/dOmega = (2 ell E - c2)/Omega
//   Omega_R = Delta*/(2 Omega), Omega_P = Delta/(2 Omega), Omega_Q = -z/Omega
template <typename T>
__host__ __device__ __forceinline__ void mob_grad(const MobCoef<T> &m, T dr, T di, T zr, T zi, T ell, Cx<T> g,
                                                  StepGrad<T> &G) {
    typedef Cx<T> C;
    const C u = crcp(C{m.c.x * g.x - m.c.y * g.y + m.d.x, m.c.x * g.y + m.c.y * g.x + m.d.y});
    const C gp = cmul(C{m.a.x * g.x - m.a.y * g.y + m.b.x, m.a.x * g.y + m.a.y * g.x + m.b.y}, u);
    const C Ab = cmul(g, u);
    const C Db{-(gp.x * u.x - gp.y * u.y), -(gp.x * u.y + gp.y * u.x)};
    const C Cb = cmul(g, Db);
    const C u2 = cmul(u, u);
    const C Eu2 = cmul(m.E, u2);
    G.dg = C{T(4) * Eu2.x, T(4) * Eu2.y};
    const C kap = cmul(C{T(2) * ell * m.E.x - m.c2.x, T(2) * ell * m.E.y - m.c2.y}, m.iO);
    const C apd{Ab.x + Db.x, Ab.y + Db.y}, amd{Ab.x - Db.x, Ab.y - Db.y};
    const C t1 = cmul(m.E, apd);
    const C w1 = cmul(amd, C{zr, zi}), w2 = cmul(u, C{dr, di}), w3 = cmul(Cb, C{dr, -di});
    const C w{w1.x + w2.x - w3.x, w1.y + w2.y - w3.y};
    const C kw = cmul(kap, w);
    const T m2l = T(-2) * ell;
    const C S{m2l * t1.x - kw.y, m2l * t1.y + kw.x};          // -2 ell E (Ab + Db) + i kappa w
    const C SO = cmul(S, m.iO);                                // S / Omega
    const C sR = cmul(SO, C{T(0.5) * dr, T(-0.5) * di});       // S Delta*/(2 Omega)
    const C sP = cmul(SO, C{T(0.5) * dr, T(0.5) * di});        // S Delta/(2 Omega)
    const C sQ = cmul(SO, C{zr, zi});                          // S z / Omega
    const C cB = cmul(m.c2, u), cC = cmul(m.c2, Cb), cA = cmul(m.c2, amd);
    G.dR = C{sR.x - cB.y, sR.y + cB.x};
    G.dP = C{sP.x + cC.y, sP.y - cC.x};
    G.dQ = C{-sQ.x - cA.y, -sQ.y + cA.x};
}

// ---------------------------------------------------------------------------
// Implicit midpoint rule (App. C, Eq. riccati_midpoint):
//   g1 = g0 + ell f((g0 + g1)/2),   f(g) = i (Delta* g^2 + 2 z g + Delta),
// a quadratic c2 g1^2 + c1 g1 + c0 = 0 with c2 = i ell Delta*/4,
// c1 = 2 c2 g0 + i ell z - 1, c0 = (c1 - c2 g0 + 2) g0 + i ell Delta, whose root
// continuous in Delta is g1 = 2 c0/(-c1 + sqrt(c1^2 - 4 c2 c0)) (principal root;
// Re c1 < 0 for ell |Delta| < 2, so the denominator stays near 2).
// The per-segment factors c2 and i ell Delta are shared by all energies.
// ---------------------------------------------------------------------------
template <typename T>
struct MidSeg {
    Cx<T> c2;   // i ell Delta*/4
    Cx<T> ild;  // i ell Delta
    T ell;
};

template <typename T>
__host__ __device__ __forceinline__ MidSeg<T> mid_seg(T dr, T di, T ell) {
    const T q = T(0.25) * ell;
    return MidSeg<T>{Cx<T>{q * di, q * dr}, Cx<T>{-ell * di, ell * dr}, ell};
}

// principal square root of x + i y (Re >= 0), the branch logic of the step's Omega
template <typename T>
__host__ __device__ __forceinline__ Cx<T> csqrt_principal(T x, T y) {
    typedef Mth<T> M;
    using ::copysign;
    using ::fabs;
    // |Omega|^2 = |Omega^2|: one reciprocal square root gives both r and the
    // 1/(2 Omega) factor below
    const T n2 = x * x + y * y;
    const T rn = M::rsqrt(n2);           // 1/|Omega|^2
    const T r = n2 * rn;                 // |Omega^2|
    const T hs = T(0.5) * (r + fabs(x));
    const T q = M::rsqrt(hs);
    const T s = hs * q;
    const T yq = T(0.5) * y * q;
    if (x >= T(0)) return Cx<T>{s, yq};
    return Cx<T>{fabs(yq), copysign(s, y)};
}

template <typename T>
__host__ __device__ __forceinline__ Cx<T> midpoint_step(const MidSeg<T> &sg, T zr, T zi, Cx<T> g) {
    const Cx<T> c2g = cmul(sg.c2, g);
    const T lzr = sg.ell * zr, lzi = sg.ell * zi;
    // c1 = 2 c2 g + i ell z - 1;  c1 - c2 g + 2 = c2 g + i ell z + 1
    const Cx<T> c1{T(2) * c2g.x - lzi - T(1), T(2) * c2g.y + lzr};
    const Cx<T> u{c2g.x - lzi + T(1), c2g.y + lzr};
    const Cx<T> ug = cmul(u, g);
    const Cx<T> c0{ug.x + sg.ild.x, ug.y + sg.ild.y};
    const Cx<T> cc = cmul(sg.c2, c0);
    const Cx<T> dsc{c1.x * c1.x - c1.y * c1.y - T(4) * cc.x, T(2) * c1.x * c1.y - T(4) * cc.y};
    const Cx<T> sq = csqrt_principal<T>(dsc.x, dsc.y);
    const Cx<T> iden = crcp(Cx<T>{sq.x - c1.x, sq.y - c1.y});
    const Cx<T> r = cmul(c0, iden);
    return Cx<T>{T(2) * r.x, T(2) * r.y};
}

// Derivatives of the midpoint step g1 = Phi(g0; P = Delta*, Q = z, R = Delta)
// by implicit differentiation of g1 = g0 + ell f(m), m = (g0 + g1)/2:
//   (1 - ell f'/2) dg1 = (1 + ell f'/2) dg0 + ell (f_P dP + f_Q dQ + f_R dR),
//   f' = i (2 P m + 2 Q), f_P = i m^2, f_Q = 2 i m, f_R = i.
template <typename T>
__host__ __device__ __forceinline__ void midpoint_grad(const MidSeg<T> &sg, T dr, T di, T zr, T zi, Cx<T> g0,
                                                       StepGrad<T> &G) {
    typedef Cx<T> C;
    const C g1 = midpoint_step<T>(sg, zr, zi, g0);
    const C m{T(0.5) * (g0.x + g1.x), T(0.5) * (g0.y + g1.y)};
    // h = ell f'/2 = i ell (Delta* m + z)
    const C pm = cmul(C{dr, -di}, m);
    const C h{-sg.ell * (pm.y + zi), sg.ell * (pm.x + zr)};
    const C w = crcp(C{T(1) - h.x, -h.y});   // 1/(1 - ell f'/2)
    G.dg = cmul(C{T(1) + h.x, h.y}, w);
    const C lw{sg.ell * w.x, sg.ell * w.y};  // ell/(1 - ell f'/2)
    G.dR = C{-lw.y, lw.x};                   // i ell w
    const C mlw = cmul(m, lw);
    G.dQ = C{T(-2) * mlw.y, T(2) * mlw.x};    // 2 i m ell w
    const C m2lw = cmul(m, mlw);
    G.dP = C{-m2lw.y, m2lw.x};                // i m^2 ell w
}

}  // namespace scd
