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

template <>
struct Mth<double> {
    static __device__ __forceinline__ double rcp(double v) { return 1.0 / v; }
    static __device__ __forceinline__ double rsqrt(double v) { return 1.0 / ::sqrt(v); }
    static __device__ __forceinline__ double sqrt(double v) { return ::sqrt(v); }
    static __device__ __forceinline__ double expneg(double u) { return ::exp(-u); }
    static __device__ __forceinline__ void sincos_(double x, double *s, double *c) { ::sincos(x, s, c); }
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
__device__ __forceinline__ void step_coef(T dr, T di, T d2, T zr, T zi, T ell, StepCoef<T> &c) {
    typedef Mth<T> M;
    const T x = d2 - zr * zr + zi * zi;  // Re Omega^2
    const T y = T(-2) * zr * zi;         // Im Omega^2
    const T r = M::sqrt(x * x + y * y);
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
    // 1/w and 1/(2 Omega) from two reciprocals of squared moduli (the sweep is
    // bound by FP32 issue, not by the reciprocal unit)
    const T rw = M::rcp(wr * wr + wi * wi);
    const T iwr = wr * rw, iwi = -wi * rw;                    // 1/w
    const T ro = T(0.5) * M::rcp(Or * Or + Oi * Oi);
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
__device__ __forceinline__ void step_apply(const StepCoef<T> &c, Cx<T> &g) {
    const T dx = g.x - c.gh.x, dy = g.y - c.gh.y;
    const T nr = dx * c.E.x - dy * c.E.y, ni = dx * c.E.y + dy * c.E.x;
    const T dnr = T(1) - (c.K.x * dx - c.K.y * dy), dni = -(c.K.x * dy + c.K.y * dx);
    const T rd = Mth<T>::rcp(dnr * dnr + dni * dni);
    g.x = c.gh.x + (nr * dnr + ni * dni) * rd;
    g.y = c.gh.y + (ni * dnr - nr * dni) * rd;
}

}  // namespace scd
