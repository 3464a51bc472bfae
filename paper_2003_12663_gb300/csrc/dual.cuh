// dual.cuh -- forward-mode dual numbers (value + N directional derivatives) and
// the closed-form flat-triangle integrals written once for any scalar type, so
// that the adjoint can differentiate the near-pair integrals exactly.
#pragma once

#include "bem_internal.cuh"

template <int N>
struct Dual {
    double v;
    double d[N];
};

template <int N>
__device__ __forceinline__ Dual<N> dconst(double v)
{
    Dual<N> r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = 0.0;
    return r;
}

template <int N>
__device__ __forceinline__ Dual<N> dvar(double v, int k)
{
    Dual<N> r = dconst<N>(v);
    r.d[k] = 1.0;
    return r;
}

#define DUAL_BIN(OP, VAL, DER)                                                              \
    template <int N>                                                                        \
    __device__ __forceinline__ Dual<N> operator OP(const Dual<N>& a, const Dual<N>& b)      \
    {                                                                                       \
        Dual<N> r;                                                                          \
        r.v = VAL;                                                                          \
        _Pragma("unroll") for (int i = 0; i < N; ++i) r.d[i] = DER;                          \
        return r;                                                                           \
    }
DUAL_BIN(+, a.v + b.v, a.d[i] + b.d[i])
DUAL_BIN(-, a.v - b.v, a.d[i] - b.d[i])
DUAL_BIN(*, a.v * b.v, a.d[i] * b.v + a.v * b.d[i])
#undef DUAL_BIN

template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b)
{
    Dual<N> r;
    r.v = a.v / b.v;
    const double ib = 1.0 / b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}

template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a)
{
    Dual<N> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}

template <int N>
__device__ __forceinline__ Dual<N> operator*(double s, const Dual<N>& a)
{
    Dual<N> r;
    r.v = s * a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = s * a.d[i];
    return r;
}

template <int N>
__device__ __forceinline__ Dual<N> dscale1(const Dual<N>& a, double dv, double v)  // f(a) with f' = dv
{
    Dual<N> r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = dv * a.d[i];
    return r;
}

template <int N>
__device__ __forceinline__ Dual<N> sqrt(const Dual<N>& a)
{
    const double s = ::sqrt(a.v);
    return dscale1(a, 0.5 / s, s);
}

template <int N>
__device__ __forceinline__ Dual<N> log(const Dual<N>& a)
{
    return dscale1(a, 1.0 / a.v, ::log(a.v));
}

template <int N>
__device__ __forceinline__ Dual<N> log1p(const Dual<N>& a)
{
    return dscale1(a, 1.0 / (1.0 + a.v), ::log1p(a.v));
}

template <int N>
__device__ __forceinline__ Dual<N> atan2(const Dual<N>& y, const Dual<N>& x)
{
    Dual<N> r;
    r.v = ::atan2(y.v, x.v);
    const double q = 1.0 / (x.v * x.v + y.v * y.v);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) * q;
    return r;
}

__device__ __forceinline__ double val(double a) { return a; }
template <int N>
__device__ __forceinline__ double val(const Dual<N>& a) { return a.v; }

template <class T>
__device__ __forceinline__ T tconst(double v);
template <>
__device__ __forceinline__ double tconst<double>(double v) { return v; }
template <>
__device__ __forceinline__ Dual<3> tconst<Dual<3>>(double v) { return dconst<3>(v); }
template <>
__device__ __forceinline__ Dual<9> tconst<Dual<9>>(double v) { return dconst<9>(v); }

// Closed-form S and G of a flat triangle with vertices v[0..8] at x (the same
// formulas as tri_closed_form: edge line integrals in cancellation-free form, the
// signed solid angle of Van Oosterom & Strackee).  own: x is the triangle's own
// centroid (principal value of the normal field, h = 0).
template <class T>
__device__ void tri_cf_t(const T* v, const T* x, bool own, T& S, T* G)
{
    const T e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
    const T e2x = v[6] - v[3], e2y = v[7] - v[4], e2z = v[8] - v[5];
    const T wx = e1y * e2z - e1z * e2y, wy = e1z * e2x - e1x * e2z, wz = e1x * e2y - e1y * e2x;
    const T wn = sqrt(wx * wx + wy * wy + wz * wz);
    const T nx = wx / wn, ny = wy / wn, nz = wz / wn;
    T h = tconst<T>(0.0);
    if (!own) h = (x[0] - v[0]) * nx + (x[1] - v[1]) * ny + (x[2] - v[2]) * nz;
    T ax[3], ay[3], az[3], al[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ax[i] = v[3 * i] - x[0];
        ay[i] = v[3 * i + 1] - x[1];
        az[i] = v[3 * i + 2] - x[2];
        al[i] = sqrt(ax[i] * ax[i] + ay[i] * ay[i] + az[i] * az[i]);
    }
    T sdf = tconst<T>(0.0), fx = tconst<T>(0.0), fy = tconst<T>(0.0), fz = tconst<T>(0.0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int k = (i + 1) % 3;
        const T ex = ax[k] - ax[i], ey = ay[k] - ay[i], ez = az[k] - az[i];
        const T L = sqrt(ex * ex + ey * ey + ez * ez);
        const T tx = ex / L, ty = ey / L, tz = ez / L;
        const T mx = ty * nz - tz * ny, my = tz * nx - tx * nz, mz = tx * ny - ty * nx;
        const T s0 = ax[i] * tx + ay[i] * ty + az[i] * tz;
        const T s1 = ax[k] * tx + ay[k] * ty + az[k] * tz;
        const T r0 = al[i], r1 = al[k];
        const T d = ax[i] * mx + ay[i] * my + az[i] * mz;
        T f;
        if (val(s0) >= 0.0)
            f = log1p(L * (s0 + s1 + r0 + r1) / ((r0 + r1) * (r0 + s0)));
        else if (val(s1) <= 0.0)
            f = log1p(L * (r0 + r1 - s0 - s1) / ((r0 + r1) * (r1 - s1)));
        else
            f = log((r1 + s1) * (r0 - s0) / (d * d + h * h));
        // d f vanishes where d does, but its derivative f d' does not (a point whose
        // projection lies on the edge's line outside the edge); only on the edge itself
        // is f infinite (a singular field)
        if (isfinite(val(f))) sdf = sdf + d * f;
        fx = fx + mx * f;
        fy = fy + my * f;
        fz = fz + mz * f;
    }
    T om = tconst<T>(0.0);
    if (!own) {
        const T det = ax[0] * (ay[1] * az[2] - az[1] * ay[2]) - ay[0] * (ax[1] * az[2] - az[1] * ax[2]) +
                      az[0] * (ax[1] * ay[2] - ay[1] * ax[2]);
        const T d01 = ax[0] * ax[1] + ay[0] * ay[1] + az[0] * az[1];
        const T d02 = ax[0] * ax[2] + ay[0] * ay[2] + az[0] * az[2];
        const T d12 = ax[1] * ax[2] + ay[1] * ay[2] + az[1] * az[2];
        const T den = al[0] * al[1] * al[2] + d01 * al[2] + d02 * al[1] + d12 * al[0];
        om = 2.0 * atan2(det, den);
    }
    S = kInv4Pi * (sdf + h * om);
    G[0] = kInv4Pi * (fx - om * nx);
    G[1] = kInv4Pi * (fy - om * ny);
    G[2] = kInv4Pi * (fz - om * nz);
}
