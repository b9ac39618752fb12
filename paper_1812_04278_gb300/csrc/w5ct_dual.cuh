// w5ct_dual.cuh -- forward-mode dual numbers for the adjoint of the
// characteristic sweep: a value and N directional derivatives, with the
// arithmetic of w5ct_physics.cuh (operators and the M<> helpers).
//
// The face function of the sweep (six stencil cells of 8 values each ->
// 5 face fluxes + 2 CT transport fluxes) is evaluated with one stencil cell's
// 8 inputs seeded as the N = 8 directions; six such passes give the full
// 7 x 48 Jacobian, which the adjoint kernel contracts with the incoming
// adjoint of the fluxes.  Branches (max, |.|, the eps_B switches, the WENO-Z
// ratio clamp) follow the primal value, so the derivative is that of the
// branch the forward step takes (a consistent subgradient at ties).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "w5ct_physics.cuh"

namespace w5ct {

template <typename T, int N>
struct Dual {
    T v;
    T d[N];
    __device__ __forceinline__ Dual() {}
    __device__ __forceinline__ Dual(double c) : v((T)c) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = T(0);
    }
    // a constant of the base type itself (no detour through double)
    template <typename U, typename std::enable_if<std::is_same<U, T>::value && !std::is_same<T, double>::value,
                                                  int>::type = 0>
    __device__ __forceinline__ Dual(U c) : v(c) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = T(0);
    }
    __device__ __forceinline__ Dual &operator+=(const Dual &b) {
        v += b.v;
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] += b.d[i];
        return *this;
    }
    __device__ __forceinline__ Dual &operator-=(const Dual &b) {
        v -= b.v;
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] -= b.d[i];
        return *this;
    }
    __device__ __forceinline__ Dual &operator*=(const Dual &b) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = d[i] * b.v + v * b.d[i];
        v *= b.v;
        return *this;
    }
};

template <typename T, int N>
struct DualTraits<Dual<T, N>> {
    static constexpr bool is_dual = true;
    using base = T;
};

template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N> &a) {
    Dual<T, N> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const Dual<T, N> &a, const Dual<T, N> &b) {
    Dual<T, N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N> &a, const Dual<T, N> &b) {
    Dual<T, N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N> &a, const Dual<T, N> &b) {
    Dual<T, N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
// products with a constant of the base type (no tangent)
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N> &a, T c) {
    Dual<T, N> r;
    r.v = a.v * c;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * c;
    return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(T c, const Dual<T, N> &a) {
    return a * c;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator/(const Dual<T, N> &a, const Dual<T, N> &b) {
    Dual<T, N> r;
    const T ib = T(1) / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <typename T, int N>
__device__ __forceinline__ bool operator<(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v < b.v; }
template <typename T, int N>
__device__ __forceinline__ bool operator>(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v > b.v; }
template <typename T, int N>
__device__ __forceinline__ bool operator<=(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v <= b.v; }
template <typename T, int N>
__device__ __forceinline__ bool operator>=(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v >= b.v; }

// f(a) with f(a.v) = fv and f'(a.v) = df
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> chain(const Dual<T, N> &a, T fv, T df) {
    Dual<T, N> r;
    r.v = fv;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = df * a.d[i];
    return r;
}

template <typename T, int N>
struct M<Dual<T, N>> {
    using D = Dual<T, N>;
    static __device__ __forceinline__ D sqrt_(const D &x) {
        const T s = sqrt(x.v);
        return chain(x, s, s > T(0) ? T(0.5) / s : T(0));     // subgradient 0 at 0
    }
    static __device__ __forceinline__ D div_(const D &a, const D &b) { return a / b; }
    // -r (r x') and -r/2 (r (r x')): no r^2 or r^3 is formed, so a large r
    // (a tiny argument, e.g. eps + IS with IS = 0 in float) times a zero
    // tangent stays zero instead of inf * 0
    static __device__ __forceinline__ D rcp_(const D &x) {
        D y;
        y.v = T(1) / x.v;
#pragma unroll
        for (int i = 0; i < N; ++i) y.d[i] = -y.v * (y.v * x.d[i]);
        return y;
    }
    static __device__ __forceinline__ D rsqrt_(const D &x) {
        D y;
        y.v = T(1) / sqrt(x.v);
#pragma unroll
        for (int i = 0; i < N; ++i) y.d[i] = T(-0.5) * y.v * (y.v * (y.v * x.d[i]));
        return y;
    }
    static __device__ __forceinline__ D abs_(const D &x) { return x.v >= T(0) ? x : -x; }
    static __device__ __forceinline__ D max_(const D &a, const D &b) { return a.v >= b.v ? a : b; }
    static __device__ __forceinline__ D min_(const D &a, const D &b) { return a.v <= b.v ? a : b; }
    static __device__ __forceinline__ bool finite_pos(const D &x) { return M<T>::finite_pos(x.v); }
};

// Physical constants of the base type as constants (no tangent) of the dual type.
template <typename T, int N>
__device__ __forceinline__ Phys<Dual<T, N>> promote(const Phys<T> &K) {
    Phys<Dual<T, N>> D;
    D.gamma = Dual<T, N>(K.gamma);
    D.gm1 = Dual<T, N>(K.gm1);
    D.g1 = Dual<T, N>(K.g1);
    D.g2 = Dual<T, N>(K.g2);
    D.eps_w = Dual<T, N>(K.eps_w);
    D.eps_b = Dual<T, N>(K.eps_b);
    D.eps_b2 = Dual<T, N>(K.eps_b2);
    D.rho_min = Dual<T, N>(K.rho_min);
    D.p_min = Dual<T, N>(K.p_min);
    D.cs2_rel = Dual<T, N>(K.cs2_rel);
    D.floors = K.floors;
    return D;
}

}  // namespace w5ct
