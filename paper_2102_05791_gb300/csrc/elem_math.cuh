// Per-element math of the neo-Hookean + muscle model shared by the tiled
// kernels and the batched solver (device functions only).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace softsim {


// FP32 uses the hardware approximations (absolute log error < 2^-21 on
// [0.5, 2]; it enters the HVP at the 1e-6 relative level); FP64 is exact.
__device__ __forceinline__ float dlog(float x) { return __logf(x); }
__device__ __forceinline__ double dlog(double x) { return log(x); }
__device__ __forceinline__ float drcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double drcp(double x) { return 1.0 / x; }

template <int D>
struct FI {
    static constexpr int B = 0;               // Dm^-1, D*D fields row-major
    static constexpr int G = D * D;           // g = Dm^-1 f, D fields
    static constexpr int W = D * D + D;       // rest measure
    static constexpr int F = D * D + D + 1;   // fiber f, D fields
    static constexpr int N = D * D + 2 * D + 1;
};

template <typename T, int D>
__device__ __forceinline__ void cof(const T F[D][D], T C[D][D])
{
    if constexpr (D == 2) {
        C[0][0] = F[1][1];
        C[0][1] = -F[1][0];
        C[1][0] = -F[0][1];
        C[1][1] = F[0][0];
    } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int a = (j + 1) % 3, b = (j + 2) % 3;  // column j = F[:,a] x F[:,b]
            C[0][j] = F[1][a] * F[2][b] - F[2][a] * F[1][b];
            C[1][j] = F[2][a] * F[0][b] - F[0][a] * F[2][b];
            C[2][j] = F[0][a] * F[1][b] - F[1][a] * F[0][b];
        }
    }
}

template <typename T, int D>
__device__ __forceinline__ void dcof(const T F[D][D], const T dF[D][D], T C[D][D])
{
    if constexpr (D == 2) {
        C[0][0] = dF[1][1];
        C[0][1] = -dF[1][0];
        C[1][0] = -dF[0][1];
        C[1][1] = dF[0][0];
    } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int a = (j + 1) % 3, b = (j + 2) % 3;
            C[0][j] = dF[1][a] * F[2][b] - dF[2][a] * F[1][b] + F[1][a] * dF[2][b] - F[2][a] * dF[1][b];
            C[1][j] = dF[2][a] * F[0][b] - dF[0][a] * F[2][b] + F[2][a] * dF[0][b] - F[0][a] * dF[2][b];
            C[2][j] = dF[0][a] * F[1][b] - dF[1][a] * F[0][b] + F[0][a] * dF[1][b] - F[1][a] * dF[0][b];
        }
    }
}

// l(J), c(J) and c'(J) for P_el = mu F + c(J) cof(F).
template <typename T>
__device__ __forceinline__ void log_terms(int mode, T mu, T lam, T J, T &l, T &c, T &cp)
{
    if (mode == 0) {
        const T iJ = drcp(J);
        l = dlog(J);
        c = (lam * l - mu) * iJ;
        cp = (lam + mu - lam * l) * iJ * iJ;
    } else {
        const T jm = J - T(1);
        const T q = jm - T(0.5) * jm * jm;
        const T qp = T(1) - jm;
        l = q;
        c = (lam * q - mu) * qp;
        cp = lam * qp * qp - (lam * q - mu);
    }
}

// Active-spring muscle psi = (k/2)(s/a - 1)^2 of q = F f, s = |q|
// (Eq. active-spring-potential with s = l/l0): dpsi/dq = c1 q and
// (d2psi/dq2) dq = c1 dq + c2 (q . dq) q with c1 = k (s/a - 1)/(a s) and
// c2 = k/(a s^3).  A padding element (live = false) contributes nothing.
template <typename T>
__device__ __forceinline__ void spring_terms(bool live, T k, T a, T s, T &c1, T &c2)
{
    if (!live) {
        c1 = c2 = T(0);
        return;
    }
    const T ia = drcp(a), is = drcp(s);
    c1 = k * (s * ia - T(1)) * ia * is;
    c2 = k * ia * is * is * is;
}

template <typename T, int D>
__device__ __forceinline__ void load_B(const ElemDev<T> &ed, int64_t e, T B[D][D])
{
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) B[i][j] = __ldg(ed.field(FI<D>::B + i * D + j) + e);
}

// Edge matrix (columns k = vertex k+1 minus vertex 0) of a staged vertex field.
template <typename T, int D>
__device__ __forceinline__ void edges(const T *s, const int lid[D + 1], T E[D][D])
{
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const T v0 = s[lid[0] * D + i];
#pragma unroll
        for (int k = 0; k < D; ++k) E[i][k] = s[lid[k + 1] * D + i] - v0;
    }
}

// M = A B (D x D), plus the identity when add_eye.
template <typename T, int D>
__device__ __forceinline__ void mul(const T A[D][D], const T B[D][D], T M[D][D], bool add_eye)
{
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            T s = (add_eye && i == j) ? T(1) : T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) s += A[i][k] * B[k][j];
            M[i][j] = s;
        }
}

template <typename T, int D>
__device__ __forceinline__ T detF(const T F[D][D], const T C[D][D])
{
    T J = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) J += F[i][0] * C[i][0];
    return J;
}

template <int D>
__device__ __forceinline__ void unpack(uint32_t cw, int lid[D + 1])
{
#pragma unroll
    for (int k = 0; k <= D; ++k) lid[k] = (cw >> (8 * k)) & 0xffu;
}


}  // namespace softsim
