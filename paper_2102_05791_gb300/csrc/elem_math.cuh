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

// The N words of a record (N even, record aligned to a pair) with pair
// loads: 8-byte in FP32, 16-byte in FP64.
template <typename T, int N>
__device__ __forceinline__ void load_pairs(const T *r, T out[N])
{
    static_assert(N % 2 == 0, "records are read in pairs");
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
        if constexpr (sizeof(T) == 4) {
            const float2 p = reinterpret_cast<const float2 *>(r)[q];
            out[2 * q] = p.x;
            out[2 * q + 1] = p.y;
        } else {
            const double2 p = reinterpret_cast<const double2 *>(r)[q];
            out[2 * q] = p.x;
            out[2 * q + 1] = p.y;
        }
    }
}

// Edge matrices of u and v from interleaved per-vertex records [u (D), v (D)]
// with 2D*sizeof(T) bytes each: every record is read with 8- or 16-byte
// vector loads (three float2 / double2 in 3D, one float4 or two double2 in
// 2D) instead of 2D scalar loads.  s must be 16-byte aligned.
template <typename T, int D>
__device__ __forceinline__ void load_uv(const T *s, int k, T u[D], T v[D])
{
    if constexpr (sizeof(T) == 4 && D == 3) {
        const float2 *r = reinterpret_cast<const float2 *>(s) + 3 * k;
        const float2 a = r[0], b = r[1], c = r[2];
        u[0] = a.x; u[1] = a.y; u[2] = b.x;
        v[0] = b.y; v[1] = c.x; v[2] = c.y;
    } else if constexpr (sizeof(T) == 4 && D == 2) {
        const float4 a = reinterpret_cast<const float4 *>(s)[k];
        u[0] = a.x; u[1] = a.y;
        v[0] = a.z; v[1] = a.w;
    } else {
        const double2 *r = reinterpret_cast<const double2 *>(s) + D * k;
        T w[2 * D];
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const double2 a = r[q];
            w[2 * q] = a.x;
            w[2 * q + 1] = a.y;
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            u[c] = w[c];
            v[c] = w[D + c];
        }
    }
}

template <typename T, int D>
__device__ __forceinline__ void edges_uv(const T *s, const int lid[D + 1], T Eu[D][D], T Ev[D][D])
{
    T u0[D], v0[D];
    load_uv<T, D>(s, lid[0], u0, v0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        T uk[D], vk[D];
        load_uv<T, D>(s, lid[k + 1], uk, vk);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            Eu[i][k] = uk[i] - u0[i];
            Ev[i][k] = vk[i] - v0[i];
        }
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
