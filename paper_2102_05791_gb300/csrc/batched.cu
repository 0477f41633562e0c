// Batched persistent solver: many independent meshes of uneven size, each
// simulated for n_steps backward-Euler steps (Eq. opt-be) and then
// differentiated by backpropagation through time (Sec. 4: implicit
// differentiation of each step, Eq. dLda-re-ordered, plus plain backprop of
// v1 = (x1 - x0)/h), all inside ONE kernel launch.
//
// Every CTA takes the next mesh (largest first) from an integer work counter
// and runs that mesh's whole forward rollout and backward pass: Newton-CG
// with backtracking for every step, then for every step in reverse the
// adjoint CG solve with FP64 refinement and the parameter VJP.  Between the
// phases of an iteration the CTA only needs __syncthreads, so a CG iteration
// costs a few microseconds instead of several kernel launches.  A mesh is
// always computed by one CTA with a fixed thread count and fixed-order sums,
// so results do not depend on which CTA takes it.
//
// Precision follows the single-mesh mixed path: FP32 HVP and CG vectors,
// FP64 state, gradient, energies, dot products and adjoint residuals.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "elem_math.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "softsim.h"

using namespace softsim;

namespace {

constexpr int kBatchThreads = 256;

struct BatchDev {
    int M = 0, dim = 0;
    const int64_t *voff = nullptr, *eoff = nullptr;  // [M+1]
    const int32_t *order = nullptr;                  // [M] processing order
    const double *X = nullptr, *mass = nullptr;      // [V][d], [V]
    const uint8_t *fixed = nullptr;                  // [V]
    const int32_t *conn = nullptr;                   // [E][d+1] mesh-local vertex ids
    const int64_t *vinc_ptr = nullptr;               // [V+1]
    const int32_t *vinc = nullptr;                   // [E*(d+1)] mesh-local corner ids (elem*(d+1)+corner)
    const float *e32 = nullptr;                      // SoA fields over E
    const double *e64 = nullptr;
    int64_t estride = 0;
    const double *mu = nullptr, *lam = nullptr;      // [M]
    double k = 0, grav = 0, kc = 0, dt = 0;
    double kf = 0, feps = 0;  // ground friction k_f and its height; kf == 0: off
    float k_f = 0, dt2_f = 0;  // FP32 copies of k and dt^2
    int cpow = 3, log_mode = 0, muscle = 0;
    double newton_rtol = 1e-8, adj_rtol = 1e-6;
    int max_newton = 100, max_cg = 500, max_adj_cg = 2000, max_ls = 30;
    // workspace [V][d]
    double *u = nullptr, *uhat = nullptr, *g = nullptr, *w64 = nullptr, *r64 = nullptr, *Hx = nullptr,
           *lacc = nullptr, *xbar = nullptr, *vbar = nullptr;
    double *fw = nullptr, *u0 = nullptr;  // friction: [V] 2 k_f ReLU(eps - y0), [V][d] x0 - X (kf > 0 only)
    float *u32 = nullptr, *d = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr;
    // FP32 HVP inputs fixed during one CG solve (no FP64 arithmetic or
    // conversion inside the CG loop; GB300's FP64 rate is 1/64 of FP32):
    float *a32 = nullptr;   // [E] the step's activations
    float *dg32 = nullptr;  // [V][2] vertex diagonal: horizontal (m + fw), vertical (m + h^2 contact'')
    float *c32 = nullptr;   // corners [E*(d+1)][d]
    double *c64 = nullptr;
    int *counter = nullptr;
    int *mstat = nullptr;   // [M][4]: status, newton iters, cg iters fwd, cg iters adj
    double *mgrad = nullptr;  // [M][3]: dL/dmu, dL/dlambda, dL/dk of each mesh over the rollout
};

struct Mesh {
    int64_t v0, e0;
    int nv, ne;
    double mu, lam;
    float mu_f, lam_f;
};

// Block-wide sum broadcast to every thread (fixed order).
__device__ double bsum(double v, double *red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Block-wide compensated sum of FP32 values (TwoSum pairs), as FP64,
// broadcast to every thread (fixed order).
__device__ double bsum_f(float v, double *red)
{
    float h = v, l = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, h, o), l2 = __shfl_down_sync(0xffffffffu, l, o);
        ds_merge(h, l, h2, l2);
    }
    float2 *rf = reinterpret_cast<float2 *>(red);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) rf[w] = make_float2(h, l);
    __syncthreads();
    if (w == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        h = in ? rf[lane].x : 0.0f;
        l = in ? rf[lane].y : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_down_sync(0xffffffffu, h, o), l2 = __shfl_down_sync(0xffffffffu, l, o);
            ds_merge(h, l, h2, l2);
        }
        if (lane == 0) red[32] = (double)h + (double)l;
    }
    __syncthreads();
    return red[32];
}

template <typename T, int D>
__device__ __forceinline__ void load_elem(const T *ed, int64_t stride, int64_t e, T B[D][D], T gv[D], T &W, T f[D])
{
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) B[i][j] = ed[(FI<D>::B + i * D + j) * stride + e];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        gv[i] = ed[(FI<D>::G + i) * stride + e];
        f[i] = ed[(FI<D>::F + i) * stride + e];
    }
    W = ed[FI<D>::W * stride + e];
}

// Edge matrix of a vertex field for element e of mesh m (field indexed globally).
template <typename T, typename S, int D>
__device__ __forceinline__ void edge_of(const S *x, const Mesh &m, const int lid[D + 1], T E[D][D])
{
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const T x0 = T(x[(m.v0 + lid[0]) * D + i]);
#pragma unroll
        for (int k = 0; k < D; ++k) E[i][k] = T(x[(m.v0 + lid[k + 1]) * D + i]) - x0;
    }
}

template <int D>
__device__ __forceinline__ void elem_ids(const BatchDev &b, int64_t e, int lid[D + 1])
{
#pragma unroll
    for (int k = 0; k <= D; ++k) lid[k] = b.conn[e * (D + 1) + k];
}

// Sum of the corners of mesh m touching local vertex lv (fixed order).
template <typename T, int D>
__device__ __forceinline__ void corner_sum(const BatchDev &b, const Mesh &m, const T *c, int lv, T acc[D])
{
#pragma unroll
    for (int q = 0; q < D; ++q) acc[q] = T(0);
    const int64_t v = m.v0 + lv;
    for (int64_t s = b.vinc_ptr[v]; s < b.vinc_ptr[v + 1]; ++s) {
        const int64_t base = (m.e0 * (D + 1) + b.vinc[s]) * D;
#pragma unroll
        for (int q = 0; q < D; ++q) acc[q] += c[base + q];
    }
}

template <typename T, int D>
__device__ __forceinline__ void put_corners(T *c, int64_t e, const T G[D][D])
{
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            c[(e * (D + 1) + j + 1) * D + i] = G[i][j];
            s += G[i][j];
        }
        c[(e * (D + 1)) * D + i] = -s;
    }
}

__device__ __forceinline__ double contact_d1(double y, double kc, int p)
{
    const double pen = y < 0.0 ? -y : 0.0;
    return pen > 0.0 ? -p * kc * (p == 2 ? pen : pen * pen) : 0.0;
}
__device__ __forceinline__ double contact_d2(double y, double kc, int p)
{
    const double pen = y < 0.0 ? -y : 0.0;
    return pen > 0.0 ? p * (p - 1) * kc * (p == 2 ? 1.0 : pen) : 0.0;
}

// ---------------------------------------------------------------- passes (CTA-wide)

// Muscle energy density from |F f|^2: contractile (k/2) a |F f|^2 or the
// active spring (k/2)(|F f|/a - 1)^2.
__device__ __forceinline__ double muscle_psi(const BatchDev &b, double a, double Ff2)
{
    if (!b.muscle) return 0.5 * b.k * a * Ff2;
    const double r = sqrt(Ff2) / a - 1.0;
    return 0.5 * b.k * r * r;
}

// FP64 gradient of the incremental potential at u; returns |g|^2 over free entries.
template <int D>
__device__ double grad_pass(const BatchDev &b, const Mesh &m, const double *a_t, double *red)
{
    const double s_el = b.dt * b.dt;
    for (int le = threadIdx.x; le < m.ne; le += blockDim.x) {
        const int64_t e = m.e0 + le;
        int lid[D + 1];
        elem_ids<D>(b, e, lid);
        double B[D][D], gv[D], W, f[D], Du[D][D], F[D][D], C[D][D];
        load_elem<double, D>(b.e64, b.estride, e, B, gv, W, f);
        edge_of<double, double, D>(b.u, m, lid, Du);
        mul<double, D>(Du, B, F, true);
        cof<double, D>(F, C);
        const double J = detF<double, D>(F, C);
        double l, cc, cp;
        log_terms<double>(b.log_mode, m.mu, m.lam, J, l, cc, cp);
        double Ff[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < D; ++q) s += F[i][q] * f[q];
            Ff[i] = s;
        }
        double ka = b.k * a_t[e];  // dpsi_m/dq = ka q
        if (b.muscle) {
            double s2 = 0.0, c2;
#pragma unroll
            for (int i = 0; i < D; ++i) s2 += Ff[i] * Ff[i];
            spring_terms<double>(W != 0.0, b.k, a_t[e], sqrt(s2), ka, c2);
        }
        double G[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < D; ++q) s += (m.mu * F[i][q] + cc * C[i][q]) * B[j][q];
                G[i][j] = s_el * W * (s + ka * Ff[i] * gv[j]);
            }
        put_corners<double, D>(b.c64, e, G);
    }
    __syncthreads();
    double g2 = 0.0;
    for (int lv = threadIdx.x; lv < m.nv; lv += blockDim.x) {
        const int64_t v = m.v0 + lv;
        double acc[D];
        corner_sum<double, D>(b, m, b.c64, lv, acc);
        const double mass = b.mass[v];
        const double y = b.X[v * D + 1] + b.u[v * D + 1];
        acc[1] += s_el * (mass * b.grav + contact_d1(y, b.kc, b.cpow));
#pragma unroll
        for (int q = 0; q < D; ++q) acc[q] += mass * (b.u[v * D + q] - b.uhat[v * D + q]);
        if (b.fw) {
            const double fv = b.fw[v];
#pragma unroll
            for (int q = 0; q < D; ++q)
                if (q != 1) acc[q] += fv * (b.u[v * D + q] - b.u0[v * D + q]);
        }
        const bool fx = b.fixed[v] != 0;
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const double o = fx ? 0.0 : acc[q];
            b.g[v * D + q] = o;
            g2 += o * o;
        }
    }
    return bsum(g2, red);
}

// FP64 incremental potential at u + t dir (dir may be null); returns E and the
// sum of |terms| through S.
template <int D>
__device__ double energy_pass(const BatchDev &b, const Mesh &m, const double *a_t, const double *dir, double t,
                              double *S, double *red)
{
    const double s_el = b.dt * b.dt;
    double E = 0.0, A = 0.0;
    for (int le = threadIdx.x; le < m.ne; le += blockDim.x) {
        const int64_t e = m.e0 + le;
        int lid[D + 1];
        elem_ids<D>(b, e, lid);
        double B[D][D], gv[D], W, f[D], Du[D][D], Dd[D][D], F[D][D], C[D][D];
        load_elem<double, D>(b.e64, b.estride, e, B, gv, W, f);
        edge_of<double, double, D>(b.u, m, lid, Du);
        if (dir) {
            edge_of<double, double, D>(dir, m, lid, Dd);
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int q = 0; q < D; ++q) Du[i][q] += t * Dd[i][q];
        }
        mul<double, D>(Du, B, F, true);
        cof<double, D>(F, C);
        const double J = detF<double, D>(F, C);
        double I1 = 0.0, Ff2 = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double ff = 0.0;
#pragma unroll
            for (int q = 0; q < D; ++q) {
                I1 += F[i][q] * F[i][q];
                ff += F[i][q] * f[q];
            }
            Ff2 += ff * ff;
        }
        double l;
        if (b.log_mode == 0)
            l = J > 0.0 ? log(J) : 0.0;
        else
            l = (J - 1.0) - 0.5 * (J - 1.0) * (J - 1.0);
        double w = s_el * W *
                   (0.5 * m.mu * (I1 - D) - m.mu * l + 0.5 * m.lam * l * l + muscle_psi(b, a_t[e], Ff2));
        if (b.log_mode == 0 && J <= 0.0) w = INFINITY;  // a NaN J (non-finite input) stays NaN
        E += w;
        A += fabs(w);
    }
    for (int lv = threadIdx.x; lv < m.nv; lv += blockDim.x) {
        const int64_t v = m.v0 + lv;
        const double mass = b.mass[v];
        double in = 0.0, yv = 0.0;
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const double uq = b.u[v * D + q] + (dir ? t * dir[v * D + q] : 0.0);
            const double rq = uq - b.uhat[v * D + q];
            in += 0.5 * mass * rq * rq;
            if (q == 1) yv = b.X[v * D + 1] + uq;
            else if (b.fw) {
                const double rf = uq - b.u0[v * D + q];
                in += 0.5 * b.fw[v] * rf * rf;
            }
        }
        const double pen = yv < 0.0 ? -yv : 0.0;
        const double w = s_el * (mass * b.grav * yv + b.kc * (b.cpow == 2 ? pen * pen : pen * pen * pen));
        E += w + in;
        A += fabs(w) + in;
    }
    const double Et = bsum(E, red);
    *S = bsum(A, red);
    return Et;
}

// y = (M + h^2 H(u)) v with pinned rows/columns dropped; returns v.y (FP64
// sum for T = double, compensated FP32 block sum for T = float).
template <typename T, int D>
__device__ double hvp_pass(const BatchDev &b, const Mesh &m, const double *a_t, const T *us, const T *v, T *y, T *c,
                           const T *ed, double *red)
{
    constexpr bool F32 = sizeof(T) == 4;
    const T s_el = pick<T>(b.dt * b.dt, b.dt2_f);
    const T mu = pick<T>(m.mu, m.mu_f), lam = pick<T>(m.lam, m.lam_f);
    const T kk = pick<T>(b.k, b.k_f);
    for (int le = threadIdx.x; le < m.ne; le += blockDim.x) {
        const int64_t e = m.e0 + le;
        int lid[D + 1];
        elem_ids<D>(b, e, lid);
        const T ae = F32 ? T(b.a32[e]) : T(a_t[e]);
        T B[D][D], gv[D], W, f[D], Du[D][D], Dv[D][D], F[D][D], dF[D][D], C[D][D], dC[D][D];
        load_elem<T, D>(ed, b.estride, e, B, gv, W, f);
        edge_of<T, T, D>(us, m, lid, Du);
        T vv[D + 1][D];
#pragma unroll
        for (int k = 0; k <= D; ++k) {
            const int64_t gvid = m.v0 + lid[k];
            const bool fx = b.fixed[gvid] != 0;
#pragma unroll
            for (int q = 0; q < D; ++q) vv[k][q] = fx ? T(0) : v[gvid * D + q];
        }
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) Dv[i][k] = vv[k + 1][i] - vv[0][i];
        mul<T, D>(Du, B, F, true);
        mul<T, D>(Dv, B, dF, false);
        cof<T, D>(F, C);
        dcof<T, D>(F, dF, dC);
        const T J = detF<T, D>(F, C);
        T dJ = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) dJ += C[i][j] * dF[i][j];
        T l, cc, cp;
        log_terms<T>(b.log_mode, mu, lam, J, l, cc, cp);
        const T ka = F32 ? kk * ae : T(b.k * a_t[e]);
        T dvg[D];  // (d2psi_m/dq2) dq with dq = Dv g
#pragma unroll
        for (int i = 0; i < D; ++i) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) s += Dv[i][k] * gv[k];
            dvg[i] = s;
        }
        if (b.muscle) {  // spring, q = F f = f + Du g
            T q[D], s2 = T(0), qdq = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                T s = f[i];
#pragma unroll
                for (int k = 0; k < D; ++k) s += Du[i][k] * gv[k];
                q[i] = s;
                s2 += s * s;
                qdq += s * dvg[i];
            }
            T c1, c2;
            spring_terms<T>(W != T(0), kk, ae, sqrt(s2), c1, c2);
#pragma unroll
            for (int i = 0; i < D; ++i) dvg[i] = c1 * dvg[i] + c2 * qdq * q[i];
        } else {
#pragma unroll
            for (int i = 0; i < D; ++i) dvg[i] *= ka;
        }
        T G[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                T s = T(0);
#pragma unroll
                for (int k = 0; k < D; ++k) s += (mu * dF[i][k] + cp * dJ * C[i][k] + cc * dC[i][k]) * B[j][k];
                G[i][j] = s_el * W * (s + dvg[i] * gv[j]);
            }
        put_corners<T, D>(c, e, G);
    }
    __syncthreads();
    T dot = T(0);
    for (int lv = threadIdx.x; lv < m.nv; lv += blockDim.x) {
        const int64_t vg = m.v0 + lv;
        T acc[D];
        corner_sum<T, D>(b, m, c, lv, acc);
        const bool fx = b.fixed[vg] != 0;
        T dh, dy;  // diagonal: horizontal axes (inertia + friction), y (inertia + contact)
        if constexpr (F32) {
            dh = b.dg32[2 * vg];
            dy = b.dg32[2 * vg + 1];
        } else {
            const double mass = b.mass[vg];
            const double yy = b.X[vg * D + 1] + us[vg * D + 1];
            dh = b.fw ? mass + b.fw[vg] : mass;  // friction stiffens the horizontal axes
            dy = mass + b.dt * b.dt * contact_d2(yy, b.kc, b.cpow);
        }
        T vv[D];
#pragma unroll
        for (int q = 0; q < D; ++q) vv[q] = fx ? T(0) : v[vg * D + q];
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const T o = fx ? T(0) : acc[q] + (q == 1 ? dy : dh) * vv[q];
            y[vg * D + q] = o;
            dot += vv[q] * o;
        }
    }
    if constexpr (F32)
        return bsum_f(dot, red);
    else
        return bsum(dot, red);
}

// CG on (M + h^2 H) d = rhs (FP64 rhs, FP32 vectors); returns iterations.
template <int D>
__device__ int cg_solve(const BatchDev &b, const Mesh &m, const double *a_t, const double *rhs, double rtol, int max_it,
                        double *red)
{
    const int64_t o = m.v0 * D, n = (int64_t)m.nv * D;
    float rr32 = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float ri = (float)rhs[o + i];
        b.r[o + i] = ri;
        b.p[o + i] = ri;
        b.d[o + i] = 0.0f;
        rr32 += ri * ri;
    }
    double rr = bsum_f(rr32, red);
    const double tol2 = rtol * rtol * rr;
    int k = 0;
    for (; k < max_it; ++k) {
        if (!(rr > tol2)) break;
        const double pAp = hvp_pass<float, D>(b, m, a_t, b.u32, b.p, b.Ap, b.c32, b.e32, red);
        if (!(pAp > 0.0)) {
            if (k == 0)
                for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b.d[o + i] = b.p[o + i];
            __syncthreads();
            break;
        }
        const float alpha = (float)(rr / pAp);
        float rn32 = 0.0f;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            b.d[o + i] += alpha * b.p[o + i];
            const float ri = b.r[o + i] - alpha * b.Ap[o + i];
            b.r[o + i] = ri;
            rn32 += ri * ri;
        }
        const double rn = bsum_f(rn32, red);
        const float beta = (float)(rn / rr);
        rr = rn;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b.p[o + i] = b.r[o + i] + beta * b.p[o + i];
        __syncthreads();
    }
    return k;
}

// FP32 state and vertex diagonals of mesh m for the CG solves at the current
// u (the caller synchronises before the next pass reads them).
template <int D>
__device__ void set_fp32_state(const BatchDev &b, const Mesh &m)
{
    const int64_t o = m.v0 * D, n = (int64_t)m.nv * D;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b.u32[o + i] = (float)b.u[o + i];
    for (int lv = threadIdx.x; lv < m.nv; lv += blockDim.x) {
        const int64_t v = m.v0 + lv;
        const double mass = b.mass[v];
        const double yy = b.X[v * D + 1] + b.u[v * D + 1];
        b.dg32[2 * v] = (float)(b.fw ? mass + b.fw[v] : mass);
        b.dg32[2 * v + 1] = (float)(mass + b.dt * b.dt * contact_d2(yy, b.kc, b.cpow));
    }
}

// FP32 activations of mesh m for this step.
__device__ void set_a32(const BatchDev &b, const Mesh &m, const double *a_t)
{
    for (int le = threadIdx.x; le < m.ne; le += blockDim.x) b.a32[m.e0 + le] = (float)a_t[m.e0 + le];
}

// Friction data of a step of mesh m started at x0: u0 = x0 - X and
// fw = 2 k_f ReLU(eps - y0) per vertex.
template <int D>
__device__ void friction_prep(const BatchDev &b, const Mesh &m, const double *x0)
{
    for (int lv = threadIdx.x; lv < m.nv; lv += blockDim.x) {
        const int64_t v = m.v0 + lv;
#pragma unroll
        for (int q = 0; q < D; ++q) b.u0[v * D + q] = x0[v * D + q] - b.X[v * D + q];
        const double r = b.feps - x0[v * D + 1];
        b.fw[v] = r > 0.0 ? 2.0 * b.kf * r : 0.0;
    }
}

// Backward-Euler step of mesh m: x1 = argmin of the incremental potential,
// started from x0; returns the step's status and adds iteration counts.
template <int D>
__device__ int step_forward(const BatchDev &b, const Mesh &m, const double *x0, const double *v0, const double *a_t,
                            double *x1, double *v1, int *newton_it, int *cg_it, double *red)
{
    const int64_t o = m.v0 * D, n = (int64_t)m.nv * D;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        b.u[o + i] = b.fixed[m.v0 + i / D] ? 0.0 : x0[o + i] - b.X[o + i];
        b.uhat[o + i] = x0[o + i] + b.dt * v0[o + i] - b.X[o + i];
    }
    if (b.fw) friction_prep<D>(b, m, x0);
    set_a32(b, m, a_t);
    __syncthreads();
    double S0;
    double gn = sqrt(grad_pass<D>(b, m, a_t, red));
    double E = energy_pass<D>(b, m, a_t, nullptr, 0.0, &S0, red);
    const double g0 = gn;
    int status = SIM_ENOTCONVERGED;
    const double eps = 2.220446049250313e-16;
    for (int it = 0;; ++it) {
        if (gn <= b.newton_rtol * g0) {
            status = SIM_OK;
            break;
        }
        if (it >= b.max_newton || !isfinite(gn) || !isfinite(E)) {
            status = (!isfinite(gn) || !isfinite(E)) ? SIM_ENAN : SIM_ENOTCONVERGED;
            break;
        }
        ++*newton_it;
        set_fp32_state<D>(b, m);
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b.w64[o + i] = -b.g[o + i];
        __syncthreads();
        const double eta = fmin(0.5, sqrt(gn / g0));
        *cg_it += cg_solve<D>(b, m, a_t, b.w64, eta, b.max_cg, red);
        double gd = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) gd += b.g[o + i] * (double)b.d[o + i];
        gd = bsum(gd, red);
        if (!(gd < 0.0)) {
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b.d[o + i] = (float)(-b.g[o + i]);
            gd = -gn * gn;
        }
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b.r64[o + i] = (double)b.d[o + i];
        __syncthreads();
        bool ok = false;
        double t = 1.0, Et = INFINITY, St = 0.0;
        for (int ls = 0; ls < b.max_ls; ++ls) {
            Et = energy_pass<D>(b, m, a_t, b.r64, t, &St, red);
            if (isfinite(Et) && Et <= E + 1e-4 * t * gd + 64.0 * eps * fmax(S0, St)) {
                ok = true;
                break;
            }
            t *= 0.5;
        }
        if (!ok) {
            status = SIM_ELINESEARCH;
            break;
        }
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b.u[o + i] += t * b.r64[o + i];
        __syncthreads();
        E = Et;
        S0 = St;
        gn = sqrt(grad_pass<D>(b, m, a_t, red));
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double xi = b.X[o + i] + b.u[o + i];
        x1[o + i] = xi;
        v1[o + i] = (xi - x0[o + i]) / b.dt;
    }
    __syncthreads();
    return status;
}

// Backward of one step at its converged state x1: lambda = (M + h^2 H)^-1
// (xbar + vbar/h) with FP64 refinement, then xbar <- M lambda - vbar/h,
// vbar <- h M lambda, abar_t = -h^2 lambda^T d2E/dx da.
template <int D>
__device__ int step_backward(const BatchDev &b, const Mesh &m, const double *x0, const double *x1, const double *a_t,
                             double *abar_t, int *cg_it, double mat[3], double *red)
{
    const int64_t o = m.v0 * D, n = (int64_t)m.nv * D;
    const double h = b.dt;
    if (b.fw) friction_prep<D>(b, m, x0);
    double bn = 0.0;
    set_a32(b, m, a_t);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        b.u[o + i] = x1[o + i] - b.X[o + i];
        const double bi = b.fixed[m.v0 + i / D] ? 0.0 : b.xbar[o + i] + b.vbar[o + i] / h;
        b.w64[o + i] = bi;
        b.r64[o + i] = bi;
        b.lacc[o + i] = 0.0;
        bn += bi * bi;
    }
    bn = sqrt(bsum(bn, red));
    set_fp32_state<D>(b, m);
    __syncthreads();
    double rn = bn;
    int status = SIM_ENOTCONVERGED;
    int budget = b.max_adj_cg;
    for (int pass = 0; pass < 12 && isfinite(bn); ++pass) {
        if (rn <= b.adj_rtol * bn || !(rn > 0.0)) {
            status = SIM_OK;
            break;
        }
        if (budget <= 0) break;
        const int it = cg_solve<D>(b, m, a_t, b.r64, fmax(fmax(b.adj_rtol, 1e-4), 0.5 * b.adj_rtol * bn / rn), budget,
                                   red);
        *cg_it += it;
        budget -= it > 0 ? it : 1;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b.lacc[o + i] += (double)b.d[o + i];
        __syncthreads();
        hvp_pass<double, D>(b, m, a_t, b.u, b.lacc, b.Hx, b.c64, b.e64, red);
        double r2 = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const double ri = b.w64[o + i] - b.Hx[o + i];
            b.r64[o + i] = ri;
            r2 += ri * ri;
        }
        const double rnew = sqrt(bsum(r2, red));
        if (!isfinite(rnew)) {
            status = SIM_ENAN;
            break;
        }
        if (rnew >= rn) {
            rn = rnew;
            break;
        }
        rn = rnew;
    }
    if (rn <= b.adj_rtol * bn) status = SIM_OK;
    if (!isfinite(bn)) status = SIM_ENAN;  // non-finite right-hand side
    // xbar0 = M lambda - vbar1/h, vbar0 = h M lambda; with friction, plus
    // fw lambda_h on the horizontal axes and 2 k_f [y0 < eps] lambda_h . (x1 - x0)_h on y
    for (int lv = threadIdx.x; lv < m.nv; lv += blockDim.x) {
        const int64_t v = m.v0 + lv;
        const bool fx = b.fixed[v] != 0;
        const double fv = b.fw ? b.fw[v] : 0.0;
        double ysum = 0.0;
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const int64_t i = v * D + q;
            const double l = b.lacc[i];
            const double ml = b.mass[v] * l;
            const double vb = b.vbar[i];
            double xb = ml - vb / h;
            if (q != 1 && fv > 0.0) {
                xb += fv * l;
                ysum += l * (x1[i] - x0[i]);
            }
            b.xbar[i] = fx ? 0.0 : xb;
            b.vbar[i] = fx ? 0.0 : h * ml;
        }
        if (fv > 0.0 && !fx) b.xbar[v * D + 1] += 2.0 * b.kf * ysum;
    }
    // parameter VJP at x1, and this step's material VJPs summed over the mesh:
    // -h^2 W (dP/dtheta) : dF(lambda), dP/dmu = F - l' cof F, dP/dlambda = l l' cof F
    double tmu = 0.0, tlam = 0.0, tk = 0.0;
    for (int le = threadIdx.x; le < m.ne; le += blockDim.x) {
        const int64_t e = m.e0 + le;
        int lid[D + 1];
        elem_ids<D>(b, e, lid);
        double B[D][D], gv[D], W, f[D], Du[D][D], Dl[D][D], F[D][D], dF[D][D], C[D][D];
        load_elem<double, D>(b.e64, b.estride, e, B, gv, W, f);
        edge_of<double, double, D>(b.u, m, lid, Du);
        edge_of<double, double, D>(b.lacc, m, lid, Dl);
        mul<double, D>(Du, B, F, true);
        mul<double, D>(Dl, B, dF, false);
        cof<double, D>(F, C);
        const double J = detF<double, D>(F, C);
        double FdF = 0.0, CdF = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                FdF += F[i][j] * dF[i][j];
                CdF += C[i][j] * dF[i][j];
            }
        double l, lp;
        if (b.log_mode == 0) {
            l = log(J);
            lp = 1.0 / J;
        } else {
            l = (J - 1.0) - 0.5 * (J - 1.0) * (J - 1.0);
            lp = 2.0 - J;
        }
        const double sW = -h * h * W;
        tmu += sW * (FdF - lp * CdF);
        tlam += sW * l * lp * CdF;
        double dot = 0.0, s2 = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double Ff = 0.0, dFf = 0.0;
#pragma unroll
            for (int q = 0; q < D; ++q) {
                Ff += F[i][q] * f[q];
                dFf += Dl[i][q] * gv[q];
            }
            dot += Ff * dFf;
            s2 += Ff * Ff;
        }
        double kq = b.k;                  // d2psi_m/dq da = kq q
        double ck = a_t[e];               // d2psi_m/dq dk = ck q
        if (b.muscle) {
            const double s = sqrt(s2), ia = 1.0 / a_t[e];
            kq = b.k * (ia * ia - 2.0 * s * ia * ia * ia) / s;
            ck = (s * ia - 1.0) * ia / s;
        }
        abar_t[e] = -h * h * W * kq * dot;
        tk += sW * ck * dot;
    }
    mat[0] += bsum(tmu, red);
    mat[1] += bsum(tlam, red);
    mat[2] += bsum(tk, red);
    __syncthreads();
    return status;
}

// BT threads per mesh CTA (128, 256 or 512; every variant may use up to
// 128 registers a thread).
template <int D, int BT>
__global__ void __launch_bounds__(BT, 512 / BT)
    k_batch_rollout(BatchDev b, int n_steps, const double *__restrict__ a_seq, double *xs, double *vs,
                    const double *__restrict__ xbarT, const double *__restrict__ vbarT, double *__restrict__ abar_seq,
                    int64_t V, int64_t E)
{
    __shared__ double red[33];
    __shared__ int sm_mesh;
    for (;;) {
        if (threadIdx.x == 0) sm_mesh = atomicAdd(b.counter, 1);
        __syncthreads();
        const int slot = sm_mesh;
        __syncthreads();
        if (slot >= b.M) break;
        const int mi = b.order[slot];
        Mesh m;
        m.v0 = b.voff[mi];
        m.e0 = b.eoff[mi];
        m.nv = (int)(b.voff[mi + 1] - m.v0);
        m.ne = (int)(b.eoff[mi + 1] - m.e0);
        m.mu = b.mu[mi];
        m.lam = b.lam[mi];
        m.mu_f = (float)m.mu;
        m.lam_f = (float)m.lam;
        int status = SIM_OK, newton_it = 0, cg_f = 0, cg_a = 0;
        const size_t VD = (size_t)V * D;
        for (int t = 0; t < n_steps; ++t) {
            const int st = step_forward<D>(b, m, xs + t * VD, vs + t * VD, a_seq + (size_t)t * E, xs + (t + 1) * VD,
                                           vs + (t + 1) * VD, &newton_it, &cg_f, red);
            if (st != SIM_OK) status = st;
        }
        const int64_t o = m.v0 * D, n = (int64_t)m.nv * D;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            b.xbar[o + i] = xbarT[o + i];
            b.vbar[o + i] = vbarT[o + i];
        }
        __syncthreads();
        double mat[3] = {0.0, 0.0, 0.0};
        for (int t = n_steps - 1; t >= 0; --t) {
            const int st = step_backward<D>(b, m, xs + t * VD, xs + (t + 1) * VD, a_seq + (size_t)t * E,
                                            abar_seq + (size_t)t * E, &cg_a, mat, red);
            if (st != SIM_OK && status == SIM_OK) status = st;
        }
        if (threadIdx.x == 0) {
            b.mgrad[3 * mi + 0] = mat[0];
            b.mgrad[3 * mi + 1] = mat[1];
            b.mgrad[3 * mi + 2] = mat[2];
            b.mstat[4 * mi + 0] = status;
            b.mstat[4 * mi + 1] = newton_it;
            b.mstat[4 * mi + 2] = cg_f;
            b.mstat[4 * mi + 3] = cg_a;
        }
        __syncthreads();
    }
}

thread_local std::string g_batch_error;

}  // namespace

using BatchKernel = void (*)(BatchDev, int, const double *, double *, double *, const double *, const double *,
                             double *, int64_t, int64_t);

static BatchKernel batch_kernel(int dim, int threads)
{
    if (dim == 2)
        return threads == 128 ? k_batch_rollout<2, 128> : threads == 512 ? k_batch_rollout<2, 512> : k_batch_rollout<2, 256>;
    return threads == 128 ? k_batch_rollout<3, 128> : threads == 512 ? k_batch_rollout<3, 512> : k_batch_rollout<3, 256>;
}

struct sim_batch {
    int M = 0, dim = 0;
    int64_t V = 0, E = 0;
    BatchDev dev;
    std::vector<void *> allocs;
    std::vector<int64_t> voff, eoff;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = -1;
    const void *graph_args[8] = {};
    int threads = kBatchThreads;  // threads per mesh CTA
    std::string err;
};

static int bfail(sim_batch *b, int code, const std::string &msg)
{
    if (b)
        b->err = msg;
    else
        g_batch_error = msg;
    return code;
}

#define BCK(b, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail((b), SIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename V>
static V *bupload(sim_batch *b, const std::vector<V> &v)
{
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(v.size() * sizeof(V), 16)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    b->allocs.push_back(p);
    if (!v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<V *>(p);
}

template <typename V>
static V *balloc(sim_batch *b, size_t n)
{
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n * sizeof(V), 16)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    b->allocs.push_back(p);
    return static_cast<V *>(p);
}

extern "C" const char *sim_batch_last_error(const sim_batch *b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

extern "C" int sim_batch_destroy(sim_batch *b)
{
    if (!b) return SIM_EINVAL;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (void *p : b->allocs) cudaFree(p);
    delete b;
    return SIM_OK;
}

static int batch_create_impl(sim_batch *bt, int M, const sim_mesh *meshes, const sim_material *mats,
                             const sim_options *opt)
{
    const int d = meshes[0].dim;
    const int nc = d + 1;
    bt->M = M;
    bt->dim = d;
    sim_options o;
    if (opt)
        o = *opt;
    else
        sim_default_options(&o);
    if (o.threads != 0 && o.threads != 128 && o.threads != 256 && o.threads != 512)
        return bfail(bt, SIM_EINVAL, "batched threads per mesh must be 0 (default 256), 128, 256 or 512");
    bt->threads = o.threads ? o.threads : kBatchThreads;
    bt->voff.assign(M + 1, 0);
    bt->eoff.assign(M + 1, 0);
    for (int m = 0; m < M; ++m) {
        if (meshes[m].dim != d) return bfail(bt, SIM_EINVAL, "all meshes of a batch must have the same dim");
        if (meshes[m].n_vert <= 0 || meshes[m].n_elem <= 0 || !meshes[m].rest_pos || !meshes[m].elems)
            return bfail(bt, SIM_EINVAL, "empty mesh in batch");
        if (!(mats[m].dt > 0.0)) return bfail(bt, SIM_EINVAL, "batched rollouts need dt > 0");
        bt->voff[m + 1] = bt->voff[m] + meshes[m].n_vert;
        bt->eoff[m + 1] = bt->eoff[m] + meshes[m].n_elem;
    }
    const sim_material &m0 = mats[0];
    for (int m = 1; m < M; ++m)
        if (mats[m].k_muscle != m0.k_muscle || mats[m].gravity != m0.gravity || mats[m].k_contact != m0.k_contact ||
            mats[m].contact_power != m0.contact_power || mats[m].log_mode != m0.log_mode || mats[m].dt != m0.dt ||
            mats[m].density != m0.density || mats[m].k_friction != m0.k_friction ||
            mats[m].eps_friction != m0.eps_friction || mats[m].muscle_model != m0.muscle_model)
            return bfail(bt, SIM_EINVAL, "batched meshes may differ only in mu and lambda");
    if (!(m0.k_friction >= 0.0) || !std::isfinite(m0.k_friction) || !std::isfinite(m0.eps_friction))
        return bfail(bt, SIM_EINVAL, "k_friction must be finite and >= 0, eps_friction finite");
    if (m0.contact_power != 2 && m0.contact_power != 3) return bfail(bt, SIM_EINVAL, "contact_power must be 2 or 3");
    if (m0.muscle_model != SIM_MUSCLE_CONTRACTILE && m0.muscle_model != SIM_MUSCLE_SPRING)
        return bfail(bt, SIM_EINVAL, "muscle_model must be SIM_MUSCLE_CONTRACTILE or SIM_MUSCLE_SPRING");
    const int64_t V = bt->voff[M], E = bt->eoff[M];
    bt->V = V;
    bt->E = E;
    const int nf = d * d + 2 * d + 1;
    std::vector<double> X(V * d), mass(V, 0.0), e64((size_t)nf * E, 0.0), mu(M), lam(M);
    std::vector<uint8_t> fixed(V, 0);
    std::vector<int32_t> conn(E * nc), vinc(E * nc);
    std::vector<int64_t> vinc_ptr(V + 1, 0);
    for (int m = 0; m < M; ++m) {
        const sim_mesh &mh = meshes[m];
        const int64_t v0 = bt->voff[m], e0 = bt->eoff[m];
        mu[m] = mats[m].mu;
        lam[m] = mats[m].lambda;
        for (int64_t i = 0; i < mh.n_vert * d; ++i) X[v0 * d + i] = mh.rest_pos[i];
        if (mh.fixed)
            for (int64_t i = 0; i < mh.n_vert; ++i) fixed[v0 + i] = mh.fixed[i] ? 1 : 0;
        for (int64_t e = 0; e < mh.n_elem; ++e) {
            const int32_t *t = mh.elems + e * nc;
            for (int k = 0; k < nc; ++k) {
                if (t[k] < 0 || t[k] >= mh.n_vert) return bfail(bt, SIM_EINVAL, "element vertex id out of range");
                conn[(e0 + e) * nc + k] = t[k];
                vinc_ptr[v0 + t[k] + 1] += 1;
            }
            double Dm[3][3] = {{0}}, B[3][3] = {{0}}, det;
            for (int k = 0; k < d; ++k)
                for (int i = 0; i < d; ++i) Dm[i][k] = mh.rest_pos[(int64_t)t[k + 1] * d + i] - mh.rest_pos[(int64_t)t[0] * d + i];
            if (d == 2) {
                det = Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0];
                B[0][0] = Dm[1][1] / det;
                B[0][1] = -Dm[0][1] / det;
                B[1][0] = -Dm[1][0] / det;
                B[1][1] = Dm[0][0] / det;
            } else {
                double C[3][3];
                for (int j = 0; j < 3; ++j) {
                    const int a = (j + 1) % 3, c = (j + 2) % 3;
                    C[0][j] = Dm[1][a] * Dm[2][c] - Dm[2][a] * Dm[1][c];
                    C[1][j] = Dm[2][a] * Dm[0][c] - Dm[0][a] * Dm[2][c];
                    C[2][j] = Dm[0][a] * Dm[1][c] - Dm[1][a] * Dm[0][c];
                }
                det = Dm[0][0] * C[0][0] + Dm[1][0] * C[1][0] + Dm[2][0] * C[2][0];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) B[i][j] = C[j][i] / det;
            }
            if (!(det > 0.0)) return bfail(bt, SIM_EINVERTED, "element with non-positive rest volume");
            const double W = det / (d == 2 ? 2.0 : 6.0);
            double f[3] = {0, 0, 0};
            if (mats[m].fiber)
                for (int c = 0; c < d; ++c) f[c] = mats[m].fiber[e * d + c];
            const int64_t ge = e0 + e;
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) e64[(size_t)(i * d + j) * E + ge] = B[i][j];
            for (int i = 0; i < d; ++i) {
                double s = 0.0;
                for (int j = 0; j < d; ++j) s += B[i][j] * f[j];
                e64[(size_t)(d * d + i) * E + ge] = s;
                e64[(size_t)(d * d + d + 1 + i) * E + ge] = f[i];
            }
            e64[(size_t)(d * d + d) * E + ge] = W;
            for (int k = 0; k < nc; ++k) mass[v0 + t[k]] += mats[m].density * W / nc;
        }
    }
    for (int64_t v = 0; v < V; ++v) vinc_ptr[v + 1] += vinc_ptr[v];
    {
        std::vector<int64_t> fill(vinc_ptr.begin(), vinc_ptr.end() - 1);
        for (int m = 0; m < M; ++m) {
            const int64_t v0 = bt->voff[m], e0 = bt->eoff[m], ne = bt->eoff[m + 1] - e0;
            for (int64_t e = 0; e < ne; ++e)
                for (int k = 0; k < nc; ++k) vinc[fill[v0 + conn[(e0 + e) * nc + k]]++] = (int32_t)(e * nc + k);
        }
    }
    std::vector<int32_t> order(M);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return bt->eoff[a + 1] - bt->eoff[a] > bt->eoff[c + 1] - bt->eoff[c];
    });
    std::vector<float> e32(e64.begin(), e64.end());
    BatchDev &b = bt->dev;
    b.M = M;
    b.dim = d;
    b.voff = bupload(bt, bt->voff);
    b.eoff = bupload(bt, bt->eoff);
    b.order = bupload(bt, order);
    b.X = bupload(bt, X);
    b.mass = bupload(bt, mass);
    b.fixed = bupload(bt, fixed);
    b.conn = bupload(bt, conn);
    b.vinc_ptr = bupload(bt, vinc_ptr);
    b.vinc = bupload(bt, vinc);
    b.e32 = bupload(bt, e32);
    b.e64 = bupload(bt, e64);
    b.estride = E;
    b.mu = bupload(bt, mu);
    b.lam = bupload(bt, lam);
    b.k = m0.k_muscle;
    b.grav = m0.gravity;
    b.kc = m0.k_contact;
    b.dt = m0.dt;
    b.kf = m0.k_friction;
    b.k_f = (float)m0.k_muscle;
    b.dt2_f = (float)(m0.dt * m0.dt);
    b.feps = m0.eps_friction;
    b.cpow = m0.contact_power;
    b.log_mode = m0.log_mode;
    b.muscle = m0.muscle_model;
    b.newton_rtol = o.newton_rtol;
    b.adj_rtol = o.adjoint_rtol;
    b.max_newton = o.max_newton;
    b.max_cg = o.max_cg;
    b.max_adj_cg = o.max_adjoint_cg > 0 ? o.max_adjoint_cg : 2000;
    b.max_ls = o.max_ls;
    const size_t VD = (size_t)V * d;
    b.u = balloc<double>(bt, VD);
    b.uhat = balloc<double>(bt, VD);
    b.g = balloc<double>(bt, VD);
    b.w64 = balloc<double>(bt, VD);
    b.r64 = balloc<double>(bt, VD);
    b.Hx = balloc<double>(bt, VD);
    b.lacc = balloc<double>(bt, VD);
    b.xbar = balloc<double>(bt, VD);
    b.vbar = balloc<double>(bt, VD);
    if (b.kf > 0.0) {
        b.fw = balloc<double>(bt, V);
        b.u0 = balloc<double>(bt, VD);
    }
    b.u32 = balloc<float>(bt, VD);
    b.a32 = balloc<float>(bt, (size_t)E);
    b.dg32 = balloc<float>(bt, (size_t)2 * V);
    b.d = balloc<float>(bt, VD);
    b.r = balloc<float>(bt, VD);
    b.p = balloc<float>(bt, VD);
    b.Ap = balloc<float>(bt, VD);
    b.c32 = balloc<float>(bt, (size_t)E * nc * d);
    b.c64 = balloc<double>(bt, (size_t)E * nc * d);
    b.counter = balloc<int>(bt, 1);
    b.mstat = balloc<int>(bt, (size_t)4 * M);
    b.mgrad = balloc<double>(bt, (size_t)3 * M);
    const void *ptrs[] = {b.voff, b.eoff, b.order, b.X, b.mass, b.fixed, b.conn, b.vinc_ptr, b.vinc, b.e32, b.e64,
                          b.mu, b.lam, b.u, b.uhat, b.g, b.w64, b.r64, b.Hx, b.lacc, b.xbar, b.vbar, b.u32,
                          b.d, b.r, b.p, b.Ap, b.c32, b.c64, b.counter, b.mstat, b.mgrad, b.a32, b.dg32};
    for (const void *p : ptrs)
        if (!p) return bfail(bt, SIM_ENOMEM, "device allocation or upload failed");
    if (b.kf > 0.0 && (!b.fw || !b.u0)) return bfail(bt, SIM_ENOMEM, "device allocation failed");
    return SIM_OK;
}

extern "C" int sim_batch_create(int n_meshes, const sim_mesh *meshes, const sim_material *mats,
                                const sim_options *opt, sim_batch **out)
{
    if (out) *out = nullptr;
    if (n_meshes <= 0 || !meshes || !mats || !out) return bfail(nullptr, SIM_EINVAL, "bad batch arguments");
    if (meshes[0].dim != 2 && meshes[0].dim != 3) return bfail(nullptr, SIM_EINVAL, "dim must be 2 or 3");
    sim_batch *b = new sim_batch();
    const int rc = batch_create_impl(b, n_meshes, meshes, mats, opt);
    if (rc != SIM_OK) {
        g_batch_error = b->err;
        sim_batch_destroy(b);
        return rc;
    }
    *out = b;
    return SIM_OK;
}

extern "C" int sim_batch_sizes(const sim_batch *b, int *n_meshes, int64_t *total_vert, int64_t *total_elem)
{
    if (!b) return SIM_EINVAL;
    if (n_meshes) *n_meshes = b->M;
    if (total_vert) *total_vert = b->V;
    if (total_elem) *total_elem = b->E;
    return SIM_OK;
}

extern "C" int sim_batch_rollout(sim_batch *bt, int n_steps, double *states_x, double *states_v, const double *a_seq,
                                 const double *xbarT, const double *vbarT, double *abar_seq, double *xbar0,
                                 double *vbar0, int *mesh_stats, double *mat_grad, void *stream)
{
    if (!bt) return SIM_EINVAL;
    if (n_steps <= 0 || !states_x || !states_v || !a_seq || !xbarT || !vbarT || !abar_seq || !xbar0 || !vbar0)
        return bfail(bt, SIM_EINVAL, "null or bad rollout argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const BatchDev &b = bt->dev;
    const size_t VD = (size_t)bt->V * bt->dim;
    int dev = 0, sms = 0, occ = 0;
    BCK(bt, cudaGetDevice(&dev));
    BCK(bt, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const BatchKernel kfun = batch_kernel(bt->dim, bt->threads);
    BCK(bt, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfun, bt->threads, 0));
    const int grid = std::max(1, std::min(bt->M, sms * std::max(occ, 1)));
    const void *args[8] = {states_x, states_v, a_seq, xbarT, vbarT, abar_seq, (const void *)(intptr_t)n_steps, nullptr};
    const bool reuse = bt->graph && bt->graph_steps == n_steps && memcmp(args, bt->graph_args, sizeof(args)) == 0;
    if (!reuse) {
        if (bt->graph) {
            cudaGraphExecDestroy(bt->graph);
            bt->graph = nullptr;
        }
        cudaStream_t cap;
        BCK(bt, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(b.counter, 0, sizeof(int), cap);
            kfun<<<grid, bt->threads, 0, cap>>>(b, n_steps, a_seq, states_x, states_v, xbarT, vbarT, abar_seq, bt->V,
                                                bt->E);
            e = cudaGetLastError();
            cudaError_t e2 = cudaStreamEndCapture(cap, &g);
            if (e == cudaSuccess) e = e2;
        }
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(bt, SIM_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&bt->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(bt, SIM_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
        bt->graph_steps = n_steps;
        memcpy(bt->graph_args, args, sizeof(args));
    }
    BCK(bt, cudaGraphLaunch(bt->graph, s));
    BCK(bt, cudaMemcpyAsync(xbar0, b.xbar, VD * sizeof(double), cudaMemcpyDeviceToDevice, s));
    BCK(bt, cudaMemcpyAsync(vbar0, b.vbar, VD * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (mesh_stats) BCK(bt, cudaMemcpyAsync(mesh_stats, b.mstat, sizeof(int) * 4 * bt->M, cudaMemcpyDeviceToDevice, s));
    if (mat_grad) BCK(bt, cudaMemcpyAsync(mat_grad, b.mgrad, sizeof(double) * 3 * bt->M, cudaMemcpyDeviceToDevice, s));
    return SIM_OK;
}
