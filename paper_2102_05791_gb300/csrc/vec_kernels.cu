// Vector kernels of the conjugate-gradient and Newton loops.
//
// CG (Sec. 3: the adjoint system is solved matrix-free by conjugate
// gradients; the same CG gives the Newton direction) keeps its scalars in
// device memory: the HVP tile kernel and k_cg_alpha form p.Ap and alpha,
// k_cg_update_halo and k_cg_beta form r.r and beta and raise `done`, so a
// whole block of iterations runs without a host round trip and can be
// captured in a CUDA graph.  Reductions are fixed-order; vectors are float
// (mixed precision) or double.  In the float CG loop (GB300's FP64 rate is
// 1/64 of FP32) r.r is summed in compensated FP32 at every level above a
// single term (per thread, over a block, over the blocks' (hi, lo) pairs);
// p.Ap is summed in plain FP32 within a tile (inside the HVP tile kernel)
// and with compensation over the tiles.  The double loop sums in FP64.
#include <algorithm>

#include "internal.h"
#include "reduce.cuh"
#include "pdl.cuh"

namespace softsim {

static inline int vec_grid(int64_t n)
{
    int64_t g = (n + 1023) / 1024;
    if (g < 1) g = 1;
    if (g > 1216) g = 1216;  // 152 SMs x 8
    return (int)g;
}

// Grids of the CG loop's vector kernels: every thread takes one vertex
// (update) or four consecutive entries (direction) and issues all of its
// loads at once, so each kernel waits on DRAM about once instead of once per
// grid-stride step.
static inline int cg_vert_grid(int64_t nv) { return (int)std::max<int64_t>(1, (nv + 255) / 256); }
static inline int cg_vec4_grid(int64_t n) { return (int)std::max<int64_t>(1, ((n + 3) / 4 + 255) / 256); }

template <typename T>
__global__ void __launch_bounds__(256) k_cg_init(int64_t n, const double *__restrict__ b, double sign,
                                                 T *__restrict__ d, T *__restrict__ r, T *__restrict__ p, double rtol,
                                                 int max_iter, int max_rounds, double *__restrict__ partials,
                                                 DevScalars *sc)
{
    double rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T ri = T(sign * b[i]);
        r[i] = ri;
        p[i] = ri;
        d[i] = T(0);
        rr += (double)ri * (double)ri;
    }
    const double s = block_sum(rr);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(&sc->ticket[TK_CGINIT], gridDim.x)) {
        const double tot = sum_partials(partials, gridDim.x);
        if (threadIdx.x == 0) {
            sc->rr = tot;
            sc->tol2 = rtol * rtol * tot;
            sc->iter = 0;
            sc->max_iter = max_iter;
            sc->negcurv = 0;
            sc->alpha = sc->beta = sc->pAp = 0.0;
            sc->alpha_f = sc->beta_f = 0.0f;
            sc->done = (tot <= sc->tol2 || max_iter <= 0 || !isfinite(tot)) ? 1 : 0;
            sc->cg_rounds = 0;
            sc->cg_max_rounds = max_rounds;
        }
    }
}

// Sets the WHILE condition of the device-side CG loop after each body round;
// the round cap ends the loop even if `done` were never raised.
__global__ void k_cg_cond(cudaGraphConditionalHandle hnd, DevScalars *sc)
{
    const int r = ++sc->cg_rounds;
    cudaGraphSetConditional(hnd, (!sc->done && !sc->kerr && r < sc->cg_max_rounds) ? 1u : 0u);
}

// d += alpha p, r -= alpha A p, r.r -> beta / done, with A p completed here for
// halo vertices (partial sums in tile order + per-vertex terms).
template <typename T, int D>
__global__ void __launch_bounds__(256) k_cg_update_halo(TileDev td, VertDev vd, Phys ph, const T *__restrict__ u,
                                                        T *__restrict__ d, T *__restrict__ r, const T *__restrict__ p,
                                                        const T *__restrict__ Ap, const T *__restrict__ hp,
                                                        double *__restrict__ partials, DevScalars *sc)
{
    pdl_trigger();
    pdl_wait();  // upstream results are visible past this point
    if (sc->done) return;
    const bool neg = sc->negcurv != 0;
    const bool first = sc->iter == 0;
    const T alpha = pick<T>(sc->alpha, sc->alpha_f);
    const bool contact = ph.kc > 0.0;
    CompSum<T> rr;  // r.r of this thread's vertices (compensated in FP32)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vd.nv;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (neg) {
            if (first)
#pragma unroll
                for (int c = 0; c < D; ++c) d[i * D + c] = p[i * D + c];
            continue;
        }
        // every load of the vertex is issued before any is used (Ap is read at
        // halo vertices too and ignored there)
        const int f = td.vfin[i];
        T a[D], pv[D], rv[D], dv[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            a[c] = Ap[i * D + c];
            pv[c] = p[i * D + c];
            rv[c] = r[i * D + c];
            dv[c] = d[i * D + c];
        }
        if (f >= 0) {
            const bool fx = vd.fixed[i] != 0;
#pragma unroll
            for (int c = 0; c < D; ++c) a[c] = T(0);
            for (int s = td.fin_ptr[f]; s < td.fin_ptr[f + 1]; ++s)
#pragma unroll
                for (int c = 0; c < D; ++c) a[c] += hp[(int64_t)s * D + c];
            if (contact) {
                const double yy = vd.X[i * D + 1] + (double)u[i * D + 1];
                const double pen = yy < 0.0 ? -yy : 0.0;
                const double d2 = pen > 0.0 ? ph.cpow * (ph.cpow - 1) * ph.kc * (ph.cpow == 2 ? 1.0 : pen) : 0.0;
                a[1] += T(ph.s_el * d2) * pv[1];
            }
            if (ph.dyn) {
                const T m = T(vd.mass[i]);
                const T mh = ph.fw ? m + T(ph.fw[i]) : m;
#pragma unroll
                for (int c = 0; c < D; ++c) a[c] += (c == 1 ? m : mh) * pv[c];
            }
            if (fx)
#pragma unroll
                for (int c = 0; c < D; ++c) a[c] = T(0);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            d[i * D + c] = dv[c] + alpha * pv[c];
            const T ri = rv[c] - alpha * a[c];
            r[i * D + c] = ri;
            rr.add(ri * ri);
        }
    }
    store_block_partial<T>(rr, partials + blockIdx.x);  // reduced by k_cg_beta<T>
}

// One block: p.Ap from the HVP tile partials -> alpha (or non-positive curvature).
// T is the CG precision (float: FP32 tile partials, summed with compensation).
template <typename T>
__global__ void __launch_bounds__(1024) k_cg_alpha(const double *__restrict__ partials, int n, DevScalars *sc)
{
    pdl_trigger();
    pdl_wait();  // upstream results are visible past this point
    if (sc->done) return;
    const double pAp = sum_partials(reinterpret_cast<const T *>(partials), n);
    if (threadIdx.x == 0) {
        sc->pAp = pAp;
        if (pAp > 0.0 && isfinite(pAp)) {
            sc->alpha = sc->rr / pAp;
            sc->alpha_f = (float)sc->alpha;
        } else {
            sc->alpha = 0.0;
            sc->alpha_f = 0.0f;
            sc->negcurv = 1;
        }
    }
}

// One block: the HVP tile kernel's v.Av partials summed as k_cg_alpha sums
// them, into *out (for sim_hvp_dot).
template <typename T>
__global__ void __launch_bounds__(1024) k_tile_dot(const double *__restrict__ partials, int n, double *out)
{
    const double v = sum_partials(reinterpret_cast<const T *>(partials), n);
    if (threadIdx.x == 0) *out = v;
}

// One block: r.r from the update partials -> beta, iteration count, done.
template <typename T>
__global__ void __launch_bounds__(1024) k_cg_beta(const double *__restrict__ partials, int n, DevScalars *sc)
{
    pdl_trigger();
    pdl_wait();  // upstream results are visible past this point
    if (sc->done) return;
    const double tot = sum_block_partials<T>(partials, n);
    if (threadIdx.x == 0) {
        if (sc->negcurv) {
            sc->done = 1;
        } else {
            sc->beta = tot / sc->rr;
            sc->beta_f = (float)sc->beta;
            sc->rr = tot;
            sc->iter += 1;
            if (tot <= sc->tol2 || sc->iter >= sc->max_iter || !isfinite(tot)) sc->done = 1;
        }
    }
}

// Four entries of a vector in one aligned load or store (the vectors are
// allocated with 256-byte alignment).
template <typename T>
struct alignas(4 * sizeof(T)) Vec4 {
    T v[4];
};

template <typename T>
__global__ void __launch_bounds__(256) k_cg_dir(int64_t n, T *__restrict__ p, const T *__restrict__ r,
                                                const DevScalars *sc)
{
    pdl_trigger();
    pdl_wait();  // upstream results are visible past this point
    if (sc->done) return;
    const T beta = pick<T>(sc->beta, sc->beta_f);
    // four consecutive entries per thread and step, both loads issued first
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, n4 = n >> 2;
    for (int64_t j = q; j < n4; j += (int64_t)gridDim.x * blockDim.x) {
        Vec4<T> pv = reinterpret_cast<const Vec4<T> *>(p)[j];
        const Vec4<T> rv = reinterpret_cast<const Vec4<T> *>(r)[j];
#pragma unroll
        for (int k = 0; k < 4; ++k) pv.v[k] = rv.v[k] + beta * pv.v[k];
        reinterpret_cast<Vec4<T> *>(p)[j] = pv;
    }
    const int64_t t = (n4 << 2) + q;  // the last n mod 4 entries
    if (t < n) p[t] = r[t] + beta * p[t];
}

template <typename T>
__global__ void __launch_bounds__(256) k_dir_check(int64_t n, const double *__restrict__ g, const T *__restrict__ d,
                                                   double *__restrict__ partials, DevScalars *sc)
{
    double gd = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        gd += g[i] * (double)d[i];
    const double s = block_sum(gd);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(&sc->ticket[TK_GD], gridDim.x)) {
        const double tot = sum_partials(partials, gridDim.x);
        if (threadIdx.x == 0) {
            if (tot < 0.0 && isfinite(tot)) {
                sc->gd = tot;
                sc->dir_fix = 0;
            } else {
                sc->gd = -sc->gn2;
                sc->dir_fix = 1;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_dir_fix(int64_t n, const double *__restrict__ g, T *__restrict__ d,
                                                 const DevScalars *sc)
{
    if (!sc->dir_fix) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = T(-g[i]);
}

template <typename T>
__global__ void k_step_update(int64_t n, double *__restrict__ u, const T *__restrict__ d, double t,
                              float *__restrict__ u32)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ui = u[i] + t * (double)d[i];
        u[i] = ui;
        if (u32) u32[i] = (float)ui;
    }
}

__global__ void k_x_to_u(int64_t nv, int dim, const double *__restrict__ x, const double *__restrict__ X,
                         const uint8_t *__restrict__ fixed, double *__restrict__ u, float *__restrict__ u32)
{
    const int64_t n = nv * dim;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ui = (fixed && fixed[i / dim]) ? 0.0 : x[i] - X[i];
        u[i] = ui;
        if (u32) u32[i] = (float)ui;
    }
}

__global__ void k_u_to_x(int64_t n, const double *__restrict__ u, const double *__restrict__ X, double *__restrict__ x)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = X[i] + u[i];
}

__global__ void k_uhat(int64_t n, const double *__restrict__ x0, const double *__restrict__ v0, double dt,
                       const double *__restrict__ X, double *__restrict__ uhat)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        uhat[i] = (x0[i] + dt * v0[i]) - X[i];
}

template <typename T>
__global__ void k_gather_elem(int64_t ne_int, const int32_t *__restrict__ perm, const double *__restrict__ user,
                              T *__restrict__ internal, int64_t stride)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne_int; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t pe = perm[e];
        internal[e * stride] = pe >= 0 ? T(user[pe]) : T(0);
    }
}

template <typename Tin, typename Tout>
__global__ void k_convert(int64_t n, const Tin *__restrict__ in, Tout *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = Tout(in[i]);
}

__global__ void k_mask_copy(int64_t nv, int dim, const uint8_t *__restrict__ fixed, const double *__restrict__ in,
                            double *__restrict__ out)
{
    const int64_t n = nv * dim;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = fixed[i / dim] ? 0.0 : in[i];
}

// Friction data of one backward-Euler step: the start displacement
// u0 = x0 - X and the weight fw = 2 k_f ReLU(eps - y0) of every vertex.
__global__ void k_friction_prep(int64_t nv, int dim, const double *__restrict__ x0, const double *__restrict__ X,
                                double kf, double eps, double *__restrict__ u0, double *__restrict__ fw)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < dim; ++c) u0[i * dim + c] = x0[i * dim + c] - X[i * dim + c];
        const double r = eps - x0[i * dim + 1];
        fw[i] = r > 0.0 ? 2.0 * kf * r : 0.0;
    }
}

// xbar0 = M lambda - vbar1/dt, vbar0 = dt M lambda, plus, with friction
// (fw non-null), the derivative of fw_i (x1 - x0)_h by x0: fw_i lambda_h on
// the horizontal axes and 2 k_f [y0 < eps] lambda_h . (x1 - x0)_h on y.
__global__ void k_step_bwd_combine(int64_t nv, int dim, const uint8_t *__restrict__ fixed,
                                   const double *__restrict__ mass, const double *__restrict__ lam,
                                   const double *__restrict__ vbar1, double dt, const double *__restrict__ fw,
                                   double kf, const double *__restrict__ x0, const double *__restrict__ x1,
                                   double *__restrict__ xbar0, double *__restrict__ vbar0)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        const bool fx = fixed[v] != 0;
        const double m = mass[v];
        const double f = fw ? fw[v] : 0.0;
        double ysum = 0.0;
        for (int c = 0; c < dim; ++c) {
            const int64_t i = v * dim + c;
            const double l = lam[i];
            double xb = m * l - vbar1[i] / dt;
            if (c != 1 && f > 0.0) {
                xb += f * l;
                ysum += l * (x1[i] - x0[i]);
            }
            xbar0[i] = fx ? 0.0 : xb;
            vbar0[i] = fx ? 0.0 : dt * m * l;
        }
        if (f > 0.0 && !fx) xbar0[v * dim + 1] += 2.0 * kf * ysum;
    }
}

__global__ void k_axpy_out(int64_t n, const double *__restrict__ x, const double *__restrict__ y, double beta,
                           double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = x[i] + beta * y[i];
}

__global__ void k_velocity(int64_t n, const double *__restrict__ x1, const double *__restrict__ x0, double dt,
                           double *__restrict__ v1)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v1[i] = (x1[i] - x0[i]) / dt;
}

// r = b - Ax (FP64) and |r|^2 into sc->gn2 (used by the adjoint refinement).
__global__ void __launch_bounds__(256) k_residual(int64_t n, const double *__restrict__ b, const double *__restrict__ Ax,
                                                  double *__restrict__ r, double *__restrict__ partials, DevScalars *sc)
{
    double rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = b[i] - (Ax ? Ax[i] : 0.0);
        r[i] = ri;
        rr += ri * ri;
    }
    const double s = block_sum(rr);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(&sc->ticket[TK_MISC], gridDim.x)) {
        const double tot = sum_partials(partials, gridDim.x);
        if (threadIdx.x == 0) sc->gn2 = tot;
    }
}

template <typename T>
__global__ void k_accumulate(int64_t n, double *__restrict__ x, const T *__restrict__ d)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

// ---------------------------------------------------------------- launchers

void launch_residual(const Ctx &c, const double *b, const double *Ax, double *r, cudaStream_t s)
{
    c.n_launch += 1;
    const int64_t n = c.nv * c.dim;
    k_residual<<<vec_grid(n), 256, 0, s>>>(n, b, Ax, r, c.partials, c.sc);
}

template <typename T>
void launch_accumulate(const Ctx &c, double *x, const T *d, cudaStream_t s)
{
    c.n_launch += 1;
    const int64_t n = c.nv * c.dim;
    k_accumulate<T><<<vec_grid(n), 256, 0, s>>>(n, x, d);
}

template <typename T>
void launch_cg_init(const Ctx &c, const double *b, double sign, T *d, T *r, T *p, double rtol, int max_iter,
                    int max_rounds, cudaStream_t s)
{
    c.n_launch += 1;
    const int64_t n = c.nv * c.dim;
    k_cg_init<T><<<vec_grid(n), 256, 0, s>>>(n, b, sign, d, r, p, rtol, max_iter, max_rounds, c.partials, c.sc);
}

void launch_cg_cond(const Ctx &c, cudaGraphConditionalHandle hnd, cudaStream_t s)
{
    k_cg_cond<<<1, 1, 0, s>>>(hnd, c.sc);
}

template <typename T>
void launch_cg_update_halo(const Ctx &c, const Phys &ph, const T *u, T *d, T *r, const T *p, const T *Ap,
                           const T *hp, cudaStream_t s)
{
    c.n_launch += 2;
    const int g = cg_vert_grid(c.nv);
    if (c.dim == 2)
        launch_k(c.pdl, k_cg_update_halo<T, 2>, dim3(g), dim3(256), 0, s, c.td, c.vd, ph, u, d, r, p, Ap, hp,
                 c.partials, c.sc);
    else
        launch_k(c.pdl, k_cg_update_halo<T, 3>, dim3(g), dim3(256), 0, s, c.td, c.vd, ph, u, d, r, p, Ap, hp,
                 c.partials, c.sc);
    launch_k(c.pdl, k_cg_beta<T>, dim3(1), dim3(1024), 0, s, (const double *)c.partials, g, c.sc);
}

template <typename T>
void launch_cg_alpha(const Ctx &c, int n_partials, cudaStream_t s)
{
    c.n_launch += 1;
    launch_k(c.pdl, k_cg_alpha<T>, dim3(1), dim3(1024), 0, s, (const double *)c.partials, n_partials, c.sc);
}

template <typename T>
void launch_cg_dir(const Ctx &c, T *p, const T *r, cudaStream_t s)
{
    c.n_launch += 1;
    const int64_t n = c.nv * c.dim;
    launch_k(c.pdl, k_cg_dir<T>, dim3(cg_vec4_grid(n)), dim3(256), 0, s, n, p, (const T *)r, (const DevScalars *)c.sc);
}

template <typename T>
void launch_tile_dot(const Ctx &c, double *out, cudaStream_t s)
{
    c.n_launch += 1;
    k_tile_dot<T><<<1, 1024, 0, s>>>(c.partials, c.td.n_tiles, out);
}

template <typename T>
void launch_dir_check(const Ctx &c, const double *g, T *d, cudaStream_t s)
{
    c.n_launch += 2;
    const int64_t n = c.nv * c.dim;
    k_dir_check<T><<<vec_grid(n), 256, 0, s>>>(n, g, d, c.partials, c.sc);
    k_dir_fix<T><<<vec_grid(n), 256, 0, s>>>(n, g, d, c.sc);
}

template <typename T>
void launch_step_update(const Ctx &c, double *u, const T *d, double t, float *u32, cudaStream_t s)
{
    c.n_launch += 1;
    const int64_t n = c.nv * c.dim;
    k_step_update<T><<<vec_grid(n), 256, 0, s>>>(n, u, d, t, u32);
}

void launch_x_to_u(const Ctx &c, const double *x, double *u, float *u32, const uint8_t *fixed, cudaStream_t s)
{
    c.n_launch += 1;
    k_x_to_u<<<vec_grid(c.nv * c.dim), 256, 0, s>>>(c.nv, c.dim, x, c.vd.X, fixed, u, u32);
}

void launch_u_to_x(const Ctx &c, const double *u, double *x, cudaStream_t s)
{
    c.n_launch += 1;
    const int64_t n = c.nv * c.dim;
    k_u_to_x<<<vec_grid(n), 256, 0, s>>>(n, u, c.vd.X, x);
}

void launch_uhat(const Ctx &c, const double *x0, const double *v0, double dt, double *uhat, cudaStream_t s)
{
    c.n_launch += 1;
    const int64_t n = c.nv * c.dim;
    k_uhat<<<vec_grid(n), 256, 0, s>>>(n, x0, v0, dt, c.vd.X, uhat);
}

template <typename T>
void launch_gather_elem(const Ctx &c, const double *user, T *internal, cudaStream_t s, int64_t stride)
{
    c.n_launch += 1;
    k_gather_elem<T><<<vec_grid(c.ne_int), 256, 0, s>>>(c.ne_int, c.td.perm, user, internal, stride);
}

template <typename Tin, typename Tout>
void launch_convert(int64_t n, const Tin *in, Tout *out, cudaStream_t s)
{
    k_convert<Tin, Tout><<<vec_grid(n), 256, 0, s>>>(n, in, out);
}

void launch_mask_copy(const Ctx &c, const double *in, double *out, cudaStream_t s)
{
    c.n_launch += 1;
    k_mask_copy<<<vec_grid(c.nv * c.dim), 256, 0, s>>>(c.nv, c.dim, c.vd.fixed, in, out);
}

void launch_friction_prep(const Ctx &c, const double *x0, double kf, double eps, double *u0, double *fw,
                          cudaStream_t s)
{
    c.n_launch += 1;
    k_friction_prep<<<vec_grid(c.nv), 256, 0, s>>>(c.nv, c.dim, x0, c.vd.X, kf, eps, u0, fw);
}

void launch_step_bwd_combine(const Ctx &c, const double *lam, const double *vbar1, double dt, const double *fw,
                             double kf, const double *x0, const double *x1, double *xbar0, double *vbar0,
                             cudaStream_t s)
{
    c.n_launch += 1;
    k_step_bwd_combine<<<vec_grid(c.nv), 256, 0, s>>>(c.nv, c.dim, c.vd.fixed, c.vd.mass, lam, vbar1, dt, fw, kf, x0,
                                                     x1, xbar0, vbar0);
}

void launch_axpy_out(int64_t n, const double *x, const double *y, double beta, double *out, cudaStream_t s)
{
    k_axpy_out<<<vec_grid(n), 256, 0, s>>>(n, x, y, beta, out);
}

void launch_velocity(int64_t n, const double *x1, const double *x0, double dt, double *v1, cudaStream_t s)
{
    k_velocity<<<vec_grid(n), 256, 0, s>>>(n, x1, x0, dt, v1);
}

__global__ void k_pad_rows4(int64_t nv, const float *__restrict__ u, float4 *__restrict__ u4)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x)
        u4[i] = make_float4(u[3 * i], u[3 * i + 1], u[3 * i + 2], 0.0f);
}

void launch_pad_rows4(const Ctx &c, const float *u, float *u4, cudaStream_t s)
{
    c.n_launch += 1;
    k_pad_rows4<<<vec_grid(c.nv), 256, 0, s>>>(c.nv, u, reinterpret_cast<float4 *>(u4));
}

int vec_grid_size(int64_t n) { return vec_grid(n); }
int cg_update_grid_size(int64_t nv) { return cg_vert_grid(nv); }

#define INST(T)                                                                                                     \
    template void launch_cg_init<T>(const Ctx &, const double *, double, T *, T *, T *, double, int, int,            \
                                    cudaStream_t);                                                                \
    template void launch_cg_update_halo<T>(const Ctx &, const Phys &, const T *, T *, T *, const T *, const T *,    \
                                           const T *, cudaStream_t);                                                \
    template void launch_cg_dir<T>(const Ctx &, T *, const T *, cudaStream_t);                                      \
    template void launch_cg_alpha<T>(const Ctx &, int, cudaStream_t);                                               \
    template void launch_dir_check<T>(const Ctx &, const double *, T *, cudaStream_t);                              \
    template void launch_tile_dot<T>(const Ctx &, double *, cudaStream_t);                                          \
    template void launch_step_update<T>(const Ctx &, double *, const T *, double, float *, cudaStream_t);           \
    template void launch_gather_elem<T>(const Ctx &, const double *, T *, cudaStream_t, int64_t);                   \
    template void launch_accumulate<T>(const Ctx &, double *, const T *, cudaStream_t);
INST(float)
INST(double)
#undef INST
template void launch_convert<double, float>(int64_t, const double *, float *, cudaStream_t);
template void launch_convert<float, double>(int64_t, const float *, double *, cudaStream_t);
template void launch_convert<double, double>(int64_t, const double *, double *, cudaStream_t);

}  // namespace softsim
