// Element kernels: energy, gradient, Hessian-vector product and parameter
// VJP of the neo-Hookean + muscle energy on triangle (D = 2) and tet (D = 3)
// meshes.
//
// Model (Sec. 2, Eq. neohookean-psi; 3D form with I1 - 3):
//   F = Ds Dm^-1 = I + Du Dm^-1 (Du: edge matrix of the displacement u = x - X,
//   which keeps F accurate in FP32), J = det F,
//   Psi = mu/2 (|F|^2 - D) - mu l(J) + lambda/2 l(J)^2,
//   l = log (exact) or q(J) = (J-1) - (J-1)^2/2 (quadratic stand-in),
//   muscle Psi_m = k/2 a |F f|^2 (contractile) or k/2 (|F f|/a - 1)^2 (active
//   spring, Eq. active-spring-potential).
// Writing P_el = mu F + c(J) cof(F) with c = (lambda l - mu) l', the
// differential is dP = mu dF + c'(J) (cof F : dF) cof F + c(J) dcof(F)[dF].
// The element force matrix is G = W dPsi/dF Dm^-T; column j goes to vertex
// j+1 and minus the column sum to vertex 0 (f = -grad E, Eq. f-as-grad; the
// HVP is the paper's Eq. matrix-free-dfdx written out analytically).
//
// Each CTA processes one tile: it stages the tile's vertex values in shared
// memory, evaluates its elements (one thread per element, coalesced SoA
// loads), writes the per-corner results to shared memory, and then one
// thread per tile vertex adds that vertex's corners in a fixed order.
// Vertices shared with other tiles go through halo slots and a finalize
// kernel, so every sum has one fixed order: no float atomics.
#include <cstdio>

#include "internal.h"
#include "reduce.cuh"
#include "tma.cuh"
#include "elem_math.cuh"
#include "pdl.cuh"
#include "tile_device.cuh"

namespace softsim {

// Per-vertex potential terms: gravity m g y and ground penalty kc max(0,-y)^p.
__device__ __forceinline__ double pen_pow(double pen, int p) { return p == 2 ? pen * pen : pen * pen * pen; }

// ---------------------------------------------------------------- energy

// One launch evaluates the energy at u + t_j dir for n_trials step lengths,
// sharing the element loads; FP64 throughout.
template <int D>
__global__ void __launch_bounds__(256) k_tile_energy(TileDev td, ElemDev<double> ed, VertDev vd, Phys ph,
                                                     const double *__restrict__ u, const double *__restrict__ dir,
                                                     const double *__restrict__ uhat, const double *__restrict__ a,
                                                     TrialT tr, double *__restrict__ partials,
                                                     DevScalars *__restrict__ sc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *su = reinterpret_cast<double *>(smem);
    double *sd = su + td.max_tv * D;
    const int t = blockIdx.x;
    const int es = td.tile_elem[t], ne_t = td.tile_elem[t + 1] - es;
    const int vs = td.tile_vert[t], nlv = td.tile_vert[t + 1] - vs;
    const int nt = tr.n;
    for (int k = threadIdx.x; k < nlv; k += blockDim.x) {
        const int64_t gid = td.lv_gid[vs + k];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            su[k * D + c] = u[gid * D + c];
            sd[k * D + c] = dir ? dir[gid * D + c] : 0.0;
        }
    }
    __syncthreads();
    double Eacc[kMaxTrials], Sacc[kMaxTrials];
#pragma unroll
    for (int j = 0; j < kMaxTrials; ++j) Eacc[j] = Sacc[j] = 0.0;
    double minJ = INFINITY;
    const double mu = ph.mu, lam = ph.lam;
    for (int le = threadIdx.x; le < ne_t; le += blockDim.x) {
        const int64_t e = es + le;
        int lid[D + 1];
        unpack<D>(td.conn[e], lid);
        double B[D][D], Du[D][D], Dd[D][D], Z0[D][D], Zd[D][D];
        load_B<double, D>(ed, e, B);
        edges<double, D>(su, lid, Du);
        edges<double, D>(sd, lid, Dd);
        mul<double, D>(Du, B, Z0, true);
        mul<double, D>(Dd, B, Zd, false);
        const double W = __ldg(ed.field(FI<D>::W) + e);
        double f[D];
#pragma unroll
        for (int i = 0; i < D; ++i) f[i] = __ldg(ed.field(FI<D>::F + i) + e);
        const double ka = ph.k * a[e];
#pragma unroll
        for (int j = 0; j < kMaxTrials; ++j) {
            if (j >= nt) break;
            const double tj = tr.t[j];
            double F[D][D], C[D][D];
#pragma unroll
            for (int r = 0; r < D; ++r)
#pragma unroll
                for (int q = 0; q < D; ++q) F[r][q] = Z0[r][q] + tj * Zd[r][q];
            cof<double, D>(F, C);
            const double J = detF<double, D>(F, C);
            if (j == 0) minJ = fmin(minJ, J);
            double I1 = 0.0, Ff2 = 0.0;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                double ff = 0.0;
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    I1 += F[r][q] * F[r][q];
                    ff += F[r][q] * f[q];
                }
                Ff2 += ff * ff;
            }
            double l;
            if (ph.log_mode == 0) {
                l = J > 0.0 ? log(J) : 0.0;
            } else {
                const double jm = J - 1.0;
                l = jm - 0.5 * jm * jm;
            }
            double musc = 0.5 * ka * Ff2;
            if (ph.muscle) {
                const double r = sqrt(Ff2) / a[e] - 1.0;
                musc = W != 0.0 ? 0.5 * ph.k * r * r : 0.0;
            }
            double w = ph.s_el * W * (0.5 * mu * (I1 - D) - mu * l + 0.5 * lam * l * l + musc);
            if (ph.log_mode == 0 && J <= 0.0) w = INFINITY;  // a NaN J (non-finite input) stays NaN
            Eacc[j] += w;
            Sacc[j] += fabs(w);
        }
    }
    // per-vertex terms, added by each vertex's owner tile
    for (int k = threadIdx.x; k < nlv; k += blockDim.x) {
        const int code = td.lv_code[vs + k];
        if (code == LV_PAD || (code >= 0 && !(code & 1))) continue;  // padding, or not the owner
        const int64_t gid = td.lv_gid[vs + k];
        const double m = vd.mass[gid];
        const double X1 = vd.X[gid * D + 1];
#pragma unroll
        for (int j = 0; j < kMaxTrials; ++j) {
            if (j >= nt) break;
            const double tj = tr.t[j];
            const double y = X1 + su[k * D + 1] + tj * sd[k * D + 1];
            const double pen = y < 0.0 ? -y : 0.0;
            double w = ph.s_el * (m * ph.grav * y + ph.kc * pen_pow(pen, ph.cpow));
            double s = fabs(w);
            if (ph.dyn) {
                double in = 0.0;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const double r = su[k * D + c] + tj * sd[k * D + c] - uhat[gid * D + c];
                    in += 0.5 * m * r * r;
                }
                if (ph.fw) {
                    const double f = ph.fw[gid];
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        if (c == 1) continue;
                        const double r = su[k * D + c] + tj * sd[k * D + c] - ph.u0[gid * D + c];
                        in += 0.5 * f * r * r;
                    }
                }
                w += in;
                s += in;
            }
            Eacc[j] += w;
            Sacc[j] += s;
        }
    }
    const int nb = gridDim.x;
    for (int j = 0; j < nt; ++j) {
        double e = block_sum(Eacc[j]);
        double s = block_sum(Sacc[j]);
        if (threadIdx.x == 0) {
            partials[(size_t)j * nb + t] = e;
            partials[(size_t)(kMaxTrials + j) * nb + t] = s;
        }
    }
    double mj = block_min(minJ);
    if (threadIdx.x == 0) partials[(size_t)(2 * kMaxTrials) * nb + t] = mj;
    if (last_block(&sc->ticket[TK_ENERGY], nb)) {
        for (int j = 0; j < nt; ++j) {
            double e = sum_partials(partials + (size_t)j * nb, nb);
            double s = sum_partials(partials + (size_t)(kMaxTrials + j) * nb, nb);
            if (threadIdx.x == 0) {
                sc->E[j] = e;
                sc->S[j] = s;
            }
        }
        double m = min_partials(partials + (size_t)(2 * kMaxTrials) * nb, nb);
        if (threadIdx.x == 0) sc->minJ = m;
    }
}

// ---------------------------------------------------------------- gradient

template <int D>
__global__ void __launch_bounds__(256) k_tile_grad(TileDev td, ElemDev<double> ed, VertDev vd, Phys ph,
                                                   const double *__restrict__ u, const double *__restrict__ uhat,
                                                   const double *__restrict__ a, double *__restrict__ g,
                                                   double *__restrict__ hp, double *__restrict__ partials)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *su = reinterpret_cast<double *>(smem);
    double *scr = su + td.max_tv * D;
    const int t = blockIdx.x;
    const int es = td.tile_elem[t], ne_t = td.tile_elem[t + 1] - es;
    const int vs = td.tile_vert[t], nlv = td.tile_vert[t + 1] - vs;
    for (int k = threadIdx.x; k < nlv; k += blockDim.x) {
        const int64_t gid = td.lv_gid[vs + k];
#pragma unroll
        for (int c = 0; c < D; ++c) su[k * D + c] = u[gid * D + c];
    }
    __syncthreads();
    const double mu = ph.mu, lam = ph.lam;
    for (int le = threadIdx.x; le < ne_t; le += blockDim.x) {
        const int64_t e = es + le;
        int lid[D + 1];
        unpack<D>(td.conn[e], lid);
        double B[D][D], Du[D][D], F[D][D], C[D][D];
        load_B<double, D>(ed, e, B);
        edges<double, D>(su, lid, Du);
        mul<double, D>(Du, B, F, true);
        cof<double, D>(F, C);
        const double J = detF<double, D>(F, C);
        double l, cc, cp;
        log_terms<double>(ph.log_mode, mu, lam, J, l, cc, cp);
        const double W = __ldg(ed.field(FI<D>::W) + e) * ph.s_el;
        double f[D], gv[D], Ff[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            f[i] = __ldg(ed.field(FI<D>::F + i) + e);
            gv[i] = __ldg(ed.field(FI<D>::G + i) + e);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < D; ++q) s += F[i][q] * f[q];
            Ff[i] = s;
        }
        double ka = ph.k * a[e];  // dpsi_m/dq = ka q
        if (ph.muscle) {
            double s2 = 0.0, c2;
#pragma unroll
            for (int i = 0; i < D; ++i) s2 += Ff[i] * Ff[i];
            spring_terms<double>(W != 0.0, ph.k, a[e], sqrt(s2), ka, c2);
        }
        double G[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) s += (mu * F[i][k] + cc * C[i][k]) * B[j][k];
                G[i][j] = W * (s + ka * Ff[i] * gv[j]);
            }
        store_corners<double, D>(scr + (int64_t)le * td.rs + corner_base(le), G);
    }
    __syncthreads();
    double gn2 = 0.0;
    const uint16_t *tinc = td.inc + (int64_t)es * (D + 1);
    for (int k = threadIdx.x; k < nlv; k += blockDim.x) {
        const int code = td.lv_code[vs + k];
        if (code == LV_PAD) continue;
        double acc[D];
        gather_corners<double, D>(tinc, td.lv_inc[vs + k], scr, acc);
        const int64_t gid = td.lv_gid[vs + k];
        if (code == LV_INTERIOR) {
            const double m = vd.mass[gid];
            const double y = vd.X[gid * D + 1] + su[k * D + 1];
            const double pen = y < 0.0 ? -y : 0.0;
            const double dcon = pen > 0.0 ? -ph.cpow * ph.kc * (ph.cpow == 2 ? pen : pen * pen) : 0.0;
            acc[1] += ph.s_el * (m * ph.grav + dcon);
            if (ph.dyn)
#pragma unroll
                for (int c = 0; c < D; ++c) acc[c] += m * (su[k * D + c] - uhat[gid * D + c]);
            if (ph.fw) {
                const double f = ph.fw[gid];
#pragma unroll
                for (int c = 0; c < D; ++c)
                    if (c != 1) acc[c] += f * (su[k * D + c] - ph.u0[gid * D + c]);
            }
            const bool fx = vd.fixed[gid] != 0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const double o = fx ? 0.0 : acc[c];
                g[gid * D + c] = o;
                gn2 += o * o;
            }
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) hp[(int64_t)(code >> 1) * D + c] = acc[c];
        }
    }
    const double s = block_sum(gn2);
    if (threadIdx.x == 0) partials[t] = s;
}

template <int D>
__global__ void __launch_bounds__(256) k_fin_grad(TileDev td, VertDev vd, Phys ph, const double *__restrict__ u,
                                                  const double *__restrict__ uhat, const double *__restrict__ hp,
                                                  double *__restrict__ g, double *__restrict__ partials,
                                                  DevScalars *__restrict__ sc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double gn2 = 0.0;
    if (i < td.n_fin) {
        const int64_t gid = td.fin_gid[i];
        double acc[D];
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = 0.0;
        for (int s = td.fin_ptr[i]; s < td.fin_ptr[i + 1]; ++s)
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] += hp[(int64_t)s * D + c];
        const double m = vd.mass[gid];
        const double y = vd.X[gid * D + 1] + u[gid * D + 1];
        const double pen = y < 0.0 ? -y : 0.0;
        const double dcon = pen > 0.0 ? -ph.cpow * ph.kc * (ph.cpow == 2 ? pen : pen * pen) : 0.0;
        acc[1] += ph.s_el * (m * ph.grav + dcon);
        if (ph.dyn)
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] += m * (u[gid * D + c] - uhat[gid * D + c]);
        if (ph.fw) {
            const double f = ph.fw[gid];
#pragma unroll
            for (int c = 0; c < D; ++c)
                if (c != 1) acc[c] += f * (u[gid * D + c] - ph.u0[gid * D + c]);
        }
        const bool fx = vd.fixed[gid] != 0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double o = fx ? 0.0 : acc[c];
            g[gid * D + c] = o;
            gn2 += o * o;
        }
    }
    const double s = block_sum(gn2);
    const int base = td.n_tiles;
    if (threadIdx.x == 0) partials[base + blockIdx.x] = s;
    if (last_block(&sc->ticket[TK_GRAD], gridDim.x)) {
        const double tot = sum_partials(partials, base + gridDim.x);
        if (threadIdx.x == 0) sc->gn2 = tot;
    }
}

// ---------------------------------------------------------------- HVP

// Shared-memory plan of the HVP tile kernel (offsets in bytes, all 16-byte
// aligned because max_te is a multiple of 8, max_tv of 4 and rs even).
template <typename T, int D>
struct HvpSmem {
    size_t e, rec, conn, inc, gid, code, linc, uv, total;
    __host__ __device__ HvpSmem(int max_te, int max_tv, int rs)
    {
        e = 16;  // two mbarriers
        rec = e;  // [max_te][rs] element records
        conn = rec + (size_t)rs * max_te * sizeof(T);
        inc = conn + (size_t)max_te * 4;
        gid = inc + (size_t)max_te * (D + 1) * 2;
        code = gid + (size_t)max_tv * 4;
        linc = code + (size_t)max_tv * 4;
        uv = linc + (size_t)max_tv * 4;  // [max_tv][2D]: u then v of each local vertex
        total = uv + (size_t)max_tv * 2 * D * sizeof(T);
    }
};

// HVP of one tile per CTA.  Thread 0 pulls the tile's element records
// (fields and activation), connectivity, incidence lists and local-vertex
// tables into shared memory with bulk copies on two mbarriers; the tile's
// vertex values are then gathered, each thread evaluates dP(dF) for its
// elements from their records (pair loads), the element's corner forces
// overwrite its own record in place (slots corner_base(le) .. +(D+1)*D <= RS),
// and one thread
// per local vertex adds its corners in fixed order.
// SPRING selects the active-spring muscle at compile time, so the
// contractile kernel carries none of its code or its extra fields.
template <typename T, int D, bool CG, int MINB, int MTE, bool SPRING>
__global__ void __launch_bounds__(256, MINB) k_tile_hvp(TileDev td, const T *__restrict__ erec, VertDev vd,
                                                  Phys ph, const T *__restrict__ u, const T *__restrict__ v,
                                                  T *__restrict__ y, T *__restrict__ hp,
                                                  double *__restrict__ partials, DevScalars *__restrict__ sc)
{
    extern __shared__ __align__(128) unsigned char smem[];
    // MTE != 0: the tile capacity is a compile-time constant, so every
    // record and corner offset below folds into an immediate
    constexpr int NF = hvp_fields(D, SPRING);
    constexpr int RS = rec_stride(NF);  // record: NF fields, the activation at slot NF, padding
    const HvpSmem<T, D> L(MTE ? MTE : td.max_te, td.max_tv, RS);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);  // [0]: vertex tables, [1]: element data
    T *sRec = reinterpret_cast<T *>(smem + L.rec);
    // vertex table: [gid, code, lv_inc] per local vertex (stride 3 words:
    // a warp's lanes read distinct banks)
    const int32_t *sLv = reinterpret_cast<const int32_t *>(smem + L.gid);
    T *suv = reinterpret_cast<T *>(smem + L.uv);  // per local vertex: u (D values), then v (D values)
    const int t = blockIdx.x;
    // a tile's ranges: from its index for equal tiles (no dependent load before
    // the bulk copies can be issued), else from the offset tables
    const int es = td.uni_te ? t * td.uni_te : td.tile_elem[t];
    const int ne_t = td.uni_te ? td.uni_te : td.tile_elem[t + 1] - es;
    const int vs = td.uni_tv ? t * td.uni_tv : td.tile_vert[t];
    const int nlv = td.uni_tv ? td.uni_tv : td.tile_vert[t + 1] - vs;
    // the tile's connectivity and incidence block arrive as one blob: conn
    // [ne_t] then inc [ne_t (D+1)] (both 16-byte multiples)
    const uint32_t *sConn = reinterpret_cast<const uint32_t *>(smem + L.conn);
    const uint16_t *sInc = reinterpret_cast<const uint16_t *>(smem + L.conn + (size_t)ne_t * 4);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        // vertex table first: the vertex gather below overlaps the element copy
        mbar_arrive_expect_tx(bar, 12u * nlv);
        bulk_g2s(smem + L.gid, td.lv3 + (int64_t)vs * 3, 12u * nlv, bar);
        const uint32_t brec = (uint32_t)ne_t * RS * sizeof(T), bci = (uint32_t)ne_t * (4 + 2 * (D + 1));
        mbar_arrive_expect_tx(bar + 1, brec + bci);
        const uint64_t pol = l2_evict_first_policy();  // element data is read once per launch
        bulk_g2s_stream(sRec, erec + (int64_t)es * RS, brec, bar + 1, pol);
        bulk_g2s_stream(smem + L.conn, td.ci + (int64_t)es * (4 + 2 * (D + 1)), bci, bar + 1, pol);
    }
    __syncthreads();
    // Everything copied so far is static during a solve; state (u, v) and the
    // CG scalars are read only after the predecessor kernel has completed.
    pdl_wait();
    // the flag is read before the wait so that its load overlaps the copies
    // in flight; the previous kernel has completed, so every thread reads the
    // same value
    const int cg_done = CG ? sc->done : 0;
    // every thread takes the same decision, so no thread is left at a barrier
    if (__syncthreads_or(!mbar_wait_bounded(bar, 0, td.wait_polls))) {
        if (threadIdx.x == 0) {
            atomicOr(&sc->kerr, 1);
            mbar_wait_bounded(bar, 0);  // give copies in flight a last chance before the CTA exits
            mbar_wait_bounded(bar + 1, 0);
        }
        return;
    }
    if (cg_done) {  // CG already finished: drain the second copy, then leave
        if (threadIdx.x == 0) mbar_wait_bounded(bar + 1, 0);
        return;
    }
    for (int k = threadIdx.x; k < nlv; k += blockDim.x) {
        const int64_t gid = sLv[3 * k];
        const bool fx = ((uint32_t)sLv[3 * k + 2] & kLvPinned) != 0;
        if constexpr (CG && sizeof(T) == 4 && D == 3) {
            // the CG loop's 3D FP32 displacement comes in 16-byte rows
            const float4 u4 = reinterpret_cast<const float4 *>(u)[gid];
            suv[k * 6 + 0] = u4.x;
            suv[k * 6 + 1] = u4.y;
            suv[k * 6 + 2] = u4.z;
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) suv[k * 2 * D + c] = u[gid * D + c];
        }
#pragma unroll
        for (int c = 0; c < D; ++c) suv[k * 2 * D + D + c] = fx ? T(0) : v[gid * D + c];
    }
    if (__syncthreads_or(!mbar_wait_bounded(bar + 1, 0))) {
        if (threadIdx.x == 0) {
            atomicOr(&sc->kerr, 1);
            mbar_wait_bounded(bar + 1, 0);
        }
        return;
    }
    const T mu = pick<T>(ph.mu, ph.mu_f), lam = pick<T>(ph.lam, ph.lam_f);
    const T sel = pick<T>(ph.s_el, ph.s_el_f), kk = pick<T>(ph.k, ph.k_f);
    // CG: p.Ap of this tile from the element quadratic forms v_e . (H_e v_e)
    // and the owners' vertex terms, in the kernel's precision.  In the mixed
    // kernel the per-thread and block sums stay plain FP32 (GB300's FP64 pipe
    // runs at 1/64 of FP32, and compensating them here cost ~7 % of the
    // kernel's time); k_cg_alpha sums the tiles' partials with compensation.
    T dot = T(0);
    for (int le = threadIdx.x; le < ne_t; le += blockDim.x)
        hvp_element<T, D, CG, SPRING, RS>(sRec + le * RS, le, sConn[le], suv, ph, mu, lam, sel, kk, dot,
                                          sRec + le * RS);
    __syncthreads();
    for (int k = threadIdx.x; k < nlv; k += blockDim.x)
        hvp_vertex<T, D, CG>(sLv[3 * k + 1], (uint32_t)sLv[3 * k + 2], sLv[3 * k], suv + k * 2 * D, sInc, sRec, vd, ph,
                             y, hp, dot);
    pdl_trigger();  // the alpha reduction may be scheduled once every tile is done
    if (CG) {
        const T sum = block_sum(dot);
        if (threadIdx.x == 0) reinterpret_cast<T *>(partials)[t] = sum;  // reduced by k_cg_alpha<T>
    }
}

// Completes y = A v at halo vertices: the tiles' partial sums in tile order
// plus the per-vertex terms.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_fin_hvp(TileDev td, VertDev vd, Phys ph, const T *__restrict__ u,
                                                 const T *__restrict__ v, const T *__restrict__ hp, T *__restrict__ y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= td.n_fin) return;
    const int64_t gid = td.fin_gid[i];
    const bool fx = vd.fixed[gid] != 0;
    T acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = T(0);
    for (int s = td.fin_ptr[i]; s < td.fin_ptr[i + 1]; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] += hp[(int64_t)s * D + c];
    T vv[D];
#pragma unroll
    for (int c = 0; c < D; ++c) vv[c] = fx ? T(0) : v[gid * D + c];
    if (ph.kc > 0.0) {
        const double yy = vd.X[gid * D + 1] + (double)u[gid * D + 1];
        const double pen = yy < 0.0 ? -yy : 0.0;
        const double d2 = pen > 0.0 ? ph.cpow * (ph.cpow - 1) * ph.kc * (ph.cpow == 2 ? 1.0 : pen) : 0.0;
        acc[1] += T(ph.s_el * d2) * vv[1];
    }
    if (ph.dyn) {
        const T m = T(vd.mass[gid]);
        const T mh = ph.fw ? m + T(ph.fw[gid]) : m;
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] += (c == 1 ? m : mh) * vv[c];
    }
#pragma unroll
    for (int c = 0; c < D; ++c) y[gid * D + c] = fx ? T(0) : acc[c];
}

// ---------------------------------------------------------------- parameter VJP

template <int D>
__global__ void __launch_bounds__(256) k_tile_vjp(TileDev td, ElemDev<double> ed, VertDev vd, Phys ph,
                                                  const double *__restrict__ u, const double *__restrict__ a,
                                                  const double *__restrict__ lam, double *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *su = reinterpret_cast<double *>(smem);
    double *sl = su + td.max_tv * D;
    const int t = blockIdx.x;
    const int es = td.tile_elem[t], ne_t = td.tile_elem[t + 1] - es;
    const int vs = td.tile_vert[t], nlv = td.tile_vert[t + 1] - vs;
    for (int k = threadIdx.x; k < nlv; k += blockDim.x) {
        const int64_t gid = td.lv_gid[vs + k];
        const bool fx = vd.fixed[gid] != 0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            su[k * D + c] = u[gid * D + c];
            sl[k * D + c] = fx ? 0.0 : lam[gid * D + c];
        }
    }
    __syncthreads();
    for (int le = threadIdx.x; le < ne_t; le += blockDim.x) {
        const int64_t e = es + le;
        int lid[D + 1];
        unpack<D>(td.conn[e], lid);
        double B[D][D], Du[D][D], Dl[D][D], F[D][D];
        load_B<double, D>(ed, e, B);
        edges<double, D>(su, lid, Du);
        edges<double, D>(sl, lid, Dl);
        mul<double, D>(Du, B, F, true);
        double f[D], gv[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            f[i] = __ldg(ed.field(FI<D>::F + i) + e);
            gv[i] = __ldg(ed.field(FI<D>::G + i) + e);
        }
        double dot = 0.0, s2 = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double Ff = 0.0, dFf = 0.0;
#pragma unroll
            for (int q = 0; q < D; ++q) {
                Ff += F[i][q] * f[q];
                dFf += Dl[i][q] * gv[q];  // dF(lam) f = Dlam Dm^-1 f = Dlam g
            }
            dot += Ff * dFf;
            s2 += Ff * Ff;
        }
        const double W = __ldg(ed.field(FI<D>::W) + e);
        const int32_t pe = td.perm[e];
        // d2psi/dq da = k q (contractile) or k (1/a^2 - 2 s/a^3)/s q (spring, s = |q|)
        double kq = ph.k;
        if (ph.muscle && pe >= 0) {
            const double s = sqrt(s2), ia = 1.0 / a[e];
            kq = ph.k * (ia * ia - 2.0 * s * ia * ia * ia) / s;
        }
        if (pe >= 0) out[pe] = -ph.s_el * W * kq * dot;
    }
}

// Material-parameter VJPs per element: -s W (dP/dtheta) : dF(lam) with
// dP/dmu = F - l'(J) cof F, dP/dlambda = l(J) l'(J) cof F, and for the
// muscle stiffness -s W (d2psi_m/dq dk) . dq(lam).  Null outputs are skipped.
template <int D>
__global__ void __launch_bounds__(256) k_tile_mat_vjp(TileDev td, ElemDev<double> ed, VertDev vd, Phys ph,
                                                      const double *__restrict__ u, const double *__restrict__ a,
                                                      const double *__restrict__ lam, double *__restrict__ dmu,
                                                      double *__restrict__ dlam, double *__restrict__ dk)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *su = reinterpret_cast<double *>(smem);
    double *sl = su + td.max_tv * D;
    const int t = blockIdx.x;
    const int es = td.tile_elem[t], ne_t = td.tile_elem[t + 1] - es;
    const int vs = td.tile_vert[t], nlv = td.tile_vert[t + 1] - vs;
    for (int k = threadIdx.x; k < nlv; k += blockDim.x) {
        const int64_t gid = td.lv_gid[vs + k];
        const bool fx = vd.fixed[gid] != 0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            su[k * D + c] = u[gid * D + c];
            sl[k * D + c] = fx ? 0.0 : lam[gid * D + c];
        }
    }
    __syncthreads();
    for (int le = threadIdx.x; le < ne_t; le += blockDim.x) {
        const int64_t e = es + le;
        const int32_t pe = td.perm[e];
        if (pe < 0) continue;  // padding
        int lid[D + 1];
        unpack<D>(td.conn[e], lid);
        double B[D][D], Du[D][D], Dl[D][D], F[D][D], dF[D][D], C[D][D];
        load_B<double, D>(ed, e, B);
        edges<double, D>(su, lid, Du);
        edges<double, D>(sl, lid, Dl);
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
        double l, lp;  // l(J) and l'(J)
        if (ph.log_mode == 0) {
            l = log(J);
            lp = 1.0 / J;
        } else {
            l = (J - 1.0) - 0.5 * (J - 1.0) * (J - 1.0);
            lp = 2.0 - J;
        }
        const double sW = -ph.s_el * __ldg(ed.field(FI<D>::W) + e);
        if (dmu) dmu[pe] = sW * (FdF - lp * CdF);
        if (dlam) dlam[pe] = sW * l * lp * CdF;
        if (dk) {
            double qdq = 0.0, s2 = 0.0;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                double q = 0.0, dq = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    q += F[i][k] * __ldg(ed.field(FI<D>::F + k) + e);
                    dq += Dl[i][k] * __ldg(ed.field(FI<D>::G + k) + e);  // dF(lam) f = Dlam g
                }
                qdq += q * dq;
                s2 += q * q;
            }
            double c = a[e];  // d2psi_m/dq dk = c q
            if (ph.muscle) {
                const double sq = sqrt(s2);
                c = (sq / a[e] - 1.0) / (a[e] * sq);
            }
            dk[pe] = sW * c * qdq;
        }
    }
}

// ---------------------------------------------------------------- launchers

static inline size_t smem_verts(const Ctx &c, size_t elt, int nfields)
{
    return (size_t)c.td.max_tv * c.dim * nfields * elt;
}

void launch_energy(const Ctx &c, const Phys &ph, const double *u, const double *dir, const double *uhat,
                   const double *a, const double *t, int n_trials, cudaStream_t s)
{
    c.n_launch += 1;
    TrialT tr;
    tr.n = n_trials;
    for (int j = 0; j < kMaxTrials; ++j) tr.t[j] = j < n_trials ? t[j] : 0.0;
    const size_t sm = smem_verts(c, sizeof(double), 2);
    if (c.dim == 2)
        k_tile_energy<2><<<c.td.n_tiles, c.threads, sm, s>>>(c.td, c.e64, c.vd, ph, u, dir, uhat, a, tr, c.partials, c.sc);
    else
        k_tile_energy<3><<<c.td.n_tiles, c.threads, sm, s>>>(c.td, c.e64, c.vd, ph, u, dir, uhat, a, tr, c.partials, c.sc);
}

void launch_grad(const Ctx &c, const Phys &ph, const double *u, const double *uhat, const double *a, double *g,
                 double *hp, cudaStream_t s)
{
    c.n_launch += 2;
    const size_t sm = smem_verts(c, sizeof(double), 1) + (size_t)c.td.max_te * c.td.rs * sizeof(double);
    const int fb = c.n_fin_blocks;
    if (c.dim == 2) {
        k_tile_grad<2><<<c.td.n_tiles, c.threads, sm, s>>>(c.td, c.e64, c.vd, ph, u, uhat, a, g, hp, c.partials);
        k_fin_grad<2><<<fb, 256, 0, s>>>(c.td, c.vd, ph, u, uhat, hp, g, c.partials, c.sc);
    } else {
        k_tile_grad<3><<<c.td.n_tiles, c.threads, sm, s>>>(c.td, c.e64, c.vd, ph, u, uhat, a, g, hp, c.partials);
        k_fin_grad<3><<<fb, 256, 0, s>>>(c.td, c.vd, ph, u, uhat, hp, g, c.partials, c.sc);
    }
}

template <typename T>
static const T *erec(const Ctx &c);
template <>
const float *erec<float>(const Ctx &c) { return c.rec32; }
template <>
const double *erec<double>(const Ctx &c) { return c.rec64; }

template <typename T>
size_t hvp_smem(const Ctx &c)
{
    return c.dim == 2 ? HvpSmem<T, 2>(c.td.max_te, c.td.max_tv, c.td.rs).total
                      : HvpSmem<T, 3>(c.td.max_te, c.td.max_tv, c.td.rs).total;
}

// Resident CTAs per SM that the tile's shared memory allows (at most 4);
// the kernel variant compiled for that count caps registers to match.  (At
// 128 threads and 7 resident tiles, the 64-register FP32 variant measured
// faster in-solve than the 72-register one before the element used paired
// FP32 arithmetic: 66.3 vs 68.4 us on the large body; with it, the CG variant
// spills at 64 and runs at 58.4 us with 72 against 60.7 us.)
template <typename T>
int hvp_blocks_per_sm(const Ctx &c)
{
    const size_t per = hvp_smem<T>(c) + 1024;  // + static shared memory and reserve
    int b = (int)((227 * 1024) / per);
    return b < 1 ? 1 : (b > 4 ? 4 : b);
}

// Tile capacities with a compile-time specialisation (the library defaults).
constexpr int kCap2 = 512, kCap3 = 384;

template <typename T, int D, bool CG, int MINB>
static void hvp_tile_v(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y, T *hp, cudaStream_t s)
{
    constexpr int CAP = D == 2 ? kCap2 : kCap3;
    if (c.muscle)  // the spring variant exists for the runtime tile capacity only
        launch_k(c.pdl, k_tile_hvp<T, D, CG, MINB, 0, true>, dim3(c.td.n_tiles), dim3(c.threads), hvp_smem<T>(c), s,
                 c.td, erec<T>(c), c.vd, ph, u, v, y, hp, c.partials, c.sc);
    else if (sizeof(T) == 4 && c.td.max_te == CAP)
        launch_k(c.pdl, k_tile_hvp<T, D, CG, MINB, (sizeof(T) == 4 ? CAP : 0), false>, dim3(c.td.n_tiles),
                 dim3(c.threads), hvp_smem<T>(c), s, c.td, erec<T>(c), c.vd, ph, u, v, y, hp, c.partials, c.sc);
    else
        launch_k(c.pdl, k_tile_hvp<T, D, CG, MINB, 0, false>, dim3(c.td.n_tiles), dim3(c.threads), hvp_smem<T>(c), s,
                 c.td, erec<T>(c), c.vd, ph, u, v, y, hp, c.partials, c.sc);
}

template <typename T, bool CG>
static void hvp_tile(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y, T *hp, cudaStream_t s)
{
    c.n_launch += 1;
    const int b = hvp_blocks_per_sm<T>(c);
    if constexpr (sizeof(T) == 4) {
        if (c.dim == 2)
            (b >= 4 ? hvp_tile_v<T, 2, CG, 4> : hvp_tile_v<T, 2, CG, 3>)(c, ph, u, v, y, hp, s);
        else
            // the CG variant also forms p.Ap: at 64 registers it spilled, at
            // the 3-CTA bound it takes 72, which still lets 7 of the
            // 128-thread tiles be resident (shared memory allows 7)
            ((b >= 4 && !CG) ? hvp_tile_v<T, 3, CG, 4> : hvp_tile_v<T, 3, CG, 3>)(c, ph, u, v, y, hp, s);
    } else {
        if (c.dim == 2)
            (b >= 2 ? hvp_tile_v<T, 2, CG, 2> : hvp_tile_v<T, 2, CG, 1>)(c, ph, u, v, y, hp, s);
        else
            (b >= 2 ? hvp_tile_v<T, 3, CG, 2> : hvp_tile_v<T, 3, CG, 1>)(c, ph, u, v, y, hp, s);
    }
}

template <typename T>
static void hvp_fin(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y, const T *hp, cudaStream_t s)
{
    c.n_launch += 1;
    if (c.dim == 2)
        k_fin_hvp<T, 2><<<c.n_fin_blocks, 256, 0, s>>>(c.td, c.vd, ph, u, v, hp, y);
    else
        k_fin_hvp<T, 3><<<c.n_fin_blocks, 256, 0, s>>>(c.td, c.vd, ph, u, v, hp, y);
}

template <typename T>
void launch_hvp(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y, T *hp, cudaStream_t s)
{
    hvp_tile<T, false>(c, ph, u, v, y, hp, s);
    hvp_fin<T>(c, ph, u, v, y, hp, s);
}

template <typename T>
void launch_hvp_cg(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y, T *hp, cudaStream_t s)
{
    hvp_tile<T, true>(c, ph, u, v, y, hp, s);
}

template <typename T>
void launch_hvp_tile_only(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y, T *hp, cudaStream_t s)
{
    hvp_tile<T, false>(c, ph, u, v, y, hp, s);
}

template <typename T>
void launch_hvp_finalize_only(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y, const T *hp,
                              cudaStream_t s)
{
    hvp_fin<T>(c, ph, u, v, y, hp, s);
}

void launch_param_vjp(const Ctx &c, const Phys &ph, const double *u, const double *a, const double *lam,
                      double *dLda, cudaStream_t s)
{
    c.n_launch += 1;
    const size_t sm = smem_verts(c, sizeof(double), 2);
    if (c.dim == 2)
        k_tile_vjp<2><<<c.td.n_tiles, c.threads, sm, s>>>(c.td, c.e64, c.vd, ph, u, a, lam, dLda);
    else
        k_tile_vjp<3><<<c.td.n_tiles, c.threads, sm, s>>>(c.td, c.e64, c.vd, ph, u, a, lam, dLda);
}

void launch_material_vjp(const Ctx &c, const Phys &ph, const double *u, const double *a, const double *lam,
                         double *dmu, double *dlam, double *dk, cudaStream_t s)
{
    c.n_launch += 1;
    const size_t sm = smem_verts(c, sizeof(double), 2);
    if (c.dim == 2)
        k_tile_mat_vjp<2><<<c.td.n_tiles, c.threads, sm, s>>>(c.td, c.e64, c.vd, ph, u, a, lam, dmu, dlam, dk);
    else
        k_tile_mat_vjp<3><<<c.td.n_tiles, c.threads, sm, s>>>(c.td, c.e64, c.vd, ph, u, a, lam, dmu, dlam, dk);
}

// Opt every kernel that may need more than 48 KB of dynamic shared memory into
// the larger carve-out.
cudaError_t configure_elem_kernels()
{
    const int big = 200 * 1024;
    cudaError_t e = cudaSuccess;
#define SET(k) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, big)
    SET((k_tile_energy<2>));
    SET((k_tile_energy<3>));
    SET((k_tile_grad<2>));
    SET((k_tile_grad<3>));
#define SET_HVP(T, MB)                                                       \
    SET((k_tile_hvp<T, 2, true, MB, 0, false>));                             \
    SET((k_tile_hvp<T, 3, true, MB, 0, false>));                             \
    SET((k_tile_hvp<T, 2, false, MB, 0, false>));                            \
    SET((k_tile_hvp<T, 3, false, MB, 0, false>));                            \
    SET((k_tile_hvp<T, 2, true, MB, 0, true>));                              \
    SET((k_tile_hvp<T, 3, true, MB, 0, true>));                              \
    SET((k_tile_hvp<T, 2, false, MB, 0, true>));                             \
    SET((k_tile_hvp<T, 3, false, MB, 0, true>));                             \
    SET((k_tile_hvp<T, 2, true, MB, (sizeof(T) == 4 ? kCap2 : 0), false>));  \
    SET((k_tile_hvp<T, 3, true, MB, (sizeof(T) == 4 ? kCap3 : 0), false>));  \
    SET((k_tile_hvp<T, 2, false, MB, (sizeof(T) == 4 ? kCap2 : 0), false>)); \
    SET((k_tile_hvp<T, 3, false, MB, (sizeof(T) == 4 ? kCap3 : 0), false>));
    SET_HVP(float, 3)
    SET_HVP(float, 4)
    SET_HVP(double, 1)
    SET_HVP(double, 2)
#undef SET_HVP
    SET((k_tile_vjp<2>));
    SET((k_tile_vjp<3>));
    SET((k_tile_mat_vjp<2>));
    SET((k_tile_mat_vjp<3>));
#undef SET
    return e;
}

template void launch_hvp<float>(const Ctx &, const Phys &, const float *, const float *, float *, float *,
                                cudaStream_t);
template void launch_hvp<double>(const Ctx &, const Phys &, const double *, const double *, double *, double *,
                                 cudaStream_t);
template void launch_hvp_cg<float>(const Ctx &, const Phys &, const float *, const float *, float *, float *,
                                   cudaStream_t);
template void launch_hvp_cg<double>(const Ctx &, const Phys &, const double *, const double *, double *, double *,
                                    cudaStream_t);
template void launch_hvp_tile_only<float>(const Ctx &, const Phys &, const float *, const float *, float *, float *,
                                          cudaStream_t);
template void launch_hvp_tile_only<double>(const Ctx &, const Phys &, const double *, const double *, double *,
                                           double *, cudaStream_t);
template void launch_hvp_finalize_only<float>(const Ctx &, const Phys &, const float *, const float *, float *,
                                              const float *, cudaStream_t);
template void launch_hvp_finalize_only<double>(const Ctx &, const Phys &, const double *, const double *,
                                               double *, const double *, cudaStream_t);
template size_t hvp_smem<float>(const Ctx &);
template size_t hvp_smem<double>(const Ctx &);

}  // namespace softsim
