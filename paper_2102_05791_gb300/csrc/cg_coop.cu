// Conjugate gradients of a whole solve in ONE cooperative kernel, for meshes
// whose tiles can all be resident on the GPU at once (every CTA holds one
// tile; the launch fails instead of running if they do not fit).
//
// The per-iteration path (vec_kernels.cu, elem_kernels.cu) launches the HVP
// tile kernel and four small kernels per CG iteration and re-stages every
// tile's element records from global memory each time.  For small and
// medium meshes that cost is launch latency, not bandwidth.  Here each CTA
// stages its tile's element records, connectivity, incidence lists and
// vertex tables in shared memory once, then runs the CG iterations (Sec. 3:
// the adjoint and Newton systems are solved matrix-free by CG, the HVP of
// Eq. matrix-free-dfdx written out analytically) with two grid-wide barriers
// per iteration:
//   1. gather u, r and the previous p at the tile's vertices and form the
//      new direction p = r + beta p there (every CTA that touches a vertex
//      computes the same bits); element phase (corner forces into a separate
//      shared buffer, so the records stay); vertex phase (A p at single-tile
//      vertices, halo partials, the tile's p.Ap partial); barrier;
//   2. every CTA sums the p.Ap partials in the same fixed order (so all
//      take the same alpha and the same decisions); over its own contiguous
//      range of vertices it forms p again and stores it, completes A p at halo
//      vertices, updates d and r and forms its r.r partial; barrier; then
//      every CTA sums the r.r partials, takes beta and the convergence test.
// Meshes of at most 16 tiles run the same kernel as ONE thread-block cluster
// (a grid of n_tiles CTAs = one cluster, co-scheduled by construction): the
// two barriers are then the cluster's hardware barrier and the per-CTA
// partial sums are read from the other CTAs' shared memory, which costs
// about 0.75 us per barrier and sum against about 2.0 us through L2 atomics
// and loads (measured on GB300 with 8-32 CTAs).
// Cross-CTA data are read through L2 (ld.global.cg), never from a stale L1
// line.  Sums are fixed-order (FP32 within a CTA and compensated FP32 across
// CTAs for float vectors; FP64 for double), so results are deterministic.
// Every barrier wait is bounded: a CTA that gives up raises an error flag
// that the host reads and leaves; the others give up at their next barrier.
#include <cstdint>

#include "grid_sync.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "tile_device.cuh"
#include "tma.cuh"

namespace softsim {

template <typename T>
__device__ __forceinline__ T ldcg(const T *p)
{
    return __ldcg(p);
}

// Fixed-order sum of the G per-CTA partials (FP32 (hi, lo) pairs stored in
// 8-byte slots, or doubles), computed the same way by every CTA; valid in
// every thread.
template <typename T>
__device__ __forceinline__ double grid_sum(const double *slots, int G)
{
    __shared__ double bc;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double r;
        if constexpr (sizeof(T) == 4) {
            float hi = 0.0f, lo = 0.0f;
            for (int i = lane; i < G; i += 32) {
                const float2 v = __ldcg(reinterpret_cast<const float2 *>(slots) + i);
                ds_merge(hi, lo, v.x, v.y);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float h2 = __shfl_down_sync(0xffffffffu, hi, o), l2 = __shfl_down_sync(0xffffffffu, lo, o);
                ds_merge(hi, lo, h2, l2);
            }
            r = (double)hi + (double)lo;
        } else {
            double acc = 0.0;
            for (int i = lane; i < G; i += 32) acc += __ldcg(slots + i);
            r = warp_sum(acc);
        }
        if (lane == 0) bc = r;
    }
    __syncthreads();
    const double v = bc;
    __syncthreads();  // bc is reused by the next call
    return v;
}

// The same fixed-order sum over the G CTAs of a one-cluster grid, each CTA's
// partial read from its shared-memory slot (distributed shared memory) in rank
// order; valid in every thread.
template <typename T>
__device__ __forceinline__ double cluster_sum(const double *slot, int G)
{
    __shared__ double bc;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double r;
        if constexpr (sizeof(T) == 4) {
            float hi = 0.0f, lo = 0.0f;
            if (lane < G) {
                const float2 v = ld_dsmem_f2(slot, (uint32_t)lane);
                ds_merge(hi, lo, v.x, v.y);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float h2 = __shfl_down_sync(0xffffffffu, hi, o), l2 = __shfl_down_sync(0xffffffffu, lo, o);
                ds_merge(hi, lo, h2, l2);
            }
            r = (double)hi + (double)lo;
        } else {
            const double acc = lane < G ? ld_dsmem_f64(slot, (uint32_t)lane) : 0.0;
            r = warp_sum(acc);
        }
        if (lane == 0) bc = r;
    }
    __syncthreads();
    const double v = bc;
    __syncthreads();  // bc is reused by the next call
    return v;
}

// Shared-memory plan (bytes; 16-byte aligned: max_te is a multiple of 8,
// max_tv of 4, rs even).
template <typename T, int D>
struct CoopSmem {
    size_t rec, cor, conn, inc, gid, code, linc, uv, total;
    __host__ __device__ CoopSmem(int max_te, int max_tv, int rs)
    {
        rec = 16;  // one mbarrier
        cor = rec + (size_t)rs * max_te * sizeof(T);
        conn = cor + (size_t)rs * max_te * sizeof(T);
        inc = conn + (size_t)max_te * 4;
        gid = inc + (size_t)max_te * (D + 1) * 2;
        code = gid + (size_t)max_tv * 4;
        linc = code + (size_t)max_tv * 4;
        uv = linc + (size_t)max_tv * 4;
        total = uv + (size_t)max_tv * 2 * D * sizeof(T);
        total = (total + 15) / 16 * 16;
    }
};

// The CG iterations of one solve (the CG scalars rr, tol2, max_iter and done
// come from k_cg_init; the iteration count, the non-positive-curvature flag
// and the final r.r go back to sc).  part: 2 G slots of partial sums.
// CL: the grid is one thread-block cluster (at most 16 CTAs): the barriers
// are the cluster's hardware barrier and the partial sums are read from the
// other CTAs' shared memory instead of through L2.
template <typename T, int D, bool SPRING, bool CL>
__global__ void __launch_bounds__(256) k_cg_coop(TileDev td, const T *__restrict__ erec, VertDev vd, Phys ph,
                                                 const T *__restrict__ u, T *__restrict__ d, T *__restrict__ r,
                                                 T *p, T *Ap, T *hp, double *part, DevScalars *sc)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int NF = hvp_fields(D, SPRING);
    constexpr int RS = rec_stride(NF);
    const CoopSmem<T, D> L(td.max_te, td.max_tv, RS);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    T *sRec = reinterpret_cast<T *>(smem + L.rec);
    T *sCor = reinterpret_cast<T *>(smem + L.cor);
    const uint32_t *sConn = reinterpret_cast<const uint32_t *>(smem + L.conn);
    const uint16_t *sInc = reinterpret_cast<const uint16_t *>(smem + L.inc);
    const int32_t *sGid = reinterpret_cast<const int32_t *>(smem + L.gid);
    const int32_t *sCode = reinterpret_cast<const int32_t *>(smem + L.code);
    const uint32_t *sLinc = reinterpret_cast<const uint32_t *>(smem + L.linc);
    T *suv = reinterpret_cast<T *>(smem + L.uv);
    const int t = blockIdx.x, G = gridDim.x;
    const int es = td.tile_elem[t], ne_t = td.tile_elem[t + 1] - es;
    const int vs = td.tile_vert[t], nlv = td.tile_vert[t + 1] - vs;
    unsigned int *gword = &sc->gs_count;
    __shared__ __align__(16) double cl_slot[2];  // CL: this CTA's p.Ap and r.r partials
    __shared__ int cl_bad;

    // the tile's static data, once for the whole solve
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        const uint32_t brec = (uint32_t)ne_t * RS * sizeof(T);
        mbar_arrive_expect_tx(bar, brec + (uint32_t)ne_t * 4 + (uint32_t)ne_t * (D + 1) * 2 + 3u * nlv * 4);
        bulk_g2s(sRec, erec + (int64_t)es * RS, brec, bar);
        bulk_g2s(smem + L.conn, td.conn + es, (uint32_t)ne_t * 4, bar);
        bulk_g2s(smem + L.inc, td.inc + (int64_t)es * (D + 1), (uint32_t)ne_t * (D + 1) * 2, bar);
        bulk_g2s(smem + L.gid, td.lv_gid + vs, (uint32_t)nlv * 4, bar);
        bulk_g2s(smem + L.code, td.lv_code + vs, (uint32_t)nlv * 4, bar);
        bulk_g2s(smem + L.linc, td.lv_inc + vs, (uint32_t)nlv * 4, bar);
    }
    __syncthreads();
    const int bad = __syncthreads_or(!mbar_wait_bounded(bar, 0, td.wait_polls));
    if constexpr (CL) {
        // no CTA of a cluster may leave alone while the others wait at a
        // cluster barrier: the CTAs agree on the outcome first
        if (threadIdx.x == 0) cl_bad = bad;
        cluster_sync();
        const int any = __syncthreads_or(threadIdx.x < G ? ld_dsmem_s32(&cl_bad, (uint32_t)threadIdx.x) : 0);
        if (any) {
            if (bad && threadIdx.x == 0) {
                atomicOr(&sc->kerr, 1);
                mbar_wait_bounded(bar, 0);  // let copies in flight land before the CTA exits
            }
            cluster_sync();  // the flags have been read everywhere
            return;
        }
    } else if (bad) {
        if (threadIdx.x == 0) {
            atomicOr(&sc->kerr, 1);
            mbar_wait_bounded(bar, 0);  // let copies in flight land before the CTA exits
        }
        return;
    }

    const int64_t nv = vd.nv;
    const int64_t v0 = nv * t / G, v1 = nv * (t + 1) / G;  // this CTA's vertex range for the vector updates
    const T mu = pick<T>(ph.mu, ph.mu_f), lam = pick<T>(ph.lam, ph.lam_f);
    const T sel = pick<T>(ph.s_el, ph.s_el_f), kk = pick<T>(ph.k, ph.k_f);
    const bool contact = ph.kc > 0.0;
    double rr = sc->rr;
    const double tol2 = sc->tol2;
    const int max_iter = sc->max_iter;
    int done = sc->done, neg = 0, it = 0, fail = 0;
    T b_t = T(0);  // beta of this iteration (0 first: p = r; k_cg_init left p = r as well)
    while (!done) {
        // 1. p = r + beta p and A p on the tile
        for (int k = threadIdx.x; k < nlv; k += blockDim.x) {
            const int64_t gid = sGid[k];
            const bool fx = (sLinc[k] & kLvPinned) != 0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                suv[k * 2 * D + c] = u[gid * D + c];
                const T pn = ldcg(r + gid * D + c) + b_t * ldcg(p + gid * D + c);
                suv[k * 2 * D + D + c] = fx ? T(0) : pn;
            }
        }
        __syncthreads();
        T dot = T(0);
        for (int le = threadIdx.x; le < ne_t; le += blockDim.x)
            hvp_element<T, D, true, SPRING, RS>(sRec + le * RS, le, sConn[le], suv, ph, mu, lam, sel, kk, dot,
                                                sCor + le * RS);
        __syncthreads();
        for (int k = threadIdx.x; k < nlv; k += blockDim.x)
            hvp_vertex<T, D, true>(sCode[k], sLinc[k], sGid[k], suv + k * 2 * D, sInc, sCor, vd, ph, Ap, hp, dot);
        {
            CompSum<T> acc;
            acc.add(dot);
            store_block_partial<T>(acc, CL ? &cl_slot[0] : part + t);
        }
        if constexpr (CL) {
            cluster_sync();
        } else if (!grid_barrier(gword, G)) {
            fail = 1;
            break;
        }
        // 2. alpha; p, d and r over this CTA's vertices; r.r
        const double pAp = CL ? cluster_sum<T>(&cl_slot[0], G) : grid_sum<T>(part, G);
        if (!(pAp > 0.0) || !isfinite(pAp)) {
            neg = 1;
            if (it == 0)  // steepest descent: d = p (= the initial residual)
                for (int64_t i = v0 * D + threadIdx.x; i < v1 * D; i += blockDim.x) d[i] = r[i];
            break;
        }
        const double alpha = rr / pAp;
        const T a_t = pick<T>(alpha, (float)alpha);
        CompSum<T> rrs;
        for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x) {
            T a[D], pv[D];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                pv[c] = r[i * D + c] + b_t * p[i * D + c];  // the same bits the gathers formed
                p[i * D + c] = pv[c];
            }
            const int f = td.vfin[i];
            if (f < 0) {
#pragma unroll
                for (int c = 0; c < D; ++c) a[c] = ldcg(Ap + i * D + c);
            } else {
#pragma unroll
                for (int c = 0; c < D; ++c) a[c] = T(0);
                for (int q = td.fin_ptr[f]; q < td.fin_ptr[f + 1]; ++q)
#pragma unroll
                    for (int c = 0; c < D; ++c) a[c] += ldcg(hp + (int64_t)q * D + c);
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
                if (vd.fixed[i])
#pragma unroll
                    for (int c = 0; c < D; ++c) a[c] = T(0);
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                d[i * D + c] += a_t * pv[c];
                const T ri = r[i * D + c] - a_t * a[c];
                r[i * D + c] = ri;
                rrs.add(ri * ri);
            }
        }
        store_block_partial<T>(rrs, CL ? &cl_slot[1] : part + G + t);
        if constexpr (CL) {
            cluster_sync();
        } else if (!grid_barrier(gword, G)) {
            fail = 1;
            break;
        }
        // beta and the convergence test, the same in every CTA
        const double rr_new = CL ? cluster_sum<T>(&cl_slot[1], G) : grid_sum<T>(part + G, G);
        ++it;
        const double beta = rr_new / rr;
        rr = rr_new;
        if (rr <= tol2 || it >= max_iter || !isfinite(rr)) break;
        b_t = pick<T>(beta, (float)beta);
    }
    if constexpr (CL) cluster_sync();  // every CTA has read the others' last partials
    if (fail && threadIdx.x == 0) atomicOr(&sc->kerr, 2);
    if (t == 0 && threadIdx.x == 0) {
        sc->iter = it;
        sc->negcurv = neg;
        sc->rr = rr;
        sc->done = 1;
    }
}

// ---------------------------------------------------------------- host side

template <typename T, int D, bool SPRING, bool CL>
static void coop_kernel_ptr(void **k)
{
    *k = (void *)k_cg_coop<T, D, SPRING, CL>;
}

template <typename T, bool CL = false>
static void *coop_kernel(const Ctx &c)
{
    void *k = nullptr;
    if (c.dim == 2)
        c.muscle ? coop_kernel_ptr<T, 2, true, CL>(&k) : coop_kernel_ptr<T, 2, false, CL>(&k);
    else
        c.muscle ? coop_kernel_ptr<T, 3, true, CL>(&k) : coop_kernel_ptr<T, 3, false, CL>(&k);
    return k;
}

template <typename T>
static size_t coop_smem(const Ctx &c)
{
    return c.dim == 2 ? CoopSmem<T, 2>(c.td.max_te, c.td.max_tv, c.td.rs).total
                      : CoopSmem<T, 3>(c.td.max_te, c.td.max_tv, c.td.rs).total;
}

constexpr int kMaxClusterCtas = 16;  // the largest (non-portable) cluster GB300 schedules

// Launch configuration of the one-cluster grid (cluster = grid = n_tiles CTAs).
static cudaLaunchConfig_t cluster_config(const Ctx &c, size_t smem, cudaStream_t s, cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.td.n_tiles);
    cfg.blockDim = dim3(c.threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c.td.n_tiles;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// Whether the mesh's tiles fit in one thread-block cluster (at most 16 CTAs,
// one resident cluster possible with this kernel's shared memory).
template <typename T>
static bool cg_cluster_fits(const Ctx &c)
{
    int &fit = c.coop_fit[sizeof(T) == 4 ? 2 : 3];
    if (fit < 0) {
        fit = 0;
        const size_t sm = coop_smem<T>(c);
        void *k = coop_kernel<T, true>(c);
        int n_clusters = 0;
        cudaLaunchAttribute at[1];
        const cudaLaunchConfig_t cfg = cluster_config(c, sm, nullptr, at);
        if (c.td.n_tiles >= 1 && c.td.n_tiles <= kMaxClusterCtas && sm <= 220 * 1024 &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess &&
            cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
            cudaOccupancyMaxActiveClusters(&n_clusters, k, &cfg) == cudaSuccess)
            fit = n_clusters >= 1 ? 1 : 0;
        cudaGetLastError();
    }
    return fit == 1;
}

template <typename T>
bool cg_coop_fits(const Ctx &c)
{
    if (cg_cluster_fits<T>(c)) return true;
    int &fit = c.coop_fit[sizeof(T) == 4 ? 0 : 1];
    if (fit < 0) {
        fit = 0;
        const size_t sm = coop_smem<T>(c);
        void *k = coop_kernel<T>(c);
        int dev = 0, n_sm = 0, per_sm = 0;
        if (sm <= 220 * 1024 && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, c.threads, sm) == cudaSuccess)
            fit = (int64_t)per_sm * n_sm >= c.td.n_tiles ? 1 : 0;
        cudaGetLastError();
    }
    return fit == 1;
}

template <typename T>
cudaError_t launch_cg_coop(const Ctx &c, const Phys &ph, const T *u, T *d, T *r, T *p, T *Ap, T *hp,
                           cudaStream_t s)
{
    const bool cl = cg_cluster_fits<T>(c);
    if (!cl) {
        cudaError_t e = cudaMemsetAsync(&c.sc->gs_count, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
    }
    c.n_launch += 1;
    const T *er = sizeof(T) == 4 ? reinterpret_cast<const T *>(c.rec32) : reinterpret_cast<const T *>(c.rec64);
    double *part = c.partials;
    DevScalars *sc = c.sc;
    TileDev td = c.td;
    VertDev vd = c.vd;
    Phys phv = ph;
    void *args[] = {&td, (void *)&er, &vd, &phv, (void *)&u, &d, &r, &p, &Ap, &hp, &part, &sc};
    if (cl) {  // one cluster: every CTA co-scheduled by construction
        cudaLaunchAttribute at[1];
        const cudaLaunchConfig_t cfg = cluster_config(c, coop_smem<T>(c), s, at);
        return cudaLaunchKernelExC(&cfg, coop_kernel<T, true>(c), args);
    }
    return cudaLaunchCooperativeKernel(coop_kernel<T>(c), dim3(c.td.n_tiles), dim3(c.threads), args,
                                       coop_smem<T>(c), s);
}

template bool cg_coop_fits<float>(const Ctx &);
template bool cg_coop_fits<double>(const Ctx &);
template cudaError_t launch_cg_coop<float>(const Ctx &, const Phys &, const float *, float *, float *, float *,
                                           float *, float *, cudaStream_t);
template cudaError_t launch_cg_coop<double>(const Ctx &, const Phys &, const double *, double *, double *,
                                            double *, double *, double *, cudaStream_t);

}  // namespace softsim
