// Internal structures shared by the translation units of libsoftsim.
//
// Data layout in device memory (one handle = one mesh):
//   * Elements are stored in "tile order": a locality-preserving (Morton)
//     order cut into tiles of at most max_te elements touching at most
//     max_tv (<= 256) vertices.  perm[e] maps tile order -> caller order.
//   * Per-element static data is structure-of-arrays, one field per array of
//     `stride` entries: Dm^-1 (dim*dim fields, row-major), g = Dm^-1 f (dim),
//     W (1), f (dim); FP64, read by the energy, gradient and VJP kernels.
//   * The HVP kernels read per-element records instead, [ne_int][rs] (FP32 and
//     FP64 copies): the hvp_fields() fields in the order above (f only with
//     the spring muscle), the activation, padding to rs = rec_stride(), and
//     in shared memory the element's corner forces overwrite its own record
//     from slot corner_base(local elem).
//   * conn[e] packs the element's dim+1 tile-local vertex ids, 8 bits each.
//   * A tile's local vertices are lv_gid[tile_vert[t] .. tile_vert[t+1]),
//     sorted by global id.  lv_code < 0: the vertex belongs to this tile only
//     and the tile writes its final value; otherwise the tile writes a partial
//     sum to halo slot (lv_code >> 1) and bit 0 says whether this tile is the
//     vertex's owner (first tile touching it; owners add per-vertex energy
//     terms).  Halo and element-less vertices are listed in fin_gid; their
//     partial-sum slots are fin_ptr[i] .. fin_ptr[i+1], in tile order, so
//     every vertex sum is formed in one fixed order (deterministic, no float
//     atomics).
//   * inc[tile_elem[t]*(dim+1) + s], s in [first, first+count) of lv_inc[lv],
//     lists the corners that touch local vertex lv, each encoded as the
//     offset local_elem*rs + corner_base(local_elem) + corner*dim of its dim
//     values among the tile's records; the tile builder picks the order of
//     each list and where it starts so that the lanes of a warp read from
//     distinct shared-memory banks.  lv_inc also flags pinned vertices.
//   * Per-tile ranges are padded to 16-byte multiples for bulk copies;
//     padding elements have W = 0 and perm -1, padding local vertices have
//     lv_code == LV_PAD and no incidences.
//   * Vertex fields are row-major [n_vert][dim].
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "layout.h"

namespace softsim {

constexpr int kMaxTileVerts = 256;   // local ids fit in 8 bits
constexpr int kMaxTrials = 8;        // step lengths evaluated per energy launch

struct TileDev {
    int n_tiles = 0;
    int max_te = 0, max_tv = 0;
    int n_fin = 0;
    int rs = 0;                          // element-record stride (words), rec_stride(hvp_fields(dim, spring))
    // when every tile has the same padded element and local-vertex counts
    // (a regular mesh cut into equal blocks), those counts: a tile's ranges
    // then follow from its index without loading tile_elem / tile_vert
    int uni_te = 0, uni_tv = 0;
    const int32_t *tile_elem = nullptr;  // [n_tiles + 1]
    const int32_t *tile_vert = nullptr;  // [n_tiles + 1]
    const int32_t *lv_gid = nullptr;     // [n_lv]
    const int32_t *lv_code = nullptr;    // [n_lv]
    const uint32_t *lv_inc = nullptr;    // [n_lv] first incidence (within the tile) | count << 16 | pinned
    // inc entries: the offset of a corner's dim values among the tile's element
    // records, local element * rs + corner_base(local element) + corner * dim
    const uint16_t *inc = nullptr;       // [ne_int * (dim+1)]
    const uint32_t *conn = nullptr;      // [ne_int]
    const int32_t *perm = nullptr;       // [ne_int] tile order -> caller order, -1 = padding
    const int32_t *fin_gid = nullptr;    // [n_fin]
    const int32_t *fin_ptr = nullptr;    // [n_fin + 1]
    const int32_t *vfin = nullptr;       // [nv] halo index of a vertex, -1 if one tile owns it
    // the same tables packed for the HVP tile kernel's bulk copies:
    const int32_t *lv3 = nullptr;        // [n_lv][3] gid, code, lv_inc of each local vertex
    const uint8_t *ci = nullptr;         // per tile at byte es * (4 + 2 (dim+1)): conn [ne_t] u32, then the
                                         // tile's incidence block [ne_t (dim+1)] u16
    // poll limit of the HVP tile kernel's first bulk-copy wait (the copies of
    // the vertex tables); the library default is the same bound as every
    // other wait, and sim_set_wait_limit lowers it to exercise the error path
    int wait_polls = 1 << 22;
};

template <typename T>
struct ElemDev {
    const T *base = nullptr;  // SoA block
    int64_t stride = 0;       // entries per field
    __host__ __device__ const T *field(int k) const { return base + (int64_t)k * stride; }
};

struct VertDev {
    int64_t nv = 0;
    const double *X = nullptr;      // [nv][dim] rest positions
    const double *mass = nullptr;   // [nv]
    const uint8_t *fixed = nullptr; // [nv]
};

// Physical scalars of one evaluation.  s_el scales the potential-energy
// terms (dt^2 for the backward-Euler incremental potential, else 1); dyn
// adds the inertia term 1/2 |x - xhat|_M^2 and its derivatives.  With ground
// friction (dynamics only), fw is non-null and the potential gains
// sum_i fw_i/2 |x_i - x0_i|^2 over the horizontal axes (all but y), which is
// dt^2 k_f |v_h|^2 ReLU(eps - y0_i) at v = (x - x0)/dt.
struct Phys {
    double mu = 0, lam = 0, k = 0, grav = 0, kc = 0;
    int cpow = 3;
    int log_mode = 0;
    int dyn = 0;
    double s_el = 1.0;
    int muscle = 0;              // 0: contractile (k/2) a |F f|^2; 1: active spring (k/2)(|F f|/a - 1)^2
    // FP32 copies for the FP32 kernels (GB300 converts FP64 at the FP64 rate, 1/64 of FP32)
    float mu_f = 0, lam_f = 0, k_f = 0, s_el_f = 1;
    int contact = 0;             // kc > 0
    const double *fw = nullptr;  // [nv] 2 k_f ReLU(eps - y0), or null: no friction
    const double *u0 = nullptr;  // [nv][dim] displacement x0 - X of the step's start
};

#ifdef __CUDACC__
// A constant in the kernel's precision, from its FP64 value or its FP32 copy
// rounded once elsewhere (no conversion in every thread).
template <typename T>
__device__ __forceinline__ T pick(double d, float f)
{
    if constexpr (sizeof(T) == 4)
        return f;
    else
        return d;
}
#endif

// Scalars that the kernels exchange in device memory (no host round trip).
struct DevScalars {
    // conjugate gradients
    double rr, tol2, pAp, alpha, beta;
    float alpha_f, beta_f;  // FP32 copies of alpha and beta for the FP32 vector kernels
    int iter, max_iter, done, negcurv;
    int cg_rounds, cg_max_rounds;  // body rounds of the device-side CG loop and their cap
    unsigned int gs_count, gs_pad;  // grid-barrier word of the cooperative CG kernel (zeroed before each launch)
    // Newton
    double gn2;      // |g|^2 of the FP64 gradient
    double gd;       // g . d
    int dir_fix;     // 1: CG gave no descent direction, d := -g
    int pad0;
    // energies of the line-search trials: E, sum |terms|, min J
    double E[kMaxTrials], S[kMaxTrials];
    double minJ;
    int inverted;
    int kerr;        // kernel-side error flags (1: bulk-copy wait timed out)
    unsigned int ticket[8];  // last-block-done counters, reset by the last block
};

struct TrialT {
    int n;
    double t[kMaxTrials];
};

enum Ticket { TK_CGINIT = 0, TK_ENERGY = 1, TK_GD = 2, TK_GRAD = 3, TK_MISC = 4 };

// Everything a launcher needs about one mesh.
struct Ctx {
    int dim = 0;
    int64_t nv = 0, ne = 0, ne_int = 0;
    TileDev td;
    VertDev vd;
    ElemDev<double> e64;
    // HVP element records [ne_int][td.rs] in tile order: the hvp_fields()
    // element fields, then the activation (written by set_activation)
    float *rec32 = nullptr;   // mixed precision only
    double *rec64 = nullptr;
    int threads = 256;
    int muscle = 0;              // muscle model (the spring's HVP also stages the fiber)
    double *partials = nullptr;  // [n_partials] FP64 block partial sums
    int n_fin_blocks = 1;
    DevScalars *sc = nullptr;
    mutable int64_t n_launch = 0;  // kernels launched through this context
    mutable bool pdl = false;      // launch CG-loop kernels with programmatic dependent launch
    // [FP32, FP64] the cooperative CG kernel fits as a cooperative grid, then
    // [FP32, FP64] as one thread-block cluster: 1 / 0, -1 = not checked
    mutable int coop_fit[4] = {-1, -1, -1, -1};
};

// ---------------------------------------------------------------- launchers
// Element kernels (elem_kernels.cu).  All vertex fields are displacements
// u = x - X or directions, [nv][dim]; `a` is in tile order.

// Multi-trial energy: for j < n_trials, E_j = energy at u + t_j dir (dir may
// be null with n_trials = 1, t = 0).  Writes sc->E[j], sc->S[j], sc->minJ.
void launch_energy(const Ctx &c, const Phys &ph, const double *u, const double *dir,
                   const double *uhat, const double *a, const double *t, int n_trials,
                   cudaStream_t s);

// FP64 gradient of the energy (with inertia when ph.dyn), masked; writes
// sc->gn2 = |g|^2.  hp: halo scratch [n_slots][dim] double.
void launch_grad(const Ctx &c, const Phys &ph, const double *u, const double *uhat,
                 const double *a, double *g, double *hp, cudaStream_t s);

// HVP y = A v (A = H, or M + dt^2 H when ph.dyn), masked; the activations
// come from the element records.
template <typename T>
void launch_hvp(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y, T *hp, cudaStream_t s);
template <typename T>
void launch_hvp_tile_only(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y, T *hp, cudaStream_t s);
template <typename T>
void launch_hvp_finalize_only(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y,
                              const T *hp, cudaStream_t s);

template <typename T>
size_t hvp_smem(const Ctx &c);
cudaError_t configure_elem_kernels();

// dLda[perm[e]] = -s_el W (d2psi_m/dq da).(dF(lam) f), q = F f; a in tile order
void launch_param_vjp(const Ctx &c, const Phys &ph, const double *u, const double *a, const double *lam,
                      double *dLda, cudaStream_t s);
// per-element dL/dmu, dL/dlambda, dL/dk (caller order; null outputs skipped)
void launch_material_vjp(const Ctx &c, const Phys &ph, const double *u, const double *a, const double *lam,
                         double *dmu, double *dlam, double *dk, cudaStream_t s);

// ---------------------------------------------------------------- cooperative CG (cg_coop.cu)
// Whether every tile can be resident at once for the cooperative CG kernel.
template <typename T>
bool cg_coop_fits(const Ctx &c);
// The CG iterations of one solve in one cooperative launch (after
// launch_cg_init; results in sc as from the per-iteration kernels).
template <typename T>
cudaError_t launch_cg_coop(const Ctx &c, const Phys &ph, const T *u, T *d, T *r, T *p, T *Ap, T *hp,
                           cudaStream_t s);

// ---------------------------------------------------------------- vector kernels (vec_kernels.cu)
template <typename T>
void launch_cg_init(const Ctx &c, const double *b, double sign, T *d, T *r, T *p, double rtol,
                    int max_iter, int max_rounds, cudaStream_t s);
// Condition of the device-side CG loop (last node of a WHILE body): go on
// while CG runs, no kernel gave up on a wait, and fewer than max_rounds
// bodies have run.
void launch_cg_cond(const Ctx &c, cudaGraphConditionalHandle hnd, cudaStream_t s);
// CG update that first completes A p: vertices of one tile take it from Ap
// (written by the HVP tile kernel), halo vertices add their partial sums hp
// and their per-vertex terms; then d += alpha p, r -= alpha A p, r.r, beta.
template <typename T>
void launch_cg_update_halo(const Ctx &c, const Phys &ph, const T *u, T *d, T *r, const T *p, const T *Ap,
                           const T *hp, cudaStream_t s);
// HVP tile kernel of the CG loop: A p for single-tile vertices, halo
// partials, and p.Ap partials from element quadratic forms (no finalize; the
// caller launches launch_cg_alpha next).
template <typename T>
void launch_hvp_cg(const Ctx &c, const Phys &ph, const T *u, const T *v, T *y, T *hp, cudaStream_t s);
template <typename T>
void launch_cg_dir(const Ctx &c, T *p, const T *r, cudaStream_t s);
template <typename T>
void launch_dir_check(const Ctx &c, const double *g, T *d, cudaStream_t s);
// *out = sum of the HVP tile kernel's v.Av partials, summed as k_cg_alpha does
template <typename T>
void launch_tile_dot(const Ctx &c, double *out, cudaStream_t s);
template <typename T>
void launch_step_update(const Ctx &c, double *u, const T *d, double t, float *u32, cudaStream_t s);

void launch_x_to_u(const Ctx &c, const double *x, double *u, float *u32, const uint8_t *fixed_pin,
                   cudaStream_t s);
void launch_u_to_x(const Ctx &c, const double *u, double *x, cudaStream_t s);
void launch_uhat(const Ctx &c, const double *x0, const double *v0, double dt, double *uhat,
                 cudaStream_t s);
template <typename T>
// internal[e * stride] = user[perm[e]] (0 for padding elements), e in tile order
void launch_gather_elem(const Ctx &c, const double *user, T *internal, cudaStream_t s, int64_t stride = 1);
template <typename Tin, typename Tout>
void launch_convert(int64_t n, const Tin *in, Tout *out, cudaStream_t s);
void launch_mask_copy(const Ctx &c, const double *in, double *out, cudaStream_t s);
// step backward: xbar0 = M lam - vbar1/dt, vbar0 = dt M lam (masked)
// u0 = x0 - X and fw = 2 k_f ReLU(eps - y0) for the friction of one step
void launch_friction_prep(const Ctx &c, const double *x0, double kf, double eps, double *u0, double *fw,
                          cudaStream_t s);
void launch_step_bwd_combine(const Ctx &c, const double *lam, const double *vbar1, double dt, const double *fw,
                             double kf, const double *x0, const double *x1, double *xbar0, double *vbar0,
                             cudaStream_t s);
// b = xbar1 + vbar1/dt
void launch_axpy_out(int64_t n, const double *x, const double *y, double beta, double *out,
                     cudaStream_t s);
// u4[i] = (u[3i], u[3i+1], u[3i+2], 0) for the 3D FP32 CG tile kernel
void launch_pad_rows4(const Ctx &c, const float *u, float *u4, cudaStream_t s);
// blocks of the grid-stride vector kernels for n entries
int vec_grid_size(int64_t n);
int cg_update_grid_size(int64_t nv);  // blocks of the CG update kernel (one vertex per thread)
// One block: p.Ap from the HVP tile partials (type T: FP32 partials are summed
// with compensation) -> sc->alpha, or non-positive curvature.
template <typename T>
void launch_cg_alpha(const Ctx &c, int n_partials, cudaStream_t s);
// r = b - Ax, |r|^2 -> sc->gn2
void launch_residual(const Ctx &c, const double *b, const double *Ax, double *r, cudaStream_t s);
// x += d
template <typename T>
void launch_accumulate(const Ctx &c, double *x, const T *d, cudaStream_t s);
// v1 = (x1 - x0)/dt
void launch_velocity(int64_t n, const double *x1, const double *x0, double dt, double *v1,
                     cudaStream_t s);

}  // namespace softsim
