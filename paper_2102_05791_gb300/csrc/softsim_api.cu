// C ABI of libsoftsim: handle construction and the solvers.
//
// Forward: x* = argmin_x E(x, a) (Eq. x1-quasistatic-argmin) or the
// backward-Euler incremental potential (Eq. opt-be), by Newton-CG.  The
// paper minimises with a first-order descent method and line search and
// states that the forward minimiser may be chosen freely (Sec. 2, Sec. 5);
// Newton-CG is used here because the HVP is available anyway.
// Backward: CG on H lambda = dL/dx, then dL/da = -lambda^T d2E/dx da
// (Eq. dLda-re-ordered), with H applied matrix-free (Eq. matrix-free-dfdx).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "softsim.h"
#include "tiling.h"

using namespace softsim;

namespace {

thread_local std::string g_create_error;
constexpr int kCgBlock = 16;  // CG iterations per captured graph (host-driven loop)
constexpr int kCgBody = 8;    // CG iterations per round of the device-side loop

struct Graph {
    cudaGraphExec_t exec = nullptr;
    bool valid = false;
};

// The whole CG solve as one graph: a WHILE conditional node whose body runs
// kCgBody iterations and then sets the condition on the device.
struct WhileGraph {
    cudaGraphExec_t exec = nullptr;
    int state = 0;  // 0: not built yet, 1: built, -1: refused by this CUDA build (host-driven loop instead)
};

}  // namespace

struct sim_handle {
    int dim = 0, precision = SIM_PREC_MIXED, device = 0;
    int64_t nv = 0, ne = 0;
    sim_material mat{};
    sim_options opt{};
    Ctx ctx;
    TileBuild tb;
    std::vector<void *> allocs;
    // device state
    double *X = nullptr, *mass = nullptr;
    uint8_t *fixed = nullptr;
    double *u = nullptr, *uhat = nullptr, *g = nullptr, *hp64 = nullptr, *a64 = nullptr;
    double *fw = nullptr, *u0 = nullptr;  // ground friction of the current step (null when off)
    float *u32 = nullptr, *hp32 = nullptr;
    float *u4 = nullptr;  // 3D FP32 displacement in 16-byte rows, as the CG tile kernel gathers it
    void *vd = nullptr, *vr = nullptr, *vp = nullptr, *vAp = nullptr;  // CG vectors in the HVP precision
    double *work = nullptr, *lam = nullptr, *lacc = nullptr, *r64 = nullptr, *Hx = nullptr;
    int verbose = 0;
    double *rx[2] = {nullptr, nullptr}, *rv[2] = {nullptr, nullptr};  // rollout ping-pong
    DevScalars *sc = nullptr;
    DevScalars *sc_host = nullptr;  // pinned mirror
    cudaStream_t cap = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    Graph cg_graph[2][2];           // [dyn][kernel timing]
    WhileGraph cg_while[2];         // [dyn]
    int timing = 0;                 // record events around HVP tile launches in solves
    cudaEvent_t tev[2 * kCgBlock] = {};
    double t_hvp_ms = 0.0;          // accumulated in-solve HVP tile-kernel time
    int64_t n_hvp_timed = 0;
    std::string err;
};

// ---------------------------------------------------------------- helpers

static int fail(sim_handle *h, int code, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return code;
}

#define CK(h, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), SIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKL(h) CK(h, cudaGetLastError())

static void *dalloc(sim_handle *h, size_t bytes)
{
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    h->allocs.push_back(p);
    return p;
}

template <typename V>
static int upload(sim_handle *h, const std::vector<V> &v, const V **dst)
{
    V *p = (V *)dalloc(h, v.size() * sizeof(V));
    if (!p) return fail(h, SIM_ENOMEM, "device allocation failed");
    if (!v.empty()) CK(h, cudaMemcpy(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
    *dst = p;
    return SIM_OK;
}

static Phys make_phys(const sim_handle *h, bool dyn)
{
    Phys ph;
    ph.mu = h->mat.mu;
    ph.lam = h->mat.lambda;
    ph.k = h->mat.k_muscle;
    ph.grav = h->mat.gravity;
    ph.kc = h->mat.k_contact;
    ph.cpow = h->mat.contact_power;
    ph.log_mode = h->mat.log_mode;
    ph.muscle = h->mat.muscle_model;
    ph.dyn = dyn ? 1 : 0;
    ph.s_el = dyn ? h->mat.dt * h->mat.dt : 1.0;
    ph.mu_f = (float)ph.mu;
    ph.lam_f = (float)ph.lam;
    ph.k_f = (float)ph.k;
    ph.s_el_f = (float)ph.s_el;
    ph.contact = ph.kc > 0.0 ? 1 : 0;
    if (dyn && h->fw) {
        ph.fw = h->fw;
        ph.u0 = h->u0;
    }
    return ph;
}

static int read_scalars(sim_handle *h, cudaStream_t s)
{
    CK(h, cudaMemcpyAsync(h->sc_host, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    if (h->sc_host->kerr) {
        // clear the flag so that the handle's next call starts clean
        CK(h, cudaMemsetAsync(&h->sc->kerr, 0, sizeof(int), s));
        CK(h, cudaStreamSynchronize(s));
        return fail(h, SIM_ECUDA, h->sc_host->kerr & 2 ? "a kernel gave up waiting at a grid barrier"
                                                       : "a kernel gave up waiting for its bulk copies");
    }
    return SIM_OK;
}

static void drop_graphs(sim_handle *h)
{
    for (auto &row : h->cg_graph)
        for (auto &gr : row) {
            if (gr.exec) cudaGraphExecDestroy(gr.exec);
            gr.exec = nullptr;
            gr.valid = false;
        }
    for (auto &wg : h->cg_while) {
        if (wg.exec) cudaGraphExecDestroy(wg.exec);
        wg.exec = nullptr;
        wg.state = 0;
    }
}

static bool is_mixed(const sim_handle *h) { return h->precision == SIM_PREC_MIXED; }

// ---------------------------------------------------------------- options

extern "C" int sim_default_options(sim_options *o)
{
    if (!o) return SIM_EINVAL;
    memset(o, 0, sizeof(*o));
    o->precision = SIM_PREC_MIXED;
    o->newton_rtol = 1e-8;
    o->newton_forcing = 0.5;
    o->adjoint_rtol = 1e-6;
    o->max_newton = 100;
    o->max_cg = 500;
    o->max_adjoint_cg = 0;  // 0 = 4 * n_dof
    o->max_ls = 30;
    o->tile_elems = 0;
    o->threads = 0;
    return SIM_OK;
}

extern "C" const char *sim_last_error(const sim_handle *h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

extern "C" int sim_sizes(const sim_handle *h, int *dim, int64_t *nv, int64_t *ne)
{
    if (!h) return SIM_EINVAL;
    if (dim) *dim = h->dim;
    if (nv) *nv = h->nv;
    if (ne) *ne = h->ne;
    return SIM_OK;
}

extern "C" int sim_tile_stats(const sim_handle *h, int *n_tiles, double *ept, double *vpt, double *halo)
{
    if (!h) return SIM_EINVAL;
    const int nt = h->tb.n_tiles;
    if (n_tiles) *n_tiles = nt;
    if (ept) *ept = nt ? (double)h->ne / nt : 0.0;
    if (vpt) *vpt = nt ? (double)h->tb.n_real_lv / nt : 0.0;
    if (halo) *halo = h->nv ? (double)h->tb.fin_gid.size() / h->nv : 0.0;
    return SIM_OK;
}

extern "C" int sim_destroy(sim_handle *h)
{
    if (!h) return SIM_EINVAL;
    drop_graphs(h);
    for (auto &e : h->tev)
        if (e) cudaEventDestroy(e);
    for (void *p : h->allocs) cudaFree(p);
    if (h->sc_host) cudaFreeHost(h->sc_host);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
    return SIM_OK;
}

// ---------------------------------------------------------------- create

static int create_impl(sim_handle *h, const sim_mesh *mesh, const sim_material *mat, const sim_options *opt)
{
    const int d = mesh->dim;
    const int nc = d + 1;
    const int64_t nv = mesh->n_vert, ne = mesh->n_elem;
    h->dim = d;
    h->nv = nv;
    h->ne = ne;
    h->mat = *mat;
    h->mat.fiber = nullptr;
    if (opt)
        h->opt = *opt;
    else
        sim_default_options(&h->opt);
    if (h->opt.max_adjoint_cg <= 0) h->opt.max_adjoint_cg = (int)std::min<int64_t>(4 * nv * d, 1 << 30);
    h->precision = h->opt.precision;
    {
        const char *v = getenv("SOFTSIM_VERBOSE");
        h->verbose = (v && *v && *v != '0') ? 1 : 0;
    }
    CK(h, cudaGetDevice(&h->device));

    // --- validation and rest data (host, FP64)
    for (int64_t i = 0; i < ne * nc; ++i)
        if (mesh->elems[i] < 0 || mesh->elems[i] >= nv) return fail(h, SIM_EINVAL, "element vertex id out of range");
    for (int64_t i = 0; i < nv * d; ++i)
        if (!std::isfinite(mesh->rest_pos[i])) return fail(h, SIM_ENAN, "non-finite rest position");
    const int nf = d * d + 2 * d + 1;
    std::vector<double> mass(nv, 0.0);
    std::vector<double> Wv(ne);
    for (int64_t e = 0; e < ne; ++e) {
        double Dm[3][3] = {{0}};
        const int32_t *t = mesh->elems + e * nc;
        for (int k = 0; k < d; ++k)
            for (int i = 0; i < d; ++i) Dm[i][k] = mesh->rest_pos[(int64_t)t[k + 1] * d + i] - mesh->rest_pos[(int64_t)t[0] * d + i];
        double det, B[3][3] = {{0}};
        if (d == 2) {
            det = Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0];
            B[0][0] = Dm[1][1] / det;
            B[0][1] = -Dm[0][1] / det;
            B[1][0] = -Dm[1][0] / det;
            B[1][1] = Dm[0][0] / det;
        } else {
            double C[3][3];
            for (int j = 0; j < 3; ++j) {
                const int a = (j + 1) % 3, b = (j + 2) % 3;
                C[0][j] = Dm[1][a] * Dm[2][b] - Dm[2][a] * Dm[1][b];
                C[1][j] = Dm[2][a] * Dm[0][b] - Dm[0][a] * Dm[2][b];
                C[2][j] = Dm[0][a] * Dm[1][b] - Dm[1][a] * Dm[0][b];
            }
            det = Dm[0][0] * C[0][0] + Dm[1][0] * C[1][0] + Dm[2][0] * C[2][0];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) B[i][j] = C[j][i] / det;  // Dm^-1 = cof^T / det
        }
        if (!(det > 0.0)) return fail(h, SIM_EINVERTED, "element " + std::to_string(e) + " has non-positive rest volume");
        const double W = det / (d == 2 ? 2.0 : 6.0);
        Wv[e] = W;
        for (int k = 0; k < nc; ++k) mass[t[k]] += mat->density * W / nc;
    }
    std::vector<uint8_t> fixed(nv, 0);
    if (mesh->fixed)
        for (int64_t i = 0; i < nv; ++i) fixed[i] = mesh->fixed[i] ? 1 : 0;

    // --- tiles
    int te = h->opt.tile_elems > 0 ? h->opt.tile_elems : (d == 3 ? 384 : 512);
    const int nf_hvp = hvp_fields(d, h->mat.muscle_model == SIM_MUSCLE_SPRING);
    const int rs = rec_stride(nf_hvp);
    std::string terr;
    if (!build_tiles(d, nv, ne, mesh->rest_pos, mesh->elems, mesh->fixed, te, kMaxTileVerts, rs, h->tb, terr))
        return fail(h, SIM_EINVAL, "tiling: " + terr);
    const TileBuild &tb = h->tb;
    const int64_t ne_int = tb.ne_int;

    // element SoA in (padded) tile order; padding elements stay all-zero (W = 0)
    std::vector<double> edata((size_t)nf * ne_int, 0.0);
    for (int64_t i = 0; i < ne_int; ++i) {
        const int64_t e = tb.perm[i];
        if (e < 0) continue;
        const int32_t *t = mesh->elems + e * nc;
        double Dm[3][3] = {{0}}, B[3][3] = {{0}};
        for (int k = 0; k < d; ++k)
            for (int r = 0; r < d; ++r) Dm[r][k] = mesh->rest_pos[(int64_t)t[k + 1] * d + r] - mesh->rest_pos[(int64_t)t[0] * d + r];
        // recompute Dm^-1 (cheap) in tile order
        if (d == 2) {
            const double det = Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0];
            B[0][0] = Dm[1][1] / det;
            B[0][1] = -Dm[0][1] / det;
            B[1][0] = -Dm[1][0] / det;
            B[1][1] = Dm[0][0] / det;
        } else {
            double C[3][3];
            for (int j = 0; j < 3; ++j) {
                const int a = (j + 1) % 3, b = (j + 2) % 3;
                C[0][j] = Dm[1][a] * Dm[2][b] - Dm[2][a] * Dm[1][b];
                C[1][j] = Dm[2][a] * Dm[0][b] - Dm[0][a] * Dm[2][b];
                C[2][j] = Dm[0][a] * Dm[1][b] - Dm[1][a] * Dm[0][b];
            }
            const double det = Dm[0][0] * C[0][0] + Dm[1][0] * C[1][0] + Dm[2][0] * C[2][0];
            for (int r = 0; r < 3; ++r)
                for (int j = 0; j < 3; ++j) B[r][j] = C[j][r] / det;
        }
        double f[3] = {0, 0, 0};
        if (mat->fiber)
            for (int c = 0; c < d; ++c) f[c] = mat->fiber[e * d + c];
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) edata[(size_t)(r * d + c) * ne_int + i] = B[r][c];
        for (int r = 0; r < d; ++r) {
            double s = 0.0;
            for (int c = 0; c < d; ++c) s += B[r][c] * f[c];
            edata[(size_t)(d * d + r) * ne_int + i] = s;
            edata[(size_t)(d * d + d + 1 + r) * ne_int + i] = f[r];
        }
        edata[(size_t)(d * d + d) * ne_int + i] = Wv[e];
    }

    // --- upload
    int rc;
    const double *cX, *cm;
    const uint8_t *cf;
    std::vector<double> Xv(mesh->rest_pos, mesh->rest_pos + nv * d);
    if ((rc = upload(h, Xv, &cX))) return rc;
    if ((rc = upload(h, mass, &cm))) return rc;
    if ((rc = upload(h, fixed, &cf))) return rc;
    h->X = const_cast<double *>(cX);
    h->mass = const_cast<double *>(cm);
    h->fixed = const_cast<uint8_t *>(cf);
    const double *ce64;
    if ((rc = upload(h, edata, &ce64))) return rc;
    Ctx &c = h->ctx;
    c.dim = d;
    c.nv = nv;
    c.ne = ne;
    c.ne_int = ne_int;
    c.e64.base = ce64;
    c.e64.stride = ne_int;
    {
        // HVP records: the first nf_hvp fields in the FI order, activation slot and padding zero
        std::vector<double> rec((size_t)rs * ne_int, 0.0);
        for (int64_t i = 0; i < ne_int; ++i)
            for (int f = 0; f < nf_hvp; ++f) rec[(size_t)i * rs + f] = edata[(size_t)f * ne_int + i];
        const double *cr64;
        if ((rc = upload(h, rec, &cr64))) return rc;
        c.rec64 = const_cast<double *>(cr64);
        if (is_mixed(h)) {
            std::vector<float> rec32(rec.begin(), rec.end());
            const float *cr32;
            if ((rc = upload(h, rec32, &cr32))) return rc;
            c.rec32 = const_cast<float *>(cr32);
        }
    }
    c.vd.nv = nv;
    c.vd.X = h->X;
    c.vd.mass = h->mass;
    c.vd.fixed = h->fixed;
    TileDev &td = c.td;
    td.n_tiles = tb.n_tiles;
    td.max_te = tb.max_te;
    td.max_tv = tb.max_tv;
    td.n_fin = (int)tb.fin_gid.size();
    td.rs = tb.rs;
    {
        bool uni = tb.n_tiles > 0;
        const int te0 = tb.tile_elem[1] - tb.tile_elem[0], tv0 = tb.tile_vert[1] - tb.tile_vert[0];
        for (int t = 1; uni && t < tb.n_tiles; ++t)
            uni = tb.tile_elem[t + 1] - tb.tile_elem[t] == te0 && tb.tile_vert[t + 1] - tb.tile_vert[t] == tv0;
        td.uni_te = uni ? te0 : 0;
        td.uni_tv = uni ? tv0 : 0;
    }
    if ((rc = upload(h, tb.tile_elem, &td.tile_elem))) return rc;
    if ((rc = upload(h, tb.tile_vert, &td.tile_vert))) return rc;
    if ((rc = upload(h, tb.lv_gid, &td.lv_gid))) return rc;
    if ((rc = upload(h, tb.lv_code, &td.lv_code))) return rc;
    if ((rc = upload(h, tb.lv_inc, &td.lv_inc))) return rc;
    if ((rc = upload(h, tb.inc, &td.inc))) return rc;
    if ((rc = upload(h, tb.conn, &td.conn))) return rc;
    if ((rc = upload(h, tb.perm, &td.perm))) return rc;
    if ((rc = upload(h, tb.fin_gid, &td.fin_gid))) return rc;
    if ((rc = upload(h, tb.fin_ptr, &td.fin_ptr))) return rc;
    if ((rc = upload(h, tb.vfin, &td.vfin))) return rc;
    {
        // packed copies of the vertex tables and of conn + incidence lists,
        // so that the HVP tile kernel stages a tile with three bulk copies
        std::vector<int32_t> lv3(tb.lv_gid.size() * 3);
        for (size_t k = 0; k < tb.lv_gid.size(); ++k) {
            lv3[3 * k] = tb.lv_gid[k];
            lv3[3 * k + 1] = tb.lv_code[k];
            lv3[3 * k + 2] = (int32_t)tb.lv_inc[k];
        }
        if ((rc = upload(h, lv3, &td.lv3))) return rc;
        const size_t per = 4 + 2 * (size_t)nc;
        std::vector<uint8_t> ci((size_t)tb.ne_int * per);
        for (int t = 0; t < tb.n_tiles; ++t) {
            const int64_t es = tb.tile_elem[t], ne_t = tb.tile_elem[t + 1] - es;
            uint8_t *dst = ci.data() + (size_t)es * per;
            std::memcpy(dst, tb.conn.data() + es, (size_t)ne_t * 4);
            std::memcpy(dst + (size_t)ne_t * 4, tb.inc.data() + es * nc, (size_t)ne_t * nc * 2);
        }
        if ((rc = upload(h, ci, &td.ci))) return rc;
    }
    c.threads = h->opt.threads > 0 ? h->opt.threads : (d == 3 ? 128 : 256);
    c.muscle = h->mat.muscle_model;
    if (c.threads % 32 || c.threads > 256) return fail(h, SIM_EINVAL, "threads must be a multiple of 32, at most 256");
    c.n_fin_blocks = std::max(1, (td.n_fin + 255) / 256);

    // --- work buffers
    const int64_t nd = nv * d;
    const int n_part = std::max({td.n_tiles + c.n_fin_blocks, vec_grid_size(nd), vec_grid_size(ne_int),
                                  cg_update_grid_size(nv), 1});
    c.partials = (double *)dalloc(h, sizeof(double) * (size_t)n_part * (2 * kMaxTrials + 1));
    h->sc = (DevScalars *)dalloc(h, sizeof(DevScalars));
    c.sc = h->sc;
    const size_t vbytes = is_mixed(h) ? sizeof(float) : sizeof(double);
    h->u = (double *)dalloc(h, sizeof(double) * nd);
    h->uhat = (double *)dalloc(h, sizeof(double) * nd);
    h->g = (double *)dalloc(h, sizeof(double) * nd);
    h->work = (double *)dalloc(h, sizeof(double) * nd);
    h->lam = (double *)dalloc(h, sizeof(double) * nd);
    h->lacc = (double *)dalloc(h, sizeof(double) * nd);
    h->r64 = (double *)dalloc(h, sizeof(double) * nd);
    h->Hx = (double *)dalloc(h, sizeof(double) * nd);
    h->hp64 = (double *)dalloc(h, sizeof(double) * std::max<int64_t>(tb.n_slots, 1) * d);
    h->a64 = (double *)dalloc(h, sizeof(double) * ne_int);
    h->vd = dalloc(h, vbytes * nd);
    h->vr = dalloc(h, vbytes * nd);
    h->vp = dalloc(h, vbytes * nd);
    h->vAp = dalloc(h, vbytes * nd);
    if (is_mixed(h)) {
        h->u32 = (float *)dalloc(h, sizeof(float) * nd);
        h->hp32 = (float *)dalloc(h, sizeof(float) * std::max<int64_t>(tb.n_slots, 1) * d);
        if (d == 3) {
            h->u4 = (float *)dalloc(h, sizeof(float) * 4 * nv);
            if (!h->u4) return fail(h, SIM_ENOMEM, "device allocation failed");
        }
    }
    if (!c.partials || !h->sc || !h->u || !h->uhat || !h->g || !h->work || !h->lam || !h->lacc || !h->r64 || !h->Hx || !h->hp64 || !h->a64 || !h->vd ||
        !h->vr || !h->vp || !h->vAp || (is_mixed(h) && (!h->u32 || !h->hp32)))
        return fail(h, SIM_ENOMEM, "device allocation failed");
    CK(h, cudaMemset(h->sc, 0, sizeof(DevScalars)));
    CK(h, cudaMemset(h->u, 0, sizeof(double) * nd));
    CK(h, cudaMemset(h->uhat, 0, sizeof(double) * nd));
    if (h->mat.dt > 0.0 && h->mat.k_friction > 0.0) {
        h->fw = (double *)dalloc(h, sizeof(double) * nv);
        h->u0 = (double *)dalloc(h, sizeof(double) * nd);
        if (!h->fw || !h->u0) return fail(h, SIM_ENOMEM, "device allocation failed");
        CK(h, cudaMemset(h->fw, 0, sizeof(double) * nv));
        CK(h, cudaMemset(h->u0, 0, sizeof(double) * nd));
    }
    CK(h, cudaMemset(h->vp, 0, vbytes * nd));
    if (h->u32) CK(h, cudaMemset(h->u32, 0, sizeof(float) * nd));
    CK(h, cudaMallocHost((void **)&h->sc_host, sizeof(DevScalars)));
    CK(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    CK(h, cudaEventCreate(&h->ev0));
    CK(h, cudaEventCreate(&h->ev1));
    CK(h, configure_elem_kernels());
    const size_t sm_need = is_mixed(h) ? hvp_smem<float>(c) : hvp_smem<double>(c);
    const size_t sm_grad = (size_t)td.max_tv * d * sizeof(double) + (size_t)td.max_te * td.rs * sizeof(double);
    if (std::max(sm_need, sm_grad) > 200 * 1024) return fail(h, SIM_EINVAL, "tile too large for shared memory");
    CK(h, cudaDeviceSynchronize());
    return SIM_OK;
}

extern "C" int sim_create(const sim_mesh *mesh, const sim_material *mat, const sim_options *opt, sim_handle **out)
{
    if (out) *out = nullptr;
    if (!mesh || !mat || !out) return fail(nullptr, SIM_EINVAL, "null argument");
    if (mesh->dim != 2 && mesh->dim != 3) return fail(nullptr, SIM_EINVAL, "dim must be 2 or 3");
    if (mesh->n_vert <= 0 || mesh->n_elem <= 0 || !mesh->rest_pos || !mesh->elems)
        return fail(nullptr, SIM_EINVAL, "empty mesh");
    if (mesh->n_vert > (int64_t)1 << 30 || mesh->n_elem > (int64_t)1 << 30)
        return fail(nullptr, SIM_EINVAL, "mesh too large for 32-bit indices");
    if (mat->contact_power != 2 && mat->contact_power != 3)
        return fail(nullptr, SIM_EINVAL, "contact_power must be 2 or 3");
    if (mat->log_mode != SIM_LOG_EXACT && mat->log_mode != SIM_LOG_QUAD)
        return fail(nullptr, SIM_EINVAL, "log_mode must be SIM_LOG_EXACT or SIM_LOG_QUAD");
    if (mat->muscle_model != SIM_MUSCLE_CONTRACTILE && mat->muscle_model != SIM_MUSCLE_SPRING)
        return fail(nullptr, SIM_EINVAL, "muscle_model must be SIM_MUSCLE_CONTRACTILE or SIM_MUSCLE_SPRING");
    if (!(mat->dt >= 0.0) || !std::isfinite(mat->mu) || !std::isfinite(mat->lambda) || !std::isfinite(mat->k_muscle) ||
        !std::isfinite(mat->density) || !std::isfinite(mat->gravity) || !std::isfinite(mat->k_contact))
        return fail(nullptr, SIM_EINVAL, "bad material scalar");
    if (!(mat->k_friction >= 0.0) || !std::isfinite(mat->k_friction) || !std::isfinite(mat->eps_friction))
        return fail(nullptr, SIM_EINVAL, "k_friction must be finite and >= 0, eps_friction finite");
    if (opt && opt->precision != SIM_PREC_FP64 && opt->precision != SIM_PREC_MIXED)
        return fail(nullptr, SIM_EINVAL, "precision must be SIM_PREC_FP64 or SIM_PREC_MIXED");
    if (opt && opt->cg_kernel != SIM_CG_AUTO && opt->cg_kernel != SIM_CG_ITERATION)
        return fail(nullptr, SIM_EINVAL, "cg_kernel must be SIM_CG_AUTO or SIM_CG_ITERATION");
    sim_handle *h = new sim_handle();
    const int rc = create_impl(h, mesh, mat, opt);
    if (rc != SIM_OK) {
        g_create_error = h->err;
        sim_destroy(h);
        return rc;
    }
    *out = h;
    return SIM_OK;
}

// ---------------------------------------------------------------- typed views

template <typename T>
struct View;
template <>
struct View<float> {
    static float *u(sim_handle *h) { return h->u32; }
    // the displacement as the CG tile kernel reads it (refresh_cg_u first)
    static const float *ucg(sim_handle *h) { return h->u4 ? h->u4 : h->u32; }
    static float *hp(sim_handle *h) { return h->hp32; }
};
template <>
struct View<double> {
    static double *u(sim_handle *h) { return h->u; }
    static const double *ucg(sim_handle *h) { return h->u; }
    static double *hp(sim_handle *h) { return h->hp64; }
};

// Set the internal activation copies from the caller's array.
static int set_activation(sim_handle *h, const double *a, cudaStream_t s)
{
    const Ctx &c = h->ctx;
    const int slot = hvp_fields(c.dim, c.muscle == SIM_MUSCLE_SPRING);  // after the HVP fields
    launch_gather_elem<double>(c, a, h->a64, s);
    launch_gather_elem<double>(c, a, c.rec64 + slot, s, c.td.rs);
    if (is_mixed(h)) launch_gather_elem<float>(c, a, c.rec32 + slot, s, c.td.rs);
    CKL(h);
    return SIM_OK;
}

// Set the internal displacement from positions; pin = clamp pinned vertices to rest.
static int set_state(sim_handle *h, const double *x, bool pin, cudaStream_t s)
{
    launch_x_to_u(h->ctx, x, h->u, h->u32, pin ? h->fixed : nullptr, s);
    CKL(h);
    return SIM_OK;
}

// ---------------------------------------------------------------- CG

// Copies the FP32 displacement into the padded rows the 3D CG tile kernel
// gathers (one 16-byte load per vertex); the displacement is constant during
// a CG solve.
static void refresh_cg_u(sim_handle *h, cudaStream_t s)
{
    if (h->u4) launch_pad_rows4(h->ctx, h->u32, h->u4, s);
}

template <typename T>
static void enqueue_cg_block(sim_handle *h, const Phys &ph, cudaStream_t s, int n_iter = kCgBlock, bool pdl = true)
{
    T *d = (T *)h->vd, *r = (T *)h->vr, *p = (T *)h->vp, *Ap = (T *)h->vAp;
    h->ctx.pdl = pdl;  // programmatic edges between the kernels of the captured block
    for (int k = 0; k < n_iter; ++k) {
        // the timing events bracket the HVP tile kernel alone
        if (h->timing) cudaEventRecordWithFlags(h->tev[2 * k], s, cudaEventRecordExternal);
        launch_hvp_cg<T>(h->ctx, ph, View<T>::ucg(h), p, Ap, View<T>::hp(h), s);
        if (h->timing) cudaEventRecordWithFlags(h->tev[2 * k + 1], s, cudaEventRecordExternal);
        launch_cg_alpha<T>(h->ctx, h->ctx.td.n_tiles, s);
        launch_cg_update_halo<T>(h->ctx, ph, View<T>::u(h), d, r, p, Ap, View<T>::hp(h), s);
        launch_cg_dir<T>(h->ctx, p, r, s);
    }
    h->ctx.pdl = false;
}

template <typename T>
static int get_cg_graph(sim_handle *h, const Phys &ph, cudaGraphExec_t *exec)
{
    Graph &gr = h->cg_graph[ph.dyn ? 1 : 0][h->timing ? 1 : 0];
    if (!gr.valid) {
        cudaGraph_t graph = nullptr;
        CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        enqueue_cg_block<T>(h, ph, h->cap);
        cudaError_t e1 = cudaGetLastError();
        cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(h, SIM_ECUDA, std::string("CG graph capture failed: ") +
                                          cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
        }
        cudaError_t e3 = cudaGraphInstantiate(&gr.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) return fail(h, SIM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
        gr.valid = true;
    }
    *exec = gr.exec;
    return SIM_OK;
}

// Builds the device-side CG loop: graph = WHILE(cond) { kCgBody iterations;
// k_cg_cond }, the condition starting at 1 on every launch.
template <typename T>
static cudaError_t build_cg_while(sim_handle *h, const Phys &ph, bool pdl, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle hnd = 0;
    cudaGraphNode_t node = nullptr;
    cudaGraphNodeParams np = {};
    e = cudaGraphConditionalHandleCreate(&hnd, g, 1u, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = hnd;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue_cg_block<T>(h, ph, h->cap, kCgBody, pdl);
            launch_cg_cond(h->ctx, hnd, h->cap);
            const cudaError_t e1 = cudaGetLastError();
            cudaGraph_t cap_out = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(h->cap, &cap_out);
            e = e1 != cudaSuccess ? e1 : e2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

// The device-side CG loop of this handle (PDL edges inside the body if the
// CUDA build accepts them), or null if conditional nodes are refused.
template <typename T>
static cudaGraphExec_t get_cg_while(sim_handle *h, const Phys &ph)
{
    WhileGraph &wg = h->cg_while[ph.dyn ? 1 : 0];
    if (wg.state == 0) {
        cudaError_t e = build_cg_while<T>(h, ph, true, &wg.exec);
        if (e != cudaSuccess) e = build_cg_while<T>(h, ph, false, &wg.exec);
        wg.state = e == cudaSuccess ? 1 : -1;
        if (e != cudaSuccess) {
            wg.exec = nullptr;
            if (h->verbose)
                fprintf(stderr, "[softsim] device-side CG loop unavailable (%s); host-driven blocks\n",
                        cudaGetErrorString(e));
        }
    }
    return wg.state == 1 ? wg.exec : nullptr;
}

// Rounds of the device-side loop that cover max_iter iterations, plus slack.
static int cg_max_rounds(int max_iter) { return max_iter / kCgBody + 2; }

// Runs CG until the device raises `done`: one launch of the device-side loop
// (a single host synchronisation), or, with in-solve kernel timing on or
// without conditional graph nodes, replays of a kCgBlock-iteration graph with
// a host check between replays.  Returns the iteration count through
// sc_host->iter.
template <typename T>
static int run_cg(sim_handle *h, const Phys &ph, int max_iter, cudaStream_t s)
{
    int rc;
    if (!h->timing && h->opt.cg_kernel == SIM_CG_AUTO && cg_coop_fits<T>(h->ctx)) {
        CK(h, launch_cg_coop<T>(h->ctx, ph, View<T>::u(h), (T *)h->vd, (T *)h->vr, (T *)h->vp, (T *)h->vAp,
                                View<T>::hp(h), s));
        return read_scalars(h, s);
    }
    refresh_cg_u(h, s);
    if (!h->timing) {
        cudaGraphExec_t wexec = get_cg_while<T>(h, ph);
        if (wexec) {
            CK(h, cudaGraphLaunch(wexec, s));
            if ((rc = read_scalars(h, s))) return rc;
            h->ctx.n_launch += (int64_t)h->sc_host->cg_rounds * (5 * kCgBody + 1);
            if (!h->sc_host->done) return fail(h, SIM_ECUDA, "CG control did not terminate");
            return SIM_OK;
        }
    }
    cudaGraphExec_t exec;
    rc = get_cg_graph<T>(h, ph, &exec);
    if (rc) return rc;
    if ((rc = read_scalars(h, s))) return rc;
    const int max_blocks = max_iter / kCgBlock + 2;
    for (int b = 0; b < max_blocks && !h->sc_host->done; ++b) {
        const int it0 = h->sc_host->iter;
        const int neg0 = h->sc_host->negcurv;
        CK(h, cudaGraphLaunch(exec, s));
        h->ctx.n_launch += 5 * kCgBlock;
        if ((rc = read_scalars(h, s))) return rc;
        if (h->timing) {
            // tile launches that did work in this replay (later ones exit at once)
            int active = h->sc_host->iter - it0 + ((h->sc_host->negcurv && !neg0) ? 1 : 0);
            active = std::min(active, kCgBlock);
            for (int k = 0; k < active; ++k) {
                float ms = 0.f;
                CK(h, cudaEventElapsedTime(&ms, h->tev[2 * k], h->tev[2 * k + 1]));
                h->t_hvp_ms += ms;
            }
            h->n_hvp_timed += active;
        }
    }
    if (!h->sc_host->done) return fail(h, SIM_ECUDA, "CG control did not terminate");
    return SIM_OK;
}

// ---------------------------------------------------------------- Newton

template <typename T>
static int newton_impl(sim_handle *h, bool dyn, sim_solve_stats *st, cudaStream_t s)
{
    const Phys ph = make_phys(h, dyn);
    Ctx &c = h->ctx;
    sim_solve_stats S;
    memset(&S, 0, sizeof(S));
    S.status = SIM_ENOTCONVERGED;
    int rc;
    const double *uh = dyn ? h->uhat : nullptr;
    const double t0 = 0.0;
    launch_grad(c, ph, h->u, uh, h->a64, h->g, h->hp64, s);
    launch_energy(c, ph, h->u, nullptr, uh, h->a64, &t0, 1, s);
    CKL(h);
    if ((rc = read_scalars(h, s))) return rc;
    double gn = std::sqrt(h->sc_host->gn2);
    const double g0 = gn;
    double E = h->sc_host->E[0], Sabs = h->sc_host->S[0];
    S.res0 = g0;
    if (!std::isfinite(E) || !std::isfinite(gn)) {
        S.status = std::isinf(E) ? SIM_EINVERTED : SIM_ENAN;
        S.res_final = gn;
        S.min_J = h->sc_host->minJ;
        if (st) *st = S;
        return S.status;
    }
    const double eps = 2.220446049250313e-16;
    int it = 0;
    for (;; ++it) {
        if (gn <= h->opt.newton_rtol * g0) {
            S.status = SIM_OK;
            break;
        }
        if (it >= h->opt.max_newton) break;
        const double eta = std::min(h->opt.newton_forcing, std::sqrt(gn / g0));
        launch_cg_init<T>(c, h->g, -1.0, (T *)h->vd, (T *)h->vr, (T *)h->vp, eta, h->opt.max_cg,
                          cg_max_rounds(h->opt.max_cg), s);
        CKL(h);
        if ((rc = run_cg<T>(h, ph, h->opt.max_cg, s))) return rc;
        S.cg_iters_total += h->sc_host->iter;
        launch_dir_check<T>(c, h->g, (T *)h->vd, s);
        CKL(h);
        // line search: t = 1, then batches of halvings
        bool ok = false;
        double t_acc = 0.0, E_acc = 0.0, S_acc = 0.0;
        int j0 = 0;
        const double *dir64 = nullptr;
        if (is_mixed(h)) {
            launch_convert<float, double>(c.nv * c.dim, (const float *)h->vd, h->work, s);
            c.n_launch += 1;
            dir64 = h->work;
        } else {
            dir64 = (const double *)h->vd;
        }
        while (j0 < h->opt.max_ls && !ok) {
            const int nt = j0 == 0 ? 1 : std::min(kMaxTrials, h->opt.max_ls - j0);
            double ts[kMaxTrials];
            for (int j = 0; j < nt; ++j) ts[j] = std::ldexp(1.0, -(j0 + j));
            launch_energy(c, ph, h->u, dir64, uh, h->a64, ts, nt, s);
            CKL(h);
            if ((rc = read_scalars(h, s))) return rc;
            const double gd = h->sc_host->gd;
            for (int j = 0; j < nt; ++j) {
                const double Et = h->sc_host->E[j], St = h->sc_host->S[j];
                const double slack = 64.0 * eps * std::max(Sabs, St);
                if (std::isfinite(Et) && Et <= E + 1e-4 * ts[j] * gd + slack) {
                    ok = true;
                    t_acc = ts[j];
                    E_acc = Et;
                    S_acc = St;
                    S.ls_halvings += j0 + j;
                    break;
                }
            }
            if (!ok) j0 += nt;
        }
        if (!ok) {
            if (h->verbose) fprintf(stderr, "[softsim] newton %d: line search failed, |g|/|g0| %.3e\n", it, gn / g0);
            S.ls_halvings += h->opt.max_ls;
            S.status = SIM_ELINESEARCH;
            break;
        }
        if (h->verbose)
            fprintf(stderr, "[softsim] newton %d: |g|/|g0| %.3e, eta %.2e, cg %d%s, t %.3g, E %.10e\n", it, gn / g0, eta,
                    h->sc_host->iter, h->sc_host->dir_fix ? " (steepest descent)" : "", t_acc, E_acc);
        launch_step_update<T>(c, h->u, (const T *)h->vd, t_acc, h->u32, s);
        E = E_acc;
        Sabs = S_acc;
        launch_grad(c, ph, h->u, uh, h->a64, h->g, h->hp64, s);
        CKL(h);
        if ((rc = read_scalars(h, s))) return rc;
        gn = std::sqrt(h->sc_host->gn2);
        if (!std::isfinite(gn)) {
            S.status = SIM_ENAN;
            break;
        }
    }
    S.newton_iters = it;
    S.res_final = gn;
    launch_energy(c, ph, h->u, nullptr, uh, h->a64, &t0, 1, s);
    CKL(h);
    if ((rc = read_scalars(h, s))) return rc;
    S.min_J = h->sc_host->minJ;
    if (st) *st = S;
    return S.status;
}

// ---------------------------------------------------------------- adjoint

// lambda = A^-1 b on free entries, A at the current internal state, by CG
// with iterative refinement: each pass runs CG (in the HVP precision) on the
// current FP64 residual, adds the correction to an FP64 accumulator, and
// recomputes the exact residual b - A lambda with the FP64 HVP.  The solve
// stops when that FP64 residual meets adjoint_rtol, so the mixed-precision
// path reaches the same accuracy as the FP64 one.
template <typename T>
static int adjoint_impl(sim_handle *h, bool dyn, const double *b, double *lambda, sim_solve_stats *st,
                        cudaStream_t s)
{
    const Phys ph = make_phys(h, dyn);
    Ctx &c = h->ctx;
    int rc;
    const int64_t nd = c.nv * c.dim;
    launch_mask_copy(c, b, h->work, s);
    CK(h, cudaMemsetAsync(h->lacc, 0, sizeof(double) * nd, s));
    launch_residual(c, h->work, nullptr, h->r64, s);
    CKL(h);
    if ((rc = read_scalars(h, s))) return rc;
    const double bn = std::sqrt(h->sc_host->gn2);
    sim_solve_stats S;
    memset(&S, 0, sizeof(S));
    S.res0 = bn;
    S.min_J = NAN;
    S.status = SIM_ENOTCONVERGED;
    if (!std::isfinite(bn)) {  // non-finite right-hand side: nothing to solve
        S.status = SIM_ENAN;
        S.res_final = bn;
        CK(h, cudaMemcpyAsync(lambda, h->lacc, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s));
        if (st) *st = S;
        return S.status;
    }
    double rn = bn;
    const double target = h->opt.adjoint_rtol * bn;
    const double inner = is_mixed(h) ? std::max(h->opt.adjoint_rtol, 1e-4) : h->opt.adjoint_rtol;
    int budget = h->opt.max_adjoint_cg;
    for (int pass = 0; pass < 12; ++pass) {
        if (rn <= target || !(rn > 0.0)) {
            S.status = SIM_OK;
            break;
        }
        if (budget <= 0) break;
        launch_cg_init<T>(c, h->r64, 1.0, (T *)h->vd, (T *)h->vr, (T *)h->vp, std::max(inner, 0.5 * target / rn),
                          budget, cg_max_rounds(budget), s);
        CKL(h);
        if ((rc = run_cg<T>(h, ph, budget, s))) return rc;
        const int it = h->sc_host->iter;
        const bool neg = h->sc_host->negcurv != 0;
        S.cg_iters_total += it;
        budget -= std::max(it, 1);
        launch_accumulate<T>(c, h->lacc, (const T *)h->vd, s);
        launch_hvp<double>(c, ph, h->u, h->lacc, h->Hx, h->hp64, s);
        launch_residual(c, h->work, h->Hx, h->r64, s);
        CKL(h);
        if ((rc = read_scalars(h, s))) return rc;
        const double rn_new = std::sqrt(h->sc_host->gn2);
        if (h->verbose)
            fprintf(stderr, "[softsim] adjoint pass %d: cg %d, |r|/|b| %.3e -> %.3e%s\n", pass, it, rn / bn,
                    rn_new / bn, neg ? " (non-positive curvature)" : "");
        if (!std::isfinite(rn_new)) {
            S.status = SIM_ENAN;
            rn = rn_new;
            break;
        }
        if (neg || rn_new >= rn) {  // no progress: the operator is not positive definite here
            rn = rn_new;
            S.status = rn <= target ? SIM_OK : SIM_ENOTCONVERGED;
            break;
        }
        rn = rn_new;
    }
    if (rn <= target) S.status = SIM_OK;
    S.res_final = rn;
    CK(h, cudaMemcpyAsync(lambda, h->lacc, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s));
    if (st) *st = S;
    return S.status;
}

// ---------------------------------------------------------------- API

#define CHECK_H(h) \
    if (!(h)) return SIM_EINVAL

extern "C" int sim_energy_grad(sim_handle *h, const double *x, const double *a, double *E_dev, double *grad,
                               void *stream)
{
    CHECK_H(h);
    if (!x || !a) return fail(h, SIM_EINVAL, "null x or a");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = set_state(h, x, false, s))) return rc;
    if ((rc = set_activation(h, a, s))) return rc;
    const Phys ph = make_phys(h, false);
    if (grad) launch_grad(h->ctx, ph, h->u, nullptr, h->a64, grad, h->hp64, s);
    if (E_dev) {
        const double t0 = 0.0;
        launch_energy(h->ctx, ph, h->u, nullptr, nullptr, h->a64, &t0, 1, s);
        CK(h, cudaMemcpyAsync(E_dev, &h->sc->E[0], sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CKL(h);
    return SIM_OK;
}

extern "C" int sim_hvp(sim_handle *h, const double *x, const double *a, const void *v, void *Hv, void *stream)
{
    CHECK_H(h);
    if (!x || !a || !v || !Hv) return fail(h, SIM_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = set_state(h, x, false, s))) return rc;
    if ((rc = set_activation(h, a, s))) return rc;
    const Phys ph = make_phys(h, false);
    if (is_mixed(h))
        launch_hvp<float>(h->ctx, ph, h->u32, (const float *)v, (float *)Hv, h->hp32, s);
    else
        launch_hvp<double>(h->ctx, ph, h->u, (const double *)v, (double *)Hv, h->hp64, s);
    CKL(h);
    return SIM_OK;
}

template <typename T>
static int hvp_dot_impl(sim_handle *h, const void *v, void *Hv, double *vHv, cudaStream_t s)
{
    Ctx &c = h->ctx;
    const Phys ph = make_phys(h, false);
    const int64_t nd = c.nv * c.dim;
    T *p = (T *)h->vp, *Ap = (T *)h->vAp;
    CK(h, cudaMemcpyAsync(p, v, sizeof(T) * nd, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemsetAsync(&h->sc->done, 0, sizeof(int), s));  // the CG tile kernel skips its work once CG is done
    refresh_cg_u(h, s);
    launch_hvp_cg<T>(c, ph, View<T>::ucg(h), p, Ap, View<T>::hp(h), s);
    launch_hvp_finalize_only<T>(c, ph, View<T>::u(h), p, Ap, View<T>::hp(h), s);
    launch_tile_dot<T>(c, &h->sc->pAp, s);
    CKL(h);
    CK(h, cudaMemcpyAsync(Hv, Ap, sizeof(T) * nd, cudaMemcpyDeviceToDevice, s));
    int rc = read_scalars(h, s);
    if (rc) return rc;
    *vHv = h->sc_host->pAp;
    return SIM_OK;
}

extern "C" int sim_hvp_dot(sim_handle *h, const double *x, const double *a, const void *v, void *Hv, double *vHv,
                           void *stream)
{
    CHECK_H(h);
    if (!x || !a || !v || !Hv || !vHv) return fail(h, SIM_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = set_state(h, x, false, s))) return rc;
    if ((rc = set_activation(h, a, s))) return rc;
    return is_mixed(h) ? hvp_dot_impl<float>(h, v, Hv, vHv, s) : hvp_dot_impl<double>(h, v, Hv, vHv, s);
}

extern "C" int sim_newton_solve(sim_handle *h, const double *x_init, const double *a, const double *x0,
                                const double *v0, double *x_out, sim_solve_stats *st, void *stream)
{
    CHECK_H(h);
    const bool dyn = h->mat.dt > 0.0;
    if (!a || !x_out) return fail(h, SIM_EINVAL, "null a or x_out");
    if (dyn && (!x0 || !v0)) return fail(h, SIM_EINVAL, "backward Euler needs x0 and v0");
    if (!dyn && (x0 || v0)) return fail(h, SIM_EINVAL, "x0/v0 given but dt == 0");
    if (!x_init) x_init = x0;
    if (!x_init) return fail(h, SIM_EINVAL, "null x_init");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = set_activation(h, a, s))) return rc;
    if (dyn) launch_uhat(h->ctx, x0, v0, h->mat.dt, h->uhat, s);
    if (dyn && h->fw) launch_friction_prep(h->ctx, x0, h->mat.k_friction, h->mat.eps_friction, h->u0, h->fw, s);
    if ((rc = set_state(h, x_init, true, s))) return rc;
    const int status = is_mixed(h) ? newton_impl<float>(h, dyn, st, s) : newton_impl<double>(h, dyn, st, s);
    if (status == SIM_ECUDA) return status;
    launch_u_to_x(h->ctx, h->u, x_out, s);
    CKL(h);
    CK(h, cudaStreamSynchronize(s));
    if (status != SIM_OK) fail(h, status, "Newton solve did not converge (status " + std::to_string(status) + ")");
    return status;
}

extern "C" int sim_adjoint_solve(sim_handle *h, const double *x_star, const double *a, const double *dLdx,
                                 double *lambda, sim_solve_stats *st, void *stream)
{
    CHECK_H(h);
    if (!x_star || !a || !dLdx || !lambda) return fail(h, SIM_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = set_state(h, x_star, false, s))) return rc;
    if ((rc = set_activation(h, a, s))) return rc;
    const bool dyn = h->mat.dt > 0.0;
    const int status = is_mixed(h) ? adjoint_impl<float>(h, dyn, dLdx, lambda, st, s)
                                   : adjoint_impl<double>(h, dyn, dLdx, lambda, st, s);
    if (status == SIM_ECUDA) return status;
    CK(h, cudaStreamSynchronize(s));
    if (status != SIM_OK) fail(h, status, "adjoint CG did not converge");
    return status;
}

extern "C" int sim_param_vjp(sim_handle *h, const double *x_star, const double *a, const double *lambda,
                             double *dLda, void *stream)
{
    CHECK_H(h);
    if (!x_star || !a || !lambda || !dLda) return fail(h, SIM_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = set_state(h, x_star, false, s))) return rc;
    if ((rc = set_activation(h, a, s))) return rc;
    const Phys ph = make_phys(h, h->mat.dt > 0.0);
    launch_param_vjp(h->ctx, ph, h->u, h->a64, lambda, dLda, s);
    CKL(h);
    return SIM_OK;
}

extern "C" int sim_material_vjp(sim_handle *h, const double *x_star, const double *a, const double *lambda,
                                double *dLdmu, double *dLdlambda, double *dLdk, void *stream)
{
    CHECK_H(h);
    if (!x_star || !a || !lambda) return fail(h, SIM_EINVAL, "null argument");
    if (!dLdmu && !dLdlambda && !dLdk) return SIM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = set_state(h, x_star, false, s))) return rc;
    if ((rc = set_activation(h, a, s))) return rc;
    const Phys ph = make_phys(h, h->mat.dt > 0.0);
    launch_material_vjp(h->ctx, ph, h->u, h->a64, lambda, dLdmu, dLdlambda, dLdk, s);
    CKL(h);
    return SIM_OK;
}

extern "C" int sim_step_forward(sim_handle *h, const double *x0, const double *v0, const double *a, double *x1,
                                double *v1, sim_solve_stats *st, void *stream)
{
    CHECK_H(h);
    if (!(h->mat.dt > 0.0)) return fail(h, SIM_EINVAL, "sim_step_forward needs dt > 0");
    if (!x0 || !v0 || !a || !x1 || !v1) return fail(h, SIM_EINVAL, "null argument");
    const int rc = sim_newton_solve(h, x0, a, x0, v0, x1, st, stream);
    if (rc != SIM_OK) return rc;
    launch_velocity(h->nv * h->dim, x1, x0, h->mat.dt, v1, (cudaStream_t)stream);
    h->ctx.n_launch += 1;
    CKL(h);
    return SIM_OK;
}

extern "C" int sim_step_backward(sim_handle *h, const double *x0, const double *v0, const double *x1, const double *a,
                                 const double *xbar1, const double *vbar1, double *xbar0, double *vbar0, double *abar,
                                 sim_solve_stats *st, void *stream)
{
    CHECK_H(h);
    (void)v0;  // the backward needs the converged state x1, and x0 only for friction
    if (!(h->mat.dt > 0.0)) return fail(h, SIM_EINVAL, "sim_step_backward needs dt > 0");
    if (!x1 || !a || !xbar1 || !vbar1 || !xbar0 || !vbar0 || !abar) return fail(h, SIM_EINVAL, "null argument");
    if (h->fw && !x0) return fail(h, SIM_EINVAL, "friction needs x0 in the step backward");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->fw) launch_friction_prep(h->ctx, x0, h->mat.k_friction, h->mat.eps_friction, h->u0, h->fw, s);
    const double dt = h->mat.dt;
    const int64_t nd = h->nv * h->dim;
    // b = xbar1 + vbar1/dt lives in h->lam until the adjoint overwrites it
    launch_axpy_out(nd, xbar1, vbar1, 1.0 / dt, h->lam, s);
    h->ctx.n_launch += 1;
    CKL(h);
    int rc = sim_adjoint_solve(h, x1, a, h->lam, h->lam, st, stream);
    if (rc != SIM_OK) return rc;
    launch_step_bwd_combine(h->ctx, h->lam, vbar1, dt, h->fw, h->mat.k_friction, x0, x1, xbar0, vbar0, s);
    CKL(h);
    return sim_param_vjp(h, x1, a, h->lam, abar, stream);
}

static int ensure_rollout_buffers(sim_handle *h)
{
    if (h->rx[0]) return SIM_OK;
    const size_t b = sizeof(double) * h->nv * h->dim;
    for (int k = 0; k < 2; ++k) {
        h->rx[k] = (double *)dalloc(h, b);
        h->rv[k] = (double *)dalloc(h, b);
        if (!h->rx[k] || !h->rv[k]) return fail(h, SIM_ENOMEM, "device allocation failed");
    }
    return SIM_OK;
}

static void accumulate(sim_solve_stats *acc, const sim_solve_stats &s)
{
    acc->newton_iters += s.newton_iters;
    acc->cg_iters_total += s.cg_iters_total;
    acc->ls_halvings += s.ls_halvings;
    acc->res0 = std::max(acc->res0, s.res0);
    acc->res_final = std::max(acc->res_final, s.res_final);
    acc->min_J = std::isnan(acc->min_J) ? s.min_J : std::min(acc->min_J, s.min_J);
    if (s.status != SIM_OK) acc->status = s.status;
}

extern "C" int sim_rollout(sim_handle *h, int n_steps, const double *x0, const double *v0, const double *a_seq,
                           int ckpt_every, double *ckpt_x, double *ckpt_v, double *xT, double *vT,
                           sim_solve_stats *st, void *stream)
{
    CHECK_H(h);
    if (n_steps < 0 || ckpt_every <= 0 || !x0 || !v0 || (n_steps > 0 && !a_seq) || !xT || !vT)
        return fail(h, SIM_EINVAL, "bad rollout arguments");
    if (n_steps > 0 && (!ckpt_x || !ckpt_v)) return fail(h, SIM_EINVAL, "null checkpoint buffers");
    int rc;
    if ((rc = ensure_rollout_buffers(h))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nd = h->nv * h->dim;
    const size_t bytes = sizeof(double) * nd;
    sim_solve_stats acc;
    memset(&acc, 0, sizeof(acc));
    acc.min_J = NAN;
    CK(h, cudaMemcpyAsync(h->rx[0], x0, bytes, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(h->rv[0], v0, bytes, cudaMemcpyDeviceToDevice, s));
    int cur = 0;
    for (int t = 0; t < n_steps; ++t) {
        if (t % ckpt_every == 0) {
            const int k = t / ckpt_every;
            CK(h, cudaMemcpyAsync(ckpt_x + (size_t)k * nd, h->rx[cur], bytes, cudaMemcpyDeviceToDevice, s));
            CK(h, cudaMemcpyAsync(ckpt_v + (size_t)k * nd, h->rv[cur], bytes, cudaMemcpyDeviceToDevice, s));
        }
        sim_solve_stats ss;
        rc = sim_step_forward(h, h->rx[cur], h->rv[cur], a_seq + (size_t)t * h->ne, h->rx[1 - cur], h->rv[1 - cur], &ss,
                              stream);
        accumulate(&acc, ss);
        if (rc != SIM_OK) {
            if (st) *st = acc;
            return rc;
        }
        cur = 1 - cur;
    }
    CK(h, cudaMemcpyAsync(xT, h->rx[cur], bytes, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(vT, h->rv[cur], bytes, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaStreamSynchronize(s));
    if (st) *st = acc;
    return SIM_OK;
}

extern "C" int sim_rollout_backward(sim_handle *h, int n_steps, const double *a_seq, int ckpt_every,
                                    const double *ckpt_x, const double *ckpt_v, const double *xbarT,
                                    const double *vbarT, double *xbar0, double *vbar0, double *abar_seq,
                                    double *seg_x, double *seg_v, sim_solve_stats *st, void *stream)
{
    CHECK_H(h);
    if (n_steps < 0 || ckpt_every <= 0 || !xbarT || !vbarT || !xbar0 || !vbar0)
        return fail(h, SIM_EINVAL, "bad rollout arguments");
    if (n_steps > 0 && (!a_seq || !ckpt_x || !ckpt_v || !abar_seq || !seg_x || !seg_v))
        return fail(h, SIM_EINVAL, "null rollout buffers");
    int rc;
    if ((rc = ensure_rollout_buffers(h))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nd = h->nv * h->dim;
    const size_t bytes = sizeof(double) * nd;
    sim_solve_stats acc;
    memset(&acc, 0, sizeof(acc));
    acc.min_J = NAN;
    // running adjoints live in rx/rv ping-pong buffers
    CK(h, cudaMemcpyAsync(h->rx[0], xbarT, bytes, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(h->rv[0], vbarT, bytes, cudaMemcpyDeviceToDevice, s));
    int cur = 0;
    const int n_ckpt = (n_steps + ckpt_every - 1) / ckpt_every;
    for (int k = n_ckpt - 1; k >= 0; --k) {
        const int t0 = k * ckpt_every, t1 = std::min(n_steps, t0 + ckpt_every);
        CK(h, cudaMemcpyAsync(seg_x, ckpt_x + (size_t)k * nd, bytes, cudaMemcpyDeviceToDevice, s));
        CK(h, cudaMemcpyAsync(seg_v, ckpt_v + (size_t)k * nd, bytes, cudaMemcpyDeviceToDevice, s));
        for (int t = t0; t < t1; ++t) {  // recompute the segment's states
            sim_solve_stats ss;
            const int j = t - t0;
            rc = sim_step_forward(h, seg_x + (size_t)j * nd, seg_v + (size_t)j * nd, a_seq + (size_t)t * h->ne,
                                  seg_x + (size_t)(j + 1) * nd, seg_v + (size_t)(j + 1) * nd, &ss, stream);
            accumulate(&acc, ss);
            if (rc != SIM_OK) {
                if (st) *st = acc;
                return rc;
            }
        }
        for (int t = t1 - 1; t >= t0; --t) {
            sim_solve_stats ss;
            const int j = t - t0;
            rc = sim_step_backward(h, seg_x + (size_t)j * nd, seg_v + (size_t)j * nd, seg_x + (size_t)(j + 1) * nd,
                                   a_seq + (size_t)t * h->ne, h->rx[cur], h->rv[cur], h->rx[1 - cur], h->rv[1 - cur],
                                   abar_seq + (size_t)t * h->ne, &ss, stream);
            accumulate(&acc, ss);
            if (rc != SIM_OK) {
                if (st) *st = acc;
                return rc;
            }
            cur = 1 - cur;
        }
    }
    CK(h, cudaMemcpyAsync(xbar0, h->rx[cur], bytes, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(vbar0, h->rv[cur], bytes, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaStreamSynchronize(s));
    if (st) *st = acc;
    return SIM_OK;
}

extern "C" int sim_set_kernel_timing(sim_handle *h, int on)
{
    CHECK_H(h);
    if (on && !h->tev[0])
        for (auto &e : h->tev) CK(h, cudaEventCreate(&e));
    h->timing = on ? 1 : 0;
    h->t_hvp_ms = 0.0;
    h->n_hvp_timed = 0;
    return SIM_OK;
}

extern "C" int sim_kernel_timing(const sim_handle *h, double *hvp_tile_ms, int64_t *hvp_launches)
{
    if (!h) return SIM_EINVAL;
    if (hvp_tile_ms) *hvp_tile_ms = h->t_hvp_ms;
    if (hvp_launches) *hvp_launches = h->n_hvp_timed;
    return SIM_OK;
}

extern "C" int sim_set_wait_limit(sim_handle *h, int polls)
{
    CHECK_H(h);
    const int v = polls < 0 ? TileDev{}.wait_polls : polls;
    if (v != h->ctx.td.wait_polls) {
        CK(h, cudaDeviceSynchronize());  // no captured graph may still be running
        drop_graphs(h);                  // they hold the old limit
        h->ctx.td.wait_polls = v;
    }
    return SIM_OK;
}

extern "C" int sim_counters(const sim_handle *h, int64_t *kernel_launches)
{
    if (!h) return SIM_EINVAL;
    if (kernel_launches) *kernel_launches = h->ctx.n_launch;
    return SIM_OK;
}

extern "C" int sim_time_hvp(sim_handle *h, int n, float *ms, void *stream)
{
    CHECK_H(h);
    if (n <= 0 || !ms) return fail(h, SIM_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const Phys ph = make_phys(h, false);
    float t_tile = 0.f, t_fin = 0.f;
    CK(h, cudaStreamSynchronize(s));
    CK(h, cudaEventRecord(h->ev0, s));
    for (int i = 0; i < n; ++i) {
        if (is_mixed(h))
            launch_hvp_tile_only<float>(h->ctx, ph, h->u32, (const float *)h->vp, (float *)h->vAp, h->hp32, s);
        else
            launch_hvp_tile_only<double>(h->ctx, ph, h->u, (const double *)h->vp, (double *)h->vAp, h->hp64, s);
    }
    CK(h, cudaEventRecord(h->ev1, s));
    CKL(h);
    CK(h, cudaEventSynchronize(h->ev1));
    CK(h, cudaEventElapsedTime(&t_tile, h->ev0, h->ev1));
    CK(h, cudaEventRecord(h->ev0, s));
    for (int i = 0; i < n; ++i) {
        if (is_mixed(h))
            launch_hvp_finalize_only<float>(h->ctx, ph, h->u32, (const float *)h->vp, (float *)h->vAp, h->hp32, s);
        else
            launch_hvp_finalize_only<double>(h->ctx, ph, h->u, (const double *)h->vp, (double *)h->vAp, h->hp64, s);
    }
    CK(h, cudaEventRecord(h->ev1, s));
    CKL(h);
    CK(h, cudaEventSynchronize(h->ev1));
    CK(h, cudaEventElapsedTime(&t_fin, h->ev0, h->ev1));
    ms[0] = t_tile / n;
    ms[1] = t_fin / n;
    return SIM_OK;
}
