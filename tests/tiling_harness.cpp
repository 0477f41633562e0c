// Test harness: exposes the host tile builder (paper_2102_05791_gb300/csrc/
// tiling.cpp) through a C interface so the CPU tests can check its output.
#include <cstring>
#include <new>
#include <string>

#include "tiling.h"

using softsim::TileBuild;

extern "C" {

void *tb_build(int dim, int64_t nv, int64_t ne, const double *X, const int32_t *T, const uint8_t *fixed, int te_max,
               int tv_max, int rec_stride, char *err, int err_len)
{
    TileBuild *tb = new (std::nothrow) TileBuild();
    std::string e;
    if (!tb || !softsim::build_tiles(dim, nv, ne, X, T, fixed, te_max, tv_max, rec_stride, *tb, e)) {
        if (err && err_len > 0) {
            std::strncpy(err, e.c_str(), err_len - 1);
            err[err_len - 1] = 0;
        }
        delete tb;
        return nullptr;
    }
    return tb;
}

void tb_free(void *h) { delete static_cast<TileBuild *>(h); }

int64_t tb_scalar(void *h, int which)
{
    const TileBuild *t = static_cast<TileBuild *>(h);
    switch (which) {
    case 0: return t->n_tiles;
    case 1: return t->max_te;
    case 2: return t->max_tv;
    case 3: return t->ne_int;
    case 4: return t->n_slots;
    default: return -1;
    }
}

// which: 0 perm, 1 tile_elem, 2 tile_vert, 3 lv_gid, 4 lv_code, 5 lv_inc(u32), 6 inc(u16), 7 conn(u32),
// 8 fin_gid, 9 fin_ptr, 10 vfin
int64_t tb_len(void *h, int which)
{
    const TileBuild *t = static_cast<TileBuild *>(h);
    switch (which) {
    case 0: return t->perm.size();
    case 1: return t->tile_elem.size();
    case 2: return t->tile_vert.size();
    case 3: return t->lv_gid.size();
    case 4: return t->lv_code.size();
    case 5: return t->lv_inc.size();
    case 6: return t->inc.size();
    case 7: return t->conn.size();
    case 8: return t->fin_gid.size();
    case 9: return t->fin_ptr.size();
    case 10: return t->vfin.size();
    default: return -1;
    }
}

void tb_copy(void *h, int which, void *dst)
{
    const TileBuild *t = static_cast<TileBuild *>(h);
    switch (which) {
    case 0: std::memcpy(dst, t->perm.data(), t->perm.size() * 4); break;
    case 1: std::memcpy(dst, t->tile_elem.data(), t->tile_elem.size() * 4); break;
    case 2: std::memcpy(dst, t->tile_vert.data(), t->tile_vert.size() * 4); break;
    case 3: std::memcpy(dst, t->lv_gid.data(), t->lv_gid.size() * 4); break;
    case 4: std::memcpy(dst, t->lv_code.data(), t->lv_code.size() * 4); break;
    case 5: std::memcpy(dst, t->lv_inc.data(), t->lv_inc.size() * 4); break;
    case 6: std::memcpy(dst, t->inc.data(), t->inc.size() * 2); break;
    case 7: std::memcpy(dst, t->conn.data(), t->conn.size() * 4); break;
    case 8: std::memcpy(dst, t->fin_gid.data(), t->fin_gid.size() * 4); break;
    case 9: std::memcpy(dst, t->fin_ptr.data(), t->fin_ptr.size() * 4); break;
    case 10: std::memcpy(dst, t->vfin.data(), t->vfin.size() * 4); break;
    }
}

// The element-record layout constants shared by the builder and the kernels.
int tb_hvp_fields(int dim, int spring) { return softsim::hvp_fields(dim, spring != 0); }
int tb_rec_stride(int nf) { return softsim::rec_stride(nf); }
int tb_corner_base(int le) { return softsim::corner_base(le); }
}
