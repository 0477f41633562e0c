// Host-side construction of the tile structure used by the element kernels
// (see internal.h for the layout).  Plain C++, no CUDA.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "layout.h"

namespace softsim {

// Padding makes every per-tile range start and end on a 16-byte boundary so
// that it can be copied with one bulk (TMA) copy: element ranges are padded
// to multiples of kElemPad entries (padding elements have W = 0, zero
// connectivity and perm = -1) and local-vertex ranges to multiples of
// kVertPad (padding entries have lv_code = LV_PAD and no incidences).

struct TileBuild {
    int dim = 0;
    int64_t nv = 0, ne = 0;
    int64_t ne_int = 0;              // padded element count (tile order)
    int n_tiles = 0, max_te = 0, max_tv = 0;   // padded per-tile maxima
    int rs = 0;                      // element-record stride (words) the corner offsets assume
    int64_t n_slots = 0;
    int64_t n_real_lv = 0;           // local vertices without padding
    std::vector<int32_t> perm;       // [ne_int] tile order -> caller order, -1 for padding
    std::vector<int32_t> tile_elem;  // [n_tiles + 1] padded element offsets
    std::vector<int32_t> tile_vert;  // [n_tiles + 1] padded local-vertex offsets
    std::vector<int32_t> lv_gid, lv_code;
    std::vector<uint32_t> lv_inc;    // first incidence | count << 16 | kLvPinned
    std::vector<uint16_t> inc;       // [ne_int * (dim+1)] corner offsets le*rs + corner_base(le) + corner*dim
    std::vector<uint32_t> conn;      // [ne_int]
    std::vector<int32_t> fin_gid, fin_ptr;
    std::vector<int32_t> vfin;       // [nv] index into fin_gid, or -1 for a vertex of one tile
};

// Orders the elements along a Morton curve of their centroids (cells of the
// mean element size) and cuts the order greedily into tiles of at most
// te_max elements and at most tv_max (<= 256) distinct vertices.  `T` is
// [ne][dim+1] in caller order; rec_stride is the stride (in words) of the
// per-element records whose slots corner_base(le) + corner*dim .. + dim-1
// hold the corner forces in the kernels.  Returns false and sets err if some vertex
// belongs to no element or a single element exceeds the limits.
bool build_tiles(int dim, int64_t nv, int64_t ne, const double *X, const int32_t *T, const uint8_t *fixed,
                 int te_max, int tv_max, int rec_stride, TileBuild &out, std::string &err);

}  // namespace softsim
