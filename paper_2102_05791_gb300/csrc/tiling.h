// Host-side construction of the tile structure used by the element kernels
// (see internal.h for the layout).  Plain C++, no CUDA.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace softsim {

struct TileBuild {
    int dim = 0;
    int64_t nv = 0, ne = 0;
    int n_tiles = 0, max_te = 0, max_tv = 0;
    int64_t n_slots = 0;
    std::vector<int32_t> perm;       // tile order -> caller order
    std::vector<int32_t> tile_elem;  // [n_tiles + 1]
    std::vector<int32_t> tile_vert;  // [n_tiles + 1]
    std::vector<int32_t> lv_gid, lv_code, inc_start;
    std::vector<uint16_t> inc;
    std::vector<uint32_t> conn;
    std::vector<int32_t> fin_gid, fin_ptr;
};

// Orders the elements along a Morton curve of their centroids (cells of the
// mean element size) and cuts the order greedily into tiles of at most
// te_max elements and at most tv_max (<= 256) distinct vertices.  `T` is
// [ne][dim+1] in caller order.  Returns false and sets err if some vertex
// belongs to no element or a single element exceeds the limits.
bool build_tiles(int dim, int64_t nv, int64_t ne, const double *X, const int32_t *T, int te_max, int tv_max,
                 TileBuild &out, std::string &err);

}  // namespace softsim
