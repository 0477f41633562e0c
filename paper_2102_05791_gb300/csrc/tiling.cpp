// Tile construction for the deterministic element -> vertex reduction.
#include "tiling.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace softsim {

static uint64_t spread3(uint64_t x)
{
    x &= 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

static uint64_t spread2(uint64_t x)
{
    x &= 0xffffffffull;
    x = (x | x << 16) & 0x0000ffff0000ffffull;
    x = (x | x << 8) & 0x00ff00ff00ff00ffull;
    x = (x | x << 4) & 0x0f0f0f0f0f0f0f0full;
    x = (x | x << 2) & 0x3333333333333333ull;
    x = (x | x << 1) & 0x5555555555555555ull;
    return x;
}

// Orders each local vertex's incidence list for the vertex phase of the tile
// kernels, where lane j of a warp walks the list of local vertex 32w + j:
// at every step the lanes read corner forces from the tile's element records
// in shared memory, whose bank is the entry's word offset mod 32.  Greedily, step by
// step, each lane takes the remaining entry whose bank the other lanes of the
// step have used least (lanes with the fewest entries left choose first;
// ties go to the lower offset), so the lanes of a step mostly hit distinct
// banks.  Any fixed order gives a deterministic sum; this one is a function
// of the tile alone.  inc: the tile's incidence block; bucket[j]..bucket[j+1]
// is local vertex j's list.
static void bank_order(uint16_t *inc, const std::vector<int32_t> &bucket, int nl)
{
    std::vector<uint16_t> src;
    std::vector<char> taken;
    std::vector<int> lanes;
    for (int g0 = 0; g0 < nl; g0 += 32) {
        const int g1 = std::min(nl, g0 + 32);
        const int b0 = bucket[g0];
        src.assign(inc + b0, inc + bucket[g1]);
        taken.assign(src.size(), 0);
        int m = 0;
        for (int j = g0; j < g1; ++j) m = std::max(m, bucket[j + 1] - bucket[j]);
        for (int i = 0; i < m; ++i) {
            int used[32] = {0};
            lanes.clear();
            for (int j = g0; j < g1; ++j)
                if (bucket[j + 1] - bucket[j] > i) lanes.push_back(j);
            std::stable_sort(lanes.begin(), lanes.end(),
                             [&](int a, int b) { return bucket[a + 1] - bucket[a] < bucket[b + 1] - bucket[b]; });
            for (int j : lanes) {
                int best = -1;
                for (int q = bucket[j] - b0; q < bucket[j + 1] - b0; ++q) {
                    if (taken[q]) continue;
                    if (best < 0 || used[src[q] % 32] < used[src[best] % 32] ||
                        (used[src[q] % 32] == used[src[best] % 32] && src[q] < src[best]))
                        best = q;
                }
                taken[best] = 1;
                used[src[best] % 32] += 1;
                inc[bucket[j] + i] = src[best];
            }
        }
    }
}

// Places the tile's incidence lists in its incidence block so that the lanes
// of a warp load their list entries from distinct banks.  At step i lane j
// loads the 16-bit entry first_j + i, i.e. word (first_j + i) >> 1; two lanes
// of one warp conflict on every step both are active when their firsts agree
// mod 64, and on every other step when they differ by 1 mod 64.  The lists
// are laid end to end; at each position the builder places the unplaced list
// whose warp has the fewest such conflicts with its lanes placed so far
// (ties: longer list, then lower local id).  Returns each vertex's first
// entry; moves the entries accordingly.  bucket[j]..bucket[j+1]: vertex j's
// list before placement.
static std::vector<int32_t> bank_place(uint16_t *inc, const std::vector<int32_t> &bucket, int nl)
{
    std::vector<int32_t> first(nl, 0);
    std::vector<uint16_t> src(inc + bucket[0], inc + bucket[nl]);
    std::vector<int> used(((nl + 31) / 32) * 64, 0);
    std::vector<char> placed(nl, 0);
    int p = 0;
    for (int n_left = nl; n_left > 0; --n_left) {
        const int r = p % 64;
        int best = -1, best_score = 0;
        for (int j = 0; j < nl; ++j) {
            if (placed[j]) continue;
            const int *u = &used[(j / 32) * 64];
            const int score = 2 * u[r] + u[(r + 1) % 64] + u[(r + 63) % 64];
            const int len = bucket[j + 1] - bucket[j], blen = best < 0 ? 0 : bucket[best + 1] - bucket[best];
            if (best < 0 || score < best_score || (score == best_score && len > blen)) {
                best = j;
                best_score = score;
            }
        }
        placed[best] = 1;
        first[best] = p;
        const int len = bucket[best + 1] - bucket[best];
        if (len > 0) used[(best / 32) * 64 + r] += 1;
        for (int q = 0; q < len; ++q) inc[p + q] = src[bucket[best] + q];
        p += len;
    }
    return first;
}

bool build_tiles(int dim, int64_t nv, int64_t ne, const double *X, const int32_t *T, const uint8_t *fixed,
                 int te_max, int tv_max, int rec_stride, TileBuild &out, std::string &err)
{
    const int nc = dim + 1;
    out = TileBuild();
    out.dim = dim;
    out.nv = nv;
    out.ne = ne;
    if (tv_max > 256) tv_max = 256;
    if (te_max < 1) te_max = 1;
    if (rec_stride < nc * dim + 2) {
        err = "element record stride too small for the corner forces";
        return false;
    }
    out.rs = rec_stride;
    if ((int64_t)te_max * rec_stride > 65535) te_max = 65535 / rec_stride / kElemPad * kElemPad;

    // --- Morton order of element centroids, quantised at the mean element size
    std::vector<double> lo(dim, INFINITY), hi(dim, -INFINITY);
    for (int64_t i = 0; i < nv; ++i)
        for (int c = 0; c < dim; ++c) {
            lo[c] = std::min(lo[c], X[i * dim + c]);
            hi[c] = std::max(hi[c], X[i * dim + c]);
        }
    double vol = 1.0;
    for (int c = 0; c < dim; ++c) vol *= std::max(hi[c] - lo[c], 1e-300);
    double cell = std::pow(vol / std::max<int64_t>(ne, 1) * (dim == 2 ? 2.0 : 6.0), 1.0 / dim);
    if (!(cell > 0.0) || !std::isfinite(cell)) cell = 1.0;
    const uint64_t qmax = dim == 2 ? 0xffffffffull : 0x1fffffull;
    std::vector<uint64_t> code(ne);
    for (int64_t e = 0; e < ne; ++e) {
        uint64_t q[3] = {0, 0, 0};
        for (int c = 0; c < dim; ++c) {
            double s = 0.0;
            for (int k = 0; k < nc; ++k) s += X[(int64_t)T[e * nc + k] * dim + c];
            double v = std::floor((s / nc - lo[c]) / cell);
            if (v < 0) v = 0;
            q[c] = std::min<uint64_t>((uint64_t)v, qmax);
        }
        code[e] = dim == 2 ? (spread2(q[0]) | spread2(q[1]) << 1)
                           : (spread3(q[0]) | spread3(q[1]) << 1 | spread3(q[2]) << 2);
    }
    out.perm.resize(ne);
    std::iota(out.perm.begin(), out.perm.end(), 0);
    std::stable_sort(out.perm.begin(), out.perm.end(), [&](int32_t a, int32_t b) { return code[a] < code[b]; });

    // --- greedy cut into tiles
    std::vector<int32_t> stamp(nv, -1);
    out.tile_elem.push_back(0);
    int cur = 0, cur_ne = 0, cur_nv = 0;
    for (int64_t i = 0; i < ne; ++i) {
        const int32_t *t = T + (int64_t)out.perm[i] * nc;
        int fresh = 0;
        for (int k = 0; k < nc; ++k)
            if (stamp[t[k]] != cur) ++fresh;
        if (cur_ne > 0 && (cur_ne + 1 > te_max || cur_nv + fresh > tv_max)) {
            out.tile_elem.push_back((int32_t)i);
            ++cur;
            cur_ne = cur_nv = 0;
            fresh = nc;
        }
        if (fresh > tv_max) {
            err = "element has more vertices than a tile allows";
            return false;
        }
        for (int k = 0; k < nc; ++k)
            if (stamp[t[k]] != cur) {
                stamp[t[k]] = cur;
                ++cur_nv;
            }
        ++cur_ne;
    }
    if (ne > 0) out.tile_elem.push_back((int32_t)ne);
    out.n_tiles = (int)out.tile_elem.size() - 1;

    // --- padded layout: local vertices, packed connectivity, incidence lists
    auto round_up = [](int64_t v, int64_t m) { return (v + m - 1) / m * m; };
    std::vector<int32_t> cut = out.tile_elem;  // unpadded cut points in Morton order
    std::vector<int32_t> order = out.perm;
    out.tile_elem.assign(1, 0);
    for (int ti = 0; ti < out.n_tiles; ++ti)
        out.tile_elem.push_back((int32_t)round_up(out.tile_elem.back() + (cut[ti + 1] - cut[ti]), kElemPad));
    out.ne_int = out.tile_elem.back();
    for (int ti = 0; ti < out.n_tiles; ++ti)
        out.max_te = std::max(out.max_te, out.tile_elem[ti + 1] - out.tile_elem[ti]);
    if ((int64_t)out.max_te * rec_stride > 65535) {
        err = "tile too large for 16-bit corner offsets";
        return false;
    }
    out.perm.assign(out.ne_int, -1);
    for (int ti = 0; ti < out.n_tiles; ++ti)
        for (int i = cut[ti]; i < cut[ti + 1]; ++i) out.perm[out.tile_elem[ti] + (i - cut[ti])] = order[i];
    std::vector<int32_t> loc(nv, -1), cnt(nv, 0), first_tile(nv, -1);
    out.conn.assign(out.ne_int, 0u);
    out.inc.assign((size_t)out.ne_int * nc, 0);
    out.tile_vert.push_back(0);
    std::vector<int32_t> verts, bucket;
    for (int ti = 0; ti < out.n_tiles; ++ti) {
        const int es = out.tile_elem[ti];
        const int n_real = cut[ti + 1] - cut[ti];
        verts.clear();
        for (int i = es; i < es + n_real; ++i)
            for (int k = 0; k < nc; ++k) verts.push_back(T[(int64_t)out.perm[i] * nc + k]);
        std::sort(verts.begin(), verts.end());
        verts.erase(std::unique(verts.begin(), verts.end()), verts.end());
        const int nl = (int)verts.size();
        const int nl_pad = (int)round_up(nl, kVertPad);
        out.max_tv = std::max(out.max_tv, nl_pad);
        for (int j = 0; j < nl; ++j) {
            loc[verts[j]] = j;
            cnt[verts[j]] += 1;
            if (first_tile[verts[j]] < 0) first_tile[verts[j]] = ti;
        }
        bucket.assign(nl + 1, 0);
        for (int i = es; i < es + n_real; ++i) {
            uint32_t w = 0;
            for (int k = 0; k < nc; ++k) {
                const int l = loc[T[(int64_t)out.perm[i] * nc + k]];
                w |= (uint32_t)l << (8 * k);
                bucket[l + 1] += 1;
            }
            out.conn[i] = w;
        }
        for (int j = 0; j < nl; ++j) bucket[j + 1] += bucket[j];
        const int64_t base = (int64_t)es * nc;
        std::vector<int> fill(bucket.begin(), bucket.end() - 1);
        for (int i = es; i < es + n_real; ++i)
            for (int k = 0; k < nc; ++k) {
                const int l = loc[T[(int64_t)out.perm[i] * nc + k]];
                out.inc[base + fill[l]++] =
                    (uint16_t)((i - es) * rec_stride + corner_base(i - es) + k * dim);
            }
        bank_order(out.inc.data() + base, bucket, nl);
        const std::vector<int32_t> first = bank_place(out.inc.data() + base, bucket, nl);
        for (int j = 0; j < nl; ++j)
            out.lv_inc.push_back((uint32_t)first[j] | ((uint32_t)(bucket[j + 1] - bucket[j]) << 16) |
                                 ((fixed && fixed[verts[j]]) ? kLvPinned : 0u));
        for (int j = 0; j < nl; ++j) out.lv_gid.push_back(verts[j]);
        for (int j = nl; j < nl_pad; ++j) {
            out.lv_gid.push_back(verts[0]);  // a valid id, never written
            out.lv_inc.push_back(0u);
        }
        out.n_real_lv += nl;
        out.tile_vert.push_back((int32_t)out.lv_gid.size());
    }

    // --- halo vertices and their partial-sum slots
    std::vector<int32_t> fin_index(nv, -1);
    out.fin_ptr.push_back(0);
    for (int64_t v = 0; v < nv; ++v) {
        if (cnt[v] == 0) {
            err = "vertex " + std::to_string(v) + " belongs to no element";
            return false;
        }
        if (cnt[v] >= 2) {
            fin_index[v] = (int32_t)out.fin_gid.size();
            out.fin_gid.push_back((int32_t)v);
            out.fin_ptr.push_back(out.fin_ptr.back() + cnt[v]);
        }
    }
    out.n_slots = out.fin_ptr.back();
    out.vfin = fin_index;
    std::vector<int32_t> next(out.fin_ptr.begin(), out.fin_ptr.end() - 1);
    out.lv_code.assign(out.lv_gid.size(), LV_PAD);
    for (int ti = 0; ti < out.n_tiles; ++ti)
        for (int j = out.tile_vert[ti]; j < out.tile_vert[ti + 1]; ++j) {
            if (((out.lv_inc[j] >> 16) & kLvCountMask) == 0) continue;  // padding entry
            const int32_t v = out.lv_gid[j];
            if (cnt[v] == 1) {
                out.lv_code[j] = LV_INTERIOR;
            } else {
                const int32_t slot = next[fin_index[v]]++;
                out.lv_code[j] = slot * 2 + (first_tile[v] == ti ? 1 : 0);
            }
        }
    return true;
}

}  // namespace softsim
