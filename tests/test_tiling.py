"""Host-side tile builder (CPU only): every invariant the element kernels rely
on for the deterministic element -> vertex reduction."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2102_05791_gb300", "csrc")
HERE = os.path.dirname(os.path.abspath(__file__))
LV_INTERIOR, LV_PAD = -1, -2
PINNED, COUNT_MASK = 0x80000000, 0x7FFF


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("tiling") / "libtiling.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "tiling_harness.cpp"), os.path.join(CSRC, "tiling.cpp"), "-o", out],
                   check=True)
    L = C.CDLL(out)
    vp = C.c_void_p
    L.tb_build.argtypes = [C.c_int, C.c_int64, C.c_int64, vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_char_p,
                           C.c_int]
    L.tb_build.restype = vp
    L.tb_free.argtypes = [vp]
    L.tb_scalar.argtypes = [vp, C.c_int]
    L.tb_scalar.restype = C.c_int64
    L.tb_len.argtypes = [vp, C.c_int]
    L.tb_len.restype = C.c_int64
    L.tb_copy.argtypes = [vp, C.c_int, vp]
    for f, n in (("tb_hvp_fields", 2), ("tb_rec_stride", 1), ("tb_corner_base", 1)):
        getattr(L, f).argtypes = [C.c_int] * n
        getattr(L, f).restype = C.c_int
    return L


DT = [np.int32, np.int32, np.int32, np.int32, np.int32, np.uint32, np.uint16, np.uint32, np.int32, np.int32, np.int32]
NAMES = ["perm", "tile_elem", "tile_vert", "lv_gid", "lv_code", "lv_inc", "inc", "conn", "fin_gid", "fin_ptr", "vfin"]


def tile_lists(t, ti, nc):
    """Tile ti's incidence lists, one array per local vertex in the kernels'
    summation order (vertex k's list starts at its first-incidence field)."""
    es, vs, ve = t["tile_elem"][ti], t["tile_vert"][ti], t["tile_vert"][ti + 1]
    linc = t["lv_inc"][vs:ve].astype(np.int64)
    first, count = linc & 0xFFFF, (linc >> 16) & COUNT_MASK
    inc = t["inc"][es * nc:t["tile_elem"][ti + 1] * nc].astype(np.int64)
    return [inc[first[k]:first[k] + count[k]] for k in range(ve - vs)]


def rec_stride(dim, spring=False):
    """Element-record stride of the HVP kernels: the element fields (Dm^-1, g,
    W, and f with the spring muscle) plus the activation, padded to 2 mod 4."""
    nf = dim * dim + dim + 1 + (dim if spring else 0)
    rs = nf + 1
    while rs % 4 != 2:
        rs += 1
    return rs


def build(L, p, te, tv=256, rs=None):
    X = np.ascontiguousarray(p.X, np.float64)
    T = np.ascontiguousarray(p.T, np.int32)
    fx = np.ascontiguousarray(p.fixed, np.uint8)
    err = C.create_string_buffer(256)
    rs = rec_stride(p.dim) if rs is None else rs
    h = L.tb_build(p.dim, len(X), len(T), X.ctypes.data, T.ctypes.data, fx.ctypes.data, te, tv, rs, err, 256)
    if not h:
        raise ValueError(err.value.decode())
    out = {n: np.zeros(L.tb_len(h, i), DT[i]) for i, n in enumerate(NAMES)}
    for i, n in enumerate(NAMES):
        if len(out[n]):
            L.tb_copy(h, i, out[n].ctypes.data)
    for i, n in enumerate(["n_tiles", "max_te", "max_tv", "ne_int", "n_slots"]):
        out[n] = L.tb_scalar(h, i)
    out["rs"] = rs
    L.tb_free(h)
    return out


CASES = {
    "c1": (synth.make_config1, 64),
    "c1_one_tile": (synth.make_config1, 1024),
    "tet5": (lambda: synth.make_small3d(6, 4, 4, split=5), 96),
    "tet6": (lambda: synth.make_small3d(8, 4, 4, split=6), 200),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_tile_layout_invariants(lib, name):
    make, te = CASES[name]
    p = make()
    t = build(lib, p, te)
    d, nc = p.dim, p.dim + 1
    nt = t["n_tiles"]
    te_, tv_ = t["tile_elem"], t["tile_vert"]
    # padding and alignment for the bulk copies
    assert (te_ % 8 == 0).all() and (tv_ % 4 == 0).all()
    assert t["ne_int"] == te_[-1] and t["max_tv"] <= 256
    assert t["max_te"] == np.diff(te_).max() and t["max_tv"] == np.diff(tv_).max()
    # every element exactly once, padding marked -1
    real = t["perm"][t["perm"] >= 0]
    assert np.array_equal(np.sort(real), np.arange(p.n_elem))
    tiles_of = [set() for _ in range(p.n_vert)]
    max_te = t["max_te"]
    for ti in range(nt):
        es, ee = te_[ti], te_[ti + 1]
        vs, ve = tv_[ti], tv_[ti + 1]
        perm = t["perm"][es:ee]
        n_real = int((perm >= 0).sum())
        assert n_real <= te and (perm[:n_real] >= 0).all() and (perm[n_real:] == -1).all()
        gid = t["lv_gid"][vs:ve]
        code = t["lv_code"][vs:ve]
        linc = t["lv_inc"][vs:ve]
        count = (linc >> 16) & COUNT_MASK
        real_lv = count > 0
        assert (code[~real_lv] == LV_PAD).all() and (code[real_lv] != LV_PAD).all()
        g_real = gid[real_lv]
        assert np.array_equal(g_real, np.unique(g_real))  # sorted, unique
        # local connectivity unpacks to the element's global vertices
        conn = t["conn"][es:es + n_real]
        lids = np.stack([(conn >> (8 * k)) & 0xFF for k in range(nc)], axis=1)
        assert np.array_equal(gid[lids], p.T[perm[:n_real]])
        assert set(g_real.tolist()) == set(p.T[perm[:n_real]].ravel().tolist())
        # incidence lists: offsets local elem*rs + corner*d, each corner exactly once
        lists = tile_lists(t, ti, nc)
        seen = np.zeros((n_real, nc), int)
        rs = t["rs"]
        for k in np.nonzero(real_lv)[0]:
            offs = lists[k]
            assert len(offs) == count[k]
            le, slot = offs // rs, offs % rs
            slot = slot - 2 * ((le >> 6) & 1)  # corner block moved by two words in half the records
            assert (slot >= 0).all() and (slot % d == 0).all() and (slot < nc * d).all()
            corner = slot // d
            assert (le < n_real).all()
            assert (lids[le, corner] == k).all()
            seen[le, corner] += 1
            # pinned flag
            assert bool(linc[k] & PINNED) == bool(p.fixed[gid[k]])
        assert (seen == 1).all()
        for v in g_real:
            tiles_of[v].add(ti)
    # halo bookkeeping
    ntile = np.array([len(s) for s in tiles_of])
    assert (ntile >= 1).all()
    halo = np.nonzero(ntile >= 2)[0]
    assert np.array_equal(t["fin_gid"], halo)
    assert np.array_equal(np.diff(t["fin_ptr"]), ntile[halo])
    assert t["n_slots"] == ntile[halo].sum()
    assert ((t["vfin"] >= 0) == (ntile >= 2)).all()
    assert np.array_equal(t["fin_gid"][t["vfin"][halo]], halo)
    slot_owner = {}
    for ti in range(nt):
        vs, ve = tv_[ti], tv_[ti + 1]
        for k in range(vs, ve):
            c = int(t["lv_code"][k])
            v = int(t["lv_gid"][k])
            if c == LV_PAD:
                continue
            if ntile[v] == 1:
                assert c == LV_INTERIOR
            else:
                slot, owner = c >> 1, c & 1
                f = t["vfin"][v]
                assert t["fin_ptr"][f] <= slot < t["fin_ptr"][f + 1]
                assert owner == (ti == min(tiles_of[v]))
                assert slot not in slot_owner
                slot_owner[slot] = ti
    # slots of each halo vertex are in tile order
    for f, v in enumerate(halo):
        s = [slot_owner[q] for q in range(t["fin_ptr"][f], t["fin_ptr"][f + 1])]
        assert s == sorted(s)


def _corner_wavefronts(t, nc, element_order=False):
    # mean shared-memory wavefronts per corner load of the vertex phase, where
    # lane j of a warp walks the list of local vertex 32w + j (bank = word
    # offset mod 32; one wavefront per distinct address in the busiest bank)
    tot = n = 0
    for ti in range(t["n_tiles"]):
        lists = tile_lists(t, ti, nc)
        if element_order:
            lists = [np.sort(x) for x in lists]  # offsets grow with the local element
        for g0 in range(0, len(lists), 32):
            ks = range(g0, min(g0 + 32, len(lists)))
            for i in range(max(len(lists[k]) for k in ks)):
                offs = np.array([lists[k][i] for k in ks if len(lists[k]) > i])
                tot += np.bincount(np.unique(offs) % 32, minlength=32).max()
                n += 1
    return tot / n


def test_incidence_lists_are_bank_aware(lib):
    # a block of 6-tet hexes cut into tiles of 384 tets (the default 3D tile,
    # records of 14 words): the builder's order of each vertex's incidences
    # spreads the lanes of a warp over the banks; listing them in element
    # order instead conflicts about twice as often
    p = synth.make_small3d(16, 8, 8, split=6)
    t = build(lib, p, 384)
    nc = p.dim + 1
    ours = _corner_wavefronts(t, nc)
    base = _corner_wavefronts(t, nc, element_order=True)
    assert ours <= 1.6 and base >= 1.8 * ours, (ours, base)


def _list_wavefronts(t, packed=False):
    # mean wavefronts per 16-bit list-entry load of the vertex phase: lane j
    # of a warp loads entry first_j + i at step i (word (first_j + i) >> 1);
    # packed=True lays the lists end to end in local-vertex order instead
    tot = n = 0
    for ti in range(t["n_tiles"]):
        vs, ve = t["tile_vert"][ti], t["tile_vert"][ti + 1]
        linc = t["lv_inc"][vs:ve].astype(np.int64)
        first, count = linc & 0xFFFF, (linc >> 16) & COUNT_MASK
        if packed:
            first = np.concatenate([[0], np.cumsum(count)[:-1]])
        for g0 in range(0, ve - vs, 32):
            ks = range(g0, min(g0 + 32, ve - vs))
            for i in range(max(int(count[k]) for k in ks)):
                words = np.unique([(first[k] + i) >> 1 for k in ks if count[k] > i])
                tot += np.bincount(words % 32, minlength=32).max()
                n += 1
    return tot / n


def test_incidence_lists_are_placed_bank_aware(lib):
    # where each vertex's list starts in the tile's block is chosen so that the
    # lanes of a warp load their entries from distinct banks; laying the lists
    # end to end in local-vertex order conflicts about twice as often
    p = synth.make_small3d(16, 8, 8, split=6)
    t = build(lib, p, 384)
    ours, packed = _list_wavefronts(t), _list_wavefronts(t, packed=True)
    assert ours <= 2.0 and packed >= 1.5 * ours, (ours, packed)
    # the lists tile the block exactly: no overlap, no gap
    for ti in range(t["n_tiles"]):
        vs, ve = t["tile_vert"][ti], t["tile_vert"][ti + 1]
        linc = t["lv_inc"][vs:ve].astype(np.int64)
        first, count = linc & 0xFFFF, (linc >> 16) & COUNT_MASK
        cover = np.zeros(int(count.sum()), int)
        for f, c in zip(first, count):
            cover[f:f + c] += 1
        assert (cover == 1).all()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("spring", [0, 1])
def test_element_record_layout(lib, dim, spring):
    # the HVP record: the element fields (Dm^-1, g, W; f with the spring), the
    # activation, padding to a stride of 2 mod 4 words (conflict-free pair
    # loads across a warp); the corner block fits after its base in every
    # record and starts pair-aligned
    nf = lib.tb_hvp_fields(dim, spring)
    assert nf == dim * dim + dim + 1 + (dim if spring else 0)
    rs = lib.tb_rec_stride(nf)
    assert rs == rec_stride(dim, bool(spring)) and rs >= nf + 1 and rs % 4 == 2 and rs < nf + 5
    for le in range(1024):
        base = lib.tb_corner_base(le)
        assert base % 2 == 0 and base + (dim + 1) * dim <= rs
    # pair loads of 32 consecutive records hit 16 distinct 8-byte bank pairs per half warp
    pairs = [(rs * le // 2) % 16 for le in range(16)]
    assert len(set(pairs)) == 16


def test_single_tile_has_no_halo(lib):
    t = build(lib, synth.make_config1(), 1024)
    assert t["n_tiles"] == 1 and len(t["fin_gid"]) == 0 and (t["lv_code"][t["lv_code"] != LV_PAD] == LV_INTERIOR).all()


def test_isolated_vertex_is_rejected(lib):
    p = synth.make_small2d(2, 1)
    X = np.vstack([p.X, [[5.0, 5.0]]])
    q = synth.SynthProblem("iso", 2, X, p.T, np.zeros(len(X), np.uint8), p.fiber, p.a, p.target)
    with pytest.raises(ValueError, match="belongs to no element"):
        build(lib, q, 64)
