// Constants of the padded tile layout shared by the host builder and the kernels.
#pragma once

#include <cstdint>

namespace softsim {

constexpr int kElemPad = 8;           // element ranges padded to this many entries
constexpr int kVertPad = 4;           // local-vertex ranges padded to this many entries
constexpr int32_t LV_INTERIOR = -1;   // vertex touched by this tile only
constexpr int32_t LV_PAD = -2;        // padding entry
// lv_inc word: bits 0-15 first incidence within the tile, bits 16-30 count,
// bit 31 set when the vertex is pinned (Dirichlet).
constexpr uint32_t kLvPinned = 0x80000000u;
constexpr uint32_t kLvCountMask = 0x7fffu;

// Element record of the HVP tile kernels: the nf element fields (Dm^-1, g, W,
// and the fiber f with the spring muscle) followed by the activation a,
// padded to a stride of 2 mod 4 words so that the pair loads of a warp's
// records (8 bytes in FP32, 16 in FP64) fall in distinct banks.  In shared
// memory the same record later holds the element's (d+1)*d corner forces.
#ifdef __CUDACC__
#define SOFTSIM_HD __host__ __device__
#else
#define SOFTSIM_HD
#endif
SOFTSIM_HD constexpr int hvp_fields(int dim, bool spring) { return dim * dim + dim + 1 + (spring ? dim : 0); }
SOFTSIM_HD constexpr int rec_stride(int nf) { return nf + 1 + ((2 - (nf + 1) % 4) + 4) % 4; }
// First slot of the corner forces in the record of local element le: 0 or 2.
// With an even stride, records le and le + 16 start in the same bank; moving
// the corner block of half the elements by two words (pair-aligned) spreads
// the vertex phase's corner loads over more banks (bit 6 measured best on
// the tiles of a 6-tet hex mesh; any bit from 4 up does about as well).
SOFTSIM_HD constexpr int corner_base(int le) { return 2 * ((le >> 6) & 1); }
#undef SOFTSIM_HD

}  // namespace softsim
