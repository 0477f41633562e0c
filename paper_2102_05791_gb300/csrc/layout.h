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

}  // namespace softsim
