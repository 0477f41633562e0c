// Constants of the padded tile layout shared by the host builder and the kernels.
#pragma once

#include <cstdint>

namespace softsim {

constexpr int kElemPad = 8;           // element ranges padded to this many entries
constexpr int kVertPad = 4;           // local-vertex ranges padded to this many entries
constexpr int32_t LV_INTERIOR = -1;   // vertex touched by this tile only
constexpr int32_t LV_PAD = -2;        // padding entry

}  // namespace softsim
