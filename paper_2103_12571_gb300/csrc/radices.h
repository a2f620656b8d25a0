// Radix plan of a mixed-radix FFT length (plain C++, shared by the host
// planner and the kernels).
#pragma once

namespace ac {

// n = r[0] r[1] ... r[ns-1], each r[s] in {2, 3, 4, 5, 7, 8}; stage s of the
// Stockham transform takes radix r[s].  ns = 0 for n = 1.
struct FftRadices {
    int ns;
    int r[15];
};

}  // namespace ac
