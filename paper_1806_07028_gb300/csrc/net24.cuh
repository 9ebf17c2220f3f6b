// A sorting network for up to 24 elements held in one thread's registers.
//
// Batcher's odd-even merge sort on 32 positions, every comparator putting the
// element that comes first at its lower position. Padding that comes after
// every element never moves down, so with the positions from kNet24 on holding
// padding no comparator reaching them ever swaps; they are left out, and 132
// comparators sort 24 positions. Used with the comparators as template
// arguments, so every register index is a compile-time constant. The header
// also compiles as plain C++ (the host-side check of the network).
#pragma once

#if defined(__CUDACC__)
#define PC_NET24_HD __host__ __device__
#else
#define PC_NET24_HD
#endif

namespace pc {

constexpr int kNet24 = 24;

// comparator q's lower (first = true) or upper position; for q < 0 the number
// of comparators
PC_NET24_HD constexpr int net24(int q, bool first) {
    int m = 0;
    for (int p = 1; p < 32; p <<= 1)
        for (int k = p; k >= 1; k >>= 1)
            for (int j = k % p; j + k < 32; j += 2 * k)
                for (int i = 0; i < k; ++i) {
                    const int a = i + j, c = i + j + k;
                    if (c < kNet24 && a / (2 * p) == c / (2 * p)) {
                        if (m == q) return first ? a : c;
                        ++m;
                    }
                }
    return m;
}

constexpr int kNet24Size = net24(-1, true);
static_assert(kNet24Size == 132, "odd-even merge network on 24 of 32 positions");

}  // namespace pc
