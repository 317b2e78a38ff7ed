// neighbours.cuh -- walk over the hashed cell list (built in cells.cu).
#pragma once
#include "sd_internal.h"

namespace sd {

// Calls f(j) for every particle j != i whose cell is one of the 27 cells around
// cell ci, in fixed order (cells by offset, bucket entries by index).
template <typename Fn>
__device__ __forceinline__ void for_each_neighbour(const CellList &c, int i, int4 ci, Fn &&f) {
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int cx = ci.x + ox, cy = ci.y + oy, cz = ci.z + oz;
                const uint32_t b = cell_hash(cx, cy, cz, c.H);
                const int s1 = c.start[b + 1];
                for (int s = c.start[b]; s < s1; ++s) {
                    const int j = c.sorted[s];
                    if (j == i) continue;
                    const int4 cj = c.cell[j];
                    if (cj.x != cx || cj.y != cy || cj.z != cz) continue;  // another cell in the same bucket
                    f(j);
                }
            }
}

}  // namespace sd
