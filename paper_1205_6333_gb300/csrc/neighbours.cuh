// neighbours.cuh -- walk over the hashed cell list (built in cells.cu).
#pragma once
#include "sd_internal.h"

namespace sd {

// Calls f(j) for every particle j != i whose cell is one of the 27 cells around
// cell ci, in fixed order (cells by offset, bucket entries by index).
// A neighbour cell coordinate: wrapped in a periodic dimension (nc > 0).
__device__ __forceinline__ int cell_wrap(int c, int nc) {
    if (nc <= 0) return c;
    return c < 0 ? c + nc : (c >= nc ? c - nc : c);
}

template <typename Fn>
__device__ __forceinline__ void for_each_neighbour(const CellList &c, int i, int4 ci, Fn &&f) {
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int cx = cell_wrap(ci.x + ox, c.nc[0]), cy = cell_wrap(ci.y + oy, c.nc[1]),
                          cz = cell_wrap(ci.z + oz, c.nc[2]);
                const uint32_t b = cell_hash(cx, cy, cz, c.H);
                const int s1 = c.start[b + 1];
                for (int s = c.start[b]; s < s1; ++s) {
                    const int j = static_cast<int>(dbg_index(c.sorted[dbg_index(s, c.n, c.err)], c.n, c.err));
                    if (j == i) continue;
                    const int4 cj = c.cell[j];
                    if (cj.x != cx || cj.y != cy || cj.z != cz) continue;  // another cell in the same bucket
                    f(j);
                }
            }
}

// The same walk split over `step` cooperating threads: this thread visits the
// neighbour cells first, first + step, ... of the 27 (same per-cell order).
template <typename Fn>
__device__ __forceinline__ void for_each_neighbour_part(const CellList &c, int i, int4 ci, int first, int step,
                                                        Fn &&f) {
    for (int k = first; k < 27; k += step) {
        const int cx = cell_wrap(ci.x + (k % 3) - 1, c.nc[0]), cy = cell_wrap(ci.y + (k / 3) % 3 - 1, c.nc[1]),
                  cz = cell_wrap(ci.z + k / 9 - 1, c.nc[2]);
        const uint32_t b = cell_hash(cx, cy, cz, c.H);
        const int s1 = c.start[b + 1];
        for (int s = c.start[b]; s < s1; ++s) {
            const int j = static_cast<int>(dbg_index(c.sorted[dbg_index(s, c.n, c.err)], c.n, c.err));
            if (j == i) continue;
            const int4 cj = c.cell[j];
            if (cj.x != cx || cj.y != cy || cj.z != cz) continue;
            f(j);
        }
    }
}

// Nearest-image FP64 separation r_i - r_j (identity in unbounded dimensions).
__device__ __forceinline__ void box_image(const Box &b, double &dx, double &dy, double &dz) {
    if (!b.periodic) return;
    dx = min_image_f64(dx, b.L[0], b.invL[0]);
    dy = min_image_f64(dy, b.L[1], b.invL[1]);
    dz = min_image_f64(dz, b.L[2], b.invL[2]);
}

// Threads per particle in the neighbour-walking kernels (a power of two <= 32;
// consecutive lanes of one warp), and the fixed-order sum over them.
constexpr int kWalkLanes = 8;

__device__ __forceinline__ double walk_sum(double v) {
    for (int o = kWalkLanes / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Lanes of this thread's group whose flag `b` is set (bit k = sub-lane k).
__device__ __forceinline__ unsigned walk_mask(bool b) {
    const unsigned m = __ballot_sync(0xffffffffu, b);
    const int lane = threadIdx.x & 31;
    return (m >> (lane & ~(kWalkLanes - 1))) & ((1u << kWalkLanes) - 1u);
}

// Combine per-lane FP64 partial sums v[0..K) of a group.  Most groups have at
// most one lane with a non-zero contribution (that lane's sums are the result,
// no arithmetic); only when some group in the warp has two or more does the
// warp run the fixed shuffle tree.  Returns the sub-lane that holds the result.
template <int K>
__device__ __forceinline__ int walk_combine(double (&v)[K], bool contributed, int sub) {
    const unsigned gm = walk_mask(contributed);
    const bool many = __popc(gm) > 1;
    if (__any_sync(0xffffffffu, many)) {
        for (int d = 0; d < K; ++d) v[d] = walk_sum(v[d]);
        return 0;
    }
    (void)sub;
    return gm ? __ffs(gm) - 1 : 0;
}
__device__ __forceinline__ bool walk_any(bool b) {
    const unsigned m = __ballot_sync(0xffffffffu, b);
    const int lane = threadIdx.x & 31;
    const unsigned grp = ((1u << kWalkLanes) - 1u) << (lane & ~(kWalkLanes - 1));
    return (m & grp) != 0u;
}

}  // namespace sd
