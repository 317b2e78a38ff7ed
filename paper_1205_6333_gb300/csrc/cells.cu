// cells.cu -- staging of FP64 state into the dense kernels' mirrors, the hashed
// cell list, and force assembly (Sec. 3.1, step 2: F_ext + pair interactions,
// the primed sums accelerated by neighbour lists; the paper notes that particle
// sorting is needed for these short-ranged parts but not for the all-pairs sum,
// Sec. 3.2).
//
// Cell list: cells of side h >= max(r_near, repulsion cutoff) over FP64
// positions; the integer cell (cx, cy, cz) is hashed into H = 2^k >= 2n buckets,
// so unbounded domains need no bounding box.  Build = count, exclusive scan,
// scatter, and an insertion sort of each bucket by particle index (makes every
// neighbour walk, hence every FP64 near-pair sum, independent of atomics order).
#include <type_traits>

#include "neighbours.cuh"

namespace sd {

// ---------------------------------------------------------------- staging

// Entry i of a mirror: (x, y, z, 0) in the AoS array and, if present, the SoA copy.
template <typename V4>
__device__ __forceinline__ void put_mirror(V4 *aos, float *soa, int npad, int i, double x, double y, double z) {
    V4 v;
    v.x = x;
    v.y = y;
    v.z = z;
    v.w = 0;
    aos[i] = v;
    if (soa) {
        soa[i] = static_cast<float>(x);
        soa[npad + i] = static_cast<float>(y);
        soa[2 * static_cast<size_t>(npad) + i] = static_cast<float>(z);
    }
}

// u wrapped into [0, L) in a periodic dimension (L > 0), unchanged otherwise.
__device__ __forceinline__ double wrap_box(double u, double L, double invL) {
    return L > 0.0 ? u - L * floor(u * invL) : u;
}

// Mirror entry of a position: relative to particle 0 (only differences enter the
// pair terms, and small coordinates keep FP32 separations accurate), wrapped into
// the box in periodic dimensions (the pair terms take the nearest image).
template <typename V4>
__device__ __forceinline__ void put_pos_mirror(V4 *m, float *soa, int npad, int i, const double *x, const Box &b) {
    const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
    put_mirror(m, soa, npad, i, wrap_box(px - x[0], b.L[0], b.invL[0]), wrap_box(py - x[1], b.L[1], b.invL[1]),
               wrap_box(pz - x[2], b.L[2], b.invL[2]));
}

template <typename V4>
__global__ void stage_pos_kernel(const double *__restrict__ x, V4 *__restrict__ m, float *__restrict__ soa, int n,
                                 int npad, Box b, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
    if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) atomicOr(err, DEV_ERR_NONFINITE);
    put_pos_mirror(m, soa, npad, i, x, b);
}

cudaError_t launch_stage_pos(sd_handle *h, cudaStream_t st, const double *x64, Mirror posm) {
    if (h->n == 0) return cudaSuccess;
    const int nb = (h->n + 255) / 256;
    if (h->mode == MODE_FP64)
        stage_pos_kernel<dbl4><<<nb, 256, 0, st>>>(x64, static_cast<dbl4 *>(posm.aos), posm.soa, h->n, h->npad,
                                                   h->cl.box, h->d_err);
    else
        stage_pos_kernel<float4><<<nb, 256, 0, st>>>(x64, static_cast<float4 *>(posm.aos), posm.soa, h->n, h->npad,
                                                     h->cl.box, h->d_err);
    ++h->launches;
    return cudaGetLastError();
}

// The Verlet step's first kernel: the mirror of x (as the cell-list build writes it),
// the rebuild decision and the clamp flag of the step, both written by the last block
// to finish (vl[0] and *flag; vl[1] counts the blocks, vl[2] gathers their bits).
//   * The list holds the pairs within r_near + skin of the positions xref it was
//     built from.  While every particle's displacement since then, relative to
//     particle 0's, stays below skin / 2, pair distances have changed by less than
//     the skin (a uniform translation moves no pair), so the list still holds every
//     pair within r_near.  It is rebuilt early, from skin / 4 on, so that this holds
//     in the step that rebuilds it too.
//   * The clamp flag (some pair closer than r_safe: the all-pairs kernel then clamps
//     every tile) comes from the pairs of that list, in FP64 exactly as the near pass
//     tests them, so the all-pairs kernel need not wait for the near pass.  It is
//     raised outright when the list may miss pairs: no list yet (bit 2 of vl[0]:
//     positions never set), overflowed (its particles corrected in place), or a
//     displacement of skin / 2 or more.  (The list is the steps' own, built when the
//     positions are set and by the steps' rebuilds; no other pass touches it.)
template <typename V4>
__global__ void verlet_check_kernel(const double *__restrict__ x, const double *__restrict__ xref, int n, int npad,
                                    Box b, double quarter_skin2, double half_skin2, double rsafe2,
                                    V4 *__restrict__ m, float *__restrict__ soa, int *flag, int *vl,
                                    const unsigned long long *near_n, int cap, const int2 *__restrict__ ent,
                                    const int *__restrict__ noff, const int *__restrict__ ncnt, int *err) {
    __shared__ int s_invalid;
    if (threadIdx.x == 0) s_invalid = (vl[0] & 2) != 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int bits = s_invalid ? 3 : 0;   // 1: rebuild; 2: clamp every tile
    if (i < n) {
        const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
        if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) atomicOr(err, DEV_ERR_NONFINITE);
        put_pos_mirror(m, soa, npad, i, x, b);
        const double ux = (px - xref[3 * i]) - (x[0] - xref[0]);
        const double uy = (py - xref[3 * i + 1]) - (x[1] - xref[1]);
        const double uz = (pz - xref[3 * i + 2]) - (x[2] - xref[2]);
        const double u2 = ux * ux + uy * uy + uz * uz;
        if (!(u2 < quarter_skin2)) bits |= 1;   // (also NaN)
        if (!(u2 < half_skin2)) bits |= 3;
        if (i == 0 && *near_n > static_cast<unsigned long long>(cap)) bits |= 3;
        if (!(bits & 2)) {   // the list is complete around i: its pairs closer than r_safe
            const int c = ncnt[i];
            if (c < 0) {
                bits |= 3;
            } else {
                const long long e0 = dbg_index(noff[i], static_cast<long long>(cap) - c + 1, err);
                for (int k = 0; k < c; ++k) {
                    const int j = static_cast<int>(dbg_index(ent[e0 + k].y, n, err));
                    double dx = px - x[3 * j], dy = py - x[3 * j + 1], dz = pz - x[3 * j + 2];
                    box_image(b, dx, dy, dz);
                    if (dx * dx + dy * dy + dz * dz < rsafe2) bits |= 2;
                }
            }
        }
    }
    const int any = (__syncthreads_or(bits & 1) ? 1 : 0) | (__syncthreads_or(bits & 2) ? 2 : 0);
    if (threadIdx.x == 0) {
        if (any) atomicOr(&vl[2], any);
        __threadfence();
        const int done = atomicAdd(&vl[1], 1);
        if (done == static_cast<int>(gridDim.x) - 1) {   // every block's bits are in
            __threadfence();
            const int all = atomicExch(&vl[2], 0);
            *flag = (all & 2) ? 1 : 0;
            vl[0] = all & 1;
            vl[1] = 0;
        }
    }
}

cudaError_t launch_verlet_check(sd_handle *h, cudaStream_t st, const double *x64, Mirror posm) {
    if (h->n == 0) return cudaSuccess;
    const int nb = (h->n + 255) / 256;
    const double hs2 = 0.25 * h->skin * h->skin, qs2 = 0.0625 * h->skin * h->skin;
    const double rs2 = kRSafe * kRSafe * h->pc.a * h->pc.a;
    prof_begin(h, SD_KERNEL_CELLS, st);
    if (h->mode == MODE_FP64)
        verlet_check_kernel<dbl4><<<nb, 256, 0, st>>>(x64, h->xref, h->n, h->npad, h->cl.box, qs2, hs2, rs2,
                                                      static_cast<dbl4 *>(posm.aos), posm.soa, h->d_flag, h->d_vl,
                                                      h->vn, h->near_cap, h->vent, h->voff, h->vcnt, h->d_err);
    else
        verlet_check_kernel<float4><<<nb, 256, 0, st>>>(x64, h->xref, h->n, h->npad, h->cl.box, qs2, hs2, rs2,
                                                        static_cast<float4 *>(posm.aos), posm.soa, h->d_flag,
                                                        h->d_vl, h->vn, h->near_cap, h->vent, h->voff, h->vcnt,
                                                        h->d_err);
    prof_end(h, SD_KERNEL_CELLS, st);
    ++h->launches;
    return cudaGetLastError();
}

// dst64 = src (+ fext + gravity when add_ext) and its mirror; src is n x 3 float or double.
template <typename V4, typename Src>
__global__ void stage_forces_kernel(const Src *__restrict__ src, const double *__restrict__ fext, double gx,
                                    double gy, double gz, double *__restrict__ dst, V4 *__restrict__ m,
                                    float *__restrict__ soa, int n, int npad, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double f[3];
    for (int d = 0; d < 3; ++d) f[d] = src ? static_cast<double>(src[3 * i + d]) : 0.0;
    if (fext) {
        f[0] += fext[3 * i] + gx;
        f[1] += fext[3 * i + 1] + gy;
        f[2] += fext[3 * i + 2] + gz;
    }
    if (!isfinite(f[0]) || !isfinite(f[1]) || !isfinite(f[2])) atomicOr(err, DEV_ERR_NONFINITE);
    dst[3 * i] = f[0];
    dst[3 * i + 1] = f[1];
    dst[3 * i + 2] = f[2];
    put_mirror(m, soa, npad, i, f[0], f[1], f[2]);
}

template <typename V4, typename Src>
static void stage_forces_launch(sd_handle *h, cudaStream_t st, const void *src, const double *fe, double *dst64,
                                Mirror dstm) {
    const int nb = (h->n + 255) / 256;
    const double *g = h->cfg.gravity;
    stage_forces_kernel<V4, Src><<<nb, 256, 0, st>>>(static_cast<const Src *>(src), fe, g[0], g[1], g[2], dst64,
                                                     static_cast<V4 *>(dstm.aos), dstm.soa, h->n, h->npad, h->d_err);
}

// src_dtype: SD_DTYPE_F32 / SD_DTYPE_F64 (src may be NULL = zeros); add_ext: add
// the handle's F_ext and gravity.
cudaError_t launch_stage_forces(sd_handle *h, cudaStream_t st, const void *src, int src_dtype, int add_ext,
                                double *dst64, Mirror dstm) {
    if (h->n == 0) return cudaSuccess;
    const double *fe = add_ext ? h->fext64 : nullptr;
    if (h->mode == MODE_FP64) {
        if (src_dtype == SD_DTYPE_F32) stage_forces_launch<dbl4, float>(h, st, src, fe, dst64, dstm);
        else stage_forces_launch<dbl4, double>(h, st, src, fe, dst64, dstm);
    } else {
        if (src_dtype == SD_DTYPE_F32) stage_forces_launch<float4, float>(h, st, src, fe, dst64, dstm);
        else stage_forces_launch<float4, double>(h, st, src, fe, dst64, dstm);
    }
    ++h->launches;
    return cudaGetLastError();
}

// Padding entries n..npad-1 of a position mirror: far from every particle
// (1e18, 0, 0), so that with their zero padding force each pair term with them is
// exactly zero even where the all-pairs kernel does not clamp r^2.
template <typename V4>
__global__ void pad_mirror_kernel(V4 *__restrict__ m, float *__restrict__ soa, int n, int npad) {
    const int i = n + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    put_mirror(m, soa, npad, i, 1.0e18, 0.0, 0.0);
}

cudaError_t launch_pad_mirror(sd_handle *h, cudaStream_t st, Mirror m) {
    const int npad = h->npad > 0 ? h->npad : kPadTo;
    const int cnt = npad - h->n;
    if (cnt <= 0) return cudaSuccess;
    const int nb = (cnt + 255) / 256;
    if (h->mode == MODE_FP64)
        pad_mirror_kernel<dbl4><<<nb, 256, 0, st>>>(static_cast<dbl4 *>(m.aos), m.soa, h->n, npad);
    else
        pad_mirror_kernel<float4><<<nb, 256, 0, st>>>(static_cast<float4 *>(m.aos), m.soa, h->n, npad);
    ++h->launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- cell list

__device__ __forceinline__ int cell_coord(double x, double inv_h) {
    double c = floor(x * inv_h);
    c = fmin(fmax(c, -1.0e9), 1.0e9);  // keep the integer in range for absurd coordinates
    return static_cast<int>(c);
}

// Cell coordinate in dimension d: nc[d] cells over [0, L) of the wrapped coordinate
// in a periodic dimension, cells of side h otherwise.
__device__ __forceinline__ int cell_coord_d(const CellList &c, int d, double x) {
    const int nc = c.nc[d];
    if (nc <= 0) return cell_coord(x, c.inv_h);
    const int k = static_cast<int>(floor(wrap_box(x, c.box.L[d], c.box.invL[d]) * c.box.invL[d] * nc));
    return k < 0 ? 0 : (k >= nc ? nc - 1 : k);
}

// Bins particle i and writes its mirror (position relative to particle 0, in the
// dense kernels' precision), so the mirror is a pure function of the FP64 state.  A
// Verlet list build (xref given) records the positions in xref instead and leaves
// the mirror and the clamp flag to the step's check kernel.
template <typename V4>
__global__ void cells_hash_kernel(const double *__restrict__ x, int n, CellList c, int4 *__restrict__ cell,
                                  uint32_t *__restrict__ key, int *__restrict__ cnt, V4 *__restrict__ m,
                                  float *__restrict__ soa, int npad, int *flag, unsigned long long *near_n,
                                  double *__restrict__ xref, const int *gate, int *err) {
    if (gate && *gate == 0) return;   // a Verlet step without a rebuild request
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0) {
        *near_n = 0;                // the near pass fills its candidate list from the start
        if (!xref) *flag = 0;       // ... and raises the flag again if needed
    }
    const int H = c.H;
    const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
    if (xref) {   // a Verlet step's rebuild: the flag and the mirror are its check kernel's
        xref[3 * i] = px;
        xref[3 * i + 1] = py;
        xref[3 * i + 2] = pz;
    } else {
        if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) atomicOr(err, DEV_ERR_NONFINITE);
        put_pos_mirror(m, soa, npad, i, x, c.box);
    }
    const int cx = cell_coord_d(c, 0, px);
    const int cy = cell_coord_d(c, 1, py);
    const int cz = cell_coord_d(c, 2, pz);
    cell[i] = make_int4(cx, cy, cz, 0);
    const uint32_t k = cell_hash(cx, cy, cz, H);
    key[i] = k;
    atomicAdd(&cnt[k], 1);
}

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 16;
constexpr int kScanBlock = kScanThreads * kScanPer;   // buckets one scan block covers (one kernel up to this)

// Exclusive scan of kScanPer values per thread across a block; returns the
// block total.  Warp shuffles within warps, shared memory across warps.
__device__ __forceinline__ int block_exclusive_scan(int v[kScanPer], int *s_warp) {
    int tsum = 0;
    for (int k = 0; k < kScanPer; ++k) {
        const int t = v[k];
        v[k] = tsum;
        tsum += t;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = tsum;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < kScanThreads / 32) ? s_warp[lane] : 0;
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        s_warp[lane] = wi - w;  // exclusive warp offsets
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    const int off = s_warp[wid] + incl - tsum;
    for (int k = 0; k < kScanPer; ++k) v[k] += off;
    const int total = s_warp[32];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(const int *__restrict__ in, int *__restrict__ out,
                                                                   int *__restrict__ bsum, int H, const int *gate) {
    if (gate && *gate == 0) return;
    __shared__ int s_warp[33];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    int v[kScanPer];
    for (int k = 0; k < kScanPer; ++k) v[k] = (base + k < H) ? in[base + k] : 0;
    const int total = block_exclusive_scan(v, s_warp);
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < H) out[base + k] = v[k];
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = total;
        if (gridDim.x == 1) out[H] = total;   // one block: the scan is complete
    }
}

// One block: exclusive scan of the block totals in place (nblk <= kScanBlock
// per pass, looping with a carry), then start[H] = grand total.
__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(int *__restrict__ bsum, int nblk,
                                                                int *__restrict__ start, int H, const int *gate) {
    if (gate && *gate == 0) return;
    __shared__ int s_warp[33];
    int carry = 0;
    for (int b0 = 0; b0 < nblk; b0 += kScanBlock) {
        const int base = b0 + threadIdx.x * kScanPer;
        int v[kScanPer];
        for (int k = 0; k < kScanPer; ++k) v[k] = (base + k < nblk) ? bsum[base + k] : 0;
        const int total = block_exclusive_scan(v, s_warp);
        for (int k = 0; k < kScanPer; ++k)
            if (base + k < nblk) bsum[base + k] = v[k] + carry;
        carry += total;
    }
    if (threadIdx.x == 0) start[H] = carry;
}

__global__ void scan_add_kernel(int *__restrict__ start, const int *__restrict__ bsum, int H, const int *gate) {
    if (gate && *gate == 0) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < H) start[e] += bsum[e / kScanBlock];
}

// Each particle takes a place in its bucket by counting the bucket's occupancy
// down, which leaves every counter at zero for the next build (no memset).
__global__ void cells_scatter_kernel(const uint32_t *__restrict__ key, int n, const int *__restrict__ start,
                                     int *__restrict__ cnt, int *__restrict__ sorted, const int *gate, int *err) {
    if (gate && *gate == 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = key[i];
    const int pos = start[k] + atomicSub(&cnt[k], 1) - 1;
    if (pos >= start[k] && pos < start[k + 1])   // always, unless a counter was left non-zero
        sorted[pos] = i;
    else
        atomicOr(err, DEV_ERR_BOUNDS);
}

// Sort each bucket by particle index (buckets hold ~1 particle; a bucket larger
// than 256 -- only possible for unphysically dense input -- stays unsorted, which
// changes only the FP64 summation order of its near pairs).
__global__ void cells_sort_kernel(const int *__restrict__ start, int *__restrict__ sorted, int H, const int *gate) {
    if (gate && *gate == 0) return;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= H) return;
    const int s0 = start[b], s1 = start[b + 1];
    if (s1 - s0 < 2 || s1 - s0 > 256) return;
    for (int p = s0 + 1; p < s1; ++p) {
        const int v = sorted[p];
        int q = p - 1;
        while (q >= s0 && sorted[q] > v) {
            sorted[q + 1] = sorted[q];
            --q;
        }
        sorted[q + 1] = v;
    }
}

cudaError_t launch_build_cells(sd_handle *h, cudaStream_t st, const double *x64, Mirror posm, double *xref) {
    CellList &c = h->cl;
    if (h->n == 0) return cudaSuccess;
    // a Verlet build runs only when the step's check asked for it: every kernel reads
    // the request and returns at once without it
    const int *gate = xref ? h->d_vl : nullptr;
    prof_begin(h, SD_KERNEL_CELLS, st);
    // (the bucket counters are zero: zeroed at creation, counted back to zero by
    // every build's scatter)
    const int nb = (h->n + 255) / 256;
    if (h->mode == MODE_FP64)
        cells_hash_kernel<dbl4><<<nb, 256, 0, st>>>(x64, h->n, c, c.cell, c.key, c.cnt,
                                                    static_cast<dbl4 *>(posm.aos), posm.soa, h->npad, h->d_flag,
                                                    xref ? h->vn : h->near_n, xref, gate, h->d_err);
    else
        cells_hash_kernel<float4><<<nb, 256, 0, st>>>(x64, h->n, c, c.cell, c.key, c.cnt,
                                                      static_cast<float4 *>(posm.aos), posm.soa, h->npad,
                                                      h->d_flag, xref ? h->vn : h->near_n, xref, gate, h->d_err);
    scan_blocks_kernel<<<c.nblk, kScanThreads, 0, st>>>(c.cnt, c.start, c.bsum, c.H, gate);
    if (c.nblk > 1) {
        scan_top_kernel<<<1, kScanThreads, 0, st>>>(c.bsum, c.nblk, c.start, c.H, gate);
        scan_add_kernel<<<(c.H + 255) / 256, 256, 0, st>>>(c.start, c.bsum, c.H, gate);
        h->launches += 2;
    }
    cells_scatter_kernel<<<nb, 256, 0, st>>>(c.key, h->n, c.start, c.cnt, c.sorted, gate, h->d_err);
    cells_sort_kernel<<<(c.H + 255) / 256, 256, 0, st>>>(c.start, c.sorted, c.H, gate);
    prof_end(h, SD_KERNEL_CELLS, st);
    h->launches += 4;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- forces (Sec. 3.1, step 2)

// F_i = F_ext,i + g + sum_{j: r_ij < r_c} 12 eps (2a)^12 r^-14 (r_i - r_j)
// (U = eps (2a/r)^12, truncated at r_c, F = -grad U; Sec. 3.1 step 2), and with
// lubrication (vlag != nullptr) the singular friction of Sec. 2.3 Eq. lubrication,
//   F_i -= (1/mu0) sum_{j: 0 < s < 1} [(1/(4s) - (9/40) ln s) e e^T - (1/6) ln s (I - e e^T)] (v_i - v_j),
// s = r/a - 2, e = r_ij / r, with the previous step's velocities vlag (Sec. 3.1:
// the forces are corrected for lubrication before the velocity update).  FP64;
// writes F64 and its mirror.
template <typename V4>
__global__ void forces_rep_kernel(const double *__restrict__ x, const double *__restrict__ fext, double gx, double gy,
                                  double gz, double eps, double rc, double s12, const double *__restrict__ vlag,
                                  double inv_a, double inv_mu0, CellList c, int n, int npad, double *__restrict__ F,
                                  V4 *__restrict__ m, float *__restrict__ soa, int *err) {
    // kWalkLanes threads per particle, partial sums meet in a fixed shuffle tree
    const long long gt = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int i = static_cast<int>(gt / kWalkLanes), sub = static_cast<int>(gt % kWalkLanes);
    const bool active = i < n;
    const bool rep = eps != 0.0, lub = vlag != nullptr;
    const double rc2 = rep ? rc * rc : 0.0;
    const double rl2 = lub ? 9.0 / (inv_a * inv_a) : 0.0;   // (3a)^2
    const double rmax2 = rc2 > rl2 ? rc2 : rl2;
    double f[3] = {0.0, 0.0, 0.0};
    bool coincident = false, found = false;
    if (active) {
        const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
        for_each_neighbour_part(c, i, c.cell[i], sub, kWalkLanes, [&](int j) {
            double dx = xi - x[3 * j], dy = yi - x[3 * j + 1], dz = zi - x[3 * j + 2];
            box_image(c.box, dx, dy, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= rmax2) return;
            found = true;
            if (r2 == 0.0) {
                if (rep) coincident = true;   // s = -2: no lubrication term
                return;
            }
            const double ri = rsqrt_nr64(r2);   // no FP64 division (scarce FP64 throughput)
            if (r2 < rc2) {
                const double ir2 = ri * ri;
                const double ir6 = ir2 * ir2 * ir2;
                const double coef = 12.0 * eps * s12 * ir6 * ir6 * ir2;
                f[0] += coef * dx;
                f[1] += coef * dy;
                f[2] += coef * dz;
            }
            if (lub) {
                // the gap s in FP64 (it cancels: r/a - 2); the coefficients in the
                // working precision of the pair terms (FP32 in the FP32 modes)
                const double sg = r2 * ri * inv_a - 2.0;
                if (sg > 0.0 && sg < 1.0) {
                    double zn, zt;
                    if constexpr (std::is_same<V4, float4>::value) {
                        const float sf = static_cast<float>(sg), ls = logf(sf);
                        zn = __fsub_rn(__fdiv_rn(0.25f, sf), __fmul_rn(0.225f, ls));
                        zt = __fmul_rn(ls, -1.0f / 6.0f);
                    } else {
                        const double ls = log(sg);
                        zn = 0.25 / sg - 0.225 * ls;
                        zt = -ls / 6.0;
                    }
                    const double ex = dx * ri, ey = dy * ri, ez = dz * ri;
                    const double wx = vlag[3 * i] - vlag[3 * j], wy = vlag[3 * i + 1] - vlag[3 * j + 1],
                                 wz = vlag[3 * i + 2] - vlag[3 * j + 2];
                    const double en = ex * wx + ey * wy + ez * wz;
                    // zeta w = zn (e.w) e + zt (w - (e.w) e)
                    const double kn = (zn - zt) * en;
                    f[0] -= inv_mu0 * (kn * ex + zt * wx);
                    f[1] -= inv_mu0 * (kn * ey + zt * wy);
                    f[2] -= inv_mu0 * (kn * ez + zt * wz);
                }
            }
        });
    }
    const int writer = walk_combine(f, found, sub);
    coincident = walk_any(coincident);
    if (!active || sub != writer) return;
    const double f0 = f[0] + fext[3 * i] + gx, f1 = f[1] + fext[3 * i + 1] + gy, f2v = f[2] + fext[3 * i + 2] + gz;
    if (coincident) atomicOr(err, DEV_ERR_COINCIDENT);
    if (!isfinite(f0) || !isfinite(f1) || !isfinite(f2v)) atomicOr(err, DEV_ERR_NONFINITE);
    F[3 * i] = f0;
    F[3 * i + 1] = f1;
    F[3 * i + 2] = f2v;
    put_mirror(m, soa, npad, i, f0, f1, f2v);
}

// Forces of a Verlet step (Sec. 3.1, step 2) with soft repulsion and/or lubrication:
// the pairs come from the steps' near-pair list (it holds every pair within the
// largest cutoff while the list is valid), one thread per particle over its run in
// ascending partner order, in FP64; the terms are forces_rep_kernel's.  Plus F_ext and
// gravity.  Writes F64 and the force mirror.
template <typename V4>
__global__ void forces_list_kernel(const double *__restrict__ x, const double *__restrict__ fext, double gx,
                                   double gy, double gz, double eps, double rc, double s12,
                                   const double *__restrict__ vlag, double inv_a, double inv_mu0, CellList c,
                                   const int2 *__restrict__ ent, const int *__restrict__ noff,
                                   const int *__restrict__ ncnt, int cap, int n, int npad, double *__restrict__ F,
                                   V4 *__restrict__ m, float *__restrict__ soa, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool rep = eps != 0.0, lub = vlag != nullptr;
    const double rc2 = rep ? rc * rc : 0.0;
    const double rl2 = lub ? 9.0 / (inv_a * inv_a) : 0.0;   // (3a)^2
    const double rmax2 = rc2 > rl2 ? rc2 : rl2;
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    double f[3] = {0.0, 0.0, 0.0};
    bool coincident = false;
    auto pair = [&](int j) {
        double dx = xi - x[3 * j], dy = yi - x[3 * j + 1], dz = zi - x[3 * j + 2];
        box_image(c.box, dx, dy, dz);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= rmax2) return;
        if (r2 == 0.0) {
            if (rep) coincident = true;   // s = -2: no lubrication term
            return;
        }
        const double ri = rsqrt_nr64(r2);
        if (r2 < rc2) {
            const double ir2 = ri * ri;
            const double ir6 = ir2 * ir2 * ir2;
            const double coef = 12.0 * eps * s12 * ir6 * ir6 * ir2;
            f[0] += coef * dx;
            f[1] += coef * dy;
            f[2] += coef * dz;
        }
        if (lub) {
            const double sg = r2 * ri * inv_a - 2.0;
            if (sg > 0.0 && sg < 1.0) {
                double zn, zt;
                if constexpr (std::is_same<V4, float4>::value) {
                    const float sf = static_cast<float>(sg), ls = logf(sf);
                    zn = __fsub_rn(__fdiv_rn(0.25f, sf), __fmul_rn(0.225f, ls));
                    zt = __fmul_rn(ls, -1.0f / 6.0f);
                } else {
                    const double ls = log(sg);
                    zn = 0.25 / sg - 0.225 * ls;
                    zt = -ls / 6.0;
                }
                const double ex = dx * ri, ey = dy * ri, ez = dz * ri;
                const double wx = vlag[3 * i] - vlag[3 * j], wy = vlag[3 * i + 1] - vlag[3 * j + 1],
                             wz = vlag[3 * i + 2] - vlag[3 * j + 2];
                const double en = ex * wx + ey * wy + ez * wz;
                const double kn = (zn - zt) * en;
                f[0] -= inv_mu0 * (kn * ex + zt * wx);
                f[1] -= inv_mu0 * (kn * ey + zt * wy);
                f[2] -= inv_mu0 * (kn * ez + zt * wz);
            }
        }
    };
    const int cnt = ncnt[i];
    if (cnt < 0) {   // a particle the overflowed list corrects in place: the cell list (rebuilt
                     // every step while the list overflows) gives its pairs
        for_each_neighbour_part(c, i, c.cell[i], 0, 1, pair);
    } else {
        const long long e0 = dbg_index(noff[i], static_cast<long long>(cap) - cnt + 1, err);
        for (int k = 0; k < cnt; ++k) pair(static_cast<int>(dbg_index(ent[e0 + k].y, n, err)));
    }
    const double f0 = f[0] + fext[3 * i] + gx, f1 = f[1] + fext[3 * i + 1] + gy, f2v = f[2] + fext[3 * i + 2] + gz;
    if (coincident) atomicOr(err, DEV_ERR_COINCIDENT);
    if (!isfinite(f0) || !isfinite(f1) || !isfinite(f2v)) atomicOr(err, DEV_ERR_NONFINITE);
    F[3 * i] = f0;
    F[3 * i + 1] = f1;
    F[3 * i + 2] = f2v;
    put_mirror(m, soa, npad, i, f0, f1, f2v);
}

cudaError_t launch_forces_list(sd_handle *h, cudaStream_t st, const double *x64) {
    if (h->n == 0) return cudaSuccess;
    const int nb = (h->n + 127) / 128;
    const double *g = h->cfg.gravity;
    const double s12 = pow(2.0 * h->cfg.a, 12.0);
    const double *vlag = h->lub ? h->vlag : nullptr;
    const double inv_a = 1.0 / h->pc.a, inv_mu0 = 1.0 / h->pc.mu0;
    prof_begin(h, SD_KERNEL_FORCES, st);
    if (h->mode == MODE_FP64)
        forces_list_kernel<dbl4><<<nb, 128, 0, st>>>(x64, h->fext64, g[0], g[1], g[2], h->cfg.rep_eps, h->rep_rc,
                                                     s12, vlag, inv_a, inv_mu0, h->cl, h->vent, h->voff, h->vcnt,
                                                     h->near_cap, h->n, h->npad, h->F64,
                                                     static_cast<dbl4 *>(h->frcm.aos), h->frcm.soa, h->d_err);
    else
        forces_list_kernel<float4><<<nb, 128, 0, st>>>(x64, h->fext64, g[0], g[1], g[2], h->cfg.rep_eps, h->rep_rc,
                                                       s12, vlag, inv_a, inv_mu0, h->cl, h->vent, h->voff, h->vcnt,
                                                       h->near_cap, h->n, h->npad, h->F64,
                                                       static_cast<float4 *>(h->frcm.aos), h->frcm.soa, h->d_err);
    prof_end(h, SD_KERNEL_FORCES, st);
    ++h->launches;
    return cudaGetLastError();
}

cudaError_t launch_forces_rep(sd_handle *h, cudaStream_t st, const double *x64) {
    if (h->n == 0) return cudaSuccess;
    const int nb = static_cast<int>((static_cast<long long>(h->n) * kWalkLanes + 127) / 128);
    const double *g = h->cfg.gravity;
    const double s12 = pow(2.0 * h->cfg.a, 12.0);
    prof_begin(h, SD_KERNEL_FORCES, st);
    const double *vlag = h->lub ? h->vlag : nullptr;
    const double inv_a = 1.0 / h->pc.a, inv_mu0 = 1.0 / h->pc.mu0;
    if (h->mode == MODE_FP64)
        forces_rep_kernel<dbl4><<<nb, 128, 0, st>>>(x64, h->fext64, g[0], g[1], g[2], h->cfg.rep_eps, h->rep_rc, s12,
                                                    vlag, inv_a, inv_mu0, h->cl, h->n, h->npad, h->F64,
                                                    static_cast<dbl4 *>(h->frcm.aos), h->frcm.soa, h->d_err);
    else
        forces_rep_kernel<float4><<<nb, 128, 0, st>>>(x64, h->fext64, g[0], g[1], g[2], h->cfg.rep_eps, h->rep_rc,
                                                      s12, vlag, inv_a, inv_mu0, h->cl, h->n, h->npad, h->F64,
                                                      static_cast<float4 *>(h->frcm.aos), h->frcm.soa, h->d_err);
    prof_end(h, SD_KERNEL_FORCES, st);
    ++h->launches;
    return cudaGetLastError();
}

}  // namespace sd
