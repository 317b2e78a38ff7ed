// dense.cu -- the all-pairs mobility sum (Sec. 3.1 step 3; Sec. 2.2 Eq. rotneMobility).
//
// Design (GB300, CUDA cores; the pair term is not a dense contraction):
//   * persistent grid of (SMs x resident CTAs); the (i-block, j-tile) plane is cut
//     into equal contiguous runs of tiles, one run per CTA, so every SM gets the
//     same number of pair interactions whatever N is;
//   * each thread keeps R target particles i in registers (position + running sum);
//   * j-tiles of positions and forces (float4 / dbl4, 16 / 32 B each, Sec. 3.2
//     layout) are staged in shared memory by 1-D bulk copies (cp.async.bulk with
//     mbarrier completion), double-buffered, and read back as warp-wide broadcasts;
//   * FP32C: each tile's FP32 partial sum is folded into a two-float (hi, lo)
//     accumulator with TwoSum (Sec. 3.2: single-precision pair terms, higher-precision
//     accumulation); FP64: plain FP64 sums; FP32: plain FP32 sums (ablation);
//   * each CTA writes its partial sum for every i-block it touched into a fixed slot
//     (FP32C: the (hi, lo) float pair; FP64, FP32: one double); the epilogue adds the
//     slots in ascending order (deterministic result).
// Self and overlapping pairs take r^2 clamped to (2a)^2 here; the FP64 epilogue
// replaces them (and every pair closer than r_near) by their exact terms.
#include <algorithm>
#include "sd_internal.h"

namespace sd {

// Failure injection for tests (sd_inject_stall): the launcher passes the watchdog
// limit negated, and the first CTA of the launch then never issues the copy of its
// first tile.  Its bounded waits on that stage run out, the kernel records
// DEV_ERR_TIMEOUT, stops issuing copies, drains the copies it did issue and exits;
// no wait is unbounded and no memory outside the kernel's buffers is touched.
__device__ __forceinline__ bool stall_first_copy(long long wd) { return wd < 0 && blockIdx.x == 0; }

template <int MODE>
struct DenseT;
template <>
struct DenseT<MODE_FP32C> {
    using V4 = float4;
    using S = float;
    static constexpr int R = kR32;
};
template <>
struct DenseT<MODE_FP32> {
    using V4 = float4;
    using S = float;
    static constexpr int R = kR32;
};
template <>
struct DenseT<MODE_FP64> {
    using V4 = dbl4;
    using S = double;
    static constexpr int R = kR64;
};

template <int TENSOR, int MODE, bool PER>
__device__ __forceinline__ void dense_pair(typename DenseT<MODE>::S xi, typename DenseT<MODE>::S yi,
                                           typename DenseT<MODE>::S zi, const typename DenseT<MODE>::V4 &p,
                                           const typename DenseT<MODE>::V4 &f, const PairConst &c,
                                           typename DenseT<MODE>::S &ax, typename DenseT<MODE>::S &ay,
                                           typename DenseT<MODE>::S &az) {
    if constexpr (MODE == MODE_FP64)
        pair_f64<TENSOR, PER>(xi, yi, zi, p, f, c, ax, ay, az);
    else
        pair_f32<TENSOR, true, PER>(xi, yi, zi, p, f, c, ax, ay, az);
}

template <int TENSOR, int MODE, bool PER>
__global__ void __launch_bounds__(kNT) dense_kernel(const typename DenseT<MODE>::V4 *__restrict__ pos,
                                                    const typename DenseT<MODE>::V4 *__restrict__ frc,
                                                    double *__restrict__ part, int npad, DenseGeom g, PairConst c,
                                                    int *__restrict__ err, long long wd, TileWin w) {
    using V4 = typename DenseT<MODE>::V4;
    using S = typename DenseT<MODE>::S;
    constexpr int R = DenseT<MODE>::R;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    V4 *s_pos = reinterpret_cast<V4 *>(smem);
    V4 *s_frc = s_pos + 2 * g.J;

    const int tid = threadIdx.x;
    const long long T = static_cast<long long>(g.nIB) * g.nJT;
    const int cta = static_cast<int>(blockIdx.x) + w.b0;   // index in the full launch
    const long long tb = static_cast<long long>(cta) * g.chunk;
    const long long thi = (w.hi >= 0 && w.hi < T) ? w.hi : T;
    const long long t0 = tb > w.lo ? tb : w.lo;
    const long long t1 = (tb + g.chunk < thi) ? tb + g.chunk : thi;
    if (t0 >= t1) return;  // uniform over the CTA
    const uint32_t tile_bytes = static_cast<uint32_t>(g.J * sizeof(V4));
    const long long lim = wd < 0 ? -wd : wd;   // wd < 0: injected stall (stall_first_copy)

    int issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0;  // bookkeeping of thread 0 only
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int q = 0; q < 2 && t0 + q < t1; ++q) {
            if (q == 0 && stall_first_copy(wd)) continue;
            const size_t jt = static_cast<size_t>((t0 + q) % g.nJT);
            mbar_arrive_expect_tx(&bars[q], 2 * tile_bytes);
            bulk_g2s(s_pos + q * g.J, pos + jt * g.J, tile_bytes, &bars[q]);
            bulk_g2s(s_frc + q * g.J, frc + jt * g.J, tile_bytes, &bars[q]);
            if (q == 0) ++issued0; else ++issued1;
        }
    }

    S xi[R], yi[R], zi[R], ax[R], ay[R], az[R];
    float hx[R], hy[R], hz[R], lx[R], ly[R], lz[R];
    int cur_ib = -1;
    bool aborted = false;

    auto flush = [&](int ib) {
        const int slot = cta - geom_first(g, ib);
        double *dst = part + static_cast<size_t>(slot) * 3 * npad;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const size_t i = static_cast<size_t>(ib) * g.I + tid + k * kNT;
            double vx, vy, vz;
            if constexpr (MODE == MODE_FP32C) {
                vx = static_cast<double>(hx[k]) + static_cast<double>(lx[k]);
                vy = static_cast<double>(hy[k]) + static_cast<double>(ly[k]);
                vz = static_cast<double>(hz[k]) + static_cast<double>(lz[k]);
            } else {
                vx = static_cast<double>(ax[k]);
                vy = static_cast<double>(ay[k]);
                vz = static_cast<double>(az[k]);
            }
            dst[i] = vx;
            dst[npad + i] = vy;
            dst[2 * static_cast<size_t>(npad) + i] = vz;
        }
    };

    for (long long t = t0; t < t1; ++t) {
        const int ib = static_cast<int>(t / g.nJT);
        if (ib != cur_ib) {
            if (cur_ib >= 0) flush(cur_ib);
            cur_ib = ib;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const V4 p = pos[static_cast<size_t>(ib) * g.I + tid + k * kNT];
                xi[k] = p.x;
                yi[k] = p.y;
                zi[k] = p.z;
                ax[k] = ay[k] = az[k] = S(0);
                hx[k] = hy[k] = hz[k] = lx[k] = ly[k] = lz[k] = 0.0f;
            }
        }
        const int q = static_cast<int>(t - t0);
        const int st = q & 1;
        if (!aborted) {
            if (mbar_wait_bounded(&bars[st], (q >> 1) & 1, lim)) {
                if (tid == 0) { if (st == 0) ++waited0; else ++waited1; }
            } else {
                atomicOr(err, DEV_ERR_TIMEOUT);
                s_abort = 1;
            }
        }
        const V4 *P = s_pos + st * g.J;
        const V4 *Fq = s_frc + st * g.J;
#pragma unroll 2
        for (int jj = 0; jj < g.J; ++jj) {
            const V4 p = P[jj];
            const V4 f = Fq[jj];
#pragma unroll
            for (int k = 0; k < R; ++k)
                dense_pair<TENSOR, MODE, PER>(xi[k], yi[k], zi[k], p, f, c, ax[k], ay[k], az[k]);
        }
        if constexpr (MODE == MODE_FP32C) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                fold2(hx[k], lx[k], ax[k]);
                fold2(hy[k], ly[k], ay[k]);
                fold2(hz[k], lz[k], az[k]);
                ax[k] = ay[k] = az[k] = 0.0f;
            }
        }
        __syncthreads();  // every thread is done with stage st
        aborted = s_abort != 0;
        if (tid == 0 && !aborted && t + 2 < t1) {
            const size_t jt = static_cast<size_t>((t + 2) % g.nJT);
            mbar_arrive_expect_tx(&bars[st], 2 * tile_bytes);
            bulk_g2s(s_pos + st * g.J, pos + jt * g.J, tile_bytes, &bars[st]);
            bulk_g2s(s_frc + st * g.J, frc + jt * g.J, tile_bytes, &bars[st]);
            if (st == 0) ++issued0; else ++issued1;
        }
    }
    flush(cur_ib);
    if (tid == 0) {
        // After a time-out, wait (bounded) for copies still in flight into this CTA's
        // shared memory before the CTA exits.
        for (int k = waited0; k < issued0; ++k)
            if (!mbar_wait_bounded(&bars[0], k & 1, drain_limit(lim))) atomicOr(err, DEV_ERR_TIMEOUT);
        for (int k = waited1; k < issued1; ++k)
            if (!mbar_wait_bounded(&bars[1], k & 1, drain_limit(lim))) atomicOr(err, DEV_ERR_TIMEOUT);
    }
}

// ---------------------------------------------------------------- FP32, packed (f32x2)

// The FP32 all-pairs kernel.  Same persistent tiling as above, but the j-tiles
// are staged as six float arrays (x, y, z, Fx, Fy, Fz; six bulk copies) so that
// two consecutive j's form one 64-bit operand, and every instruction of the pair
// term (pair_f32x2) evaluates the pairs (i, j) and (i, j+1) together.  Each thread
// owns R targets i, duplicated into both lanes; its packed accumulators sum even
// and odd j's separately, and both lanes are folded into the (hi, lo) TwoSum
// accumulators (kept in shared memory) after every tile.  COMP = false keeps one
// plain FP32 running sum per lane instead (ablation).
// One staged j-tile against the thread's R targets: 4 j's (two packed pairs) per
// step, six 128-bit shared loads per step.
template <int TENSOR, bool CLAMP, int R, bool PER>
__device__ __forceinline__ void tile_pairs(uint32_t base, uint32_t astride, int J, const f2 (&XI)[R],
                                           const f2 (&YI)[R], const f2 (&ZI)[R], const PairConst2 &c, f2 (&AX)[R],
                                           f2 (&AY)[R], f2 (&AZ)[R]) {
#pragma unroll kJUnroll
    for (int jj = 0; jj < J; jj += 4) {
        f2 P[6][2];
#pragma unroll
        for (int a = 0; a < 6; ++a)
            asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];"
                         : "=l"(P[a][0]), "=l"(P[a][1])
                         : "r"(base + a * astride + jj * 4));
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
            for (int k = 0; k < R; ++k)
                pair_f32x2<TENSOR, CLAMP, PER>(XI[k], YI[k], ZI[k], P[0][h2], P[1][h2], P[2][h2], P[3][h2],
                                               P[4][h2], P[5][h2], c, AX[k], AY[k], AZ[k]);
    }
}

template <int TENSOR, bool COMP, bool PER>
__global__ void __launch_bounds__(kNT) dense2_kernel(const float *__restrict__ pos, const float *__restrict__ frc,
                                                     double *__restrict__ part, int npad, DenseGeom g, PairConst2 c,
                                                     const int *__restrict__ flag, int *__restrict__ err,
                                                     long long wd, TileWin w) {
    constexpr int R = kR32;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    float *s_tile = reinterpret_cast<float *>(smem);          // [2 stages][6 arrays][J]
    float *s_acc = s_tile + 12 * g.J;                          // [R][6][kNT]: hx hy hz lx ly lz

    const int tid = threadIdx.x;
    const long long T = static_cast<long long>(g.nIB) * g.nJT;
    const int cta = static_cast<int>(blockIdx.x) + w.b0;   // index in the full launch
    const long long tb = static_cast<long long>(cta) * g.chunk;
    const long long thi = (w.hi >= 0 && w.hi < T) ? w.hi : T;
    const long long t0 = tb > w.lo ? tb : w.lo;
    const long long t1 = (tb + g.chunk < thi) ? tb + g.chunk : thi;
    if (t0 >= t1) return;
    const uint32_t arr_bytes = static_cast<uint32_t>(g.J * sizeof(float));
    const long long lim = wd < 0 ? -wd : wd;   // wd < 0: injected stall (stall_first_copy)

    int issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0;  // bookkeeping of thread 0 only
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](long long t, int stg) {
        const size_t j0 = static_cast<size_t>(t % g.nJT) * g.J;
        float *dst = s_tile + stg * 6 * g.J;
        mbar_arrive_expect_tx(&bars[stg], 6 * arr_bytes);
        for (int a = 0; a < 3; ++a) {
            bulk_g2s(dst + a * g.J, pos + a * static_cast<size_t>(npad) + j0, arr_bytes, &bars[stg]);
            bulk_g2s(dst + (3 + a) * g.J, frc + a * static_cast<size_t>(npad) + j0, arr_bytes, &bars[stg]);
        }
        if (stg == 0) ++issued0; else ++issued1;
    };
    if (tid == 0)
        for (int q = 0; q < 2 && t0 + q < t1; ++q)
            if (q != 0 || !stall_first_copy(wd)) issue(t0 + q, q);

    f2 XI[R], YI[R], ZI[R], AX[R], AY[R], AZ[R];
    int cur_ib = -1;
    bool aborted = false;
    const bool clamp_all = *flag != 0;

    auto flush = [&](int ib) {
        const int slot = cta - geom_first(g, ib);
        double *dst = part + static_cast<size_t>(slot) * 3 * npad;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const size_t i = static_cast<size_t>(ib) * g.I + tid + k * kNT;
            const f2 acc[3] = {AX[k], AY[k], AZ[k]};
            for (int d = 0; d < 3; ++d) {
                if constexpr (COMP) {   // the (hi, lo) pair itself, for the epilogue's FP32 TwoSum
                    const float *q = s_acc + (k * 6) * kNT + tid;
                    reinterpret_cast<float2 *>(dst)[d * static_cast<size_t>(npad) + i] =
                        make_float2(q[d * kNT], q[(3 + d) * kNT]);
                } else {
                    float lo, hi;
                    upk2(acc[d], lo, hi);
                    dst[d * static_cast<size_t>(npad) + i] = static_cast<double>(__fadd_rn(lo, hi));
                }
            }
        }
    };

    for (long long t = t0; t < t1; ++t) {
        const int ib = static_cast<int>(t / g.nJT);
        if (ib != cur_ib) {
            if (cur_ib >= 0) flush(cur_ib);
            cur_ib = ib;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const size_t i = static_cast<size_t>(ib) * g.I + tid + k * kNT;
                const float x = pos[i], y = pos[npad + i], z = pos[2 * static_cast<size_t>(npad) + i];
                XI[k] = pk2(x, x);
                YI[k] = pk2(y, y);
                ZI[k] = pk2(z, z);
                AX[k] = AY[k] = AZ[k] = 0ull;
                if constexpr (COMP)
                    for (int d = 0; d < 6; ++d) s_acc[(k * 6 + d) * kNT + tid] = 0.0f;
            }
        }
        const int q = static_cast<int>(t - t0);
        const int st = q & 1;
        if (!aborted) {
            if (mbar_wait_bounded(&bars[st], (q >> 1) & 1, lim)) {
                if (tid == 0) { if (st == 0) ++waited0; else ++waited1; }
            } else {
                atomicOr(err, DEV_ERR_TIMEOUT);
                s_abort = 1;
            }
        }
        const uint32_t base = smem_addr(s_tile + st * 6 * g.J);
        const uint32_t astride = static_cast<uint32_t>(g.J * sizeof(float));
        // r^2 is clamped to (2a)^2 only in tiles that hold self pairs, unless the
        // near pass found a pair closer than r_safe (then everywhere)
        const long long i0 = static_cast<long long>(ib) * g.I, j0 = (t % g.nJT) * static_cast<long long>(g.J);
        const bool diag = (j0 < i0 + g.I) && (i0 < j0 + g.J);
        if (clamp_all || diag || (PER && geom_pad_tile(g, c.n, i0, j0)))
            tile_pairs<TENSOR, true, R, PER>(base, astride, g.J, XI, YI, ZI, c, AX, AY, AZ);
        else
            tile_pairs<TENSOR, false, R, PER>(base, astride, g.J, XI, YI, ZI, c, AX, AY, AZ);
        if constexpr (COMP) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                float *qa = s_acc + (k * 6) * kNT + tid;
                const f2 acc[3] = {AX[k], AY[k], AZ[k]};
                for (int d = 0; d < 3; ++d) {
                    float lo, hi2;
                    upk2(acc[d], lo, hi2);
                    float h = qa[d * kNT], l = qa[(3 + d) * kNT];
                    fold2(h, l, lo);
                    fold2(h, l, hi2);
                    qa[d * kNT] = h;
                    qa[(3 + d) * kNT] = l;
                }
                AX[k] = AY[k] = AZ[k] = 0ull;
            }
        }
        __syncthreads();  // every thread is done with stage st
        aborted = s_abort != 0;
        if (tid == 0 && !aborted && t + 2 < t1) issue(t + 2, st);
    }
    flush(cur_ib);
    if (tid == 0) {
        // After a time-out, wait (bounded) for copies still in flight into this CTA's
        // shared memory before the CTA exits.
        for (int k = waited0; k < issued0; ++k)
            if (!mbar_wait_bounded(&bars[0], k & 1, drain_limit(lim))) atomicOr(err, DEV_ERR_TIMEOUT);
        for (int k = waited1; k < issued1; ++k)
            if (!mbar_wait_bounded(&bars[1], k & 1, drain_limit(lim))) atomicOr(err, DEV_ERR_TIMEOUT);
    }
}

// ---------------------------------------------------------------- FP32, symmetric

// The FP32 all-pairs kernel using mu_ij = mu_ji (Sec. 2.2).  The paper's GPU
// kernel evaluates every pair twice, once per thread of each particle (Sec. 3.2):
// on its hardware, handing a result to another thread cost global-memory traffic.
// Here the hand-off stays on chip:
//   * the particles are cut into blocks of B = 128 R (R = 2, or R = 4 for large
//     N); a tile is an unordered pair of blocks (ib <= jb), laid out row-major over
//     the upper triangle and partitioned over the persistent grid like the
//     directed kernel's plane;
//   * off-diagonal tiles: each warp holds 32 R targets of block ib (R per lane,
//     duplicated into both halves of a packed register) and walks block jb in
//     groups of 64 sources = 32 packets of two.  At step m lane l takes packet
//     (l + m) mod 32, so the 32 lanes read 32 different packets (conflict-free
//     64-bit shared loads) and each packet's running source-side sum (3 packed
//     registers) moves one lane down per step with a shuffle; after 32 steps
//     lane l holds packet l, having met all 32 R targets of the warp.  The four
//     warps' source sums are added in fixed order and written, in FP32, to the
//     tile's own slot of `jpart`; the epilogue adds a block's column of slots in
//     FP64 in ascending ib;
//   * diagonal tiles (ib == jb) hold the self pairs: they run the directed step
//     (tile_pairs, clamped) and write no source-side sums;
//   * target-side sums are kept and written exactly as in dense2_kernel (TwoSum
//     fold per tile, one slot per CTA and row).
// Per directed pair this spends 16 FP32-pipe operations instead of 22 (RP), at
// the price of one shuffle of 6 words and six 64-bit shared loads per 8 pairs.
// A pair in an off-diagonal tile is clamped iff the near pass raised the flag,
// exactly as in dense2_kernel, and each direction's FP32 term is bit-identical to
// dense2_kernel's; only the order of the sums differs.
#ifndef SD_SYM_UNROLL
#define SD_SYM_UNROLL 4
#endif
#ifndef SD_SYM_MINB
#define SD_SYM_MINB 1
#endif
constexpr int kSymUnroll = SD_SYM_UNROLL;

template <int TENSOR, bool CLAMP, bool PER, int R, int B>
__device__ __forceinline__ void sym_tile(const f2 *__restrict__ sp, int lane, const f2 (&XI)[R], const f2 (&YI)[R],
                                         const f2 (&ZI)[R], const f2 (&GX)[R], const f2 (&GY)[R], const f2 (&GZ)[R],
                                         const PairConst2 &c, f2 (&AX)[R], f2 (&AY)[R], f2 (&AZ)[R],
                                         float *__restrict__ jw) {
    constexpr int S = B / 2;   // packets per array
    const int nxt = (lane + 1) & 31;
#pragma unroll 1
    for (int g = 0; g < B / 64; ++g) {
        const f2 *gp = sp + g * 32;
        f2 JX = 0ull, JY = 0ull, JZ = 0ull;
#pragma unroll kSymUnroll
        for (int m = 0; m < 32; ++m) {
            const int p = (lane + m) & 31;
            const f2 PX = gp[p], PY = gp[S + p], PZ = gp[2 * S + p];
            const f2 FX = gp[3 * S + p], FY = gp[4 * S + p], FZ = gp[5 * S + p];
#pragma unroll
            for (int k = 0; k < R; ++k)
                pair_sym_f32x2<TENSOR, CLAMP, PER>(XI[k], YI[k], ZI[k], GX[k], GY[k], GZ[k], PX, PY, PZ, FX, FY,
                                                   FZ, c, AX[k], AY[k], AZ[k], JX, JY, JZ);
            JX = __shfl_sync(0xffffffffu, JX, nxt);
            JY = __shfl_sync(0xffffffffu, JY, nxt);
            JZ = __shfl_sync(0xffffffffu, JZ, nxt);
        }
        // lane holds packet `lane` of group g: sources 64 g + 2 lane (+1)
        f2 *jd = reinterpret_cast<f2 *>(jw) + g * 32 + lane;
        jd[0] = JX;
        jd[S] = JY;
        jd[2 * S] = JZ;
    }
}

template <int TENSOR, bool COMP, bool PER, int B, int NT>
__global__ void __launch_bounds__(NT, SD_SYM_MINB) dense_sym_kernel(const float *__restrict__ pos,
                                                           const float *__restrict__ frc, double *__restrict__ part,
                                                           float *__restrict__ jpart, int npad, DenseGeom g,
                                                           PairConst2 c, const int *__restrict__ flag,
                                                           int *__restrict__ err, long long wd, int b0) {
    constexpr int R = B / NT, NW = NT / 32;
    static_assert(B == NT * R, "a block is R targets per thread");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    float *s_tile = reinterpret_cast<float *>(smem);   // [2 stages][6 arrays][B]
    float *s_acc = s_tile + 12 * B;                     // [R][6][NT]: hx hy hz lx ly lz
    float *s_jacc = s_acc + R * 6 * NT;                 // [NW][3][B] source-side sums per warp

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = g.nIB;
    const int cta = static_cast<int>(blockIdx.x) + b0;   // index in the full launch
    const long long t0 = static_cast<long long>(cta) * g.chunk;
    const long long t1 = (t0 + g.chunk < g.nT) ? t0 + g.chunk : g.nT;
    if (t0 >= t1) return;
    constexpr uint32_t arr_bytes = B * sizeof(float);
    const long long lim = wd < 0 ? -wd : wd;   // wd < 0: injected stall (stall_first_copy)

    // (ib, jb) of tile t0: row ib starts at ib nb - ib (ib - 1) / 2
    int ib0;
    {
        const double q = 2.0 * nb + 1.0;
        ib0 = static_cast<int>(0.5 * (q - sqrt(q * q - 8.0 * static_cast<double>(t0))));
        ib0 = ib0 < 0 ? 0 : (ib0 > nb - 1 ? nb - 1 : ib0);
        while (ib0 > 0 && geom_rowstart(g, ib0) > t0) --ib0;
        while (ib0 + 1 < nb && geom_rowstart(g, ib0 + 1) <= t0) ++ib0;
    }
    const int jb0 = ib0 + static_cast<int>(t0 - geom_rowstart(g, ib0));

    int issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0;  // bookkeeping of thread 0 only
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    int qi = ib0, qj = jb0;   // next tile to stage (thread 0)
    auto issue = [&](int stg) {
        float *dst = s_tile + stg * 6 * B;
        const size_t j0 = static_cast<size_t>(qj) * B;
        mbar_arrive_expect_tx(&bars[stg], 6 * arr_bytes);
        for (int a = 0; a < 3; ++a) {
            bulk_g2s(dst + a * B, pos + a * static_cast<size_t>(npad) + j0, arr_bytes, &bars[stg]);
            bulk_g2s(dst + (3 + a) * B, frc + a * static_cast<size_t>(npad) + j0, arr_bytes, &bars[stg]);
        }
        if (stg == 0) ++issued0; else ++issued1;
        if (++qj == nb) { ++qi; qj = qi; }
    };
    if (tid == 0)
        for (int q = 0; q < 2 && t0 + q < t1; ++q) {
            if (q == 0 && stall_first_copy(wd)) {   // the tile is skipped, not staged
                if (++qj == nb) { ++qi; qj = qi; }
                continue;
            }
            issue(q);
        }

    f2 XI[R], YI[R], ZI[R], GX[R], GY[R], GZ[R], AX[R], AY[R], AZ[R];
    int cur_ib = -1;
    bool aborted = false;
    const bool clamp_all = *flag != 0;

    auto flush = [&](int ib) {
        const int slot = cta - geom_first(g, ib);
        double *dst = part + static_cast<size_t>(slot) * 3 * npad;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const size_t i = static_cast<size_t>(ib) * B + tid + k * NT;
            const f2 acc[3] = {AX[k], AY[k], AZ[k]};
            for (int d = 0; d < 3; ++d) {
                if constexpr (COMP) {   // the (hi, lo) pair itself, for the epilogue's FP32 TwoSum
                    const float *qa = s_acc + (k * 6) * NT + tid;
                    reinterpret_cast<float2 *>(dst)[d * static_cast<size_t>(npad) + i] =
                        make_float2(qa[d * NT], qa[(3 + d) * NT]);
                } else {
                    float lo, hi;
                    upk2(acc[d], lo, hi);
                    dst[d * static_cast<size_t>(npad) + i] = static_cast<double>(__fadd_rn(lo, hi));
                }
            }
        }
    };

    int ib = ib0, jb = jb0;
    for (long long t = t0; t < t1; ++t) {
        if (ib != cur_ib) {
            if (cur_ib >= 0) flush(cur_ib);
            cur_ib = ib;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const size_t i = static_cast<size_t>(ib) * B + tid + k * NT;
                const float x = pos[i], y = pos[npad + i], z = pos[2 * static_cast<size_t>(npad) + i];
                const float fx = frc[i], fy = frc[npad + i], fz = frc[2 * static_cast<size_t>(npad) + i];
                XI[k] = pk2(x, x);
                YI[k] = pk2(y, y);
                ZI[k] = pk2(z, z);
                GX[k] = pk2(fx, fx);
                GY[k] = pk2(fy, fy);
                GZ[k] = pk2(fz, fz);
                AX[k] = AY[k] = AZ[k] = 0ull;
                if constexpr (COMP)
                    for (int d = 0; d < 6; ++d) s_acc[(k * 6 + d) * NT + tid] = 0.0f;
            }
        }
        const int q = static_cast<int>(t - t0);
        const int st = q & 1;
        if (!aborted) {
            if (mbar_wait_bounded(&bars[st], (q >> 1) & 1, lim)) {
                if (tid == 0) { if (st == 0) ++waited0; else ++waited1; }
            } else {
                atomicOr(err, DEV_ERR_TIMEOUT);
                s_abort = 1;
            }
        }
        const bool diag = ib == jb;
        if (diag) {
            const uint32_t base = smem_addr(s_tile + st * 6 * B);
            tile_pairs<TENSOR, true, R, PER>(base, B * sizeof(float), B, XI, YI, ZI, c, AX, AY, AZ);
        } else {
            const f2 *sp = reinterpret_cast<const f2 *>(s_tile + st * 6 * B);
            float *jw = s_jacc + warp * 3 * B;
            const bool pad = PER && geom_pad_tile(g, c.n, static_cast<long long>(ib) * B, static_cast<long long>(jb) * B);
            if (clamp_all || pad)
                sym_tile<TENSOR, true, PER, R, B>(sp, lane, XI, YI, ZI, GX, GY, GZ, c, AX, AY, AZ, jw);
            else
                sym_tile<TENSOR, false, PER, R, B>(sp, lane, XI, YI, ZI, GX, GY, GZ, c, AX, AY, AZ, jw);
        }
        if constexpr (COMP) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                float *qa = s_acc + (k * 6) * NT + tid;
                const f2 acc[3] = {AX[k], AY[k], AZ[k]};
                for (int d = 0; d < 3; ++d) {
                    float lo, hi2;
                    upk2(acc[d], lo, hi2);
                    float h = qa[d * NT], l = qa[(3 + d) * NT];
                    fold2(h, l, lo);
                    fold2(h, l, hi2);
                    qa[d * NT] = h;
                    qa[(3 + d) * NT] = l;
                }
                AX[k] = AY[k] = AZ[k] = 0ull;
            }
        }
        __syncthreads();  // stage st consumed; every warp's source sums are in s_jacc
        if (!diag) {
            float *dst = jpart + static_cast<size_t>(t) * 3 * B;
            for (int e = tid; e < 3 * B; e += NT) {
                float v = s_jacc[e];
#pragma unroll
                for (int w = 1; w < NW; ++w) v = __fadd_rn(v, s_jacc[w * 3 * B + e]);
                dst[e] = v;
            }
            __syncthreads();  // s_jacc free for the next tile
        }
        aborted = s_abort != 0;
        if (tid == 0 && !aborted && t + 2 < t1) issue(st);
        if (++jb == nb) { ++ib; jb = ib; }
    }
    flush(cur_ib);
    if (tid == 0) {
        // After a time-out, wait (bounded) for copies still in flight into this CTA's
        // shared memory before the CTA exits.
        for (int k = waited0; k < issued0; ++k)
            if (!mbar_wait_bounded(&bars[0], k & 1, drain_limit(lim))) atomicOr(err, DEV_ERR_TIMEOUT);
        for (int k = waited1; k < issued1; ++k)
            if (!mbar_wait_bounded(&bars[1], k & 1, drain_limit(lim))) atomicOr(err, DEV_ERR_TIMEOUT);
    }
}

// ---------------------------------------------------------------- FP64, symmetric

// The FP64 all-pairs kernel using mu_ij = mu_ji (Sec. 2.2), the reference path's
// counterpart of dense_sym_kernel.  GB300 issues FP64 at a small fraction of its
// FP32 rate, so this kernel is bound by the FP64 pipe alone and its only aim is
// fewer FP64 operations per pair: r, 1/r, A and B are formed once per unordered
// pair (pair_sym_f64), 19 FP64 operations per ordered pair against 30 directed.
//   * blocks of kB64 = 128 particles, one target per thread (128 threads); a tile
//     is an unordered block pair (ib <= jb), partitioned over the persistent grid
//     as in dense_sym_kernel; the positions and forces of block jb (dbl4, AoS) are
//     staged by two bulk copies per tile, double-buffered;
//   * off-diagonal tiles: warp w holds targets 32 w .. 32 w + 31 of block ib and
//     walks block jb in groups of 32 sources; at step m lane l takes source
//     (l + m) mod 32 of the group, and the source's running sum (3 doubles) moves one
//     lane down per step by shuffle, so after 32 steps lane l holds source l.  The
//     four warps' source sums are added in fixed order into the tile's row of
//     `jpart` (FP64);
//   * diagonal tiles hold the self pairs and run the directed pair term;
//   * r^2 is clamped to (2a)^2 everywhere, as in the directed FP64 kernel, so the
//     near pass's FP64 correction applies unchanged.
constexpr int kB64 = 128;

template <int TENSOR, bool PER>
__global__ void __launch_bounds__(kB64) dense_sym64_kernel(const dbl4 *__restrict__ pos, const dbl4 *__restrict__ frc,
                                                          double *__restrict__ part, double *__restrict__ jpart,
                                                          int npad, DenseGeom g, PairConst c,
                                                          int *__restrict__ err, long long wd, int b0) {
    constexpr int B = kB64, NW = B / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    dbl4 *s_pos = reinterpret_cast<dbl4 *>(smem);            // [2 stages][B]
    dbl4 *s_frc = s_pos + 2 * B;                              // [2 stages][B]
    double *s_jacc = reinterpret_cast<double *>(s_frc + 2 * B);   // [NW][3][B]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = g.nIB;
    const int cta = static_cast<int>(blockIdx.x) + b0;   // index in the full launch
    const long long t0 = static_cast<long long>(cta) * g.chunk;
    const long long t1 = (t0 + g.chunk < g.nT) ? t0 + g.chunk : g.nT;
    if (t0 >= t1) return;
    constexpr uint32_t tile_bytes = B * sizeof(dbl4);
    const long long lim = wd < 0 ? -wd : wd;   // wd < 0: injected stall (stall_first_copy)

    int ib0;
    {
        const double q = 2.0 * nb + 1.0;
        ib0 = static_cast<int>(0.5 * (q - sqrt(q * q - 8.0 * static_cast<double>(t0))));
        ib0 = ib0 < 0 ? 0 : (ib0 > nb - 1 ? nb - 1 : ib0);
        while (ib0 > 0 && geom_rowstart(g, ib0) > t0) --ib0;
        while (ib0 + 1 < nb && geom_rowstart(g, ib0 + 1) <= t0) ++ib0;
    }
    const int jb0 = ib0 + static_cast<int>(t0 - geom_rowstart(g, ib0));

    int issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0;  // bookkeeping of thread 0 only
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    int qi = ib0, qj = jb0;   // next tile to stage (thread 0)
    auto issue = [&](int stg) {
        const size_t j0 = static_cast<size_t>(qj) * B;
        mbar_arrive_expect_tx(&bars[stg], 2 * tile_bytes);
        bulk_g2s(s_pos + stg * B, pos + j0, tile_bytes, &bars[stg]);
        bulk_g2s(s_frc + stg * B, frc + j0, tile_bytes, &bars[stg]);
        if (stg == 0) ++issued0; else ++issued1;
        if (++qj == nb) { ++qi; qj = qi; }
    };
    if (tid == 0)
        for (int q = 0; q < 2 && t0 + q < t1; ++q) {
            if (q == 0 && stall_first_copy(wd)) {   // the tile is skipped, not staged
                if (++qj == nb) { ++qi; qj = qi; }
                continue;
            }
            issue(q);
        }

    double xi = 0.0, yi = 0.0, zi = 0.0, gx = 0.0, gy = 0.0, gz = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
    int cur_ib = -1;
    bool aborted = false;
    auto flush = [&](int ib) {
        const int slot = cta - geom_first(g, ib);
        double *dst = part + static_cast<size_t>(slot) * 3 * npad + static_cast<size_t>(ib) * B + tid;
        dst[0] = ax;
        dst[npad] = ay;
        dst[2 * static_cast<size_t>(npad)] = az;
    };

    int ib = ib0, jb = jb0;
    for (long long t = t0; t < t1; ++t) {
        if (ib != cur_ib) {
            if (cur_ib >= 0) flush(cur_ib);
            cur_ib = ib;
            const dbl4 p = pos[static_cast<size_t>(ib) * B + tid], f = frc[static_cast<size_t>(ib) * B + tid];
            xi = p.x; yi = p.y; zi = p.z;
            gx = f.x; gy = f.y; gz = f.z;
            ax = ay = az = 0.0;
        }
        const int q = static_cast<int>(t - t0);
        const int st = q & 1;
        if (!aborted) {
            if (mbar_wait_bounded(&bars[st], (q >> 1) & 1, lim)) {
                if (tid == 0) { if (st == 0) ++waited0; else ++waited1; }
            } else {
                atomicOr(err, DEV_ERR_TIMEOUT);
                s_abort = 1;
            }
        }
        const dbl4 *P = s_pos + st * B;
        const dbl4 *Fq = s_frc + st * B;
        const bool diag = ib == jb;
        if (diag) {
#pragma unroll 2
            for (int jj = 0; jj < B; ++jj) pair_f64<TENSOR, PER>(xi, yi, zi, P[jj], Fq[jj], c, ax, ay, az);
        } else {
            const int nxt = (lane + 1) & 31;
#pragma unroll 1
            for (int gq = 0; gq < B / 32; ++gq) {
                double bx = 0.0, by = 0.0, bz = 0.0;
#pragma unroll 4
                for (int m = 0; m < 32; ++m) {
                    const int k = gq * 32 + ((lane + m) & 31);
                    pair_sym_f64<TENSOR, PER>(xi, yi, zi, gx, gy, gz, P[k], Fq[k], c, ax, ay, az, bx, by, bz);
                    bx = __shfl_sync(0xffffffffu, bx, nxt);
                    by = __shfl_sync(0xffffffffu, by, nxt);
                    bz = __shfl_sync(0xffffffffu, bz, nxt);
                }
                double *jw = s_jacc + warp * 3 * B + gq * 32 + lane;   // source 32 gq + lane
                jw[0] = bx;
                jw[B] = by;
                jw[2 * B] = bz;
            }
        }
        __syncthreads();  // stage st consumed; every warp's source sums are in s_jacc
        if (!diag) {
            double *dst = jpart + static_cast<size_t>(t) * 3 * B;
            for (int e = tid; e < 3 * B; e += B) {
                double v = s_jacc[e];
#pragma unroll
                for (int w = 1; w < NW; ++w) v += s_jacc[w * 3 * B + e];
                dst[e] = v;
            }
            __syncthreads();  // s_jacc free for the next tile
        }
        aborted = s_abort != 0;
        if (tid == 0 && !aborted && t + 2 < t1) issue(st);
        if (++jb == nb) { ++ib; jb = ib; }
    }
    flush(cur_ib);
    if (tid == 0) {
        // After a time-out, wait (bounded) for copies still in flight into this CTA's
        // shared memory before the CTA exits.
        for (int k = waited0; k < issued0; ++k)
            if (!mbar_wait_bounded(&bars[0], k & 1, drain_limit(lim))) atomicOr(err, DEV_ERR_TIMEOUT);
        for (int k = waited1; k < issued1; ++k)
            if (!mbar_wait_bounded(&bars[1], k & 1, drain_limit(lim))) atomicOr(err, DEV_ERR_TIMEOUT);
    }
}

constexpr size_t sym64_smem() {
    return 4 * static_cast<size_t>(kB64) * sizeof(dbl4) + (kB64 / 32) * 3 * static_cast<size_t>(kB64) * sizeof(double);
}

// ---------------------------------------------------------------- dispatch

template <bool PER>
static void *pick_dense_t(int tensor, int mode) {
    const bool oseen = tensor == T_OSEEN;
    switch (mode) {
        case MODE_FP32C:
            return oseen ? reinterpret_cast<void *>(&dense2_kernel<T_OSEEN, true, PER>)
                         : reinterpret_cast<void *>(&dense2_kernel<T_RP, true, PER>);
        case MODE_FP64:
            return oseen ? reinterpret_cast<void *>(&dense_kernel<T_OSEEN, MODE_FP64, PER>)
                         : reinterpret_cast<void *>(&dense_kernel<T_RP, MODE_FP64, PER>);
        default:
            return oseen ? reinterpret_cast<void *>(&dense2_kernel<T_OSEEN, false, PER>)
                         : reinterpret_cast<void *>(&dense2_kernel<T_RP, false, PER>);
    }
}
static void *pick_dense(int tensor, int mode, bool per) {
    return per ? pick_dense_t<true>(tensor, mode) : pick_dense_t<false>(tensor, mode);
}

template <bool PER, int B, int NT>
static void *pick_sym_t(int tensor, int mode) {
    const bool oseen = tensor == T_OSEEN, comp = mode == MODE_FP32C;
    if (oseen)
        return comp ? reinterpret_cast<void *>(&dense_sym_kernel<T_OSEEN, true, PER, B, NT>)
                    : reinterpret_cast<void *>(&dense_sym_kernel<T_OSEEN, false, PER, B, NT>);
    return comp ? reinterpret_cast<void *>(&dense_sym_kernel<T_RP, true, PER, B, NT>)
                : reinterpret_cast<void *>(&dense_sym_kernel<T_RP, false, PER, B, NT>);
}
template <bool PER>
static void *pick_sym_p(int tensor, int mode, int B, int NT) {
    if (B == 512) return pick_sym_t<PER, 512, 128>(tensor, mode);
    if (B == 128) return pick_sym_t<PER, 128, 64>(tensor, mode);
    if (NT == 64) return pick_sym_t<PER, 256, 64>(tensor, mode);
    return pick_sym_t<PER, 256, 128>(tensor, mode);
}
static void *pick_sym(int tensor, int mode, bool per, int B, int NT) {
    return per ? pick_sym_p<true>(tensor, mode, B, NT) : pick_sym_p<false>(tensor, mode, B, NT);
}

// Dynamic shared memory of the dense kernel of this mode for tile J.
static size_t dense_smem(int mode, int J) {
    if (mode == MODE_FP64) return 4 * static_cast<size_t>(J) * sizeof(dbl4);
    return 12 * static_cast<size_t>(J) * sizeof(float) + static_cast<size_t>(kR32) * 6 * kNT * sizeof(float);
}
// Dynamic shared memory of the symmetric kernel for blocks of B: two stages of six
// source arrays, the (hi, lo) target accumulators, the warps' source-side sums.
static constexpr size_t sym_smem(int B, int NT) {
    return (12 * static_cast<size_t>(B) + static_cast<size_t>(B / NT) * 6 * NT +
            static_cast<size_t>(NT / 32) * 3 * static_cast<size_t>(B)) * sizeof(float);
}

// The symmetric kernel replaces the directed FP32 kernel once the triangle holds at
// least one tile per SD_DENSE_SYM_SMS_PER_TILE SMs.  Measured on GB300 (step time,
// N = 2^k at volume fraction 0.05): directed faster at N <= 2048 (36 tiles),
// symmetric faster from N = 4096 (136 tiles) on.  From SD_DENSE_SYM_LARGE_N
// particles on, blocks of 512 (4 targets per thread: more independent work per
// warp, half the source-side partial rows) replace blocks of 256: all-pairs kernel
// 2.29 -> 2.23 ms at N = 65,536 and 36.3 -> 34.2 ms at 262,144, but 0.159 -> 0.170
// ms at 16,384 (too few tiles for 2 CTAs per SM of 174 registers).
#ifndef SD_DENSE_SYM_SMS_PER_TILE
#define SD_DENSE_SYM_SMS_PER_TILE 2
#endif
#ifndef SD_DENSE_SYM_LARGE_N
#define SD_DENSE_SYM_LARGE_N 32768
#endif
// Below SD_DENSE_SYM_LARGE_N and from SD_DENSE_SYM_MID_N on, blocks of 256 go to
// 64-thread CTAs (4 targets per thread): 0.159 -> 0.151 ms at N = 16,384 and
// 0.053 -> 0.050 ms at 8,192; at 4,096 they leave too few CTAs (0.020 -> 0.030).
#ifndef SD_DENSE_SYM_MID_N
#define SD_DENSE_SYM_MID_N 8192
#endif
// Below SD_DENSE_SYM_SMALL_N, blocks of 128 particles in 64-thread CTAs (2 targets
// per thread): four times the tiles of 256-blocks, so a small system still spreads
// over every SM.
#ifndef SD_DENSE_SYM_SMALL_N
#define SD_DENSE_SYM_SMALL_N 8192
#endif
// CTA oversubscription of the symmetric kernel's grid (see SD_DENSE_CTA_SCALE): runs
// of ceil(tiles / (SD_DENSE_SYM_CTA_SCALE x resident CTAs)) tiles, or one tile per CTA
// while the tiles number at most SD_DENSE_SYM_ONE_TILE x the resident CTAs.  Measured
// all-pairs kernel (blocks of 512, 2 CTAs per SM):
//   N = 65,536 (8,256 tiles): one tile per CTA 2.179 ms, runs of 2 (16x) 2.209 ms;
//   N = 131,072: runs of 7 (16x) 8.571 ms, runs of 4 (32x) 8.646 ms;
//   N = 262,144: runs of 27 (16x) 34.07 ms, runs of 14 (32x) 34.19 ms.
// Longer runs write fewer target-side partial rows; at N = 65,536 the shorter work
// units balance the SMs better.
#ifndef SD_DENSE_SYM_CTA_SCALE
#define SD_DENSE_SYM_CTA_SCALE 16
#endif
#ifndef SD_DENSE_SYM_ONE_TILE
#define SD_DENSE_SYM_ONE_TILE 32
#endif
static long long sym_chunk(long long nT, long long resident) {
    if (nT <= resident * SD_DENSE_SYM_ONE_TILE) return 1;
    const long long want = resident * SD_DENSE_SYM_CTA_SCALE;
    return (nT + want - 1) / want;
}

// Choose the tile J and the persistent grid for h->npad, and size the partials.
cudaError_t dense_setup(sd_handle *h) {
    const int R = (h->mode == MODE_FP64) ? kR64 : kR32;
    DenseGeom g{};
    g.I = kNT * R;
    // Blocks and tiles cover the n particles, not the padded arrays (the slots past n
    // hold far-away particles with zero force, so a partly filled block or tile is
    // harmless): at small n the padding would otherwise be most of the work, which
    // matters in FP64 (GB300 issues FP64 at 1/64 the FP32 rate).
    const int nreal = std::max(h->n, 1);
    g.nIB = (nreal + g.I - 1) / g.I;
    void *fn = pick_dense(h->tensor, h->mode, h->pc.periodic != 0);
    const int Jcand[4] = {kJmax, 128, 64, 32};
    int occ = 0;
    for (int ci = 0; ci < 4; ++ci) {
        const int J = Jcand[ci];
        if (h->mode == MODE_FP64 && J > 128) continue;
        if (h->mode != MODE_FP64 && J < 64) continue;   // (32-source tiles: FP64 only)
        const size_t smem = dense_smem(h->mode, J);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kNT, smem);
        if (e != cudaSuccess) return e;
        g.J = J;
        g.nJT = (nreal + J - 1) / J;
        const long long T = static_cast<long long>(g.nIB) * g.nJT;
        if (T >= 4LL * h->num_sms * std::max(occ, 1)) break;
    }
    occ = std::max(occ, 1);
    const long long T = static_cast<long long>(g.nIB) * g.nJT;
// The grid holds SD_DENSE_CTA_SCALE times as many CTAs as fit at once: the
// hardware block scheduler then balances uneven per-SM progress (measured on
// GB300: 58% -> 60% of the FP32 peak going from 1 to 8).
#ifndef SD_DENSE_CTA_SCALE
#define SD_DENSE_CTA_SCALE 8
#endif
    const long long want = static_cast<long long>(h->num_sms) * occ * SD_DENSE_CTA_SCALE;
    g.chunk = (T + want - 1) / want;
    if (g.chunk < 1) g.chunk = 1;
    g.grid = static_cast<int>((T + g.chunk - 1) / g.chunk);
    g.nT = T;
    g.sym = 0;
    const int want_sym = h->cfg.dense_kernel;
    // block shape: 512 particles x 128 threads (4 targets each) for large N, 256 x 64
    // (4 each) for mid-size N, 256 x 128 (2 each) below
    const bool large = h->npad >= SD_DENSE_SYM_LARGE_N && h->npad % 512 == 0;
    const bool small = h->npad < SD_DENSE_SYM_SMALL_N;
    const int B = large ? 512 : (small ? 128 : 256);
    const int NT = large ? 128 : (small ? 64 : (h->npad < SD_DENSE_SYM_MID_N ? 128 : 64));
    if (h->mode == MODE_FP64 && want_sym != SD_DENSE_DIRECTED) {
        void *sfn = h->tensor == T_OSEEN ? (h->pc.periodic ? reinterpret_cast<void *>(&dense_sym64_kernel<T_OSEEN, true>)
                                                           : reinterpret_cast<void *>(&dense_sym64_kernel<T_OSEEN, false>))
                                         : (h->pc.periodic ? reinterpret_cast<void *>(&dense_sym64_kernel<T_RP, true>)
                                                           : reinterpret_cast<void *>(&dense_sym64_kernel<T_RP, false>));
        cudaError_t e = cudaFuncSetAttribute(sfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(sym64_smem()));
        if (e != cudaSuccess) return e;
        int socc = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&socc, sfn, kB64, sym64_smem());
        if (e != cudaSuccess) return e;
        socc = std::max(socc, 1);
        DenseGeom s{};
        s.sym = 1;
        s.I = s.J = kB64;
        s.nIB = s.nJT = (nreal + kB64 - 1) / kB64;
        s.nT = static_cast<long long>(s.nIB) * (s.nIB + 1) / 2;
        if (want_sym == SD_DENSE_SYMMETRIC || s.nT * SD_DENSE_SYM_SMS_PER_TILE >= h->num_sms) {
            s.chunk = sym_chunk(s.nT, static_cast<long long>(h->num_sms) * socc);
            s.grid = static_cast<int>((s.nT + s.chunk - 1) / s.chunk);
            g = s;
            occ = socc;
            h->sym_nt = kB64;
        }
    }
    if (h->mode != MODE_FP64 && h->npad % B == 0 && want_sym != SD_DENSE_DIRECTED) {
        void *sfn = pick_sym(h->tensor, h->mode, h->pc.periodic != 0, B, NT);
        cudaError_t e = cudaFuncSetAttribute(sfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(sym_smem(B, NT)));
        if (e != cudaSuccess) return e;
        int socc = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&socc, sfn, NT, sym_smem(B, NT));
        if (e != cudaSuccess) return e;
        socc = std::max(socc, 1);
        DenseGeom s{};
        s.sym = 1;
        s.I = s.J = B;
        s.nIB = s.nJT = (nreal + B - 1) / B;
        s.nT = static_cast<long long>(s.nIB) * (s.nIB + 1) / 2;
        // (blocks of 128: four times as many, and smaller, tiles are needed to beat the
        // directed kernel: measured directed faster at n = 2048, symmetric at 4096)
        const long long need = static_cast<long long>(h->num_sms) * (B == 128 ? 4 : 1);
        if (want_sym == SD_DENSE_SYMMETRIC || s.nT * SD_DENSE_SYM_SMS_PER_TILE >= need) {
            s.chunk = sym_chunk(s.nT, static_cast<long long>(h->num_sms) * socc);
            s.grid = static_cast<int>((s.nT + s.chunk - 1) / s.chunk);
            g = s;
            occ = socc;
            h->sym_nt = NT;
        }
    }
    int ms = 0;
    for (int ib = 0; ib < g.nIB; ++ib) ms = std::max(ms, geom_last(g, ib) - geom_first(g, ib) + 1);
    g.maxSlots = ms;
    h->geom = g;
    h->dense_occ = occ;
    return cudaSuccess;
}

// The watchdog limit the all-pairs kernels get: negated while a stall is injected.
static long long dense_wd(const sd_handle *h) { return h->inject_stall ? -h->watchdog : h->watchdog; }

template <bool PER>
static void launch_dense_t(sd_handle *h, cudaStream_t st, Mirror posm, Mirror frcm, double *part, const TileWin &w,
                           int grid) {
    const DenseGeom &g = h->geom;
    const size_t smem = dense_smem(h->mode, g.J);
    const bool oseen = h->tensor == T_OSEEN;
    if (h->mode == MODE_FP64) {
        const dbl4 *p = static_cast<const dbl4 *>(posm.aos), *f = static_cast<const dbl4 *>(frcm.aos);
        if (g.sym) {
            double *jp = static_cast<double *>(h->jpart);
            if (oseen)
                dense_sym64_kernel<T_OSEEN, PER><<<grid, kB64, sym64_smem(), st>>>(p, f, part, jp, h->npad, g, h->pc,
                                                                                 h->d_err, dense_wd(h), w.b0);
            else
                dense_sym64_kernel<T_RP, PER><<<grid, kB64, sym64_smem(), st>>>(p, f, part, jp, h->npad, g, h->pc,
                                                                              h->d_err, dense_wd(h), w.b0);
            return;
        }
        if (oseen)
            dense_kernel<T_OSEEN, MODE_FP64, PER><<<grid, kNT, smem, st>>>(p, f, part, h->npad, g, h->pc,
                                                                            h->d_err, dense_wd(h), w);
        else
            dense_kernel<T_RP, MODE_FP64, PER><<<grid, kNT, smem, st>>>(p, f, part, h->npad, g, h->pc, h->d_err,
                                                                         dense_wd(h), w);
        return;
    }
    PairConst2 c2{};
    c2.c1 = pk2_host(h->pc.c1_f);
    c2.c3 = pk2_host(h->pc.c3_f);
    c2.m3c3 = pk2_host(h->pc.m3c3_f);
    c2.r2min = h->pc.r2min_f;
    for (int d = 0; d < 3; ++d) {
        c2.negL[d] = pk2_host(-h->pc.Lf[d]);
        c2.invL[d] = pk2_host(h->pc.invLf[d]);
    }
    c2.n = h->n;
    const bool comp = h->mode == MODE_FP32C;
    if (g.sym) {
#define SD_DS(TT, CC, BB, NN)                                                                                  \
    dense_sym_kernel<TT, CC, PER, BB, NN><<<grid, NN, sym_smem(BB, NN), st>>>(posm.soa, frcm.soa, part,       \
                                                                              static_cast<float *>(h->jpart), h->npad, \
                                                                              g, c2, h->d_flag, h->d_err, dense_wd(h), \
                                                                              w.b0)
#define SD_DS_SHAPE(BB, NN)                                                                                    \
    if (oseen) {                                                                                               \
        if (comp) SD_DS(T_OSEEN, true, BB, NN); else SD_DS(T_OSEEN, false, BB, NN);                            \
    } else {                                                                                                   \
        if (comp) SD_DS(T_RP, true, BB, NN); else SD_DS(T_RP, false, BB, NN);                                  \
    }
        if (g.I == 512) {
            SD_DS_SHAPE(512, 128)
        } else if (g.I == 128) {
            SD_DS_SHAPE(128, 64)
        } else if (h->sym_nt == 64) {
            SD_DS_SHAPE(256, 64)
        } else {
            SD_DS_SHAPE(256, 128)
        }
#undef SD_DS_SHAPE
#undef SD_DS
        return;
    }
#define SD_D2(TT, CC)                                                                                          \
    dense2_kernel<TT, CC, PER><<<grid, kNT, smem, st>>>(posm.soa, frcm.soa, part, h->npad, g, c2, h->d_flag, \
                                                        h->d_err, dense_wd(h), w)
    if (oseen) {
        if (comp) SD_D2(T_OSEEN, true); else SD_D2(T_OSEEN, false);
    } else {
        if (comp) SD_D2(T_RP, true); else SD_D2(T_RP, false);
    }
#undef SD_D2
}

cudaError_t launch_dense(sd_handle *h, cudaStream_t st, Mirror posm, Mirror frcm, double *part,
                         const TileWin *win) {
    const DenseGeom &g = h->geom;
    TileWin w{};
    int grid = g.grid;
    if (win) {   // a window of tiles: the CTAs of the full launch touching it
        w = *win;
        const long long T = g.nT;
        const long long hi = (w.hi >= 0 && w.hi < T) ? w.hi : T;
        if (w.lo >= hi) return cudaSuccess;
        w.b0 = static_cast<int>(w.lo / g.chunk);
        grid = static_cast<int>((hi - 1) / g.chunk) - w.b0 + 1;
        // the symmetric kernels take whole CTAs of the full launch only
        if (g.sym && (w.lo != w.b0 * g.chunk || (hi != T && hi % g.chunk != 0))) return cudaErrorInvalidValue;
    }
    prof_begin(h, SD_KERNEL_DENSE, st);
    if (h->pc.periodic)
        launch_dense_t<true>(h, st, posm, frcm, part, w, grid);
    else
        launch_dense_t<false>(h, st, posm, frcm, part, w, grid);
    prof_end(h, SD_KERNEL_DENSE, st);
    ++h->launches;
    return cudaGetLastError();
}

}  // namespace sd
