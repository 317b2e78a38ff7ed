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
//   * each CTA writes its partial sum for every i-block it touched into a fixed slot;
//     the epilogue adds the slots in ascending order (deterministic result).
// Self and overlapping pairs take r^2 clamped to (2a)^2 here; the FP64 epilogue
// replaces them (and every pair closer than r_near) by their exact terms.
#include <algorithm>
#include "sd_internal.h"

namespace sd {

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

template <int TENSOR, int MODE>
__device__ __forceinline__ void dense_pair(typename DenseT<MODE>::S xi, typename DenseT<MODE>::S yi,
                                           typename DenseT<MODE>::S zi, const typename DenseT<MODE>::V4 &p,
                                           const typename DenseT<MODE>::V4 &f, const PairConst &c,
                                           typename DenseT<MODE>::S &ax, typename DenseT<MODE>::S &ay,
                                           typename DenseT<MODE>::S &az) {
    if constexpr (MODE == MODE_FP64)
        pair_f64<TENSOR>(xi, yi, zi, p, f, c, ax, ay, az);
    else
        pair_f32<TENSOR>(xi, yi, zi, p, f, c, ax, ay, az);
}

template <int TENSOR, int MODE>
__global__ void __launch_bounds__(kNT) dense_kernel(const typename DenseT<MODE>::V4 *__restrict__ pos,
                                                    const typename DenseT<MODE>::V4 *__restrict__ frc,
                                                    double *__restrict__ part, int npad, DenseGeom g, PairConst c,
                                                    int *__restrict__ err, long long wd) {
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
    const long long t0 = static_cast<long long>(blockIdx.x) * g.chunk;
    const long long t1 = (t0 + g.chunk < T) ? t0 + g.chunk : T;
    if (t0 >= t1) return;  // uniform over the CTA
    const uint32_t tile_bytes = static_cast<uint32_t>(g.J * sizeof(V4));

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
        const int slot = static_cast<int>(blockIdx.x) - geom_first(g, ib);
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
            if (mbar_wait_bounded(&bars[st], (q >> 1) & 1, wd)) {
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
            for (int k = 0; k < R; ++k) dense_pair<TENSOR, MODE>(xi[k], yi[k], zi[k], p, f, c, ax[k], ay[k], az[k]);
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
            if (!mbar_wait_bounded(&bars[0], k & 1, drain_limit(wd))) atomicOr(err, DEV_ERR_TIMEOUT);
        for (int k = waited1; k < issued1; ++k)
            if (!mbar_wait_bounded(&bars[1], k & 1, drain_limit(wd))) atomicOr(err, DEV_ERR_TIMEOUT);
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
template <int TENSOR, bool CLAMP, int R>
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
                pair_f32x2<TENSOR, CLAMP>(XI[k], YI[k], ZI[k], P[0][h2], P[1][h2], P[2][h2], P[3][h2], P[4][h2],
                                          P[5][h2], c, AX[k], AY[k], AZ[k]);
    }
}

template <int TENSOR, bool COMP>
__global__ void __launch_bounds__(kNT) dense2_kernel(const float *__restrict__ pos, const float *__restrict__ frc,
                                                     double *__restrict__ part, int npad, DenseGeom g, PairConst2 c,
                                                     const int *__restrict__ flag, int *__restrict__ err,
                                                     long long wd) {
    constexpr int R = kR32;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    float *s_tile = reinterpret_cast<float *>(smem);          // [2 stages][6 arrays][J]
    float *s_acc = s_tile + 12 * g.J;                          // [R][6][kNT]: hx hy hz lx ly lz

    const int tid = threadIdx.x;
    const long long T = static_cast<long long>(g.nIB) * g.nJT;
    const long long t0 = static_cast<long long>(blockIdx.x) * g.chunk;
    const long long t1 = (t0 + g.chunk < T) ? t0 + g.chunk : T;
    if (t0 >= t1) return;
    const uint32_t arr_bytes = static_cast<uint32_t>(g.J * sizeof(float));

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
        for (int q = 0; q < 2 && t0 + q < t1; ++q) issue(t0 + q, q);

    f2 XI[R], YI[R], ZI[R], AX[R], AY[R], AZ[R];
    int cur_ib = -1;
    bool aborted = false;
    const bool clamp_all = *flag != 0;

    auto flush = [&](int ib) {
        const int slot = static_cast<int>(blockIdx.x) - geom_first(g, ib);
        double *dst = part + static_cast<size_t>(slot) * 3 * npad;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const size_t i = static_cast<size_t>(ib) * g.I + tid + k * kNT;
            const f2 acc[3] = {AX[k], AY[k], AZ[k]};
            for (int d = 0; d < 3; ++d) {
                double v;
                if constexpr (COMP) {
                    const float *q = s_acc + (k * 6) * kNT + tid;
                    v = static_cast<double>(q[d * kNT]) + static_cast<double>(q[(3 + d) * kNT]);
                } else {
                    float lo, hi;
                    upk2(acc[d], lo, hi);
                    v = static_cast<double>(__fadd_rn(lo, hi));
                }
                dst[d * static_cast<size_t>(npad) + i] = v;
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
            if (mbar_wait_bounded(&bars[st], (q >> 1) & 1, wd)) {
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
        if (clamp_all || diag)
            tile_pairs<TENSOR, true, R>(base, astride, g.J, XI, YI, ZI, c, AX, AY, AZ);
        else
            tile_pairs<TENSOR, false, R>(base, astride, g.J, XI, YI, ZI, c, AX, AY, AZ);
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
            if (!mbar_wait_bounded(&bars[0], k & 1, drain_limit(wd))) atomicOr(err, DEV_ERR_TIMEOUT);
        for (int k = waited1; k < issued1; ++k)
            if (!mbar_wait_bounded(&bars[1], k & 1, drain_limit(wd))) atomicOr(err, DEV_ERR_TIMEOUT);
    }
}

// ---------------------------------------------------------------- dispatch

static void *pick_dense(int tensor, int mode) {
    const bool oseen = tensor == T_OSEEN;
    switch (mode) {
        case MODE_FP32C:
            return oseen ? reinterpret_cast<void *>(&dense2_kernel<T_OSEEN, true>)
                         : reinterpret_cast<void *>(&dense2_kernel<T_RP, true>);
        case MODE_FP64:
            return oseen ? reinterpret_cast<void *>(&dense_kernel<T_OSEEN, MODE_FP64>)
                         : reinterpret_cast<void *>(&dense_kernel<T_RP, MODE_FP64>);
        default:
            return oseen ? reinterpret_cast<void *>(&dense2_kernel<T_OSEEN, false>)
                         : reinterpret_cast<void *>(&dense2_kernel<T_RP, false>);
    }
}

// Dynamic shared memory of the dense kernel of this mode for tile J.
static size_t dense_smem(int mode, int J) {
    if (mode == MODE_FP64) return 4 * static_cast<size_t>(J) * sizeof(dbl4);
    return 12 * static_cast<size_t>(J) * sizeof(float) + static_cast<size_t>(kR32) * 6 * kNT * sizeof(float);
}

// Choose the tile J and the persistent grid for h->npad, and size the partials.
cudaError_t dense_setup(sd_handle *h) {
    const int R = (h->mode == MODE_FP64) ? kR64 : kR32;
    DenseGeom g{};
    g.I = kNT * R;
    g.nIB = h->npad / g.I;
    void *fn = pick_dense(h->tensor, h->mode);
    const int Jcand[3] = {kJmax, 128, 64};
    int occ = 0;
    for (int ci = 0; ci < 3; ++ci) {
        const int J = Jcand[ci];
        if (h->mode == MODE_FP64 && J > 128) continue;
        const size_t smem = dense_smem(h->mode, J);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kNT, smem);
        if (e != cudaSuccess) return e;
        g.J = J;
        g.nJT = h->npad / J;
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
    int ms = 0;
    for (int ib = 0; ib < g.nIB; ++ib) ms = std::max(ms, geom_last(g, ib) - geom_first(g, ib) + 1);
    g.maxSlots = ms;
    h->geom = g;
    h->dense_occ = occ;
    return cudaSuccess;
}

cudaError_t launch_dense(sd_handle *h, cudaStream_t st, Mirror posm, Mirror frcm, double *part) {
    const DenseGeom &g = h->geom;
    const size_t smem = dense_smem(h->mode, g.J);
    const bool oseen = h->tensor == T_OSEEN;
    prof_begin(h, SD_KERNEL_DENSE, st);
    if (h->mode == MODE_FP64) {
        const dbl4 *p = static_cast<const dbl4 *>(posm.aos), *f = static_cast<const dbl4 *>(frcm.aos);
        if (oseen)
            dense_kernel<T_OSEEN, MODE_FP64><<<g.grid, kNT, smem, st>>>(p, f, part, h->npad, g, h->pc, h->d_err,
                                                                         h->watchdog);
        else
            dense_kernel<T_RP, MODE_FP64><<<g.grid, kNT, smem, st>>>(p, f, part, h->npad, g, h->pc, h->d_err,
                                                                      h->watchdog);
    } else {
        PairConst2 c2;
        c2.c1 = pk2_host(h->pc.c1_f);
        c2.c3 = pk2_host(h->pc.c3_f);
        c2.m3c3 = pk2_host(h->pc.m3c3_f);
        c2.r2min = h->pc.r2min_f;
        const bool comp = h->mode == MODE_FP32C;
#define SD_D2(TT, CC) \
    dense2_kernel<TT, CC><<<g.grid, kNT, smem, st>>>(posm.soa, frcm.soa, part, h->npad, g, c2, h->d_flag, h->d_err, \
                                                     h->watchdog)
        if (oseen) {
            if (comp) SD_D2(T_OSEEN, true); else SD_D2(T_OSEEN, false);
        } else {
            if (comp) SD_D2(T_RP, true); else SD_D2(T_RP, false);
        }
#undef SD_D2
    }
    prof_end(h, SD_KERNEL_DENSE, st);
    ++h->launches;
    return cudaGetLastError();
}

}  // namespace sd
