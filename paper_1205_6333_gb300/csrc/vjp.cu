// vjp.cu -- vector-Jacobian products of v(x, F) = mu(x) F (derivative of
// Sec. 2.2, Eq. rotneMobility; the paper has no adjoint):
//
//   (mu W)_i  = mu0 [ W_i + sum_{j != i} (A W_j + B (r.W_j) r) ]
//   gX_i      = mu0 sum_{j != i} grad_r [ W_i.T^(r) F_j + W_j.T^(r) F_i ],  r = x_i - x_j
//
// with T^ = T/mu0 = A I + B r r^T (pair.cuh).  mu is symmetric, so mu^T W = mu W
// is the force gradient.  One all-pairs kernel evaluates both sums from the same
// r, 1/r and tensor profile; the layout is the dense kernel's (persistent grid,
// bulk-copied j-tiles of positions, forces and cotangents, per-tile TwoSum folds,
// fixed-order slots), and the epilogue again swaps the self term and the pairs
// closer than r_near for their exact FP64 values.
#include <algorithm>
#include "neighbours.cuh"

namespace sd {

template <int MODE>
struct VjpT {
    using V4 = float4;
    using V3 = float3;
    using S = float;
};
template <>
struct VjpT<MODE_FP64> {
    using V4 = dbl4;
    using V3 = double3;
    using S = double;
};

template <int TENSOR, int MODE, bool PER>
__device__ __forceinline__ void vjp_term(typename VjpT<MODE>::S xi, typename VjpT<MODE>::S yi,
                                         typename VjpT<MODE>::S zi, const typename VjpT<MODE>::V3 &Fi,
                                         const typename VjpT<MODE>::V3 &Wi, const typename VjpT<MODE>::V4 &p,
                                         const typename VjpT<MODE>::V4 &f, const typename VjpT<MODE>::V4 &w,
                                         const PairConst &c, typename VjpT<MODE>::V3 &m,
                                         typename VjpT<MODE>::V3 &g) {
    if constexpr (MODE == MODE_FP64)
        vjp_pair_f64<TENSOR, PER>(xi, yi, zi, Fi, Wi, p, f, w, c, m, g);
    else
        vjp_pair_f32<TENSOR, PER>(xi, yi, zi, Fi, Wi, p, f, w, c, m, g);
}

// The FP64 VJP kernel (the FP32C path runs vjp2_kernel below): plain FP64 sums.
template <int TENSOR, int MODE, bool PER>
__global__ void __launch_bounds__(kNT) vjp_kernel(const typename VjpT<MODE>::V4 *__restrict__ pos,
                                                  const typename VjpT<MODE>::V4 *__restrict__ frc,
                                                  const typename VjpT<MODE>::V4 *__restrict__ wv,
                                                  double *__restrict__ partM, double *__restrict__ partG, int npad,
                                                  DenseGeom g, PairConst c, int *__restrict__ err, long long wd) {
    using V4 = typename VjpT<MODE>::V4;
    using V3 = typename VjpT<MODE>::V3;
    using S = typename VjpT<MODE>::S;
    constexpr int R = kRV;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    V4 *s_pos = reinterpret_cast<V4 *>(smem);
    V4 *s_frc = s_pos + 2 * g.J;
    V4 *s_w = s_frc + 2 * g.J;

    const int tid = threadIdx.x;
    const long long T = static_cast<long long>(g.nIB) * g.nJT;
    const long long t0 = static_cast<long long>(blockIdx.x) * g.chunk;
    const long long t1 = (t0 + g.chunk < T) ? t0 + g.chunk : T;
    if (t0 >= t1) return;
    const uint32_t tile_bytes = static_cast<uint32_t>(g.J * sizeof(V4));

    int issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](long long t, int stg) {
        const size_t jt = static_cast<size_t>(t % g.nJT);
        mbar_arrive_expect_tx(&bars[stg], 3 * tile_bytes);
        bulk_g2s(s_pos + stg * g.J, pos + jt * g.J, tile_bytes, &bars[stg]);
        bulk_g2s(s_frc + stg * g.J, frc + jt * g.J, tile_bytes, &bars[stg]);
        bulk_g2s(s_w + stg * g.J, wv + jt * g.J, tile_bytes, &bars[stg]);
        if (stg == 0) ++issued0; else ++issued1;
    };
    if (tid == 0)
        for (int q = 0; q < 2 && t0 + q < t1; ++q) issue(t0 + q, q);

    S xi[R], yi[R], zi[R];
    V3 Fi[R], Wi[R], m[R], gg[R];
    int cur_ib = -1;
    bool aborted = false;

    auto flush = [&](int ib) {
        const int slot = static_cast<int>(blockIdx.x) - geom_first(g, ib);
        double *dM = partM + static_cast<size_t>(slot) * 3 * npad;
        double *dG = partG + static_cast<size_t>(slot) * 3 * npad;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const size_t i = static_cast<size_t>(ib) * g.I + tid + k * kNT;
            dM[i] = m[k].x;
            dM[npad + i] = m[k].y;
            dM[2 * static_cast<size_t>(npad) + i] = m[k].z;
            dG[i] = gg[k].x;
            dG[npad + i] = gg[k].y;
            dG[2 * static_cast<size_t>(npad) + i] = gg[k].z;
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
                const V4 p = pos[i], f = frc[i], w = wv[i];
                xi[k] = p.x;
                yi[k] = p.y;
                zi[k] = p.z;
                Fi[k].x = f.x; Fi[k].y = f.y; Fi[k].z = f.z;
                Wi[k].x = w.x; Wi[k].y = w.y; Wi[k].z = w.z;
                m[k].x = m[k].y = m[k].z = S(0);
                gg[k].x = gg[k].y = gg[k].z = S(0);
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
        const V4 *Wq = s_w + st * g.J;
        for (int jj = 0; jj < g.J; ++jj) {
            const V4 p = P[jj], f = Fq[jj], w = Wq[jj];
#pragma unroll
            for (int k = 0; k < R; ++k)
                vjp_term<TENSOR, MODE, PER>(xi[k], yi[k], zi[k], Fi[k], Wi[k], p, f, w, c, m[k], gg[k]);
        }
        __syncthreads();
        aborted = s_abort != 0;
        if (tid == 0 && !aborted && t + 2 < t1) issue(t + 2, st);
    }
    flush(cur_ib);
    if (tid == 0) {
        for (int k = waited0; k < issued0; ++k)
            if (!mbar_wait_bounded(&bars[0], k & 1, drain_limit(wd))) atomicOr(err, DEV_ERR_TIMEOUT);
        for (int k = waited1; k < issued1; ++k)
            if (!mbar_wait_bounded(&bars[1], k & 1, drain_limit(wd))) atomicOr(err, DEV_ERR_TIMEOUT);
    }
}

// FP32C: the same sums with the pair terms packed over pairs of sources.  The j-tiles
// are staged as nine float arrays (x, y, z, Fx, Fy, Fz, Wx, Wy, Wz: nine bulk copies),
// so two consecutive j's form one 64-bit operand and every instruction of
// vjp_pair_f32x2 evaluates (i, j) and (i, j + 1): half the issued instructions of the
// scalar loop (N = 4,096: 45 us against 48).  Each thread owns R targets, duplicated
// into both lanes; its packed
// accumulators sum even and odd j's separately, and both lanes are folded into (hi, lo)
// TwoSum accumulators in shared memory after every tile.  Slots are (hi, lo) float
// pairs, as the FP32C epilogue reads them.
// Targets per thread of the packed FP32C VJP kernel.  One keeps it at about 120
// registers (4 CTAs per SM); two took 140 and were slower at N = 4,096 (50 against 45 us).
#ifndef SD_VJP2_R
#define SD_VJP2_R 1
#endif
constexpr int kRV2 = SD_VJP2_R;

template <int TENSOR, bool PER>
__global__ void __launch_bounds__(kNT) vjp2_kernel(const float *__restrict__ pos, const float *__restrict__ frc,
                                                   const float *__restrict__ wv, double *__restrict__ partM,
                                                   double *__restrict__ partG, int npad, DenseGeom g, VjpConst2 c,
                                                   int *__restrict__ err, long long wd) {
    constexpr int R = kRV2;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    float *s_tile = reinterpret_cast<float *>(smem);   // [2 stages][9 arrays][J]
    float *s_acc = s_tile + 18 * g.J;                   // [R][12][kNT]: M hi(3) lo(3), G hi(3) lo(3)

    const int tid = threadIdx.x;
    const long long T = static_cast<long long>(g.nIB) * g.nJT;
    const long long t0 = static_cast<long long>(blockIdx.x) * g.chunk;
    const long long t1 = (t0 + g.chunk < T) ? t0 + g.chunk : T;
    if (t0 >= t1) return;
    const uint32_t arr_bytes = static_cast<uint32_t>(g.J * sizeof(float));

    int issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0;   // bookkeeping of thread 0 only
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](long long t, int stg) {
        const size_t j0 = static_cast<size_t>(t % g.nJT) * g.J;
        float *dst = s_tile + stg * 9 * g.J;
        mbar_arrive_expect_tx(&bars[stg], 9 * arr_bytes);
        for (int a = 0; a < 3; ++a) {
            bulk_g2s(dst + a * g.J, pos + a * static_cast<size_t>(npad) + j0, arr_bytes, &bars[stg]);
            bulk_g2s(dst + (3 + a) * g.J, frc + a * static_cast<size_t>(npad) + j0, arr_bytes, &bars[stg]);
            bulk_g2s(dst + (6 + a) * g.J, wv + a * static_cast<size_t>(npad) + j0, arr_bytes, &bars[stg]);
        }
        if (stg == 0) ++issued0; else ++issued1;
    };
    if (tid == 0)
        for (int q = 0; q < 2 && t0 + q < t1; ++q) issue(t0 + q, q);

    f2 XI[R], YI[R], ZI[R], FI[R][3], WI[R][3];
    int cur_ib = -1;
    bool aborted = false;

    auto flush = [&](int ib) {
        const int slot = static_cast<int>(blockIdx.x) - geom_first(g, ib);
        float2 *dM = reinterpret_cast<float2 *>(partM) + static_cast<size_t>(slot) * 3 * npad;
        float2 *dG = reinterpret_cast<float2 *>(partG) + static_cast<size_t>(slot) * 3 * npad;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const size_t i = static_cast<size_t>(ib) * g.I + tid + k * kNT;
            const float *q = s_acc + k * 12 * kNT + tid;
            for (int d = 0; d < 3; ++d) {
                dM[d * static_cast<size_t>(npad) + i] = make_float2(q[d * kNT], q[(3 + d) * kNT]);
                dG[d * static_cast<size_t>(npad) + i] = make_float2(q[(6 + d) * kNT], q[(9 + d) * kNT]);
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
                for (int d = 0; d < 3; ++d) {
                    const float fv = frc[d * static_cast<size_t>(npad) + i], wvv = wv[d * static_cast<size_t>(npad) + i];
                    FI[k][d] = pk2(fv, fv);
                    WI[k][d] = pk2(wvv, wvv);
                }
                for (int e = 0; e < 12; ++e) s_acc[(k * 12 + e) * kNT + tid] = 0.0f;
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
        const float *src = s_tile + st * 9 * g.J;
        f2 M[R][3], G[R][3];
#pragma unroll
        for (int k = 0; k < R; ++k)
            for (int d = 0; d < 3; ++d) M[k][d] = G[k][d] = 0ull;
#pragma unroll 2
        for (int jj = 0; jj < g.J; jj += 4) {
            f2 P[9][2];   // four sources: two packed pairs per array
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(src + a * g.J + jj);
                P[a][0] = v.x;
                P[a][1] = v.y;
            }
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
                for (int k = 0; k < R; ++k)
                    vjp_pair_f32x2<TENSOR, PER>(XI[k], YI[k], ZI[k], FI[k][0], FI[k][1], FI[k][2], WI[k][0], WI[k][1],
                                                WI[k][2], P[0][h2], P[1][h2], P[2][h2], P[3][h2], P[4][h2], P[5][h2],
                                                P[6][h2], P[7][h2], P[8][h2], c, M[k], G[k]);
        }
#pragma unroll
        for (int k = 0; k < R; ++k)
            for (int d = 0; d < 3; ++d) {
                float lo, hi;
                float *q0 = s_acc + (k * 12 + d) * kNT + tid;   // M hi; M lo at +3 kNT
                upk2(M[k][d], lo, hi);
                float h = q0[0], l = q0[3 * kNT];
                fold2(h, l, lo);
                fold2(h, l, hi);
                q0[0] = h;
                q0[3 * kNT] = l;
                float *q1 = s_acc + (k * 12 + 6 + d) * kNT + tid;   // G hi; G lo at +3 kNT
                upk2(G[k][d], lo, hi);
                h = q1[0];
                l = q1[3 * kNT];
                fold2(h, l, lo);
                fold2(h, l, hi);
                q1[0] = h;
                q1[3 * kNT] = l;
            }
        __syncthreads();   // every thread is done with stage st
        aborted = s_abort != 0;
        if (tid == 0 && !aborted && t + 2 < t1) issue(t + 2, st);
    }
    flush(cur_ib);
    if (tid == 0) {
        for (int k = waited0; k < issued0; ++k)
            if (!mbar_wait_bounded(&bars[0], k & 1, drain_limit(wd))) atomicOr(err, DEV_ERR_TIMEOUT);
        for (int k = waited1; k < issued1; ++k)
            if (!mbar_wait_bounded(&bars[1], k & 1, drain_limit(wd))) atomicOr(err, DEV_ERR_TIMEOUT);
    }
}

template <int TT, int MM>
static void *vjp_fn(bool per) {
    return per ? reinterpret_cast<void *>(&vjp_kernel<TT, MM, true>)
               : reinterpret_cast<void *>(&vjp_kernel<TT, MM, false>);
}

template <int TT>
static void *vjp2_fn(bool per) {
    return per ? reinterpret_cast<void *>(&vjp2_kernel<TT, true>) : reinterpret_cast<void *>(&vjp2_kernel<TT, false>);
}

static void *pick_vjp(int tensor, int mode, bool per) {
    const int dt = (tensor == T_OSEEN) ? T_OSEEN : T_RP;
    if (mode == MODE_FP64) return dt == T_OSEEN ? vjp_fn<T_OSEEN, MODE_FP64>(per) : vjp_fn<T_RP, MODE_FP64>(per);
    return dt == T_OSEEN ? vjp2_fn<T_OSEEN>(per) : vjp2_fn<T_RP>(per);
}

// Dynamic shared memory: FP64, two stages of three dbl4 arrays; FP32C, two stages of
// nine float arrays and the (hi, lo) accumulators.
static size_t vjp_smem(int mode, int J) {
    if (mode == MODE_FP64) return 6 * static_cast<size_t>(J) * sizeof(dbl4);
    return 18 * static_cast<size_t>(J) * sizeof(float) + static_cast<size_t>(kRV2) * 12 * kNT * sizeof(float);
}

// The grid holds SD_VJP_CTA_SCALE times as many CTAs as fit at once, so the block
// scheduler evens out the SMs' shares (N = 4,096: 57 -> 51 us; 8x gave the same).
#ifndef SD_VJP_CTA_SCALE
#define SD_VJP_CTA_SCALE 2
#endif
#ifndef SD_VJP_JMIN
#define SD_VJP_JMIN 64   // smallest j-tile (32 measured slower at N = 4,096)
#endif
cudaError_t vjp_setup(sd_handle *h) {
    DenseGeom g{};
    const int mode = (h->mode == MODE_FP64) ? MODE_FP64 : MODE_FP32C;
    g.I = kNT * (mode == MODE_FP64 ? kRV : kRV2);
    g.nIB = h->npad / g.I;
    void *fn = pick_vjp(h->tensor, mode, h->pc.periodic != 0);
    int occ = 0;
    const int Jc[4] = {kJmax, 128, 64, SD_VJP_JMIN};
    for (int ci = 0; ci < 4; ++ci) {
        const int J = Jc[ci];
        if (mode == MODE_FP64 && J > 128) continue;
        const size_t smem = vjp_smem(mode, J);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kNT, smem);
        if (e != cudaSuccess) return e;
        g.J = J;
        g.nJT = h->npad / J;
        if (static_cast<long long>(g.nIB) * g.nJT >= 4LL * h->num_sms * std::max(occ, 1)) break;
    }
    occ = std::max(occ, 1);
    const long long T = static_cast<long long>(g.nIB) * g.nJT;
    const long long want = static_cast<long long>(h->num_sms) * occ * SD_VJP_CTA_SCALE;
    g.chunk = std::max(1LL, (T + want - 1) / want);
    g.grid = static_cast<int>((T + g.chunk - 1) / g.chunk);
    int ms = 0;
    for (int ib = 0; ib < g.nIB; ++ib) ms = std::max(ms, geom_last(g, ib) - geom_first(g, ib) + 1);
    g.maxSlots = ms;
    h->geomv = g;
    h->vjp_occ = occ;
    return cudaSuccess;
}

cudaError_t launch_vjp_dense(sd_handle *h, cudaStream_t st, Mirror posm, Mirror frcm, Mirror wm, double *partM,
                             double *partG) {
    const DenseGeom &g = h->geomv;
    const bool f64 = h->mode == MODE_FP64;
    const size_t smem = vjp_smem(f64 ? MODE_FP64 : MODE_FP32C, g.J);
    const bool oseen = h->tensor == T_OSEEN;
    const bool per = h->pc.periodic != 0;
    prof_begin(h, SD_KERNEL_VJP, st);
    if (f64) {
#define SD_VJP_LAUNCH(TT, PP)                                                                                 \
    vjp_kernel<TT, MODE_FP64, PP><<<g.grid, kNT, smem, st>>>(                                                 \
        static_cast<const dbl4 *>(posm.aos), static_cast<const dbl4 *>(frcm.aos),                            \
        static_cast<const dbl4 *>(wm.aos), partM, partG, h->npad, g, h->pc, h->d_err, h->watchdog)
        if (oseen) {
            if (per) SD_VJP_LAUNCH(T_OSEEN, true); else SD_VJP_LAUNCH(T_OSEEN, false);
        } else {
            if (per) SD_VJP_LAUNCH(T_RP, true); else SD_VJP_LAUNCH(T_RP, false);
        }
#undef SD_VJP_LAUNCH
    } else {
        const PairConst &pc = h->pc;
        VjpConst2 c{};
        c.c1 = pk2_host(pc.c1_f);
        c.c3 = pk2_host(pc.c3_f);
        c.m3c3 = pk2_host(pc.m3c3_f);
        c.nc1 = pk2_host(-pc.c1_f);
        c.n5m3c3 = pk2_host(-5.0f * pc.m3c3_f);   // (rounded in FP32, as vjp_pair_f32 forms them)
        c.n3c1 = pk2_host(-3.0f * pc.c1_f);
        c.r2min = pc.r2min_f;
        for (int d = 0; d < 3; ++d) {
            c.negL[d] = pk2_host(-pc.Lf[d]);
            c.invL[d] = pk2_host(pc.invLf[d]);
        }
#define SD_VJP2_LAUNCH(TT, PP)                                                                                \
    vjp2_kernel<TT, PP><<<g.grid, kNT, smem, st>>>(posm.soa, frcm.soa, wm.soa, partM, partG, h->npad, g, c,   \
                                                    h->d_err, h->watchdog)
        if (oseen) {
            if (per) SD_VJP2_LAUNCH(T_OSEEN, true); else SD_VJP2_LAUNCH(T_OSEEN, false);
        } else {
            if (per) SD_VJP2_LAUNCH(T_RP, true); else SD_VJP2_LAUNCH(T_RP, false);
        }
#undef SD_VJP2_LAUNCH
    }
    prof_end(h, SD_KERNEL_VJP, st);
    ++h->launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- VJP epilogue

struct VjpEpiArgs {
    const double *partM, *partG;
    int npad;
    DenseGeom g;
    const double *x64;
    const void *posm;
    const double *F64;
    const void *frcm;
    const double *W64;
    const void *wm;
    CellList cl;
    double rnear2;
    PairConst pc;
    int n;
    int out_dtype;   // SD_DTYPE_F32 / SD_DTYPE_F64 for gX / gF, or -1 = adjoint update
    void *gx_out, *gF_out;
    double dt;
    double *lam_out;   // adjoint: lam_out = W + dt gX
    double *gF_acc;    // adjoint: gF_acc += dt mu W
    int *err;
};

// One lane's share of particle i's VJP terms: the CTA slots sub, sub + kWalkLanes, ...
// of the dense partial sums, the self term (sub-lane 0), and the FP64 near pairs of
// the neighbour cells sub, sub + kWalkLanes, ... of the 27.  MG = (M, G): the mu W
// part and the x-derivative part, before the factor mu0.
template <int TENSOR, int MODE>
__device__ __forceinline__ void vjp_epilogue_lane(const VjpEpiArgs &a, int i, int sub,
                                                  const typename VjpT<MODE>::V4 *pm,
                                                  const typename VjpT<MODE>::V4 *fm,
                                                  const typename VjpT<MODE>::V4 *wm, double (&MG)[6],
                                                  bool &coincident) {
    using V4 = typename VjpT<MODE>::V4;
    using V3 = typename VjpT<MODE>::V3;
    using S = typename VjpT<MODE>::S;
    constexpr int TD = (TENSOR == T_OSEEN) ? T_OSEEN : T_RP;
    {
        const int ib = i / a.g.I;
        const int ns = geom_last(a.g, ib) - geom_first(a.g, ib) + 1;
        if constexpr (MODE == MODE_FP64) {
            for (int s = sub; s < ns; s += kWalkLanes)
                for (int d = 0; d < 3; ++d) {
                    MG[d] += a.partM[(static_cast<size_t>(s) * 3 + d) * a.npad + i];
                    MG[3 + d] += a.partG[(static_cast<size_t>(s) * 3 + d) * a.npad + i];
                }
        } else {   // (hi, lo) float pairs, summed with FP32 TwoSum (FP64 issues at 1/64 the rate)
            const float2 *pM = reinterpret_cast<const float2 *>(a.partM);
            const float2 *pG = reinterpret_cast<const float2 *>(a.partG);
            float hi[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, lo[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            for (int s = sub; s < ns; s += kWalkLanes)
                for (int d = 0; d < 3; ++d) {
                    const float2 qm = pM[(static_cast<size_t>(s) * 3 + d) * a.npad + i];
                    const float2 qg = pG[(static_cast<size_t>(s) * 3 + d) * a.npad + i];
                    fold2(hi[d], lo[d], qm.x);
                    lo[d] = __fadd_rn(lo[d], qm.y);
                    fold2(hi[3 + d], lo[3 + d], qg.x);
                    lo[3 + d] = __fadd_rn(lo[3 + d], qg.y);
                }
            for (int d = 0; d < 6; ++d) MG[d] += static_cast<double>(hi[d]) + static_cast<double>(lo[d]);
        }
    }
    const V4 pi = pm[i], fi4 = fm[i], wi4 = wm[i];
    V3 Fi, Wi;
    Fi.x = fi4.x; Fi.y = fi4.y; Fi.z = fi4.z;
    Wi.x = wi4.x; Wi.y = wi4.y; Wi.z = wi4.z;
    auto dense = [&](const V4 &pj, const V4 &fj, const V4 &wj, double tm[3], double tg[3]) {
        V3 m, g;
        m.x = m.y = m.z = S(0);
        g.x = g.y = g.z = S(0);
        if (a.pc.periodic)
            vjp_term<TD, MODE, true>(pi.x, pi.y, pi.z, Fi, Wi, pj, fj, wj, a.pc, m, g);
        else
            vjp_term<TD, MODE, false>(pi.x, pi.y, pi.z, Fi, Wi, pj, fj, wj, a.pc, m, g);
        tm[0] = m.x; tm[1] = m.y; tm[2] = m.z;
        tg[0] = g.x; tg[1] = g.y; tg[2] = g.z;
    };
    if (sub == 0) {   // self: mu_ii W_i / mu0 = W_i; its x-derivative is zero
        double tm[3], tg[3];
        dense(pi, fi4, wi4, tm, tg);
        for (int d = 0; d < 3; ++d) {
            MG[d] += a.W64[3 * i + d] - tm[d];
            MG[3 + d] -= tg[d];
        }
    }
    const double xi = a.x64[3 * i], yi = a.x64[3 * i + 1], zi = a.x64[3 * i + 2];
    const double Fx = a.F64[3 * i], Fy = a.F64[3 * i + 1], Fz = a.F64[3 * i + 2];
    const double Wx = a.W64[3 * i], Wy = a.W64[3 * i + 1], Wz = a.W64[3 * i + 2];
    for_each_neighbour_part(a.cl, i, a.cl.cell[i], sub, kWalkLanes, [&](int j) {
        double dx = xi - a.x64[3 * j], dy = yi - a.x64[3 * j + 1], dz = zi - a.x64[3 * j + 2];
        box_image(a.cl.box, dx, dy, dz);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= a.rnear2) return;
        if (r2 == 0.0 && TENSOR != T_RPY) {
            coincident = true;
            return;
        }
        double A, B, dA, dB;
        profile_exact<TENSOR>(r2, a.pc, A, B, dA, dB);
        const double fx = a.F64[3 * j], fy = a.F64[3 * j + 1], fz = a.F64[3 * j + 2];
        const double wx = a.W64[3 * j], wy = a.W64[3 * j + 1], wz = a.W64[3 * j + 2];
        const double Wir = dx * Wx + dy * Wy + dz * Wz, Fir = dx * Fx + dy * Fy + dz * Fz;
        const double Wjr = dx * wx + dy * wy + dz * wz, Fjr = dx * fx + dy * fy + dz * fz;
        const double U = Wx * fx + Wy * fy + Wz * fz + wx * Fx + wy * Fy + wz * Fz;
        const double Q = Wir * Fjr + Wjr * Fir;
        const double cr = dA * U + dB * Q;
        double tm[3], tg[3];
        dense(pm[j], fm[j], wm[j], tm, tg);
        MG[0] += A * wx + B * Wjr * dx - tm[0];
        MG[1] += A * wy + B * Wjr * dy - tm[1];
        MG[2] += A * wz + B * Wjr * dz - tm[2];
        MG[3] += cr * dx + B * (Wx * Fjr + fx * Wir + wx * Fir + Fx * Wjr) - tg[0];
        MG[4] += cr * dy + B * (Wy * Fjr + fy * Wir + wy * Fir + Fy * Wjr) - tg[1];
        MG[5] += cr * dz + B * (Wz * Fjr + fz * Wir + wz * Fir + Fz * Wjr) - tg[2];
    });
}

// kWalkLanes threads per particle; their partial sums meet in the fixed shuffle tree
// of walk_sum (deterministic), and sub-lane 0 writes the particle's results.
template <int TENSOR, int MODE>
__global__ void __launch_bounds__(128) vjp_epilogue_kernel(VjpEpiArgs a) {
    using V4 = typename VjpT<MODE>::V4;
    const long long gt = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int i = static_cast<int>(gt / kWalkLanes), sub = static_cast<int>(gt % kWalkLanes);
    const bool active = i < a.n;
    double MG[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    bool coincident = false;
    if (active)
        vjp_epilogue_lane<TENSOR, MODE>(a, i, sub, static_cast<const V4 *>(a.posm), static_cast<const V4 *>(a.frcm),
                                        static_cast<const V4 *>(a.wm), MG, coincident);
    for (int d = 0; d < 6; ++d) MG[d] = walk_sum(MG[d]);
    coincident = walk_any(coincident);
    if (!active || sub != 0) return;
    if (coincident) atomicOr(a.err, DEV_ERR_COINCIDENT);
    const double m0 = a.pc.mu0;
    double M[3], G[3];
    for (int d = 0; d < 3; ++d) {
        M[d] = MG[d] * m0;
        G[d] = MG[3 + d] * m0;
    }
    if (a.out_dtype == SD_DTYPE_F32) {
        float *gx = static_cast<float *>(a.gx_out), *gF = static_cast<float *>(a.gF_out);
        for (int d = 0; d < 3; ++d) {
            if (gx) gx[3 * i + d] = static_cast<float>(G[d]);
            if (gF) gF[3 * i + d] = static_cast<float>(M[d]);
        }
    } else if (a.out_dtype == SD_DTYPE_F64) {
        double *gx = static_cast<double *>(a.gx_out), *gF = static_cast<double *>(a.gF_out);
        for (int d = 0; d < 3; ++d) {
            if (gx) gx[3 * i + d] = G[d];
            if (gF) gF[3 * i + d] = M[d];
        }
    } else {
        for (int d = 0; d < 3; ++d) {
            a.lam_out[3 * i + d] = a.W64[3 * i + d] + a.dt * G[d];
            a.gF_acc[3 * i + d] += a.dt * M[d];
        }
    }
}

cudaError_t launch_vjp_epilogue(sd_handle *h, cudaStream_t st, const double *x64, const void *posm,
                                const double *F64, const void *frcm, const double *W64, const void *wm,
                                int out_dtype, void *gx_out, void *gF_out, double dt, double *lam_out,
                                double *gF_acc) {
    if (h->n == 0) return cudaSuccess;
    VjpEpiArgs a;
    a.partM = h->part;
    a.partG = h->part2;
    a.npad = h->npad;
    a.g = h->geomv;
    a.x64 = x64;
    a.posm = posm;
    a.F64 = F64;
    a.frcm = frcm;
    a.W64 = W64;
    a.wm = wm;
    a.cl = h->cl;
    a.rnear2 = h->r_near * h->r_near;
    a.pc = h->pc;
    a.n = h->n;
    a.out_dtype = out_dtype;
    a.gx_out = gx_out;
    a.gF_out = gF_out;
    a.dt = dt;
    a.lam_out = lam_out;
    a.gF_acc = gF_acc;
    a.err = h->d_err;
    const int nb = static_cast<int>((static_cast<long long>(h->n) * kWalkLanes + 127) / 128);
    prof_begin(h, SD_KERNEL_EPILOGUE, st);
    const bool f64 = h->mode == MODE_FP64;
    switch (h->tensor) {
        case T_RPY:
            if (f64) vjp_epilogue_kernel<T_RPY, MODE_FP64><<<nb, 128, 0, st>>>(a);
            else vjp_epilogue_kernel<T_RPY, MODE_FP32C><<<nb, 128, 0, st>>>(a);
            break;
        case T_RP:
            if (f64) vjp_epilogue_kernel<T_RP, MODE_FP64><<<nb, 128, 0, st>>>(a);
            else vjp_epilogue_kernel<T_RP, MODE_FP32C><<<nb, 128, 0, st>>>(a);
            break;
        default:
            if (f64) vjp_epilogue_kernel<T_OSEEN, MODE_FP64><<<nb, 128, 0, st>>>(a);
            else vjp_epilogue_kernel<T_OSEEN, MODE_FP32C><<<nb, 128, 0, st>>>(a);
            break;
    }
    prof_end(h, SD_KERNEL_EPILOGUE, st);
    ++h->launches;
    return cudaGetLastError();
}

}  // namespace sd
