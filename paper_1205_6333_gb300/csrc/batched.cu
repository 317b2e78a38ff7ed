// batched.cu -- many independent clusters, one persistent launch per Euler step.
//
// Each cluster c (particles off[c] .. off[c+1]-1, at most 256) evolves by
//   v_i = mu0 [F_i + sum_{j != i in c} T^(r_i - r_j) F_j],  x_i <- x_i + dt v_i
// (Sec. 2.2, Eq. rotneMobility; Sec. 3.1, steps 1 and 3).
//
// Work distribution: a persistent grid; every warp pops cluster tickets from a
// global atomic counter (reset by a memset node before each step) and takes the
// clusters in largest-first order (a longest-processing-time schedule), so the
// small clusters fill the tail.  A warp stages its cluster in shared memory --
// FP64 positions minus the cluster's first particle, rounded to FP32, so FP32
// separations keep full relative precision and no FP64 near-pair pass is needed
// -- and lane l owns particles l, l+32, ..., l+32(R-1), R = ceil(n/32).
//
// The j loop runs over 32-particle chunks in a lane-rotated order
// (j = 32 jb + ((l + m) mod 32)), so a particle meets itself exactly at m = 0 of
// its own chunk and that pair is skipped without a per-pair test.  Pairs use the
// dense kernel's clamped pair term; a running minimum of r^2 flags overlaps
// (r < 2a), and only then does a second pass replace the clamped terms of the
// overlapping pairs by their exact values.  FP32C keeps per-lane (hi, lo)
// accumulators in shared memory and folds each chunk's FP32 partial into them
// with TwoSum.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <type_traits>
#include <tuple>
#include <vector>

#include "sd_internal.h"

namespace sd {

constexpr int kMaxCluster = 256;

struct BatchShape {
    int warps;        // warps per CTA
    int ctas_per_sm;  // resident CTAs per SM requested
    int r = 1;        // FP32C block kernel: targets per thread (1 or 2); 0: the symmetric kernel
};

}  // namespace sd

struct sd_batch {
    sd_config cfg{};
    int C = 0, P = 0, maxn = 0;
    int mode = 0, tensor = 0, device = 0, num_sms = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    sd::Allocator al;
    sd::PairConst pc{};
    int32_t *d_off = nullptr, *d_order = nullptr;
    // largest-first layout of the FP32C block kernel (see batched_blocks_kernel)
    int32_t *qperm = nullptr, *qcl = nullptr, *cbeg = nullptr, *cend = nullptr, *canchor = nullptr;
    int32_t *tq = nullptr;   // slots of two targets (see batched_blocks_kernel)
    int M2 = 0;              // number of such slots
    int4 *stask = nullptr;   // symmetric kernel: (cluster, cluster, 32-blocks) per warp task
    int nstask = 0;
    double *x64[2] = {nullptr, nullptr};   // position ping-pong: step reads x64[cur], writes the other
    float4 *rel[2] = {nullptr, nullptr};   // FP32C: positions relative to the cluster's reference point
    int32_t *panchor = nullptr;            // first particle of each particle's cluster
    int cur = 0;
    double *F64 = nullptr, *fext64 = nullptr;
    void *frcm = nullptr;
    unsigned long long *ctr = nullptr;
    int *d_err = nullptr;
    bool pos_set = false;
    std::vector<sd::BatchShape> shapes;
    int choice = -1;
    cudaGraphExec_t gexec = nullptr;
    double g_dt = 0.0;
    int g_choice = -1, g_cur = -1;
    int64_t launches = 0;
    sd::Profiler prof;
    long long watchdog = sd::kDefaultWatchdog;
};

namespace sd {

template <int MODE>
struct BT {
    using V4 = float4;
    using S = float;
};
template <>
struct BT<MODE_FP64> {
    using V4 = dbl4;
    using S = double;
};

struct BatchArgs {
    const int32_t *off, *order;
    const int32_t *qperm, *qcl, *cbeg, *cend, *canchor;
    const int32_t *tq;   // two-target slots: q (targets q, q + 1) or ~q (q alone)
    const int4 *stask;   // symmetric kernel's tasks
    int P, M2, nblk;
    const double *x64;   // positions of this step
    double *x64n;        // positions after it
    const float4 *rel;   // FP32C: FP32 positions of this step relative to their cluster's reference point
    float4 *reln;        // ... after it, relative to the reference point of this step (x64 of the anchor)
    const int32_t *panchor;
    const double *F64;
    const void *frcm;
    unsigned long long *ctr;
    int C;
    PairConst pc;
    double dt;
    int *err;
};

// Exact pair term (overlap branch included) in the working precision, from zero.
template <int TENSOR, typename S>
__device__ __forceinline__ void exact_pair(S dx, S dy, S dz, S fx, S fy, S fz, const PairConst &c, S &ox, S &oy,
                                           S &oz, bool &coincident) {
    const S r2 = dx * dx + dy * dy + dz * dz;
    ox = oy = oz = S(0);
    if (r2 == S(0)) {
        if (TENSOR != T_RPY) coincident = true;
        else { ox = fx; oy = fy; oz = fz; }   // T^(0) = I for the RPY overlap form
        return;
    }
    const S r = sqrt(r2);
    S A, B;
    if (TENSOR == T_RPY && r < S(c.two_a)) {
        A = S(1) - S(9) * r / (S(32) * S(c.a));
        B = S(3) / (S(32) * S(c.a) * r);
    } else if (TENSOR == T_OSEEN) {
        A = S(c.c1_d) / r;
        B = A / r2;
    } else {
        const S ri = S(1) / r, ri2 = ri * ri;
        A = ri * (S(c.c1_d) + S(c.c3_d) * ri2);
        B = ri * ri2 * (S(c.c1_d) + S(c.m3c3_d) * ri2);
    }
    const S s = B * (dx * fx + dy * fy + dz * fz);
    ox = A * fx + s * dx;
    oy = A * fy + s * dy;
    oz = A * fz + s * dz;
}

template <int TENSOR, int MODE, int R>
__device__ __forceinline__ void cluster_compute(const BatchArgs &a, int o, int n, double3 anchor,
                                                const typename BT<MODE>::V4 *s_pos,
                                                const typename BT<MODE>::V4 *s_frc, float *s_acc, int lane) {
    using V4 = typename BT<MODE>::V4;
    using S = typename BT<MODE>::S;
    constexpr int TD = (TENSOR == T_OSEEN) ? T_OSEEN : T_RP;
    constexpr bool COMP = (MODE == MODE_FP32C);
    S xi[R], yi[R], zi[R], ax[R], ay[R], az[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        // slots beyond n sit far from everything (their results are discarded)
        const V4 p = s_pos[lane + 32 * k];
        const bool real = lane + 32 * k < n;
        xi[k] = real ? S(p.x) : S(-1.0e15);
        yi[k] = real ? S(p.y) : S(0);
        zi[k] = real ? S(p.z) : S(0);
        ax[k] = ay[k] = az[k] = S(0);
        if (COMP)
            for (int d = 0; d < 6; ++d) s_acc[(k * 6 + d) * 32 + lane] = 0.0f;
    }
    S mn = S(1e30);
    const int nchunk = (n + 31) >> 5;
    for (int jb = 0; jb < nchunk; ++jb) {
        // m = 0: the diagonal slot k == jb meets itself; skip that pair only
        {
            const int j = 32 * jb + lane;
            const V4 p = s_pos[j], f = s_frc[j];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if (k == jb) continue;
                const S dx = xi[k] - p.x, dy = yi[k] - p.y, dz = zi[k] - p.z;
                mn = fmin(mn, dx * dx + dy * dy + dz * dz);
                if constexpr (MODE == MODE_FP64)
                    pair_f64<TD>(xi[k], yi[k], zi[k], p, f, a.pc, ax[k], ay[k], az[k]);
                else
                    pair_f32<TD>(xi[k], yi[k], zi[k], p, f, a.pc, ax[k], ay[k], az[k]);
            }
        }
        for (int m = 1; m < 32; ++m) {
            const int j = 32 * jb + ((lane + m) & 31);
            const V4 p = s_pos[j], f = s_frc[j];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if constexpr (MODE == MODE_FP64) {
                    const double dx = xi[k] - p.x, dy = yi[k] - p.y, dz = zi[k] - p.z;
                    mn = fmin(mn, dx * dx + dy * dy + dz * dz);
                    pair_f64<TD>(xi[k], yi[k], zi[k], p, f, a.pc, ax[k], ay[k], az[k]);
                } else {
                    // the clamp in pair_f32 sees the same r^2; track it for the overlap test
                    const float dx = __fsub_rn(xi[k], p.x), dy = __fsub_rn(yi[k], p.y), dz = __fsub_rn(zi[k], p.z);
                    mn = fminf(mn, __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
                    pair_f32<TD>(xi[k], yi[k], zi[k], p, f, a.pc, ax[k], ay[k], az[k]);
                }
            }
        }
        if constexpr (COMP) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                float *q = s_acc + k * 6 * 32 + lane;
                float hx = q[0], hy = q[32], hz = q[64], lx = q[96], ly = q[128], lz = q[160];
                fold2(hx, lx, ax[k]);
                fold2(hy, ly, ay[k]);
                fold2(hz, lz, az[k]);
                q[0] = hx; q[32] = hy; q[64] = hz; q[96] = lx; q[128] = ly; q[160] = lz;
                ax[k] = ay[k] = az[k] = 0.0f;
            }
        }
    }
    // per slot: compensated dense sum, exact terms for overlapping pairs (only
    // when some lane saw r < 2a), self term mu_ii = mu0 I, Euler update in FP64
    const bool overlap = __any_sync(0xffffffffu, mn < S(a.pc.r2min_d));
    bool coincident = false;
    const double m0 = a.pc.mu0, dt = a.dt;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int i = lane + 32 * k;
        if (i >= n) continue;
        double V0, V1, V2;
        if constexpr (COMP) {
            const float *q = s_acc + k * 6 * 32 + lane;
            V0 = static_cast<double>(q[0]) + q[96];
            V1 = static_cast<double>(q[32]) + q[128];
            V2 = static_cast<double>(q[64]) + q[160];
        } else {
            V0 = ax[k];
            V1 = ay[k];
            V2 = az[k];
        }
        if (overlap) {
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                const V4 p = s_pos[j], f = s_frc[j];
                S dx, dy, dz;
                if constexpr (MODE == MODE_FP64) {
                    dx = xi[k] - p.x; dy = yi[k] - p.y; dz = zi[k] - p.z;
                } else {
                    dx = __fsub_rn(xi[k], p.x); dy = __fsub_rn(yi[k], p.y); dz = __fsub_rn(zi[k], p.z);
                }
                const S r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < S(a.pc.r2min_d))) continue;
                S cx = S(0), cy = S(0), cz = S(0);
                if constexpr (MODE == MODE_FP64)
                    pair_f64<TD>(xi[k], yi[k], zi[k], p, f, a.pc, cx, cy, cz);
                else
                    pair_f32<TD>(xi[k], yi[k], zi[k], p, f, a.pc, cx, cy, cz);
                S ex, ey, ez;
                exact_pair<TENSOR, S>(dx, dy, dz, S(f.x), S(f.y), S(f.z), a.pc, ex, ey, ez, coincident);
                V0 += static_cast<double>(ex) - static_cast<double>(cx);
                V1 += static_cast<double>(ey) - static_cast<double>(cy);
                V2 += static_cast<double>(ez) - static_cast<double>(cz);
            }
        }
        const size_t g = static_cast<size_t>(o + i);
        const double vx = m0 * (V0 + a.F64[3 * g]);
        const double vy = m0 * (V1 + a.F64[3 * g + 1]);
        const double vz = m0 * (V2 + a.F64[3 * g + 2]);
        const double nx = a.x64[3 * g] + dt * vx, ny = a.x64[3 * g + 1] + dt * vy, nz = a.x64[3 * g + 2] + dt * vz;
        if (!isfinite(nx) || !isfinite(ny) || !isfinite(nz)) atomicOr(a.err, DEV_ERR_NONFINITE);
        a.x64n[3 * g] = nx;
        a.x64n[3 * g + 1] = ny;
        a.x64n[3 * g + 2] = nz;
    }
    if (coincident) atomicOr(a.err, DEV_ERR_COINCIDENT);
    (void)anchor;
}

// FP64 path: one warp per cluster, scalar FP64 pairs.
constexpr size_t kWarpStage = 2 * kMaxCluster * sizeof(dbl4);

template <int TENSOR>
__global__ void batched_kernel(BatchArgs a) {
    using V4 = dbl4;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char *mine = smem + static_cast<size_t>(wid) * kWarpStage;
    const V4 *frcm = static_cast<const V4 *>(a.frcm);
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.ctr, 1ULL);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= static_cast<unsigned long long>(a.C)) break;
        const int c = a.order[t];
        const int o = a.off[c];
        const int n = a.off[c + 1] - o;
        if (n <= 0) continue;
        if (n > kMaxCluster) {   // rejected at creation; never reached
            if (lane == 0) atomicOr(a.err, DEV_ERR_QUEUE);
            continue;
        }
        const double3 anchor = make_double3(a.x64[3 * o], a.x64[3 * o + 1], a.x64[3 * o + 2]);
        const int R = (n + 31) >> 5;
        V4 *s_pos = reinterpret_cast<V4 *>(mine);
        V4 *s_frc = s_pos + kMaxCluster;
        for (int p = lane; p < 32 * R; p += 32) {
            V4 q, f;
            if (p < n) {
                const size_t g = static_cast<size_t>(o + p);
                q.x = a.x64[3 * g] - anchor.x;
                q.y = a.x64[3 * g + 1] - anchor.y;
                q.z = a.x64[3 * g + 2] - anchor.z;
                f = frcm[g];
            } else {
                // padding: far away (and far from the unused i-slots at -1e15), zero force
                q.x = 1.0e15;
                q.y = 0;
                q.z = 0;
                f.x = f.y = f.z = 0;
            }
            q.w = 0;
            f.w = 0;
            s_pos[p] = q;
            s_frc[p] = f;
        }
        __syncwarp();
        switch (R) {
#define SD_BR(RR) \
    case RR: cluster_compute<TENSOR, MODE_FP64, RR>(a, o, n, anchor, s_pos, s_frc, nullptr, lane); break
            SD_BR(1); SD_BR(2); SD_BR(3); SD_BR(4); SD_BR(5); SD_BR(6); SD_BR(7); SD_BR(8);
#undef SD_BR
            default: break;
        }
        __syncwarp();
    }
}

// FP32C path: target blocks.  At creation the clusters are laid out largest
// first (a longest-processing-time order) as one sequence of P particles,
// position q of the sequence being particle qperm[q] of cluster qcl[q] (whose
// particles are the positions cbeg .. cend-1).  A thread owns R targets of one
// cluster: R = 1, the target q = its slot; R = 2, the slot's entry tq[m] = q
// (targets q, q + 1) or ~q (a cluster's last, odd target q alone; the second
// lane then repeats q and is not stored).  A persistent CTA of BT threads pops
// blocks of BT consecutive slots from a ticket counter, so neighbouring threads
// have targets in clusters of equal or near-equal size (their loops are as long).
// The CTA stages every cluster its block touches -- at most R BT + 2 (256 - 1)
// particles -- in shared memory as SoA floats: positions relative to each
// cluster's first particle (FP64 difference, then rounded, so FP32 separations
// keep full relative precision) and forces.  Each thread then sums over its own
// cluster with packed pairs (two sources per f32x2 instruction, read as
// broadcasts, each load serving the R targets), r^2 clamped to (2a)^2 throughout:
//   * the self pair is met once and its clamped term subtracted again, as
//     mu_ii = mu0 I joins the sum;
//   * pairs with r < 2a are listed as they are met; only they are swapped for
//     exact terms afterwards.
// Both packed lanes, the scalar edge terms and the self terms meet in a TwoSum
// (hi, lo) sum; v stays FP32, x_{n+1} = x_n + dt v in FP64.  Positions are read
// from x64 and written to x64n (a cluster may span two blocks).
constexpr int kStageExtra = 2 * (kMaxCluster - 1);
constexpr int kNoteCap = 8;   // close pairs (self included) a target lists; more: full rescan

template <int BT, int R>
__host__ __device__ constexpr int block_stage_len() {
    return ((R * BT + kStageExtra) + 3) & ~3;   // per SoA array, floats (16-byte multiple)
}

// Resident 128-thread CTAs per SM the two-target variant is compiled for: 6 keeps
// it at 80 registers without spills (7 spills a little, and neither beats the
// one-target variant's 8 CTAs of 64 registers on the batched workload).  The
// one-target variant gets no bound.
#ifndef SD_BATCH_R2_MINB
#define SD_BATCH_R2_MINB 6
#endif

template <int TENSOR, int BT, int R>
__global__ void __launch_bounds__(BT, R == 2 ? SD_BATCH_R2_MINB * 128 / BT : 0) batched_blocks_kernel(BatchArgs a) {
    static_assert(R == 1 || R == 2, "one or two targets per thread");
    constexpr int TD = (TENSOR == T_OSEEN) ? T_OSEEN : T_RP;
    constexpr int L = block_stage_len<BT, R>();
    extern __shared__ __align__(16) float s_src[];   // [6][L]: x y z Fx Fy Fz, then int [kNoteCap][R][BT]
    __shared__ int s_blk;
    int *s_note = reinterpret_cast<int *>(s_src + 6 * L);
    const int tid = threadIdx.x;
    const float4 *frcm = static_cast<const float4 *>(a.frcm);
    PairConst2 c2{};
    c2.c1 = pk2(a.pc.c1_f, a.pc.c1_f);
    c2.c3 = pk2(a.pc.c3_f, a.pc.c3_f);
    c2.m3c3 = pk2(a.pc.m3c3_f, a.pc.m3c3_f);
    c2.r2min = a.pc.r2min_f;
    const float r2min = a.pc.r2min_f;
    const float m0dt = static_cast<float>(a.pc.mu0 * a.dt);
    const int M = R == 1 ? a.P : a.M2;   // slots
    // the first target of slot m, and whether it has a second one
    auto slot = [&](int m, int &q, bool &pair) {
        if constexpr (R == 1) {
            q = m;
            pair = false;
        } else {
            const int t = a.tq[m];
            q = t < 0 ? ~t : t;
            pair = t >= 0;
        }
    };
    for (;;) {
        if (tid == 0) s_blk = static_cast<int>(atomicAdd(a.ctr, 1ULL));
        __syncthreads();
        const int blk = s_blk;
        if (blk >= a.nblk) break;   // uniform over the CTA
        const int m0 = blk * BT, m1 = min(m0 + BT, M);
        int qf, ql;
        bool pf, pl;
        slot(m0, qf, pf);
        slot(m1 - 1, ql, pl);
        if (pl) ++ql;
        const int s0 = a.cbeg[a.qcl[qf]], s1 = a.cend[a.qcl[ql]];   // s1 - s0 <= R BT + kStageExtra
        if (s1 > s0 && tid == 0) dbg_index(s1 - s0 - 1, L, a.err);
        for (int k = s0 + tid; k < s1; k += BT) {
            const int p = a.qperm[k];
            const float4 r = a.rel[p], f = frcm[p];
            const int l = k - s0;
            s_src[l] = r.x;
            s_src[L + l] = r.y;
            s_src[2 * L + l] = r.z;
            s_src[3 * L + l] = f.x;
            s_src[4 * L + l] = f.y;
            s_src[5 * L + l] = f.z;
        }
        __syncthreads();
        const int m = m0 + tid;
        if (m < m1) {
            int q0;
            bool two;
            slot(m, q0, two);
            const int cq = a.qcl[q0];
            const int beg = a.cbeg[cq] - s0, end = a.cend[cq] - s0;
            int me[R];
            float xi[R], yi[R], zi[R];
            f2 XI[R], YI[R], ZI[R], AX[R], AY[R], AZ[R];
            float tx[R], ty[R], tz[R];
            int close[R];   // pairs with r^2 < (2a)^2 (the self pair among them), listed as met
#pragma unroll
            for (int r = 0; r < R; ++r) {
                me[r] = q0 + (two ? r : 0) - s0;
                xi[r] = s_src[me[r]];
                yi[r] = s_src[L + me[r]];
                zi[r] = s_src[2 * L + me[r]];
                XI[r] = pk2(xi[r], xi[r]);
                YI[r] = pk2(yi[r], yi[r]);
                ZI[r] = pk2(zi[r], zi[r]);
                AX[r] = AY[r] = AZ[r] = 0ull;
                tx[r] = ty[r] = tz[r] = 0.0f;
                close[r] = 0;
            }
            auto note = [&](int r, int j) {
                if (close[r] < kNoteCap) s_note[(close[r] * R + r) * BT + tid] = j;
                ++close[r];
            };
            auto scalar = [&](int j) {
                const float4 pj = make_float4(s_src[j], s_src[L + j], s_src[2 * L + j], 0.0f);
                const float4 fj = make_float4(s_src[3 * L + j], s_src[4 * L + j], s_src[5 * L + j], 0.0f);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float dx = __fsub_rn(xi[r], pj.x), dy = __fsub_rn(yi[r], pj.y),
                                dz = __fsub_rn(zi[r], pj.z);
                    if (__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) < r2min) note(r, j);
                    pair_f32<TD, true>(xi[r], yi[r], zi[r], pj, fj, a.pc, tx[r], ty[r], tz[r]);
                }
            };
            int j = beg;
            while ((j & 3) && j < end) scalar(j++);   // 128-bit loads need an index that is a multiple of 4
            for (; j + 3 < end; j += 4) {
                // four sources: one 128-bit broadcast load per SoA array (j and L are multiples
                // of 4, so every load is 16-byte aligned); plain loads leave the compiler free
                // to schedule them (2.4% faster than volatile inline loads)
                f2 P[6][2];
                const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(s_src + j);
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    const ulonglong2 v = src[d * (L / 4)];
                    P[d][0] = v.x;
                    P[d][1] = v.y;
                }
                float rr[R][4];
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        pair_f32x2_t<TD, true, true>(XI[r], YI[r], ZI[r], P[0][h], P[1][h], P[2][h], P[3][h], P[4][h],
                                                     P[5][h], c2, AX[r], AY[r], AZ[r], rr[r][2 * h], rr[r][2 * h + 1]);
                float mn = fminf(fminf(rr[0][0], rr[0][1]), fminf(rr[0][2], rr[0][3]));
                if constexpr (R == 2) mn = fminf(mn, fminf(fminf(rr[1][0], rr[1][1]), fminf(rr[1][2], rr[1][3])));
                if (mn < r2min) {   // rare: overlaps, and the self pair once per target
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (rr[r][u] < r2min) note(r, j + u);
                }
            }
            while (j < end) scalar(j++);
            bool coincident = false;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r > 0 && !two) break;   // the repeated target of an odd cluster's last slot
                // the clamped self term, met once in the loop, bit for bit
                const float4 pi = make_float4(xi[r], yi[r], zi[r], 0.0f);
                const float4 fi = make_float4(s_src[3 * L + me[r]], s_src[4 * L + me[r]], s_src[5 * L + me[r]], 0.0f);
                float sx = 0.0f, sy = 0.0f, sz = 0.0f;
                pair_f32<TD, true>(xi[r], yi[r], zi[r], pi, fi, a.pc, sx, sy, sz);
                const f2 acc[3] = {AX[r], AY[r], AZ[r]};
                const float tsc[3] = {tx[r], ty[r], tz[r]}, ssc[3] = {sx, sy, sz}, fsc[3] = {fi.x, fi.y, fi.z};
                float V[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    float lo, hi, h, l;
                    upk2(acc[d], lo, hi);
                    two_sum(lo, hi, h, l);
                    fold2(h, l, tsc[d]);
                    fold2(h, l, -ssc[d]);
                    fold2(h, l, fsc[d]);   // mu_ii F_i / mu0 = F_i
                    V[d] = __fadd_rn(h, l);
                }
                auto fix = [&](int k) {   // swap the clamped term of an overlapping pair for the exact one
                    const float4 pj = make_float4(s_src[k], s_src[L + k], s_src[2 * L + k], 0.0f);
                    const float4 fj = make_float4(s_src[3 * L + k], s_src[4 * L + k], s_src[5 * L + k], 0.0f);
                    const float dx = __fsub_rn(xi[r], pj.x), dy = __fsub_rn(yi[r], pj.y), dz = __fsub_rn(zi[r], pj.z);
                    float cx = 0.0f, cy = 0.0f, cz = 0.0f, ex, ey, ez;
                    pair_f32<TD, true>(xi[r], yi[r], zi[r], pj, fj, a.pc, cx, cy, cz);
                    exact_pair<TENSOR, float>(dx, dy, dz, fj.x, fj.y, fj.z, a.pc, ex, ey, ez, coincident);
                    V[0] = __fadd_rn(V[0], __fsub_rn(ex, cx));
                    V[1] = __fadd_rn(V[1], __fsub_rn(ey, cy));
                    V[2] = __fadd_rn(V[2], __fsub_rn(ez, cz));
                };
                if (close[r] > 1 && close[r] <= kNoteCap) {   // the listed pairs, in the order met
                    for (int e = 0; e < close[r]; ++e) {
                        const int k = s_note[(e * R + r) * BT + tid];
                        if (k != me[r] && k >= beg && k < end) fix(k);   // every listed entry lies in [beg, end)
                    }
                } else if (close[r] > kNoteCap) {   // list overflow: scan the cluster again
                    for (int k = beg; k < end; ++k) {
                        if (k == me[r]) continue;
                        const float dx = __fsub_rn(xi[r], s_src[k]), dy = __fsub_rn(yi[r], s_src[L + k]),
                                    dz = __fsub_rn(zi[r], s_src[2 * L + k]);
                        if (__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) < r2min) fix(k);
                    }
                }
                const size_t g = static_cast<size_t>(a.qperm[me[r] + s0]);
                // the positions are finite (checked when set), so x + dt v is finite iff dt v is
                const float ux = __fmul_rn(m0dt, V[0]), uy = __fmul_rn(m0dt, V[1]), uz = __fmul_rn(m0dt, V[2]);
                if (!isfinite(ux) || !isfinite(uy) || !isfinite(uz)) atomicOr(a.err, DEV_ERR_NONFINITE);
                const double nx = a.x64[3 * g] + static_cast<double>(ux);
                const double ny = a.x64[3 * g + 1] + static_cast<double>(uy);
                const double nz = a.x64[3 * g + 2] + static_cast<double>(uz);
                a.x64n[3 * g] = nx;
                a.x64n[3 * g + 1] = ny;
                a.x64n[3 * g + 2] = nz;
                // the next step's FP32 position, relative to this step's position of the cluster's
                // first particle (the same reference point for the whole cluster; unchanged
                // during this step, x64 being read-only)
                const size_t an = static_cast<size_t>(a.panchor[g]);
                a.reln[g] = make_float4(static_cast<float>(nx - a.x64[3 * an]),
                                        static_cast<float>(ny - a.x64[3 * an + 1]),
                                        static_cast<float>(nz - a.x64[3 * an + 2]), 0.0f);
            }
            if (coincident) atomicOr(a.err, DEV_ERR_COINCIDENT);
        }
        __syncthreads();   // the stage and s_blk are free for the next block
    }
}

// ---------------------------------------------------------------- FP32C, symmetric

// The symmetric batched kernel: each unordered pair of a cluster once, its term
// used for both particles (mu_ij = mu_ji, Sec. 2.2), as dense_sym_kernel does for
// one large system.
//   * A warp takes a task from the ticket counter: two clusters of the largest-first
//     order (equal or nearly equal sizes), cut into the same number nb of 32-particle
//     blocks.  The two clusters ride the two halves of every packed f32x2 register,
//     so each packed instruction evaluates one pair of each cluster.  The warp stages
//     both clusters in its shared memory, interleaved (slot k holds particle k of
//     each), with padding slots far apart and far away, with zero force.
//   * Block pairs (p, q), p <= q: lane l holds target 32 p + l; at step m it takes
//     source 32 q + ((l + m) mod 32), and the source's running sum moves one lane down
//     per step by shuffle (after 32 steps lane l holds source l again).  A diagonal
//     block (p = q) takes the steps m = 1 .. 16 only (lanes l < 16 at m = 16): every
//     pair of the block once, no self pair.
//   * Sums: a tile's FP32 partials; the target's are folded into a TwoSum (hi, lo)
//     per block row, the sources' added to a per-particle shared sum.  Block p is
//     complete after its row (every tile that reaches it has run) and is finalised
//     at once: + F_i (the self term mu_ii = mu0 I), v = mu0 V, x <- x + dt v in FP64.
//   * r^2 is clamped to (2a)^2; the smallest unclamped r^2 of each tile is tracked,
//     and in a tile that met a pair with r < 2a the warp screens the targets of the
//     lanes that met one against the tile's sources, in parallel, listing each such
//     pair.  Before a row pair is finalised, the lanes take the listed pairs one each
//     and replace their clamped terms (bit-identical, recomputed) by the exact ones,
//     in both directions.
constexpr int kSymSlots = kMaxCluster;                 // particles per cluster half (8 blocks of 32)
constexpr int kSymFixCap = 128;                       // entries of a warp's list of pairs closer than 2a
constexpr int kSymTileCap = 16;                       // flagged tiles of a row pair (at most 9 walks)
constexpr size_t kSymWarpSmem = 9 * static_cast<size_t>(kSymSlots) * sizeof(f2)    // 6 staged + 3 sum arrays
                                + kSymFixCap * sizeof(int)                           // + the pair list
                                + kSymTileCap * sizeof(int2);                        // + the flagged tiles

// One pair of each half, both directions, with the unclamped r^2 of each half
// tracked (the order of operations of pair_sym_f32x2 with CLAMP).
template <int TENSOR>
__device__ __forceinline__ void bsym_pair(f2 XI, f2 YI, f2 ZI, f2 GX, f2 GY, f2 GZ, f2 PX, f2 PY, f2 PZ, f2 FX,
                                          f2 FY, f2 FZ, const PairConst2 &c, f2 &AX, f2 &AY, f2 &AZ, f2 &JX,
                                          f2 &JY, f2 &JZ, float &mn0, float &mn1) {
    const f2 dx = sub2(XI, PX), dy = sub2(YI, PY), dz = sub2(ZI, PZ);
    const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    float ra, rb;
    upk2(r2, ra, rb);
    mn0 = fminf(mn0, ra);
    mn1 = fminf(mn1, rb);
    ra = fmaxf(ra, c.r2min);
    rb = fmaxf(rb, c.r2min);
    const f2 ri = pk2(rsqrt_sfu(ra), rsqrt_sfu(rb));
    const f2 ri2 = mul2(ri, ri);
    f2 A, B;
    if (TENSOR == T_OSEEN) {
        A = mul2(c.c1, ri);
        B = mul2(A, ri2);
    } else {
        A = mul2(ri, fma2(c.c3, ri2, c.c1));
        const f2 ri3 = mul2(ri, ri2);
        B = mul2(ri3, fma2(c.m3c3, ri2, c.c1));
    }
    const f2 s = mul2(B, fma2(dz, FZ, fma2(dy, FY, mul2(dx, FX))));
    AX = fma2(s, dx, fma2(A, FX, AX));
    AY = fma2(s, dy, fma2(A, FY, AY));
    AZ = fma2(s, dz, fma2(A, FZ, AZ));
    const f2 u = mul2(B, fma2(dz, GZ, fma2(dy, GY, mul2(dx, GX))));
    JX = fma2(u, dx, fma2(A, GX, JX));
    JY = fma2(u, dy, fma2(A, GY, JY));
    JZ = fma2(u, dz, fma2(A, GZ, JZ));
}

__device__ __forceinline__ float half_of(f2 v, int h) {
    float lo, hi;
    upk2(v, lo, hi);
    return h ? hi : lo;
}
__device__ __forceinline__ f2 add_half(f2 v, int h, float d) {
    float lo, hi;
    upk2(v, lo, hi);
    if (h) hi = __fadd_rn(hi, d);
    else lo = __fadd_rn(lo, d);
    return pk2(lo, hi);
}

// Tile (p, q) of the warp's task: lane l holds target 32 p + l (XI..GZ); adds the
// tile's target partials to AX..AZ and its source sums to the shared sums.
template <int TENSOR, bool DIAG>
__device__ __forceinline__ void bsym_tile(const f2 *__restrict__ S, f2 *__restrict__ SUM, int q, int lane, f2 XI,
                                          f2 YI, f2 ZI, f2 GX, f2 GY, f2 GZ, const PairConst2 &c, f2 &AX, f2 &AY,
                                          f2 &AZ, float &mn0, float &mn1) {
    const f2 *SX = S + 32 * q, *SY = SX + kSymSlots, *SZ = SY + kSymSlots, *SFX = SZ + kSymSlots,
             *SFY = SFX + kSymSlots, *SFZ = SFY + kSymSlots;
    const int nxt = (lane + 1) & 31;
    f2 JX = 0ull, JY = 0ull, JZ = 0ull;
    constexpr int M0 = DIAG ? 1 : 0, M1 = DIAG ? 15 : 31;
#pragma unroll 4
    for (int m = M0; m <= M1; ++m) {
        const int k = (lane + m) & 31;
        bsym_pair<TENSOR>(XI, YI, ZI, GX, GY, GZ, SX[k], SY[k], SZ[k], SFX[k], SFY[k], SFZ[k], c, AX, AY, AZ, JX, JY,
                          JZ, mn0, mn1);
        JX = __shfl_sync(0xffffffffu, JX, nxt);
        JY = __shfl_sync(0xffffffffu, JY, nxt);
        JZ = __shfl_sync(0xffffffffu, JZ, nxt);
    }
    int sj = (lane + M1 + 1) & 31;   // the source whose sum this lane holds
    if (DIAG) {   // m = 16: the pair (l, l + 16) once, by the lanes l < 16
        const int k = (lane + 16) & 31;
        if (lane < 16)
            bsym_pair<TENSOR>(XI, YI, ZI, GX, GY, GZ, SX[k], SY[k], SZ[k], SFX[k], SFY[k], SFZ[k], c, AX, AY, AZ, JX,
                              JY, JZ, mn0, mn1);
        sj = k;
    }
    f2 *D = SUM + 32 * q + sj;
    D[0] = add2(D[0], JX);
    D[kSymSlots] = add2(D[kSymSlots], JY);
    D[2 * kSymSlots] = add2(D[2 * kSymSlots], JZ);
    __syncwarp();
}

// Tiles (p, q) and (p + 1, q), q > p + 1, in one walk of source block q: lane l holds
// targets 32 p + l (T0) and 32 (p + 1) + l (T1); each source's running sum collects
// both targets' terms before it moves on, and every source load serves both.
template <int TENSOR>
__device__ __forceinline__ void bsym_tile2(const f2 *__restrict__ S, f2 *__restrict__ SUM, int q, int lane,
                                           const f2 (&T0)[6], const f2 (&T1)[6], const PairConst2 &c, f2 (&A0)[3],
                                           f2 (&A1)[3], float &mn0, float &mn1) {
    const f2 *SX = S + 32 * q, *SY = SX + kSymSlots, *SZ = SY + kSymSlots, *SFX = SZ + kSymSlots,
             *SFY = SFX + kSymSlots, *SFZ = SFY + kSymSlots;
    const int nxt = (lane + 1) & 31;
    f2 JX = 0ull, JY = 0ull, JZ = 0ull;
#pragma unroll 2
    for (int m = 0; m < 32; ++m) {
        const int k = (lane + m) & 31;
        const f2 PX = SX[k], PY = SY[k], PZ = SZ[k], FX = SFX[k], FY = SFY[k], FZ = SFZ[k];
        bsym_pair<TENSOR>(T0[0], T0[1], T0[2], T0[3], T0[4], T0[5], PX, PY, PZ, FX, FY, FZ, c, A0[0], A0[1], A0[2], JX,
                          JY, JZ, mn0, mn1);
        bsym_pair<TENSOR>(T1[0], T1[1], T1[2], T1[3], T1[4], T1[5], PX, PY, PZ, FX, FY, FZ, c, A1[0], A1[1], A1[2], JX,
                          JY, JZ, mn0, mn1);
        JX = __shfl_sync(0xffffffffu, JX, nxt);
        JY = __shfl_sync(0xffffffffu, JY, nxt);
        JZ = __shfl_sync(0xffffffffu, JZ, nxt);
    }
    f2 *D = SUM + 32 * q + lane;
    D[0] = add2(D[0], JX);
    D[kSymSlots] = add2(D[kSymSlots], JY);
    D[2 * kSymSlots] = add2(D[2 * kSymSlots], JZ);
    __syncwarp();
}

// Pairs closer than 2a.  The walk only records the tiles that met one (with the
// lanes that did); one out-of-line call per row pair (bsym_rowfix) screens those
// tiles and fixes the pairs found, so the walk's code stays as it would be without
// them.
// The exact pair term (overlap branch included) for the fix below, without divides:
// 1/r from one SFU reciprocal square root.  inv32a = 1 / (32 a).
template <int TENSOR>
__device__ __forceinline__ void exact_pair_sfu(float dx, float dy, float dz, float fx, float fy, float fz,
                                               const PairConst &c, float inv32a, float &ox, float &oy, float &oz,
                                               bool &coincident) {
    const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    if (r2 == 0.0f) {
        if (TENSOR != T_RPY) coincident = true;
        ox = TENSOR == T_RPY ? fx : 0.0f;   // T^(0) = I for the RPY overlap form
        oy = TENSOR == T_RPY ? fy : 0.0f;
        oz = TENSOR == T_RPY ? fz : 0.0f;
        return;
    }
    const float ri = rsqrt_sfu(r2), ri2 = __fmul_rn(ri, ri);
    float A, B;
    if (TENSOR == T_RPY && r2 < c.r2min_f) {   // r < 2a: 1 - 9 r / (32 a), 3 / (32 a r)
        A = __fmaf_rn(-9.0f * inv32a, __fmul_rn(r2, ri), 1.0f);
        B = __fmul_rn(3.0f * inv32a, ri);
    } else if (TENSOR == T_OSEEN) {
        A = __fmul_rn(c.c1_f, ri);
        B = __fmul_rn(A, ri2);
    } else {
        A = __fmul_rn(ri, __fmaf_rn(c.c3_f, ri2, c.c1_f));
        B = __fmul_rn(__fmul_rn(ri, ri2), __fmaf_rn(c.m3c3_f, ri2, c.c1_f));
    }
    const float s = __fmul_rn(B, __fmaf_rn(dz, fz, __fmaf_rn(dy, fy, __fmul_rn(dx, fx))));
    ox = __fmaf_rn(s, dx, __fmul_rn(A, fx));
    oy = __fmaf_rn(s, dy, __fmul_rn(A, fy));
    oz = __fmaf_rn(s, dz, __fmul_rn(A, fz));
}

// Adds v (3 dims, half h) to the shared sum of slot `to` for every lane whose `on` is
// set: in parallel when the lanes' slots are distinct, else one entry at a time in
// lane order (each sum by the lane that owns its slot, slot mod 32).
__device__ __forceinline__ void bsym_add_sums(f2 *__restrict__ SUM, bool on, int to, int h, const float (&v)[3],
                                              int lane) {
    const unsigned grp = __match_any_sync(0xffffffffu, on ? to : -1 - lane);
    if (__all_sync(0xffffffffu, __popc(grp) == 1)) {
        if (on)
#pragma unroll
            for (int d = 0; d < 3; ++d) SUM[d * kSymSlots + to] = add_half(SUM[d * kSymSlots + to], h, v[d]);
    } else {
        unsigned act = __ballot_sync(0xffffffffu, on);
        while (act) {
            const int u = __ffs(act) - 1;
            act &= act - 1;
            const int tu = __shfl_sync(0xffffffffu, to, u), hu = __shfl_sync(0xffffffffu, h, u);
            float vu[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) vu[d] = __shfl_sync(0xffffffffu, v[d], u);
            if (lane == (tu & 31))
#pragma unroll
                for (int d = 0; d < 3; ++d) SUM[d * kSymSlots + tu] = add_half(SUM[d * kSymSlots + tu], hu, vu[d]);
        }
    }
    __syncwarp();
}

// Fix (bsym_fix_list): in place of the clamped terms of the nfix listed pairs, the
// exact ones (Yamakawa form for RPY), in both directions.  Each lane computes the
// corrections of one entry: the exact term minus the clamped one, the latter
// recomputed bit for bit.  The target sides are then added to the targets' shared
// sums, then the source sides to the sources' (bsym_add_sums).
template <int TENSOR>
__device__ __forceinline__ void bsym_fix_list(const f2 *__restrict__ S, f2 *__restrict__ SUM,
                                              const int *__restrict__ FL, int nfix, int lane, const PairConst &pc,
                                              int *err) {
    constexpr int TD = (TENSOR == T_OSEEN) ? T_OSEEN : T_RP;
    const float inv32a = 1.0f / (32.0f * static_cast<float>(pc.a));
    bool coincident = false;
    __syncwarp();   // the list and the walks' shared sums are visible
    for (int e0 = 0; e0 < nfix; e0 += 32) {
        float ct[3] = {0.0f, 0.0f, 0.0f}, cs[3] = {0.0f, 0.0f, 0.0f};
        const bool on = e0 + lane < nfix;
        int i = 0, k = 0, h = 0;
        if (on) {
            const int ent = FL[e0 + lane];
            i = ent >> 9;
            k = (ent >> 1) & 255;
            h = ent & 1;
            const float4 pi = make_float4(half_of(S[i], h), half_of(S[kSymSlots + i], h),
                                          half_of(S[2 * kSymSlots + i], h), 0.0f);
            const float4 fi = make_float4(half_of(S[3 * kSymSlots + i], h), half_of(S[4 * kSymSlots + i], h),
                                          half_of(S[5 * kSymSlots + i], h), 0.0f);
            const float4 pj = make_float4(half_of(S[k], h), half_of(S[kSymSlots + k], h),
                                          half_of(S[2 * kSymSlots + k], h), 0.0f);
            const float4 fj = make_float4(half_of(S[3 * kSymSlots + k], h), half_of(S[4 * kSymSlots + k], h),
                                          half_of(S[5 * kSymSlots + k], h), 0.0f);
            const float dx = __fsub_rn(pi.x, pj.x), dy = __fsub_rn(pi.y, pj.y), dz = __fsub_rn(pi.z, pj.z);
            float cx = 0.0f, cy = 0.0f, cz = 0.0f, ex, ey, ez;
            pair_f32<TD, true>(pi.x, pi.y, pi.z, pj, fj, pc, cx, cy, cz);
            exact_pair_sfu<TENSOR>(dx, dy, dz, fj.x, fj.y, fj.z, pc, inv32a, ex, ey, ez, coincident);
            ct[0] = __fsub_rn(ex, cx);
            ct[1] = __fsub_rn(ey, cy);
            ct[2] = __fsub_rn(ez, cz);
            float bx = 0.0f, by = 0.0f, bz = 0.0f;
            pair_f32<TD, true>(pj.x, pj.y, pj.z, pi, fi, pc, bx, by, bz);
            exact_pair_sfu<TENSOR>(-dx, -dy, -dz, fi.x, fi.y, fi.z, pc, inv32a, ex, ey, ez, coincident);
            cs[0] = __fsub_rn(ex, bx);
            cs[1] = __fsub_rn(ey, by);
            cs[2] = __fsub_rn(ez, bz);
        }
        bsym_add_sums(SUM, on, i, h, ct, lane);
        bsym_add_sums(SUM, on, k, h, cs, lane);
    }
    if (coincident) atomicOr(err, DEV_ERR_COINCIDENT);
}

// Screening, then fix (bsym_rowfix), for the row blocks p, p + 1: TL holds ntl flagged
// walks, each (source block q | rows << 8 | diagonal << 10, lanes).  rows = r for the
// tile (p + r, q) alone, 2 for the walk of both rows.  For each lane L that met a pair
// closer than 2a the warp tests L's target against the tile's 32 sources, one
// source per lane: the walk's r^2, recomputed bit for bit, and only the pairs the
// walk gave lane L.  Each pair found goes to the warp's list FL as (target slot,
// source slot, half); a list that could overflow is fixed and emptied first.
template <int TENSOR>
__device__ __noinline__ void bsym_rowfix(const f2 *__restrict__ S, f2 *__restrict__ SUM, int *__restrict__ FL,
                                         const int2 *__restrict__ TL, int ntl, int p, int lane, int nh0, int nh1,
                                         const PairConst &pc, int *err) {
    __syncwarp();   // the recorded walks are visible
    const unsigned below = (1u << lane) - 1u;
    int nfix = 0;
    for (int t = 0; t < ntl; ++t) {
        const int2 w = TL[t];
        const int q = w.x & 255, rows = (w.x >> 8) & 3;
        const bool diag = (w.x >> 10) & 1;
        const int j = 32 * q + lane;
        const f2 PX = S[j], PY = S[kSymSlots + j], PZ = S[2 * kSymSlots + j];
        for (int r = (rows == 1 ? 1 : 0); r <= (rows == 0 ? 0 : 1); ++r) {
            unsigned who = static_cast<unsigned>(w.y);
            while (who) {
                const int L = __ffs(who) - 1;
                who &= who - 1;
                if (nfix > kSymFixCap - 64) {   // room for one target's 32 sources x 2 halves
                    bsym_fix_list<TENSOR>(S, SUM, FL, nfix, lane, pc, err);
                    nfix = 0;
                }
                const int i = 32 * (p + r) + L;
                const int m = (lane - L) & 31;   // the step of the walk at which lane L met this lane's source
                const bool mine = !diag || (m >= 1 && m <= 15) || (m == 16 && L < 16);
                const f2 dx = sub2(S[i], PX), dy = sub2(S[kSymSlots + i], PY), dz = sub2(S[2 * kSymSlots + i], PZ);
                const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                float ra, rb;
                upk2(r2, ra, rb);
                const unsigned h0 = __ballot_sync(0xffffffffu, mine && i < nh0 && j < nh0 && ra < pc.r2min_f);
                if ((h0 >> lane) & 1u) FL[nfix + __popc(h0 & below)] = (i << 9) | (j << 1);
                nfix += __popc(h0);
                const unsigned h1 = __ballot_sync(0xffffffffu, mine && i < nh1 && j < nh1 && rb < pc.r2min_f);
                if ((h1 >> lane) & 1u) FL[nfix + __popc(h1 & below)] = (i << 9) | (j << 1) | 1;
                nfix += __popc(h1);
            }
        }
    }
    if (nfix) bsym_fix_list<TENSOR>(S, SUM, FL, nfix, lane, pc, err);
}

template <int TENSOR>
__global__ void __launch_bounds__(128, 3) batched_sym_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    f2 *S = reinterpret_cast<f2 *>(smem + static_cast<size_t>(wid) * kSymWarpSmem);    // x y z Fx Fy Fz
    f2 *SUM = S + 6 * kSymSlots;                                                         // sums x y z
    int *FL = reinterpret_cast<int *>(SUM + 3 * kSymSlots);                              // pair list
    int2 *TL = reinterpret_cast<int2 *>(FL + kSymFixCap);                                // flagged walks
    const float4 *frcm = static_cast<const float4 *>(a.frcm);
    PairConst2 c2{};
    c2.c1 = pk2(a.pc.c1_f, a.pc.c1_f);
    c2.c3 = pk2(a.pc.c3_f, a.pc.c3_f);
    c2.m3c3 = pk2(a.pc.m3c3_f, a.pc.m3c3_f);
    c2.r2min = a.pc.r2min_f;
    const float m0dt = static_cast<float>(a.pc.mu0 * a.dt);
    const float far = 1.0e4f * static_cast<float>(a.pc.a), gap = 4.0f * static_cast<float>(a.pc.a);
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.ctr, 1ULL);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= static_cast<unsigned long long>(a.nblk)) break;
        const int4 task = a.stask[t];
        const int cl[2] = {task.x, task.y};
        const int nb = task.z;
        int o[2], nh[2];
        for (int h = 0; h < 2; ++h) {
            o[h] = cl[h] >= 0 ? a.off[cl[h]] : 0;
            nh[h] = cl[h] >= 0 ? a.off[cl[h] + 1] - o[h] : 0;
        }
        // stage both clusters, interleaved; padding slots far away, 4a apart, zero force
        for (int k = lane; k < 32 * nb; k += 32) {
            float v[2][6];
            for (int h = 0; h < 2; ++h) {
                if (k < nh[h]) {
                    const float4 r = a.rel[o[h] + k], f = frcm[o[h] + k];
                    v[h][0] = r.x; v[h][1] = r.y; v[h][2] = r.z;
                    v[h][3] = f.x; v[h][4] = f.y; v[h][5] = f.z;
                } else {
                    v[h][0] = far + gap * static_cast<float>(k);
                    v[h][1] = v[h][2] = v[h][3] = v[h][4] = v[h][5] = 0.0f;
                }
            }
            for (int d = 0; d < 6; ++d) S[d * kSymSlots + k] = pk2(v[0][d], v[1][d]);
            for (int d = 0; d < 3; ++d) SUM[d * kSymSlots + k] = 0ull;
        }
        __syncwarp();
        // the block rows in pairs (p, p + 1): their tiles against the blocks q > p + 1
        // share each walk of q (bsym_tile2); the rest run one row at a time
        for (int p = 0; p < nb; p += 2) {
            const bool two = p + 1 < nb;
            f2 T[2][6];
            for (int r = 0; r < 2; ++r) {
                const int i = 32 * (p + r) + lane;   // (a padding row when !two: never used)
                for (int d = 0; d < 6; ++d) T[r][d] = S[d * kSymSlots + i];
            }
            // (hi, lo) sums of the rows' targets [row][half][dim]
            float hs[2][2][3] = {}, ls[2][2][3] = {};
            auto fold = [&](int r, const f2 (&A)[3]) {
                for (int d = 0; d < 3; ++d) {
                    float v0, v1;
                    upk2(A[d], v0, v1);
                    fold2(hs[r][0][d], ls[r][0][d], v0);
                    fold2(hs[r][1][d], ls[r][1][d], v1);
                }
            };
            int ntl = 0;   // walks of rows p, p + 1 that met a pair closer than 2a
            auto record = [&](int rows, int q, bool diag, unsigned who) {
                if (lane == 0) TL[ntl] = make_int2(q | (rows << 8) | (diag ? 1 << 10 : 0), static_cast<int>(who));
                ++ntl;
            };
            auto one = [&](int r, int q) {   // tile (p + r, q) alone
                f2 A[3] = {0ull, 0ull, 0ull};
                float mn0 = 3.0e38f, mn1 = 3.0e38f;
                if (q == p + r)
                    bsym_tile<TENSOR, true>(S, SUM, q, lane, T[r][0], T[r][1], T[r][2], T[r][3], T[r][4], T[r][5], c2,
                                            A[0], A[1], A[2], mn0, mn1);
                else
                    bsym_tile<TENSOR, false>(S, SUM, q, lane, T[r][0], T[r][1], T[r][2], T[r][3], T[r][4], T[r][5],
                                             c2, A[0], A[1], A[2], mn0, mn1);
                fold(r, A);
                const unsigned who = __ballot_sync(0xffffffffu, fminf(mn0, mn1) < c2.r2min);
                if (who) record(r, q, q == p + r, who);   // rare: pairs closer than 2a
            };
            one(0, p);
            if (two) {
                one(0, p + 1);
                one(1, p + 1);
            }
            for (int q = p + (two ? 2 : 1); q < nb; ++q) {
                if (!two) {
                    one(0, q);
                    continue;
                }
                f2 A0[3] = {0ull, 0ull, 0ull}, A1[3] = {0ull, 0ull, 0ull};
                float mn0 = 3.0e38f, mn1 = 3.0e38f;
                bsym_tile2<TENSOR>(S, SUM, q, lane, T[0], T[1], c2, A0, A1, mn0, mn1);
                fold(0, A0);
                fold(1, A1);
                const unsigned who = __ballot_sync(0xffffffffu, fminf(mn0, mn1) < c2.r2min);
                if (who) record(2, q, false, who);   // (a lane's flag covers both of its targets)
            }
            if (ntl) bsym_rowfix<TENSOR>(S, SUM, FL, TL, ntl, p, lane, nh[0], nh[1], a.pc, a.err);
            // rows p (and p + 1) are complete: finalise their particles
            for (int r = 0; r < (two ? 2 : 1); ++r)
            for (int h = 0; h < 2; ++h) {
                const int i = 32 * (p + r) + lane;
                if (i >= nh[h]) continue;
                float V[3];
                for (int d = 0; d < 3; ++d) {
                    float hh = hs[r][h][d], ll = ls[r][h][d];
                    fold2(hh, ll, half_of(SUM[d * kSymSlots + i], h));
                    fold2(hh, ll, half_of(S[(3 + d) * kSymSlots + i], h));   // mu_ii F_i / mu0 = F_i
                    V[d] = __fadd_rn(hh, ll);
                }
                const size_t g = static_cast<size_t>(o[h] + i);
                const float ux = __fmul_rn(m0dt, V[0]), uy = __fmul_rn(m0dt, V[1]), uz = __fmul_rn(m0dt, V[2]);
                if (!isfinite(ux) || !isfinite(uy) || !isfinite(uz)) atomicOr(a.err, DEV_ERR_NONFINITE);
                const double nx = a.x64[3 * g] + static_cast<double>(ux);
                const double ny = a.x64[3 * g + 1] + static_cast<double>(uy);
                const double nz = a.x64[3 * g + 2] + static_cast<double>(uz);
                a.x64n[3 * g] = nx;
                a.x64n[3 * g + 1] = ny;
                a.x64n[3 * g + 2] = nz;
                const size_t an = static_cast<size_t>(o[h]);
                a.reln[g] = make_float4(static_cast<float>(nx - a.x64[3 * an]), static_cast<float>(ny - a.x64[3 * an + 1]),
                                        static_cast<float>(nz - a.x64[3 * an + 2]), 0.0f);
            }
        }
        __syncwarp();   // the warp's shared memory is free for the next task
    }
}

// Launch shapes: FP64 -- warps per CTA (one cluster per warp) x resident CTAs;
// FP32C -- block of BT = 32 warps threads (R targets each) x resident CTAs.
static size_t shape_smem(int mode, const BatchShape &sh) {
    if (mode == MODE_FP64) return static_cast<size_t>(sh.warps) * kWarpStage;
    if (sh.r == 0) return static_cast<size_t>(sh.warps) * kSymWarpSmem;
    const size_t bt = 32 * static_cast<size_t>(sh.warps);
    const int len = sh.warps == 4 ? (sh.r == 2 ? block_stage_len<128, 2>() : block_stage_len<128, 1>())
                                  : (sh.r == 2 ? block_stage_len<256, 2>() : block_stage_len<256, 1>());
    return 6 * sizeof(float) * static_cast<size_t>(len) + kNoteCap * static_cast<size_t>(sh.r) * bt * sizeof(int);
}

template <int TENSOR>
static void *batched_fn_t(int mode, const BatchShape &sh) {
    if (mode == MODE_FP64) return reinterpret_cast<void *>(&batched_kernel<TENSOR>);
    if (sh.r == 0) return reinterpret_cast<void *>(&batched_sym_kernel<TENSOR>);
    if (sh.r == 2)
        return sh.warps == 4 ? reinterpret_cast<void *>(&batched_blocks_kernel<TENSOR, 128, 2>)
                             : reinterpret_cast<void *>(&batched_blocks_kernel<TENSOR, 256, 2>);
    return sh.warps == 4 ? reinterpret_cast<void *>(&batched_blocks_kernel<TENSOR, 128, 1>)
                         : reinterpret_cast<void *>(&batched_blocks_kernel<TENSOR, 256, 1>);
}

static void *batched_fn(int tensor, int mode, const BatchShape &sh) {
    if (tensor == T_RPY) return batched_fn_t<T_RPY>(mode, sh);
    if (tensor == T_RP) return batched_fn_t<T_RP>(mode, sh);
    return batched_fn_t<T_OSEEN>(mode, sh);
}

static cudaError_t batch_launch(sd_batch *b, cudaStream_t st, double dt, const BatchShape &sh, bool prof) {
    cudaError_t e = cudaMemsetAsync(b->ctr, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    BatchArgs a;
    a.off = b->d_off;
    a.order = b->d_order;
    a.qperm = b->qperm;
    a.qcl = b->qcl;
    a.cbeg = b->cbeg;
    a.cend = b->cend;
    a.canchor = b->canchor;
    a.tq = b->tq;
    a.stask = b->stask;
    a.P = b->P;
    a.M2 = b->M2;
    if (b->mode == MODE_FP32C && sh.r == 0) {
        a.nblk = b->nstask;   // warp tasks
    } else {
        const int slots = (b->mode == MODE_FP32C && sh.r == 2) ? b->M2 : b->P;
        a.nblk = (slots + 32 * sh.warps - 1) / (32 * sh.warps);
    }
    a.x64 = b->x64[b->cur];
    a.x64n = b->x64[1 - b->cur];
    a.rel = b->rel[b->cur];
    a.reln = b->rel[1 - b->cur];
    a.panchor = b->panchor;
    a.F64 = b->F64;
    a.frcm = b->frcm;
    a.ctr = b->ctr;
    a.C = b->C;
    a.pc = b->pc;
    a.dt = dt;
    a.err = b->d_err;
    const size_t smem = shape_smem(b->mode, sh);
    const int grid = b->num_sms * sh.ctas_per_sm;
    void *fn = batched_fn(b->tensor, b->mode, sh);
    int kk = -1;
    if (prof && b->prof.on && b->prof.npending < Profiler::kMaxPending) {
        kk = b->prof.npending;
        if (kk >= b->prof.nevents) {
            cudaEventCreate(&b->prof.ev0[kk]);
            cudaEventCreate(&b->prof.ev1[kk]);
            b->prof.nevents = kk + 1;
        }
        b->prof.kind[kk] = SD_KERNEL_BATCHED;
        cudaEventRecord(b->prof.ev0[kk], st);
    }
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(32 * sh.warps), args, smem, st);
    if (kk >= 0) {
        cudaEventRecord(b->prof.ev1[kk], st);
        ++b->prof.npending;
    }
    ++b->launches;
    b->cur = 1 - b->cur;
    return e;
}

static sd_status batch_sync_check(sd_batch *b) {
    SD_CUDA(cudaStreamSynchronize(b->stream));
    int bits = 0;
    SD_CUDA(cudaMemcpy(&bits, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (bits) SD_CUDA(cudaMemset(b->d_err, 0, sizeof(int)));
    if (bits & (DEV_ERR_TIMEOUT | DEV_ERR_QUEUE)) return set_error(SD_ERR_TIMEOUT, "batched kernel gave up");
    if (bits & DEV_ERR_COINCIDENT) return set_error(SD_ERR_COINCIDENT, "two distinct particles at zero separation");
    if (bits & DEV_ERR_NONFINITE) return set_error(SD_ERR_NONFINITE, "non-finite value in positions or forces");
    if (bits & DEV_ERR_BOUNDS) return set_error(SD_ERR_INTERNAL, "a device-side index check failed");
    return SD_OK;
}

static void *balloc(sd_batch *b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b->al.alloc) return b->al.alloc(bytes, b->al.ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void bfree(sd_batch *b, void *p) {
    if (!p) return;
    if (b->al.free) b->al.free(p, b->al.ctx);
    else cudaFree(p);
}

template <typename V4>
__global__ void batch_stage_forces_kernel(const double *__restrict__ fext, double gx, double gy, double gz,
                                          double *__restrict__ F, V4 *__restrict__ m, int P, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const double f0 = fext[3 * i] + gx, f1 = fext[3 * i + 1] + gy, f2 = fext[3 * i + 2] + gz;
    if (!isfinite(f0) || !isfinite(f1) || !isfinite(f2)) atomicOr(err, DEV_ERR_NONFINITE);
    F[3 * i] = f0;
    F[3 * i + 1] = f1;
    F[3 * i + 2] = f2;
    V4 v;
    v.x = f0;
    v.y = f1;
    v.z = f2;
    v.w = 0;
    m[i] = v;
}

__global__ void batch_check_pos_kernel(const double *__restrict__ x, int P, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * P) return;
    if (!isfinite(x[i])) atomicOr(err, DEV_ERR_NONFINITE);
}

// FP32 position of every particle relative to the first particle of its cluster
// (the reference point the FP32C block kernel stages from).
__global__ void batch_rel_kernel(const double *__restrict__ x, const int32_t *__restrict__ panchor,
                                 float4 *__restrict__ rel, int P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const size_t an = static_cast<size_t>(panchor[i]);
    rel[i] = make_float4(static_cast<float>(x[3 * static_cast<size_t>(i)] - x[3 * an]),
                         static_cast<float>(x[3 * static_cast<size_t>(i) + 1] - x[3 * an + 1]),
                         static_cast<float>(x[3 * static_cast<size_t>(i) + 2] - x[3 * an + 2]), 0.0f);
}

static cudaError_t batch_stage_forces(sd_batch *b) {
    if (b->P == 0) return cudaSuccess;
    const int nb = (b->P + 255) / 256;
    const double *g = b->cfg.gravity;
    if (b->mode == MODE_FP64)
        batch_stage_forces_kernel<dbl4><<<nb, 256, 0, b->stream>>>(b->fext64, g[0], g[1], g[2], b->F64,
                                                                   static_cast<dbl4 *>(b->frcm), b->P, b->d_err);
    else
        batch_stage_forces_kernel<float4><<<nb, 256, 0, b->stream>>>(b->fext64, g[0], g[1], g[2], b->F64,
                                                                     static_cast<float4 *>(b->frcm), b->P, b->d_err);
    ++b->launches;
    return cudaGetLastError();
}

static void drop_batch_graph(sd_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
}

constexpr int kBatchGraphSteps = 16;

static sd_status capture_batch(sd_batch *b, double dt) {
    drop_batch_graph(b);
    cudaGraph_t graph = nullptr;
    SD_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    const int64_t l0 = b->launches;
    for (int k = 0; k < kBatchGraphSteps && e == cudaSuccess; ++k) e = batch_launch(b, b->cap, dt, b->shapes[b->choice], false);
    b->launches = l0;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_status(e, "capture of batched steps");
    }
    if (e2 != cudaSuccess) return cuda_status(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate");
    b->g_dt = dt;
    b->g_choice = b->choice;
    b->g_cur = b->cur;   // 16 launches flip the buffers back: the graph starts and ends here
    return SD_OK;
}

}  // namespace sd

using namespace sd;

extern "C" {

sd_status sd_batch_create(const sd_config *cfg, const int32_t *offsets, int32_t nclusters, sd_batch **out) {
    if (!out) return set_error(SD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return set_error(SD_ERR_ARG, "cfg is NULL");
    if (nclusters < 0 || (nclusters > 0 && !offsets)) return set_error(SD_ERR_ARG, "offsets / nclusters");
    if (!(cfg->a > 0.0) || !(cfg->eta > 0.0) || !std::isfinite(cfg->a) || !std::isfinite(cfg->eta))
        return set_error(SD_ERR_ARG, "a and eta must be finite and > 0");
    if (cfg->tensor < 0 || cfg->tensor > 2) return set_error(SD_ERR_ARG, "unknown tensor");
    if (cfg->prec < 0 || cfg->prec > 2) return set_error(SD_ERR_ARG, "unknown precision");
    for (int d = 0; d < 3; ++d) {
        if (cfg->box[d] != 0.0) return set_error(SD_ERR_UNSUPPORTED, "periodic boxes are not implemented for batches");
        if (!std::isfinite(cfg->gravity[d])) return set_error(SD_ERR_ARG, "gravity must be finite");
    }
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
        return set_error(SD_ERR_ARG, "alloc and free callbacks must be given together");
    if (cfg->lubrication != 0) return set_error(SD_ERR_UNSUPPORTED, "lubrication is not implemented for batches");
    if (nclusters > 0 && offsets[0] != 0) return set_error(SD_ERR_ARG, "offsets[0] must be 0");
    int maxn = 0;
    for (int c = 0; c < nclusters; ++c) {
        const int nc = offsets[c + 1] - offsets[c];
        if (nc < 0 || nc > kMaxCluster) return set_error(SD_ERR_ARG, "cluster sizes must be in [0, 256]");
        maxn = std::max(maxn, nc);
    }
    const int P = nclusters > 0 ? offsets[nclusters] : 0;

    sd_batch *b = new (std::nothrow) sd_batch();
    if (!b) return set_error(SD_ERR_OOM, "host allocation");
    b->cfg = *cfg;
    b->C = nclusters;
    b->P = P;
    b->maxn = maxn;
    b->mode = cfg->prec == SD_PREC_FP64 ? MODE_FP64 : MODE_FP32C;
    b->tensor = cfg->tensor;
    b->device = cfg->device;
    b->stream = static_cast<cudaStream_t>(cfg->stream);
    b->al.alloc = cfg->alloc;
    b->al.free = cfg->free;
    b->al.ctx = cfg->alloc_ctx;
    const double a = cfg->a;
    PairConst &pc = b->pc;
    pc.a = a;
    pc.two_a = 2 * a;
    pc.mu0 = 1.0 / (6.0 * 3.14159265358979323846 * cfg->eta * a);
    pc.r2min_d = 4 * a * a;
    pc.c1_d = 0.75 * a;
    pc.c3_d = 0.5 * a * a * a;
    pc.m3c3_d = -1.5 * a * a * a;
    pc.r2min_f = static_cast<float>(pc.r2min_d);
    pc.c1_f = static_cast<float>(pc.c1_d);
    pc.c3_f = static_cast<float>(pc.c3_d);
    pc.m3c3_f = static_cast<float>(pc.m3c3_d);

    auto fail = [&](sd_status st, const std::string &m) {
        sd_batch_destroy(b);
        return set_error(st, m);
    };
    if (cudaSetDevice(b->device) != cudaSuccess) return fail(SD_ERR_CUDA, "cudaSetDevice");
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(SD_ERR_CUDA, "stream");
    const size_t p3 = 3 * static_cast<size_t>(std::max(P, 1));
    const size_t vb = b->mode == MODE_FP64 ? sizeof(dbl4) : sizeof(float4);
    b->d_off = static_cast<int32_t *>(balloc(b, sizeof(int32_t) * (nclusters + 1)));
    b->d_order = static_cast<int32_t *>(balloc(b, sizeof(int32_t) * std::max(nclusters, 1)));
    b->x64[0] = static_cast<double *>(balloc(b, p3 * sizeof(double)));
    b->x64[1] = static_cast<double *>(balloc(b, p3 * sizeof(double)));
    const size_t c1 = static_cast<size_t>(std::max(nclusters, 1));
    b->qperm = static_cast<int32_t *>(balloc(b, sizeof(int32_t) * std::max(P, 1)));
    b->panchor = static_cast<int32_t *>(balloc(b, sizeof(int32_t) * std::max(P, 1)));
    for (int k = 0; k < 2; ++k) b->rel[k] = static_cast<float4 *>(balloc(b, sizeof(float4) * std::max(P, 1)));
    b->qcl = static_cast<int32_t *>(balloc(b, sizeof(int32_t) * std::max(P, 1)));
    b->cbeg = static_cast<int32_t *>(balloc(b, sizeof(int32_t) * c1));
    b->cend = static_cast<int32_t *>(balloc(b, sizeof(int32_t) * c1));
    b->canchor = static_cast<int32_t *>(balloc(b, sizeof(int32_t) * c1));
    b->F64 = static_cast<double *>(balloc(b, p3 * sizeof(double)));
    b->fext64 = static_cast<double *>(balloc(b, p3 * sizeof(double)));
    b->frcm = balloc(b, std::max(P, 1) * vb);
    b->ctr = static_cast<unsigned long long *>(balloc(b, sizeof(unsigned long long)));
    b->d_err = static_cast<int *>(balloc(b, sizeof(int)));
    if (!b->d_off || !b->d_order || !b->x64[0] || !b->x64[1] || !b->F64 || !b->fext64 || !b->frcm || !b->ctr ||
        !b->d_err || !b->qperm || !b->qcl || !b->cbeg || !b->cend || !b->canchor || !b->panchor || !b->rel[0] ||
        !b->rel[1])
        return fail(SD_ERR_OOM, "device allocation of batch buffers");

    // largest-first order (stable in the cluster index)
    std::vector<int32_t> order(nclusters);
    for (int c = 0; c < nclusters; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return offsets[x + 1] - offsets[x] > offsets[y + 1] - offsets[y];
    });
    // the largest-first sequence of particles (block kernel)
    std::vector<int32_t> qperm(std::max(P, 1)), qcl(std::max(P, 1)), cbeg(c1), cend(c1), canchor(c1),
        panchor(std::max(P, 1));
    for (int c = 0; c < nclusters; ++c)
        for (int i = offsets[c]; i < offsets[c + 1]; ++i) panchor[i] = offsets[c];
    int pos = 0;
    for (int k = 0; k < nclusters; ++k) {
        const int c = order[k], o = offsets[c], n = offsets[c + 1] - o;
        cbeg[k] = pos;
        canchor[k] = o;
        for (int i = 0; i < n; ++i) {
            qperm[pos + i] = o + i;
            qcl[pos + i] = k;
        }
        pos += n;
        cend[k] = pos;
    }
    // two-target slots over the same sequence: pairs of neighbours in a cluster, an odd
    // cluster's last target alone (stored as ~q)
    std::vector<int32_t> tq;
    tq.reserve(static_cast<size_t>(P) / 2 + nclusters + 1);
    for (int k = 0; k < nclusters; ++k)
        for (int q = cbeg[k]; q < cend[k]; q += 2) tq.push_back(q + 1 < cend[k] ? q : ~q);
    b->M2 = static_cast<int>(tq.size());
    b->tq = static_cast<int32_t *>(balloc(b, sizeof(int32_t) * std::max<size_t>(tq.size(), 1)));
    if (!b->tq) return fail(SD_ERR_OOM, "device allocation of batch buffers");
    // symmetric kernel: neighbouring non-empty clusters of the largest-first order in
    // pairs, each pair with its number of 32-particle blocks
    std::vector<int4> stask;
    {
        std::vector<int> ne;
        for (int k = 0; k < nclusters; ++k)
            if (offsets[order[k] + 1] > offsets[order[k]]) ne.push_back(order[k]);
        for (size_t k = 0; k < ne.size(); k += 2) {
            const int cA = ne[k], cB = k + 1 < ne.size() ? ne[k + 1] : -1;
            const int nA = offsets[cA + 1] - offsets[cA], nB = cB >= 0 ? offsets[cB + 1] - offsets[cB] : 0;
            stask.push_back(make_int4(cA, cB, (std::max(nA, nB) + 31) / 32, 0));
        }
    }
    b->nstask = static_cast<int>(stask.size());
    b->stask = static_cast<int4 *>(balloc(b, sizeof(int4) * std::max<size_t>(stask.size(), 1)));
    if (!b->stask) return fail(SD_ERR_OOM, "device allocation of batch buffers");
    cudaStream_t st = b->stream;
    cudaError_t e = cudaMemcpyAsync(b->d_off, offsets, sizeof(int32_t) * (nclusters + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nclusters > 0)
        e = cudaMemcpyAsync(b->d_order, order.data(), sizeof(int32_t) * nclusters, cudaMemcpyHostToDevice, st);
    // (pageable host vectors: cudaMemcpyAsync returns once they are staged, so they may go out of scope)
    for (auto [dst, src, cnt] : {std::make_tuple(b->qperm, qperm.data(), static_cast<size_t>(P)),
                                 std::make_tuple(b->qcl, qcl.data(), static_cast<size_t>(P)),
                                 std::make_tuple(b->panchor, panchor.data(), static_cast<size_t>(P)),
                                 std::make_tuple(b->cbeg, cbeg.data(), static_cast<size_t>(nclusters)),
                                 std::make_tuple(b->cend, cend.data(), static_cast<size_t>(nclusters)),
                                 std::make_tuple(b->canchor, canchor.data(), static_cast<size_t>(nclusters)),
                                 std::make_tuple(b->tq, tq.data(), tq.size())})
        if (e == cudaSuccess && cnt > 0)
            e = cudaMemcpyAsync(dst, src, sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !stask.empty())
        e = cudaMemcpyAsync(b->stask, stask.data(), sizeof(int4) * stask.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->fext64, 0, p3 * sizeof(double), st);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMemsetAsync(b->x64[k], 0, p3 * sizeof(double), st);
    if (e == cudaSuccess) e = batch_stage_forces(b);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SD_ERR_CUDA, std::string("batch initialisation: ") + cudaGetErrorString(e));

    // candidate launch shapes that fit: FP64 -- warps per CTA x resident CTAs per SM;
    // FP32C -- blocks of 128 or 256 threads (4 or 8 warps) with 1 or 2 targets per
    // thread x resident CTAs per SM
    for (int r : {1, 2, 0}) {
        if (r != 1 && b->mode != MODE_FP32C) continue;
        for (int w : {4, 8}) {
            if (r == 0 && w != 4) continue;   // symmetric kernel: 4 warps (tasks) per CTA
            const BatchShape sh1{w, 1, r};
            void *fn = batched_fn(b->tensor, b->mode, sh1);
            const size_t smem = shape_smem(b->mode, sh1);
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
                cudaSuccess)
                return fail(SD_ERR_CUDA, "shared-memory opt-in for the batched kernel");
            int occ = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * w, smem) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            for (int c = 1; c <= occ; ++c) b->shapes.push_back({w, c, r});
        }
    }
    if (b->shapes.empty()) return fail(SD_ERR_CUDA, "no launch shape fits the device");
    b->choice = -1;   // autotune on first step
    *out = b;
    return SD_OK;
}

void sd_batch_destroy(sd_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_batch_graph(b);
    for (int k = 0; k < b->prof.nevents; ++k) {
        cudaEventDestroy(b->prof.ev0[k]);
        cudaEventDestroy(b->prof.ev1[k]);
    }
    void *bufs[] = {b->d_off, b->d_order, b->x64[0], b->x64[1], b->F64, b->fext64, b->frcm, b->ctr, b->d_err,
                    b->qperm, b->qcl, b->cbeg, b->cend, b->canchor, b->panchor, b->rel[0], b->rel[1], b->tq,
                    b->stask};
    for (void *p : bufs) bfree(b, p);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

sd_status sd_batch_set_positions(sd_batch *b, const double *xyz, int on_device) {
    if (!b) return set_error(SD_ERR_ARG, "batch is NULL");
    if (on_device != 0 && on_device != 1) return set_error(SD_ERR_ARG, "on_device must be 0 or 1");
    if (b->P > 0 && !xyz) return set_error(SD_ERR_ARG, "positions pointer is NULL");
    cudaSetDevice(b->device);
    if (!on_device)
        for (size_t k = 0; k < 3 * static_cast<size_t>(b->P); ++k)
            if (!std::isfinite(xyz[k])) return set_error(SD_ERR_NONFINITE, "non-finite position");
    if (b->P > 0) {
        SD_CUDA(cudaMemcpyAsync(b->x64[b->cur], xyz, 3 * sizeof(double) * b->P,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
        batch_check_pos_kernel<<<(3 * b->P + 255) / 256, 256, 0, b->stream>>>(b->x64[b->cur], b->P, b->d_err);
        ++b->launches;
        if (b->mode != MODE_FP64) {
            batch_rel_kernel<<<(b->P + 255) / 256, 256, 0, b->stream>>>(b->x64[b->cur], b->panchor, b->rel[b->cur],
                                                                       b->P);
            ++b->launches;
        }
        SD_CUDA(cudaGetLastError());
    }
    b->pos_set = true;
    return on_device ? SD_OK : batch_sync_check(b);
}

sd_status sd_batch_get_positions(sd_batch *b, double *xyz, int on_device) {
    if (!b) return set_error(SD_ERR_ARG, "batch is NULL");
    if (on_device != 0 && on_device != 1) return set_error(SD_ERR_ARG, "on_device must be 0 or 1");
    if (b->P > 0 && !xyz) return set_error(SD_ERR_ARG, "positions pointer is NULL");
    if (!b->pos_set) return set_error(SD_ERR_STATE, "positions were never set");
    cudaSetDevice(b->device);
    if (b->P > 0)
        SD_CUDA(cudaMemcpyAsync(xyz, b->x64[b->cur], 3 * sizeof(double) * b->P,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    return on_device ? SD_OK : batch_sync_check(b);
}

sd_status sd_batch_set_forces(sd_batch *b, const double *f, int on_device) {
    if (!b) return set_error(SD_ERR_ARG, "batch is NULL");
    if (on_device != 0 && on_device != 1) return set_error(SD_ERR_ARG, "on_device must be 0 or 1");
    if (b->P > 0 && !f) return set_error(SD_ERR_ARG, "forces pointer is NULL");
    cudaSetDevice(b->device);
    if (!on_device)
        for (size_t k = 0; k < 3 * static_cast<size_t>(b->P); ++k)
            if (!std::isfinite(f[k])) return set_error(SD_ERR_NONFINITE, "non-finite force");
    if (b->P > 0) {
        SD_CUDA(cudaMemcpyAsync(b->fext64, f, 3 * sizeof(double) * b->P,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
        SD_CUDA(batch_stage_forces(b));
    }
    return on_device ? SD_OK : batch_sync_check(b);
}

sd_status sd_batch_synchronize(sd_batch *b) {
    if (!b) return set_error(SD_ERR_ARG, "batch is NULL");
    cudaSetDevice(b->device);
    return batch_sync_check(b);
}

sd_status sd_batch_autotune(sd_batch *b, int32_t *choice) {
    if (!b) return set_error(SD_ERR_ARG, "batch is NULL");
    if (!b->pos_set) return set_error(SD_ERR_STATE, "positions were never set");
    cudaSetDevice(b->device);
    if (b->C == 0 || b->P == 0) {
        b->choice = 0;
        if (choice) *choice = 0;
        return SD_OK;
    }
    // time every shape on a scratch copy of the positions (dt = 0 keeps them fixed)
    cudaEvent_t e0, e1;
    SD_CUDA(cudaEventCreate(&e0));
    SD_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best = 0;
    const int64_t l0 = b->launches;
    for (int k = 0; k < static_cast<int>(b->shapes.size()); ++k) {
        const BatchShape &sh = b->shapes[k];
        cudaError_t e = cudaSuccess;
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = batch_launch(b, b->stream, 0.0, sh, false);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = batch_launch(b, b->stream, 0.0, sh, false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_status(e, "autotune launch");
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = k;
        }
    }
    b->launches = l0;   // tuning launches are not part of the user's work
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->choice = best;
    drop_batch_graph(b);
    if (choice) *choice = best;
    return batch_sync_check(b);
}

int32_t sd_batch_shape_count(const sd_batch *b) { return b ? static_cast<int32_t>(b->shapes.size()) : 0; }

sd_status sd_batch_shape_info(const sd_batch *b, int32_t k, int32_t *threads, int32_t *ctas_per_sm,
                              int32_t *targets_per_thread) {
    if (!b) return set_error(SD_ERR_ARG, "batch is NULL");
    if (k < 0 || k >= static_cast<int32_t>(b->shapes.size())) return set_error(SD_ERR_ARG, "shape index out of range");
    const BatchShape &sh = b->shapes[k];
    if (threads) *threads = 32 * sh.warps;
    if (ctas_per_sm) *ctas_per_sm = sh.ctas_per_sm;
    if (targets_per_thread) *targets_per_thread = sh.r;
    return SD_OK;
}

sd_status sd_batch_set_shape(sd_batch *b, int32_t k) {
    if (!b) return set_error(SD_ERR_ARG, "batch is NULL");
    if (k < 0 || k >= static_cast<int32_t>(b->shapes.size())) return set_error(SD_ERR_ARG, "shape index out of range");
    cudaSetDevice(b->device);
    b->choice = k;
    drop_batch_graph(b);
    return SD_OK;
}

sd_status sd_step_batched(sd_batch *b, double dt, int64_t nsteps) {
    NvtxRange nvtx_range("sd_step_batched");
    if (!b) return set_error(SD_ERR_ARG, "batch is NULL");
    if (nsteps < 0 || !std::isfinite(dt)) return set_error(SD_ERR_ARG, "nsteps must be >= 0 and dt finite");
    if (!b->pos_set) return set_error(SD_ERR_STATE, "positions were never set");
    if (b->C == 0 || b->P == 0 || nsteps == 0) return SD_OK;
    cudaSetDevice(b->device);
    if (b->choice < 0) {
        sd_status s = sd_batch_autotune(b, nullptr);
        if (s != SD_OK) return s;
    }
    int64_t left = nsteps;
    if (!b->prof.on) {
        while (left >= kBatchGraphSteps) {
            if (!b->gexec || b->g_dt != dt || b->g_choice != b->choice || b->g_cur != b->cur) {
                sd_status s = capture_batch(b, dt);
                if (s != SD_OK) return s;
            }
            SD_CUDA(cudaGraphLaunch(b->gexec, b->stream));
            b->launches += kBatchGraphSteps;
            left -= kBatchGraphSteps;
        }
    }
    for (; left > 0; --left) SD_CUDA(batch_launch(b, b->stream, dt, b->shapes[b->choice], true));
    return SD_OK;
}

sd_status sd_batch_profile(sd_batch *b, int on) {
    if (!b) return set_error(SD_ERR_ARG, "batch is NULL");
    cudaSetDevice(b->device);
    SD_CUDA(cudaStreamSynchronize(b->stream));
    b->prof.on = on != 0;
    b->prof.npending = 0;
    for (int k = 0; k < SD_KERNEL_COUNT; ++k) {
        b->prof.ms[k] = 0;
        b->prof.launches[k] = 0;
    }
    return SD_OK;
}

sd_status sd_batch_profile_read(sd_batch *b, int kernel, double *ms, int64_t *launches) {
    if (!b || kernel < 0 || kernel >= SD_KERNEL_COUNT) return set_error(SD_ERR_ARG, "bad batch or kernel id");
    cudaSetDevice(b->device);
    Profiler &p = b->prof;
    for (int k = 0; k < p.npending; ++k) {
        float t = 0.0f;
        SD_CUDA(cudaEventSynchronize(p.ev1[k]));
        SD_CUDA(cudaEventElapsedTime(&t, p.ev0[k], p.ev1[k]));
        p.ms[p.kind[k]] += t;
        p.launches[p.kind[k]] += 1;
    }
    p.npending = 0;
    if (ms) *ms = p.ms[kernel];
    if (launches) *launches = p.launches[kernel];
    return SD_OK;
}

int64_t sd_batch_launch_count(const sd_batch *b) { return b ? b->launches : 0; }

}  // extern "C"
