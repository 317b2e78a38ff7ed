// epilogue.cu -- the FP64 parts of the mobility product and the Euler update
// (Sec. 3.1, steps 1 and 3), around the all-pairs kernel:
//
//   near pass (before the all-pairs kernel), per particle i:
//     C_i = sum_{j: |r_ij| < r_near} [Texact(r_ij) F_j - Tdense(r_ij) F_j]
//     for both variants of Tdense (r^2 clamped to (2a)^2, and unclamped), and a
//     device flag raised when some pair is closer than r_safe (then the
//     all-pairs kernel clamps every tile, else only the tiles holding self pairs);
//     in a Verlet step the flag comes from the step's check kernel instead, and the
//     near pass runs beside the all-pairs kernel;
//   epilogue (after it):
//     V_i = sum over the CTA slots of the dense partial sums (and, after the
//           symmetric kernel, over the source-side slots of the particle's block
//           column), in a fixed order
//         + F_i - Tdense(0) F_i                  self term mu_ii = mu0 I (Sec. 2.2)
//         + C_i                                  (the variant the kernel used)
//     v_i = mu0 V_i;  output v, or x_{n+1} = x_n + dt v_n in FP64.
//
// Tdense is re-evaluated with the very same device function and inputs the
// all-pairs kernel used; Texact is the FP64 tensor in use (Rotne-Prager, Oseen,
// or the RPY overlap form) at the FP64 separation.  These are the pairs whose
// FP32 evaluation suffers from cancellation in r_i - r_j (large coordinates,
// small separations) or that the clamp altered (r < 2a).
#include <algorithm>
#include <type_traits>
#include "neighbours.cuh"

namespace sd {

template <int MODE>
struct EpiT {
    using V4 = float4;
    using S = float;
};
template <>
struct EpiT<MODE_FP64> {
    using V4 = dbl4;
    using S = double;
};

template <int TDENSE, int MODE, bool CLAMP, bool PER = false>
__device__ __forceinline__ void dense_term(const typename EpiT<MODE>::V4 &pi, const typename EpiT<MODE>::V4 &pj,
                                           const typename EpiT<MODE>::V4 &fj, const PairConst &c, double out[3]) {
    using S = typename EpiT<MODE>::S;
    S ax = S(0), ay = S(0), az = S(0);
    if constexpr (MODE == MODE_FP64)
        pair_f64<TDENSE, PER>(pi.x, pi.y, pi.z, pj, fj, c, ax, ay, az);
    else
        pair_f32<TDENSE, CLAMP, PER>(pi.x, pi.y, pi.z, pj, fj, c, ax, ay, az);
    out[0] = static_cast<double>(ax);
    out[1] = static_cast<double>(ay);
    out[2] = static_cast<double>(az);
}

// The all-pairs kernels' term of the pair (i, j), nearest image in a periodic box.
template <int TDENSE, int MODE, bool CLAMP>
__device__ __forceinline__ void dense_term_box(const typename EpiT<MODE>::V4 &pi, const typename EpiT<MODE>::V4 &pj,
                                               const typename EpiT<MODE>::V4 &fj, const PairConst &c,
                                               double out[3]) {
    if (c.periodic)
        dense_term<TDENSE, MODE, CLAMP, true>(pi, pj, fj, c, out);
    else
        dense_term<TDENSE, MODE, CLAMP, false>(pi, pj, fj, c, out);
}

// Mirror separation (nearest image in a periodic box) rounded to FP32, for the
// near pass's screen.
__device__ __forceinline__ float screen_r2(const float4 &pi, const float4 &pj, const PairConst &c) {
    float sx = __fsub_rn(pi.x, pj.x), sy = __fsub_rn(pi.y, pj.y), sz = __fsub_rn(pi.z, pj.z);
    if (c.periodic) {
        sx = min_image_f32(sx, c.Lf[0], c.invLf[0]);
        sy = min_image_f32(sy, c.Lf[1], c.invLf[1]);
        sz = min_image_f32(sz, c.Lf[2], c.invLf[2]);
    }
    return sx * sx + sy * sy + sz * sz;
}
__device__ __forceinline__ float screen_r2(const dbl4 &pi, const dbl4 &pj, const PairConst &c) {
    double ux = pi.x - pj.x, uy = pi.y - pj.y, uz = pi.z - pj.z;
    if (c.periodic) {
        ux = min_image_f64(ux, c.Ld[0], c.invLd[0]);
        uy = min_image_f64(uy, c.Ld[1], c.invLd[1]);
        uz = min_image_f64(uz, c.Ld[2], c.invLd[2]);
    }
    const float sx = static_cast<float>(ux), sy = static_cast<float>(uy), sz = static_cast<float>(uz);
    return sx * sx + sy * sy + sz * sz;
}

// ---------------------------------------------------------------- near pass

struct NearArgs {
    const double *x64;
    const void *posm;
    const double *F64;
    const void *frcm;
    CellList cl;
    double rnear2, rsafe2;
    float rscreen2;   // (1.01 r_near)^2: FP32 screen of candidates before the FP64 test
    PairConst pc;
    int n;
    double *near;   // [n][6]: clamped-variant correction (3), unclamped-variant correction (3)
    int *flag;      // raised when some pair has r < r_safe
    int *err;
    DenseGeom g;    // the all-pairs kernel's tiling (which tiles clamp r^2)
    // compacted candidate list (near_collect_kernel -> near_pair_kernel -> epilogue)
    int2 *ent;        // [cap] (i, j), or (-1, -1) for a slot that holds no pair
    double *ent_out;  // [cap][6] the pair's two correction variants, as `near`
    unsigned long long *ent_n;   // entries claimed (zeroed before the collect kernel)
    int *noff, *ncnt; // per particle: first entry and count; ncnt = -1: correction is in near[i]
    int cap;
    const int *gate;  // Verlet list build: run only when the step's check asked for a rebuild
};

// The correction of one near pair (FP64 r^2 < r_near^2), added to c6: the exact
// FP64 term minus the all-pairs kernel's FP32 term with r^2 clamped (c6[0..2]),
// and the further difference when that kernel did not clamp (c6[3..5]).
template <int TENSOR, int MODE>
__device__ __forceinline__ void near_pair_term(const NearArgs &a, int i, int j, double dx, double dy, double dz,
                                               double r2, double (&c6)[6], bool &coincident) {
    using V4 = typename EpiT<MODE>::V4;
    constexpr int TDENSE = (TENSOR == T_OSEEN) ? T_OSEEN : T_RP;
    const V4 *pm = static_cast<const V4 *>(a.posm);
    const V4 *fm = static_cast<const V4 *>(a.frcm);
    if (r2 == 0.0 && TENSOR != T_RPY) {
        coincident = true;
        return;
    }
    double A, B, dA, dB;
    profile_exact<TENSOR>(r2, a.pc, A, B, dA, dB);
    const double fx = a.F64[3 * j], fy = a.F64[3 * j + 1], fz = a.F64[3 * j + 2];
    const double s = B * (dx * fx + dy * fy + dz * fz);
    const double e[3] = {A * fx + s * dx, A * fy + s * dy, A * fz + s * dz};
    const V4 pi = pm[i], pj = pm[j];
    double tc[3];
    dense_term_box<TDENSE, MODE, true>(pi, pj, fm[j], a.pc, tc);
    for (int d = 0; d < 3; ++d) c6[d] += e[d] - tc[d];
    // The unclamped variant differs only where the clamp was active, i.e. the
    // pair's FP32 r^2 < (2a)^2, and outside the tiles holding self pairs (clamped
    // in both variants); c6[3..5] collects that difference.
    if constexpr (MODE != MODE_FP64) {
        float ux = __fsub_rn(pi.x, pj.x), uy = __fsub_rn(pi.y, pj.y), uz = __fsub_rn(pi.z, pj.z);
        if (a.pc.periodic) {
            ux = min_image_f32(ux, a.pc.Lf[0], a.pc.invLf[0]);
            uy = min_image_f32(uy, a.pc.Lf[1], a.pc.invLf[1]);
            uz = min_image_f32(uz, a.pc.Lf[2], a.pc.invLf[2]);
        }
        const float r2f = __fmaf_rn(uz, uz, __fmaf_rn(uy, uy, __fmul_rn(ux, ux)));
        const long long i0 = static_cast<long long>(i / a.g.I) * a.g.I, j0 = static_cast<long long>(j / a.g.J) * a.g.J;
        const bool diag = (j0 < i0 + a.g.I) && (i0 < j0 + a.g.J);
        if (r2f < a.pc.r2min_f && !diag && !(a.pc.periodic && geom_pad_tile(a.g, a.n, i0, j0))) {
            double tu[3];
            dense_term_box<TDENSE, MODE, false>(pi, pj, fm[j], a.pc, tu);
            for (int d = 0; d < 3; ++d) c6[3 + d] += tc[d] - tu[d];
        }
    }
}

// In-place correction of particle i by its kWalkLanes lanes (used when the
// candidate list has no room): the walk, the FP64 test and the term per lane,
// then the fixed shuffle tree.  Warp-collective.
template <int TENSOR, int MODE>
__device__ void near_direct(const NearArgs &a, int i, int sub, bool active) {
    using V4 = typename EpiT<MODE>::V4;
    const V4 *pm = static_cast<const V4 *>(a.posm);
    double c6[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    bool coincident = false, close = false, found = false;
    if (active) {
        const V4 pi = pm[i];
        const double xi = a.x64[3 * i], yi = a.x64[3 * i + 1], zi = a.x64[3 * i + 2];
        for_each_neighbour_part(a.cl, i, a.cl.cell[i], sub, kWalkLanes, [&](int j) {
            if (screen_r2(pi, pm[j], a.pc) > a.rscreen2) return;
            double dx = xi - a.x64[3 * j], dy = yi - a.x64[3 * j + 1], dz = zi - a.x64[3 * j + 2];
            box_image(a.cl.box, dx, dy, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= a.rnear2) return;
            found = true;
            if (r2 < a.rsafe2) close = true;
            near_pair_term<TENSOR, MODE>(a, i, j, dx, dy, dz, r2, c6, coincident);
        });
    }
    const int writer = walk_combine(c6, found, sub);
    coincident = walk_any(coincident);
    close = walk_any(close);
    if (!active || sub != writer) return;
    if (coincident) atomicOr(a.err, DEV_ERR_COINCIDENT);
    if (close && a.flag) atomicOr(a.flag, 1);
    double *o = a.near + 6 * static_cast<size_t>(i);
    for (int d = 0; d < 3; ++d) {
        o[d] = c6[d];                 // correction when every tile is clamped
        o[3 + d] = c6[d] + c6[3 + d]; // correction when only self-pair tiles are
    }
}

// Step 1 of the near pass: kWalkLanes lanes per particle walk the 27 cells and keep
// the neighbours that pass an FP32 screen on the mirror.  Particles are taken in
// cell-list order, so the groups of a warp are spatial neighbours and share the
// cells they read.  The candidates go to a list in (particle, lane, walk) order: a
// warp-wide prefix sum places each lane's run, one atomicAdd per warp claims the
// warp's range (where the warps' ranges land does not matter: each particle's run
// is contiguous and read in order).  The FP64 arithmetic is left to
// near_pair_kernel, where every lane of a warp has a pair (here only ~1 lane in 20
// would).
constexpr int kNearRegs = 4;   // candidates a lane keeps in registers; more -> second walk

template <int TENSOR, int MODE>
__global__ void __launch_bounds__(128) near_collect_kernel(NearArgs a) {
    if (a.gate && *a.gate == 0) return;   // (uniform over the grid)
    using V4 = typename EpiT<MODE>::V4;
    const V4 *pm = static_cast<const V4 *>(a.posm);
    const long long gt = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int q = static_cast<int>(gt / kWalkLanes), sub = static_cast<int>(gt % kWalkLanes);
    const bool active = q < a.n;
    const int i = active ? a.cl.sorted[q] : 0;
    const int lane = threadIdx.x & 31;
    int cnt = 0, j0 = -1, j1 = -1, j2 = -1, j3 = -1;
    auto screen = [&](const V4 &pi, int j) { return screen_r2(pi, pm[j], a.pc) <= a.rscreen2; };
    if (active) {
        const V4 pi = pm[i];
        for_each_neighbour_part(a.cl, i, a.cl.cell[i], sub, kWalkLanes, [&](int j) {
            if (!screen(pi, j)) return;
            if (cnt == 0) j0 = j;
            else if (cnt == 1) j1 = j;
            else if (cnt == 2) j2 = j;
            else if (cnt == 3) j3 = j;
            ++cnt;
        });
    }
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - cnt;
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    long long base = 0;
    if (lane == 0 && tot > 0) base = static_cast<long long>(atomicAdd(a.ent_n, static_cast<unsigned long long>(tot)));
    base = __shfl_sync(0xffffffffu, base, 0);
    const bool fits = base + tot <= a.cap;
    // this lane's first entry (only used when the warp's range fits below the capacity)
    const int first = fits ? static_cast<int>(base) + excl : 0;
    const int pfirst = __shfl_sync(0xffffffffu, first, lane & ~(kWalkLanes - 1));
    int pcnt = cnt;
    for (int o = kWalkLanes / 2; o >= 1; o >>= 1) pcnt += __shfl_xor_sync(0xffffffffu, pcnt, o);
    if (fits) {
        if (active) {
            const int js[kNearRegs] = {j0, j1, j2, j3};
#pragma unroll
            for (int k = 0; k < kNearRegs; ++k)
                if (k < cnt) a.ent[first + k] = make_int2(i, js[k]);
            for (int k = 0; k < kNearRegs && k < cnt; ++k) dbg_index(first + k, a.cap, a.err);
            if (cnt > kNearRegs) {   // rare: walk again for the candidates beyond the registers
                const V4 pi = pm[i];
                int k = 0;
                for_each_neighbour_part(a.cl, i, a.cl.cell[i], sub, kWalkLanes, [&](int j) {
                    if (!screen(pi, j)) return;
                    if (k >= kNearRegs && k < cnt) a.ent[first + k] = make_int2(i, j);
                    ++k;
                });
            }
            if (sub == 0) {
                a.noff[i] = pfirst;
                a.ncnt[i] = pcnt;
            }
        }
    } else {
        // The list is full: mark this warp's claimed slots below the capacity as
        // empty and correct its particles in place.
        for (long long e = base + lane; e < base + tot && e < a.cap; e += 32) a.ent[e] = make_int2(-1, -1);
        if (active && sub == 0) a.ncnt[i] = -1;
        near_direct<TENSOR, MODE>(a, i, sub, active);
    }
    // A Verlet list (a.gate set): each particle's run in ascending partner index, so
    // that the epilogue adds a particle's near terms in an order that does not depend
    // on when, or from which cell list, the list was built (entries beyond r_near add
    // exact zeros).  The run was written by this warp's lanes of the particle.
    __syncwarp();
    if (a.gate && fits && active && sub == 0 && pcnt > 1) {
        for (int p = pfirst + 1; p < pfirst + pcnt; ++p) {
            const int2 v = a.ent[p];
            int q = p - 1;
            while (q >= pfirst && a.ent[q].y > v.y) {
                a.ent[q + 1] = a.ent[q];
                --q;
            }
            a.ent[q + 1] = v;
        }
    }
}

// Step 2: one thread per listed pair: the FP64 test r < r_near, the flags, and the
// two correction variants of the pair, written to its entry.
template <int TENSOR, int MODE>
__global__ void __launch_bounds__(128) near_pair_kernel(NearArgs a) {
    const int total = static_cast<int>(min(*a.ent_n, static_cast<unsigned long long>(a.cap)));
    bool coincident = false, close = false;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int2 p = a.ent[e];
        double c6[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (p.x >= 0) {
            const int i = static_cast<int>(dbg_index(p.x, a.n, a.err)), j = static_cast<int>(dbg_index(p.y, a.n, a.err));
            double dx = a.x64[3 * i] - a.x64[3 * j], dy = a.x64[3 * i + 1] - a.x64[3 * j + 1],
                   dz = a.x64[3 * i + 2] - a.x64[3 * j + 2];
            box_image(a.cl.box, dx, dy, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < a.rnear2) {
                if (r2 < a.rsafe2) close = true;
                near_pair_term<TENSOR, MODE>(a, i, j, dx, dy, dz, r2, c6, coincident);
            }
        }
        double *o = a.ent_out + 6 * static_cast<size_t>(e);
        for (int d = 0; d < 3; ++d) {
            o[d] = c6[d];
            o[3 + d] = c6[d] + c6[3 + d];
        }
    }
    if (coincident) atomicOr(a.err, DEV_ERR_COINCIDENT);
    if (close && a.flag) atomicOr(a.flag, 1);
}

template <int TENSOR, int MODE>
static void near_launch_collect(int nb, cudaStream_t st, const NearArgs &a) {
    near_collect_kernel<TENSOR, MODE><<<nb, 128, 0, st>>>(a);
}
template <int TENSOR, int MODE>
static void near_launch_pairs(int np, cudaStream_t st, const NearArgs &a) {
    near_pair_kernel<TENSOR, MODE><<<np, 128, 0, st>>>(a);
}

static NearArgs near_args(sd_handle *h, const double *x64, const void *posm, const double *F64, const void *frcm,
                          double screen, bool vlist = false) {
    NearArgs a;
    a.x64 = x64;
    a.posm = posm;
    a.F64 = F64;
    a.frcm = frcm;
    a.cl = h->cl;
    a.rnear2 = h->r_near * h->r_near;
    a.rsafe2 = kRSafe * kRSafe * h->pc.a * h->pc.a;
    a.rscreen2 = static_cast<float>(1.0201 * screen * screen);
    a.pc = h->pc;
    a.n = h->n;
    a.near = h->near64;
    a.flag = h->d_flag;
    a.err = h->d_err;
    a.g = h->geom;
    a.ent = vlist ? h->vent : h->near_ent;   // (the Verlet steps' own list)
    a.ent_out = h->near_out;
    a.ent_n = vlist ? h->vn : h->near_n;
    a.noff = vlist ? h->voff : h->near_off;
    a.ncnt = vlist ? h->vcnt : h->near_cnt;
    a.cap = h->near_cap;
    a.gate = nullptr;
    return a;
}

#define SD_NEAR_DISPATCH(FN, ARG)                                                                                \
    do {                                                                                                         \
        const bool f64_ = h->mode == MODE_FP64;                                                                  \
        switch (h->tensor) {                                                                                     \
            case T_RPY: if (f64_) FN<T_RPY, MODE_FP64>(ARG, st, a); else FN<T_RPY, MODE_FP32C>(ARG, st, a); break; \
            case T_RP: if (f64_) FN<T_RP, MODE_FP64>(ARG, st, a); else FN<T_RP, MODE_FP32C>(ARG, st, a); break;    \
            default: if (f64_) FN<T_OSEEN, MODE_FP64>(ARG, st, a); else FN<T_OSEEN, MODE_FP32C>(ARG, st, a); break; \
        }                                                                                                        \
    } while (0)

cudaError_t launch_near_collect(sd_handle *h, cudaStream_t st, const double *x64, const void *posm,
                                const double *F64, const void *frcm, bool count_zeroed, bool verlet_list) {
    if (h->n == 0) return cudaSuccess;
    NearArgs a = near_args(h, x64, posm, F64, frcm, verlet_list ? h->list_cut + h->skin : h->r_near, verlet_list);
    if (verlet_list) {   // a Verlet step's rebuild: the clamp flag is its check kernel's
        a.gate = h->d_vl;
        a.flag = nullptr;
    }
    const int nb = static_cast<int>((static_cast<long long>(h->n) * kWalkLanes + 127) / 128);
    if (!count_zeroed) {
        cudaError_t e = cudaMemsetAsync(a.ent_n, 0, sizeof(*a.ent_n), st);
        if (e != cudaSuccess) return e;
    }
    SD_NEAR_DISPATCH(near_launch_collect, nb);
    ++h->launches;
    return cudaGetLastError();
}

cudaError_t launch_near_pairs(sd_handle *h, cudaStream_t st, const double *x64, const void *posm, const double *F64,
                              const void *frcm, bool verlet_step) {
    if (h->n == 0) return cudaSuccess;
    NearArgs a = near_args(h, x64, posm, F64, frcm, h->r_near, verlet_step);
    if (verlet_step) a.flag = nullptr;   // (the check kernel's; the all-pairs kernel may be reading it)
    const int np = static_cast<int>(std::min<long long>((static_cast<long long>(a.cap) + 127) / 128,
                                                        8LL * h->num_sms));
    SD_NEAR_DISPATCH(near_launch_pairs, np);
    ++h->launches;
    return cudaGetLastError();
}
#undef SD_NEAR_DISPATCH

cudaError_t launch_near(sd_handle *h, cudaStream_t st, const double *x64, const void *posm, const double *F64,
                        const void *frcm, bool count_zeroed) {
    if (h->n == 0) return cudaSuccess;
    prof_begin(h, SD_KERNEL_NEAR, st);
    cudaError_t e = launch_near_collect(h, st, x64, posm, F64, frcm, count_zeroed, false);
    if (e == cudaSuccess) e = launch_near_pairs(h, st, x64, posm, F64, frcm, false);
    prof_end(h, SD_KERNEL_NEAR, st);
    return e;
}

// ---------------------------------------------------------------- epilogue

struct EpiArgs {
    const double *ent_out;   // near-pass list results, per particle noff/ncnt
    const int *noff, *ncnt;
    const double *part;
    const float *jpart;     // source-side sums of the symmetric kernel (g.sym), FP32 modes
    const double *jpart64;  // ... FP64 mode
    int npad;
    DenseGeom g;
    const double *x64;
    const void *posm;
    const double *F64;
    const void *frcm;
    const double *near;
    const int *flag;
    PairConst pc;
    int n;
    void *vout;
    double dt;
    double *x64n;
    double *vlag;   // OUT_EULER with lubrication: this step's FP64 velocities, for the next step's forces
    int *err;
    int cap;        // capacity of the near-pass list
    int row0, row1; // rows written (a shard); vout holds rows row0 .. row1-1
    EpiShard sh;    // a tile shard's share, or the shards' results to combine
};

// First r in [0, ib] whose source-side row of block ib, tile rowstart(r) + ib - r,
// is >= t (the row index grows with r).
__device__ __forceinline__ int first_row_at(const DenseGeom &g, int ib, long long t) {
    int lo = 0, hi = ib;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (geom_rowstart(g, mid) + (ib - mid) >= t) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Each CTA finishes 32 consecutive particles.  Warp w of the kEpiWarps adds the
// slots s = w, w + kEpiWarps, ... of the dense partial sums (and, after the
// symmetric kernel, the source-side tiles r = w, w + kEpiWarps, ... of the
// particle's block column); lane l reads particle 32 b + l, so every warp load is
// one coalesced 128-byte row.  Warp 0 adds the warps' results in ascending w
// (fixed order: deterministic) and applies the FP64 terms.  Four warps per 32
// particles measured best at N = 65,536 (40 us against 45 for 8, 51 for 2, 79 for 16):
// the kernel waits on DRAM latency, and fewer warps per group leave fewer idle
// during warp 0's FP64 tail.  With one tile per all-pairs CTA (twice the target-side
// slots): 53 us at 4 warps, 55 at 8; source loop unrolled 1 / 2 / 4: 52.6 / 53.0 /
// 70 us; launch bounds for 16 or 12 resident CTAs per SM (32 or 40 registers, all
// CTAs in one wave): 53 / 61 us.  Two particles per lane (one 16-byte load for both
// particles' (hi, lo) pairs): 43 us, the loads then reaching 63% of the HBM copy
// rate instead of 50%.
#ifndef SD_EPI_WARPS
#define SD_EPI_WARPS 4
#endif
#ifndef SD_EPI_UNROLL
#define SD_EPI_UNROLL 2
#endif
#ifndef SD_EPI_PAIRS
#define SD_EPI_PAIRS 1
#endif
constexpr int kEpiWarps = SD_EPI_WARPS;
constexpr int kEpiUnroll = SD_EPI_UNROLL;
constexpr bool kEpiPairs = SD_EPI_PAIRS != 0;   // FP32C: two particles per lane in the sums

// P particles per lane in the sums (P = 2: FP32C without shard shares, row0 even):
// a lane then reads the (hi, lo) pairs of particles i0, i0 + 1 as one 16-byte load
// and their source-side partials as one 8-byte load, so each load instruction
// carries twice the bytes; every particle's sums take the same operations in the
// same order as with P = 1.
template <int TDENSE, int MODE, int OUT, int P>
__global__ void __launch_bounds__(32 * kEpiWarps) epilogue_kernel(EpiArgs a) {
    using V4 = typename EpiT<MODE>::V4;
    constexpr int NP = 32 * P;   // particles per CTA
    static_assert(P == 1 || (P == 2 && MODE == MODE_FP32C), "two particles per lane: FP32C only");
    __shared__ double s_v[kEpiWarps][3][NP];
    __shared__ float s_h[kEpiWarps][3][NP], s_l[kEpiWarps][3][NP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // CTAs in reverse particle order: the last blocks have the longest source-side
    // columns, so they start first instead of forming the tail
    const int base = a.row0 + (gridDim.x - 1 - blockIdx.x) * NP;

    // This warp's share of the dense sum: the CTA slots of the particle's i-block,
    // then (symmetric kernel) the source-side slots of the tiles (r, ib), r < ib.
    // FP32C sums both with TwoSum in FP32 (hi, lo) -- the slots are (hi, lo) pairs
    // themselves -- because FP64 issues at 1/64 the FP32 rate on GB300.
    {
        const int i = base + P * lane;   // this lane's particles: i .. i + P - 1 (one i-block)
        const bool active = i < a.row1;
        double v[P][3];
        float hi[P][3], lo[P][3];
        for (int k = 0; k < P; ++k)
            for (int d = 0; d < 3; ++d) {
                v[k][d] = 0.0;
                hi[k][d] = lo[k][d] = 0.0f;
            }
        if (active && a.sh.pall) {   // (P = 1)
            // the shards' results, added in shard order (warp 0)
            if (w == 0)
                for (int q = 0; q < a.sh.nparts; ++q)
                    for (int d = 0; d < 3; ++d) v[0][d] += a.sh.pall[(static_cast<size_t>(q) * a.n + i) * 3 + d];
        } else if (active) {
            const int ib = i / a.g.I;
            const int first = geom_first(a.g, ib);
            const int s0 = max(0, a.sh.b0 - first);
            const int ns = min(geom_last(a.g, ib) - first + 1, a.sh.b1 - first);
            if (ns > 0) dbg_index(ns - 1, a.g.maxSlots, a.err);
            if (a.g.sym && ib > 0) dbg_index(geom_rowstart(a.g, ib - 1) + 1, a.g.nT, a.err);
            int r0 = 0, nc = a.g.sym ? ib : 0;
            if (a.g.sym && (a.sh.tlo > 0 || a.sh.thi < a.g.nT)) {
                r0 = first_row_at(a.g, ib, a.sh.tlo);
                nc = first_row_at(a.g, ib, a.sh.thi);
            }
            const int o = i - ib * a.g.I;
            const int J = a.g.J;
            const size_t cs = 3 * static_cast<size_t>(J);
            if constexpr (MODE == MODE_FP32) {
                for (int s = s0 + w; s < ns; s += kEpiWarps)
                    for (int d = 0; d < 3; ++d)
                        hi[0][d] = __fadd_rn(hi[0][d], static_cast<float>(
                                                           a.part[(static_cast<size_t>(s) * 3 + d) * a.npad + i]));
                for (int r = r0 + w; r < nc; r += kEpiWarps) {
                    const float *src = a.jpart + static_cast<size_t>(geom_rowstart(a.g, r) + (ib - r)) * cs + o;
                    for (int d = 0; d < 3; ++d) hi[0][d] = __fadd_rn(hi[0][d], src[d * J]);
                }
            } else if constexpr (MODE == MODE_FP64) {
                for (int s = s0 + w; s < ns; s += kEpiWarps)
                    for (int d = 0; d < 3; ++d) v[0][d] += a.part[(static_cast<size_t>(s) * 3 + d) * a.npad + i];
                for (int r = r0 + w; r < nc; r += kEpiWarps) {
                    const double *src = a.jpart64 + static_cast<size_t>(geom_rowstart(a.g, r) + (ib - r)) * cs + o;
                    for (int d = 0; d < 3; ++d) v[0][d] += src[d * J];
                }
            } else if constexpr (P == 1) {   // FP32C: each slot is a (hi, lo) float pair
                const float2 *pp = reinterpret_cast<const float2 *>(a.part);
#pragma unroll 4
                for (int s = s0 + w; s < ns; s += kEpiWarps)
                    for (int d = 0; d < 3; ++d) {
                        const float2 q = pp[(static_cast<size_t>(s) * 3 + d) * a.npad + i];
                        fold2(hi[0][d], lo[0][d], q.x);
                        lo[0][d] = __fadd_rn(lo[0][d], q.y);
                    }
#pragma unroll kEpiUnroll
                for (int r = r0 + w; r < nc; r += kEpiWarps) {
                    const float *src = a.jpart + static_cast<size_t>(geom_rowstart(a.g, r) + (ib - r)) * cs + o;
                    for (int d = 0; d < 3; ++d) fold2(hi[0][d], lo[0][d], src[d * J]);
                }
            } else {   // FP32C, two particles: i even, npad, I and J even, so both loads are aligned
                const float2 *pp = reinterpret_cast<const float2 *>(a.part);
#pragma unroll 4
                for (int s = s0 + w; s < ns; s += kEpiWarps)
                    for (int d = 0; d < 3; ++d) {
                        const float4 q =
                            *reinterpret_cast<const float4 *>(pp + (static_cast<size_t>(s) * 3 + d) * a.npad + i);
                        fold2(hi[0][d], lo[0][d], q.x);
                        lo[0][d] = __fadd_rn(lo[0][d], q.y);
                        fold2(hi[1][d], lo[1][d], q.z);
                        lo[1][d] = __fadd_rn(lo[1][d], q.w);
                    }
#pragma unroll kEpiUnroll
                for (int r = r0 + w; r < nc; r += kEpiWarps) {
                    const float *src = a.jpart + static_cast<size_t>(geom_rowstart(a.g, r) + (ib - r)) * cs + o;
                    for (int d = 0; d < 3; ++d) {
                        const float2 q = *reinterpret_cast<const float2 *>(src + d * J);
                        fold2(hi[0][d], lo[0][d], q.x);
                        fold2(hi[1][d], lo[1][d], q.y);
                    }
                }
            }
        }
        for (int k = 0; k < P; ++k)
            for (int d = 0; d < 3; ++d) {
                s_v[w][d][P * lane + k] = v[k][d];
                s_h[w][d][P * lane + k] = hi[k][d];
                s_l[w][d][P * lane + k] = lo[k][d];
            }
    }
    __syncthreads();
    // one particle per lane from here: warps 0 .. P - 1
    if (w >= P) return;
    const int j = 32 * w + lane;   // the particle's place in the CTA's sums
    const int i = base + j;
    if (i >= a.row1) return;
    const V4 *pm = static_cast<const V4 *>(a.posm);
    const V4 *fm = static_cast<const V4 *>(a.frcm);
    double V[3];
    for (int d = 0; d < 3; ++d) {
        if constexpr (MODE == MODE_FP32) {
            float f = s_h[0][d][j];
            for (int q = 1; q < kEpiWarps; ++q) f = __fadd_rn(f, s_h[q][d][j]);
            V[d] = f;
        } else {
            double v = s_v[0][d][j];
            float h = s_h[0][d][j], l = s_l[0][d][j];
            for (int q = 1; q < kEpiWarps; ++q) {
                v += s_v[q][d][j];
                fold2(h, l, s_h[q][d][j]);
                l = __fadd_rn(l, s_l[q][d][j]);
            }
            V[d] = v + (static_cast<double>(h) + static_cast<double>(l));
        }
    }
    if constexpr (OUT == OUT_PART) {   // a shard's raw share: no self or near terms, no mu0
        double *o = static_cast<double *>(a.vout) + 3 * static_cast<size_t>(i);
        o[0] = V[0];
        o[1] = V[1];
        o[2] = V[2];
        return;
    }
    // self term: the tile holding it was clamped; replace by mu_ii / mu0 = I
    {
        const V4 pi = pm[i];
        double t[3];
        dense_term<TDENSE, MODE, true>(pi, pi, fm[i], a.pc, t);
        for (int d = 0; d < 3; ++d) V[d] += a.F64[3 * i + d] - t[d];
    }
    // near pairs: the variant matching the kernel's clamping, from the particle's
    // entries of the candidate list in list order (or from its in-place result)
    {
        const int var = (*a.flag) ? 0 : 3;
        const int cnt = a.ncnt[i];
        if (cnt < 0) {
            const double *c = a.near + 6 * static_cast<size_t>(i) + var;
            for (int d = 0; d < 3; ++d) V[d] += c[d];
        } else {
            const long long e0 = dbg_index(a.noff[i], static_cast<long long>(a.cap) - cnt + 1, a.err);
            const double *c = a.ent_out + 6 * static_cast<size_t>(e0) + var;
            for (int k = 0; k < cnt; ++k, c += 6)
                for (int d = 0; d < 3; ++d) V[d] += c[d];
        }
    }
    const double m0 = a.pc.mu0;
    const double v0 = m0 * V[0], v1 = m0 * V[1], v2 = m0 * V[2];
    if constexpr (OUT == OUT_F32) {
        float *o = static_cast<float *>(a.vout) + 3 * static_cast<size_t>(i - a.row0);
        o[0] = static_cast<float>(v0);
        o[1] = static_cast<float>(v1);
        o[2] = static_cast<float>(v2);
    } else if constexpr (OUT == OUT_F64) {
        double *o = static_cast<double *>(a.vout) + 3 * static_cast<size_t>(i - a.row0);
        o[0] = v0;
        o[1] = v1;
        o[2] = v2;
    } else {
        const double xi = a.x64[3 * i], yi = a.x64[3 * i + 1], zi = a.x64[3 * i + 2];
        const double nx = xi + a.dt * v0, ny = yi + a.dt * v1, nz = zi + a.dt * v2;
        if (a.vlag) {
            a.vlag[3 * i] = v0;
            a.vlag[3 * i + 1] = v1;
            a.vlag[3 * i + 2] = v2;
        }
        if (!isfinite(nx) || !isfinite(ny) || !isfinite(nz)) atomicOr(a.err, DEV_ERR_NONFINITE);
        a.x64n[3 * i] = nx;
        a.x64n[3 * i + 1] = ny;
        a.x64n[3 * i + 2] = nz;
    }
}

template <int TDENSE, int MODE, int P>
static void epi_launch(int out, cudaStream_t st, const EpiArgs &a) {
    const int nb = (a.row1 - a.row0 + 32 * P - 1) / (32 * P);
    switch (out) {
        case OUT_F32: epilogue_kernel<TDENSE, MODE, OUT_F32, P><<<nb, 32 * kEpiWarps, 0, st>>>(a); break;
        case OUT_F64: epilogue_kernel<TDENSE, MODE, OUT_F64, P><<<nb, 32 * kEpiWarps, 0, st>>>(a); break;
        case OUT_PART: epilogue_kernel<TDENSE, MODE, OUT_PART, P><<<nb, 32 * kEpiWarps, 0, st>>>(a); break;
        default: epilogue_kernel<TDENSE, MODE, OUT_EULER, P><<<nb, 32 * kEpiWarps, 0, st>>>(a); break;
    }
}

template <int TDENSE>
static void epi_launch_mode(int mode, int out, cudaStream_t st, const EpiArgs &a) {
    switch (mode) {
        case MODE_FP32C:
            // two particles per lane needs an even first row (aligned loads) and no shard shares
            if (kEpiPairs && (a.row0 & 1) == 0 && !a.sh.pall)
                epi_launch<TDENSE, MODE_FP32C, 2>(out, st, a);
            else
                epi_launch<TDENSE, MODE_FP32C, 1>(out, st, a);
            break;
        case MODE_FP64: epi_launch<TDENSE, MODE_FP64, 1>(out, st, a); break;
        default: epi_launch<TDENSE, MODE_FP32, 1>(out, st, a); break;
    }
}

cudaError_t launch_epilogue(sd_handle *h, cudaStream_t st, int out, const double *x64, const void *posm,
                            const double *F64, const void *frcm, void *vout, double dt, double *x64n, int row0,
                            int row1, const EpiShard *shard, bool vlist) {
    if (h->n == 0) return cudaSuccess;
    if (row1 < 0 || row1 > h->n) row1 = h->n;
    if (row0 < 0) row0 = 0;
    if (row0 >= row1) return cudaSuccess;
    EpiArgs a;
    a.ent_out = h->near_out;
    a.noff = vlist ? h->voff : h->near_off;   // (a Verlet step: its own candidate list)
    a.ncnt = vlist ? h->vcnt : h->near_cnt;
    a.part = h->part;
    a.jpart = h->mode == MODE_FP64 ? nullptr : static_cast<const float *>(h->jpart);
    a.jpart64 = h->mode == MODE_FP64 ? static_cast<const double *>(h->jpart) : nullptr;
    a.npad = h->npad;
    a.g = h->geom;
    a.x64 = x64;
    a.posm = posm;
    a.F64 = F64;
    a.frcm = frcm;
    a.near = h->near64;
    a.flag = h->d_flag;
    a.pc = h->pc;
    a.n = h->n;
    a.vout = vout;
    a.dt = dt;
    a.x64n = x64n;
    a.vlag = (out == OUT_EULER && h->lub) ? h->vlag : nullptr;
    a.err = h->d_err;
    a.cap = h->near_cap;
    a.row0 = row0;
    a.row1 = row1;
    if (shard) a.sh = *shard;
    prof_begin(h, SD_KERNEL_EPILOGUE, st);
    if (h->tensor == T_OSEEN)
        epi_launch_mode<T_OSEEN>(h->mode, out, st, a);
    else
        epi_launch_mode<T_RP>(h->mode, out, st, a);
    prof_end(h, SD_KERNEL_EPILOGUE, st);
    ++h->launches;
    return cudaGetLastError();
}

}  // namespace sd
