// sd_internal.h -- handle layout and kernel launchers shared by the .cu files
// of the library (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sd.h"
#include "pair.cuh"

namespace sd {

// Device error word bits (atomicOr'ed by kernels, read at synchronising calls).
enum : int {
    DEV_ERR_NONFINITE = 1,
    DEV_ERR_COINCIDENT = 2,
    DEV_ERR_TIMEOUT = 4,
    DEV_ERR_QUEUE = 8,
    DEV_ERR_BOUNDS = 16,   // a device-side index check failed (SD_DEBUG builds)
};

// Debug builds (-DSD_DEBUG) check the data-dependent indices of the kernels (cell
// list, near-pair list, partial-sum slots, batched staging) against the buffers they
// address: an index outside [0, bound) sets DEV_ERR_BOUNDS (reported as
// SD_ERR_INTERNAL) and is replaced by 0, so the access stays inside the buffer and no
// thread leaves a warp-collective section early.  Release builds compile the check
// away.
__device__ __forceinline__ long long dbg_index(long long idx, long long bound, int *err) {
#ifdef SD_DEBUG
    if (idx < 0 || idx >= bound) {
        if (err) atomicOr(err, DEV_ERR_BOUNDS);
        return 0;
    }
#else
    (void)bound;
    (void)err;
#endif
    return idx;
}

enum { MODE_FP32C = 0, MODE_FP64 = 1, MODE_FP32 = 2 };
// Epilogue outputs: velocities (FP32 / FP64), the Euler update, or (OUT_PART) a
// shard's raw share of the all-pairs sum (FP64, no self or near-pair terms).
enum { OUT_F32 = 0, OUT_F64 = 1, OUT_EULER = 2, OUT_PART = 3 };

// A shard of the all-pairs sum for the epilogue: only the slots written by CTAs
// b0 .. b1-1 of the full launch, and (symmetric kernels) the source-side rows of the
// tiles tlo .. thi-1, enter the sum; or, with pall, the sum is replaced by the
// nparts shard results pall[g][n][3] added in shard order.
struct EpiShard {
    int b0 = 0, b1 = 0x7fffffff;
    long long tlo = 0, thi = 0x7fffffffffffffffLL;
    const double *pall = nullptr;
    int nparts = 0;
};

constexpr int kPadTo = 1024;     // particle arrays are padded to a multiple of this
#ifndef SD_DENSE_THREADS
#define SD_DENSE_THREADS 128
#endif
#ifndef SD_DENSE_R32
#define SD_DENSE_R32 2
#endif
#ifndef SD_DENSE_JUNROLL
#define SD_DENSE_JUNROLL 1
#endif
constexpr int kNT = SD_DENSE_THREADS;   // threads per CTA of the dense kernels
constexpr int kR32 = SD_DENSE_R32;      // i-particles per thread, FP32 (packed) dense kernel
constexpr int kJUnroll = SD_DENSE_JUNROLL;  // unroll of the packed kernel's 4-particle j step
constexpr int kR64 = 2;          // i-particles per thread, FP64 dense kernel
constexpr int kRV = 2;           // i-particles per thread, VJP dense kernel
constexpr int kJmax = 256;       // largest j-tile
constexpr double kRSafe = 1.0;   // pairs closer than kRSafe * a make the FP32 kernel clamp every tile
constexpr long long kDefaultWatchdog = 1LL << 22;
constexpr int kNearPerParticle = 32;  // near-pass list capacity per particle (overflow: in-place path); an fcc
                                      // lattice at the paper's density lists 18 partners within 3a + skin

// Partition of the (i-block, j-tile) plane over a persistent grid: CTA b takes
// the row-major tile range [b*chunk, min((b+1)*chunk, nIB*nJT)).  The CTAs that
// touch i-block ib are first(ib) .. last(ib); each writes its partial sum for ib
// into slot (b - first(ib)), and the epilogue adds slots in ascending order.
// With sym != 0 (the symmetric FP32 kernel, I == J) only the tiles ib <= jb of
// the plane exist, still row-major: row ib holds jb = ib .. nJT-1.
struct DenseGeom {
    int I;          // i-particles per CTA (threads x R)
    int J;          // j-particles per tile
    int nIB, nJT;   // i-blocks, j-tiles
    long long chunk;
    int grid;
    int maxSlots;
    int sym;        // upper triangle of the plane (mu_ij = mu_ji used once per pair)
    long long nT;   // tiles
};

// A window on the directed kernels' persistent grid, for a shard of rows: the CTAs
// b0 .. b0 + grid - 1 of the full launch, restricted to the tiles [lo, hi) (whole
// i-blocks).  Every CTA computes the same partial sums for the rows it keeps as in
// the full launch, so a shard's rows are bit-identical to the unsharded result.
struct TileWin {
    long long lo = 0, hi = -1;   // hi < 0: every tile
    int b0 = 0;
};

// In a periodic box the padding entries n .. npad-1 have no far-away position under
// the nearest image, so a tile whose i- or j-range reaches index n clamps r^2 (its
// padding terms stay exactly zero).  (The particle count travels with the pair
// constants, not in DenseGeom: a larger DenseGeom cost the symmetric kernel six
// registers.)
__host__ __device__ inline bool geom_pad_tile(const DenseGeom &g, int n, long long i0, long long j0) {
    return i0 + g.I > n || j0 + g.J > n;
}

// First tile of row ib.
__host__ __device__ inline long long geom_rowstart(const DenseGeom &g, int ib) {
    const long long b = ib;
    return g.sym ? b * g.nJT - b * (b - 1) / 2 : b * g.nJT;
}
__host__ __device__ inline int geom_first(const DenseGeom &g, int ib) {
    return static_cast<int>(geom_rowstart(g, ib) / g.chunk);
}
__host__ __device__ inline int geom_last(const DenseGeom &g, int ib) {
    return static_cast<int>((geom_rowstart(g, ib + 1) - 1) / g.chunk);
}

// Periodic box, nearest image only (Sec. 3.1 footnote): side L[d] and 1/L[d] in
// each periodic dimension, 0 and 0 in the others.
struct Box {
    double L[3] = {0.0, 0.0, 0.0};
    double invL[3] = {0.0, 0.0, 0.0};
    int periodic = 0;
};

// Hashed cell list over FP64 positions: cells of side h in unbounded dimensions
// (no bounding box needed), nc[d] >= 3 cells of side L[d] / nc[d] >= h in a
// periodic one (coordinates wrapped into [0, L)); H buckets (power of two),
// particles sorted by bucket, each bucket ascending.
struct CellList {
    double h = 0.0, inv_h = 0.0;
    Box box;
    int nc[3] = {0, 0, 0};          // cells per periodic dimension (0: unbounded)
    int H = 0;
    int nblk = 0;          // scan blocks
    int4 *cell = nullptr;  // [n] integer cell coordinates (w unused)
    uint32_t *key = nullptr;  // [n] bucket of each particle
    int *cnt = nullptr;    // [H] occupancy (zero between builds)
    int *start = nullptr;  // [H+1]
    int *bsum = nullptr;   // [nblk]
    int *sorted = nullptr; // [n]
    int n = 0;             // particles binned
    int *err = nullptr;    // device error word (debug index checks)
};

__device__ __forceinline__ uint32_t cell_hash(int cx, int cy, int cz, int H) {
    return ((static_cast<uint32_t>(cx) * 73856093u) ^ (static_cast<uint32_t>(cy) * 19349663u) ^
            (static_cast<uint32_t>(cz) * 83492791u)) &
           static_cast<uint32_t>(H - 1);
}

// A mirror of an n x 3 FP64 array in the dense kernels' precision: `aos` holds
// float4 / double4 [npad] (x, y, z, 0); for the FP32 modes `soa` additionally
// holds the same values as three float arrays [3][npad] (x..., y..., z...), the
// layout the packed FP32 kernel stages j-tiles from.  Padding entries are zero.
struct Mirror {
    void *aos = nullptr;
    float *soa = nullptr;
};

struct Profiler {
    bool on = false;
    double ms[SD_KERNEL_COUNT] = {};
    int64_t launches[SD_KERNEL_COUNT] = {};
    static constexpr int kMaxPending = 4096;
    cudaEvent_t ev0[kMaxPending] = {}, ev1[kMaxPending] = {};
    int kind[kMaxPending] = {};
    int npending = 0;
    int nevents = 0;  // created event pairs
    bool open = false;   // a range is open (ranges do not nest: an inner one is ignored)
};

struct Allocator {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*free)(void *, void *) = nullptr;
    void *ctx = nullptr;
};

}  // namespace sd

struct sd_handle {
    sd_config cfg{};
    int n = 0, npad = 0;
    int mode = 0;      // MODE_*
    int tensor = 0;    // T_*
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;   // caller's stream
    cudaStream_t cap = nullptr;      // private stream used for graph capture
    sd::Allocator al;
    sd::PairConst pc{};
    double r_near = 0.0, rep_rc = 0.0;
    long long watchdog = sd::kDefaultWatchdog;
    bool inject_stall = false;   // sd_inject_stall: the all-pairs kernels' first CTA skips a copy

    // FP64 state (ping-pong) and the mirror the dense kernel reads: float4 or
    // double4 [npad], positions relative to particle 0 of the state, rewritten by
    // the cell-list build of every step (a pure function of the FP64 state)
    double *x64[2] = {nullptr, nullptr};
    sd::Mirror posm;
    int cur = 0;
    bool pos_set = false;
    bool cells_valid = false;             // cell list matches x64[cur]

    double *fext64 = nullptr;   // [n*3] per-particle external forces
    double *F64 = nullptr;      // [n*3] total force of the current step
    sd::Mirror frcm;            // mirror of F64
    bool forces_const = true;   // no repulsion, no lubrication: F64 depends on nothing that changes
    bool lub = false;           // lubrication friction (Sec. 2.3) in the forces of sd_step
    double *vlag = nullptr;     // [n*3] velocities of the previous step (lubrication), zeroed by set_positions

    // apply / vjp scratch
    double *Fa64 = nullptr;  sd::Mirror frcam;
    double *Wa64 = nullptr;  sd::Mirror wam;
    double *part = nullptr;  size_t part_bytes = 0;   // dense partial sums
    double *part2 = nullptr; size_t part2_bytes = 0;  // second output of the VJP kernel
    void *jpart = nullptr;  size_t jpart_bytes = 0;   // symmetric kernels: source-side sums [tile][3][block],
                                                       // float (FP32 modes) or double (FP64)
    sd::DenseGeom geom{}, geomv{};
    int dense_occ = 0, vjp_occ = 0;
    int sym_nt = 128;   // threads per CTA of the symmetric kernel's chosen block shape

    sd::CellList cl;
    double *near64 = nullptr;   // [n][6] FP64 near-pair corrections (clamped / unclamped variant)
    int2 *near_ent = nullptr;   // [near_cap] candidate pairs of the near pass
    double *near_out = nullptr; // [near_cap][6] their corrections
    unsigned long long *near_n = nullptr;   // entries claimed this pass
    int *near_off = nullptr, *near_cnt = nullptr;   // [n] each particle's run of entries
    int near_cap = 0;
    int *d_flag = nullptr;      // set by the near pass when some pair has r < kRSafe a
    int *d_err = nullptr;

    // graph cache for sd_step: [0] 16 steps, [1] one step; each for both parities of
    // the position buffer the first step reads
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    double g_dt[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    int64_t g_kernels[2][2] = {{0, 0}, {0, 0}};   // kernel nodes in each cached graph

    // adjoint storage (allocated on first use)
    double *ckpt = nullptr; size_t ckpt_bytes = 0;
    double *seg = nullptr;  size_t seg_bytes = 0;
    double *lam = nullptr;  double *gFacc = nullptr;
    // adjoint graphs of one full checkpoint segment (cached per dt and segment length;
    // they hold seg, lam and gFacc: dropped whenever seg is reallocated)
    cudaGraphExec_t adj_rec = nullptr, adj_rev = nullptr;
    double adj_dt = 0.0;
    int64_t adj_K = 0, adj_rec_kernels = 0, adj_rev_kernels = 0;

    sd::Profiler prof;
    int64_t launches = 0;
    bool capturing = false;
    int part_kind = 0;   // 1: sd_mobility_apply_part done, 2: sd_step_part done (their combine may follow)

    // Verlet neighbour lists of sd_step (constant forces only): the near-pair list holds
    // the pairs within r_near + skin of the positions xref it was built from
    bool verlet = false;
    double skin = 0.0;
    double list_cut = 0.0;         // cutoff of the Verlet list: max(r_near, r_c with repulsion, 3a with lubrication)
    double *xref = nullptr;        // [n*3] positions of the last build
    int *d_vl = nullptr;           // [0] rebuild request (bit 2: no list yet), [1] [2] check kernel's
    // the Verlet steps' own candidate list, kept across steps (every other near pass
    // uses near_ent / near_off / near_cnt / near_n): entries, each particle's run, count
    int2 *vent = nullptr;
    int *voff = nullptr, *vcnt = nullptr;
    unsigned long long *vn = nullptr;
    cudaStream_t side = nullptr;   // the rebuild and the near pass, beside the all-pairs kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace sd {

// An NVTX range around an entry point (visible to Nsight tools; a no-op without one).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// errors
sd_status set_error(sd_status st, const std::string &msg);
sd_status cuda_status(cudaError_t e, const char *what);
#define SD_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return ::sd::cuda_status(e_, #call);    \
    } while (0)

// profiling hooks around launches on `st`
void prof_begin(sd_handle *h, int kind, cudaStream_t st);
void prof_end(sd_handle *h, int kind, cudaStream_t st);

// ---- launchers (return cudaGetLastError of the launch)
// cells.cu
cudaError_t launch_stage_pos(sd_handle *h, cudaStream_t st, const double *x64, Mirror posm);
cudaError_t launch_stage_forces(sd_handle *h, cudaStream_t st, const void *src, int src_dtype, int add_ext,
                                double *dst64, Mirror dstm);
// xref != nullptr: a Verlet-list build (copies x64 to xref and clears the rebuild
// request); otherwise any build requests a rebuild of the step's list.
cudaError_t launch_build_cells(sd_handle *h, cudaStream_t st, const double *x64, Mirror posm,
                               double *xref = nullptr);
// Verlet step: the mirror of x64, the clamp flag reset, and the rebuild decision
// (displacements relative to particle 0 since xref; list overflow) in d_vl[0].
cudaError_t launch_verlet_check(sd_handle *h, cudaStream_t st, const double *x64, Mirror posm);
cudaError_t launch_forces_rep(sd_handle *h, cudaStream_t st, const double *x64);
// Verlet step with soft repulsion: the forces from the steps' near-pair list.
cudaError_t launch_forces_list(sd_handle *h, cudaStream_t st, const double *x64);
cudaError_t launch_pad_mirror(sd_handle *h, cudaStream_t st, Mirror m);
// dense.cu
cudaError_t dense_setup(sd_handle *h);
cudaError_t launch_dense(sd_handle *h, cudaStream_t st, Mirror posm, Mirror frcm, double *part,
                         const TileWin *win = nullptr);
// epilogue.cu
// count_zeroed: the list counter is already zero (launch_build_cells zeroes it), so
// the pass needs no memset of its own.
cudaError_t launch_near(sd_handle *h, cudaStream_t st, const double *x64, const void *posm, const double *F64,
                        const void *frcm, bool count_zeroed = false);
// The two halves of the near pass: the candidate list (cutoff r_near, or r_near + skin
// for a Verlet list, which is then sorted by partner within each particle) and the
// FP64 terms of the listed pairs.
cudaError_t launch_near_collect(sd_handle *h, cudaStream_t st, const double *x64, const void *posm,
                                const double *F64, const void *frcm, bool count_zeroed, bool verlet_list);
cudaError_t launch_near_pairs(sd_handle *h, cudaStream_t st, const double *x64, const void *posm, const double *F64,
                              const void *frcm, bool verlet_step = false);
cudaError_t launch_epilogue(sd_handle *h, cudaStream_t st, int out, const double *x64, const void *posm,
                            const double *F64, const void *frcm, void *vout, double dt, double *x64n, int row0 = 0,
                            int row1 = -1, const EpiShard *shard = nullptr, bool vlist = false);
// vjp.cu
cudaError_t vjp_setup(sd_handle *h);
cudaError_t launch_vjp_dense(sd_handle *h, cudaStream_t st, Mirror posm, Mirror frcm, Mirror wm, double *partM,
                             double *partG);
cudaError_t launch_vjp_epilogue(sd_handle *h, cudaStream_t st, const double *x64, const void *posm,
                                const double *F64, const void *frcm, const double *W64, const void *wm,
                                int out_dtype, void *gx_out, void *gF_out, double dt, double *lam_acc,
                                double *gF_acc);

}  // namespace sd
