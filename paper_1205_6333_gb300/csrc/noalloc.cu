// noalloc.cu -- sd_mobility_apply_noalloc: the mobility product v = mu(x) F for
// callers that must not allocate GPU memory.
//
// Who needs it: code that runs while a CUDA stream is being captured into a
// graph (cudaMalloc cannot be captured and a graph replay could not repeat it),
// hosts that hand a plug-in a fixed device-memory budget and forbid further
// allocation, and latency-critical loops that cannot afford cudaMalloc/cudaFree
// (which may synchronise the device).  Such a caller cannot create an sd_handle,
// because a handle allocates its buffers.
//
// This entry point allocates nothing.  Its only working memory (FP32 copies of
// the inputs and the per-split partial sums of the all-pairs kernel) lives in
// one file-scope __device__ array of kScratchBytes (about 14 MB), which every
// GPU that loads the library holds until the process exits.  That array bounds
// the problem size to n <= kMaxN (65,536 particles).
//
// The kernels here are a self-contained variant of the all-pairs sum of
// dense.cu: FP32 pair terms with compensated (two-float) accumulation,
// j-split across CTAs with partial sums in the scratch array, the self term and
// overlapping pairs handled exactly inside the pair loop (so no cell list and
// no FP64 near-pair pass are needed), and a final FP64 reduction.
#include <cmath>
#include <mutex>
#include <string>

#include "sd_internal.h"

namespace sd {
namespace {

constexpr int kMaxN = 65536;          // largest n the scratch array holds
constexpr int kSplits = 8;            // j-splits (partial sums per particle)
constexpr int kThreads = 128;         // threads per CTA = i-particles per CTA
constexpr int kTile = 128;            // j-particles per shared-memory tile
constexpr size_t kMirrorFloats = 6 * static_cast<size_t>(kMaxN);                  // x y z Fx Fy Fz (SoA)
constexpr size_t kPartialDoubles = static_cast<size_t>(kSplits) * 3 * kMaxN;       // [split][dim][i]
constexpr size_t kScratchBytes = kMirrorFloats * sizeof(float) + kPartialDoubles * sizeof(double);
constexpr int kMaxDevices = 64;

static_assert(kMaxN % kTile == 0, "the scratch stride must hold whole tiles");

// The scratch array.  Host code must not pass its name to a kernel: on the host
// the name is only a stand-in, so its device address is looked up once per
// device with cudaGetSymbolAddress (noalloc_scratch below).
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call on each device).
sd_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(SD_ERR_UNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_status(e, "cudaGetSymbolAddress of the no-alloc scratch");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SD_OK;
}

struct NaArgs {
    const double *x, *F;
    double *V;
    int n, npad;       // npad: n rounded up to a whole tile
    int chunk;         // j-particles per split (a multiple of kTile)
    float *mir;        // scratch: SoA x, y, z, Fx, Fy, Fz with stride kMaxN
    double *part;      // scratch: [split][dim][kMaxN]
    PairConst pc;
};

// Mirror of positions (relative to particle 0) and forces in FP32; entries
// n..npad-1 are rewritten on every call (far away, zero force), since the array
// keeps whatever an earlier call left there.
__global__ void na_stage_kernel(NaArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.npad) return;
    float v[6];
    if (i < a.n) {
        for (int d = 0; d < 3; ++d) {
            v[d] = static_cast<float>(a.x[3 * i + d] - a.x[d]);
            v[3 + d] = static_cast<float>(a.F[3 * i + d]);
        }
    } else {
        v[0] = 1.0e18f;
        v[1] = v[2] = v[3] = v[4] = v[5] = 0.0f;
    }
    for (int k = 0; k < 6; ++k) a.mir[k * static_cast<size_t>(kMaxN) + i] = v[k];
}

// Exact pair term from zero (the overlap form for RPY when r < 2a), FP32.
template <int TENSOR>
__device__ __forceinline__ void na_exact(float dx, float dy, float dz, float fx, float fy, float fz,
                                         const PairConst &c, float &ax, float &ay, float &az) {
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0f) {
        if (TENSOR == T_RPY) {   // coincident spheres: T^(0) = I
            ax += fx;
            ay += fy;
            az += fz;
        } else {                 // undefined for RP / Oseen: poison the result
            ax = ay = az = __int_as_float(0x7fc00000);
        }
        return;
    }
    const float r = sqrtf(r2);
    float A, B;
    if (TENSOR == T_RPY && r < static_cast<float>(c.two_a)) {
        A = 1.0f - 9.0f * r / (32.0f * static_cast<float>(c.a));
        B = 3.0f / (32.0f * static_cast<float>(c.a) * r);
    } else if (TENSOR == T_OSEEN) {
        A = c.c1_f / r;
        B = A / r2;
    } else {
        const float ri = 1.0f / r, ri2 = ri * ri;
        A = ri * (c.c1_f + c.c3_f * ri2);
        B = ri * ri2 * (c.c1_f + c.m3c3_f * ri2);
    }
    const float s = B * (dx * fx + dy * fy + dz * fz);
    ax += A * fx + s * dx;
    ay += A * fy + s * dy;
    az += A * fz + s * dz;
}

// CTA (ib, s): targets ib*kThreads + tid against j in [s*chunk, (s+1)*chunk).
template <int TENSOR>
__global__ void __launch_bounds__(kThreads) na_dense_kernel(NaArgs a) {
    constexpr int TD = (TENSOR == T_OSEEN) ? T_OSEEN : T_RP;
    __shared__ float4 s_p[kTile], s_f[kTile];
    const int tid = threadIdx.x;
    const int i = blockIdx.x * kThreads + tid;
    const int j0 = blockIdx.y * a.chunk;
    const int j1 = min(j0 + a.chunk, a.npad);
    const size_t M = kMaxN;
    const float xi = a.mir[i], yi = a.mir[M + i], zi = a.mir[2 * M + i];
    float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
    for (int jt = j0; jt < j1; jt += kTile) {
        const int j = jt + tid;
        s_p[tid] = make_float4(a.mir[j], a.mir[M + j], a.mir[2 * M + j], 0.0f);
        s_f[tid] = make_float4(a.mir[3 * M + j], a.mir[4 * M + j], a.mir[5 * M + j], 0.0f);
        __syncthreads();
        float ax = 0.f, ay = 0.f, az = 0.f;
        for (int k = 0; k < kTile; ++k) {
            const float4 p = s_p[k], f = s_f[k];
            const float dx = xi - p.x, dy = yi - p.y, dz = zi - p.z;
            if (dx * dx + dy * dy + dz * dz >= a.pc.r2min_f) {
                pair_f32<TD, false>(xi, yi, zi, p, f, a.pc, ax, ay, az);
            } else if (jt + k != i) {   // overlapping pair (rare); the self pair is skipped
                na_exact<TENSOR>(dx, dy, dz, f.x, f.y, f.z, a.pc, ax, ay, az);
            }
        }
        fold2(hx, lx, ax);
        fold2(hy, ly, ay);
        fold2(hz, lz, az);
        __syncthreads();
    }
    double *p = a.part + static_cast<size_t>(blockIdx.y) * 3 * M;
    p[i] = static_cast<double>(hx) + lx;
    p[M + i] = static_cast<double>(hy) + ly;
    p[2 * M + i] = static_cast<double>(hz) + lz;
}

// V_i = mu0 (F_i + sum of the split partials in split order), FP64.
__global__ void na_finish_kernel(NaArgs a, int nsplit) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const size_t M = kMaxN;
    for (int d = 0; d < 3; ++d) {
        double v = a.F[3 * i + d];
        for (int s = 0; s < nsplit; ++s) v += a.part[(static_cast<size_t>(s) * 3 + d) * M + i];
        a.V[3 * i + d] = a.pc.mu0 * v;
    }
}

}  // namespace
}  // namespace sd

using namespace sd;

extern "C" sd_status sd_mobility_apply_noalloc(const double *x, const double *F, double *V, int32_t n, double a,
                                               double eta, int32_t tensor, void *stream) {
    if (n < 0) return set_error(SD_ERR_ARG, "n must be >= 0");
    if (n > kMaxN)
        return set_error(SD_ERR_ARG, "sd_mobility_apply_noalloc: n = " + std::to_string(n) +
                                         " exceeds the limit of its fixed scratch array (65536 particles)");
    if (!(a > 0.0) || !(eta > 0.0) || !std::isfinite(a) || !std::isfinite(eta))
        return set_error(SD_ERR_ARG, "a and eta must be finite and > 0");
    if (tensor < 0 || tensor > 2) return set_error(SD_ERR_ARG, "unknown tensor");
    if (n == 0) return SD_OK;
    if (!x || !F || !V) return set_error(SD_ERR_ARG, "x, F and V must be device pointers");
    void *base = nullptr;
    sd_status s = noalloc_scratch(&base);
    if (s != SD_OK) return s;

    NaArgs g;
    g.x = x;
    g.F = F;
    g.V = V;
    g.n = n;
    g.npad = ((n + kTile - 1) / kTile) * kTile;
    const int tiles = g.npad / kTile;
    const int split = std::min(kSplits, tiles);
    g.chunk = ((tiles + split - 1) / split) * kTile;
    const int nsplit = (g.npad + g.chunk - 1) / g.chunk;
    g.mir = static_cast<float *>(base);
    g.part = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + kMirrorFloats * sizeof(float));
    PairConst &pc = g.pc;
    pc.a = a;
    pc.two_a = 2.0 * a;
    pc.mu0 = 1.0 / (6.0 * 3.14159265358979323846 * eta * a);
    pc.r2min_d = 4.0 * a * a;
    pc.c1_d = 0.75 * a;
    pc.c3_d = 0.5 * a * a * a;
    pc.m3c3_d = -1.5 * a * a * a;
    pc.r2min_f = static_cast<float>(pc.r2min_d);
    pc.c1_f = static_cast<float>(pc.c1_d);
    pc.c3_f = static_cast<float>(pc.c3_d);
    pc.m3c3_f = static_cast<float>(pc.m3c3_d);

    // An error left by the caller's earlier work is reported as such and left in
    // place (peeked, not cleared); each launch below is then checked on its own.
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess)
        return set_error(SD_ERR_CUDA, std::string("sd_mobility_apply_noalloc: a CUDA error from earlier work is "
                                                  "pending (not cleared): ") + cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    na_stage_kernel<<<(g.npad + 255) / 256, 256, 0, st>>>(g);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "sd_mobility_apply_noalloc: staging launch");
    const dim3 grid(g.npad / kThreads, nsplit);
    switch (tensor) {
        case SD_TENSOR_RPY: na_dense_kernel<T_RPY><<<grid, kThreads, 0, st>>>(g); break;
        case SD_TENSOR_RP: na_dense_kernel<T_RP><<<grid, kThreads, 0, st>>>(g); break;
        default: na_dense_kernel<T_OSEEN><<<grid, kThreads, 0, st>>>(g); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "sd_mobility_apply_noalloc: all-pairs launch");
    na_finish_kernel<<<(n + 127) / 128, 128, 0, st>>>(g, nsplit);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "sd_mobility_apply_noalloc: reduction launch");
    return SD_OK;
}
