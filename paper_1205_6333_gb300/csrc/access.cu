// access.cu -- the memory-access study of the paper's appendix (App. A,
// Algorithms 3 and 4), on GB300.
//
// N threads; thread j starts from in[j] and adds the N elements in[map(k)],
// k = 0 .. N-1, then stores its sum.  The maps (p = 131, M = 32):
//   linear     k -> k
//   strided    k -> k p mod N
//   unordered  k -> (k p + j M) mod N        (j: the global thread index)
// The kernels:
//   naive        every thread loads its own map(k) from global memory;
//   tiling       the block loads a tile of blockDim elements into shared memory,
//                one per thread (thread n of the block loads map(m + n) with its
//                own j), and every thread adds the whole tile;
//   smalltiling  the same with warp-size tiles loaded by the first warp;
//   bulk         (linear map only) tiling whose tiles arrive by cp.async.bulk
//                copies into a double buffer, completing on an mbarrier.
// Elements are float or float4 (added componentwise).  The maps advance by one
// addition and a conditional subtraction per k instead of a modulo, so the loops
// measure memory access, not integer division.
#include "sd_internal.h"

namespace sd {

enum { ACC_NAIVE = 0, ACC_TILING = 1, ACC_SMALLTILING = 2, ACC_BULK = 3 };
enum { MAP_LINEAR = 0, MAP_STRIDED = 1, MAP_UNORDERED = 2 };
constexpr unsigned kAccP = 131, kAccM = 32;

__device__ int g_access_err;   // bounded-wait time-outs of the bulk kernel

template <typename T>
__device__ __forceinline__ void acc_add(T &s, const T &v);
template <>
__device__ __forceinline__ void acc_add<float>(float &s, const float &v) {
    s = __fadd_rn(s, v);
}
template <>
__device__ __forceinline__ void acc_add<float4>(float4 &s, const float4 &v) {
    s.x = __fadd_rn(s.x, v.x);
    s.y = __fadd_rn(s.y, v.y);
    s.z = __fadd_rn(s.z, v.z);
    s.w = __fadd_rn(s.w, v.w);
}
template <typename T>
__device__ __forceinline__ T acc_zero();
template <>
__device__ __forceinline__ float acc_zero<float>() {
    return 0.0f;
}
template <>
__device__ __forceinline__ float4 acc_zero<float4>() {
    return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// map(k) for the thread of global index j, advanced by `stride` positions of k per
// call of next() (one addition and a conditional subtraction instead of a modulo).
template <int MAP>
struct AccMap {
    unsigned idx, step, n;
    __device__ __forceinline__ AccMap(unsigned k0, unsigned j, unsigned N, unsigned stride) : n(N) {
        const unsigned long long base = MAP == MAP_UNORDERED ? static_cast<unsigned long long>(j) * kAccM : 0ull;
        const unsigned long long mult = MAP == MAP_LINEAR ? 1ull : kAccP;
        idx = static_cast<unsigned>((static_cast<unsigned long long>(k0) * mult + base) % N);
        step = static_cast<unsigned>(static_cast<unsigned long long>(stride) * mult % N);
    }
    __device__ __forceinline__ void next() {
        idx += step;   // idx, step < N <= 2^31 - 1: no wrap-around
        if (idx >= n) idx -= n;
    }
};

template <typename T, int MAP>
__global__ void access_naive(const T *__restrict__ in, T *__restrict__ out, unsigned N) {
    const unsigned j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    T sum = in[j];
    AccMap<MAP> m(0, j, N, 1);
    for (unsigned k = 0; k < N; ++k) {
        acc_add(sum, in[m.idx]);
        m.next();
    }
    out[j] = sum;
}

// TILE = 0: tiles of blockDim elements loaded by all threads; TILE = 32: warp-size
// tiles loaded by the first warp.  Elements past N load as zero.
template <typename T, int MAP, int TILE>
__global__ void access_tiling(const T *__restrict__ in, T *__restrict__ out, unsigned N) {
    extern __shared__ __align__(16) unsigned char acc_smem[];
    T *s_data = reinterpret_cast<T *>(acc_smem);
    const unsigned n = threadIdx.x;
    const unsigned j = blockIdx.x * blockDim.x + n;
    const unsigned tile = TILE ? TILE : blockDim.x;
    T sum = j < N ? in[j] : acc_zero<T>();
    AccMap<MAP> m(n, j, N, tile);   // this thread loads map(m0 + n), m0 = 0, tile, 2 tile, ...
    for (unsigned m0 = 0; m0 < N; m0 += tile) {
        if (n < tile) {
            s_data[n] = (m0 + n < N) ? in[m.idx] : acc_zero<T>();
            m.next();
        }
        __syncthreads();
        for (unsigned k = 0; k < tile; ++k) acc_add(sum, s_data[k]);
        __syncthreads();
    }
    if (j < N) out[j] = sum;
}

// Linear map, tiles of blockDim elements copied by cp.async.bulk (thread 0 issues,
// double buffer, mbarrier completion with bounded waits); the ragged last tile is
// loaded by the threads.
template <typename T>
__global__ void access_bulk(const T *__restrict__ in, T *__restrict__ out, unsigned N, long long wd) {
    extern __shared__ __align__(128) unsigned char acc_smem[];
    __shared__ __align__(8) uint64_t bars[2];
    T *s_data = reinterpret_cast<T *>(acc_smem);   // [2][blockDim]
    const unsigned n = threadIdx.x, B = blockDim.x;
    const unsigned j = blockIdx.x * B + n;
    const unsigned nfull = N / B;                  // tiles copied in bulk
    const uint32_t tile_bytes = B * sizeof(T);     // a multiple of 16 (host-checked)
    T sum = j < N ? in[j] : acc_zero<T>();
    int issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0;
    if (n == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](unsigned t, int st) {
        mbar_arrive_expect_tx(&bars[st], tile_bytes);
        bulk_g2s(s_data + st * B, in + static_cast<size_t>(t) * B, tile_bytes, &bars[st]);
        if (st == 0) ++issued0; else ++issued1;
    };
    if (n == 0)
        for (unsigned t = 0; t < 2 && t < nfull; ++t) issue(t, static_cast<int>(t));
    bool aborted = false;
    for (unsigned t = 0; t < nfull; ++t) {
        const int st = static_cast<int>(t & 1);
        const bool ok = mbar_wait_bounded(&bars[st], (t >> 1) & 1, wd);
        if (ok && n == 0) {
            if (st == 0) ++waited0; else ++waited1;
        }
        const T *tp = s_data + st * B;
        for (unsigned k = 0; k < B; ++k) acc_add(sum, tp[k]);
        aborted = __syncthreads_or(!ok) != 0;   // uniform over the block
        if (aborted) break;
        if (n == 0 && t + 2 < nfull) issue(t + 2, st);
    }
    if (aborted) {
        if (n == 0) atomicOr(&g_access_err, 1);
    } else if (nfull * B < N) {   // the ragged last tile by plain loads
        const unsigned m0 = nfull * B;
        s_data[n] = (m0 + n < N) ? in[m0 + n] : acc_zero<T>();
        __syncthreads();
        for (unsigned k = 0; k < B; ++k) acc_add(sum, s_data[k]);
    }
    if (j < N) out[j] = sum;
    if (n == 0) {
        for (int k = waited0; k < issued0; ++k)
            if (!mbar_wait_bounded(&bars[0], k & 1, drain_limit(wd))) atomicOr(&g_access_err, 1);
        for (int k = waited1; k < issued1; ++k)
            if (!mbar_wait_bounded(&bars[1], k & 1, drain_limit(wd))) atomicOr(&g_access_err, 1);
    }
}

template <typename T, int MAP>
static cudaError_t access_launch_t(int algo, unsigned N, int block, const void *in, void *out, cudaStream_t st) {
    const T *src = static_cast<const T *>(in);
    T *dst = static_cast<T *>(out);
    const unsigned grid = (N + block - 1) / block;
    switch (algo) {
        case ACC_NAIVE: access_naive<T, MAP><<<grid, block, 0, st>>>(src, dst, N); break;
        case ACC_TILING:
            access_tiling<T, MAP, 0><<<grid, block, block * sizeof(T), st>>>(src, dst, N);
            break;
        case ACC_SMALLTILING:
            access_tiling<T, MAP, 32><<<grid, block, 32 * sizeof(T), st>>>(src, dst, N);
            break;
        default:
            if constexpr (MAP == MAP_LINEAR) {
                access_bulk<T><<<grid, block, 2 * block * sizeof(T), st>>>(src, dst, N, kDefaultWatchdog);
            } else {
                return cudaErrorInvalidValue;
            }
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t access_launch_m(int algo, int map, unsigned N, int block, const void *in, void *out,
                                   cudaStream_t st) {
    switch (map) {
        case MAP_LINEAR: return access_launch_t<T, MAP_LINEAR>(algo, N, block, in, out, st);
        case MAP_STRIDED: return access_launch_t<T, MAP_STRIDED>(algo, N, block, in, out, st);
        default: return access_launch_t<T, MAP_UNORDERED>(algo, N, block, in, out, st);
    }
}

}  // namespace sd

using namespace sd;

extern "C" sd_status sd_access_run(int32_t algo, int32_t map, int32_t vec4, int32_t n, int32_t block, const void *in,
                                   void *out, void *stream) {
    if (algo < ACC_NAIVE || algo > ACC_BULK || map < MAP_LINEAR || map > MAP_UNORDERED || n < 0)
        return set_error(SD_ERR_ARG, "unknown algorithm / map, or n < 0");
    if (algo == ACC_BULK && map != MAP_LINEAR) return set_error(SD_ERR_ARG, "the bulk kernel reads linear tiles only");
    if (block < 32 || block > 1024 || block % 32) return set_error(SD_ERR_ARG, "block must be a multiple of 32 in [32, 1024]");
    if (algo == ACC_BULK && (reinterpret_cast<uintptr_t>(in) & 15))
        return set_error(SD_ERR_ARG, "the bulk kernel needs a 16-byte aligned input");
    if (n > 0 && (!in || !out)) return set_error(SD_ERR_ARG, "in or out is NULL");
    if (n == 0) return SD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = vec4 ? access_launch_m<float4>(algo, map, static_cast<unsigned>(n), block, in, out, st)
                         : access_launch_m<float>(algo, map, static_cast<unsigned>(n), block, in, out, st);
    if (e != cudaSuccess) return cuda_status(e, "access study kernel");
    return SD_OK;
}

extern "C" sd_status sd_access_status(void) {
    int bits = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&bits, g_access_err, sizeof(int));
    if (e != cudaSuccess) return cuda_status(e, "access study status");
    if (bits) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_access_err, &zero, sizeof(int));
        return set_error(SD_ERR_TIMEOUT, "bulk copy wait gave up");
    }
    return SD_OK;
}
