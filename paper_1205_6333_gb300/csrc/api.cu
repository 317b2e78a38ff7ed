// api.cu -- the C ABI of include/sd.h for single systems: handle life cycle,
// argument checks, buffers, error reporting, CUDA-graph replay of Euler steps
// (Sec. 3.1), the adjoint sweep, and the per-kernel event profiler.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sd_internal.h"

namespace sd {

static thread_local std::string g_last_error;

sd_status set_error(sd_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

sd_status cuda_status(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(SD_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return set_error(SD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------- profiler

void prof_begin(sd_handle *h, int kind, cudaStream_t st) {
    Profiler &p = h->prof;
    if (!p.on || h->capturing || p.open || p.npending >= Profiler::kMaxPending) return;
    const int k = p.npending;
    if (k >= p.nevents) {
        cudaEventCreate(&p.ev0[k]);
        cudaEventCreate(&p.ev1[k]);
        p.nevents = k + 1;
    }
    p.kind[k] = kind;
    cudaEventRecord(p.ev0[k], st);
    p.open = true;
}

void prof_end(sd_handle *h, int kind, cudaStream_t st) {
    Profiler &p = h->prof;
    if (!p.on || h->capturing || !p.open || p.kind[p.npending] != kind) return;
    cudaEventRecord(p.ev1[p.npending], st);
    ++p.npending;
    p.open = false;
}

static cudaError_t prof_collect(Profiler &p) {
    for (int k = 0; k < p.npending; ++k) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(p.ev1[k]);
        if (e != cudaSuccess) return e;
        e = cudaEventElapsedTime(&ms, p.ev0[k], p.ev1[k]);
        if (e != cudaSuccess) return e;
        p.ms[p.kind[k]] += ms;
        p.launches[p.kind[k]] += 1;
    }
    p.npending = 0;
    return cudaSuccess;
}

static void prof_destroy(Profiler &p) {
    for (int k = 0; k < p.nevents; ++k) {
        cudaEventDestroy(p.ev0[k]);
        cudaEventDestroy(p.ev1[k]);
    }
    p.nevents = p.npending = 0;
}

// ---------------------------------------------------------------- memory

static void *dalloc(sd_handle *h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (h->al.alloc) return h->al.alloc(bytes, h->al.ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void dfree(sd_handle *h, void *p) {
    if (!p) return;
    if (h->al.free)
        h->al.free(p, h->al.ctx);
    else
        cudaFree(p);
}

template <typename T>
static bool dalloc_t(sd_handle *h, T *&p, size_t count) {
    p = static_cast<T *>(dalloc(h, count * sizeof(T)));
    return p != nullptr;
}

static size_t v4size(const sd_handle *h) { return h->mode == MODE_FP64 ? sizeof(dbl4) : sizeof(float4); }

// ---------------------------------------------------------------- device status

static sd_status status_from_bits(int bits) {
    if (bits & DEV_ERR_TIMEOUT) return set_error(SD_ERR_TIMEOUT, "a bounded device-side wait timed out");
    if (bits & DEV_ERR_QUEUE) return set_error(SD_ERR_TIMEOUT, "batched work queue inconsistent");
    if (bits & DEV_ERR_COINCIDENT)
        return set_error(SD_ERR_COINCIDENT, "two distinct particles at zero separation (RP/Oseen tensor undefined)");
    if (bits & DEV_ERR_NONFINITE) return set_error(SD_ERR_NONFINITE, "non-finite value in positions or forces");
    if (bits & DEV_ERR_BOUNDS) return set_error(SD_ERR_INTERNAL, "a device-side index check failed");
    return SD_OK;
}

// Synchronise the stream, read and clear the device error word.
static sd_status sync_check(sd_handle *h) {
    SD_CUDA(cudaStreamSynchronize(h->stream));
    int bits = 0;
    SD_CUDA(cudaMemcpy(&bits, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (bits) SD_CUDA(cudaMemset(h->d_err, 0, sizeof(int)));
    return status_from_bits(bits);
}

static sd_status launch_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) return cuda_status(e, what);
    return SD_OK;
}

// ---------------------------------------------------------------- one Euler step

// A Verlet step (constant forces).  The check kernel writes the mirror, the rebuild
// decision and the clamp flag.  Then two branches run side by side: the all-pairs
// kernel on st, and on the side stream the rebuild kernels (cell list and
// xref = x_in; the candidate list within r_near + skin, each particle's run sorted by
// partner), which read the decision and return at once when no rebuild is due,
// followed by the FP64 terms of the listed pairs.  The Euler epilogue joins them.
// Neither branch writes what the other reads.  A fresh and a reused list give the
// same result bit for bit: each particle's list is sorted by partner and entries
// beyond r_near add exact zeros.
static cudaError_t launch_verlet_step(sd_handle *h, cudaStream_t st, double dt, const double *x_in, double *x_out) {
    cudaError_t e = launch_verlet_check(h, st, x_in, h->posm);
    // with soft repulsion the forces need the list: rebuild (when due) and forces first
    cudaStream_t rb = h->forces_const ? h->side : st;
    if (!h->forces_const) {
        if (e == cudaSuccess) e = launch_build_cells(h, st, x_in, h->posm, h->xref);
        if (e == cudaSuccess) e = launch_near_collect(h, st, x_in, h->posm.aos, h->F64, h->frcm.aos, true, true);
        if (e == cudaSuccess) e = launch_forces_list(h, st, x_in);
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    if (h->forces_const && e == cudaSuccess) e = launch_build_cells(h, rb, x_in, h->posm, h->xref);
    prof_begin(h, SD_KERNEL_NEAR, h->side);
    if (h->forces_const && e == cudaSuccess)
        e = launch_near_collect(h, rb, x_in, h->posm.aos, h->F64, h->frcm.aos, true, true);
    if (e == cudaSuccess) e = launch_near_pairs(h, h->side, x_in, h->posm.aos, h->F64, h->frcm.aos, true);
    prof_end(h, SD_KERNEL_NEAR, h->side);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->side);
    if (e == cudaSuccess) e = launch_dense(h, st, h->posm, h->frcm, h->part);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_join, 0);
    if (e == cudaSuccess)
        e = launch_epilogue(h, st, OUT_EULER, x_in, h->posm.aos, h->F64, h->frcm.aos, nullptr, dt, x_out, 0, -1,
                            nullptr, true);
    return e;
}

// x_out = x_in + dt mu(x_in) F(x_in); the cell-list build also writes the mirror of x_in.
static cudaError_t launch_step(sd_handle *h, cudaStream_t st, double dt, const double *x_in, double *x_out) {
    if (h->verlet) return launch_verlet_step(h, st, dt, x_in, x_out);
    cudaError_t e = launch_build_cells(h, st, x_in, h->posm);
    if (e == cudaSuccess && !h->forces_const) e = launch_forces_rep(h, st, x_in);
    if (e == cudaSuccess) e = launch_near(h, st, x_in, h->posm.aos, h->F64, h->frcm.aos, true);
    if (e == cudaSuccess) e = launch_dense(h, st, h->posm, h->frcm, h->part);
    if (e == cudaSuccess) e = launch_epilogue(h, st, OUT_EULER, x_in, h->posm.aos, h->F64, h->frcm.aos, nullptr, dt, x_out);
    return e;
}

constexpr int kGraphSteps = 16;   // steps per captured graph (even: ends on the starting buffer)

static void drop_adjoint_graphs(sd_handle *h) {
    if (h->adj_rec) cudaGraphExecDestroy(h->adj_rec);
    if (h->adj_rev) cudaGraphExecDestroy(h->adj_rev);
    h->adj_rec = h->adj_rev = nullptr;
    h->adj_K = 0;
}

static void drop_graphs(sd_handle *h) {
    for (int k = 0; k < 2; ++k)
        for (int c = 0; c < 2; ++c) {
            if (h->gexec[k][c]) cudaGraphExecDestroy(h->gexec[k][c]);
            h->gexec[k][c] = nullptr;
        }
    drop_adjoint_graphs(h);
}

// The handle's one staging buffer `seg` (host-pointer calls, the adjoint's recompute
// segment) holds at least `need` bytes.  Every reallocation goes through here: the
// cached adjoint graphs captured the old address, so they are dropped first.
static sd_status ensure_seg(sd_handle *h, size_t need, const char *what) {
    if (h->seg && h->seg_bytes >= need) return SD_OK;
    drop_adjoint_graphs(h);
    dfree(h, h->seg);
    h->seg = static_cast<double *>(dalloc(h, need));
    h->seg_bytes = h->seg ? need : 0;
    if (!h->seg) return set_error(SD_ERR_OOM, what);
    return SD_OK;
}

// kGraphSteps (k = 0) or one (k = 1) Euler steps from buffer `cur`, captured into a
// graph and cached per (k, cur, dt): a step's dozen launches become one graph launch
// (the GPU no longer waits on each small launch at small N, nor after a host round trip).
static sd_status capture_steps(sd_handle *h, double dt, int cur, int k) {
    if (h->gexec[k][cur]) cudaGraphExecDestroy(h->gexec[k][cur]);
    h->gexec[k][cur] = nullptr;
    cudaGraph_t graph = nullptr;
    SD_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    const int64_t l0 = h->launches;
    cudaError_t e = cudaSuccess;
    int c = cur;
    const int steps = k == 0 ? kGraphSteps : 1;
    for (int q = 0; q < steps && e == cudaSuccess; ++q) {
        e = launch_step(h, h->cap, dt, h->x64[c], h->x64[1 - c]);
        c = 1 - c;
    }
    h->capturing = false;
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
    h->g_kernels[k][cur] = h->launches - l0;
    h->launches = l0;
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_status(e, "capture of Euler steps");
    }
    if (e2 != cudaSuccess) return cuda_status(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->gexec[k][cur], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate");
    h->g_dt[k][cur] = dt;
    return SD_OK;
}

// nsteps Euler steps: cached 16-step graphs, then cached single-step graphs; with the
// profiler on, eager launches so that every kernel family gets its own event pair.
static sd_status run_steps(sd_handle *h, double dt, int64_t nsteps) {
    int64_t left = nsteps;
    auto replay = [&](int k) -> sd_status {
        const int c = h->cur;
        if (!h->gexec[k][c] || h->g_dt[k][c] != dt) {
            sd_status s = capture_steps(h, dt, c, k);
            if (s != SD_OK) return s;
        }
        SD_CUDA(cudaGraphLaunch(h->gexec[k][c], h->stream));
        h->launches += h->g_kernels[k][c];
        return SD_OK;
    };
    if (!h->prof.on) {
        while (left >= kGraphSteps) {
            sd_status s = replay(0);
            if (s != SD_OK) return s;
            left -= kGraphSteps;   // even count: the state ends in buffer h->cur again
        }
    }
    for (; left > 0; --left) {
        const int c = h->cur;
        if (!h->prof.on) {
            sd_status s = replay(1);
            if (s != SD_OK) return s;
        } else {
            sd_status s = launch_check(launch_step(h, h->stream, dt, h->x64[c], h->x64[1 - c]), "Euler step");
            if (s != SD_OK) return s;
        }
        h->cur = 1 - c;
    }
    h->cells_valid = false;
    return SD_OK;
}

// The adjoint's work on one checkpoint segment of K steps, on stream st:
//   recompute (part 0): x_{k+1} = x_k + dt v(x_k) into seg, k = 0 .. K-2;
//   reverse (part 1), k = K-1 .. 0: W = lambda; lambda += dt (dv/dx(x_k))^T W; gF += dt mu(x_k) W.
static cudaError_t adjoint_segment(sd_handle *h, cudaStream_t st, double dt, int64_t len, int part) {
    const size_t n3 = 3 * static_cast<size_t>(h->n);
    auto segx = [&](int64_t k) { return h->seg + static_cast<size_t>(k) * n3; };
    cudaError_t e = cudaSuccess;
    if (part == 0) {
        for (int64_t k = 0; k + 1 < len && e == cudaSuccess; ++k) e = launch_step(h, st, dt, segx(k), segx(k + 1));
        return e;
    }
    for (int64_t k = len - 1; k >= 0 && e == cudaSuccess; --k) {
        e = launch_stage_forces(h, st, h->lam, SD_DTYPE_F64, 0, h->Wa64, h->wam);
        if (e == cudaSuccess) e = launch_build_cells(h, st, segx(k), h->posm);
        if (e == cudaSuccess) e = launch_vjp_dense(h, st, h->posm, h->frcm, h->wam, h->part, h->part2);
        if (e == cudaSuccess)
            e = launch_vjp_epilogue(h, st, segx(k), h->posm.aos, h->F64, h->frcm.aos, h->Wa64, h->wam.aos, -1,
                                    nullptr, nullptr, dt, h->lam, h->gFacc);
    }
    return e;
}

// Graphs of both parts for a full segment of K steps (the recompute part only when
// K > 1), cached per (dt, K).
static sd_status capture_adjoint(sd_handle *h, double dt, int64_t K) {
    drop_adjoint_graphs(h);
    for (int part = 0; part < 2; ++part) {
        if (part == 0 && K < 2) continue;
        cudaGraph_t graph = nullptr;
        SD_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        h->capturing = true;
        const int64_t l0 = h->launches;
        cudaError_t e = adjoint_segment(h, h->cap, dt, K, part);
        h->capturing = false;
        cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
        const int64_t kernels = h->launches - l0;
        h->launches = l0;
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            drop_adjoint_graphs(h);
            return cuda_status(e, "capture of an adjoint segment");
        }
        if (e2 != cudaSuccess) {
            drop_adjoint_graphs(h);
            return cuda_status(e2, "cudaStreamEndCapture");
        }
        e = cudaGraphInstantiate(part == 0 ? &h->adj_rec : &h->adj_rev, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            drop_adjoint_graphs(h);
            return cuda_status(e, "cudaGraphInstantiate");
        }
        (part == 0 ? h->adj_rec_kernels : h->adj_rev_kernels) = kernels;
    }
    h->adj_dt = dt;
    h->adj_K = K;
    return SD_OK;
}

}  // namespace sd

using namespace sd;

extern "C" {

const char *sd_last_error(void) { return g_last_error.c_str(); }

const char *sd_version(void) { return "sd-gb300 1.0 (sm_103a)"; }

void sd_config_init(sd_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->a = 1.0;
    cfg->eta = 1.0;
    cfg->tensor = SD_TENSOR_RPY;
    cfg->prec = SD_PREC_FP32C;
    cfg->r_near = 2.5;
    cfg->rep_rc = 2.5;
    cfg->verlet_skin = 0.5;
}

static sd_status validate_common(const sd_config *cfg) {
    if (!cfg) return set_error(SD_ERR_ARG, "cfg is NULL");
    if (!(cfg->a > 0.0) || !std::isfinite(cfg->a)) return set_error(SD_ERR_ARG, "radius a must be finite and > 0");
    if (!(cfg->eta > 0.0) || !std::isfinite(cfg->eta)) return set_error(SD_ERR_ARG, "viscosity eta must be > 0");
    if (cfg->tensor < 0 || cfg->tensor > 2) return set_error(SD_ERR_ARG, "unknown tensor");
    if (cfg->prec < 0 || cfg->prec > 2) return set_error(SD_ERR_ARG, "unknown precision");
    for (int d = 0; d < 3; ++d) {
        if (cfg->box[d] < 0.0 || !std::isfinite(cfg->box[d])) return set_error(SD_ERR_ARG, "box must be >= 0");
        if (!std::isfinite(cfg->gravity[d])) return set_error(SD_ERR_ARG, "gravity must be finite");
    }
    if (cfg->dense_kernel < 0 || cfg->dense_kernel > 2) return set_error(SD_ERR_ARG, "unknown dense kernel");
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
        return set_error(SD_ERR_ARG, "alloc and free callbacks must be given together");
    return SD_OK;
}

sd_status sd_create(const sd_config *cfg, sd_handle **out) {
    if (!out) return set_error(SD_ERR_ARG, "out is NULL");
    *out = nullptr;
    sd_status s = validate_common(cfg);
    if (s != SD_OK) return s;
    if (cfg->n < 0 || cfg->n > (1 << 24)) return set_error(SD_ERR_ARG, "n must be in [0, 2^24]");
    const double a = cfg->a;
    const double r_near = cfg->r_near > 0.0 ? cfg->r_near : 2.5 * a;
    if (!(r_near >= 2.2 * a) || !std::isfinite(r_near)) return set_error(SD_ERR_ARG, "r_near must be >= 2.2 a");
    const double rep_rc = cfg->rep_rc > 0.0 ? cfg->rep_rc : 2.5 * a;
    if (!std::isfinite(cfg->rep_eps) || !std::isfinite(rep_rc)) return set_error(SD_ERR_ARG, "repulsion parameters");
    // cell side: every FP64 neighbour pass (near pairs, repulsion, lubrication) within one cell
    const double cutoff = std::max(r_near, std::max(cfg->rep_eps != 0.0 ? rep_rc : 0.0,
                                                    cfg->lubrication != 0 ? 3.0 * a : 0.0));
    for (int d = 0; d < 3; ++d)
        if (cfg->box[d] > 0.0 && cfg->box[d] < 3.0 * cutoff)
            return set_error(SD_ERR_ARG, "a periodic box side must be at least 3 max(r_near, rep_rc, 3a if "
                                         "lubrication)");
    if (!std::isfinite(cfg->verlet_skin)) return set_error(SD_ERR_ARG, "verlet_skin must be finite");
    // Verlet lists for the steps, when the box allows cells of side cutoff + skin: the
    // list holds every pair within the largest cutoff, so the repulsive and lubricated
    // pairs come from it too
    double skin = cfg->verlet_skin == 0.0 ? 0.5 * a : cfg->verlet_skin;
    bool verlet = skin > 0.0;
    for (int d = 0; d < 3 && verlet; ++d)
        if (cfg->box[d] > 0.0 && cfg->box[d] < 3.0 * (cutoff + skin)) verlet = false;
    if (!verlet) skin = 0.0;
    const double cell_h = cutoff + skin;

    sd_handle *h = new (std::nothrow) sd_handle();
    if (!h) return set_error(SD_ERR_OOM, "host allocation");
    h->cfg = *cfg;
    h->n = cfg->n;
    h->npad = ((cfg->n + kPadTo - 1) / kPadTo) * kPadTo;
    h->mode = cfg->prec == SD_PREC_FP64 ? MODE_FP64 : (cfg->prec == SD_PREC_FP32 ? MODE_FP32 : MODE_FP32C);
    h->tensor = cfg->tensor;
    h->device = cfg->device;
    h->stream = static_cast<cudaStream_t>(cfg->stream);
    h->al.alloc = cfg->alloc;
    h->al.free = cfg->free;
    h->al.ctx = cfg->alloc_ctx;
    h->r_near = r_near;
    h->rep_rc = rep_rc;
    h->lub = cfg->lubrication != 0;
    h->forces_const = (cfg->rep_eps == 0.0) && !h->lub;
    h->verlet = verlet;
    h->skin = skin;
    h->list_cut = cutoff;

    PairConst &pc = h->pc;
    pc.a = a;
    pc.two_a = 2.0 * a;
    pc.mu0 = 1.0 / (6.0 * 3.14159265358979323846 * cfg->eta * a);
    pc.r2min_d = 4.0 * a * a;
    pc.c1_d = 0.75 * a;
    pc.c3_d = 0.5 * a * a * a;
    pc.m3c3_d = -1.5 * a * a * a;
    pc.r2min_f = static_cast<float>(pc.r2min_d);
    pc.c1_f = static_cast<float>(pc.c1_d);
    pc.c3_f = static_cast<float>(pc.c3_d);
    pc.m3c3_f = static_cast<float>(pc.m3c3_d);
    // periodic box, nearest image only (Sec. 3.1 footnote)
    pc.periodic = 0;
    for (int d = 0; d < 3; ++d) {
        const double L = cfg->box[d];
        pc.Ld[d] = L;
        pc.invLd[d] = L > 0.0 ? 1.0 / L : 0.0;
        pc.Lf[d] = static_cast<float>(pc.Ld[d]);
        pc.invLf[d] = static_cast<float>(pc.invLd[d]);
        if (L > 0.0) pc.periodic = 1;
    }

    auto fail = [&](sd_status st, const std::string &m) {
        sd_destroy(h);
        return set_error(st, m);
    };
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail(SD_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    int major = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->device);
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return fail(SD_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(SD_ERR_CUDA, "stream creation");
    if (h->verlet) {   // the side branch of a Verlet step
        e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(SD_ERR_CUDA, "stream creation");
    }

    const size_t n3 = 3 * static_cast<size_t>(std::max(h->n, 1));
    const size_t np = static_cast<size_t>(std::max(h->npad, kPadTo));
    const size_t vb = v4size(h);
    h->near_cap = static_cast<int>(std::min<long long>(static_cast<long long>(kNearPerParticle) * h->n + 1024,
                                                        1LL << 30));
    bool ok = dalloc_t(h, h->d_err, 1) && dalloc_t(h, h->d_flag, 1) && dalloc_t(h, h->d_vl, 3) &&
              dalloc_t(h, h->near64, 2 * n3) &&
              dalloc_t(h, h->near_ent, h->near_cap) && dalloc_t(h, h->near_out, 6 * static_cast<size_t>(h->near_cap)) &&
              dalloc_t(h, h->near_n, 1) && dalloc_t(h, h->near_off, n3 / 3 + 1) && dalloc_t(h, h->near_cnt, n3 / 3 + 1);
    for (int b = 0; b < 2 && ok; ++b) ok = dalloc_t(h, h->x64[b], n3);
    if (ok && h->lub) ok = dalloc_t(h, h->vlag, n3);
    if (ok && h->verlet)
        ok = dalloc_t(h, h->xref, n3) && dalloc_t(h, h->vent, h->near_cap) && dalloc_t(h, h->voff, n3 / 3 + 1) &&
             dalloc_t(h, h->vcnt, n3 / 3 + 1) && dalloc_t(h, h->vn, 1);
    ok = ok && dalloc_t(h, h->fext64, n3) && dalloc_t(h, h->F64, n3) && dalloc_t(h, h->Fa64, n3) &&
         dalloc_t(h, h->Wa64, n3);
    const bool soa = h->mode != MODE_FP64;
    for (Mirror *m : {&h->posm, &h->frcm, &h->frcam, &h->wam}) {
        if (!ok) break;
        m->aos = dalloc(h, np * vb);
        ok = m->aos != nullptr;
        if (ok && soa) {   // (the cotangents' too: the packed FP32C VJP kernel stages SoA tiles)
            m->soa = static_cast<float *>(dalloc(h, 3 * np * sizeof(float)));
            ok = m->soa != nullptr;
        }
    }
    if (!ok) return fail(SD_ERR_OOM, "device allocation of particle buffers");

    // cell list
    CellList &c = h->cl;
    c.h = cell_h;
    c.inv_h = 1.0 / c.h;
    for (int d = 0; d < 3; ++d) {
        c.box.L[d] = pc.Ld[d];
        c.box.invL[d] = pc.invLd[d];
        c.nc[d] = pc.Ld[d] > 0.0 ? static_cast<int>(std::floor(pc.Ld[d] / c.h)) : 0;   // >= 3, checked above
    }
    c.box.periodic = pc.periodic;
    c.n = h->n;
    c.err = h->d_err;
    int H = 1024;
    while (H < 2 * h->n) H <<= 1;
    c.H = H;
    c.nblk = (H + 16383) / 16384;   // scan blocks of 16,384 buckets (cells.cu)
    ok = dalloc_t(h, c.cell, n3 / 3) && dalloc_t(h, c.key, n3 / 3) && dalloc_t(h, c.cnt, H) &&
         dalloc_t(h, c.start, H + 1) && dalloc_t(h, c.bsum, c.nblk) &&
         dalloc_t(h, c.sorted, n3 / 3);
    if (!ok) return fail(SD_ERR_OOM, "device allocation of the cell list");

    if (h->n > 0) {
        e = dense_setup(h);
        if (e == cudaSuccess) e = vjp_setup(h);
        if (e != cudaSuccess) return fail(SD_ERR_CUDA, std::string("kernel set-up: ") + cudaGetErrorString(e));
        const int slots = std::max(h->geom.maxSlots, h->geomv.maxSlots);
        h->part_bytes = static_cast<size_t>(slots) * 3 * h->npad * sizeof(double);
        h->part2_bytes = static_cast<size_t>(h->geomv.maxSlots) * 3 * h->npad * sizeof(double);
        h->part = static_cast<double *>(dalloc(h, h->part_bytes));
        h->part2 = static_cast<double *>(dalloc(h, h->part2_bytes));
        if (!h->part || !h->part2) return fail(SD_ERR_OOM, "device allocation of partial sums");
        if (h->geom.sym) {
            const size_t es = h->mode == MODE_FP64 ? sizeof(double) : sizeof(float);
            h->jpart_bytes = static_cast<size_t>(h->geom.nT) * 3 * h->geom.I * es;
            h->jpart = dalloc(h, h->jpart_bytes);
            if (!h->jpart) return fail(SD_ERR_OOM, "device allocation of source-side partial sums");
        }
    }

    // zero everything that padding or defaults rely on
    cudaStream_t st = h->stream;
    e = cudaMemsetAsync(h->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_vl, 0, 3 * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_vl, 0xff, sizeof(int), st);   // no list until positions are set
    if (e == cudaSuccess && h->vn) e = cudaMemsetAsync(h->vn, 0, sizeof(*h->vn), st);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMemsetAsync(h->x64[b], 0, n3 * sizeof(double), st);
    for (Mirror *m : {&h->posm, &h->frcm, &h->frcam, &h->wam}) {
        if (e == cudaSuccess) e = cudaMemsetAsync(m->aos, 0, np * vb, st);
        if (e == cudaSuccess && m->soa) e = cudaMemsetAsync(m->soa, 0, 3 * np * sizeof(float), st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->fext64, 0, n3 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->cl.cnt, 0, sizeof(int) * static_cast<size_t>(h->cl.H), st);
    if (e == cudaSuccess && h->vlag) e = cudaMemsetAsync(h->vlag, 0, n3 * sizeof(double), st);
    if (e == cudaSuccess) e = launch_pad_mirror(h, st, h->posm);
    if (e == cudaSuccess) e = launch_stage_forces(h, st, nullptr, SD_DTYPE_F64, 1, h->F64, h->frcm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SD_ERR_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
    *out = h;
    return SD_OK;
}

void sd_destroy(sd_handle *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->side) cudaStreamSynchronize(h->side);   // (a step that failed before its join)
    drop_graphs(h);
    prof_destroy(h->prof);
    for (int b = 0; b < 2; ++b) dfree(h, h->x64[b]);
    for (Mirror *m : {&h->posm, &h->frcm, &h->frcam, &h->wam}) {
        dfree(h, m->aos);
        dfree(h, m->soa);
    }
    void *bufs[] = {h->fext64, h->F64, h->Fa64, h->Wa64, h->part, h->part2, h->jpart,
                    h->cl.cell, h->cl.key, h->cl.cnt, h->cl.start, h->cl.bsum, h->cl.sorted,
                    h->ckpt, h->seg, h->lam, h->gFacc, h->near64, h->d_flag, h->d_err,
                    h->near_ent, h->near_out, h->near_n, h->near_off, h->near_cnt, h->vlag, h->xref, h->d_vl,
                    h->vent, h->voff, h->vcnt, h->vn};
    for (void *p : bufs) dfree(h, p);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    delete h;
}

// Memory kind of a caller pointer (the on_device argument): 0 host (the call
// synchronises), 1 device, 2 host memory the caller keeps alive and unchanged until
// the stream reaches the copy (asynchronous; pinned memory makes it a DMA).
static bool valid_kind(int on_device) { return on_device >= 0 && on_device <= 2; }
static cudaMemcpyKind to_device_kind(int on_device) {
    return on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
static cudaMemcpyKind from_device_kind(int on_device) {
    return on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

// True when any of the k doubles is NaN or infinite (exponent bits all set); a
// branch-free OR over the array, so the check costs a pass over memory.
static bool any_nonfinite(const double *v, size_t k) {
    uint64_t bad = 0;
    for (size_t i = 0; i < k; ++i) {
        uint64_t b;
        std::memcpy(&b, v + i, sizeof(b));
        bad |= static_cast<uint64_t>((b & 0x7ff0000000000000ull) == 0x7ff0000000000000ull);
    }
    return bad != 0;
}

sd_status sd_set_positions(sd_handle *h, const double *xyz, int on_device) {
    NvtxRange nvtx_range("sd_set_positions");
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (!xyz && h->n > 0) return set_error(SD_ERR_ARG, "positions pointer is NULL");
    if (!valid_kind(on_device)) return set_error(SD_ERR_ARG, "on_device must be 0, 1 or 2");
    cudaSetDevice(h->device);
    if (on_device == 0 && any_nonfinite(xyz, 3 * static_cast<size_t>(h->n)))
        return set_error(SD_ERR_NONFINITE, "non-finite position");
    if (h->n > 0) {
        SD_CUDA(cudaMemcpyAsync(h->x64[h->cur], xyz, 3 * sizeof(double) * h->n, to_device_kind(on_device),
                                h->stream));
        sd_status s = launch_check(launch_stage_pos(h, h->stream, h->x64[h->cur], h->posm), "stage positions");
        if (s != SD_OK) return s;
        // new positions: the previous step's velocities no longer apply (lubrication),
        // and the steps' neighbour list is built afresh around them, so that a
        // trajectory resumed from positions read back continues bit for bit
        if (h->vlag) SD_CUDA(cudaMemsetAsync(h->vlag, 0, 3 * sizeof(double) * h->n, h->stream));
        if (h->verlet) {
            SD_CUDA(cudaMemsetAsync(h->d_vl, 0, sizeof(int), h->stream));
            SD_CUDA(cudaMemsetAsync(h->d_vl, 1, 1, h->stream));   // a rebuild request (bit 2 clear)
            s = launch_check(launch_build_cells(h, h->stream, h->x64[h->cur], h->posm, h->xref), "neighbour list");
            if (s == SD_OK)
                s = launch_check(launch_near_collect(h, h->stream, h->x64[h->cur], h->posm.aos, h->F64,
                                                     h->frcm.aos, true, true),
                                 "neighbour list");
            if (s != SD_OK) return s;
        }
    }
    h->pos_set = true;
    h->cells_valid = false;
    return on_device ? SD_OK : sync_check(h);
}

sd_status sd_get_positions(sd_handle *h, double *xyz, int on_device) {
    NvtxRange nvtx_range("sd_get_positions");
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (!xyz && h->n > 0) return set_error(SD_ERR_ARG, "positions pointer is NULL");
    if (!valid_kind(on_device)) return set_error(SD_ERR_ARG, "on_device must be 0, 1 or 2");
    if (!h->pos_set) return set_error(SD_ERR_STATE, "positions were never set");
    cudaSetDevice(h->device);
    if (h->n > 0)
        SD_CUDA(cudaMemcpyAsync(xyz, h->x64[h->cur], 3 * sizeof(double) * h->n, from_device_kind(on_device),
                                h->stream));
    return on_device ? SD_OK : sync_check(h);
}

sd_status sd_set_forces(sd_handle *h, const double *f, int on_device) {
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (!f && h->n > 0) return set_error(SD_ERR_ARG, "forces pointer is NULL");
    if (!valid_kind(on_device)) return set_error(SD_ERR_ARG, "on_device must be 0, 1 or 2");
    cudaSetDevice(h->device);
    if (on_device == 0 && any_nonfinite(f, 3 * static_cast<size_t>(h->n)))
        return set_error(SD_ERR_NONFINITE, "non-finite force");
    if (h->n > 0) {
        SD_CUDA(cudaMemcpyAsync(h->fext64, f, 3 * sizeof(double) * h->n, to_device_kind(on_device), h->stream));
        sd_status s =
            launch_check(launch_stage_forces(h, h->stream, nullptr, SD_DTYPE_F64, 1, h->F64, h->frcm), "stage forces");
        if (s != SD_OK) return s;
    }
    return on_device ? SD_OK : sync_check(h);
}

sd_status sd_synchronize(sd_handle *h) {
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    cudaSetDevice(h->device);
    return sync_check(h);
}

// Device staging buffers for host-pointer calls.
static sd_status host_io(sd_handle *h, void *&in, void *&out) {
    const size_t bytes = 3 * sizeof(double) * static_cast<size_t>(std::max(h->n, 1));
    sd_status s = ensure_seg(h, 2 * bytes, "device allocation of staging buffers");
    if (s != SD_OK) return s;
    in = h->seg;
    out = reinterpret_cast<char *>(h->seg) + bytes;
    return SD_OK;
}

static sd_status ensure_cells(sd_handle *h) {
    if (h->cells_valid) return SD_OK;
    sd_status s = launch_check(launch_build_cells(h, h->stream, h->x64[h->cur], h->posm), "cell list");
    if (s == SD_OK) h->cells_valid = true;
    return s;
}

// The tile window of the rows [row0, row1): whole i-blocks of the directed kernel.
static TileWin row_window(const sd_handle *h, int row0, int row1) {
    const DenseGeom &g = h->geom;
    TileWin w;
    w.lo = static_cast<long long>(row0 / g.I) * g.nJT;
    w.hi = static_cast<long long>((row1 + g.I - 1) / g.I) * g.nJT;
    return w;
}

// v for rows [row0, row1) (all rows: the whole product, either all-pairs kernel).
static sd_status apply_rows(sd_handle *h, const void *F, void *V, int dtype, int on_device, int row0, int row1) {
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (dtype != SD_DTYPE_F32 && dtype != SD_DTYPE_F64) return set_error(SD_ERR_ARG, "dtype must be F32 or F64");
    if (row0 < 0 || row1 < row0 || row1 > h->n) return set_error(SD_ERR_ARG, "rows must satisfy 0 <= row0 <= row1 <= n");
    if (on_device != 0 && on_device != 1) return set_error(SD_ERR_ARG, "on_device must be 0 or 1");
    const bool all = row0 == 0 && row1 == h->n;
    if (!all && h->geom.sym)
        return set_error(SD_ERR_UNSUPPORTED, "row shards need the directed all-pairs kernel (SD_DENSE_DIRECTED)");
    if (h->n > 0 && (!F || (!V && row1 > row0))) return set_error(SD_ERR_ARG, "F or V is NULL");
    if (!h->pos_set) return set_error(SD_ERR_STATE, "positions were never set");
    if (h->n == 0 || row0 == row1) return SD_OK;
    cudaSetDevice(h->device);
    const size_t es = dtype == SD_DTYPE_F32 ? sizeof(float) : sizeof(double);
    const size_t bytes_in = 3 * es * h->n, bytes_out = 3 * es * static_cast<size_t>(row1 - row0);
    const void *Fd = F;
    void *Vd = V;
    if (!on_device) {
        void *in = nullptr, *out = nullptr;
        sd_status s = host_io(h, in, out);
        if (s != SD_OK) return s;
        SD_CUDA(cudaMemcpyAsync(in, F, bytes_in, cudaMemcpyHostToDevice, h->stream));
        Fd = in;
        Vd = out;
    }
    const TileWin w = row_window(h, row0, row1);
    sd_status s = launch_check(launch_stage_forces(h, h->stream, Fd, dtype, 0, h->Fa64, h->frcam), "stage F");
    if (s == SD_OK) s = ensure_cells(h);
    if (s == SD_OK)
        s = launch_check(launch_near(h, h->stream, h->x64[h->cur], h->posm.aos, h->Fa64, h->frcam.aos), "near pass");
    if (s == SD_OK)
        s = launch_check(launch_dense(h, h->stream, h->posm, h->frcam, h->part, all ? nullptr : &w), "dense kernel");
    if (s == SD_OK)
        s = launch_check(launch_epilogue(h, h->stream, dtype == SD_DTYPE_F32 ? OUT_F32 : OUT_F64, h->x64[h->cur],
                                         h->posm.aos, h->Fa64, h->frcam.aos, Vd, 0.0, nullptr, row0, row1),
                         "epilogue");
    if (s != SD_OK) return s;
    if (!on_device) {
        SD_CUDA(cudaMemcpyAsync(V, Vd, bytes_out, cudaMemcpyDeviceToHost, h->stream));
        return sync_check(h);
    }
    return SD_OK;
}

sd_status sd_mobility_apply(sd_handle *h, const void *F, void *V, int dtype, int on_device) {
    NvtxRange nvtx_range("sd_mobility_apply");
    return apply_rows(h, F, V, dtype, on_device, 0, h ? h->n : 0);
}

sd_status sd_mobility_apply_rows(sd_handle *h, const void *F, void *V, int dtype, int on_device, int32_t row0,
                                 int32_t row1) {
    NvtxRange nvtx_range("sd_mobility_apply_rows");
    return apply_rows(h, F, V, dtype, on_device, row0, row1);
}

sd_status sd_step_rows(sd_handle *h, double dt, int32_t row0, int32_t row1) {
    NvtxRange nvtx_range("sd_step_rows");
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (!std::isfinite(dt)) return set_error(SD_ERR_ARG, "dt must be finite");
    if (row0 < 0 || row1 < row0 || row1 > h->n) return set_error(SD_ERR_ARG, "rows must satisfy 0 <= row0 <= row1 <= n");
    if (h->geom.sym && !(row0 == 0 && row1 == h->n))
        return set_error(SD_ERR_UNSUPPORTED, "row shards need the directed all-pairs kernel (SD_DENSE_DIRECTED)");
    if (h->lub) return set_error(SD_ERR_UNSUPPORTED, "sharded steps with lubrication are not implemented");
    if (!h->pos_set) return set_error(SD_ERR_STATE, "positions were never set");
    if (h->n == 0) return SD_OK;
    cudaSetDevice(h->device);
    cudaStream_t st = h->stream;
    const double *x_in = h->x64[h->cur];
    double *x_out = h->x64[1 - h->cur];
    const TileWin w = row_window(h, row0, row1);
    cudaError_t e = launch_build_cells(h, st, x_in, h->posm);
    if (e == cudaSuccess && !h->forces_const) e = launch_forces_rep(h, st, x_in);
    if (e == cudaSuccess) e = launch_near(h, st, x_in, h->posm.aos, h->F64, h->frcm.aos);
    if (e == cudaSuccess) e = launch_dense(h, st, h->posm, h->frcm, h->part, &w);
    if (e == cudaSuccess)
        e = launch_epilogue(h, st, OUT_EULER, x_in, h->posm.aos, h->F64, h->frcm.aos, nullptr, dt, x_out, row0, row1);
    // the rows of other shards keep their positions
    const size_t rb = 3 * sizeof(double);
    if (e == cudaSuccess && row0 > 0) e = cudaMemcpyAsync(x_out, x_in, rb * row0, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && row1 < h->n)
        e = cudaMemcpyAsync(x_out + 3 * static_cast<size_t>(row1), x_in + 3 * static_cast<size_t>(row1),
                            rb * (h->n - row1), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_status(e, "sharded step");
    h->cur = 1 - h->cur;
    h->cells_valid = false;
    return SD_OK;
}

// ---------------------------------------------------------------- tile shards

enum { PART_NONE = 0, PART_APPLY = 1, PART_STEP = 2 };

// Shard `shard` of `nshards`: CTAs [b0, b1) of the all-pairs kernel's persistent grid
// (either kernel), i.e. the tiles [b0 chunk, min(b1 chunk, nT)).  The CTAs hold equal
// runs of tiles, so the shards get equal pair work.
static void shard_window(const sd_handle *h, int shard, int nshards, TileWin &w, EpiShard &es) {
    const DenseGeom &g = h->geom;
    const int b0 = static_cast<int>(static_cast<long long>(shard) * g.grid / nshards);
    const int b1 = static_cast<int>(static_cast<long long>(shard + 1) * g.grid / nshards);
    w.b0 = b0;
    w.lo = static_cast<long long>(b0) * g.chunk;
    w.hi = std::min(static_cast<long long>(b1) * g.chunk, g.nT);
    es.b0 = b0;
    es.b1 = b1;
    es.tlo = w.lo;
    es.thi = w.hi;
}

static sd_status check_shard(const sd_handle *h, int shard, int nshards, const double *P) {
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (nshards < 1 || shard < 0 || shard >= nshards) return set_error(SD_ERR_ARG, "need 0 <= shard < nshards");
    if (!P && h->n > 0) return set_error(SD_ERR_ARG, "P is NULL");
    if (!h->pos_set) return set_error(SD_ERR_STATE, "positions were never set");
    return SD_OK;
}

}  // extern "C"

// This shard's raw share of the all-pairs sum for the staged positions and forces:
// near pass (every shard: the all-pairs kernel's clamping follows its flag), the
// shard's CTAs of the all-pairs kernel, and the epilogue's sum over their slots.
static sd_status run_part(sd_handle *h, int shard, int nshards, const double *F64, Mirror frcm, double *P) {
    TileWin w;
    EpiShard es;
    shard_window(h, shard, nshards, w, es);
    cudaStream_t st = h->stream;
    sd_status s = launch_check(launch_near(h, st, h->x64[h->cur], h->posm.aos, F64, frcm.aos), "near pass");
    if (s == SD_OK) s = launch_check(launch_dense(h, st, h->posm, frcm, h->part, &w), "dense kernel (shard)");
    if (s == SD_OK)
        s = launch_check(launch_epilogue(h, st, OUT_PART, h->x64[h->cur], h->posm.aos, F64, frcm.aos, P, 0.0, nullptr,
                                         0, h->n, &es),
                         "epilogue (shard)");
    return s;
}

extern "C" {

sd_status sd_mobility_apply_part(sd_handle *h, const void *F, int dtype, int on_device, int32_t shard,
                                 int32_t nshards, double *P) {
    NvtxRange nvtx_range("sd_mobility_apply_part");
    sd_status s = check_shard(h, shard, nshards, P);
    if (s != SD_OK) return s;
    if (dtype != SD_DTYPE_F32 && dtype != SD_DTYPE_F64) return set_error(SD_ERR_ARG, "dtype must be F32 or F64");
    if (on_device != 0 && on_device != 1) return set_error(SD_ERR_ARG, "on_device must be 0 or 1");
    if (h->n > 0 && !F) return set_error(SD_ERR_ARG, "F is NULL");
    h->part_kind = PART_NONE;
    if (h->n == 0) {
        h->part_kind = PART_APPLY;
        return SD_OK;
    }
    cudaSetDevice(h->device);
    const void *Fd = F;
    if (!on_device) {
        void *in = nullptr, *out = nullptr;
        s = host_io(h, in, out);
        if (s != SD_OK) return s;
        const size_t es = dtype == SD_DTYPE_F32 ? sizeof(float) : sizeof(double);
        SD_CUDA(cudaMemcpyAsync(in, F, 3 * es * h->n, cudaMemcpyHostToDevice, h->stream));
        Fd = in;
    }
    s = launch_check(launch_stage_forces(h, h->stream, Fd, dtype, 0, h->Fa64, h->frcam), "stage F");
    if (s == SD_OK) s = ensure_cells(h);
    if (s == SD_OK) s = run_part(h, shard, nshards, h->Fa64, h->frcam, P);
    if (s != SD_OK) return s;
    h->part_kind = PART_APPLY;
    return on_device ? SD_OK : sync_check(h);
}

sd_status sd_mobility_apply_combine(sd_handle *h, const double *Pall, int32_t nparts, void *V, int dtype,
                                    int on_device) {
    NvtxRange nvtx_range("sd_mobility_apply_combine");
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (dtype != SD_DTYPE_F32 && dtype != SD_DTYPE_F64) return set_error(SD_ERR_ARG, "dtype must be F32 or F64");
    if (on_device != 0 && on_device != 1) return set_error(SD_ERR_ARG, "on_device must be 0 or 1");
    if (nparts < 1 || (h->n > 0 && (!Pall || !V))) return set_error(SD_ERR_ARG, "Pall, nparts or V");
    if (h->part_kind != PART_APPLY) return set_error(SD_ERR_STATE, "sd_mobility_apply_part must come first");
    h->part_kind = PART_NONE;
    if (h->n == 0) return SD_OK;
    cudaSetDevice(h->device);
    EpiShard es;
    es.pall = Pall;
    es.nparts = nparts;
    void *Vd = V;
    if (!on_device) {
        void *in = nullptr, *out = nullptr;
        sd_status s = host_io(h, in, out);
        if (s != SD_OK) return s;
        Vd = out;
    }
    sd_status s = launch_check(launch_epilogue(h, h->stream, dtype == SD_DTYPE_F32 ? OUT_F32 : OUT_F64, h->x64[h->cur],
                                               h->posm.aos, h->Fa64, h->frcam.aos, Vd, 0.0, nullptr, 0, h->n, &es),
                               "epilogue (combine)");
    if (s != SD_OK) return s;
    if (!on_device) {
        const size_t es2 = dtype == SD_DTYPE_F32 ? sizeof(float) : sizeof(double);
        SD_CUDA(cudaMemcpyAsync(V, Vd, 3 * es2 * h->n, cudaMemcpyDeviceToHost, h->stream));
        return sync_check(h);
    }
    return SD_OK;
}

sd_status sd_step_part(sd_handle *h, int32_t shard, int32_t nshards, double *P) {
    NvtxRange nvtx_range("sd_step_part");
    sd_status s = check_shard(h, shard, nshards, P);
    if (s != SD_OK) return s;
    h->part_kind = PART_NONE;
    if (h->n == 0) {
        h->part_kind = PART_STEP;
        return SD_OK;
    }
    cudaSetDevice(h->device);
    cudaStream_t st = h->stream;
    const double *x_in = h->x64[h->cur];
    cudaError_t e = launch_build_cells(h, st, x_in, h->posm);
    if (e == cudaSuccess && !h->forces_const) e = launch_forces_rep(h, st, x_in);
    if (e != cudaSuccess) return cuda_status(e, "cells / forces (shard)");
    h->cells_valid = true;
    s = run_part(h, shard, nshards, h->F64, h->frcm, P);
    if (s != SD_OK) return s;
    h->part_kind = PART_STEP;
    return SD_OK;
}

sd_status sd_step_combine(sd_handle *h, double dt, const double *Pall, int32_t nparts) {
    NvtxRange nvtx_range("sd_step_combine");
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (!std::isfinite(dt)) return set_error(SD_ERR_ARG, "dt must be finite");
    if (nparts < 1 || (h->n > 0 && !Pall)) return set_error(SD_ERR_ARG, "Pall or nparts");
    if (h->part_kind != PART_STEP) return set_error(SD_ERR_STATE, "sd_step_part must come first");
    h->part_kind = PART_NONE;
    if (h->n == 0) return SD_OK;
    cudaSetDevice(h->device);
    EpiShard es;
    es.pall = Pall;
    es.nparts = nparts;
    const double *x_in = h->x64[h->cur];
    sd_status s = launch_check(launch_epilogue(h, h->stream, OUT_EULER, x_in, h->posm.aos, h->F64, h->frcm.aos, nullptr,
                                               dt, h->x64[1 - h->cur], 0, h->n, &es),
                               "epilogue (combine)");
    if (s != SD_OK) return s;
    h->cur = 1 - h->cur;
    h->cells_valid = false;
    return SD_OK;
}

sd_status sd_step(sd_handle *h, double dt, int64_t nsteps) {
    NvtxRange nvtx_range("sd_step");
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (nsteps < 0 || !std::isfinite(dt)) return set_error(SD_ERR_ARG, "nsteps must be >= 0 and dt finite");
    if (!h->pos_set) return set_error(SD_ERR_STATE, "positions were never set");
    if (h->n == 0 || nsteps == 0) return SD_OK;
    cudaSetDevice(h->device);
    return run_steps(h, dt, nsteps);
}

sd_status sd_mobility_vjp(sd_handle *h, const void *F, const void *W, void *gX, void *gF, int dtype, int on_device) {
    NvtxRange nvtx_range("sd_mobility_vjp");
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (dtype != SD_DTYPE_F32 && dtype != SD_DTYPE_F64) return set_error(SD_ERR_ARG, "dtype must be F32 or F64");
    if (h->n > 0 && (!F || !W || (!gX && !gF))) return set_error(SD_ERR_ARG, "null argument");
    if (on_device != 0 && on_device != 1) return set_error(SD_ERR_ARG, "on_device must be 0 or 1");
    if (!h->pos_set) return set_error(SD_ERR_STATE, "positions were never set");
    if (h->n == 0) return SD_OK;
    cudaSetDevice(h->device);
    const size_t es = dtype == SD_DTYPE_F32 ? sizeof(float) : sizeof(double);
    const size_t bytes = 3 * es * h->n;
    const void *Fd = F, *Wd = W;
    void *gXd = gX, *gFd = gF;
    if (!on_device) {
        // four n x 3 arrays: F, W in; gX, gF out
        const size_t need = 4 * 3 * sizeof(double) * static_cast<size_t>(h->n);
        sd_status s0 = ensure_seg(h, need, "device allocation of staging buffers");
        if (s0 != SD_OK) return s0;
        char *b = reinterpret_cast<char *>(h->seg);
        SD_CUDA(cudaMemcpyAsync(b, F, bytes, cudaMemcpyHostToDevice, h->stream));
        SD_CUDA(cudaMemcpyAsync(b + bytes, W, bytes, cudaMemcpyHostToDevice, h->stream));
        Fd = b;
        Wd = b + bytes;
        gXd = gX ? b + 2 * bytes : nullptr;
        gFd = gF ? b + 3 * bytes : nullptr;
    }
    sd_status s = launch_check(launch_stage_forces(h, h->stream, Fd, dtype, 0, h->Fa64, h->frcam), "stage F");
    if (s == SD_OK) s = launch_check(launch_stage_forces(h, h->stream, Wd, dtype, 0, h->Wa64, h->wam), "stage W");
    if (s == SD_OK) s = ensure_cells(h);
    if (s == SD_OK)
        s = launch_check(launch_vjp_dense(h, h->stream, h->posm, h->frcam, h->wam, h->part, h->part2),
                         "vjp kernel");
    if (s == SD_OK)
        s = launch_check(launch_vjp_epilogue(h, h->stream, h->x64[h->cur], h->posm.aos, h->Fa64, h->frcam.aos,
                                             h->Wa64, h->wam.aos, dtype, gXd, gFd, 0.0, nullptr, nullptr),
                         "vjp epilogue");
    if (s != SD_OK) return s;
    if (!on_device) {
        if (gX) SD_CUDA(cudaMemcpyAsync(gX, gXd, bytes, cudaMemcpyDeviceToHost, h->stream));
        if (gF) SD_CUDA(cudaMemcpyAsync(gF, gFd, bytes, cudaMemcpyDeviceToHost, h->stream));
        return sync_check(h);
    }
    return SD_OK;
}

sd_status sd_adjoint(sd_handle *h, double dt, int64_t nsteps, int32_t ckpt_every, const double *gxT, double *gx0,
                     double *gF, int on_device) {
    NvtxRange nvtx_range("sd_adjoint");
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    if (nsteps < 0 || ckpt_every < 1 || !std::isfinite(dt)) return set_error(SD_ERR_ARG, "nsteps, ckpt_every or dt");
    if (h->n > 0 && (!gxT || !gx0 || !gF)) return set_error(SD_ERR_ARG, "null argument");
    if (on_device != 0 && on_device != 1) return set_error(SD_ERR_ARG, "on_device must be 0 or 1");
    if (!h->forces_const)
        return set_error(SD_ERR_UNSUPPORTED, "adjoint with soft repulsion or lubrication is not implemented");
    if (!h->pos_set) return set_error(SD_ERR_STATE, "positions were never set");
    if (h->n == 0) return SD_OK;
    cudaSetDevice(h->device);
    cudaStream_t st = h->stream;
    const size_t n3 = 3 * static_cast<size_t>(h->n);
    const size_t xb = n3 * sizeof(double);
    const size_t mb = static_cast<size_t>(h->npad) * v4size(h);
    const int64_t K = ckpt_every;
    const int64_t nck = nsteps / K + 1;
    // storage: checkpoints, one segment of positions + mirrors, lambda, gF accumulator
    const size_t ck_need = static_cast<size_t>(nck) * xb;
    if (!h->ckpt || h->ckpt_bytes < ck_need) {
        dfree(h, h->ckpt);
        h->ckpt = static_cast<double *>(dalloc(h, ck_need));
        h->ckpt_bytes = h->ckpt ? ck_need : 0;
        if (!h->ckpt) return set_error(SD_ERR_OOM, "device allocation of checkpoints");
    }
    const size_t seg_need = static_cast<size_t>(K) * xb;
    {
        sd_status s0 = ensure_seg(h, seg_need, "device allocation of the recompute segment");
        if (s0 != SD_OK) return s0;
    }
    if (!h->lam) {
        if (!dalloc_t(h, h->lam, n3) || !dalloc_t(h, h->gFacc, n3))
            return set_error(SD_ERR_OOM, "device allocation of adjoint vectors");
    }
    auto segx = [&](int64_t k) { return h->seg + static_cast<size_t>(k) * n3; };

    const int c0 = h->cur;
    const int64_t nseg = (nsteps + K - 1) / K;
    // forward with checkpoints, segment by segment through the step graphs (the state
    // ping-pongs through x64[0], x64[1])
    SD_CUDA(cudaMemcpyAsync(h->ckpt, h->x64[c0], xb, cudaMemcpyDeviceToDevice, st));
    for (int64_t sg = 0; sg < nseg; ++sg) {
        const int64_t len = std::min(K, nsteps - sg * K);
        sd_status ss = run_steps(h, dt, len);
        if (ss != SD_OK) return ss;
        const int64_t s1 = sg * K + len;
        if (s1 % K == 0 && s1 / K < nck)
            SD_CUDA(cudaMemcpyAsync(h->ckpt + static_cast<size_t>(s1 / K) * n3, h->x64[h->cur], xb,
                                    cudaMemcpyDeviceToDevice, st));
    }
    // lambda_T
    if (on_device)
        SD_CUDA(cudaMemcpyAsync(h->lam, gxT, xb, cudaMemcpyDeviceToDevice, st));
    else
        SD_CUDA(cudaMemcpyAsync(h->lam, gxT, xb, cudaMemcpyHostToDevice, st));
    SD_CUDA(cudaMemsetAsync(h->gFacc, 0, xb, st));
    // reverse sweep, last segment first: recompute the segment's positions from its
    // checkpoint, then walk it backwards.  Full segments replay cached graphs (eager
    // with the profiler on, and for a shorter last segment).
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
        const int64_t len = std::min(K, nsteps - sg * K);
        SD_CUDA(cudaMemcpyAsync(segx(0), h->ckpt + static_cast<size_t>(sg) * n3, xb, cudaMemcpyDeviceToDevice, st));
        if (len == K && !h->prof.on) {
            if (!h->adj_rev || h->adj_dt != dt || h->adj_K != K) {
                sd_status ss = capture_adjoint(h, dt, K);
                if (ss != SD_OK) return ss;
            }
            if (h->adj_rec) {
                SD_CUDA(cudaGraphLaunch(h->adj_rec, st));
                h->launches += h->adj_rec_kernels;
            }
            SD_CUDA(cudaGraphLaunch(h->adj_rev, st));
            h->launches += h->adj_rev_kernels;
        } else {
            sd_status ss = launch_check(adjoint_segment(h, st, dt, len, 0), "recompute");
            if (ss == SD_OK) ss = launch_check(adjoint_segment(h, st, dt, len, 1), "adjoint sweep");
            if (ss != SD_OK) return ss;
        }
    }
    // restore x0 into the current buffers
    SD_CUDA(cudaMemcpyAsync(h->x64[c0], h->ckpt, xb, cudaMemcpyDeviceToDevice, st));
    sd_status ss = launch_check(launch_stage_pos(h, st, h->x64[c0], h->posm), "restore positions");
    if (ss != SD_OK) return ss;
    h->cur = c0;
    h->cells_valid = false;
    if (on_device) {
        SD_CUDA(cudaMemcpyAsync(gx0, h->lam, xb, cudaMemcpyDeviceToDevice, st));
        SD_CUDA(cudaMemcpyAsync(gF, h->gFacc, xb, cudaMemcpyDeviceToDevice, st));
        return SD_OK;
    }
    SD_CUDA(cudaMemcpyAsync(gx0, h->lam, xb, cudaMemcpyDeviceToHost, st));
    SD_CUDA(cudaMemcpyAsync(gF, h->gFacc, xb, cudaMemcpyDeviceToHost, st));
    return sync_check(h);
}

sd_status sd_profile(sd_handle *h, int on) {
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    cudaSetDevice(h->device);
    SD_CUDA(cudaStreamSynchronize(h->stream));
    Profiler &p = h->prof;
    p.on = on != 0;
    p.npending = 0;
    p.open = false;
    for (int k = 0; k < SD_KERNEL_COUNT; ++k) {
        p.ms[k] = 0.0;
        p.launches[k] = 0;
    }
    return SD_OK;
}

sd_status sd_profile_read(sd_handle *h, int kernel, double *ms, int64_t *launches) {
    if (!h || kernel < 0 || kernel >= SD_KERNEL_COUNT) return set_error(SD_ERR_ARG, "bad handle or kernel id");
    cudaSetDevice(h->device);
    SD_CUDA(prof_collect(h->prof));
    if (ms) *ms = h->prof.ms[kernel];
    if (launches) *launches = h->prof.launches[kernel];
    return SD_OK;
}

int64_t sd_launch_count(const sd_handle *h) { return h ? h->launches : 0; }
int32_t sd_dense_kernel_used(const sd_handle *h) {
    if (!h || h->n == 0) return SD_DENSE_AUTO;
    return h->geom.sym ? SD_DENSE_SYMMETRIC : SD_DENSE_DIRECTED;
}

sd_status sd_set_watchdog(sd_handle *h, int64_t iterations) {
    if (!h || iterations < 1) return set_error(SD_ERR_ARG, "bad handle or iteration limit");
    h->watchdog = iterations;
    drop_graphs(h);   // graphs captured the old limit
    return SD_OK;
}

sd_status sd_inject_stall(sd_handle *h, int32_t on) {
    if (!h) return set_error(SD_ERR_ARG, "handle is NULL");
    h->inject_stall = on != 0;
    drop_graphs(h);   // graphs captured the launch arguments
    return SD_OK;
}

}  // extern "C"
