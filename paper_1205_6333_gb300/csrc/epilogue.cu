// epilogue.cu -- per-particle completion of the mobility product and the Euler
// update (Sec. 3.1, steps 1 and 3):
//
//   V_i = sum over the CTA slots of the dense partial sums (ascending slot order)
//       + F_i - Tdense(0) F_i                        self term mu_ii = mu0 I (Sec. 2.2)
//       + sum_{j: |r_ij| < r_near} [Texact(r_ij) F_j - Tdense(r_ij) F_j]
//   v_i = mu0 V_i
//
// Tdense is re-evaluated with the very same device function and inputs the dense
// kernel used; Texact is the FP64 tensor in use (Rotne-Prager, Oseen, or the RPY
// overlap form) at the FP64 separation.  The near-pair terms are the ones whose
// FP32 evaluation suffers from cancellation in r_i - r_j (large coordinates,
// small separations) or that the dense kernel clamped (r < 2a).  Output: the
// velocities (apply), or x_{n+1} = x_n + dt v_n in FP64 (step).
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

struct EpiArgs {
    const double *part;
    int npad;
    DenseGeom g;
    const double *x64;
    const void *posm;
    const double *F64;
    const void *frcm;
    CellList cl;
    double rnear2;
    PairConst pc;
    int n;
    void *vout;
    double dt;
    double *x64n;
    int *err;
};

template <int TDENSE, int MODE>
__device__ __forceinline__ void dense_term(const typename EpiT<MODE>::V4 &pi, const typename EpiT<MODE>::V4 &pj,
                                           const typename EpiT<MODE>::V4 &fj, const PairConst &c, double out[3]) {
    using S = typename EpiT<MODE>::S;
    S ax = S(0), ay = S(0), az = S(0);
    if constexpr (MODE == MODE_FP64)
        pair_f64<TDENSE>(pi.x, pi.y, pi.z, pj, fj, c, ax, ay, az);
    else
        pair_f32<TDENSE>(pi.x, pi.y, pi.z, pj, fj, c, ax, ay, az);
    out[0] = static_cast<double>(ax);
    out[1] = static_cast<double>(ay);
    out[2] = static_cast<double>(az);
}

template <int TENSOR, int MODE, int OUT>
__global__ void __launch_bounds__(128) epilogue_kernel(EpiArgs a) {
    using V4 = typename EpiT<MODE>::V4;
    constexpr int TDENSE = (TENSOR == T_OSEEN) ? T_OSEEN : T_RP;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const V4 *pm = static_cast<const V4 *>(a.posm);
    const V4 *fm = static_cast<const V4 *>(a.frcm);

    // dense sum over the CTA slots of this particle's i-block, in slot order
    double V[3] = {0.0, 0.0, 0.0};
    {
        const int ib = i / a.g.I;
        const int ns = geom_last(a.g, ib) - geom_first(a.g, ib) + 1;
        if constexpr (MODE == MODE_FP32) {
            float vf[3] = {0.0f, 0.0f, 0.0f};
            for (int s = 0; s < ns; ++s)
                for (int d = 0; d < 3; ++d)
                    vf[d] = __fadd_rn(vf[d], static_cast<float>(a.part[(static_cast<size_t>(s) * 3 + d) * a.npad + i]));
            for (int d = 0; d < 3; ++d) V[d] = vf[d];
        } else {
            for (int s = 0; s < ns; ++s)
                for (int d = 0; d < 3; ++d) V[d] += a.part[(static_cast<size_t>(s) * 3 + d) * a.npad + i];
        }
    }
    const V4 pi = pm[i];
    const double xi = a.x64[3 * i], yi = a.x64[3 * i + 1], zi = a.x64[3 * i + 2];
    // self term: replace the clamped dense value by mu_ii / mu0 = I
    {
        double t[3];
        dense_term<TDENSE, MODE>(pi, pi, fm[i], a.pc, t);
        for (int d = 0; d < 3; ++d) V[d] += a.F64[3 * i + d] - t[d];
    }
    // near pairs in FP64
    bool coincident = false;
    for_each_neighbour(a.cl, i, a.cl.cell[i], [&](int j) {
        const double dx = xi - a.x64[3 * j], dy = yi - a.x64[3 * j + 1], dz = zi - a.x64[3 * j + 2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= a.rnear2) return;
        if (r2 == 0.0 && TENSOR != T_RPY) {
            coincident = true;
            return;
        }
        double A, B, dA, dB;
        profile_exact<TENSOR>(r2, a.pc, A, B, dA, dB);
        const double fx = a.F64[3 * j], fy = a.F64[3 * j + 1], fz = a.F64[3 * j + 2];
        const double s = B * (dx * fx + dy * fy + dz * fz);
        double t[3];
        dense_term<TDENSE, MODE>(pi, pm[j], fm[j], a.pc, t);
        V[0] += (A * fx + s * dx) - t[0];
        V[1] += (A * fy + s * dy) - t[1];
        V[2] += (A * fz + s * dz) - t[2];
    });
    if (coincident) atomicOr(a.err, DEV_ERR_COINCIDENT);
    const double m0 = a.pc.mu0;
    const double v0 = m0 * V[0], v1 = m0 * V[1], v2 = m0 * V[2];
    if constexpr (OUT == OUT_F32) {
        float *o = static_cast<float *>(a.vout);
        o[3 * i] = static_cast<float>(v0);
        o[3 * i + 1] = static_cast<float>(v1);
        o[3 * i + 2] = static_cast<float>(v2);
    } else if constexpr (OUT == OUT_F64) {
        double *o = static_cast<double *>(a.vout);
        o[3 * i] = v0;
        o[3 * i + 1] = v1;
        o[3 * i + 2] = v2;
    } else {
        const double nx = xi + a.dt * v0, ny = yi + a.dt * v1, nz = zi + a.dt * v2;
        if (!isfinite(nx) || !isfinite(ny) || !isfinite(nz)) atomicOr(a.err, DEV_ERR_NONFINITE);
        a.x64n[3 * i] = nx;
        a.x64n[3 * i + 1] = ny;
        a.x64n[3 * i + 2] = nz;
    }
}

template <int TENSOR, int MODE>
static void epi_launch(int out, int nb, cudaStream_t st, const EpiArgs &a) {
    switch (out) {
        case OUT_F32: epilogue_kernel<TENSOR, MODE, OUT_F32><<<nb, 128, 0, st>>>(a); break;
        case OUT_F64: epilogue_kernel<TENSOR, MODE, OUT_F64><<<nb, 128, 0, st>>>(a); break;
        default: epilogue_kernel<TENSOR, MODE, OUT_EULER><<<nb, 128, 0, st>>>(a); break;
    }
}

template <int TENSOR>
static void epi_launch_mode(int mode, int out, int nb, cudaStream_t st, const EpiArgs &a) {
    switch (mode) {
        case MODE_FP32C: epi_launch<TENSOR, MODE_FP32C>(out, nb, st, a); break;
        case MODE_FP64: epi_launch<TENSOR, MODE_FP64>(out, nb, st, a); break;
        default: epi_launch<TENSOR, MODE_FP32>(out, nb, st, a); break;
    }
}

cudaError_t launch_epilogue(sd_handle *h, cudaStream_t st, int out, const double *x64, const void *posm,
                            const double *F64, const void *frcm, void *vout, double dt, double *x64n) {
    if (h->n == 0) return cudaSuccess;
    EpiArgs a;
    a.part = h->part;
    a.npad = h->npad;
    a.g = h->geom;
    a.x64 = x64;
    a.posm = posm;
    a.F64 = F64;
    a.frcm = frcm;
    a.cl = h->cl;
    a.rnear2 = h->r_near * h->r_near;
    a.pc = h->pc;
    a.n = h->n;
    a.vout = vout;
    a.dt = dt;
    a.x64n = x64n;
    a.err = h->d_err;
    const int nb = (h->n + 127) / 128;
    prof_begin(h, SD_KERNEL_EPILOGUE, st);
    switch (h->tensor) {
        case T_RPY: epi_launch_mode<T_RPY>(h->mode, out, nb, st, a); break;
        case T_RP: epi_launch_mode<T_RP>(h->mode, out, nb, st, a); break;
        default: epi_launch_mode<T_OSEEN>(h->mode, out, nb, st, a); break;
    }
    prof_end(h, SD_KERNEL_EPILOGUE, st);
    ++h->launches;
    return cudaGetLastError();
}

}  // namespace sd
