// pair.cuh -- the pair term of the mobility sum, in the scalar form
//
//   T(r) / mu0 = A(r) I + B(r) r r^T        (r unnormalised)
//
// which is Eq. rotneMobility (Sec. 2.2) regrouped with rr = r r^T / r^2:
//   Rotne-Prager, r >= 2a : A = c1/r + c3/r^3,   B = c1/r^3 - 3 c3/r^5,   c1 = 3a/4, c3 = a^3/2
//   Oseen (Eq. oseenTensor): A = c1/r,           B = c1/r^3          ((I+rr)/(8 pi eta r) = mu0 (3a/4r)(I+rr))
//   RPY overlap, r < 2a   : A = 1 - 9r/(32a),    B = 3/(32 a r)      (Yamakawa continuation)
// so that T(r) F = mu0 [A F + B (r.F) r].  mu0 is applied once per particle in
// the epilogue, never per pair.
//
// The all-pairs ("dense") kernels evaluate the Rotne-Prager / Oseen branch for
// every pair, with r^2 clamped to >= (2a)^2 (one FMNMX instead of a branch) in
// the tiles that hold self pairs, and everywhere when some pair is closer than
// r_safe; an FP64 pass replaces the self term and every pair closer than r_near
// by its exact value.  Every FP32 operation is an
// explicit round-to-nearest intrinsic, so the epilogue can re-evaluate exactly
// the value a dense kernel used for a pair.
#pragma once
#include <cuda_runtime.h>
#include "ptx.cuh"

namespace sd {

enum { T_RPY = 0, T_RP = 1, T_OSEEN = 2 };

// 32-byte aligned four-double vector (position or force + padding).
using dbl4 = double4_32a;

struct PairConst {
    float r2min_f, c1_f, c3_f, m3c3_f;   // (2a)^2, 3a/4, a^3/2, -3a^3/2
    double r2min_d, c1_d, c3_d, m3c3_d;
    double a, two_a, mu0;
    // periodic box, nearest image only (Sec. 3.1 footnote): side L_d, 1/L_d; both 0
    // in a dimension without periodicity (the minimum image is then the identity)
    float Lf[3], invLf[3];
    double Ld[3], invLd[3];
    int periodic;
};

// Nearest image of a separation d in a dimension of period L (1/L = invL):
// d - L rint(d / L), with rint(t) = (t + 1.5 2^23) - 1.5 2^23, exact round-to-even
// for |t| < 2^22 (FP32; 2^51 for FP64).  The result is odd in d, bit for bit, so
// the image of r_j - r_i is the negated image of r_i - r_j; with invL = 0 it is d.
__device__ __forceinline__ float min_image_f32(float d, float L, float invL) {
    const float n = __fsub_rn(__fadd_rn(__fmul_rn(d, invL), 12582912.0f), 12582912.0f);
    return __fmaf_rn(-L, n, d);
}
__device__ __forceinline__ double min_image_f64(double d, double L, double invL) {
    const double n = __dsub_rn(__dadd_rn(__dmul_rn(d, invL), 6755399441055744.0), 6755399441055744.0);
    return __fma_rn(-L, n, d);
}

// ---------------------------------------------------------------- dense FP32

// One pair of the dense sum, accumulated into (ax, ay, az): 22 FP32-pipe ops
// (RP) or 20 (Oseen), one MUFU.RSQ, and with CLAMP one FMNMX.
template <int TENSOR, bool CLAMP = true, bool PER = false>
__device__ __forceinline__ void pair_f32(float xi, float yi, float zi, float4 p, float4 f, const PairConst &c,
                                         float &ax, float &ay, float &az) {
    float dx = __fsub_rn(xi, p.x);
    float dy = __fsub_rn(yi, p.y);
    float dz = __fsub_rn(zi, p.z);
    if (PER) {
        dx = min_image_f32(dx, c.Lf[0], c.invLf[0]);
        dy = min_image_f32(dy, c.Lf[1], c.invLf[1]);
        dz = min_image_f32(dz, c.Lf[2], c.invLf[2]);
    }
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    if (CLAMP) r2 = fmaxf(r2, c.r2min_f);
    const float ri = rsqrt_sfu(r2);
    const float ri2 = __fmul_rn(ri, ri);
    float A, B;
    if (TENSOR == T_OSEEN) {
        A = __fmul_rn(c.c1_f, ri);
        B = __fmul_rn(A, ri2);
    } else {
        A = __fmul_rn(ri, __fmaf_rn(c.c3_f, ri2, c.c1_f));
        const float ri3 = __fmul_rn(ri, ri2);
        B = __fmul_rn(ri3, __fmaf_rn(c.m3c3_f, ri2, c.c1_f));
    }
    const float dF = __fmaf_rn(dz, f.z, __fmaf_rn(dy, f.y, __fmul_rn(dx, f.x)));
    const float s = __fmul_rn(B, dF);
    ax = __fmaf_rn(s, dx, __fmaf_rn(A, f.x, ax));
    ay = __fmaf_rn(s, dy, __fmaf_rn(A, f.y, ay));
    az = __fmaf_rn(s, dz, __fmaf_rn(A, f.z, az));
}

// ---------------------------------------------------------------- dense FP32, packed

#ifndef SD_SYM_RCP
#define SD_SYM_RCP 0
#endif

// Two FP32 lanes in one 64-bit register pair, operated on by the sm_100+ packed
// instructions {add,sub,mul,fma}.rn.f32x2: one issued instruction, two IEEE
// round-to-nearest results.  Each half is bit-identical to the scalar op.
using f2 = unsigned long long;

__device__ __forceinline__ f2 pk2(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Host-side (c, c) pair: the first element of mov.b64 {lo, hi} is the low word.
inline f2 pk2_host(float c) {
    unsigned int b;
    __builtin_memcpy(&b, &c, sizeof(b));
    return (static_cast<f2>(b) << 32) | b;
}

struct PairConst2 {
    f2 c1, c3, m3c3;   // (c, c) pairs of the constants of PairConst
    float r2min;
    f2 negL[3], invL[3];   // (-L, -L), (1/L, 1/L) per dimension (zeros: not periodic)
    int n;                 // particles (periodic kernels: tiles reaching index n clamp)
};

__device__ __forceinline__ f2 min_image2(f2 d, f2 negL, f2 invL) {
    const f2 magic = 0x4B4000004B400000ull;   // (1.5 2^23, 1.5 2^23)
    const f2 n = sub2(add2(mul2(d, invL), magic), magic);
    return fma2(negL, n, d);
}

// Two pairs at once, lane by lane the operation sequence of pair_f32<TENSOR, CLAMP>:
// either (i, j0), (i, j1) with P* = (x_j0, x_j1) and XI = (x_i, x_i), or
// (i0, j), (i1, j) with XI = (x_i0, x_i1) and P* = (x_j, x_j).  With TRACK, mn0
// and mn1 receive the two unclamped r^2.
template <int TENSOR, bool CLAMP, bool TRACK, bool PER = false>
__device__ __forceinline__ void pair_f32x2_t(f2 XI, f2 YI, f2 ZI, f2 PX, f2 PY, f2 PZ, f2 FX, f2 FY, f2 FZ,
                                             const PairConst2 &c, f2 &AX, f2 &AY, f2 &AZ, float &mn0,
                                             float &mn1) {
    f2 dx = sub2(XI, PX);
    f2 dy = sub2(YI, PY);
    f2 dz = sub2(ZI, PZ);
    if (PER) {
        dx = min_image2(dx, c.negL[0], c.invL[0]);
        dy = min_image2(dy, c.negL[1], c.invL[1]);
        dz = min_image2(dz, c.negL[2], c.invL[2]);
    }
    const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    float ra, rb;
    upk2(r2, ra, rb);
    if (TRACK) {
        mn0 = ra;
        mn1 = rb;
    }
    if (CLAMP) {
        ra = fmaxf(ra, c.r2min);
        rb = fmaxf(rb, c.r2min);
    }
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
    const f2 dF = fma2(dz, FZ, fma2(dy, FY, mul2(dx, FX)));
    const f2 s = mul2(B, dF);
    AX = fma2(s, dx, fma2(A, FX, AX));
    AY = fma2(s, dy, fma2(A, FY, AY));
    AZ = fma2(s, dz, fma2(A, FZ, AZ));
}

template <int TENSOR, bool CLAMP = true, bool PER = false>
__device__ __forceinline__ void pair_f32x2(f2 XI, f2 YI, f2 ZI, f2 PX, f2 PY, f2 PZ, f2 FX, f2 FY, f2 FZ,
                                           const PairConst2 &c, f2 &AX, f2 &AY, f2 &AZ) {
    float unused0 = 0.0f, unused1 = 0.0f;
    pair_f32x2_t<TENSOR, CLAMP, false, PER>(XI, YI, ZI, PX, PY, PZ, FX, FY, FZ, c, AX, AY, AZ, unused0, unused1);
}

// The pairs (i, j0), (i, j1) used in both directions (mu_ij = mu_ji, Sec. 2.2):
// XI = (x_i, x_i), GX = (F_i, F_i), P* = (x_j0, x_j1), F* = (F_j0, F_j1).
//   AX += mu(r_i - r_j) F_j      (the target's sum, lanes j0 / j1)
//   JX += mu(r_j - r_i) F_i      (the sources' sums, lanes j0 / j1)
// r_j - r_i = -(r_i - r_j) exactly, T is even in r and round-to-nearest is odd, so
// each lane's J term is bit-identical to pair_f32x2_t evaluated for (j, i); A and B
// are shared.  32 packed FP32-pipe instructions for four pair terms (RP).
template <int TENSOR, bool CLAMP, bool PER = false>
__device__ __forceinline__ void pair_sym_f32x2(f2 XI, f2 YI, f2 ZI, f2 GX, f2 GY, f2 GZ, f2 PX, f2 PY, f2 PZ,
                                               f2 FX, f2 FY, f2 FZ, const PairConst2 &c, f2 &AX, f2 &AY,
                                               f2 &AZ, f2 &JX, f2 &JY, f2 &JZ) {
    f2 dx = sub2(XI, PX);
    f2 dy = sub2(YI, PY);
    f2 dz = sub2(ZI, PZ);
    if (PER) {
        dx = min_image2(dx, c.negL[0], c.invL[0]);
        dy = min_image2(dy, c.negL[1], c.invL[1]);
        dz = min_image2(dz, c.negL[2], c.invL[2]);
    }
    const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    float ra, rb;
    upk2(r2, ra, rb);
    if (CLAMP) {
        ra = fmaxf(ra, c.r2min);
        rb = fmaxf(rb, c.r2min);
    }
    const f2 ri = pk2(rsqrt_sfu(ra), rsqrt_sfu(rb));
#if SD_SYM_RCP
    const f2 ri2 = pk2(rcp_sfu(ra), rcp_sfu(rb));
#else
    const f2 ri2 = mul2(ri, ri);
#endif
    f2 A, B;
    if (TENSOR == T_OSEEN) {
        A = mul2(c.c1, ri);
        B = mul2(A, ri2);
    } else {
        A = mul2(ri, fma2(c.c3, ri2, c.c1));
        const f2 ri3 = mul2(ri, ri2);
        B = mul2(ri3, fma2(c.m3c3, ri2, c.c1));
    }
    const f2 dF = fma2(dz, FZ, fma2(dy, FY, mul2(dx, FX)));
    const f2 s = mul2(B, dF);
    AX = fma2(s, dx, fma2(A, FX, AX));
    AY = fma2(s, dy, fma2(A, FY, AY));
    AZ = fma2(s, dz, fma2(A, FZ, AZ));
    const f2 dG = fma2(dz, GZ, fma2(dy, GY, mul2(dx, GX)));
    const f2 u = mul2(B, dG);
    JX = fma2(u, dx, fma2(A, GX, JX));
    JY = fma2(u, dy, fma2(A, GY, JY));
    JZ = fma2(u, dz, fma2(A, GZ, JZ));
}

// ---------------------------------------------------------------- dense FP64

template <int TENSOR, bool PER = false>
__device__ __forceinline__ void pair_f64(double xi, double yi, double zi, dbl4 p, dbl4 f, const PairConst &c,
                                         double &ax, double &ay, double &az) {
    double dx = __dsub_rn(xi, p.x);
    double dy = __dsub_rn(yi, p.y);
    double dz = __dsub_rn(zi, p.z);
    if (PER) {
        dx = min_image_f64(dx, c.Ld[0], c.invLd[0]);
        dy = min_image_f64(dy, c.Ld[1], c.invLd[1]);
        dz = min_image_f64(dz, c.Ld[2], c.invLd[2]);
    }
    double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
    r2 = fmax(r2, c.r2min_d);
    const double ri = rsqrt_nr64(r2);
    const double ri2 = __dmul_rn(ri, ri);
    double A, B;
    if (TENSOR == T_OSEEN) {
        A = __dmul_rn(c.c1_d, ri);
        B = __dmul_rn(A, ri2);
    } else {
        A = __dmul_rn(ri, __fma_rn(c.c3_d, ri2, c.c1_d));
        const double ri3 = __dmul_rn(ri, ri2);
        B = __dmul_rn(ri3, __fma_rn(c.m3c3_d, ri2, c.c1_d));
    }
    const double dF = __fma_rn(dz, f.z, __fma_rn(dy, f.y, __dmul_rn(dx, f.x)));
    const double s = __dmul_rn(B, dF);
    ax = __fma_rn(s, dx, __fma_rn(A, f.x, ax));
    ay = __fma_rn(s, dy, __fma_rn(A, f.y, ay));
    az = __fma_rn(s, dz, __fma_rn(A, f.z, az));
}

// The pair (i, j) used in both directions in FP64 (mu_ij = mu_ji, Sec. 2.2): r, r^2,
// 1/r, A and B once, then
//   a += mu(r_i - r_j) F_j / mu0    (target i),   b += mu(r_j - r_i) F_i / mu0   (source j).
// r_j - r_i = -(r_i - r_j) exactly and every step is a round-to-nearest operation,
// so each direction is bit-identical to pair_f64 evaluated for that ordered pair.
template <int TENSOR, bool PER = false>
__device__ __forceinline__ void pair_sym_f64(double xi, double yi, double zi, double gx, double gy, double gz,
                                             const dbl4 &p, const dbl4 &f, const PairConst &c, double &ax,
                                             double &ay, double &az, double &bx, double &by, double &bz) {
    double dx = __dsub_rn(xi, p.x);
    double dy = __dsub_rn(yi, p.y);
    double dz = __dsub_rn(zi, p.z);
    if (PER) {
        dx = min_image_f64(dx, c.Ld[0], c.invLd[0]);
        dy = min_image_f64(dy, c.Ld[1], c.invLd[1]);
        dz = min_image_f64(dz, c.Ld[2], c.invLd[2]);
    }
    double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
    r2 = fmax(r2, c.r2min_d);
    const double ri = rsqrt_nr64(r2);
    const double ri2 = __dmul_rn(ri, ri);
    double A, B;
    if (TENSOR == T_OSEEN) {
        A = __dmul_rn(c.c1_d, ri);
        B = __dmul_rn(A, ri2);
    } else {
        A = __dmul_rn(ri, __fma_rn(c.c3_d, ri2, c.c1_d));
        const double ri3 = __dmul_rn(ri, ri2);
        B = __dmul_rn(ri3, __fma_rn(c.m3c3_d, ri2, c.c1_d));
    }
    const double s = __dmul_rn(B, __fma_rn(dz, f.z, __fma_rn(dy, f.y, __dmul_rn(dx, f.x))));
    ax = __fma_rn(s, dx, __fma_rn(A, f.x, ax));
    ay = __fma_rn(s, dy, __fma_rn(A, f.y, ay));
    az = __fma_rn(s, dz, __fma_rn(A, f.z, az));
    const double u = __dmul_rn(B, __fma_rn(dz, gz, __fma_rn(dy, gy, __dmul_rn(dx, gx))));
    bx = __fma_rn(u, dx, __fma_rn(A, gx, bx));
    by = __fma_rn(u, dy, __fma_rn(A, gy, by));
    bz = __fma_rn(u, dz, __fma_rn(A, gz, bz));
}

// ---------------------------------------------------------------- exact FP64 profile

// A(r), B(r) and the radial derivatives divided by r, dA = A'(r)/r, dB = B'(r)/r,
// of the tensor actually in use at separation |r| = sqrt(r2) (r2 > 0, or r2 = 0 for RPY).
template <int TENSOR>
__device__ __forceinline__ void profile_exact(double r2, const PairConst &c, double &A, double &B, double &dA,
                                              double &dB) {
    // 1/r from the SFU seed and two Newton steps (rsqrt_nr64): FP64 division and
    // square-root sequences are avoided because FP64 throughput is scarce on GB300
    if (TENSOR == T_RPY && r2 < c.two_a * c.two_a) {
        if (r2 > 0.0) {
            const double ri = rsqrt_nr64(r2);
            const double r = r2 * ri;
            const double k = 1.0 / (32.0 * c.a);   // constant, folded per launch
            A = 1.0 - 9.0 * k * r;
            B = 3.0 * k * ri;
            dA = -9.0 * k * ri;
            dB = -3.0 * k * ri * ri * ri;
        } else {
            A = 1.0;
            B = dA = dB = 0.0;  // the terms they multiply carry a factor r
        }
        return;
    }
    const double ri = rsqrt_nr64(r2);
    const double ri2 = ri * ri;
    const double ri3 = ri * ri2;
    const double ri5 = ri3 * ri2;
    if (TENSOR == T_OSEEN) {
        A = c.c1_d * ri;
        B = c.c1_d * ri3;
        dA = -c.c1_d * ri3;
        dB = -3.0 * c.c1_d * ri5;
    } else {
        A = c.c1_d * ri + c.c3_d * ri3;
        B = c.c1_d * ri3 - 3.0 * c.c3_d * ri5;
        dA = -c.c1_d * ri3 - 3.0 * c.c3_d * ri5;
        dB = -3.0 * c.c1_d * ri5 + 15.0 * c.c3_d * ri5 * ri2;
    }
}

// ---------------------------------------------------------------- VJP pair terms

// For the pair (i, j) at r = x_i - x_j with forces Fi, Fj and cotangents Wi, Wj:
//   m += A Wj + B (r.Wj) r                                  (row i of mu W)
//   g += (dA U + dB Q) r + B [Wi (Fj.r) + Fj (Wi.r) + Wj (Fi.r) + Fi (Wj.r)]
// with U = Wi.Fj + Wj.Fi and Q = (Wi.r)(Fj.r) + (Wj.r)(Fi.r)  -- the gradient of
// Wi.T(r)Fj + Wj.T(r)Fi with respect to x_i.  FP32, r^2 clamped like pair_f32.
template <int TENSOR, bool PER = false>
__device__ __forceinline__ void vjp_pair_f32(float xi, float yi, float zi, float3 Fi, float3 Wi, float4 p, float4 f,
                                             float4 w, const PairConst &c, float3 &m, float3 &g) {
    float dx = __fsub_rn(xi, p.x);
    float dy = __fsub_rn(yi, p.y);
    float dz = __fsub_rn(zi, p.z);
    if (PER) {
        dx = min_image_f32(dx, c.Lf[0], c.invLf[0]);
        dy = min_image_f32(dy, c.Lf[1], c.invLf[1]);
        dz = min_image_f32(dz, c.Lf[2], c.invLf[2]);
    }
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    r2 = fmaxf(r2, c.r2min_f);
    const float ri = rsqrt_sfu(r2);
    const float ri2 = __fmul_rn(ri, ri);
    const float ri3 = __fmul_rn(ri, ri2);
    const float ri5 = __fmul_rn(ri3, ri2);
    float A, B, dA, dB;
    if (TENSOR == T_OSEEN) {
        A = __fmul_rn(c.c1_f, ri);
        B = __fmul_rn(c.c1_f, ri3);
        dA = __fmul_rn(-c.c1_f, ri3);
        dB = __fmul_rn(-3.0f * c.c1_f, ri5);
    } else {
        A = __fmul_rn(ri, __fmaf_rn(c.c3_f, ri2, c.c1_f));
        B = __fmul_rn(ri3, __fmaf_rn(c.m3c3_f, ri2, c.c1_f));
        dA = __fmul_rn(ri3, __fmaf_rn(c.m3c3_f, ri2, -c.c1_f));                 // -c1/r^3 - 3c3/r^5
        dB = __fmul_rn(ri5, __fmaf_rn(-5.0f * c.m3c3_f, ri2, -3.0f * c.c1_f));  // -3c1/r^5 + 15c3/r^7
    }
    const float Wir = __fmaf_rn(dz, Wi.z, __fmaf_rn(dy, Wi.y, __fmul_rn(dx, Wi.x)));
    const float Fir = __fmaf_rn(dz, Fi.z, __fmaf_rn(dy, Fi.y, __fmul_rn(dx, Fi.x)));
    const float Wjr = __fmaf_rn(dz, w.z, __fmaf_rn(dy, w.y, __fmul_rn(dx, w.x)));
    const float Fjr = __fmaf_rn(dz, f.z, __fmaf_rn(dy, f.y, __fmul_rn(dx, f.x)));
    const float WiFj = __fmaf_rn(Wi.z, f.z, __fmaf_rn(Wi.y, f.y, __fmul_rn(Wi.x, f.x)));
    const float U = __fmaf_rn(w.z, Fi.z, __fmaf_rn(w.y, Fi.y, __fmaf_rn(w.x, Fi.x, WiFj)));
    const float Q = __fmaf_rn(Wjr, Fir, __fmul_rn(Wir, Fjr));
    const float cr = __fmaf_rn(dB, Q, __fmul_rn(dA, U));
    const float bFj = __fmul_rn(B, Fjr), bWi = __fmul_rn(B, Wir), bFi = __fmul_rn(B, Fir), bWj = __fmul_rn(B, Wjr);
    g.x = __fmaf_rn(cr, dx, __fmaf_rn(Wi.x, bFj, __fmaf_rn(f.x, bWi, __fmaf_rn(w.x, bFi, __fmaf_rn(Fi.x, bWj, g.x)))));
    g.y = __fmaf_rn(cr, dy, __fmaf_rn(Wi.y, bFj, __fmaf_rn(f.y, bWi, __fmaf_rn(w.y, bFi, __fmaf_rn(Fi.y, bWj, g.y)))));
    g.z = __fmaf_rn(cr, dz, __fmaf_rn(Wi.z, bFj, __fmaf_rn(f.z, bWi, __fmaf_rn(w.z, bFi, __fmaf_rn(Fi.z, bWj, g.z)))));
    m.x = __fmaf_rn(bWj, dx, __fmaf_rn(A, w.x, m.x));
    m.y = __fmaf_rn(bWj, dy, __fmaf_rn(A, w.y, m.y));
    m.z = __fmaf_rn(bWj, dz, __fmaf_rn(A, w.z, m.z));
}

// Packed constants of vjp_pair_f32x2: the values vjp_pair_f32 forms from PairConst,
// each as a (c, c) pair (products such as -5 m3c3 rounded in FP32 as there).
struct VjpConst2 {
    f2 c1, c3, m3c3, nc1, n5m3c3, n3c1;   // c1, c3, m3c3, -c1, -5 m3c3, -3 c1
    float r2min;
    f2 negL[3], invL[3];
};

// Two pairs at once, (i, j0) and (i, j1): XI.. FI.. WI.. = the target's values in both
// lanes, P* F* W* = (source j0, source j1).  Lane by lane the operation sequence of
// vjp_pair_f32, so each lane's terms are bit-identical to it (the epilogue subtracts
// vjp_pair_f32's value for the pairs closer than r_near).
template <int TENSOR, bool PER = false>
__device__ __forceinline__ void vjp_pair_f32x2(f2 XI, f2 YI, f2 ZI, f2 FIx, f2 FIy, f2 FIz, f2 WIx, f2 WIy, f2 WIz,
                                               f2 PX, f2 PY, f2 PZ, f2 FX, f2 FY, f2 FZ, f2 WX, f2 WY, f2 WZ,
                                               const VjpConst2 &c, f2 (&M)[3], f2 (&G)[3]) {
    f2 dx = sub2(XI, PX);
    f2 dy = sub2(YI, PY);
    f2 dz = sub2(ZI, PZ);
    if (PER) {
        dx = min_image2(dx, c.negL[0], c.invL[0]);
        dy = min_image2(dy, c.negL[1], c.invL[1]);
        dz = min_image2(dz, c.negL[2], c.invL[2]);
    }
    const f2 r2p = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    float ra, rb;
    upk2(r2p, ra, rb);
    ra = fmaxf(ra, c.r2min);
    rb = fmaxf(rb, c.r2min);
    const f2 ri = pk2(rsqrt_sfu(ra), rsqrt_sfu(rb));
    const f2 ri2 = mul2(ri, ri);
    const f2 ri3 = mul2(ri, ri2);
    const f2 ri5 = mul2(ri3, ri2);
    f2 A, B, dA, dB;
    if (TENSOR == T_OSEEN) {
        A = mul2(c.c1, ri);
        B = mul2(c.c1, ri3);
        dA = mul2(c.nc1, ri3);
        dB = mul2(c.n3c1, ri5);
    } else {
        A = mul2(ri, fma2(c.c3, ri2, c.c1));
        B = mul2(ri3, fma2(c.m3c3, ri2, c.c1));
        dA = mul2(ri3, fma2(c.m3c3, ri2, c.nc1));
        dB = mul2(ri5, fma2(c.n5m3c3, ri2, c.n3c1));
    }
    const f2 Wir = fma2(dz, WIz, fma2(dy, WIy, mul2(dx, WIx)));
    const f2 Fir = fma2(dz, FIz, fma2(dy, FIy, mul2(dx, FIx)));
    const f2 Wjr = fma2(dz, WZ, fma2(dy, WY, mul2(dx, WX)));
    const f2 Fjr = fma2(dz, FZ, fma2(dy, FY, mul2(dx, FX)));
    const f2 WiFj = fma2(WIz, FZ, fma2(WIy, FY, mul2(WIx, FX)));
    const f2 U = fma2(WZ, FIz, fma2(WY, FIy, fma2(WX, FIx, WiFj)));
    const f2 Q = fma2(Wjr, Fir, mul2(Wir, Fjr));
    const f2 cr = fma2(dB, Q, mul2(dA, U));
    const f2 bFj = mul2(B, Fjr), bWi = mul2(B, Wir), bFi = mul2(B, Fir), bWj = mul2(B, Wjr);
    G[0] = fma2(cr, dx, fma2(WIx, bFj, fma2(FX, bWi, fma2(WX, bFi, fma2(FIx, bWj, G[0])))));
    G[1] = fma2(cr, dy, fma2(WIy, bFj, fma2(FY, bWi, fma2(WY, bFi, fma2(FIy, bWj, G[1])))));
    G[2] = fma2(cr, dz, fma2(WIz, bFj, fma2(FZ, bWi, fma2(WZ, bFi, fma2(FIz, bWj, G[2])))));
    M[0] = fma2(bWj, dx, fma2(A, WX, M[0]));
    M[1] = fma2(bWj, dy, fma2(A, WY, M[1]));
    M[2] = fma2(bWj, dz, fma2(A, WZ, M[2]));
}

// The same pair in FP64 with the clamp (what the FP64 dense VJP kernel adds).
template <int TENSOR, bool PER = false>
__device__ __forceinline__ void vjp_pair_f64(double xi, double yi, double zi, double3 Fi, double3 Wi, dbl4 p,
                                             dbl4 f, dbl4 w, const PairConst &c, double3 &m, double3 &g) {
    double dx = __dsub_rn(xi, p.x);
    double dy = __dsub_rn(yi, p.y);
    double dz = __dsub_rn(zi, p.z);
    if (PER) {
        dx = min_image_f64(dx, c.Ld[0], c.invLd[0]);
        dy = min_image_f64(dy, c.Ld[1], c.invLd[1]);
        dz = min_image_f64(dz, c.Ld[2], c.invLd[2]);
    }
    double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
    r2 = fmax(r2, c.r2min_d);
    const double ri = rsqrt_nr64(r2);
    const double ri2 = ri * ri;
    const double ri3 = ri * ri2;
    const double ri5 = ri3 * ri2;
    double A, B, dA, dB;
    if (TENSOR == T_OSEEN) {
        A = c.c1_d * ri;
        B = c.c1_d * ri3;
        dA = -c.c1_d * ri3;
        dB = -3.0 * c.c1_d * ri5;
    } else {
        A = ri * fma(c.c3_d, ri2, c.c1_d);
        B = ri3 * fma(c.m3c3_d, ri2, c.c1_d);
        dA = ri3 * fma(c.m3c3_d, ri2, -c.c1_d);
        dB = ri5 * fma(-5.0 * c.m3c3_d, ri2, -3.0 * c.c1_d);
    }
    const double Wir = dx * Wi.x + dy * Wi.y + dz * Wi.z;
    const double Fir = dx * Fi.x + dy * Fi.y + dz * Fi.z;
    const double Wjr = dx * w.x + dy * w.y + dz * w.z;
    const double Fjr = dx * f.x + dy * f.y + dz * f.z;
    const double U = Wi.x * f.x + Wi.y * f.y + Wi.z * f.z + w.x * Fi.x + w.y * Fi.y + w.z * Fi.z;
    const double Q = Wir * Fjr + Wjr * Fir;
    const double cr = dA * U + dB * Q;
    const double bFj = B * Fjr, bWi = B * Wir, bFi = B * Fir, bWj = B * Wjr;
    g.x += cr * dx + Wi.x * bFj + f.x * bWi + w.x * bFi + Fi.x * bWj;
    g.y += cr * dy + Wi.y * bFj + f.y * bWi + w.y * bFi + Fi.y * bWj;
    g.z += cr * dz + Wi.z * bFj + f.z * bWi + w.z * bFi + Fi.z * bWj;
    m.x += A * w.x + bWj * dx;
    m.y += A * w.y + bWj * dy;
    m.z += A * w.z + bWj * dz;
}

// ---------------------------------------------------------------- compensated sums

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no FMA contraction).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Fold a tile partial p into the two-float accumulator (hi, lo).
__device__ __forceinline__ void fold2(float &hi, float &lo, float p) {
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
}

}  // namespace sd
