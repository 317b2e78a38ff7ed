/*
 * sd_oracle.c -- plain, slow FP64 CPU oracle for leading-order Stokesian dynamics
 * (Kopp & Hoefling, "GPU-accelerated simulation of colloidal suspensions with
 * direct hydrodynamic interactions", arXiv:1205.6333).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  It shares no
 * code, header, table or helper with the CUDA library in paper_1205_6333_gb300/,
 * and the CUDA library never calls it.
 *
 * Everything is IEEE double, written as the paper states it, with no blocking,
 * fusion or reordering:
 *   - Stokes self mobility mu0 = 1/(6 pi eta a)                     (Sec. 2.2, Eq. rotneMobility)
 *   - Rotne-Prager tensor, written literally as
 *       T(r) = mu0 3a/(4r) (I + rr) + mu0 a^3/(2 r^3) (I - 3 rr)     (Sec. 2.2, Eq. rotneMobility)
 *   - Oseen tensor G(r) = (I + rr)/(8 pi eta r)                      (Sec. 2.2, Eq. oseenTensor)
 *   - Yamakawa regularisation for overlapping spheres r < 2a (RPY):
 *       mu0 [(1 - 9r/(32a)) I + (3r/(32a)) rr]
 *     This form is not in the paper; it is the textbook continuation of the
 *     Rotne-Prager tensor inside r < 2a (reading 1 of the design notes).
 *   - mobility sum v_i = sum_j mu_ij F_j, one ascending-j loop per i,
 *     self term mu0 F_i (Sec. 2.2 Eq. rotneMobility; Sec. 3.2 Algorithm 1)
 *   - explicit Euler r_i <- r_i + dt v_i (Sec. 3.1, step 1); forces F_ext plus
 *     a truncated soft repulsion U = eps (2a/r)^12 for r < r_c (Sec. 3.1, step 2),
 *     optionally minus the singular lubrication friction of pairs closer than 3a
 *     with the previous step's velocities (Sec. 2.3 Eq. lubrication; Sec. 3.1)
 *   - adjoint of the Euler recursion with the closed-form derivative of the
 *     pair tensor (derived from Eq. rotneMobility; not in the paper).
 *
 * Periodic boxes use the nearest image only (Sec. 3.1, footnote on boundaries).
 * Parallelism: OpenMP over the target index i only (each i's sum stays a
 * sequential ascending-j loop), used solely to time the oracle on many cores.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SDO_RPY 0
#define SDO_RP 1
#define SDO_OSEEN 2

#define SDO_OK 0
#define SDO_ERR_ARG 1
#define SDO_ERR_COINCIDENT 4

static const double SDO_PI = 3.14159265358979323846;

/* Stokes mobility of one sphere, mu0 = 1/(6 pi eta a) (Sec. 2.2). */
double sdo_mu0(double a, double eta) { return 1.0 / (6.0 * SDO_PI * eta * a); }

/* Nearest-image separation: r_d <- r_d - L_d round(r_d / L_d) when L_d > 0
 * (Sec. 3.1, footnote: only the nearest image of each particle interacts). */
static void sdo_min_image(const double *box, double r[3]) {
    if (!box) return;
    for (int d = 0; d < 3; ++d)
        if (box[d] > 0.0) r[d] -= box[d] * nearbyint(r[d] / box[d]);
}

/* 3x3 pair tensor T(r) (row-major) for a separation vector r != 0.
 * Returns SDO_ERR_COINCIDENT for r == 0 in the RP and Oseen modes. */
int sdo_pair_tensor(int tensor, double a, double eta, const double r[3], double T[9]) {
    const double mu0 = sdo_mu0(a, eta);
    const double rr2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double rn = sqrt(rr2);
    double e[3] = {0.0, 0.0, 0.0};
    if (rn > 0.0) { e[0] = r[0] / rn; e[1] = r[1] / rn; e[2] = r[2] / rn; }
    if (rn == 0.0 && tensor != SDO_RPY) return SDO_ERR_COINCIDENT;
    for (int al = 0; al < 3; ++al) {
        for (int be = 0; be < 3; ++be) {
            const double I = (al == be) ? 1.0 : 0.0;
            const double ee = e[al] * e[be];
            double t;
            if (tensor == SDO_OSEEN) {
                /* G(r) = (I + rr) / (8 pi eta r), Eq. oseenTensor */
                t = (I + ee) / (8.0 * SDO_PI * eta * rn);
            } else if (tensor == SDO_RPY && rn < 2.0 * a) {
                /* Yamakawa continuation for overlapping spheres */
                t = mu0 * ((1.0 - 9.0 * rn / (32.0 * a)) * I + (3.0 * rn / (32.0 * a)) * ee);
            } else {
                /* Rotne-Prager, Eq. rotneMobility, term by term */
                t = mu0 * (3.0 * a / (4.0 * rn)) * (I + ee)
                  + mu0 * (a * a * a / (2.0 * rn * rn * rn)) * (I - 3.0 * ee);
            }
            T[3 * al + be] = t;
        }
    }
    return SDO_OK;
}

/* One row block of the mobility product:
 *   v_i = sum_{j=1..N} mu_ij F_j,  mu_ii = mu0 I,  mu_ij = T(r_i - r_j)
 * with j ascending, exactly as Algorithm 1 walks it. */
static int sdo_row(int tensor, double a, double eta, const double *box, int n,
                   const double *x, const double *F, int i, double vi[3]) {
    const double mu0 = sdo_mu0(a, eta);
    double acc[3] = {0.0, 0.0, 0.0};
    int st = SDO_OK;
    for (int j = 0; j < n; ++j) {
        if (j == i) {
            for (int d = 0; d < 3; ++d) acc[d] += mu0 * F[3 * i + d];
            continue;
        }
        double r[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
        sdo_min_image(box, r);
        double T[9];
        int s = sdo_pair_tensor(tensor, a, eta, r, T);
        if (s != SDO_OK) { st = s; continue; }
        for (int al = 0; al < 3; ++al)
            acc[al] += T[3 * al] * F[3 * j] + T[3 * al + 1] * F[3 * j + 1] + T[3 * al + 2] * F[3 * j + 2];
    }
    vi[0] = acc[0]; vi[1] = acc[1]; vi[2] = acc[2];
    return st;
}

/* v = M(x) F for all N particles.  x, F, v: n x 3 row-major doubles. */
int sdo_mobility_apply(int tensor, double a, double eta, const double *box, int n,
                       const double *x, const double *F, double *v, int nthreads) {
    if (n < 0 || a <= 0.0 || eta <= 0.0) return SDO_ERR_ARG;
    int st = SDO_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1) reduction(max : st)
#endif
    for (int i = 0; i < n; ++i) {
        int s = sdo_row(tensor, a, eta, box, n, x, F, i, &v[3 * i]);
        if (s > st) st = s;
    }
    (void)nthreads;
    return st;
}

/* Sampled rows: v_rows[k] = (M(x) F)_{rows[k]}.  Same loop as above. */
int sdo_mobility_rows(int tensor, double a, double eta, const double *box, int n,
                      const double *x, const double *F, int nrows, const int32_t *rows,
                      double *vrows, int nthreads) {
    if (n < 0 || nrows < 0 || a <= 0.0 || eta <= 0.0) return SDO_ERR_ARG;
    int st = SDO_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1) reduction(max : st)
#endif
    for (int k = 0; k < nrows; ++k) {
        int i = rows[k];
        int s = (i < 0 || i >= n) ? SDO_ERR_ARG : sdo_row(tensor, a, eta, box, n, x, F, i, &vrows[3 * k]);
        if (s > st) st = s;
    }
    (void)nthreads;
    return st;
}

/* The full 3N x 3N mobility matrix, block (i,j) = mu_ij (row-major). */
int sdo_assemble(int tensor, double a, double eta, const double *box, int n, const double *x, double *M) {
    const double mu0 = sdo_mu0(a, eta);
    const int m = 3 * n;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double T[9];
            if (i == j) {
                for (int k = 0; k < 9; ++k) T[k] = (k % 4 == 0) ? mu0 : 0.0;
            } else {
                double r[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
                sdo_min_image(box, r);
                int s = sdo_pair_tensor(tensor, a, eta, r, T);
                if (s != SDO_OK) return s;
            }
            for (int al = 0; al < 3; ++al)
                for (int be = 0; be < 3; ++be) M[(size_t)(3 * i + al) * m + 3 * j + be] = T[3 * al + be];
        }
    }
    return SDO_OK;
}

/* Step 2 of Sec. 3.1 without lubrication:
 *   F_i = F_ext,i + g + sum_{j: r_ij < r_c} F_int(r_i, r_j),
 * with F_int = -grad_i U(r_ij),  U = eps (2a/r)^12  (truncated, not shifted)
 * => F_int = 12 eps (2a)^12 r^-14 (r_i - r_j).  fext may be NULL. */
int sdo_forces(double a, const double *box, int n, const double *x, const double *fext,
               const double g[3], double rep_eps, double rep_rc, double *F) {
    const double s12 = pow(2.0 * a, 12.0);
    for (int i = 0; i < n; ++i) {
        double f[3] = {g[0], g[1], g[2]};
        if (fext) for (int d = 0; d < 3; ++d) f[d] += fext[3 * i + d];
        if (rep_eps != 0.0) {
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                double r[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
                sdo_min_image(box, r);
                double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                double rn = sqrt(r2);
                if (rn == 0.0) return SDO_ERR_COINCIDENT;
                if (rn < rep_rc) {
                    double c = 12.0 * rep_eps * s12 / pow(rn, 14.0);
                    for (int d = 0; d < 3; ++d) f[d] += c * r[d];
                }
            }
        }
        for (int d = 0; d < 3; ++d) F[3 * i + d] = f[d];
    }
    return SDO_OK;
}

/* Singular lubrication friction of close pairs, Sec. 2.3 Eq. lubrication, in the
 * form Sec. 3.1 step 2 uses it:
 *   F_i -= sum_{j: 0 < s_ij < 1} zeta_ij (v_i - v_j),   s_ij = r_ij / a - 2,
 *   mu0 zeta_ij = (1/(4s) - (9/40) ln s) e e^T - (1/6) ln s (I - e e^T),  e = r_ij / r_ij,
 * truncated at s = 1 (r = 3a) as the paper does; pairs with s <= 0 (overlapping
 * spheres, where the expansion has no value) contribute nothing.  v holds the
 * velocities of the previous step.  The result is ADDED to F. */
int sdo_lubrication(double a, double eta, const double *box, int n, const double *x, const double *v, double *F) {
    const double mu0 = sdo_mu0(a, eta);
    for (int i = 0; i < n; ++i) {
        double f[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double r[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
            sdo_min_image(box, r);
            const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            const double sg = rn / a - 2.0;
            if (!(sg > 0.0 && sg < 1.0)) continue;
            const double e[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
            const double vij[3] = {v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1], v[3 * i + 2] - v[3 * j + 2]};
            const double normal = 1.0 / (4.0 * sg) - (9.0 / 40.0) * log(sg);
            const double tangential = -(1.0 / 6.0) * log(sg);
            for (int al = 0; al < 3; ++al) {
                double zv = 0.0;
                for (int be = 0; be < 3; ++be) {
                    const double I = (al == be) ? 1.0 : 0.0;
                    const double ee = e[al] * e[be];
                    zv += (normal * ee + tangential * (I - ee)) * vij[be];
                }
                f[al] -= zv / mu0;
            }
        }
        for (int d = 0; d < 3; ++d) F[3 * i + d] += f[d];
    }
    return SDO_OK;
}

/* Explicit Euler, Sec. 3.1 steps 1-3 in the standard order
 *   F_n = F(x_n) [- lubrication with v_{n-1}];  v_n = M(x_n) F_n;  x_{n+1} = x_n + dt v_n.
 * x is updated in place.  With lub != 0 the forces of each step carry the
 * lubrication friction computed from the previous step's velocities (zero before
 * the first step).  If traj != NULL, x after every `every`-th step is appended
 * (traj holds (nsteps/every) * n * 3 doubles). */
int sdo_euler(int tensor, double a, double eta, const double *box, int n, double *x,
              const double *fext, const double g[3], double rep_eps, double rep_rc, int lub,
              double dt, int64_t nsteps, int64_t every, double *traj, int nthreads) {
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *v = (double *)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));
    if (!F || !v) { free(F); free(v); return SDO_ERR_ARG; }
    int st = SDO_OK;
    int64_t out = 0;
    for (int64_t s = 0; s < nsteps && st == SDO_OK; ++s) {
        st = sdo_forces(a, box, n, x, fext, g, rep_eps, rep_rc, F);
        if (st != SDO_OK) break;
        if (lub) sdo_lubrication(a, eta, box, n, x, v, F);
        st = sdo_mobility_apply(tensor, a, eta, box, n, x, F, v, nthreads);
        if (st != SDO_OK) break;
        for (int k = 0; k < 3 * n; ++k) x[k] += dt * v[k];
        if (traj && every > 0 && (s + 1) % every == 0) {
            memcpy(traj + out * 3 * (size_t)n, x, sizeof(double) * 3 * (size_t)n);
            ++out;
        }
    }
    free(F); free(v);
    return st;
}

/* Scalar profile of the tensor in the form T(r) = mu0 [A(r) I + B(r) r r^T]
 * (r unnormalised) and the radial derivatives A'(r), B'(r).  Each branch is the
 * same tensor as sdo_pair_tensor, rewritten with rr = r r^T / r^2. */
static void sdo_profile(int tensor, double a, double rn, double *A, double *B, double *dA, double *dB) {
    if (tensor == SDO_OSEEN) {
        /* (I + rr)/(8 pi eta r) = mu0 (3a/4r)(I + rr) */
        *A = 3.0 * a / (4.0 * rn);
        *B = 3.0 * a / (4.0 * rn * rn * rn);
        *dA = -3.0 * a / (4.0 * rn * rn);
        *dB = -9.0 * a / (4.0 * pow(rn, 4));
    } else if (tensor == SDO_RPY && rn < 2.0 * a) {
        *A = 1.0 - 9.0 * rn / (32.0 * a);
        *B = 3.0 / (32.0 * a * rn);
        *dA = -9.0 / (32.0 * a);
        *dB = -3.0 / (32.0 * a * rn * rn);
    } else {
        const double a3 = a * a * a;
        *A = 3.0 * a / (4.0 * rn) + a3 / (2.0 * rn * rn * rn);
        *B = 3.0 * a / (4.0 * pow(rn, 3)) - 3.0 * a3 / (2.0 * pow(rn, 5));
        *dA = -3.0 * a / (4.0 * rn * rn) - 3.0 * a3 / (2.0 * pow(rn, 4));
        *dB = -9.0 * a / (4.0 * pow(rn, 4)) + 15.0 * a3 / (2.0 * pow(rn, 6));
    }
}

/* dT[g][al][be] = d T_{al be}(r) / d r_g   for r != 0
 *   = mu0 [ A'(r) (r_g/r) d_ab + B'(r) (r_g/r) r_a r_b + B(r) (d_ag r_b + r_a d_bg) ]. */
static void sdo_dtensor(int tensor, double a, double eta, const double r[3], double dT[27]) {
    const double mu0 = sdo_mu0(a, eta);
    const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double A, B, dA, dB;
    sdo_profile(tensor, a, rn, &A, &B, &dA, &dB);
    for (int g = 0; g < 3; ++g)
        for (int al = 0; al < 3; ++al)
            for (int be = 0; be < 3; ++be) {
                double d_ab = (al == be) ? 1.0 : 0.0, d_ag = (al == g) ? 1.0 : 0.0, d_bg = (be == g) ? 1.0 : 0.0;
                dT[9 * g + 3 * al + be] = mu0 * (dA * (r[g] / rn) * d_ab + dB * (r[g] / rn) * r[al] * r[be]
                                                 + B * (d_ag * r[be] + r[al] * d_bg));
            }
}

/* Vector-Jacobian products of v(x, F) = M(x) F with a cotangent w:
 *   gF = M(x)^T w = M(x) w   (M is symmetric)
 *   gx_k = sum_{j != k} sum_{al,be} [ w_k,al dT_al,be/dr F_j,be + w_j,al dT_al,be/dr F_k,be ]
 *          evaluated at r = x_k - x_j.
 * gF or gx may be NULL. */
int sdo_vjp(int tensor, double a, double eta, const double *box, int n, const double *x,
            const double *F, const double *w, double *gx, double *gF, int nthreads) {
    int st = SDO_OK;
    if (gF) st = sdo_mobility_apply(tensor, a, eta, box, n, x, w, gF, nthreads);
    if (st != SDO_OK || !gx) return st;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1) reduction(max : st)
#endif
    for (int k = 0; k < n; ++k) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < n; ++j) {
            if (j == k) continue;
            double r[3] = {x[3 * k] - x[3 * j], x[3 * k + 1] - x[3 * j + 1], x[3 * k + 2] - x[3 * j + 2]};
            sdo_min_image(box, r);
            if (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0) {
                if (tensor != SDO_RPY) st = SDO_ERR_COINCIDENT;
                continue; /* RPY: |r| has no derivative at r = 0; the symmetric sub-gradient 0 is taken */
            }
            double dT[27];
            sdo_dtensor(tensor, a, eta, r, dT);
            for (int g = 0; g < 3; ++g) {
                double s = 0.0;
                for (int al = 0; al < 3; ++al)
                    for (int be = 0; be < 3; ++be)
                        s += w[3 * k + al] * dT[9 * g + 3 * al + be] * F[3 * j + be]
                           + w[3 * j + al] * dT[9 * g + 3 * al + be] * F[3 * k + be];
                acc[g] += s;
            }
        }
        gx[3 * k] = acc[0]; gx[3 * k + 1] = acc[1]; gx[3 * k + 2] = acc[2];
    }
    (void)nthreads;
    return st;
}

/* Reverse-mode gradient of a loss L(x_T) through nsteps explicit Euler steps
 *   x_{n+1} = x_n + dt M(x_n) F,   F_i = F_ext,i + g   (no repulsion)
 * given lambda_T = dL/dx_T (gxT):
 *   lambda_n = lambda_{n+1} + dt (d(M(x_n)F)/dx_n)^T lambda_{n+1}
 *   dL/dF_ext  = sum_n dt M(x_n) lambda_{n+1}
 * The whole trajectory is stored (the oracle is only run at small N). */
int sdo_adjoint(int tensor, double a, double eta, const double *box, int n, const double *x0,
                const double *fext, const double g[3], double dt, int64_t nsteps,
                const double *gxT, double *gx0, double *gF, int nthreads) {
    const size_t m = 3 * (size_t)n;
    double *traj = (double *)malloc(sizeof(double) * m * (size_t)(nsteps + 1));
    double *F = (double *)malloc(sizeof(double) * m);
    double *v = (double *)malloc(sizeof(double) * m);
    double *lam = (double *)malloc(sizeof(double) * m);
    double *tx = (double *)malloc(sizeof(double) * m);
    double *tF = (double *)malloc(sizeof(double) * m);
    int st = SDO_OK;
    if (!traj || !F || !v || !lam || !tx || !tF) { st = SDO_ERR_ARG; goto done; }
    for (size_t k = 0; k < m; ++k) F[k] = (fext ? fext[k] : 0.0) + g[k % 3];
    memcpy(traj, x0, sizeof(double) * m);
    for (int64_t s = 0; s < nsteps; ++s) {
        const double *xs = traj + (size_t)s * m;
        double *xn = traj + (size_t)(s + 1) * m;
        st = sdo_mobility_apply(tensor, a, eta, box, n, xs, F, v, nthreads);
        if (st != SDO_OK) goto done;
        for (size_t k = 0; k < m; ++k) xn[k] = xs[k] + dt * v[k];
    }
    memcpy(lam, gxT, sizeof(double) * m);
    for (size_t k = 0; k < m; ++k) gF[k] = 0.0;
    for (int64_t s = nsteps - 1; s >= 0; --s) {
        const double *xs = traj + (size_t)s * m;
        st = sdo_vjp(tensor, a, eta, box, n, xs, F, lam, tx, tF, nthreads);
        if (st != SDO_OK) goto done;
        for (size_t k = 0; k < m; ++k) {
            gF[k] += dt * tF[k];
            lam[k] += dt * tx[k];
        }
    }
    memcpy(gx0, lam, sizeof(double) * m);
done:
    free(traj); free(F); free(v); free(lam); free(tx); free(tF);
    return st;
}

int sdo_has_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
