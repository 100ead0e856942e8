/*
 * al_oracle.c -- plain FP64 CPU oracle of the actuator-line transfer
 * operators (sampling -> Morison drag -> normalised Gaussian projection).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: it exists so that tests/, the smoke check and the
 * bench's CPU-baseline leg can compare the CUDA path against a slow,
 * obviously correct restatement of the paper's equations.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Every step follows the paper (arXiv 2609.39443) in its own order and
 * notation:
 *   Sec. 3.2.2  actuator point (Eq. almActuatorPoint), tangent, preliminary
 *               relative velocity (Eq. almPreliminaryVelocity), sampling
 *               point (Eq. almSamplingPoint) with the fallback direction,
 *               relative velocity (Eq. almRelativeVelocity);
 *   Sec. 3.2.3  line force (Eq. almLineForce) and relaxation
 *               (Eq. almForceRelaxation);
 *   Sec. 3.2.4  bounding-box cull, closest segment and projection point
 *               (Eq. almProjectionPoint), truncated 2-D Gaussian
 *               (Eq. almGaussian), nodal weights w_k, normalised nodal
 *               force and momentum source (Eq. almMomentumSource);
 *   Sec. 2.1    mixture density rho = alpha rho1 + (1 - alpha) rho2.
 * Readings of points the paper leaves open (sign of the line force,
 * trilinear vs single-cell sampling, several lines, zero weights, points
 * outside the domain) are stated where they are used.
 *
 * Everything is FP64.  The projection of one line is independent of the
 * others (each line carries its own nearest segment, weights and
 * normalisation, and S is the sum over lines); lines are processed in
 * chunks in parallel, and their contributions are added to S sequentially
 * in line order, so the result does not depend on the thread count.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    double h;
    double o[3];
    int has_alpha;
    double rho1, rho2, rho_const;
} or_grid;

typedef struct {
    int n_lines;
    const int *line_off;              /* n_lines + 1 */
    const double *d, *cdn, *cdt;      /* per line */
    const double *eps, *ell_s, *alpha_f;
    const double *cv_len;             /* per point */
    double n_p[3], g_up[3], tau;
    int sample_mode;                  /* 0 trilinear, 1 containing cell, 2 Gaussian volume average */
    int drag_mode;                    /* 0 Eq. almLineForce, 1 Eq. fext_drag */
    int proj_mode;                    /* 0 nearest segment (Eq. almProjectionPoint), 1 segment-integrated */
    const double *cm_n, *cm_t;        /* per line, added-mass coefficients of Eq. fext_addedmass;
                                         NULL: no inertia term (the paper's model) */
    int wall_reflect;                 /* bit 2a (2a+1): the low (high) face of axis a reflects
                                         the kernel (the projection variant of Sec. 6) */
} or_beams;

/* status counters (same meaning as the CUDA library's) */
enum {
    OR_ST_PA_OUTSIDE = 0,   /* actuator point outside the grid: no load */
    OR_ST_PS_OUTSIDE = 1,   /* sampling point outside the grid: no load (Sec. 3.2.5) */
    OR_ST_FALLBACK = 2,     /* |u0_n| < tau: fallback upstream direction */
    OR_ST_FALLBACK_ZERO = 3,/* fallback direction parallel to the tangent */
    OR_ST_ZERO_WEIGHT = 4,  /* node with w_k = 0 */
    OR_ST_DEPOSIT_LOST = 5, /* zero-weight node outside the grid */
    OR_ST_N = 8
};

static const double OR_PI = 3.14159265358979323846;

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------ */
/* point -> cell search on the uniform grid                            */
/* ------------------------------------------------------------------ */

/* Continuous cell coordinate u = (p - o)/h per axis; the point is inside
 * the grid iff 0 <= u < n on every axis. */
static int or_locate(const or_grid *g, const double p[3], double u[3])
{
    const int n[3] = {g->nx, g->ny, g->nz};
    int inside = 1;
    for (int a = 0; a < 3; ++a) {
        u[a] = (p[a] - g->o[a]) / g->h;
        if (!(u[a] >= 0.0 && u[a] < (double)n[a])) inside = 0;
    }
    return inside;
}

/* Sample an SoA field (ncomp components, component c at f + c*N_c) at p.
 * mode 1: value stored in the single cell containing p, the operator of
 *         Eqs. almPreliminaryVelocity / almRelativeVelocity (floor rule);
 * mode 0: trilinear interpolation between the 8 surrounding cell centres.
 *         In the half cell next to a wall the index is clamped, i.e. the
 *         wall cell's value is extended to the wall.
 * mode 2: kernel-weighted volume average with the Gaussian of the
 *         projection (the smooth sampler the paper's Sec. 6 proposes):
 *         value = sum_j g_j f_j / sum_j g_j over the cells j of the grid
 *         whose centre C_j lies within 3 eps of p, g_j = exp(-(|C_j - p|/eps)^2)
 *         (the truncated profile of Eq. almGaussian; its constant factor
 *         cancels).  Cells outside the grid do not enter, so near a wall the
 *         average is one-sided.  When no cell centre lies within 3 eps the
 *         containing cell's value is returned (the limit of the normalised
 *         average as eps -> 0: the nearest centre is the containing cell's).
 * Returns 0 (and leaves out untouched) when p lies outside the grid. */
static int or_sample(const or_grid *g, const double *f, int ncomp, int mode, double eps,
                     const double p[3], double *out)
{
    double u[3];
    if (!or_locate(g, p, u)) return 0;
    const int n[3] = {g->nx, g->ny, g->nz};
    const long long nxy = (long long)g->nx * g->ny;
    const long long ncell = nxy * g->nz;
    if (mode == 2) {
        const double R = 3.0 * eps;
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            /* every centre within R of p lies in this index range (one cell of slack) */
            lo[a] = (int)floor(u[a] - 0.5 - R / g->h) - 1;
            hi[a] = (int)floor(u[a] - 0.5 + R / g->h) + 1;
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > n[a] - 1) hi[a] = n[a] - 1;
        }
        double *acc = (double *)calloc((size_t)ncomp, sizeof(double));
        double sw = 0.0;
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    const double C[3] = {g->o[0] + (i + 0.5) * g->h, g->o[1] + (j + 0.5) * g->h,
                                         g->o[2] + (k + 0.5) * g->h};
                    const double d[3] = {C[0] - p[0], C[1] - p[1], C[2] - p[2]};
                    const double r2 = dot3(d, d);
                    if (r2 > R * R) continue;
                    const double wgt = exp(-r2 / (eps * eps));
                    const long long idx = i + (long long)g->nx * j + nxy * k;
                    sw += wgt;
                    for (int q = 0; q < ncomp; ++q) acc[q] += wgt * f[q * ncell + idx];
                }
        if (sw > 0.0) {
            for (int q = 0; q < ncomp; ++q) out[q] = acc[q] / sw;
            free(acc);
            return 1;
        }
        free(acc);
        mode = 1;
    }
    if (mode == 1) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = (int)floor(u[a]);
            if (c[a] > n[a] - 1) c[a] = n[a] - 1;
        }
        long long idx = c[0] + (long long)g->nx * c[1] + nxy * c[2];
        for (int q = 0; q < ncomp; ++q) out[q] = f[q * ncell + idx];
        return 1;
    }
    int i0[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        double xc = u[a] - 0.5;               /* coordinate in cell-centre units */
        if (xc < 0.0) xc = 0.0;
        if (xc > (double)(n[a] - 1)) xc = (double)(n[a] - 1);
        if (n[a] == 1) { i0[a] = 0; t[a] = 0.0; continue; }
        int i = (int)floor(xc);
        if (i > n[a] - 2) i = n[a] - 2;
        i0[a] = i;
        t[a] = xc - (double)i;
    }
    for (int q = 0; q < ncomp; ++q) out[q] = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double wgt = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);
                int ix = i0[0] + (n[0] > 1 ? dx : 0);
                int iy = i0[1] + (n[1] > 1 ? dy : 0);
                int iz = i0[2] + (n[2] > 1 ? dz : 0);
                long long idx = ix + (long long)g->nx * iy + nxy * iz;
                for (int q = 0; q < ncomp; ++q) out[q] += wgt * f[q * ncell + idx];
            }
    return 1;
}

/* Exported for the sampler pins. */
int or_sample_field(const or_grid *g, const double *f, int ncomp, int mode, double eps,
                    const double *p, double *out)
{
    return or_sample(g, f, ncomp, mode, eps, p, out);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2.2 - 3.2.3: sampling and line force, one actuator point      */
/* ------------------------------------------------------------------ */

/* Centreline tangent e_t,i.  The paper reconstructs it from a Hermite
 * spline through the beam-cell centres without giving the formula; the
 * reading used is the Catmull-Rom (central-difference) tangent
 * P_{i+1} - P_{i-1}, one-sided at the two ends, normalised.  A line of
 * a single point has no tangent (zero vector). */
static void or_tangent(const double *P, long long np, int off, int n, int q, const double *tin,
                       double t[3])
{
    long long i = off + q;
    if (tin) {
        for (int a = 0; a < 3; ++a) t[a] = tin[a * np + i];
    } else if (n == 1) {
        t[0] = t[1] = t[2] = 0.0;
    } else {
        long long ip = (q == n - 1) ? i : i + 1;
        long long im = (q == 0) ? i : i - 1;
        for (int a = 0; a < 3; ++a) t[a] = P[a * np + ip] - P[a * np + im];
    }
    double nn = sqrt(dot3(t, t));
    if (nn > 0.0) for (int a = 0; a < 3; ++a) t[a] /= nn;
    else t[0] = t[1] = t[2] = 0.0;
}

int or_point_step(const or_grid *g, const or_beams *b,
                  const double *U, const double *alpha,
                  const double *P, const double *Pdot, const double *tangent,
                  const double *f_prev,
                  const double *U_prev, const double *Pddot, double dt,
                  double *F, double *f_out, double *e_t_out, double *P_s_out,
                  long long *status)
{
    const long long np = b->line_off[b->n_lines];
    for (int l = 0; l < b->n_lines; ++l) {
        const int off = b->line_off[l], n = b->line_off[l + 1] - off;
        for (int q = 0; q < n; ++q) {
            const long long i = off + q;
            double Pa[3], Pd[3], t[3];
            for (int a = 0; a < 3; ++a) { Pa[a] = P[a * np + i]; Pd[a] = Pdot[a * np + i]; }
            or_tangent(P, np, off, n, q, tangent, t);

            double fstar[3] = {0.0, 0.0, 0.0};
            double Ps[3] = {Pa[0], Pa[1], Pa[2]};
            double Ua[3];
            if (!or_sample(g, U, 3, b->sample_mode, b->eps[l], Pa, Ua)) {
                status[OR_ST_PA_OUTSIDE]++;            /* no load for this step */
            } else {
                /* Eq. almPreliminaryVelocity and its normal part */
                double u0r[3], u0n[3], es[3];
                for (int a = 0; a < 3; ++a) u0r[a] = Ua[a] - Pd[a];
                double ut = dot3(u0r, t);
                for (int a = 0; a < 3; ++a) u0n[a] = u0r[a] - ut * t[a];
                double nn = sqrt(dot3(u0n, u0n));
                if (nn >= b->tau) {
                    for (int a = 0; a < 3; ++a) es[a] = -u0n[a] / nn;
                } else {
                    /* fallback: global upstream direction projected onto the
                     * cross-section plane and renormalised */
                    status[OR_ST_FALLBACK]++;
                    double gt = dot3(b->g_up, t), gp[3];
                    for (int a = 0; a < 3; ++a) gp[a] = b->g_up[a] - gt * t[a];
                    double gn = sqrt(dot3(gp, gp));
                    if (gn > 0.0) for (int a = 0; a < 3; ++a) es[a] = gp[a] / gn;
                    else { es[0] = es[1] = es[2] = 0.0; status[OR_ST_FALLBACK_ZERO]++; }
                }
                /* Eq. almSamplingPoint: P_s = P_a + (I - n_p n_p^T) l_s e_s */
                double v[3];
                for (int a = 0; a < 3; ++a) v[a] = b->ell_s[l] * es[a];
                double vn = dot3(b->n_p, v);
                for (int a = 0; a < 3; ++a) Ps[a] = Pa[a] + (v[a] - b->n_p[a] * vn);

                double Us[4];
                int nc = g->has_alpha ? 1 : 0;
                if (!or_sample(g, U, 3, b->sample_mode, b->eps[l], Ps, Us) ||
                    (nc && !or_sample(g, alpha, 1, b->sample_mode, b->eps[l], Ps, Us + 3))) {
                    status[OR_ST_PS_OUTSIDE]++;        /* no load for this step */
                } else {
                    double rho = g->has_alpha ? Us[3] * g->rho1 + (1.0 - Us[3]) * g->rho2 : g->rho_const;
                    /* Eq. almRelativeVelocity and the tangential / normal split */
                    double Ur[3], Ut[3], Un[3];
                    for (int a = 0; a < 3; ++a) Ur[a] = Us[a] - Pd[a];
                    double urt = dot3(Ur, t);
                    for (int a = 0; a < 3; ++a) { Ut[a] = urt * t[a]; Un[a] = Ur[a] - Ut[a]; }
                    /* Line force on the beam.  It points along the relative
                     * flow (the sign of Eq. fext_drag); the fluid receives
                     * the opposite through the minus of Eq. almMomentumSource. */
                    double half = 0.5 * rho * b->d[l];
                    if (b->drag_mode == 0) {           /* Eq. almLineForce: |U_r| for both parts */
                        double m = sqrt(dot3(Ur, Ur));
                        for (int a = 0; a < 3; ++a)
                            fstar[a] = half * m * (b->cdn[l] * Un[a] + b->cdt[l] * Ut[a]);
                    } else {                           /* Eq. fext_drag: |V_t| V_t and |V_n| V_n */
                        double mt = sqrt(dot3(Ut, Ut)), mn = sqrt(dot3(Un, Un));
                        for (int a = 0; a < 3; ++a)
                            fstar[a] = half * (b->cdt[l] * mt * Ut[a] + b->cdn[l] * mn * Un[a]);
                    }
                    if (b->cm_n) {
                        /* Eq. fext_addedmass: fluid acceleration a_f = (U - U_prev) / dt
                         * sampled at P_s with the same operator, beam acceleration a_b;
                         * the added-mass reaction follows the fluid's acceleration
                         * relative to the beam, a_f - a_b, split along the tangent like
                         * the drag, plus the Froude-Krylov term rho A a_f */
                        double af[3] = {0.0, 0.0, 0.0}, ab[3] = {0.0, 0.0, 0.0};
                        if (U_prev) {
                            double Up[3];
                            or_sample(g, U_prev, 3, b->sample_mode, b->eps[l], Ps, Up);   /* inside: checked above */
                            for (int a = 0; a < 3; ++a) af[a] = (Us[a] - Up[a]) / dt;
                        }
                        if (Pddot) for (int a = 0; a < 3; ++a) ab[a] = Pddot[a * np + i];
                        double ar[3], art, area = 0.25 * OR_PI * b->d[l] * b->d[l];
                        for (int a = 0; a < 3; ++a) ar[a] = af[a] - ab[a];
                        art = dot3(ar, t);
                        for (int a = 0; a < 3; ++a) {
                            double at = art * t[a], an = ar[a] - at;
                            fstar[a] += rho * area * (b->cm_t[l] * at + b->cm_n[l] * an + af[a]);
                        }
                    }
                }
            }
            /* Eq. almForceRelaxation (no previous force: un-relaxed) */
            double f[3];
            for (int a = 0; a < 3; ++a) {
                f[a] = f_prev ? b->alpha_f[l] * fstar[a] + (1.0 - b->alpha_f[l]) * f_prev[a * np + i]
                              : fstar[a];
                F[a * np + i] = f[a] * b->cv_len[i];   /* per-CV load f_i L_i */
                if (f_out) f_out[a * np + i] = f[a];
                if (e_t_out) e_t_out[a * np + i] = t[a];
                if (P_s_out) P_s_out[a * np + i] = Ps[a];
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2.4: projection of one line to the fluid mesh                 */
/* ------------------------------------------------------------------ */

typedef struct { long long cell; int seg; double s, eta; } or_rec;

typedef struct {
    or_rec *rec; long long nrec, cap;
    double *fhat;          /* 3 x n nodes */
    double *w;             /* n nodes */
    long long *dep_cell;   /* deposit cell per node (-1: none / lost) */
    long long st[OR_ST_N];
} or_line_out;

static void or_push(or_line_out *o, long long cell, int seg, double s, double eta)
{
    if (o->nrec == o->cap) {
        o->cap = o->cap ? 2 * o->cap : 1024;
        o->rec = (or_rec *)realloc(o->rec, (size_t)o->cap * sizeof(or_rec));
    }
    o->rec[o->nrec].cell = cell; o->rec[o->nrec].seg = seg;
    o->rec[o->nrec].s = s; o->rec[o->nrec].eta = eta;
    o->nrec++;
}

/* Distance from c to segment [A, B] with the foot of the perpendicular
 * (Eq. almProjectionPoint): s = clamp(((c-A).(B-A)) / |B-A|^2, 0, 1),
 * foot = A + s (B - A), r^2 = |c - foot|^2.  A zero-length segment has
 * s = 0. */
static double or_seg_dist2(const double c[3], const double A[3], const double B[3], double *s_out)
{
    double D[3], q[3];
    for (int a = 0; a < 3; ++a) { D[a] = B[a] - A[a]; q[a] = c[a] - A[a]; }
    double L2 = dot3(D, D);
    double s = 0.0;
    if (L2 > 0.0) {
        s = dot3(q, D) / L2;
        if (s < 0.0) s = 0.0;
        if (s > 1.0) s = 1.0;
    }
    double e[3];
    for (int a = 0; a < 3; ++a) e[a] = q[a] - s * D[a];
    *s_out = s;
    return dot3(e, e);
}

/* Closest actuator segment of a line of n nodes X[0..n-1] to c: every
 * segment is tested and on equal distance the lower index is kept.
 * Returns r^2, the segment index and s.  A single-node line has one
 * zero-length segment. */
static double or_closest(const double (*X)[3], int n, const double c[3], int *kbest, double *sbest)
{
    const int nseg = (n == 1) ? 1 : n - 1;
    double best = INFINITY;
    *kbest = -1; *sbest = 0.0;
    for (int k = 0; k < nseg; ++k) {
        int kb = (n == 1) ? k : k + 1;
        double s, r2 = or_seg_dist2(c, X[k], X[kb], &s);
        if (r2 < best) { best = r2; *kbest = k; *sbest = s; }
    }
    return best;
}

/* Exported for the closest-segment pin: X is (3, n) row-major. */
double or_closest_segment(const double *X, int n, const double *c, int *kbest, double *sbest)
{
    double (*Y)[3] = (double (*)[3])malloc((size_t)n * sizeof(double[3]));
    for (int k = 0; k < n; ++k) for (int a = 0; a < 3; ++a) Y[k][a] = X[a * n + k];
    double r2 = or_closest((const double (*)[3])Y, n, c, kbest, sbest);
    free(Y);
    return r2;
}

/* Segment-integrated 3-D Gaussian (the projection variant of Sec. 6): for
 * the segment A -> B of length L and the point c,
 *   K0 = int_0^L G3(c - P(t)) dt,   K1 = int_0^L (t / L) G3(c - P(t)) dt,
 * P(t) = A + t (B - A) / L, G3(x) = exp(-|x|^2 / eps^2) / (pi^(3/2) eps^3),
 * the 3-D Gaussian whose integral along an infinite line is the 2-D kernel
 * of Eq. almGaussian.  With t0 the tangential coordinate of c and r_p its
 * distance from the segment's axis, G3 factors into exp(-r_p^2/eps^2) and a
 * 1-D Gaussian in t - t0, whose integral and first moment over [0, L] are
 * erf and exp terms:
 *   K0 = g E,  E = (erf((L - t0)/eps) + erf(t0/eps)) / 2,
 *   K1 = (g / L) (t0 E + eps / (2 sqrt(pi)) (exp(-t0^2/eps^2) - exp(-(L-t0)^2/eps^2))),
 *   g = exp(-r_p^2 / eps^2) / (pi eps^2).
 * A zero-length segment gives K0 = K1 = 0. */
void or_seg_kernel(const double *c, const double *A, const double *B, double eps, double *K)
{
    double D[3], x[3];
    for (int a = 0; a < 3; ++a) { D[a] = B[a] - A[a]; x[a] = c[a] - A[a]; }
    const double L = sqrt(dot3(D, D));
    if (!(L > 0.0)) { K[0] = K[1] = 0.0; return; }
    const double t0 = dot3(x, D) / L;
    double p[3];
    for (int a = 0; a < 3; ++a) p[a] = x[a] - t0 * D[a] / L;
    const double g = exp(-dot3(p, p) / (eps * eps)) / (OR_PI * eps * eps);
    const double E = 0.5 * (erf((L - t0) / eps) + erf(t0 / eps));
    K[0] = g * E;
    K[1] = g / L * (t0 * E + eps / (2.0 * sqrt(OR_PI)) *
                                 (exp(-t0 * t0 / (eps * eps)) - exp(-(L - t0) * (L - t0) / (eps * eps))));
}

/* Index of the grid cell a ghost cell beyond a reflecting face mirrors
 * onto: -1 - i below the low face, 2n - 1 - i above the high face. */
static int or_fold(int i, int n)
{
    return i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i);
}

static void or_project_line(const or_grid *g, const or_beams *b, const double *Ps, long long np,
                            const double *F, int l, int cull, or_line_out *o)
{
    const int off = b->line_off[l], n = b->line_off[l + 1] - off;
    memset(o, 0, sizeof(*o));
    if (n <= 0) return;
    const double eps = b->eps[l], R = 3.0 * eps, V = g->h * g->h * g->h;
    o->w = (double *)calloc((size_t)n, sizeof(double));
    o->fhat = (double *)calloc((size_t)3 * n, sizeof(double));
    o->dep_cell = (long long *)malloc((size_t)n * sizeof(long long));
    for (int k = 0; k < n; ++k) o->dep_cell[k] = -1;

    /* node coordinates */
    double (*X)[3] = (double (*)[3])malloc((size_t)n * sizeof(double[3]));
    for (int k = 0; k < n; ++k)
        for (int a = 0; a < 3; ++a) X[k][a] = Ps[a * np + off + k];

    /* bounding box of the actuator points inflated by 3 eps (Sec. 3.2.4);
     * cells whose centre lies outside it are skipped.  The index range is
     * widened by one cell so that rounding of the box bounds can never drop
     * a cell inside it (cells beyond the box are farther than R from every
     * segment, so extra cells change nothing). */
    /* A reflecting face (the one-sided kernel of Sec. 6, read as a mirror)
     * adds G = ceil(3 eps / h) + 1 layers of ghost cells beyond it: the
     * kernel is evaluated at their centres like at any cell's, and each
     * ghost's share goes to the grid cell it mirrors (or_fold), so the mass
     * that falls outside the domain comes back next to the wall rather than
     * being spread over the node's whole support by the normalisation.  One
     * reflection per face: at most n ghost layers. */
    const int nn[3] = {g->nx, g->ny, g->nz};
    const int G = (int)ceil(R / g->h) + 1;
    int glo[3], ghi[3];
    for (int a = 0; a < 3; ++a) {
        const int gd = G < nn[a] ? G : nn[a];
        glo[a] = ((b->wall_reflect >> (2 * a)) & 1) ? -gd : 0;
        ghi[a] = ((b->wall_reflect >> (2 * a + 1)) & 1) ? nn[a] - 1 + gd : nn[a] - 1;
    }
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        if (!cull) { lo[a] = glo[a]; hi[a] = ghi[a]; continue; }
        double mn = X[0][a], mx = X[0][a];
        for (int k = 1; k < n; ++k) { if (X[k][a] < mn) mn = X[k][a]; if (X[k][a] > mx) mx = X[k][a]; }
        double il = ceil((mn - R - g->o[a]) / g->h - 0.5) - 1.0;
        double ih = floor((mx + R - g->o[a]) / g->h - 0.5) + 1.0;
        if (il < glo[a]) il = glo[a];
        if (ih > ghi[a]) ih = ghi[a];
        lo[a] = (int)il; hi[a] = (int)ih;
    }
    const long long nxy = (long long)g->nx * g->ny;
    for (int kz = lo[2]; kz <= hi[2]; ++kz)
        for (int jy = lo[1]; jy <= hi[1]; ++jy)
            for (int ix = lo[0]; ix <= hi[0]; ++ix) {
                double c[3] = {g->o[0] + (ix + 0.5) * g->h, g->o[1] + (jy + 0.5) * g->h,
                               g->o[2] + (kz + 0.5) * g->h};
                const long long cell = or_fold(ix, g->nx) + (long long)g->nx * or_fold(jy, g->ny) +
                                       nxy * or_fold(kz, g->nz);
                if (b->proj_mode == 1 && n >= 2) {
                    /* every segment whose closest point lies within 3 eps
                     * contributes its integrated kernel; the record keeps
                     * eta = K0 and s = K1 / K0, so (1 - s) eta and s eta are
                     * the two nodes' shares */
                    for (int k = 0; k + 1 < n; ++k) {
                        double sk;
                        if (or_seg_dist2(c, X[k], X[k + 1], &sk) > R * R) continue;
                        double K[2];
                        or_seg_kernel(c, X[k], X[k + 1], eps, K);
                        if (K[0] > 0.0)
                            or_push(o, cell, k, K[1] / K[0], K[0]);
                    }
                    continue;
                }
                double sbest;
                int kbest;
                double r = sqrt(or_closest(X, n, c, &kbest, &sbest));
                if (r <= R) {                   /* truncation at 3 eps, inclusive */
                    double x = r / eps;
                    double eta = exp(-x * x) / (OR_PI * eps * eps);   /* Eq. almGaussian */
                    or_push(o, cell, kbest, sbest, eta);
                }
            }
    /* nodal weights w_k = sum_j omega_jk eta_j V_j with omega_ji = 1 - s_j,
     * omega_j,i+1 = s_j, accumulated in cell order */
    for (long long r = 0; r < o->nrec; ++r) {
        int ka = o->rec[r].seg, kb = (n == 1) ? ka : ka + 1;
        o->w[ka] += (1.0 - o->rec[r].s) * o->rec[r].eta * V;
        o->w[kb] += o->rec[r].s * o->rec[r].eta * V;
    }
    /* normalised nodal force f^_k = f_k Delta s_k / w_k with f_k Delta s_k
     * = F_k, the per-CV load (Delta s_k read as the CV length L_k).  A node
     * with no weight cannot be normalised (the paper requires w_k != 0);
     * its load is deposited in the cell containing the node so that the
     * resultant is still transferred. */
    for (int k = 0; k < n; ++k) {
        if (o->w[k] > 0.0) {
            for (int a = 0; a < 3; ++a) o->fhat[3 * k + a] = F[a * np + off + k] / o->w[k];
        } else {
            o->st[OR_ST_ZERO_WEIGHT]++;
            double u[3];
            if (or_locate(g, X[k], u)) {
                long long cc[3];
                for (int a = 0; a < 3; ++a) { cc[a] = (long long)floor(u[a]); if (cc[a] > nn[a] - 1) cc[a] = nn[a] - 1; }
                o->dep_cell[k] = cc[0] + (long long)g->nx * cc[1] + nxy * cc[2];
            } else {
                o->st[OR_ST_DEPOSIT_LOST]++;
            }
        }
    }
    free(X);
}

/* S -= contributions of one line (Eq. almMomentumSource), plus deposits */
static void or_apply_line(const or_grid *g, const or_beams *b, const double *F, long long np,
                          int l, const or_line_out *o, double *S, double *w_out, long long *status)
{
    const int off = b->line_off[l], n = b->line_off[l + 1] - off;
    if (n <= 0) return;
    const long long ncell = (long long)g->nx * g->ny * g->nz;
    const double V = g->h * g->h * g->h;
    for (long long r = 0; r < o->nrec; ++r) {
        int ka = o->rec[r].seg, kb = (n == 1) ? ka : ka + 1;
        double s = o->rec[r].s, eta = o->rec[r].eta;
        for (int a = 0; a < 3; ++a)
            S[a * ncell + o->rec[r].cell] -= eta * ((1.0 - s) * o->fhat[3 * ka + a] + s * o->fhat[3 * kb + a]);
    }
    for (int k = 0; k < n; ++k)
        if (o->dep_cell[k] >= 0)
            for (int a = 0; a < 3; ++a) S[a * ncell + o->dep_cell[k]] -= F[a * np + off + k] / V;
    if (w_out) for (int k = 0; k < n; ++k) w_out[off + k] = o->w[k];
    for (int q = 0; q < OR_ST_N; ++q) status[q] += o->st[q];
}

static void or_free_line(or_line_out *o)
{
    free(o->rec); free(o->fhat); free(o->w); free(o->dep_cell);
    memset(o, 0, sizeof(*o));
}

/* Projection of every (or every masked) line.  S is accumulated into
 * (S -= ...), the caller zeroes it.  w (optional) receives w_k. */
int or_project(const or_grid *g, const or_beams *b, const double *Pspread, const double *F,
               int cull, const unsigned char *line_mask, double *S, double *w,
               long long *status, int n_threads)
{
    const long long np = b->line_off[b->n_lines];
    const int chunk = 128;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    or_line_out *buf = (or_line_out *)calloc(chunk, sizeof(or_line_out));
    for (int l0 = 0; l0 < b->n_lines; l0 += chunk) {
        int l1 = l0 + chunk < b->n_lines ? l0 + chunk : b->n_lines;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
        for (int l = l0; l < l1; ++l) {
            if (line_mask && !line_mask[l]) { memset(&buf[l - l0], 0, sizeof(or_line_out)); continue; }
            or_project_line(g, b, Pspread, np, F, l, cull, &buf[l - l0]);
        }
        for (int l = l0; l < l1; ++l) {
            if (!(line_mask && !line_mask[l])) or_apply_line(g, b, F, np, l, &buf[l - l0], S, w, status);
            or_free_line(&buf[l - l0]);
        }
    }
    free(buf);
    return 0;
}

/* The projection restricted to one slab of a decomposition along x (the
 * parallel update of Sec. 3.2.5): only cells with x index in [x0, x1) take
 * part.  The kernel values and closest segments are those of or_project
 * (the same records); only the sums are restricted.
 *   w_in == NULL: w_out[k] += the part of w_k = sum_j omega_jk eta_j V_j
 *                 over the slab's cells (the slab's partial sum);
 *   w_in != NULL: w_in holds the full weights (every slab's partial sums
 *                 added): f^_k = F_k / w_in[k], S -= the sources of the
 *                 slab's cells (Eq. almMomentumSource), and a node with
 *                 w_in[k] = 0 deposits F_k / V in its cell when that cell
 *                 is in the slab. */
int or_project_slab(const or_grid *g, const or_beams *b, const double *Pspread, const double *F, int x0, int x1,
                    const double *w_in, double *S, double *w_out)
{
    const long long np = b->line_off[b->n_lines];
    const long long ncell = (long long)g->nx * g->ny * g->nz;
    const double V = g->h * g->h * g->h;
    for (int l = 0; l < b->n_lines; ++l) {
        const int off = b->line_off[l], n = b->line_off[l + 1] - off;
        if (n <= 0) continue;
        or_line_out o;
        or_project_line(g, b, Pspread, np, F, l, 1, &o);
        for (long long r = 0; r < o.nrec; ++r) {
            const int ix = (int)(o.rec[r].cell % g->nx);
            if (ix < x0 || ix >= x1) continue;
            const int ka = o.rec[r].seg, kb = (n == 1) ? ka : ka + 1;
            const double s = o.rec[r].s, eta = o.rec[r].eta;
            if (!w_in) {
                w_out[off + ka] += (1.0 - s) * eta * V;
                w_out[off + kb] += s * eta * V;
            } else {
                for (int a = 0; a < 3; ++a) {
                    const double fa = w_in[off + ka] > 0.0 ? F[a * np + off + ka] / w_in[off + ka] : 0.0;
                    const double fb = w_in[off + kb] > 0.0 ? F[a * np + off + kb] / w_in[off + kb] : 0.0;
                    S[a * ncell + o.rec[r].cell] -= eta * ((1.0 - s) * fa + s * fb);
                }
            }
        }
        if (w_in)
            for (int k = 0; k < n; ++k) {
                if (w_in[off + k] > 0.0) continue;
                double u[3];
                const double X[3] = {Pspread[off + k], Pspread[np + off + k], Pspread[2 * np + off + k]};
                if (!or_locate(g, X, u)) continue;
                const int nn[3] = {g->nx, g->ny, g->nz};
                long long cc[3];
                for (int a = 0; a < 3; ++a) { cc[a] = (long long)floor(u[a]); if (cc[a] > nn[a] - 1) cc[a] = nn[a] - 1; }
                if (cc[0] < x0 || cc[0] >= x1) continue;
                const long long cell = cc[0] + (long long)g->nx * cc[1] + (long long)g->nx * g->ny * cc[2];
                for (int a = 0; a < 3; ++a) S[a * ncell + cell] -= F[a * np + off + k] / V;
            }
        or_free_line(&o);
    }
    return 0;
}

/* Number of cells within 3 eps of each line (the kernel-cell updates a
 * coupling step performs), for throughput reporting. */
long long or_count_support(const or_grid *g, const or_beams *b, const double *Pspread, int n_threads)
{
    const long long np = b->line_off[b->n_lines];
    long long total = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
#else
    (void)n_threads;
#endif
    for (int l = 0; l < b->n_lines; ++l) {
        or_line_out o;
        or_project_line(g, b, Pspread, np, Pspread /* F unused for counting */, l, 1, &o);
        total += o.nrec;
        or_free_line(&o);
    }
    return total;
}

/* ------------------------------------------------------------------ */
/* Quasi-static reconstruction (Sec. 7, the E5 test): each CV's load    */
/* as a static point load on a linear Euler-Bernoulli cantilever        */
/* ------------------------------------------------------------------ */

/* Deflection at x of a cantilever clamped at 0 under a unit point load at
 * a (both measured from the root along the axis), times EI:
 *   x <= a: x^2 (3a - x) / 6,   x >= a: a^2 (3x - a) / 6. */
static double or_cantilever_g(double x, double a)
{
    return x <= a ? x * x * (3.0 * a - x) / 6.0 : a * a * (3.0 * x - a) / 6.0;
}

/* For every line: the rest positions P0 define the straight axis (unit
 * vector `axis`, root at the line's first node) and each node's station
 * a_k = (P0_k - P0_root) . axis; the loads F_k (3 x np) act at the nodes;
 * only their parts normal to the axis bend the beam.  Writes
 * P_out_i = P0_i + sum_k F_perp_k g(a_i, a_k) / EI_l. */
void or_beam_quasistatic(const or_beams *b, const double *EI, const double *axis, const double *P0,
                         const double *F, double *P_out)
{
    const long long np = b->line_off[b->n_lines];
    for (int l = 0; l < b->n_lines; ++l) {
        const int off = b->line_off[l], n = b->line_off[l + 1] - off;
        for (int q = 0; q < n; ++q) {
            const long long i = off + q;
            double xi = 0.0;
            for (int a = 0; a < 3; ++a) xi += (P0[a * np + i] - P0[a * np + off]) * axis[a];
            double w[3] = {0.0, 0.0, 0.0};
            for (int r = 0; r < n; ++r) {
                const long long k = off + r;
                double ak = 0.0, fa = 0.0;
                for (int a = 0; a < 3; ++a) {
                    ak += (P0[a * np + k] - P0[a * np + off]) * axis[a];
                    fa += F[a * np + k] * axis[a];
                }
                const double gk = or_cantilever_g(xi, ak);
                for (int a = 0; a < 3; ++a) w[a] += (F[a * np + k] - fa * axis[a]) * gk;
            }
            for (int a = 0; a < 3; ++a) P_out[a * np + i] = P0[a * np + i] + w[a] / EI[l];
        }
    }
}
