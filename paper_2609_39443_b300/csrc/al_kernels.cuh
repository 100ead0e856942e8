// al_kernels.cuh -- sm_103a kernels of the actuator-line transfer operators.
//
// One coupling step (arXiv 2609.39443, Sec. 3.2; Algorithm 1 steps 1-5, 7-8):
//   k_points    per actuator point: tangent, preliminary sample, sampling
//               point, upstream sample (+ alpha, mixture rho), Morison
//               line force, relaxation, F = f L         (Eqs. almActuatorPoint
//               .. almForceRelaxation)
//   k_segments  per segment / node: direction, 1/|D|^2, bisector normal and
//               turning half-angle of the projection geometry
//   k_lines     per line (one warp): bounding box, regularity certificate,
//               FP64 sum of F
//   k_mask      per segment: marks the bricks its 3-eps box touches
//   k_weights   per segment: w contributions of the cells whose closest
//               segment it is (Sec. 3.2.4, w_k), FP32 compensated sums
//   k_normalise per node: w_k, f^_k = F_k / w_k
//   k_spread    per brick of 16x16x8 cells: cell-centric gather of
//               Eq. almMomentumSource over the lines of the brick, every
//               cell of S written exactly once, no atomics
//   k_deposit   zero-weight nodes (w_k = 0) deposit their load in their cell
//   k_totals    FP64 sum F and sum S V
//
// Geometry runs in cell units.  FP32 instances carry point positions as
// float-float pairs (hi + lo) so that cell-relative offsets are accurate to
// ~1e-6 cells even 1000 cells from the origin.  Every geometric decision
// (closest segment, 3-eps cut-off) is taken in FP32 only when the FP32
// value is farther from the decision boundary than its error bound; inside
// that band it is re-taken in FP64 from the caller's original positions,
// with explicitly rounded operations, so both passes (weights and spread)
// always agree and match an FP64 evaluation of the paper's definition.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

namespace al {

constexpr int BX = 16, BY = 16, BZ = 8;          // spread brick (cells)
constexpr int SPREAD_THREADS = BX * BY;          // one thread per column
constexpr float BRICK_DIAG = 24.0f;              // sqrt(16^2+16^2+8^2)
constexpr double PI_D = 3.14159265358979323846;

enum { ST_PA_OUTSIDE = 0, ST_PS_OUTSIDE = 1, ST_FALLBACK = 2, ST_FALLBACK_ZERO = 3,
       ST_ZERO_WEIGHT = 4, ST_DEPOSIT_LOST = 5, ST_REFINED = 6, ST_IRREGULAR = 7, ST_SUPPORT = 8 };

struct GridC {
    int nx, ny, nz;
    long long ncell;
    int nbx, nby, nbz;
    long long nbrick;
    double h, o[3], V;
    float o_hi[3], o_lo[3];      // float-float origin
    float ih_hi, ih_lo;          // float-float 1/h
    int has_alpha;
    double rho1, rho2, rho_const;
};

struct BeamsC {
    int n_lines, n_points, mask_words;
    const int *line_off, *line_of;
    const double *d, *cdn, *cdt, *eps, *ell_s, *alpha_f, *cv_len;
    double n_p[3], g_up[3], tau;
    int sample_mode, drag_mode, tangents_given;
};

struct LineG {                   // per line, rebuilt every step
    float Rc;                    // 3 eps in cell units (box slack only)
    double R2c, inv_eps2c;       // (3 eps)^2, 1/eps^2 in cell units
    double eta0;                 // 1 / (pi eps^2) in 1/m^2
    int regular;                 // closest segment by monotone bisector walk
    int first, n;
};

template <typename T>
struct Scratch {
    T *fprev;                    // [3][np] relaxed force of the previous step
    T *uhi;                      // [3][np] P_spread in cell units (hi part)
    float *ulo;                  // [3][np] lo part (FP32 instances only)
    T *segD;                     // [3][np] D_k = u_{k+1} - u_k
    T *segIl2;                   // [np] 1 / |D_k|^2 (0 for zero length)
    T *nodeM;                    // [3][np] unit bisector at interior nodes
    float *nodeTau;              // [np] tan(theta_k / 2) at interior nodes
    double *segWa, *segWb;       // [np] weight of segment k to its two nodes
    double *w;                   // [np] w_k
    T *fhat;                     // [3][np] normalised nodal force
    double *lineF;               // [3][n_lines] sum of F per line
    LineG *lines;                // [n_lines]
    uint32_t *mask;              // [nbrick][mask_words] lines touching a brick
    double *brickSum;            // [3][nbrick] sum of S per brick
    int *zeroList;               // [np]
    int *zeroCount;              // [1]
    double *depSum;              // [3]
    int *hasPrev;                // [1] a previous relaxed force exists (set by k_totals)
};

template <typename T>
struct StepPtrs {
    const T *U[3];
    const T *alpha;
    const T *P[3];
    const T *Pdot[3];
    const T *Ps[3];              // projection positions (P when not given)
    const T *tan[3];
    T *S[3];
    T *F[3];
    int np;
};

// ---------------------------------------------------------------------------
// precision traits: guard bands (cell units) around geometric decisions
// ---------------------------------------------------------------------------
template <typename T> struct Tr;
template <> struct Tr<float> {
    // |sigma| error <= ~7e-7 |x| + 2.4e-6 cells; band 4e-6 (|x| + 8)
    static __device__ __forceinline__ float gsig(float x) { return 4e-6f * (x + 8.0f); }
    // r^2 error <= ~1e-4 cells^2 at R = 9 cells; band 1e-5 R^2 + 1e-4
    static __device__ __forceinline__ float grr(float R2) { return 1e-5f * R2 + 1e-4f; }
    static __device__ __forceinline__ float ex(float x) { return expf(x); }
};
template <> struct Tr<double> {
    static __device__ __forceinline__ double gsig(double x) { return 1e-12 * (x + 8.0); }
    static __device__ __forceinline__ double grr(double R2) { return 1e-12 * R2 + 1e-12; }
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
};

// ---------------------------------------------------------------------------
// float-float helpers (error-free transformations, Knuth / Dekker)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// cell-unit coordinate of a position p (metres) along axis a
__device__ __forceinline__ void to_cell(const GridC &g, int a, float p, float &uh, float &ul) {
    float s, e;
    two_sum(p, -g.o_hi[a], s, e);
    e = __fsub_rn(e, g.o_lo[a]);
    float dh, dl;
    fast_two_sum(s, e, dh, dl);
    float ph = __fmul_rn(dh, g.ih_hi);
    float pl = __fmaf_rn(dh, g.ih_hi, -ph);
    pl = __fmaf_rn(dh, g.ih_lo, pl);
    pl = __fmaf_rn(dl, g.ih_hi, pl);
    fast_two_sum(ph, pl, uh, ul);
}
__device__ __forceinline__ void to_cell(const GridC &g, int a, double p, double &uh, float &ul) {
    uh = (p - g.o[a]) / g.h;
    ul = 0.0f;
}
// (uh, ul) + d
__device__ __forceinline__ void ff_add(float uh, float ul, float d, float &rh, float &rl) {
    float s, e;
    two_sum(uh, d, s, e);
    e = __fadd_rn(e, ul);
    fast_two_sum(s, e, rh, rl);
}
__device__ __forceinline__ void ff_add(double uh, float ul, double d, double &rh, float &rl) {
    rh = uh + d;
    rl = ul;
}
// position relative to an integer origin B
__device__ __forceinline__ float rel(float uh, float ul, int B) {
    return __fadd_rn(__fsub_rn(uh, (float)B), ul);
}
__device__ __forceinline__ double rel(double uh, float, int B) { return uh - (double)B; }

// inside [0, n) along one axis
template <typename T>
__device__ __forceinline__ bool inside_axis(T uh, float ul, int n) {
    bool lo = (uh > (T)0) || (uh == (T)0 && ul >= 0.0f);
    bool hi = (uh < (T)n) || (uh == (T)n && ul < 0.0f);
    return lo && hi;
}
// floor of uh + ul
template <typename T>
__device__ __forceinline__ int ffloor(T uh, float ul) {
    T f = floor(uh);
    int c = (int)f;
    if (f == uh && ul < 0.0f) c -= 1;
    return c;
}

// floor / ceil in the arithmetic type (no FP64 for FP32 instances)
__device__ __forceinline__ int ifloor(float x) { return (int)floorf(x); }
__device__ __forceinline__ int ifloor(double x) { return (int)floor(x); }
__device__ __forceinline__ int iceil(float x) { return (int)ceilf(x); }
__device__ __forceinline__ int iceil(double x) { return (int)ceil(x); }

// ---------------------------------------------------------------------------
// sampling: trilinear (default) or containing cell
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void axis_stencil(T uh, float ul, int n, int &i0, T &t) {
    if (n == 1) { i0 = 0; t = (T)0; return; }
    T xh = uh - (T)0.5;                     // coordinate in cell-centre units: xh + ul
    if (xh + (T)ul <= (T)0) { i0 = 0; t = (T)0; return; }
    if (xh + (T)ul >= (T)(n - 1)) { i0 = n - 2; t = (T)1; return; }
    int i = (int)floor(xh);
    T fr = (xh - (T)i) + (T)ul;
    if (fr < (T)0) { i -= 1; fr += (T)1; }
    else if (fr >= (T)1) { i += 1; fr -= (T)1; }
    if (i < 0) { i = 0; fr = (T)0; }
    if (i > n - 2) { i = n - 2; fr = (T)1; }
    i0 = i;
    t = fr;
}

// Returns false when the point lies outside the grid.  Fields are stored as
// S and interpolated in the arithmetic type C.
template <typename S, typename C>
__device__ bool sample(const GridC &g, int mode, const S *const *f, int ncomp,
                       const C uh[3], const float ul[3], C *out) {
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a)
        if (!inside_axis(uh[a], ul[a], n[a])) return false;
    const long long nxy = (long long)g.nx * g.ny;
    if (mode == 1) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = ffloor(uh[a], ul[a]);
            c[a] = c[a] < 0 ? 0 : (c[a] > n[a] - 1 ? n[a] - 1 : c[a]);
        }
        long long idx = c[0] + (long long)g.nx * c[1] + nxy * c[2];
        for (int q = 0; q < ncomp; ++q) out[q] = (C)f[q][idx];
        return true;
    }
    int i0[3];
    C t[3];
    for (int a = 0; a < 3; ++a) axis_stencil(uh[a], ul[a], n[a], i0[a], t[a]);
    const int sx = g.nx > 1 ? 1 : 0;
    const long long sy = g.ny > 1 ? g.nx : 0, sz = g.nz > 1 ? nxy : 0;
    const long long base = i0[0] + (long long)g.nx * i0[1] + nxy * i0[2];
    const C wx0 = (C)1 - t[0], wy0 = (C)1 - t[1], wz0 = (C)1 - t[2];
    for (int q = 0; q < ncomp; ++q) {
        const S *F = f[q];
        C c00 = wx0 * (C)F[base] + t[0] * (C)F[base + sx];
        C c10 = wx0 * (C)F[base + sy] + t[0] * (C)F[base + sy + sx];
        C c01 = wx0 * (C)F[base + sz] + t[0] * (C)F[base + sz + sx];
        C c11 = wx0 * (C)F[base + sz + sy] + t[0] * (C)F[base + sz + sy + sx];
        out[q] = wz0 * (wy0 * c00 + t[1] * c10) + t[2] * (wy0 * c01 + t[1] * c11);
    }
    return true;
}

// Quasi-steady line force f* of one actuator point (Secs. 3.2.2-3.2.3) in the
// arithmetic type C from fields stored as T: preliminary sample, upstream
// direction with fallback, sampling point, upstream sample (+ alpha,
// mixture density), Morison drag.  Returns 1 without side effects when C is
// float and the upstream direction is ill-conditioned (|u0_n| below 1 % of
// the velocity scale, where FP32 rounding of the samples is amplified by
// 1/|u0_n|); the caller then repeats the evaluation in FP64.
template <typename T, typename C>
__device__ int point_fstar(const GridC &g, const BeamsC &b, const StepPtrs<T> &p, const int l, const C Pa[3],
                           const C Pd[3], const C t[3], C fstar[3], int *status, const bool refine_ok) {
    fstar[0] = fstar[1] = fstar[2] = (C)0;
    C ua[3];
    float la[3];
    for (int a = 0; a < 3; ++a) to_cell(g, a, Pa[a], ua[a], la[a]);
    C Ua[3];
    if (!sample(g, b.sample_mode, p.U, 3, ua, la, Ua)) {
        atomicAdd(&status[ST_PA_OUTSIDE], 1);
        return 0;
    }
    // Eq. almPreliminaryVelocity and its component normal to the tangent
    C u0r[3], u0n[3], es[3];
    for (int a = 0; a < 3; ++a) u0r[a] = Ua[a] - Pd[a];
    C ut = u0r[0] * t[0] + u0r[1] * t[1] + u0r[2] * t[2];
    for (int a = 0; a < 3; ++a) u0n[a] = u0r[a] - ut * t[a];
    C nn = sqrt(u0n[0] * u0n[0] + u0n[1] * u0n[1] + u0n[2] * u0n[2]);
    if (refine_ok) {
        C scale = sqrt(Ua[0] * Ua[0] + Ua[1] * Ua[1] + Ua[2] * Ua[2]) + sqrt(Pd[0] * Pd[0] + Pd[1] * Pd[1] + Pd[2] * Pd[2]);
        if (nn < (C)1e-2 * scale) return 1;
    }
    if ((double)nn >= b.tau) {
        for (int a = 0; a < 3; ++a) es[a] = -u0n[a] / nn;
    } else {
        atomicAdd(&status[ST_FALLBACK], 1);
        C gp[3];
        C gt = (C)b.g_up[0] * t[0] + (C)b.g_up[1] * t[1] + (C)b.g_up[2] * t[2];
        for (int a = 0; a < 3; ++a) gp[a] = (C)b.g_up[a] - gt * t[a];
        C gn = sqrt(gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2]);
        if (gn > (C)0) for (int a = 0; a < 3; ++a) es[a] = gp[a] / gn;
        else { es[0] = es[1] = es[2] = (C)0; atomicAdd(&status[ST_FALLBACK_ZERO], 1); }
    }
    // Eq. almSamplingPoint: offset (I - n_p n_p^T) l_s e_s
    const C ell = (C)b.ell_s[l];
    C v[3];
    for (int a = 0; a < 3; ++a) v[a] = ell * es[a];
    C vn = (C)b.n_p[0] * v[0] + (C)b.n_p[1] * v[1] + (C)b.n_p[2] * v[2];
    C us[3];
    float ls[3];
    for (int a = 0; a < 3; ++a) {
        C off_c = (v[a] - (C)b.n_p[a] * vn) * (C)(1.0 / g.h);
        ff_add(ua[a], la[a], off_c, us[a], ls[a]);
    }
    C Us[3], as = (C)0;
    bool ok = sample(g, b.sample_mode, p.U, 3, us, ls, Us);
    if (ok && g.has_alpha) {
        const T *af[1] = {p.alpha};
        ok = sample(g, b.sample_mode, af, 1, us, ls, &as);
    }
    if (!ok) {
        atomicAdd(&status[ST_PS_OUTSIDE], 1);
        return 0;
    }
    const C rho = g.has_alpha ? as * (C)g.rho1 + ((C)1 - as) * (C)g.rho2 : (C)g.rho_const;
    C Ur[3], Ut[3], Un[3];
    for (int a = 0; a < 3; ++a) Ur[a] = Us[a] - Pd[a];
    C urt = Ur[0] * t[0] + Ur[1] * t[1] + Ur[2] * t[2];
    for (int a = 0; a < 3; ++a) { Ut[a] = urt * t[a]; Un[a] = Ur[a] - Ut[a]; }
    // line force along the relative flow (sign of Eq. fext_drag)
    const C half = (C)0.5 * rho * (C)b.d[l];
    const C cdn = (C)b.cdn[l], cdt = (C)b.cdt[l];
    if (b.drag_mode == 0) {
        C m = sqrt(Ur[0] * Ur[0] + Ur[1] * Ur[1] + Ur[2] * Ur[2]);
        for (int a = 0; a < 3; ++a) fstar[a] = half * m * (cdn * Un[a] + cdt * Ut[a]);
    } else {
        C mt = sqrt(Ut[0] * Ut[0] + Ut[1] * Ut[1] + Ut[2] * Ut[2]);
        C mn = sqrt(Un[0] * Un[0] + Un[1] * Un[1] + Un[2] * Un[2]);
        for (int a = 0; a < 3; ++a) fstar[a] = half * (cdt * mt * Ut[a] + cdn * mn * Un[a]);
    }
    return 0;
}

// ---------------------------------------------------------------------------
// k_points: Sec. 3.2.2 - 3.2.3, one thread per actuator point
// ---------------------------------------------------------------------------
template <typename T>
__device__ void d_points(const GridC &g, const BeamsC &b, const StepPtrs<T> &p, const Scratch<T> &sc, int *status,
                         const int i) {
    const int has_prev = *sc.hasPrev;
    const int l = b.line_of[i];
    const int off = b.line_off[l], n = b.line_off[l + 1] - off, q = i - off;

    T Pa[3], Pd[3], t[3];
    for (int a = 0; a < 3; ++a) { Pa[a] = p.P[a][i]; Pd[a] = p.Pdot[a][i]; }
    // centreline tangent: Catmull-Rom (central difference), one-sided at the ends
    if (b.tangents_given) {
        for (int a = 0; a < 3; ++a) t[a] = p.tan[a][i];
    } else if (n == 1) {
        t[0] = t[1] = t[2] = (T)0;
    } else {
        const int ip = (q == n - 1) ? i : i + 1, im = (q == 0) ? i : i - 1;
        for (int a = 0; a < 3; ++a) t[a] = p.P[a][ip] - p.P[a][im];
    }
    {
        T nn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        if (nn > (T)0) for (int a = 0; a < 3; ++a) t[a] /= nn;
        else t[0] = t[1] = t[2] = (T)0;
    }

    T fstar[3];
    if (point_fstar<T, T>(g, b, p, l, Pa, Pd, t, fstar, status, sizeof(T) == 4)) {
        // ill-conditioned upstream direction: the same evaluation in FP64
        double Pa64[3], Pd64[3], t64[3], f64[3];
        for (int a = 0; a < 3; ++a) { Pa64[a] = (double)Pa[a]; Pd64[a] = (double)Pd[a]; }
        if (b.tangents_given) {
            for (int a = 0; a < 3; ++a) t64[a] = (double)p.tan[a][i];
        } else if (n == 1) {
            t64[0] = t64[1] = t64[2] = 0.0;
        } else {
            const int ip = (q == n - 1) ? i : i + 1, im = (q == 0) ? i : i - 1;
            for (int a = 0; a < 3; ++a) t64[a] = (double)p.P[a][ip] - (double)p.P[a][im];
        }
        double nn = sqrt(t64[0] * t64[0] + t64[1] * t64[1] + t64[2] * t64[2]);
        if (nn > 0.0) for (int a = 0; a < 3; ++a) t64[a] /= nn;
        else t64[0] = t64[1] = t64[2] = 0.0;
        point_fstar<T, double>(g, b, p, l, Pa64, Pd64, t64, f64, status, false);
        for (int a = 0; a < 3; ++a) fstar[a] = (T)f64[a];
        atomicAdd(&status[ST_REFINED], 1);
    }
    // Eq. almForceRelaxation and the per-CV load
    const T af = (T)b.alpha_f[l];
    const T L = (T)b.cv_len[i];
    const long long np = b.n_points;
    for (int a = 0; a < 3; ++a) {
        T f = has_prev ? af * fstar[a] + ((T)1 - af) * sc.fprev[a * np + i] : fstar[a];
        sc.fprev[a * np + i] = f;
        p.F[a][i] = f * L;
    }
    // projection positions in cell units
    for (int a = 0; a < 3; ++a) {
        T uh;
        float ul;
        to_cell(g, a, p.Ps[a][i], uh, ul);
        sc.uhi[a * np + i] = uh;
        sc.ulo[a * np + i] = ul;
    }
}

// ---------------------------------------------------------------------------
// k_segments: segment vectors and bisectors (projection geometry)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ff_diff(const Scratch<T> &sc, long long np, int a, int kb, int ka) {
    return (sc.uhi[a * np + kb] - sc.uhi[a * np + ka]) + (T)(sc.ulo[a * np + kb] - sc.ulo[a * np + ka]);
}

template <typename T>
__device__ void d_segments(const BeamsC &b, const Scratch<T> &sc, const int k) {
    const long long np = b.n_points;
    const int l = b.line_of[k];
    const int off = b.line_off[l], n = b.line_off[l + 1] - off, q = k - off;
    if (q < n - 1) {
        T D[3];
        for (int a = 0; a < 3; ++a) D[a] = ff_diff(sc, np, a, k + 1, k);
        T L2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
        for (int a = 0; a < 3; ++a) sc.segD[a * np + k] = D[a];
        sc.segIl2[k] = L2 > (T)0 ? (T)1 / L2 : (T)0;
    } else {
        for (int a = 0; a < 3; ++a) sc.segD[a * np + k] = (T)0;
        sc.segIl2[k] = (T)0;
    }
    if (q >= 1 && q <= n - 2) {
        T t0[3], t1[3];
        for (int a = 0; a < 3; ++a) { t0[a] = ff_diff(sc, np, a, k, k - 1); t1[a] = ff_diff(sc, np, a, k + 1, k); }
        T n0 = sqrt(t0[0] * t0[0] + t0[1] * t0[1] + t0[2] * t0[2]);
        T n1 = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
        float tau = 1e30f;
        T m[3] = {(T)0, (T)0, (T)0};
        if (n0 > (T)0 && n1 > (T)0) {
            for (int a = 0; a < 3; ++a) { t0[a] /= n0; t1[a] /= n1; m[a] = t0[a] + t1[a]; }
            T c = t0[0] * t1[0] + t0[1] * t1[1] + t0[2] * t1[2];
            T cx = t0[1] * t1[2] - t0[2] * t1[1], cy = t0[2] * t1[0] - t0[0] * t1[2],
              cz = t0[0] * t1[1] - t0[1] * t1[0];
            T sn = sqrt(cx * cx + cy * cy + cz * cz);
            if ((T)1 + c > (T)1e-3) tau = (float)(sn / ((T)1 + c));   // tan(theta/2)
            T mn = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            if (mn > (T)0) for (int a = 0; a < 3; ++a) m[a] /= mn;
        }
        for (int a = 0; a < 3; ++a) sc.nodeM[a * np + k] = m[a];
        sc.nodeTau[k] = tau;
    } else {
        for (int a = 0; a < 3; ++a) sc.nodeM[a * np + k] = (T)0;
        sc.nodeTau[k] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// k_lines: one warp per line
//
// Regularity certificate.  For a cell C and interior node k let
// sigma_k(C) = (C - P_k) . m_k with m_k the bisector of the two segment
// directions.  When the perpendicular distance rho of C from segment k's
// axis satisfies rho (tan(theta_k/2) + tan(theta_{k+1}/2)) < L_k, the sign
// of sigma_k(C) orders the distances to segments k-1 and k, and the signs
// are monotone along the line; then the closest segment is the last k with
// sigma_k(C) > 0 and a walk finds it.  The line is certified when
//   * every segment has length > 1e-3 cells,
//   * every segment direction makes an angle < ~72 deg with the chord
//     (c_a = min t.a > 0.3), so that segments within 3 eps of a cell lie in
//     one window of arc length <= 2E / c_a,
//   * Dw (tau_k + tau_{k+1}) <= L_k / 2 for every segment, with
//     E = brick diagonal + sqrt(3) R + 2 L_max and Dw = E (1 + 2 / c_a),
//     the largest distance between a cell of a brick and a node the walk
//     can evaluate for it.
// Lines that fail take the exhaustive search instead.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void d_lines(const GridC &g, const BeamsC &b, const Scratch<T> &sc, const StepPtrs<T> &p, int *status,
                        const int l, const int lane) {
    const long long np = b.n_points;
    const int off = b.line_off[l], n = b.line_off[l + 1] - off;
    const double eps = b.eps[l];
    const float Rc = (float)(3.0 * eps / g.h);
    // FP64 sum of F over the line in a fixed order
    double fs[3] = {0.0, 0.0, 0.0};
    for (int q = lane; q < n; q += 32)
        for (int a = 0; a < 3; ++a) fs[a] += (double)p.F[a][off + q];
    for (int o = 16; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) fs[a] += __shfl_down_sync(0xffffffffu, fs[a], o);
    if (lane == 0)
        for (int a = 0; a < 3; ++a) sc.lineF[3 * l + a] = fs[a];

    // certificate
    int ok = (n >= 2);
    float Lmin = 1e30f, Lmax = 0.0f, ca = 1.0f;
    T ax[3] = {(T)0, (T)0, (T)0};
    if (n >= 2) {
        for (int a = 0; a < 3; ++a) ax[a] = ff_diff(sc, np, a, off + n - 1, off);
        T an = sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
        if (an > (T)0) for (int a = 0; a < 3; ++a) ax[a] /= an;
        else ok = 0;
    }
    for (int q = lane; q < n - 1; q += 32) {
        const int k = off + q;
        T D0 = sc.segD[k], D1 = sc.segD[np + k], D2 = sc.segD[2 * np + k];
        float L = (float)sqrt(D0 * D0 + D1 * D1 + D2 * D2);
        Lmin = fminf(Lmin, L);
        Lmax = fmaxf(Lmax, L);
        float c = L > 0.0f ? (float)((D0 * ax[0] + D1 * ax[1] + D2 * ax[2])) / L : -1.0f;
        ca = fminf(ca, c);
    }
    for (int o = 16; o > 0; o >>= 1) {
        Lmin = fminf(Lmin, __shfl_xor_sync(0xffffffffu, Lmin, o));
        Lmax = fmaxf(Lmax, __shfl_xor_sync(0xffffffffu, Lmax, o));
        ca = fminf(ca, __shfl_xor_sync(0xffffffffu, ca, o));
    }
    if (!(Lmin > 1e-3f) || !(ca > 0.3f)) ok = 0;
    if (ok) {
        const float E = BRICK_DIAG + 1.7320508f * Rc + 2.0f * Lmax;
        const float Dw = E * (1.0f + 2.0f / ca);
        int bad = 0;
        for (int q = lane; q < n - 1; q += 32) {
            const int k = off + q;
            float t0 = (q >= 1) ? sc.nodeTau[k] : 0.0f;
            float t1 = (q + 1 <= n - 2) ? sc.nodeTau[k + 1] : 0.0f;
            T D0 = sc.segD[k], D1 = sc.segD[np + k], D2 = sc.segD[2 * np + k];
            float L = (float)sqrt(D0 * D0 + D1 * D1 + D2 * D2);
            if (!(Dw * (t0 + t1) <= 0.5f * L)) bad = 1;
        }
        if (__any_sync(0xffffffffu, bad)) ok = 0;
    }
    if (lane == 0) {
        LineG lg;
        const double ec = eps / g.h;
        lg.Rc = Rc;
        lg.R2c = 9.0 * ec * ec;
        lg.inv_eps2c = 1.0 / (ec * ec);
        lg.eta0 = 1.0 / (PI_D * eps * eps);
        lg.regular = ok;
        lg.first = off;
        lg.n = n;
        sc.lines[l] = lg;
        if (!ok && n > 0) atomicAdd(&status[ST_IRREGULAR], 1);
    }
}

// conservative R-inflated box of segment k (nodes ka, kb) in cell units
template <typename T>
__device__ __forceinline__ void seg_box(const Scratch<T> &sc, long long np, int ka, int kb, float R,
                                        float lo[3], float hi[3]) {
    for (int a = 0; a < 3; ++a) {
        float ua = (float)sc.uhi[a * np + ka], ub = (float)sc.uhi[a * np + kb];
        float slack = R + 0.01f + 1e-5f * (fabsf(ua) + 1.0f);
        lo[a] = fminf(ua, ub) - slack;
        hi[a] = fmaxf(ua, ub) + slack;
    }
}

// ---------------------------------------------------------------------------
// k_mask: every segment marks the bricks its inflated box touches
// ---------------------------------------------------------------------------
template <typename T>
__device__ void d_mask(const GridC &g, const BeamsC &b, const Scratch<T> &sc, const int k) {
    const long long np = b.n_points;
    const int l = b.line_of[k];
    const int off = b.line_off[l], n = b.line_off[l + 1] - off, q = k - off;
    if (n >= 2 && q == n - 1) return;           // no segment starts at the tip
    const int kb = (n == 1) ? k : k + 1;
    float lo[3], hi[3];
    seg_box(sc, np, k, kb, sc.lines[l].Rc, lo, hi);
    // cells whose centre c + 0.5 lies in [lo, hi]
    int c0[3], c1[3];
    const int nn[3] = {g.nx, g.ny, g.nz}, bs[3] = {BX, BY, BZ}, nb[3] = {g.nbx, g.nby, g.nbz};
    for (int a = 0; a < 3; ++a) {
        float fl = ceilf(lo[a] - 0.5f), fh = floorf(hi[a] - 0.5f);
        fl = fmaxf(fl, 0.0f);
        fh = fminf(fh, (float)(nn[a] - 1));
        if (fl > fh) return;
        c0[a] = (int)fl / bs[a];
        c1[a] = min((int)fh / bs[a], nb[a] - 1);
    }
    const uint32_t bit = 1u << (l & 31);
    const int word = l >> 5;
    for (int bz = c0[2]; bz <= c1[2]; ++bz)
        for (int by = c0[1]; by <= c1[1]; ++by)
            for (int bx = c0[0]; bx <= c1[0]; ++bx) {
                long long br = bx + (long long)g.nbx * (by + (long long)g.nby * bz);
                atomicOr(&sc.mask[br * b.mask_words + word], bit);
            }
}

// ---------------------------------------------------------------------------
// FP64 decisions (explicit rounding, no contraction): the paper's closest-
// segment distance evaluated from the caller's original positions.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ double dist2_f64(const GridC &g, const StepPtrs<T> &p, int ka, int kb, int ci, int cj, int ck,
                            double *s_out) {
    const double c[3] = {__dadd_rn(g.o[0], __dmul_rn((double)ci + 0.5, g.h)),
                         __dadd_rn(g.o[1], __dmul_rn((double)cj + 0.5, g.h)),
                         __dadd_rn(g.o[2], __dmul_rn((double)ck + 0.5, g.h))};
    double D[3], q[3];
    for (int a = 0; a < 3; ++a) {
        double A = (double)p.Ps[a][ka], B = (double)p.Ps[a][kb];
        D[a] = __dsub_rn(B, A);
        q[a] = __dsub_rn(c[a], A);
    }
    double L2 = __dadd_rn(__dadd_rn(__dmul_rn(D[0], D[0]), __dmul_rn(D[1], D[1])), __dmul_rn(D[2], D[2]));
    double s = 0.0;
    if (L2 > 0.0) {
        double qd = __dadd_rn(__dadd_rn(__dmul_rn(q[0], D[0]), __dmul_rn(q[1], D[1])), __dmul_rn(q[2], D[2]));
        s = __ddiv_rn(qd, L2);
        s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
    }
    double e[3];
    for (int a = 0; a < 3; ++a) e[a] = __dsub_rn(q[a], __dmul_rn(s, D[a]));
    if (s_out) *s_out = s;
    return __dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])), __dmul_rn(e[2], e[2]));
}
// node index of the far end of segment k of a line (first, n)
__device__ __forceinline__ int seg_end(int k, int n) { return n == 1 ? k : k + 1; }

// d_k < d_{k-1} in FP64 (segment k closer than k-1; ties keep k-1)
template <typename T>
__device__ bool later_closer_f64(const GridC &g, const StepPtrs<T> &p, int k, int ci, int cj, int ck) {
    double d1 = dist2_f64(g, p, k, k + 1, ci, cj, ck, nullptr);
    double d0 = dist2_f64(g, p, k - 1, k, ci, cj, ck, nullptr);
    return sqrt(d1) < sqrt(d0);
}
// r <= 3 eps in FP64 for segment k
template <typename T>
__device__ bool within_f64(const GridC &g, const StepPtrs<T> &p, double eps, int k, int n, int ci, int cj,
                           int ck) {
    double d2 = dist2_f64(g, p, k, seg_end(k, n), ci, cj, ck, nullptr);
    return __dsqrt_rn(d2) <= __dmul_rn(3.0, eps);
}
// argmin over segments [k0, k1] in FP64, lowest index on ties
template <typename T>
__device__ __noinline__ int argmin_f64(const GridC &g, const StepPtrs<T> &p, int k0, int k1, int n, int ci, int cj, int ck) {
    double best = INFINITY;
    int kb = k0;
    for (int k = k0; k <= k1; ++k) {
        double r = __dsqrt_rn(dist2_f64(g, p, k, seg_end(k, n), ci, cj, ck, nullptr));
        if (r < best) { best = r; kb = k; }
    }
    return kb;
}

// ---------------------------------------------------------------------------
// compensated FP32 / plain FP64 accumulator
// ---------------------------------------------------------------------------
template <typename T> struct Acc {
    T s = (T)0, c = (T)0;
    __device__ __forceinline__ void add(T v) {
        T y = v - c;
        T t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ---------------------------------------------------------------------------
// k_weights: Sec. 3.2.4, w_k = sum_j omega_jk eta(r_j) V_j, segment-centric.
// One warp per segment; it visits the cells whose closest segment it is.
// Lanes take columns of the segment's box (regular lines: only the slab
// between the two bisector planes along the march axis) or single cells
// (exhaustive search); lane sums are compensated FP32, combined across the
// warp as float-float pairs and stored as FP64.
// ---------------------------------------------------------------------------
template <typename T>
struct WSeg {
    int k, q, n, off, nseg, kb;
    int O[3], lo[3], hi[3];
    T A[3], Bn[3], D[3], il2;
    T m0[3], m1[3];
    bool has_lo, has_hi;
    T R2, gr, ie2, eta0;
    double eps;
};

// membership of cell cg (local centre C) in segment ctx.k and its weights
template <typename T>
__device__ __forceinline__ void w_cell(const WSeg<T> &c, const T C[3], const int cg[3], const GridC &g,
                                       const Scratch<T> &sc, const StepPtrs<T> &p, bool regular,
                                       int *status, Acc<T> &wa, Acc<T> &wb) {
    const long long np = (long long)p.np;
    T x[3];
    for (int a = 0; a < 3; ++a) x[a] = C[a] - c.A[a];
    if (regular) {
        if (c.has_lo) {
            T sg = x[0] * c.m0[0] + x[1] * c.m0[1] + x[2] * c.m0[2];
            T gs = Tr<T>::gsig(sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
            bool pos;
            if (sg > gs) pos = true;
            else if (sg < -gs) pos = false;
            else { pos = later_closer_f64(g, p, c.k, cg[0], cg[1], cg[2]); atomicAdd(&status[ST_REFINED], 1); }
            if (!pos) return;
        }
        if (c.has_hi) {
            T y[3];
            for (int a = 0; a < 3; ++a) y[a] = C[a] - c.Bn[a];
            T sg = y[0] * c.m1[0] + y[1] * c.m1[1] + y[2] * c.m1[2];
            T gs = Tr<T>::gsig(sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]));
            bool pos;
            if (sg > gs) pos = true;
            else if (sg < -gs) pos = false;
            else { pos = later_closer_f64(g, p, c.k + 1, cg[0], cg[1], cg[2]); atomicAdd(&status[ST_REFINED], 1); }
            if (pos) return;
        }
    } else {
        // exhaustive: closest segment over the whole line, FP64 near ties
        T best = (T)INFINITY, second = (T)INFINITY;
        int jb = 0;
        for (int j = 0; j < c.nseg; ++j) {
            const int ja = c.off + j;
            T xx[3], Dj[3];
            for (int a = 0; a < 3; ++a) {
                xx[a] = C[a] - rel(sc.uhi[a * np + ja], sc.ulo[a * np + ja], c.O[a]);
                Dj[a] = sc.segD[a * np + ja];
            }
            T t = (xx[0] * Dj[0] + xx[1] * Dj[1] + xx[2] * Dj[2]) * sc.segIl2[ja];
            t = t < (T)0 ? (T)0 : (t > (T)1 ? (T)1 : t);
            T e0 = xx[0] - t * Dj[0], e1 = xx[1] - t * Dj[1], e2 = xx[2] - t * Dj[2];
            T r2 = e0 * e0 + e1 * e1 + e2 * e2;
            if (r2 < best) { second = best; best = r2; jb = j; }
            else if (r2 < second) second = r2;
        }
        if (!(second - best > Tr<T>::grr(best))) {
            jb = argmin_f64(g, p, c.off, c.off + c.nseg - 1, c.n, cg[0], cg[1], cg[2]) - c.off;
            atomicAdd(&status[ST_REFINED], 1);
        }
        if (jb != c.q) return;
    }
    T s = (x[0] * c.D[0] + x[1] * c.D[1] + x[2] * c.D[2]) * c.il2;
    s = s < (T)0 ? (T)0 : (s > (T)1 ? (T)1 : s);
    T e0 = x[0] - s * c.D[0], e1 = x[1] - s * c.D[1], e2 = x[2] - s * c.D[2];
    T r2 = e0 * e0 + e1 * e1 + e2 * e2;
    bool in;
    if (r2 < c.R2 - c.gr) in = true;
    else if (r2 > c.R2 + c.gr) in = false;
    else { in = within_f64(g, p, c.eps, c.k, c.n, cg[0], cg[1], cg[2]); atomicAdd(&status[ST_REFINED], 1); }
    if (!in) return;
    T eta = c.eta0 * Tr<T>::ex(-r2 * c.ie2);
    wa.add(((T)1 - s) * eta);
    wb.add(s * eta);
}

// warp sum of compensated lane sums, as float-float (FP32) or plain FP64
__device__ __forceinline__ double warp_total(const Acc<float> &a) {
    float h = a.s, l = -a.c;
    for (int o = 16; o > 0; o >>= 1) {
        float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
        float s, e;
        two_sum(h, oh, s, e);
        e = __fadd_rn(e, __fadd_rn(l, ol));
        fast_two_sum(s, e, h, l);
    }
    return (double)h + (double)l;
}
__device__ __forceinline__ double warp_total(const Acc<double> &a) {
    double v = a.s - a.c;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// the cells of segment c.k's slab, columns along the two axes other than
// the march axis AX (compile-time, so coordinates stay in registers)
template <typename T, int AX>
__device__ __forceinline__ void w_columns(const WSeg<T> &c, const GridC &g, const Scratch<T> &sc,
                                          const StepPtrs<T> &p, int *status, const int lane, Acc<T> &wa,
                                          Acc<T> &wb) {
    constexpr int PA = (AX + 1) % 3, PB = (AX + 2) % 3;
    const int na = c.hi[PA] - c.lo[PA] + 1, nbb = c.hi[PB] - c.lo[PB] + 1;
    const int ncol = na * nbb;
    for (int col = lane; col < ncol; col += 32) {
        const int ia = c.lo[PA] + col % na, ib = c.lo[PB] + col / na;
        T C[3];
        C[PA] = (T)(ia - c.O[PA]) + (T)0.5;
        C[PB] = (T)(ib - c.O[PB]) + (T)0.5;
        // march-axis interval between the two planes (pruning only; the
        // membership test decides)
        T clo = (T)(c.lo[AX] - c.O[AX]) + (T)0.5, chi = (T)(c.hi[AX] - c.O[AX]) + (T)0.5;
        if (c.has_lo && c.m0[AX] != (T)0) {
            T r = c.A[AX] - ((C[PA] - c.A[PA]) * c.m0[PA] + (C[PB] - c.A[PB]) * c.m0[PB]) / c.m0[AX];
            if (c.m0[AX] > (T)0) clo = fmax(clo, r - (T)0.05); else chi = fmin(chi, r + (T)0.05);
        }
        if (c.has_hi && c.m1[AX] != (T)0) {
            T r = c.Bn[AX] - ((C[PA] - c.Bn[PA]) * c.m1[PA] + (C[PB] - c.Bn[PB]) * c.m1[PB]) / c.m1[AX];
            if (c.m1[AX] > (T)0) chi = fmin(chi, r + (T)0.05); else clo = fmax(clo, r - (T)0.05);
        }
        const int i0 = max(c.lo[AX], iceil(clo - (T)0.5) + c.O[AX]);
        const int i1 = min(c.hi[AX], ifloor(chi - (T)0.5) + c.O[AX]);
        for (int ic = i0; ic <= i1; ++ic) {
            C[AX] = (T)(ic - c.O[AX]) + (T)0.5;
            int cg[3];
            cg[AX] = ic; cg[PA] = ia; cg[PB] = ib;
            w_cell(c, C, cg, g, sc, p, true, status, wa, wb);
        }
    }
}

template <typename T>
__device__ void d_weights(const GridC &g, const BeamsC &b, const Scratch<T> &sc, const StepPtrs<T> &p, int *status,
                          const int k, const int lane) {
    const long long np = b.n_points;
    const int l = b.line_of[k];
    const LineG lg = sc.lines[l];
    WSeg<T> c;
    c.k = k; c.off = lg.first; c.n = lg.n; c.q = k - c.off;
    if (c.n >= 2 && c.q == c.n - 1) return;                 // the tip starts no segment
    c.nseg = (c.n == 1) ? 1 : c.n - 1;
    c.kb = seg_end(k, c.n);
    c.eps = b.eps[l];
    for (int a = 0; a < 3; ++a) c.O[a] = ifloor(sc.uhi[a * np + k]);
    for (int a = 0; a < 3; ++a) {
        c.A[a] = rel(sc.uhi[a * np + k], sc.ulo[a * np + k], c.O[a]);
        c.Bn[a] = rel(sc.uhi[a * np + c.kb], sc.ulo[a * np + c.kb], c.O[a]);
        c.D[a] = sc.segD[a * np + k];
    }
    c.il2 = sc.segIl2[k];
    c.R2 = (T)lg.R2c; c.gr = Tr<T>::grr(c.R2); c.ie2 = (T)lg.inv_eps2c; c.eta0 = (T)lg.eta0;
    const int nn[3] = {g.nx, g.ny, g.nz};
    bool empty = false;
    for (int a = 0; a < 3; ++a) {
        T l0 = fmin(c.A[a], c.Bn[a]) - (T)lg.Rc - (T)0.01, h0 = fmax(c.A[a], c.Bn[a]) + (T)lg.Rc + (T)0.01;
        c.lo[a] = max(0, iceil(l0 - (T)0.5) + c.O[a]);
        c.hi[a] = min(nn[a] - 1, ifloor(h0 - (T)0.5) + c.O[a]);
        if (c.lo[a] > c.hi[a]) empty = true;
    }
    Acc<T> wa, wb;
    const bool regular = lg.regular != 0;
    c.has_lo = regular && c.q >= 1;
    c.has_hi = regular && c.q + 1 <= c.n - 2;
    for (int a = 0; a < 3; ++a) {
        c.m0[a] = c.has_lo ? sc.nodeM[a * np + k] : (T)0;
        c.m1[a] = c.has_hi ? sc.nodeM[a * np + k + 1] : (T)0;
    }
    if (!empty && regular) {
        int ax = 0;
        if (fabs(c.D[1]) > fabs(c.D[ax])) ax = 1;
        if (fabs(c.D[2]) > fabs(c.D[ax])) ax = 2;
        if (ax == 0) w_columns<T, 0>(c, g, sc, p, status, lane, wa, wb);
        else if (ax == 1) w_columns<T, 1>(c, g, sc, p, status, lane, wa, wb);
        else w_columns<T, 2>(c, g, sc, p, status, lane, wa, wb);
    } else if (!empty) {
        const int n0 = c.hi[0] - c.lo[0] + 1, n1 = c.hi[1] - c.lo[1] + 1, n2 = c.hi[2] - c.lo[2] + 1;
        const long long ncell = (long long)n0 * n1 * n2;
        for (long long t = lane; t < ncell; t += 32) {
            const int cg[3] = {c.lo[0] + (int)(t % n0), c.lo[1] + (int)((t / n0) % n1), c.lo[2] + (int)(t / ((long long)n0 * n1))};
            T C[3];
            for (int a = 0; a < 3; ++a) C[a] = (T)(cg[a] - c.O[a]) + (T)0.5;
            w_cell(c, C, cg, g, sc, p, false, status, wa, wb);
        }
    }
    const double ta = warp_total(wa), tb = warp_total(wb);
    if (lane == 0) {
        sc.segWa[k] = ta * g.V;
        sc.segWb[k] = tb * g.V;
    }
}

// ---------------------------------------------------------------------------
// k_normalise: w_k and f^_k = F_k / w_k
// ---------------------------------------------------------------------------
template <typename T>
__device__ void d_normalise(const BeamsC &b, const Scratch<T> &sc, const StepPtrs<T> &p, int *status, const int k) {
    const long long np = b.n_points;
    const int l = b.line_of[k];
    const int off = b.line_off[l], n = b.line_off[l + 1] - off, q = k - off;
    double w = 0.0;
    if (n == 1) w = sc.segWa[k] + sc.segWb[k];
    else {
        if (q >= 1) w += sc.segWb[k - 1];
        if (q <= n - 2) w += sc.segWa[k];
    }
    sc.w[k] = w;
    if (w > 0.0) {
        const T wt = (T)w;                         // FP64 sum, divided in the field precision
        for (int a = 0; a < 3; ++a) sc.fhat[a * np + k] = p.F[a][k] / wt;
    } else {
        for (int a = 0; a < 3; ++a) sc.fhat[a * np + k] = (T)0;
        int slot = atomicAdd(sc.zeroCount, 1);
        sc.zeroList[slot] = k;
        atomicAdd(&status[ST_ZERO_WEIGHT], 1);
    }
}

// ---------------------------------------------------------------------------
// k_spread: Eq. almMomentumSource as a cell-centric gather per brick
// ---------------------------------------------------------------------------
template <typename T> struct SpreadCap;
template <> struct SpreadCap<float> { static constexpr int NODES = 768, LIST = 512, ENT = 64; };
template <> struct SpreadCap<double> { static constexpr int NODES = 384, LIST = 512, ENT = 64; };

template <typename T>
struct SpreadSmem {
    static constexpr int NN = SpreadCap<T>::NODES, LIST = SpreadCap<T>::LIST, ENT = SpreadCap<T>::ENT;
    T P[3][NN];                  // node positions relative to the brick origin
    T M[3][NN];                  // node bisectors
    T Fh[3][NN];                 // f^ at the nodes
    T D[3][NN];                  // segment vectors
    T Il2[NN];
    int list[LIST];              // candidate lines of this brick (line order)
    int nlist, nbatch;
    int e_line[ENT], e_jlo[ENT], e_jhi[ENT], e_base[ENT], e_reg[ENT], e_n[ENT], e_first[ENT];
    float e_lo[ENT][3], e_hi[ENT][3];
    T e_R2[ENT], e_gr[ENT], e_ie2[ENT], e_eta0[ENT];
    double red[3][SPREAD_THREADS / 32];
};

// rare paths of the gather, kept out of line so the unrolled cell loop stays small

// FP64 re-decision of "segment k closer than k-1" (walk inside the band)
template <typename T>
__device__ __noinline__ bool nl_later_closer(const GridC &g, const StepPtrs<T> &p, int k, int ci, int cj, int ck,
                                             int *status) {
    atomicAdd(&status[ST_REFINED], 1);
    return later_closer_f64(g, p, k, ci, cj, ck);
}
template <typename T>
__device__ __noinline__ bool nl_within(const GridC &g, const StepPtrs<T> &p, double eps, int k, int n, int ci,
                                       int cj, int ck, int *status) {
    atomicAdd(&status[ST_REFINED], 1);
    return within_f64(g, p, eps, k, n, ci, cj, ck);
}
// closest segment over [first + jlo, first + jhi] by exhaustive search
// (lines without a walk certificate, or longer than the shared-memory stage);
// returns the line-local segment index
template <typename T>
__device__ __noinline__ int nl_exhaustive(const GridC &g, const Scratch<T> &sc, const StepPtrs<T> &p, int first,
                                          int n, int jlo, int jhi, const T C[3], const int B[3], int ci, int cj,
                                          int ck, int *status) {
    const long long np = p.np;
    T best = (T)INFINITY, second = (T)INFINITY;
    int js = jlo;
    for (int jj = jlo; jj <= jhi; ++jj) {
        const int ka = first + jj;
        T x[3], Dj[3];
        for (int a = 0; a < 3; ++a) {
            x[a] = C[a] - rel(sc.uhi[a * np + ka], sc.ulo[a * np + ka], B[a]);
            Dj[a] = sc.segD[a * np + ka];
        }
        T t = (x[0] * Dj[0] + x[1] * Dj[1] + x[2] * Dj[2]) * sc.segIl2[ka];
        t = t < (T)0 ? (T)0 : (t > (T)1 ? (T)1 : t);
        T e0 = x[0] - t * Dj[0], e1 = x[1] - t * Dj[1], e2 = x[2] - t * Dj[2];
        T d2 = e0 * e0 + e1 * e1 + e2 * e2;
        if (d2 < best) { second = best; best = d2; js = jj; }
        else if (d2 < second) second = d2;
    }
    if (!(second - best > Tr<T>::grr(best))) {
        js = argmin_f64(g, p, first + jlo, first + jhi, n, ci, cj, ck) - first;
        atomicAdd(&status[ST_REFINED], 1);
    }
    return js;
}

template <typename T>
__device__ __forceinline__ bool sig_pos(const SpreadSmem<T> &sm, int s, const T C[3], const GridC &g,
                                        const StepPtrs<T> &p, int kglob, int ci, int cj, int ck, int *status) {
    const T x0 = C[0] - sm.P[0][s], x1 = C[1] - sm.P[1][s], x2 = C[2] - sm.P[2][s];
    const T sg = x0 * sm.M[0][s] + x1 * sm.M[1][s] + x2 * sm.M[2][s];
    const T gs = Tr<T>::gsig(sqrt(x0 * x0 + x1 * x1 + x2 * x2));
    if (sg > gs) return true;
    if (sg < -gs) return false;
    return nl_later_closer(g, p, kglob, ci, cj, ck, status);
}

template <typename T>
__device__ void d_spread(const GridC &g, const BeamsC &b, const Scratch<T> &sc, const StepPtrs<T> &p, int *status,
                         const long long br, SpreadSmem<T> &sm) {
    const long long np = b.n_points;
    const int bxi = (int)(br % g.nbx), byi = (int)((br / g.nbx) % g.nby), bzi = (int)(br / ((long long)g.nbx * g.nby));
    const int B0 = bxi * BX, B1 = byi * BY, B2 = bzi * BZ;
    const int Bv[3] = {B0, B1, B2};
    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gx = B0 + tx, gy = B1 + ty;
    const bool col_in = gx < g.nx && gy < g.ny;
    const float cx = tx + 0.5f, cy = ty + 0.5f;

    T acc[BZ][3];
#pragma unroll
    for (int z = 0; z < BZ; ++z) acc[z][0] = acc[z][1] = acc[z][2] = (T)0;
    int nsupp = 0;                                   // (cell, line) pairs within 3 eps

    const int W = b.mask_words;
    uint32_t *mrow = sc.mask + br * (long long)W;
    const float blo[3] = {(float)B0, (float)B1, (float)B2};
    const float bhi[3] = {(float)(B0 + BX), (float)(B1 + BY), (float)(B2 + BZ)};

    constexpr int CH = SpreadSmem<T>::LIST / 32;               // mask words per chunk
    for (int w0 = 0; w0 < W; w0 += CH) {
        // ---- candidate lines from CH mask words, in line order -------------
        __syncthreads();
        if (warp == 0) {
            const bool mine = lane < CH && w0 + lane < W;
            uint32_t m = mine ? mrow[w0 + lane] : 0u;
            if (mine && m) mrow[w0 + lane] = 0u;                 // clear for the next step
            int cnt = __popc(m), pre = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                int v = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre += v;
            }
            int total = __shfl_sync(0xffffffffu, pre, 31);
            int pos = pre - cnt;
            while (m) {
                int bit = __ffs(m) - 1;
                m &= m - 1;
                sm.list[pos++] = ((w0 + lane) << 5) + bit;
            }
            if (lane == 0) sm.nlist = total;                      // <= 32 * CH = LIST
        }
        __syncthreads();
        const int nlist = sm.nlist;
        int li = 0;
        while (li < nlist) {
            // ---- batch: candidate segment ranges, one warp per line --------
            const int nb = min(nlist - li, SpreadSmem<T>::ENT);
            for (int e = warp; e < nb; e += SPREAD_THREADS / 32) {
                const int l = sm.list[li + e];
                const LineG lg = sc.lines[l];
                const int nseg = lg.n == 1 ? 1 : lg.n - 1;
                int jlo = 0x7fffffff, jhi = -1;
                float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
                for (int j = lane; j < nseg; j += 32) {
                    const int ka = lg.first + j;
                    float sl[3], sh[3];
                    seg_box(sc, np, ka, seg_end(ka, lg.n), lg.Rc, sl, sh);
                    bool ov = true;
                    for (int a = 0; a < 3; ++a) ov = ov && (sh[a] >= blo[a] && sl[a] <= bhi[a]);
                    if (ov) {
                        jlo = min(jlo, j);
                        jhi = max(jhi, j);
                        for (int a = 0; a < 3; ++a) { lo[a] = fminf(lo[a], sl[a]); hi[a] = fmaxf(hi[a], sh[a]); }
                    }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    jlo = min(jlo, __shfl_xor_sync(0xffffffffu, jlo, o));
                    jhi = max(jhi, __shfl_xor_sync(0xffffffffu, jhi, o));
                    for (int a = 0; a < 3; ++a) {
                        lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
                        hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
                    }
                }
                if (lane == 0) {
                    sm.e_line[e] = l;
                    sm.e_jlo[e] = jlo;
                    sm.e_jhi[e] = jhi;
                    sm.e_reg[e] = lg.regular;
                    sm.e_n[e] = lg.n;
                    sm.e_first[e] = lg.first;
                    sm.e_R2[e] = (T)lg.R2c;
                    sm.e_gr[e] = Tr<T>::grr((T)lg.R2c);
                    sm.e_ie2[e] = (T)lg.inv_eps2c;
                    sm.e_eta0[e] = (T)lg.eta0;
                    for (int a = 0; a < 3; ++a) { sm.e_lo[e][a] = lo[a] - blo[a]; sm.e_hi[e][a] = hi[a] - blo[a]; }
                }
            }
            __syncthreads();
            // node budget: entries [li, li + ne) fit in shared memory
            if (threadIdx.x == 0) {
                int base = 0, e = 0;
                for (; e < nb; ++e) {
                    int cnt = sm.e_jhi[e] >= sm.e_jlo[e] ? sm.e_jhi[e] - sm.e_jlo[e] + 2 : 0;
                    if (base + cnt > SpreadSmem<T>::NN) break;
                    sm.e_base[e] = base;
                    base += cnt;
                }
                if (e == 0) { e = 1; sm.e_base[0] = -1; }  // one oversized line: global-memory path
                sm.nbatch = e;
            }
            __syncthreads();
            const int ne = sm.nbatch;
            // ---- stage nodes of the batch ----------------------------------
            for (int e = 0; e < ne; ++e) {
                const int jlo = sm.e_jlo[e], jhi = sm.e_jhi[e], base = sm.e_base[e];
                if (jhi < jlo || base < 0) continue;
                const int first = sm.e_first[e], n = sm.e_n[e];
                const int cnt = jhi - jlo + 2;
                for (int t = threadIdx.x; t < cnt; t += SPREAD_THREADS) {
                    const int k = first + jlo + t;
                    const int kn = (n == 1) ? first : k;    // single-node line: copy the node
                    const int s = base + t;
                    for (int a = 0; a < 3; ++a) {
                        sm.P[a][s] = rel(sc.uhi[a * np + kn], sc.ulo[a * np + kn], Bv[a]);
                        sm.M[a][s] = sc.nodeM[a * np + kn];
                        sm.Fh[a][s] = sc.fhat[a * np + kn];
                        sm.D[a][s] = sc.segD[a * np + kn];
                    }
                    sm.Il2[s] = sc.segIl2[kn];
                }
            }
            __syncthreads();
            // ---- gather: every thread walks only the lines near its column ----
            if (col_in) {
                uint64_t cm = 0;
                for (int e = 0; e < ne; ++e)
                    if (sm.e_jhi[e] >= sm.e_jlo[e] && cx >= sm.e_lo[e][0] && cx <= sm.e_hi[e][0] &&
                        cy >= sm.e_lo[e][1] && cy <= sm.e_hi[e][1])
                        cm |= 1ull << e;
                while (cm) {                                     // increasing e = line order
                    const int e = __ffsll((long long)cm) - 1;
                    cm &= cm - 1;
                    const int jlo = sm.e_jlo[e], jhi = sm.e_jhi[e], base = sm.e_base[e];
                    const int first = sm.e_first[e], n = sm.e_n[e], reg = sm.e_reg[e];
                    const T R2 = sm.e_R2[e], gr = sm.e_gr[e], ie2 = sm.e_ie2[e], eta0 = sm.e_eta0[e];
                    const float zlo = sm.e_lo[e][2], zhi = sm.e_hi[e][2];
                    int j = jlo;                                  // walk state (line-local segment)
#pragma unroll
                    for (int z = 0; z < BZ; ++z) {
                        const float cz = z + 0.5f;
                        if (cz < zlo || cz > zhi) continue;
                        const int gz = B2 + z;
                        if (gz >= g.nz) continue;
                        const T C[3] = {(T)cx, (T)cy, (T)cz};
                        int js;
                        if (reg && base >= 0) {
                            while (j > jlo && !sig_pos(sm, base + (j - jlo), C, g, p, first + j, gx, gy, gz, status)) --j;
                            while (j < jhi && sig_pos(sm, base + (j + 1 - jlo), C, g, p, first + j + 1, gx, gy, gz, status)) ++j;
                            js = j;
                        } else {
                            js = nl_exhaustive(g, sc, p, first, n, jlo, jhi, C, Bv, gx, gy, gz, status);
                        }
                        T s, r2, fa[3], fb[3];
                        if (base >= 0) {
                            const int ss = base + (js - jlo), sb = (n == 1) ? ss : ss + 1;
                            const T x0 = C[0] - sm.P[0][ss], x1 = C[1] - sm.P[1][ss], x2 = C[2] - sm.P[2][ss];
                            const T d0 = sm.D[0][ss], d1 = sm.D[1][ss], d2 = sm.D[2][ss];
                            s = (x0 * d0 + x1 * d1 + x2 * d2) * sm.Il2[ss];
                            s = s < (T)0 ? (T)0 : (s > (T)1 ? (T)1 : s);
                            const T e0 = x0 - s * d0, e1 = x1 - s * d1, e2 = x2 - s * d2;
                            r2 = e0 * e0 + e1 * e1 + e2 * e2;
                            for (int a = 0; a < 3; ++a) { fa[a] = sm.Fh[a][ss]; fb[a] = sm.Fh[a][sb]; }
                        } else {
                            const int ka = first + js, kb = seg_end(ka, n);
                            T x[3], Dj[3];
                            for (int a = 0; a < 3; ++a) {
                                x[a] = C[a] - rel(sc.uhi[a * np + ka], sc.ulo[a * np + ka], Bv[a]);
                                Dj[a] = sc.segD[a * np + ka];
                                fa[a] = sc.fhat[a * np + ka];
                                fb[a] = sc.fhat[a * np + kb];
                            }
                            s = (x[0] * Dj[0] + x[1] * Dj[1] + x[2] * Dj[2]) * sc.segIl2[ka];
                            s = s < (T)0 ? (T)0 : (s > (T)1 ? (T)1 : s);
                            const T e0 = x[0] - s * Dj[0], e1 = x[1] - s * Dj[1], e2 = x[2] - s * Dj[2];
                            r2 = e0 * e0 + e1 * e1 + e2 * e2;
                        }
                        bool in;
                        if (r2 < R2 - gr) in = true;
                        else if (r2 > R2 + gr) in = false;
                        else in = nl_within(g, p, b.eps[sm.e_line[e]], first + js, n, gx, gy, gz, status);
                        if (!in) continue;
                        ++nsupp;
                        const T eta = eta0 * Tr<T>::ex(-r2 * ie2);
                        const T wa = eta * ((T)1 - s), wb = eta * s;
                        acc[z][0] -= wa * fa[0] + wb * fb[0];
                        acc[z][1] -= wa * fa[1] + wb * fb[1];
                        acc[z][2] -= wa * fa[2] + wb * fb[2];
                    }
                }
            }
            li += ne;
            __syncthreads();
        }
    }
    // ---- write every cell of the brick once; brick sums of S ----------------
    T cs[3] = {(T)0, (T)0, (T)0};
    if (col_in) {
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            const int gz = B2 + z;
            if (gz < g.nz) {
                const long long idx = gx + (long long)g.nx * (gy + (long long)g.ny * gz);
                p.S[0][idx] = acc[z][0];
                p.S[1][idx] = acc[z][1];
                p.S[2][idx] = acc[z][2];
                cs[0] += acc[z][0]; cs[1] += acc[z][1]; cs[2] += acc[z][2];
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        for (int a = 0; a < 3; ++a) cs[a] += __shfl_down_sync(0xffffffffu, cs[a], o);
        nsupp += __shfl_down_sync(0xffffffffu, nsupp, o);
    }
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) sm.red[a][warp] = (double)cs[a];
        if (nsupp) atomicAdd(&status[ST_SUPPORT], nsupp);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) {
            double t = 0.0;
            for (int w = 0; w < SPREAD_THREADS / 32; ++w) t += sm.red[a][w];
            sc.brickSum[a * g.nbrick + br] = t;
        }
    }
}

// ---------------------------------------------------------------------------
// k_deposit: nodes with w_k = 0 put F_k into the cell that contains them
// (single thread, fixed order -> deterministic)
// ---------------------------------------------------------------------------
template <typename T>
__device__ void d_deposit(const GridC &g, const BeamsC &b, const Scratch<T> &sc, const StepPtrs<T> &p, int *status) {
    const int cnt = *sc.zeroCount;
    if (cnt == 0) return;
    const long long np = b.n_points;
    for (int i = 1; i < cnt; ++i) {             // insertion sort by node index
        int v = sc.zeroList[i], j = i - 1;
        while (j >= 0 && sc.zeroList[j] > v) { sc.zeroList[j + 1] = sc.zeroList[j]; --j; }
        sc.zeroList[j + 1] = v;
    }
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int i = 0; i < cnt; ++i) {
        const int k = sc.zeroList[i];
        int c[3];
        bool ins = true;
        for (int a = 0; a < 3; ++a) {
            T uh = sc.uhi[a * np + k];
            float ul = sc.ulo[a * np + k];
            if (!inside_axis(uh, ul, nn[a])) ins = false;
            c[a] = min(max(ffloor(uh, ul), 0), nn[a] - 1);
        }
        if (!ins) { atomicAdd(&status[ST_DEPOSIT_LOST], 1); continue; }
        const long long idx = c[0] + (long long)g.nx * (c[1] + (long long)g.ny * c[2]);
        for (int a = 0; a < 3; ++a) {
            T dv = p.F[a][k] / (T)g.V;
            p.S[a][idx] -= dv;
            sc.depSum[a] -= (double)dv;
        }
    }
}

// ---------------------------------------------------------------------------
// k_totals: FP64 sum F and sum S V, fixed reduction order
// ---------------------------------------------------------------------------
template <typename T>
__device__ void d_totals(const GridC &g, const BeamsC &b, const Scratch<T> &sc, double *totals, double (*red)[256]) {
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int l = threadIdx.x; l < b.n_lines; l += 256)
        for (int a = 0; a < 3; ++a) v[a] += sc.lineF[3 * l + a];
    for (long long r = threadIdx.x; r < g.nbrick; r += 256)
        for (int a = 0; a < 3; ++a) v[3 + a] += sc.brickSum[a * g.nbrick + r];
    for (int a = 0; a < 6; ++a) red[a][threadIdx.x] = v[a];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int a = 0; a < 6; ++a) red[a][threadIdx.x] += red[a][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) totals[a] = red[a][0];
        for (int a = 0; a < 3; ++a) totals[3 + a] = red[3 + a][0] * g.V + sc.depSum[a] * g.V;
        *sc.hasPrev = 1;                 // the next step relaxes against this one
    }
}


// ---------------------------------------------------------------------------
// Launchers.  Single instance: one launch per phase.  Batched: one launch per
// phase over the work items of every instance of a batch; each work item is
// mapped to its instance by a binary search over the prefix sums of the
// per-instance item counts (a device work list), so uneven instances share
// one grid and one CUDA graph.
// ---------------------------------------------------------------------------
template <typename T>
struct Inst {
    GridC g;
    BeamsC b;
    Scratch<T> sc;
    StepPtrs<T> p;
    int *status;
    double *totals;
};

// index of the instance owning global item `gid` (pre[i] <= gid < pre[i+1])
__device__ __forceinline__ int owner(const long long *pre, int n, long long gid) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= gid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) k_points(GridC g, BeamsC b, StepPtrs<T> p, Scratch<T> sc, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < b.n_points) d_points(g, b, p, sc, status, i);
}
template <typename T>
__global__ void __launch_bounds__(256) k_segments(BeamsC b, Scratch<T> sc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < b.n_points) d_segments(b, sc, k);
}
template <typename T>
__global__ void __launch_bounds__(256) k_lines(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p, int *status) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w < b.n_lines) d_lines(g, b, sc, p, status, w, threadIdx.x & 31);
}
template <typename T>
__global__ void __launch_bounds__(256) k_mask(GridC g, BeamsC b, Scratch<T> sc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < b.n_points) d_mask(g, b, sc, k);
}
template <typename T>
__global__ void __launch_bounds__(128) k_weights(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p, int *status) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k < b.n_points) d_weights(g, b, sc, p, status, k, threadIdx.x & 31);
}
template <typename T>
__global__ void __launch_bounds__(256) k_normalise(BeamsC b, Scratch<T> sc, StepPtrs<T> p, int *status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < b.n_points) d_normalise(b, sc, p, status, k);
}
template <typename T>
__global__ void __launch_bounds__(SPREAD_THREADS) k_spread(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p,
                                                           int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<T> &sm = *reinterpret_cast<SpreadSmem<T> *>(smem_raw);
    d_spread(g, b, sc, p, status, (long long)blockIdx.x, sm);
}
template <typename T>
__global__ void k_deposit(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p, int *status) {
    if (threadIdx.x == 0 && blockIdx.x == 0) d_deposit(g, b, sc, p, status);
}
template <typename T>
__global__ void __launch_bounds__(256) k_totals(GridC g, BeamsC b, Scratch<T> sc, double *totals) {
    __shared__ double red[6][256];
    d_totals(g, b, sc, totals, red);
}

// ---- batched -------------------------------------------------------------
// pre: prefix sums of the per-instance item counts (n + 1 entries) of the n
// selected instances; sel: instance index of each selected slot (NULL: slot q
// is instance q)
#define AL_SEL(q) (sel ? sel[q] : (q))
template <typename T>
__global__ void __launch_bounds__(256) kb_points(const Inst<T> *I, const int *sel, const long long *pre, int n) {
    const long long total = pre[n];
    for (long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
         gid += (long long)gridDim.x * blockDim.x) {
        const int q = owner(pre, n, gid);
        const Inst<T> &x = I[AL_SEL(q)];
        d_points(x.g, x.b, x.p, x.sc, x.status, (int)(gid - pre[q]));
    }
}
template <typename T>
__global__ void __launch_bounds__(256) kb_segments(const Inst<T> *I, const int *sel, const long long *pre, int n) {
    const long long total = pre[n];
    for (long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
         gid += (long long)gridDim.x * blockDim.x) {
        const int q = owner(pre, n, gid);
        const Inst<T> &x = I[AL_SEL(q)];
        d_segments(x.b, x.sc, (int)(gid - pre[q]));
    }
}
template <typename T>
__global__ void __launch_bounds__(256) kb_lines(const Inst<T> *I, const int *sel, const long long *pre, int n) {
    const long long total = pre[n];
    const long long nw = (long long)gridDim.x * blockDim.x / 32;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
        const int q = owner(pre, n, w);
        const Inst<T> &x = I[AL_SEL(q)];
        d_lines(x.g, x.b, x.sc, x.p, x.status, (int)(w - pre[q]), threadIdx.x & 31);
    }
}
template <typename T>
__global__ void __launch_bounds__(256) kb_mask(const Inst<T> *I, const int *sel, const long long *pre, int n) {
    const long long total = pre[n];
    for (long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
         gid += (long long)gridDim.x * blockDim.x) {
        const int q = owner(pre, n, gid);
        const Inst<T> &x = I[AL_SEL(q)];
        d_mask(x.g, x.b, x.sc, (int)(gid - pre[q]));
    }
}
template <typename T>
__global__ void __launch_bounds__(128) kb_weights(const Inst<T> *I, const int *sel, const long long *pre, int n) {
    const long long total = pre[n];
    const long long nw = (long long)gridDim.x * blockDim.x / 32;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
        const int q = owner(pre, n, w);
        const Inst<T> &x = I[AL_SEL(q)];
        d_weights(x.g, x.b, x.sc, x.p, x.status, (int)(w - pre[q]), threadIdx.x & 31);
    }
}
template <typename T>
__global__ void __launch_bounds__(256) kb_normalise(const Inst<T> *I, const int *sel, const long long *pre, int n) {
    const long long total = pre[n];
    for (long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
         gid += (long long)gridDim.x * blockDim.x) {
        const int q = owner(pre, n, gid);
        const Inst<T> &x = I[AL_SEL(q)];
        d_normalise(x.b, x.sc, x.p, x.status, (int)(gid - pre[q]));
    }
}
// persistent: a fixed grid of CTAs walks the bricks of every instance
template <typename T>
__global__ void __launch_bounds__(SPREAD_THREADS) kb_spread(const Inst<T> *I, const int *sel, const long long *pre, int n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<T> &sm = *reinterpret_cast<SpreadSmem<T> *>(smem_raw);
    const long long total = pre[n];
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        const int q = owner(pre, n, item);
        const Inst<T> &x = I[AL_SEL(q)];
        d_spread(x.g, x.b, x.sc, x.p, x.status, item - pre[q], sm);
        __syncthreads();
    }
}
template <typename T>
__global__ void kb_deposit(const Inst<T> *I, const int *sel, int n) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) {
        const Inst<T> &x = I[AL_SEL(q)];
        if (x.b.n_points > 0) d_deposit(x.g, x.b, x.sc, x.p, x.status);
    }
}
template <typename T>
__global__ void __launch_bounds__(256) kb_totals(const Inst<T> *I, const int *sel, int n) {
    __shared__ double red[6][256];
    for (int q = blockIdx.x; q < n; q += gridDim.x) {
        const Inst<T> &x = I[AL_SEL(q)];
        d_totals(x.g, x.b, x.sc, x.totals, red);
        __syncthreads();
    }
}
template <typename T>
__global__ void kb_reset(const Inst<T> *I, const int *sel, int n) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) {
        const Inst<T> &x = I[AL_SEL(q)];
        *x.sc.zeroCount = 0;
        x.sc.depSum[0] = x.sc.depSum[1] = x.sc.depSum[2] = 0.0;
    }
}
#undef AL_SEL

}  // namespace al
