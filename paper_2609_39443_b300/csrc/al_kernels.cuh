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
//               segment it is (Sec. 3.2.4, w_k), FP32 compensated sums;
//               records every such (cell, segment) pair in its brick's
//               region of the record arena
//   k_bweights  per brick: the same sums for lines without a walk
//               certificate (or all lines), exact fixed-point integers
//   k_normalise per node: w_k, f^_k = F_k / w_k, and a bound on one source
//   k_spread    per brick of 16 x 16 x h cells: Eq. almMomentumSource, the
//               recorded pairs replayed and the other lines gathered, each
//               cell's sources summed as fixed-point integers in shared
//               memory, then every cell of S written exactly once; the
//               zero-weight nodes (w_k = 0) deposit their load in their cell
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
#include <type_traits>

namespace al {

constexpr int BX = 16, BY = 16;                  // projection brick footprint (cells)
constexpr int BZ_MIN = 4, BZ_MAX = 16;           // brick heights the kernels are built for
constexpr int SPREAD_THREADS = BX * BY;          // one thread per column
constexpr float BRICK_DIAG = 27.72f;             // diagonal of the tallest brick, 16 x 16 x 16
constexpr int CM_NN = 640;
constexpr int CM_LN = 256;                        // column march: nodes of a line staged per warp in k_lines                       // column march: nodes staged per batch of lines
constexpr double PI_D = 3.14159265358979323846;

// Programmatic dependent launch, first statement of every kernel of a step:
// wait until the stream's previous kernel has completed and
// its writes are visible.  Launched with the attribute, the kernel is set up
// while its predecessor runs and starts as that one ends; launched without
// it, the wait returns at once (stream order has already waited), so each
// kernel sees what it saw with plain stream order.  No kernel triggers its
// dependents early: dependents resident before their predecessor ended
// slowed the latency-bound point pass.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

enum { ST_PA_OUTSIDE = 0, ST_PS_OUTSIDE = 1, ST_FALLBACK = 2, ST_FALLBACK_ZERO = 3,
       ST_ZERO_WEIGHT = 4, ST_DEPOSIT_LOST = 5, ST_REFINED = 6, ST_IRREGULAR = 7, ST_SUPPORT = 8,
       ST_REPLAYED = 9, ST_COLUMN = 10, ST_GUARD = 15 };

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
    int wmode;                   // 0: all weights from the brick pass; 1: segment pass for certified lines
    int bz;                      // brick height of the projection (4, 8 or 16 cells)
    int smode;                   // 0: gather (every line); 1: scatter with atomics for certified lines
    int rmode;                   // 1: the segment pass records its (cell, segment) pairs, the spread replays them
    int fx;                      // 1: the spread sums fixed-point integers (replay, integrated projection)
    long long rec_total;         // capacity of the record arena (records)
    long long nbrick_max;        // bricks at the lowest brick height (size of the per-brick arrays)
    int cm;                      // 1: bricks whose lines all take the column march use the column-march passes
    int own_bx0, own_bx1;        // brick columns along x whose cells this instance owns (a slab of a
                                 // decomposition along x): the weights and spread passes work on them only
};

// the brick's cells are owned (the weights and spread passes visit it)
__device__ __forceinline__ bool brick_owned(const GridC &g, long long br) {
    const int bx = (int)(br % g.nbx);
    return bx >= g.own_bx0 && bx < g.own_bx1;
}

// one (cell, segment) pair of a certified line inside the 3 eps support, as
// the segment pass found it: the cell within its brick (z * 256 + y * 16 + x),
// the segment's start node (REC_SINGLE: a one-node line, both ends the same
// node) and the node weights omega eta of the two ends
template <typename T> struct Rec { int cell; int ka; T wa, wb; };
constexpr int REC_SINGLE = 1 << 30;

struct BeamsC {
    int n_lines, n_points, mask_words;
    const int *line_off, *line_of;
    const double *d, *cdn, *cdt, *eps, *ell_s, *alpha_f, *cv_len;
    double n_p[3], g_up[3], tau;
    int sample_mode, drag_mode, tangents_given;
    const double *cm_n, *cm_t;   // added-mass coefficients (inertia != 0)
    int inertia;
    int proj_mode;               // 0 nearest segment, 1 segment-integrated 3-D Gaussian
    int reflect;                 // faces that reflect the kernel: bit 2a (2a + 1) low (high) face of axis a
};

struct LineG {                   // per line, rebuilt every step
    float Rc;                    // 3 eps in cell units (box slack only)
    double R2c, inv_eps2c;       // (3 eps)^2, 1/eps^2 in cell units
    double inv_eps2c_l2;         // log2(e) / eps^2 in cell units (Gaussian as a power of 2)
    double eta0;                 // 1 / (pi eps^2) in 1/m^2
    int regular;                 // 0: exhaustive search; 1: walk from any candidate; 2: walk from near the foot
    int first, n;
    float thmax;                 // largest turning angle at a node (rad)
    float Lmin, Lmax;            // shortest / longest segment (cells)
    float rho2;                  // regular == 2: a walk may start at a node within sqrt(rho2) cells
    int wshift;                  // fixed-point weights: omega eta / eta0 in units of 2^-wshift
    float R2f, ie2f, eta0f;      // FP32 copies of R2c, inv_eps2c_l2, eta0 (no conversions in the hot loops)
    int cm;                      // the line climbs (D_z / |D| >= 0.8 on every segment) and carries the
                                 // column-march certificate (FP32 instances)
};

// per-line constant in the field precision, without an FP64 conversion for FP32
template <typename T> __device__ __forceinline__ T lgc(double d, float f);
template <> __device__ __forceinline__ float lgc<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double lgc<double>(double d, float) { return d; }

struct CmEnt;                    // column march: one candidate line of a brick (al_cm.cuh)
struct CmLay;                    // column march: one brick layer of a line (al_cm.cuh)

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
    unsigned long long *wfix;    // [np] w_k / (eta0 V) in units of 2^-wshift (brick weights pass)
    double *w;                   // [np] w_k
    T *fhat;                     // [3][np] normalised nodal force
    double *lineF;               // [3][n_lines] sum of F per line
    LineG *lines;                // [n_lines]
    uint32_t *mask;              // [nbrick][mask_words] lines touching a brick
    double *brickSum;            // [3][nbrick] sum of S per brick
    double *scatSum;             // [3] sum of S added by the scatter form
    double *totPart;             // [TOT_PARTS][6] partial sums of the totals
    int *totDone;                // [1] parts of the totals done this step (the last part adds them)
    int *hasPrev;                // [1] a previous relaxed force exists (set by k_totals)
    int *anyIrr;                 // [1] some line has no walk certificate (set by k_lines)
    unsigned int *smax;          // [1] bound on one spread contribution (float bits, set by k_normalise)
    int *anyZero;                // [1] some node has w_k = 0 (set by k_normalise)
    Rec<T> *rec;                 // [rec_total] pair records, a region per brick
    int *rcnt;                   // [nbrick_max] records found this step per brick
    int *rcap;                   // [nbrick_max] capacity of the brick's region this step
    long long *roff;             // [nbrick_max] start of the brick's region
    int *rplan;                  // [2] brick height the regions of this step / of the next step were sized for
    unsigned long long *rused;   // [1] arena taken by the next step's regions
    int *cmcnt;                  // [5] bricks of this step on the column-march (with candidate lines) /
                                 // the brick passes; the next column-march brick of the spread / entry of
                                 // the weights pass; column-march bricks without candidate lines
    int *cmlist;                 // [2][nbrick_max] those bricks
    float4 *cmN;                 // [np][4] node records of the column march (NULL: not used)
    CmLay *cmlay;                // [n_lines][(nz + 3) / 4] per line and brick layer: what its entries share
    CmEnt *cment;                // [cment_cap] entries of the column-march bricks
    int *cment_n;                // [1] entries taken this step
    long long cment_cap;
    int *bent_off, *bent_n;      // [nbrick_max] a column-march brick's entries
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
    const T *Uprev[3];           // inertia: fluid velocity dt earlier (NULL: no fluid acceleration)
    const T *Pdd[3];             // inertia: actuator-point accelerations (NULL: none)
    double dt;
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
    // 2^y with the SFU's ex2 instruction (relative error below 2^-22 over the
    // arguments used here, y in [-13, 0]); the Gaussian is evaluated as
    // exp(-(r/eps)^2) = 2^(-(r/eps)^2 log2 e)
    static __device__ __forceinline__ float ex2(float y) {
        float r;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
        return r;
    }
};
template <> struct Tr<double> {
    static __device__ __forceinline__ double gsig(double x) { return 1e-12 * (x + 8.0); }
    static __device__ __forceinline__ double grr(double R2) { return 1e-12 * R2 + 1e-12; }
    static __device__ __forceinline__ double ex2(double y) { return exp2(y); }
};

// precision-dispatched math: float arguments always take the float
// instructions (a double overload would route through the FP64 pipe)
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float tabs(float a) { return fabsf(a); }
__device__ __forceinline__ double tabs(double a) { return fabs(a); }
__device__ __forceinline__ float tfloor(float a) { return floorf(a); }
__device__ __forceinline__ double tfloor(double a) { return floor(a); }

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

// explicitly rounded arithmetic (no contraction or reordering by the
// compiler): the segment pass and the brick gather compute the same
// per-pair values and must agree bit for bit
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

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
    T f = tfloor(uh);
    int c = (int)f;
    if (f == uh && ul < 0.0f) c -= 1;
    return c;
}

// floor / ceil of |x| < 2^22 as floats, by rounding with the 1.5 * 2^23
// shift (no conversion instruction)
__device__ __forceinline__ float ffloor_f(float x) {
    float r = __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
    return r > x ? r - 1.0f : r;
}
__device__ __forceinline__ float fceil_f(float x) {
    float r = __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
    return r < x ? r + 1.0f : r;
}
__device__ __forceinline__ double ffloor_f(double x) { return floor(x); }
__device__ __forceinline__ double fceil_f(double x) { return ceil(x); }

// floor / ceil in the arithmetic type (no FP64 for FP32 instances)
__device__ __forceinline__ int ifloor(float x) { return (int)floorf(x); }
__device__ __forceinline__ int ifloor(double x) { return (int)floor(x); }
__device__ __forceinline__ int iceil(float x) { return (int)ceilf(x); }
__device__ __forceinline__ int iceil(double x) { return (int)ceil(x); }

// v * 2^sh for 0 <= v <= 1, truncated, from the bits of v (integer
// operations only).  Integer sums of these are exact and independent of the
// order of the additions, so atomics keep the weights deterministic.  The
// per-line shift keeps every node's sum below 2^63.
__device__ __forceinline__ unsigned long long to_fixed(float v, int sh) {
    const unsigned int bits = __float_as_uint(v);
    const int e = (int)((bits >> 23) & 0xffu);
    if (e == 0 || (bits >> 31)) return 0ull;               // zero, subnormal or negative
    const unsigned long long m = (unsigned long long)((bits & 0x7fffffu) | 0x800000u);
    const int s = e - 150 + sh;                            // v 2^sh = m 2^(e - 150 + sh)
    if (s >= 0) return m << s;
    if (s <= -24) return 0ull;
    return m >> (-s);
}
__device__ __forceinline__ unsigned long long to_fixed(double v, int sh) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7ffull);
    if (e == 0 || (bits >> 63)) return 0ull;
    const unsigned long long m = (bits & 0xfffffffffffffull) | 0x10000000000000ull;
    const int s = e - 1075 + sh;
    if (s >= 0) return m << s;
    if (s <= -53) return 0ull;
    return m >> (-s);
}

// Signed v 2^sh truncated toward zero (odd in v), from the bits of v: the
// momentum source of a brick is summed as such integers, exactly and in any
// order, so every path that produces the same contributions produces the
// same S.  The caller keeps |v| 2^sh below 2^61.
__device__ __forceinline__ long long to_fixed_s(float v, int sh) {
    const unsigned int bits = __float_as_uint(v);
    const int e = (int)((bits >> 23) & 0xffu);
    if (e == 0) return 0ll;                                // zero or subnormal
    const long long m = (long long)((bits & 0x7fffffu) | 0x800000u);
    const int s = e - 150 + sh;
    const long long r = s >= 0 ? (m << s) : (s <= -24 ? 0ll : (m >> (-s)));
    return (bits >> 31) ? -r : r;
}
__device__ __forceinline__ long long to_fixed_s(double v, int sh) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7ffull);
    if (e == 0) return 0ll;
    const long long m = (long long)((bits & 0xfffffffffffffull) | 0x10000000000000ull);
    const int s = e - 1075 + sh;
    const long long r = s >= 0 ? (m << s) : (s <= -53 ? 0ll : (m >> (-s)));
    return (bits >> 63) ? -r : r;
}
// the fixed-point sum back in the field precision (one rounding)
__device__ __forceinline__ void from_fixed(long long a, int sh, float &v) { v = ldexpf(__ll2float_rn(a), -sh); }
__device__ __forceinline__ void from_fixed(long long a, int sh, double &v) { v = ldexp(__ll2double_rn(a), -sh); }
// shift of the spread's fixed point: M bounds every single contribution
// (|eta f^| or a deposit |F / V|) and a cell receives at most one per line
// plus one per deposited node, so |sum| 2^sh < 2^61
__device__ __forceinline__ int spread_shift(unsigned int mbits, long long ncontrib) {
    const float M = __uint_as_float(mbits);
    if (!(M > 0.0f)) return 0;
    int e;
    frexp((double)M * (double)(ncontrib + 1), &e);        // bound < 2^e
    return 61 - e;
}

// ---------------------------------------------------------------------------
// sampling: trilinear (default) or containing cell
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void axis_stencil(T uh, float ul, int n, int &i0, T &t) {
    if (n == 1) { i0 = 0; t = (T)0; return; }
    T xh = uh - (T)0.5;                     // coordinate in cell-centre units: xh + ul
    if (xh + (T)ul <= (T)0) { i0 = 0; t = (T)0; return; }
    if (xh + (T)ul >= (T)(n - 1)) { i0 = n - 2; t = (T)1; return; }
    int i = (int)tfloor(xh);
    T fr = (xh - (T)i) + (T)ul;
    if (fr < (T)0) { i -= 1; fr += (T)1; }
    else if (fr >= (T)1) { i += 1; fr -= (T)1; }
    if (i < 0) { i = 0; fr = (T)0; }
    if (i > n - 2) { i = n - 2; fr = (T)1; }
    i0 = i;
    t = fr;
}

// f2 given: the sample of f - f2, the difference taken per cell in the
// field precision (so a small time difference keeps its digits)
#define AL_FV(F, F2, i) ((C)(F2 ? (F[i] - F2[i]) : F[i]))

// Kernel-weighted volume average (the smooth sampler of Sec. 6): weights
// exp(-(r/eps)^2) of the projection's truncated Gaussian (Eq. almGaussian,
// its constant cancels) over the cells of the grid whose centre lies within
// r <= 3 eps of the point, normalised by their sum; epsc = eps / h.  One
// thread (LANES = 1) visits every cell of the support's bounding box; a warp
// (LANES = 32, all lanes calling with the same arguments) visits only the
// rows that reach the sphere, 16 neighbouring cells at a time, and a
// butterfly reduction leaves the same sums, bit for bit, in every lane.  At most 4 components.  Returns
// false when no cell centre lies within 3 eps (the caller then takes the
// containing cell).
template <int LANES, typename S, typename C>
__device__ bool gauss_avg(const GridC &g, C epsc, const S *const *f, int ncomp, const C uh[3], const float ul[3],
                          C *out, const S *const *f2) {
    const int n[3] = {g.nx, g.ny, g.nz};
    const C Rc = (C)3 * epsc, R2 = Rc * Rc;
    const C l2ie2 = (C)1.4426950408889634 / (epsc * epsc);     // log2(e) / eps^2
    int lo[3], bn[3];
    for (int a = 0; a < 3; ++a) {
        const C c = (uh[a] - (C)0.5) + (C)ul[a];                // centre-unit coordinate
        int l0 = (int)tfloor(c - Rc), h0 = (int)tfloor(c + Rc) + 1;
        l0 = l0 < 0 ? 0 : l0;
        h0 = h0 > n[a] - 1 ? n[a] - 1 : h0;
        lo[a] = l0;
        bn[a] = h0 - l0 + 1;
    }
    const long long nxy = (long long)g.nx * g.ny;
    C acc[4] = {(C)0, (C)0, (C)0, (C)0}, sw = (C)0;
    if constexpr (LANES > 1) {
        // a warp: per layer, lane r sizes row r's run of cells on the chord of
        // the sphere's disc (widened by a cell on each side; the r^2 test
        // decides), a scan places the runs end to end, and the lanes take 32
        // consecutive cells at a time, so only cells near the sphere are read
        const int lane = (int)(threadIdx.x & 31);
        const C cy = (uh[1] - (C)0.5) + (C)ul[1], cx = (uh[0] - (C)0.5) + (C)ul[0];
        const int xlo = lo[0], xhi = lo[0] + bn[0] - 1;
        for (int k = 0; k < bn[2]; ++k) {
            const int ck = lo[2] + k;
            const C dz = (((C)ck + (C)0.5) - uh[2]) - (C)ul[2];
            const C dz2 = dz * dz;
            if (dz2 > R2) continue;
            // rows of this layer whose centre can lie within the radius left
            const C dyr = tsqrt(R2 - dz2);
            int j0 = (int)tfloor(cy - dyr), j1 = (int)tfloor(cy + dyr) + 1;
            j0 = j0 < lo[1] ? lo[1] : j0;
            j1 = j1 > lo[1] + bn[1] - 1 ? lo[1] + bn[1] - 1 : j1;
            for (int r0 = j0; r0 <= j1; r0 += 32) {
                int rcnt = 0, rx0 = 0;
                const int cjr = r0 + lane;
                if (cjr <= j1) {
                    const C dy = (((C)cjr + (C)0.5) - uh[1]) - (C)ul[1];
                    const C q = R2 - dz2 - dy * dy;
                    if (q >= (C)0) {
                        const C hw = tsqrt(q);
                        int xa = (int)tfloor(cx - hw) - 1, xb = (int)tfloor(cx + hw) + 1;
                        xa = xa < xlo ? xlo : xa;
                        xb = xb > xhi ? xhi : xb;
                        rcnt = xb >= xa ? xb - xa + 1 : 0;
                        rx0 = xa;
                    }
                }
                int rinc = rcnt;
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, rinc, o);
                    if (lane >= o) rinc += v;
                }
                const int ncell = __shfl_sync(0xffffffffu, rinc, 31);
                for (int q0 = 0; q0 < ncell; q0 += 32) {
                    const int qc = q0 + lane;
                    int r = 0;                           // rows whose runs end at or before qc
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1) {
                        const int v = __shfl_sync(0xffffffffu, rinc, r + st - 1);
                        if (v <= qc) r += st;
                    }
                    const int cb = __shfl_sync(0xffffffffu, rinc - rcnt, r);
                    const int ci = __shfl_sync(0xffffffffu, rx0, r) + (qc - cb), cj = r0 + r;
                    const C dx = (((C)ci + (C)0.5) - uh[0]) - (C)ul[0];
                    const C dy = (((C)cj + (C)0.5) - uh[1]) - (C)ul[1];
                    const C r2 = dx * dx + (dy * dy + dz2);
                    if (qc < ncell && r2 <= R2) {
                        const C w = Tr<C>::ex2(-r2 * l2ie2);
                        const long long idx = ci + (long long)g.nx * cj + nxy * ck;
                        sw += w;
                        for (int qq = 0; qq < ncomp; ++qq) {
                            const S *F = f[qq], *F2 = f2 ? f2[qq] : nullptr;
                            acc[qq] += w * AL_FV(F, F2, idx);
                        }
                    }
                }
            }
        }
    } else {
    // one thread: every cell of the box in x-fastest order
    const int nplane = bn[0] * bn[1];
    const long long nbox = (long long)nplane * bn[2];
    const int lane = 0;
    int k = lane / nplane, r = lane - k * nplane, j = r / bn[0], i = r - j * bn[0];
    const int dk = LANES / nplane, dr = LANES - dk * nplane, dj = dr / bn[0], di = dr - dj * bn[0];
    for (long long t = lane; t < nbox; t += LANES) {
        const int ci = lo[0] + i, cj = lo[1] + j, ck = lo[2] + k;
        const C dx = (((C)ci + (C)0.5) - uh[0]) - (C)ul[0];
        const C dy = (((C)cj + (C)0.5) - uh[1]) - (C)ul[1];
        const C dz = (((C)ck + (C)0.5) - uh[2]) - (C)ul[2];
        const C r2 = dx * dx + dy * dy + dz * dz;
        if (r2 <= R2) {
            const C w = Tr<C>::ex2(-r2 * l2ie2);
            const long long idx = ci + (long long)g.nx * cj + nxy * ck;
            sw += w;
            for (int q = 0; q < ncomp; ++q) {
                const S *F = f[q], *F2 = f2 ? f2[q] : nullptr;
                acc[q] += w * AL_FV(F, F2, idx);
            }
        }
        i += di; j += dj; k += dk;
        if (i >= bn[0]) { i -= bn[0]; j += 1; }
        if (j >= bn[1]) { j -= bn[1]; k += 1; }
    }
    }
    if (LANES > 1) {
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            sw += __shfl_xor_sync(0xffffffffu, sw, m);
            for (int q = 0; q < 4; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], m);
        }
    }
    if (!(sw > (C)0)) return false;
    for (int q = 0; q < ncomp; ++q) out[q] = acc[q] / sw;
    return true;
}

// Returns false when the point lies outside the grid.  Fields are stored as
// S and interpolated in the arithmetic type C.  mode 2 (the volume average)
// needs the kernel width epsc = eps / h and LANES lanes calling together.
template <int LANES = 1, typename S, typename C>
__device__ bool sample(const GridC &g, int mode, C epsc, const S *const *f, int ncomp,
                       const C uh[3], const float ul[3], C *out, const S *const *f2 = nullptr) {
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a)
        if (!inside_axis(uh[a], ul[a], n[a])) return false;
    const long long nxy = (long long)g.nx * g.ny;
    if (mode == 2 && gauss_avg<LANES>(g, epsc, f, ncomp, uh, ul, out, f2)) return true;
    if (mode >= 1) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = ffloor(uh[a], ul[a]);
            c[a] = c[a] < 0 ? 0 : (c[a] > n[a] - 1 ? n[a] - 1 : c[a]);
        }
        long long idx = c[0] + (long long)g.nx * c[1] + nxy * c[2];
        for (int q = 0; q < ncomp; ++q) {
            const S *F = f[q], *F2 = f2 ? f2[q] : nullptr;
            out[q] = AL_FV(F, F2, idx);
        }
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
        const S *F = f[q], *F2 = f2 ? f2[q] : nullptr;
        C c00 = wx0 * AL_FV(F, F2, base) + t[0] * AL_FV(F, F2, base + sx);
        C c10 = wx0 * AL_FV(F, F2, base + sy) + t[0] * AL_FV(F, F2, base + sy + sx);
        C c01 = wx0 * AL_FV(F, F2, base + sz) + t[0] * AL_FV(F, F2, base + sz + sx);
        C c11 = wx0 * AL_FV(F, F2, base + sz + sy) + t[0] * AL_FV(F, F2, base + sz + sy + sx);
        out[q] = wz0 * (wy0 * c00 + t[1] * c10) + t[2] * (wy0 * c01 + t[1] * c11);
    }
    return true;
}
#undef AL_FV

// 1/h in the arithmetic type (no FP64 division for FP32 instances)
template <typename C> __device__ __forceinline__ C inv_h(const GridC &g);
template <> __device__ __forceinline__ float inv_h<float>(const GridC &g) { return g.ih_hi; }
template <> __device__ __forceinline__ double inv_h<double>(const GridC &g) { return 1.0 / g.h; }

// Quasi-steady line force f* of one actuator point (Secs. 3.2.2-3.2.3) in the
// arithmetic type C from fields stored as T: preliminary sample, upstream
// direction with fallback, sampling point, upstream sample (+ alpha,
// mixture density), Morison drag.  Returns 1 without side effects when C is
// float and the upstream direction is ill-conditioned (|u0_n| below 1 % of
// the velocity scale, where FP32 rounding of the samples is amplified by
// 1/|u0_n|); the caller then repeats the evaluation in FP64.
// With LANES = 32 a whole warp evaluates one point together (the volume-
// average sampler shares its cells among the lanes); every lane then holds
// the same result and lane 0 alone counts the status events.
template <int LANES>
__device__ __forceinline__ void st_count(int *status, int e) {
    if (LANES == 1 || (threadIdx.x & 31) == 0) atomicAdd(&status[e], 1);
}

template <typename T, typename C, int LANES = 1>
__device__ int point_fstar(const GridC &g, const BeamsC &b, const StepPtrs<T> &p, const int l, const C Pa[3],
                           const C Pd[3], const C t[3], C fstar[3], int *status, const bool refine_ok,
                           const C ab[3]) {
    fstar[0] = fstar[1] = fstar[2] = (C)0;
    C ua[3];
    float la[3];
    for (int a = 0; a < 3; ++a) to_cell(g, a, Pa[a], ua[a], la[a]);
    const C epsc = b.sample_mode == 2 ? (C)(b.eps[l] / g.h) : (C)0;
    C Ua[3];
    if (!sample<LANES>(g, b.sample_mode, epsc, p.U, 3, ua, la, Ua)) {
        st_count<LANES>(status, ST_PA_OUTSIDE);
        return 0;
    }
    // Eq. almPreliminaryVelocity and its component normal to the tangent
    C u0r[3], u0n[3], es[3];
    for (int a = 0; a < 3; ++a) u0r[a] = Ua[a] - Pd[a];
    C ut = u0r[0] * t[0] + u0r[1] * t[1] + u0r[2] * t[2];
    for (int a = 0; a < 3; ++a) u0n[a] = u0r[a] - ut * t[a];
    C nn = tsqrt(u0n[0] * u0n[0] + u0n[1] * u0n[1] + u0n[2] * u0n[2]);
    if (refine_ok) {
        C scale = tsqrt(Ua[0] * Ua[0] + Ua[1] * Ua[1] + Ua[2] * Ua[2]) + tsqrt(Pd[0] * Pd[0] + Pd[1] * Pd[1] + Pd[2] * Pd[2]);
        if (nn < (C)1e-2 * scale) return 1;
    }
    if ((double)nn >= b.tau) {
        for (int a = 0; a < 3; ++a) es[a] = -u0n[a] / nn;
    } else {
        st_count<LANES>(status, ST_FALLBACK);
        C gp[3];
        C gt = (C)b.g_up[0] * t[0] + (C)b.g_up[1] * t[1] + (C)b.g_up[2] * t[2];
        for (int a = 0; a < 3; ++a) gp[a] = (C)b.g_up[a] - gt * t[a];
        C gn = tsqrt(gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2]);
        if (gn > (C)0) for (int a = 0; a < 3; ++a) es[a] = gp[a] / gn;
        else { es[0] = es[1] = es[2] = (C)0; st_count<LANES>(status, ST_FALLBACK_ZERO); }
    }
    // Eq. almSamplingPoint: offset (I - n_p n_p^T) l_s e_s
    const C ell = (C)b.ell_s[l];
    C v[3];
    for (int a = 0; a < 3; ++a) v[a] = ell * es[a];
    C vn = (C)b.n_p[0] * v[0] + (C)b.n_p[1] * v[1] + (C)b.n_p[2] * v[2];
    C us[3];
    float ls[3];
    for (int a = 0; a < 3; ++a) {
        C off_c = (v[a] - (C)b.n_p[a] * vn) * inv_h<C>(g);
        ff_add(ua[a], la[a], off_c, us[a], ls[a]);
    }
    // U and alpha at P_s in one pass over the stencil (4 components)
    C Us[4];
    const T *fua[4] = {p.U[0], p.U[1], p.U[2], p.alpha};
    const bool ok = sample<LANES>(g, b.sample_mode, epsc, fua, g.has_alpha ? 4 : 3, us, ls, Us);
    const C as = g.has_alpha ? Us[3] : (C)0;
    if (!ok) {
        st_count<LANES>(status, ST_PS_OUTSIDE);
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
        C m = tsqrt(Ur[0] * Ur[0] + Ur[1] * Ur[1] + Ur[2] * Ur[2]);
        for (int a = 0; a < 3; ++a) fstar[a] = half * m * (cdn * Un[a] + cdt * Ut[a]);
    } else {
        C mt = tsqrt(Ut[0] * Ut[0] + Ut[1] * Ut[1] + Ut[2] * Ut[2]);
        C mn = tsqrt(Un[0] * Un[0] + Un[1] * Un[1] + Un[2] * Un[2]);
        for (int a = 0; a < 3; ++a) fstar[a] = half * (cdt * mt * Ut[a] + cdn * mn * Un[a]);
    }
    if (b.inertia) {
        // Eq. fext_addedmass with the fluid acceleration sampled at P_s and the
        // reaction following the fluid's acceleration relative to the beam
        C af[3] = {(C)0, (C)0, (C)0};
        if (p.Uprev[0]) {
            sample<LANES>(g, b.sample_mode, epsc, p.U, 3, us, ls, af, p.Uprev);   // U - U_prev at P_s
            const C idt = (C)(1.0 / p.dt);
            for (int a = 0; a < 3; ++a) af[a] *= idt;
        }
        C ar[3];
        for (int a = 0; a < 3; ++a) ar[a] = af[a] - ab[a];
        const C art = ar[0] * t[0] + ar[1] * t[1] + ar[2] * t[2];
        const C ra = rho * (C)(0.25 * PI_D * b.d[l] * b.d[l]);
        const C cmn = (C)b.cm_n[l], cmt = (C)b.cm_t[l];
        for (int a = 0; a < 3; ++a) {
            const C at = art * t[a], an = ar[a] - at;
            fstar[a] += ra * (cmt * at + cmn * an + af[a]);
        }
    }
    return 0;
}

// ---------------------------------------------------------------------------
// k_points: Sec. 3.2.2 - 3.2.3, one thread per actuator point (LANES = 1) or
// one warp per point (LANES = 32, for the volume-average sampler; every lane
// computes the same values and lane 0 stores them)
// ---------------------------------------------------------------------------
template <typename T, int LANES = 1>
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
        T nn = tsqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        if (nn > (T)0) for (int a = 0; a < 3; ++a) t[a] /= nn;
        else t[0] = t[1] = t[2] = (T)0;
    }

    T fstar[3];
    T ab[3] = {(T)0, (T)0, (T)0};
    if (b.inertia && p.Pdd[0])
        for (int a = 0; a < 3; ++a) ab[a] = p.Pdd[a][i];
    if (point_fstar<T, T, LANES>(g, b, p, l, Pa, Pd, t, fstar, status, sizeof(T) == 4, ab)) {
        // ill-conditioned upstream direction: the same evaluation in FP64
        double Pa64[3], Pd64[3], t64[3], f64[3], ab64[3];
        for (int a = 0; a < 3; ++a) { Pa64[a] = (double)Pa[a]; Pd64[a] = (double)Pd[a]; ab64[a] = (double)ab[a]; }
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
        point_fstar<T, double, LANES>(g, b, p, l, Pa64, Pd64, t64, f64, status, false, ab64);
        for (int a = 0; a < 3; ++a) fstar[a] = (T)f64[a];
        st_count<LANES>(status, ST_REFINED);
    }
    if (LANES > 1 && (threadIdx.x & 31) != 0) return;
    // Eq. almForceRelaxation and the per-CV load
    const T af = (T)b.alpha_f[l];
    const T L = (T)b.cv_len[i];
    const long long np = b.n_points;
    for (int a = 0; a < 3; ++a) {
        T f = has_prev ? af * fstar[a] + ((T)1 - af) * sc.fprev[a * np + i] : fstar[a];
        sc.fprev[a * np + i] = f;
        p.F[a][i] = f * L;
    }
    sc.wfix[i] = 0ull;                                   // fixed-point weights start at zero
    if (i == 0) {
        *sc.anyIrr = 0; *sc.smax = 0u; *sc.anyZero = 0;
        sc.cmcnt[0] = 0; sc.cmcnt[1] = 0; sc.cmcnt[2] = 0; sc.cmcnt[3] = 0; sc.cmcnt[4] = 0;
        if (sc.cment_n) *sc.cment_n = 0;
        sc.rplan[0] = sc.rplan[1];                        // the regions the last step sized
        sc.rplan[1] = 0;
        *sc.rused = 0ull;
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
        T n0 = tsqrt(t0[0] * t0[0] + t0[1] * t0[1] + t0[2] * t0[2]);
        T n1 = tsqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
        float tau = 1e30f;
        T m[3] = {(T)0, (T)0, (T)0};
        if (n0 > (T)0 && n1 > (T)0) {
            for (int a = 0; a < 3; ++a) { t0[a] /= n0; t1[a] /= n1; m[a] = t0[a] + t1[a]; }
            T c = t0[0] * t1[0] + t0[1] * t1[1] + t0[2] * t1[2];
            T cx = t0[1] * t1[2] - t0[2] * t1[1], cy = t0[2] * t1[0] - t0[0] * t1[2],
              cz = t0[0] * t1[1] - t0[1] * t1[0];
            T sn = tsqrt(cx * cx + cy * cy + cz * cz);
            if ((T)1 + c > (T)1e-3) tau = (float)(sn / ((T)1 + c));   // tan(theta/2)
            T mn = tsqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            if (mn > (T)0) for (int a = 0; a < 3; ++a) m[a] /= mn;
        }
        for (int a = 0; a < 3; ++a) sc.nodeM[a * np + k] = m[a];
        sc.nodeTau[k] = tau;
    } else {
        for (int a = 0; a < 3; ++a) sc.nodeM[a * np + k] = (T)0;
        sc.nodeTau[k] = 0.0f;
    }
    cm_write_node(sc, np, k, off);
}

// ---------------------------------------------------------------------------
// k_lines: one warp per line
//
// Walk certificate.  For a cell C and interior node k let
// sigma_k(C) = (C - P_k) . m_k with m_k the unit bisector of the two segment
// directions.  If the perpendicular distance rho of C from segment k's axis
// satisfies rho (tan(theta_k/2) + tan(theta_{k+1}/2)) < L_k, then
// sigma_k(C) <= 0 implies sigma_{k+1}(C) < 0, and the sign of sigma_k(C)
// orders the distances to segments k-1 and k (their common node is within
// reach of both feet).  On a run of nodes where this holds the signs are
// monotone, and the closest segment is the last k with sigma_k(C) > 0,
// which a walk finds.  Only cells within R = 3 eps matter (farther cells
// receive nothing).  Two certificates, both requiring every segment longer
// than 1e-3 cells and, with margin 2, the inequality above for every segment:
//
// regular = 1: for every node of the arc a walk over a brick's candidate
//   segments can visit.  That arc is at most S = min((brick diagonal +
//   2 sqrt(3) R + 2 L_max) / c_a, line length) long (c_a = min over segments
//   of direction . chord, > 0.3), so rho <= R + S min(Theta, 1) with
//   Theta = (S / L_min + 2) theta_max bounding its turning.  A walk may start
//   at any candidate segment.
//
// regular = 2: lines that climb (every segment's |D_z| / |D| >= c_z > 0.3,
//   one sign).  Let K be the nodes within rho_s of C, rho_s = r_h + L_max +
//   0.1 with r_h the crossing-disc radius below (so the segment crossing a
//   cell's layer starts within rho_s of every cell in its disc).  Two nodes
//   of K are at most 2 rho_s apart, so the arc between them is at most
//   lambda = 2 rho_s / c + L_max long, c = cos(Theta_l / 2) with Theta_l the
//   total turning of the line (all tangents of an arc lie in a cone of
//   half-angle Theta_l / 2, hence chord >= c arc), and it departs from the
//   chord by at most lambda/2 sin(Theta_w), Theta_w = min(Theta_l,
//   (lambda / L_min + 1) theta_max).  Every node between two nodes of K is
//   then within rho_s + lambda/2 sin(Theta_w) of C; certifying that radius
//   makes the signs monotone between any two nodes of K.  A walk that starts
//   in K (checked: |C - P_start| <= rho_s) ends at the closest segment when
//   that segment is within R, and a walk that ends within R has found the
//   closest segment whatever its start.
// ---------------------------------------------------------------------------
static __device__ void cm_layer_records(const GridC &g, const Scratch<float> &sc, long long np, int l, int off,
                                        int n, float Rc, float Lmax, int lane, int *status, float *sZ, float4 *sP);

template <typename T>
__device__ void d_lines(const GridC &g, const BeamsC &b, const Scratch<T> &sc, const StepPtrs<T> &p, int *status,
                        const int l, const int lane, float *sZ = nullptr, float4 *sP = nullptr) {
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

    // geometry of the line
    float Lmin = 1e30f, Lmax = 0.0f, ca = 1.0f, czp = 1.0f, czn = 1.0f;
    T ax[3] = {(T)0, (T)0, (T)0};
    int chord_ok = 0;
    if (n >= 2) {
        for (int a = 0; a < 3; ++a) ax[a] = ff_diff(sc, np, a, off + n - 1, off);
        T an = tsqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
        if (an > (T)0) { for (int a = 0; a < 3; ++a) ax[a] /= an; chord_ok = 1; }
    }
    float Ltot = 0.0f, thmax = 0.0f, thsum = 0.0f;
    for (int q = lane; q < n - 1; q += 32) {
        const int k = off + q;
        T D0 = sc.segD[k], D1 = sc.segD[np + k], D2 = sc.segD[2 * np + k];
        float L = (float)tsqrt(D0 * D0 + D1 * D1 + D2 * D2);
        Lmin = fminf(Lmin, L);
        Lmax = fmaxf(Lmax, L);
        Ltot += L;
        float c = L > 0.0f ? (float)((D0 * ax[0] + D1 * ax[1] + D2 * ax[2])) / L : -1.0f;
        ca = fminf(ca, c);
        const float cz = L > 0.0f ? (float)D2 / L : 0.0f;
        czp = fminf(czp, cz);
        czn = fminf(czn, -cz);
        if (q >= 1) {
            const float th = 2.0f * atanf(sc.nodeTau[k]);
            thmax = fmaxf(thmax, th);
            thsum += th;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        Lmin = fminf(Lmin, __shfl_xor_sync(0xffffffffu, Lmin, o));
        Lmax = fmaxf(Lmax, __shfl_xor_sync(0xffffffffu, Lmax, o));
        ca = fminf(ca, __shfl_xor_sync(0xffffffffu, ca, o));
        czp = fminf(czp, __shfl_xor_sync(0xffffffffu, czp, o));
        czn = fminf(czn, __shfl_xor_sync(0xffffffffu, czn, o));
        Ltot += __shfl_xor_sync(0xffffffffu, Ltot, o);
        thsum += __shfl_xor_sync(0xffffffffu, thsum, o);
        thmax = fmaxf(thmax, __shfl_xor_sync(0xffffffffu, thmax, o));
    }
    const bool base_ok = (n >= 2) && (Lmin > 1e-3f);
    // radius within which the bisector signs must be monotone, per certificate
    float D1c = -1.0f, D2c = -1.0f, rho_s = 0.0f;
    if (base_ok && chord_ok && ca > 0.3f) {
        const float S = fminf((BRICK_DIAG + 2.0f * 1.7320508f * Rc + 2.0f * Lmax) / ca, Ltot);
        const float Theta = (S / Lmin + 2.0f) * thmax;
        D1c = Rc + S * fminf(Theta, 1.0f) + 0.01f;
    }
    const float czl = fmaxf(czp, czn);
    if (base_ok && n >= 3 && czl > 0.3f) {
        const float lam = Rc / czl + Lmax;
        const float turn = (lam / Lmin + 1.0f) * thmax;
        const float rh = (Rc + lam * fminf(1.0f, turn) + 0.02f) / czl + 0.02f;
        rho_s = rh + Lmax + 0.1f;
        const float c = cosf(0.5f * fminf(thsum, 3.0f));
        if (c > 0.3f) {
            const float lw = 2.0f * rho_s / c + Lmax;
            const float thw = fminf(thsum, (lw / Lmin + 1.0f) * thmax);
            if (thw < 1.2f) D2c = rho_s + 0.5f * lw * sinf(thw) + 0.05f;
        }
    }
    // column-march certificate: the line climbs (every segment D_z / |D| >=
    // 0.8); a brick of height h <= 16 takes as candidates the segments whose
    // height range meets its layers' centres widened by 3 eps (+0.02), an arc
    // of at most S = (16 + 2 R + 0.06 + 2 L_max) / c_z cells, so a cell within
    // R of the line has every candidate within arc S of its foot; certifying
    // rho = R + S min(Theta, 1) (Theta = (S / L_min + 2) theta_max its
    // turning) makes the bisector signs monotone over the candidates
    float Dcm = -1.0f;
    // (a brick's candidate range, at most (16 + 2 R + 0.06) / (L_min c_z) + 2
    // segments, fits the stage; node positions relative to the line's first
    // node stay below 256 cells, so their FP32 rounding is below 8e-6 cells)
    if (sizeof(T) == 4 && base_ok && czp >= 0.8f && Ltot < 250.0f && (16.0f + 2.0f * Rc + 0.06f) / (Lmin * czp) + 3.0f < (float)CM_NN) {
        const float S = fminf((16.0f + 2.0f * Rc + 0.06f + 2.0f * Lmax) / czp, Ltot);
        const float Theta = (S / Lmin + 2.0f) * thmax;
        Dcm = Rc + S * fminf(Theta, 1.0f) + 0.01f;
    }
    int ok1 = D1c > 0.0f, ok2 = D2c > 0.0f, okc = Dcm > 0.0f;
    if (okc) {
        int badc = 0;
        for (int q = lane; q < n - 1; q += 32) {
            const int k = off + q;
            float t0 = (q >= 1) ? sc.nodeTau[k] : 0.0f;
            float t1 = (q + 1 <= n - 2) ? sc.nodeTau[k + 1] : 0.0f;
            T D0 = sc.segD[k], D1 = sc.segD[np + k], D2 = sc.segD[2 * np + k];
            float L = (float)tsqrt(D0 * D0 + D1 * D1 + D2 * D2);
            if (!(Dcm * (t0 + t1) <= 0.5f * L)) badc = 1;
        }
        if (__any_sync(0xffffffffu, badc)) okc = 0;
    }
    if (ok1 || ok2) {
        int bad1 = 0, bad2 = 0;
        for (int q = lane; q < n - 1; q += 32) {
            const int k = off + q;
            float t0 = (q >= 1) ? sc.nodeTau[k] : 0.0f;
            float t1 = (q + 1 <= n - 2) ? sc.nodeTau[k + 1] : 0.0f;
            T D0 = sc.segD[k], D1 = sc.segD[np + k], D2 = sc.segD[2 * np + k];
            float L = (float)tsqrt(D0 * D0 + D1 * D1 + D2 * D2);
            if (!(D1c * (t0 + t1) <= 0.5f * L)) bad1 = 1;
            if (!(D2c * (t0 + t1) <= 0.5f * L)) bad2 = 1;
        }
        if (__any_sync(0xffffffffu, bad1)) ok1 = 0;
        if (__any_sync(0xffffffffu, bad2)) ok2 = 0;
    }
    if (lane == 0) {
        LineG lg;
        const double ec = eps / g.h;
        lg.Rc = Rc;
        lg.R2c = 9.0 * ec * ec;
        lg.inv_eps2c = 1.0 / (ec * ec);
        lg.inv_eps2c_l2 = 1.4426950408889634 / (ec * ec);
        lg.eta0 = 1.0 / (PI_D * eps * eps);
        lg.R2f = (float)lg.R2c;
        lg.ie2f = (float)lg.inv_eps2c_l2;
        lg.eta0f = (float)lg.eta0;
        lg.regular = ok2 ? 2 : (ok1 ? 1 : 0);
        lg.cm = okc;
        lg.first = off;
        lg.n = n;
        lg.thmax = thmax;
        lg.Lmin = Lmin;
        lg.Lmax = Lmax;
        lg.rho2 = rho_s * rho_s;
        // largest possible fixed-point sum at a node: the cells within R of
        // its two segments, each omega eta / eta0 <= 1
        const float Rp = Rc + 1.0f;
        const float Q = 3.1415927f * Rp * Rp * 2.0f * (n >= 2 ? Lmax : 0.0f) + 4.1887903f * Rp * Rp * Rp + 1.0f;
        int sh = 62 - (int)ceilf(log2f(Q));
        lg.wshift = max(20, min(sh, 60));
        sc.lines[l] = lg;
        if (lg.regular == 0 && n > 0) {
            atomicAdd(&status[ST_IRREGULAR], 1);
            *sc.anyIrr = 1;
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        // what the column march's entries of each brick layer share
        if (okc && sc.cmlay && n >= 2) cm_layer_records(g, sc, np, l, off, n, Rc, Lmax, lane, status, sZ, sP);
    }
}

// node index of the far end of segment k of a line (first, n)
__device__ __forceinline__ int seg_end(int k, int n) { return n == 1 ? k : k + 1; }

// conservative R-inflated box of segment k (nodes ka, kb) in cell units
template <typename T>
__device__ __forceinline__ void seg_box(const Scratch<T> &sc, long long np, int ka, int kb, float R,
                                        float lo[3], float hi[3]) {
    for (int a = 0; a < 3; ++a) {
        float ua = (float)sc.uhi[a * np + ka], ub = (float)sc.uhi[a * np + kb];
        float slack = fmaxf(R, 0.5f) + 0.01f + 1e-5f * (fabsf(ua) + 1.0f);
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
    const int nn[3] = {g.nx, g.ny, g.nz}, bs[3] = {BX, BY, g.bz}, nb[3] = {g.nbx, g.nby, g.nbz};
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
__device__ __noinline__ double dist2_f64_raw(const T *P0, const T *P1, const T *P2, double ox, double oy,
                                             double oz, double h, int ka, int kb, int ci, int cj, int ck) {
    const double c[3] = {__dadd_rn(ox, __dmul_rn((double)ci + 0.5, h)),
                         __dadd_rn(oy, __dmul_rn((double)cj + 0.5, h)),
                         __dadd_rn(oz, __dmul_rn((double)ck + 0.5, h))};
    const T *P[3] = {P0, P1, P2};
    double D[3], q[3];
    for (int a = 0; a < 3; ++a) {
        double A = (double)P[a][ka], B = (double)P[a][kb];
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
    return __dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])), __dmul_rn(e[2], e[2]));
}
template <typename T>
__device__ __forceinline__ double dist2_f64(const GridC &g, const StepPtrs<T> &p, int ka, int kb, int ci, int cj,
                                            int ck) {
    return dist2_f64_raw(p.Ps[0], p.Ps[1], p.Ps[2], g.o[0], g.o[1], g.o[2], g.h, ka, kb, ci, cj, ck);
}

// d_k < d_{k-1} in FP64 (segment k closer than k-1; ties keep k-1)
template <typename T>
__device__ __forceinline__ bool later_closer_f64(const GridC &g, const StepPtrs<T> &p, int k, int ci, int cj, int ck) {
    double d1 = dist2_f64(g, p, k, k + 1, ci, cj, ck);
    double d0 = dist2_f64(g, p, k - 1, k, ci, cj, ck);
    return __dsqrt_rn(d1) < __dsqrt_rn(d0);
}
// r <= 3 eps in FP64 for segment k
template <typename T>
__device__ __forceinline__ bool within_f64(const GridC &g, const StepPtrs<T> &p, double eps, int k, int n, int ci,
                                           int cj, int ck) {
    double d2 = dist2_f64(g, p, k, seg_end(k, n), ci, cj, ck);
    return __dsqrt_rn(d2) <= __dmul_rn(3.0, eps);
}
// argmin over segments [k0, k1] in FP64, lowest index on ties
template <typename T>
__device__ __noinline__ int argmin_f64_raw(const T *P0, const T *P1, const T *P2, double ox, double oy, double oz,
                                           double h, int k0, int k1, int n, int ci, int cj, int ck) {
    double best = INFINITY;
    int kb = k0;
    for (int k = k0; k <= k1; ++k) {
        double r = __dsqrt_rn(dist2_f64_raw(P0, P1, P2, ox, oy, oz, h, k, seg_end(k, n), ci, cj, ck));
        if (r < best) { best = r; kb = k; }
    }
    return kb;
}
template <typename T>
__device__ __forceinline__ int argmin_f64(const GridC &g, const StepPtrs<T> &p, int k0, int k1, int n, int ci,
                                          int cj, int ck) {
    return argmin_f64_raw(p.Ps[0], p.Ps[1], p.Ps[2], g.o[0], g.o[1], g.o[2], g.h, k0, k1, n, ci, cj, ck);
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
    int k, q, n, off, nseg, kb, klo, khi;     // klo/khi unused (kept zero-cost)
    int O[3], lo[3], hi[3];
    T A[3], Bn[3], D[3], il2;
    int O1[3];                    // integer origin floor(u) of the end node kb
    T B1[3];                      // the end node relative to O1
    T m0[3], m1[3];
    bool has_lo, has_hi;
    T R2, gr, ie2, eta0;
    T gsb;                        // guard band of the bisector tests, for the farthest cell of the box
    double eps;
    int integ;                    // segment-integrated kernel (projection variant, lines of >= 2 nodes)
    T epsc;                       // eps in cells
};

// |x|^2 and x.m with every operation rounded explicitly
template <typename T>
__device__ __forceinline__ T norm2_r(const T x[3]) { return r_fma(x[2], x[2], r_fma(x[1], x[1], r_mul(x[0], x[0]))); }
template <typename T>
__device__ __forceinline__ T dot_r(const T x[3], const T m[3]) { return r_fma(x[2], m[2], r_fma(x[1], m[1], r_mul(x[0], m[0]))); }

// Foot parameter s (clamped to [0, 1]) and squared distance r^2 of a cell
// from a segment, from the cell's offset x to the segment start and the
// segment vector D (cell units), every operation rounded explicitly
template <typename T>
__device__ __forceinline__ void foot_sr(const T x[3], const T D[3], T il2, T &s, T &r2) {
    s = r_mul(dot_r(x, D), il2);
    s = s < (T)0 ? (T)0 : (s > (T)1 ? (T)1 : s);
    const T e[3] = {r_fma(-s, D[0], x[0]), r_fma(-s, D[1], x[1]), r_fma(-s, D[2], x[2])};
    r2 = norm2_r(e);
}
// offset of the global cell cg from node k, taken from the node's own
// integer origin floor(u_k)
template <typename T>
__device__ __forceinline__ void node_off(const Scratch<T> &sc, long long np, int k, const int cg[3], T x[3]) {
    for (int a = 0; a < 3; ++a) {
        const T uh = sc.uhi[a * np + k];
        const int O = ifloor(uh);
        x[a] = ((T)(cg[a] - O) + (T)0.5) - rel(uh, sc.ulo[a * np + k], O);
    }
}
// (s, r^2) of the global cell cg against segment (ka, kb): offsets from the
// start node's origin, and where the foot clamps to the end node, r^2 from
// the end node's origin, so a cell whose closest point is a node gets the
// same bits whichever of the node's two segments takes it (the segment
// pass computes the same values)
template <typename T>
__device__ __forceinline__ void pair_sr(const Scratch<T> &sc, long long np, int ka, int kb, const int cg[3], T &s,
                                        T &r2) {
    T x[3], D[3];
    node_off(sc, np, ka, cg, x);
    for (int a = 0; a < 3; ++a) D[a] = sc.segD[a * np + ka];
    foot_sr(x, D, sc.segIl2[ka], s, r2);
    if (s >= (T)1 && kb != ka) {
        node_off(sc, np, kb, cg, x);
        r2 = norm2_r(x);
    }
}
// the pair's kernel value eta split over the segment's two nodes (omega eta)
template <typename T>
__device__ __forceinline__ void pair_w(T eta, T s, T &wa, T &wb) {
    wa = r_mul(eta, r_add((T)1, -s));
    wb = r_mul(eta, s);
}
// the pair's momentum source for nodal forces fa, fb (S receives minus this)
template <typename T>
__device__ __forceinline__ T pair_src(T wa, T wb, T fa, T fb) { return r_fma(wa, fa, r_mul(wb, fb)); }

__device__ __forceinline__ float t_erf(float x) { return erff(x); }
__device__ __forceinline__ double t_erf(double x) { return erf(x); }
__device__ __forceinline__ float t_exp(float x) { return expf(x); }
__device__ __forceinline__ double t_exp(double x) { return exp(x); }

// Segment-integrated 3-D Gaussian (the projection variant of Sec. 6) of the
// global cell cg against segment (ka, kb): with t0 the cell's tangential
// coordinate along the segment, r_p its distance from the segment's axis
// and L the length (cells, eps in cells epsc),
//   K0 = g E,  K1 = (g / L) (t0 E + epsc / (2 sqrt(pi)) (e^(-t0^2/epsc^2) - e^(-(L-t0)^2/epsc^2))),
//   E = (erf((L - t0)/epsc) + erf(t0/epsc)) / 2,  g = eta0 exp(-r_p^2/epsc^2),
// the integral of exp(-|x|^2/eps^2) / (pi^(3/2) eps^3) along the segment and
// its first moment in t / L; the nodes take wa = K0 - K1, wb = K1.  One
// compiled body (not inlined) serves the segment pass and the gather, so
// both produce the same bits for a pair.
template <typename T>
__device__ __noinline__ void pair_int(const Scratch<T> &sc, long long np, int ka, const int cg[3], T epsc, T eta0,
                                      T ie2l, T &wa, T &wb) {
    T x[3], D[3];
    node_off(sc, np, ka, cg, x);
    for (int a = 0; a < 3; ++a) D[a] = sc.segD[a * np + ka];
    const T L = tsqrt(norm2_r(D));
    if (!(L > (T)0)) { wa = wb = (T)0; return; }
    const T t0 = dot_r(x, D) / L;
    T pp[3];
    for (int a = 0; a < 3; ++a) pp[a] = r_fma(-t0 / L, D[a], x[a]);
    const T g = eta0 * Tr<T>::ex2(-norm2_r(pp) * ie2l);
    const T ie = (T)1 / epsc;
    const T E = (T)0.5 * (t_erf((L - t0) * ie) + t_erf(t0 * ie));
    const T m = epsc * (T)0.28209479177387814 *                      // 1 / (2 sqrt(pi))
                (t_exp(-(t0 * ie) * (t0 * ie)) - t_exp(-((L - t0) * ie) * ((L - t0) * ie)));
    const T K0 = g * E, K1 = g / L * (t0 * E + m);
    wa = K0 - K1;
    wb = K1;
}

// Per-CTA staging of the records of a round of segments (one per warp): each
// record takes a shared-memory slot, and at the end of the round the CTA
// reserves the slots of each brick (instance, brick key) with one global
// atomic and writes the records there.  Records beyond CAP, or of a brick
// that finds the table full, reserve their own slot directly.
template <typename T> struct RecStage {
    static constexpr int CAP = 768, NB = 64;
    Rec<T> rec[CAP];
    unsigned long long rk[CAP];     // (instance << 32) | brick of each staged record
    int loc[CAP];                   // (table entry << 16) | rank within the entry; -1: written directly
    unsigned long long key[NB];     // table of the round's (instance, brick) keys; ~0: empty
    int cnt[NB], base[NB];
    int n;
};
template <typename T>
__device__ __forceinline__ void rec_init(RecStage<T> &st) {
    for (int h = threadIdx.x; h < RecStage<T>::NB; h += blockDim.x) { st.key[h] = ~0ull; st.cnt[h] = 0; }
    if (threadIdx.x == 0) st.n = 0;
    __syncthreads();
}
// the whole CTA calls this after its round; sc_of(q) gives instance q's scratch
template <typename T, typename ScOf>
__device__ void rec_flush(RecStage<T> &st, ScOf sc_of) {
    constexpr int CAP = RecStage<T>::CAP, NB = RecStage<T>::NB;
    __syncthreads();
    const int n = min(st.n, CAP);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long key = st.rk[i];
        int h = (int)((key * 0x9E3779B97F4A7C15ull) >> 58);
        int slot = -1;
        for (int t = 0; t < NB; ++t, h = (h + 1) & (NB - 1)) {
            const unsigned long long old = atomicCAS(&st.key[h], ~0ull, key);
            if (old == ~0ull || old == key) { slot = h; break; }
        }
        if (slot >= 0) {
            st.loc[i] = (slot << 16) | atomicAdd(&st.cnt[slot], 1);
        } else {
            const Scratch<T> &s = sc_of((int)(key >> 32));
            const int br = (int)(key & 0xffffffffull);
            const int pos = atomicAdd(&s.rcnt[br], 1);
            if (pos < s.rcap[br]) s.rec[s.roff[br] + pos] = st.rec[i];
            st.loc[i] = -1;
        }
    }
    __syncthreads();
    for (int h = threadIdx.x; h < NB; h += blockDim.x) {
        const unsigned long long key = st.key[h];
        if (key != ~0ull) {
            const Scratch<T> &s = sc_of((int)(key >> 32));
            st.base[h] = atomicAdd(&s.rcnt[(int)(key & 0xffffffffull)], st.cnt[h]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int lc = st.loc[i];
        if (lc < 0) continue;
        const int h = lc >> 16;
        const unsigned long long key = st.key[h];
        const Scratch<T> &s = sc_of((int)(key >> 32));
        const int br = (int)(key & 0xffffffffull);
        const int pos = st.base[h] + (lc & 0xffff);
        if (pos < s.rcap[br]) s.rec[s.roff[br] + pos] = st.rec[i];
    }
    __syncthreads();
    for (int h = threadIdx.x; h < NB; h += blockDim.x) { st.key[h] = ~0ull; st.cnt[h] = 0; }
    if (threadIdx.x == 0) st.n = 0;
    __syncthreads();
}

// What a visited cell feeds: the segment's two weight sums (SC = false), or
// in the scatter form of the projection the cell's momentum source, added
// to S with atomics (SC = true; the sums of what was added feed the totals).
template <typename T, bool SC> struct WSink;
template <typename T> struct WSink<T, false> {
    Acc<T> wa, wb;
    // rmode: each pair is also recorded in its brick's region for the spread
    Rec<T> *rec = nullptr;
    int *rcnt;
    const int *rcap;
    const long long *roff;
    int ka, nbx, nby, bzs;
    RecStage<T> *st = nullptr;   // the CTA's staging (null: each record reserves its slot)
    bool plan_ok = false;        // regions sized for this brick height: write; otherwise only count
    int q = 0;                   // instance index (key of the staging)
    __device__ __forceinline__ void add(const GridC &g, const StepPtrs<T> &p, const int cg[3], T eta, T s) {
        T a, b;
        pair_w(eta, s, a, b);
        add_w(g, p, cg, a, b);
    }
    __device__ __forceinline__ void add_w(const GridC &, const StepPtrs<T> &, const int cg[3], T a, T b) {
        wa.add(a);
        wb.add(b);
        if (rec && st && plan_ok) {
            const int br = (cg[0] >> 4) + nbx * ((cg[1] >> 4) + nby * (cg[2] >> bzs));
            // one shared-memory atomic for the lanes adding together
            const unsigned act = __activemask();
            const int lane = threadIdx.x & 31, lead = __ffs(act) - 1;
            int sbase = 0;
            if (lane == lead) sbase = atomicAdd(&st->n, __popc(act));
            sbase = __shfl_sync(act, sbase, lead);
            const int slot = sbase + __popc(act & ((1u << lane) - 1u));
            if (slot < RecStage<T>::CAP) {
                Rec<T> r;
                r.cell = ((cg[2] & ((1 << bzs) - 1)) << 8) | ((cg[1] & 15) << 4) | (cg[0] & 15);
                r.ka = ka; r.wa = a; r.wb = b;
                st->rec[slot] = r;
                st->rk[slot] = ((unsigned long long)(unsigned)q << 32) | (unsigned)br;
                return;
            }
        }
        if (rec) {
            // the lanes adding to one brick take consecutive slots with one atomic
            const int br = (cg[0] >> 4) + nbx * ((cg[1] >> 4) + nby * (cg[2] >> bzs));
            const int cell = ((cg[2] & ((1 << bzs) - 1)) << 8) | ((cg[1] & 15) << 4) | (cg[0] & 15);
            const unsigned act = __activemask();
            const unsigned grp = __match_any_sync(act, br);
            const int lane = threadIdx.x & 31, lead = __ffs(grp) - 1;
            int base = 0;
            if (lane == lead) base = atomicAdd(&rcnt[br], __popc(grp));
            base = __shfl_sync(grp, base, lead);
            const int pos = base + __popc(grp & ((1u << lane) - 1u));
            if (plan_ok && pos < rcap[br]) {
                Rec<T> r;
                r.cell = cell; r.ka = ka; r.wa = a; r.wb = b;
                rec[roff[br] + pos] = r;
            }
        }
    }
};
template <typename T> struct WSink<T, true> {
    T fa[3], fb[3];
    Acc<T> sum[3];
    int nsupp = 0;
    __device__ __forceinline__ void add(const GridC &g, const StepPtrs<T> &p, const int cg[3], T eta, T s) {
        T wa, wb;
        pair_w(eta, s, wa, wb);
        add_w(g, p, cg, wa, wb);
    }
    __device__ __forceinline__ void add_w(const GridC &g, const StepPtrs<T> &p, const int cg[3], T wa, T wb) {
        const long long idx = cg[0] + (long long)g.nx * (cg[1] + (long long)g.ny * cg[2]);
        for (int a = 0; a < 3; ++a) {
            const T v = -pair_src(wa, wb, fa[a], fb[a]);
            atomicAdd(&p.S[a][idx], v);
            sum[a].add(v);
        }
        ++nsupp;
    }
};

// "segment k closer than k-1" from float-float node positions (defined with
// the projection kernels below)
static __device__ __noinline__ int ff_later_closer(const float *uhi, const float *ulo, long long np, int k, int B0,
                                                   int B1, int B2, float cx, float cy, float cz);

// near-tie re-decision of "segment k closer than k-1" for a cell at C
// (relative to the integer origin O): float-float for FP32 instances, FP64
// where that does not decide, and for FP64 instances
template <typename T>
__device__ __noinline__ bool w_later_closer(const GridC &g, const Scratch<T> &sc, const StepPtrs<T> &p, int k,
                                            const int O[3], T c0, T c1, T c2, int *status) {
    if (sizeof(T) == 4) {
        const int r = ff_later_closer((const float *)sc.uhi, sc.ulo, (long long)p.np, k, O[0], O[1], O[2],
                                      (float)c0, (float)c1, (float)c2);
        if (r >= 0) return r == 1;
    }
    atomicAdd(&status[ST_REFINED], 1);
    return later_closer_f64(g, p, k, ifloor(c0) + O[0], ifloor(c1) + O[1], ifloor(c2) + O[2]);
}

// membership of the cell at C (relative to c.O) in segment c.k's share, and
// what it feeds
template <typename T, bool SC, bool INTEG>
__device__ __forceinline__ void w_cell(const WSeg<T> &c, const T C[3], const GridC &g,
                                       const Scratch<T> &sc, const StepPtrs<T> &p, bool regular,
                                       int *status, WSink<T, SC> &sink) {
    // global cell index, needed only by the FP64 re-decisions (rare)
#define AL_CG(a) (ifloor(C[a]) + c.O[a])
    // offsets from the start node (origin O) and from the end node (its own
    // origin O1): the test at a node's bisector plane is evaluated from that
    // node's origin, so the two segments meeting there take the same
    // decision bit for bit and exactly one of them keeps the cell
    T x[3], C1[3], y[3];
    for (int a = 0; a < 3; ++a) {
        x[a] = C[a] - c.A[a];
        C1[a] = C[a] + (T)(c.O[a] - c.O1[a]);
        y[a] = C1[a] - c.B1[a];
    }
    if (regular) {
        if (c.has_lo) {
            const T sg = dot_r(x, c.m0), gs = c.gsb;
            bool pos;
            if (sg > gs) pos = true;
            else if (sg < -gs) pos = false;
            else pos = w_later_closer(g, sc, p, c.k, c.O, C[0], C[1], C[2], status);
            if (!pos) return;
        }
        if (c.has_hi) {
            const T sg = dot_r(y, c.m1), gs = c.gsb;
            bool pos;
            if (sg > gs) pos = true;
            else if (sg < -gs) pos = false;
            else pos = w_later_closer(g, sc, p, c.k + 1, c.O1, C1[0], C1[1], C1[2], status);
            if (pos) return;
        }
    }
    T s, r2;
    foot_sr(x, c.D, c.il2, s, r2);
    if (s >= (T)1 && c.kb != c.k) r2 = norm2_r(y);         // foot on the end node
    bool in;
    if (r2 < c.R2 - c.gr) in = true;
    else if (r2 > c.R2 + c.gr) in = false;
    else { in = within_f64(g, p, c.eps, c.k, c.n, AL_CG(0), AL_CG(1), AL_CG(2)); atomicAdd(&status[ST_REFINED], 1); }
    if (!in) return;
    const int cg[3] = {AL_CG(0), AL_CG(1), AL_CG(2)};
#undef AL_CG
    if constexpr (INTEG) {                                  // the segment's integrated kernel
        T a, b;
        pair_int(sc, (long long)p.np, c.k, cg, c.epsc, c.eta0, c.ie2, a, b);
        sink.add_w(g, p, cg, a, b);
        return;
    }
    const T eta = c.eta0 * Tr<T>::ex2(-r2 * c.ie2);
    sink.add(g, p, cg, eta, s);
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
template <typename T, int AX, bool SC, bool INTEG>
__device__ __forceinline__ void w_columns(const WSeg<T> &c, const GridC &g, const Scratch<T> &sc,
                                          const StepPtrs<T> &p, int *status, const int lane,
                                          WSink<T, SC> &sink) {
    constexpr int PA = (AX + 1) % 3, PB = (AX + 2) % 3;
    const int na = c.hi[PA] - c.lo[PA] + 1, nbb = c.hi[PB] - c.lo[PB] + 1;
    const int ncol = na * nbb;
    if (lane >= ncol) return;
    // this lane's first column; later columns by stepping 32 (float
    // coordinates advance with exact additions, no conversions in the loop)
    int ia = lane % na, ib = lane / na;                       // offsets from lo
    T fa = (T)(c.lo[PA] + ia - c.O[PA]) + (T)0.5, fb = (T)(c.lo[PB] + ib - c.O[PB]) + (T)0.5;
    const T fna = (T)na;
    const T clo0 = (T)(c.lo[AX] - c.O[AX]) + (T)0.5, chi0 = (T)(c.hi[AX] - c.O[AX]) + (T)0.5;
    const bool p0 = c.has_lo && c.m0[AX] != (T)0, p1 = c.has_hi && c.m1[AX] != (T)0;
    const T i0 = p0 ? (T)1 / c.m0[AX] : (T)0, i1 = p1 ? (T)1 / c.m1[AX] : (T)0;
    // the segment projected along the march axis: a column farther than 3 eps
    // from it in the plane has no cell within 3 eps of the segment
    const T ua = c.D[PA], ub = c.D[PB];
    const T uu = ua * ua + ub * ub, iuu = uu > (T)0 ? (T)1 / uu : (T)0;
    const T lim = c.R2 + c.gr;
    for (int col = lane; col < ncol; col += 32) {
        T C[3];
        C[PA] = fa;
        C[PB] = fb;
        {
            const T qa = fa - c.A[PA], qb = fb - c.A[PB];
            T t = (qa * ua + qb * ub) * iuu;
            t = t < (T)0 ? (T)0 : (t > (T)1 ? (T)1 : t);
            const T ea = qa - t * ua, eb = qb - t * ub;
            if (ea * ea + eb * eb > lim) goto next_column;
        }
        {
        // march-axis interval between the two planes (pruning only; the
        // membership test decides)
        T clo = clo0, chi = chi0;
        if (p0) {
            T r = c.A[AX] - ((C[PA] - c.A[PA]) * c.m0[PA] + (C[PB] - c.A[PB]) * c.m0[PB]) * i0;
            if (c.m0[AX] > (T)0) clo = tmax(clo, r - (T)0.05); else chi = tmin(chi, r + (T)0.05);
        }
        if (p1) {
            T r = c.Bn[AX] - ((C[PA] - c.Bn[PA]) * c.m1[PA] + (C[PB] - c.Bn[PB]) * c.m1[PB]) * i1;
            if (c.m1[AX] > (T)0) chi = tmin(chi, r + (T)0.05); else clo = tmax(clo, r - (T)0.05);
        }
        // cell centres k + 1/2 inside [clo, chi] and inside the box
        const T z0 = tmax(fceil_f(clo - (T)0.5) + (T)0.5, clo0);
        const T z1 = tmin(ffloor_f(chi - (T)0.5) + (T)0.5, chi0);
        for (T z = z0; z <= z1; z += (T)1) {
            C[AX] = z;
            w_cell<T, SC, INTEG>(c, C, g, sc, p, true, status, sink);
        }
        }
    next_column:
        ia += 32;
        fa += (T)32;
        while (ia >= na) { ia -= na; fa -= fna; ++ib; fb += (T)1; }
    }
}

// the segment's two weight sums (in units of V): a float-float pair in the
// slot's 8 bytes for FP32 instances (combined in FP64 per node by
// k_normalise), a double for FP64 instances
__device__ __forceinline__ void w_store(double *slot, const Acc<float> &a) {
    float h = a.s, l = -a.c;
    for (int o = 16; o > 0; o >>= 1) {
        float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
        float s, e;
        two_sum(h, oh, s, e);
        e = __fadd_rn(e, __fadd_rn(l, ol));
        fast_two_sum(s, e, h, l);
    }
    if ((threadIdx.x & 31) == 0) *reinterpret_cast<float2 *>(slot) = make_float2(h, l);
}
__device__ __forceinline__ void w_store(double *slot, const Acc<double> &a) {
    const double v = warp_total(a);
    if ((threadIdx.x & 31) == 0) *slot = v;
}
template <typename T> __device__ __forceinline__ double w_load(const double *slot);
template <> __device__ __forceinline__ double w_load<float>(const double *slot) {
    const float2 v = *reinterpret_cast<const float2 *>(slot);
    return (double)v.x + (double)v.y;
}
template <> __device__ __forceinline__ double w_load<double>(const double *slot) { return *slot; }

template <typename T>
__device__ __forceinline__ void w_finish(const GridC &, const Scratch<T> &sc, int *, int k, int,
                                         WSink<T, false> &sink) {
    w_store(&sc.segWa[k], sink.wa);
    w_store(&sc.segWb[k], sink.wb);
}
template <typename T>
__device__ __forceinline__ void w_finish(const GridC &, const Scratch<T> &sc, int *status, int, int lane,
                                         WSink<T, true> &sink) {
    double t[3];
    for (int a = 0; a < 3; ++a) t[a] = warp_total(sink.sum[a]);
    int ns = sink.nsupp;
    for (int o = 16; o > 0; o >>= 1) ns += __shfl_xor_sync(0xffffffffu, ns, o);
    if (lane == 0) {
        for (int a = 0; a < 3; ++a)
            if (t[a] != 0.0) atomicAdd(&sc.scatSum[a], t[a]);
        if (ns) atomicAdd(&status[ST_SUPPORT], ns);
    }
}

template <typename T, bool SC>
__device__ void d_weights(const GridC &g, const BeamsC &b, const Scratch<T> &sc, const StepPtrs<T> &p, int *status,
                          const int k, const int lane, RecStage<T> *st = nullptr, int q = 0) {
    if (!SC && g.wmode == 0) return;                        // all weights from the brick pass
    const long long np = b.n_points;
    const int l = b.line_of[k];
    const LineG lg = sc.lines[l];
    WSeg<T> c;
    c.k = k; c.off = lg.first; c.n = lg.n; c.q = k - c.off;
    if (c.n >= 2 && c.q == c.n - 1) return;                 // the tip starts no segment
    c.nseg = (c.n == 1) ? 1 : c.n - 1;
    c.kb = seg_end(k, c.n);
    if ((!lg.regular && !b.proj_mode) || (g.cm && lg.cm)) { // the brick or column-march passes take it
        if (!SC && lane == 0) { sc.segWa[k] = 0.0; sc.segWb[k] = 0.0; }   // zero in both encodings
        return;
    }
    c.klo = 0; c.khi = c.nseg - 1;
    c.eps = b.eps[l];
    for (int a = 0; a < 3; ++a) c.O[a] = ifloor(sc.uhi[a * np + k]);
    for (int a = 0; a < 3; ++a) {
        c.A[a] = rel(sc.uhi[a * np + k], sc.ulo[a * np + k], c.O[a]);
        c.Bn[a] = rel(sc.uhi[a * np + c.kb], sc.ulo[a * np + c.kb], c.O[a]);
        c.O1[a] = ifloor(sc.uhi[a * np + c.kb]);
        c.B1[a] = rel(sc.uhi[a * np + c.kb], sc.ulo[a * np + c.kb], c.O1[a]);
        c.D[a] = sc.segD[a * np + k];
    }
    c.il2 = sc.segIl2[k];
    // every cell of the segment's box lies within |D| + sqrt(3) (3 eps + 0.01)
    // cells of either node, so one band, taken at that distance, covers the
    // rounding of every bisector test of the segment (a wider band only sends
    // more near-plane cells to the exact re-decision)
    c.gsb = Tr<T>::gsig(tsqrt(c.D[0] * c.D[0] + c.D[1] * c.D[1] + c.D[2] * c.D[2]) + (T)1.75 * ((T)lg.Rc + (T)1));
    c.R2 = lgc<T>(lg.R2c, lg.R2f); c.gr = Tr<T>::grr(c.R2); c.ie2 = lgc<T>(lg.inv_eps2c_l2, lg.ie2f);
    c.eta0 = lgc<T>(lg.eta0, lg.eta0f);
    const int nn[3] = {g.nx, g.ny, g.nz};
    bool empty = false;
    for (int a = 0; a < 3; ++a) {
        T l0 = tmin(c.A[a], c.Bn[a]) - (T)lg.Rc - (T)0.01, h0 = tmax(c.A[a], c.Bn[a]) + (T)lg.Rc + (T)0.01;
        c.lo[a] = max(0, iceil(l0 - (T)0.5) + c.O[a]);
        c.hi[a] = min(nn[a] - 1, ifloor(h0 - (T)0.5) + c.O[a]);
        if (c.lo[a] > c.hi[a]) empty = true;
    }
    WSink<T, SC> sink;
    if constexpr (SC)
        for (int a = 0; a < 3; ++a) { sink.fa[a] = sc.fhat[a * np + k]; sink.fb[a] = sc.fhat[a * np + c.kb]; }
    else if (g.rmode) {
        sink.rec = sc.rec; sink.rcnt = sc.rcnt; sink.rcap = sc.rcap; sink.roff = sc.roff;
        sink.plan_ok = sc.rplan[0] == g.bz;
        sink.ka = k | (c.n == 1 ? REC_SINGLE : 0);
        sink.nbx = g.nbx; sink.nby = g.nby;
        sink.bzs = g.bz == 4 ? 2 : (g.bz == 8 ? 3 : 4);
        sink.st = st;
        sink.q = q;
    }
    // the integrated projection takes every segment within 3 eps: no
    // bisector planes bound a segment's cells
    const bool regular = lg.regular != 0 || b.proj_mode;
    c.integ = (b.proj_mode && c.n >= 2) ? 1 : 0;
    c.epsc = (T)(b.eps[l] / g.h);
    c.has_lo = !b.proj_mode && regular && c.q >= 1;
    c.has_hi = !b.proj_mode && regular && c.q + 1 <= c.n - 2;
    for (int a = 0; a < 3; ++a) {
        c.m0[a] = c.has_lo ? sc.nodeM[a * np + k] : (T)0;
        c.m1[a] = c.has_hi ? sc.nodeM[a * np + k + 1] : (T)0;
    }
    if (!empty && regular) {
        int ax = 0;
        if (tabs(c.D[1]) > tabs(c.D[ax])) ax = 1;
        if (tabs(c.D[2]) > tabs(c.D[ax])) ax = 2;
        // the integrated projection's cell loop is a separate instantiation, so
        // the nearest-segment loop carries no call to its kernel
        if (c.integ) {
            if constexpr (!SC) {
                if (ax == 0) w_columns<T, 0, SC, true>(c, g, sc, p, status, lane, sink);
                else if (ax == 1) w_columns<T, 1, SC, true>(c, g, sc, p, status, lane, sink);
                else w_columns<T, 2, SC, true>(c, g, sc, p, status, lane, sink);
            }
        } else {
            if (ax == 0) w_columns<T, 0, SC, false>(c, g, sc, p, status, lane, sink);
            else if (ax == 1) w_columns<T, 1, SC, false>(c, g, sc, p, status, lane, sink);
            else w_columns<T, 2, SC, false>(c, g, sc, p, status, lane, sink);
        }
    }
    w_finish(g, sc, status, k, lane, sink);
}

// ---------------------------------------------------------------------------
// k_normalise: w_k and f^_k = F_k / w_k
// ---------------------------------------------------------------------------
// Returns a bound (float bits, rounded up) on what node k contributes to one
// cell of S: eta0 |f^_k| (max over components), or |F_k| / V when it is
// deposited.
template <typename T>
__device__ unsigned int d_normalise(const GridC &g, const BeamsC &b, const Scratch<T> &sc, const StepPtrs<T> &p,
                                    int *status, const int k) {
    const long long np = b.n_points;
    const int l = b.line_of[k];
    const int off = b.line_off[l], n = b.line_off[l + 1] - off, q = k - off;
    double w = 0.0;
    const LineG &lg = sc.lines[l];
    if ((g.wmode == 0 || !lg.regular || (g.cm && lg.cm)) && !b.proj_mode) {
        // brick pass: fixed-point sum of omega eta / eta0; w = sum eta0 V 2^-wshift
        w = ldexp((double)sc.wfix[k], -lg.wshift) * (lg.eta0 * g.V);
    } else if (n == 1) {
        w = (w_load<T>(&sc.segWa[k]) + w_load<T>(&sc.segWb[k])) * g.V;
    } else {
        if (q >= 1) w += w_load<T>(&sc.segWb[k - 1]);
        if (q <= n - 2) w += w_load<T>(&sc.segWa[k]);
        w *= g.V;
    }
    sc.w[k] = w;
    double mb = 0.0;
    if (w > 0.0) {
        const T wt = (T)w;                         // FP64 sum, divided in the field precision
        for (int a = 0; a < 3; ++a) {
            const T fh = p.F[a][k] / wt;
            sc.fhat[a * np + k] = fh;
            mb = fmax(mb, fabs((double)fh));
        }
        mb *= lg.eta0;
    } else {
        for (int a = 0; a < 3; ++a) mb = fmax(mb, fabs((double)p.F[a][k]));
        mb /= g.V;
        // w_k = 0: the spread deposits F_k in the cell containing the node
        for (int a = 0; a < 3; ++a) sc.fhat[a * np + k] = (T)0;
        *sc.anyZero = 1;
        atomicAdd(&status[ST_ZERO_WEIGHT], 1);
        const int nn[3] = {g.nx, g.ny, g.nz};
        bool ins = true;
        for (int a = 0; a < 3; ++a) ins = ins && inside_axis(sc.uhi[a * np + k], sc.ulo[a * np + k], nn[a]);
        if (!ins) atomicAdd(&status[ST_DEPOSIT_LOST], 1);
    }
    cm_write_fhat(sc, np, k, w);
    // rounded up to float with a relative margin (covers FP32 rounding of the products)
    return __float_as_uint(fminf(__double2float_ru(mb * 1.0000005), 3.0e38f));
}

// ---------------------------------------------------------------------------
// k_spread: Eq. almMomentumSource as a cell-centric gather per brick
// ---------------------------------------------------------------------------
template <typename T> struct SpreadCap;
template <> struct SpreadCap<float> { static constexpr int NODES = 640, LIST = 512, ENT = 32; };
template <> struct SpreadCap<double> { static constexpr int NODES = 320, LIST = 512, ENT = 32; };

template <typename T, int BZ, bool FX>
struct SpreadSmem {
    using AccT = typename std::conditional<FX, long long, T>::type;
    static constexpr int NN = SpreadCap<T>::NODES, LIST = SpreadCap<T>::LIST, ENT = SpreadCap<T>::ENT;
    T P[3][NN];                  // node positions relative to the brick origin
    T M[3][NN];                  // node bisectors
    T D[3][NN];                  // segment vectors
    T Il2[NN];
    float Tau[NN];               // tan(theta_k / 2) at the nodes (0 at the line's ends)
    T Ls[NN];                    // length |D| of the segment starting at the node, in cells
    union {
        struct {
            T Fh[3][NN];         // spread: f^ at the nodes
            int sk[NN];          // spread: global node index of each staged node
            AccT acc[BZ][3][BX * BY];   // spread: S of the brick's cells (FX: fixed point, 2^-sh)
        } s;
        unsigned long long wq[NN];   // weights pass: fixed-point w of the staged nodes
    } u;
    unsigned char zf[NN];        // spread: the node has w_k = 0 (deposit)
    int list[LIST];              // candidate lines of this brick (line order)
    int nlist, nbatch, nstaged, more;
    int e_line[ENT], e_jlo[ENT], e_jhi[ENT], e_base[ENT], e_reg[ENT], e_n[ENT], e_first[ENT];
    float e_lo[ENT][3], e_hi[ENT][3];
    T e_R2[ENT], e_gr[ENT], e_ie2[ENT], e_eta0[ENT];
    float e_cz[ENT];             // min |D_z| / |D| over the candidates (0: no crossing test)
    float e_rad[ENT];            // R + curvature slack, cells
    float e_rho2[ENT];           // regular == 2: squared start radius
    int e_canon[ENT];            // the line's weights come from the segment pass: its pairs take its values
    // per line and layer: where the line crosses the layer's height, the
    // horizontal radius beyond which no cell of the layer is within 3 eps,
    // the crossing segment, and the fractional segment index at the crossing
    // with its gradient in the layer (the walk starts near the foot)
    float l_xc[ENT][BZ], l_yc[ENT][BZ], l_rh2[ENT][BZ];
    float l_ac[ENT][BZ], l_gx[ENT][BZ], l_gy[ENT][BZ];
    int l_jc[ENT][BZ];
    double red[3][SPREAD_THREADS / 32];
    int redi[SPREAD_THREADS / 32];
};

// rare paths of the gather, kept out of line so the cell loop stays small

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
template <typename T>
__device__ __noinline__ int nl_argmin(const GridC &g, const StepPtrs<T> &p, int k0, int k1, int n, int ci, int cj,
                                      int ck, int *status) {
    atomicAdd(&status[ST_REFINED], 1);
    return argmin_f64(g, p, k0, k1, n, ci, cj, ck);
}
// closest segment over [first + jlo, first + jhi] by exhaustive search from
// global memory (lines longer than the shared-memory stage); returns the
// line-local segment index
template <typename T>
__device__ __noinline__ int nl_exhaustive(const GridC &g, const Scratch<T> &sc, const StepPtrs<T> &p, int first,
                                          int n, int jlo, int jhi, T c0, T c1, T c2, int B0, int B1, int B2,
                                          int ci, int cj, int ck, int *status) {
    const long long np = p.np;
    const T C[3] = {c0, c1, c2};
    const int B[3] = {B0, B1, B2};
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
    if (!(second - best > Tr<T>::grr(best))) js = nl_argmin(g, p, first + jlo, first + jhi, n, ci, cj, ck, status) - first;
    return js;
}
// the same over the staged candidate segments.  A near tie between the two
// closest segments that share a node is decided by the float-float test of
// the pair (ff_later_closer, defined below); other near ties by the FP64
// argmin.
template <typename T, typename SMT>
__device__ __noinline__ int nl_exhaustive_staged(const SMT &sm, const GridC &g, const StepPtrs<T> &p,
                                                 const Scratch<T> &sc, int base, int first, int n, int jlo, int jhi,
                                                 T c0, T c1, T c2, int B0, int B1, int B2, int ci, int cj, int ck,
                                                 int *status) {
    T best = (T)INFINITY, second = (T)INFINITY, third = (T)INFINITY;
    int js = jlo, j2 = jlo;
    for (int jj = jlo; jj <= jhi; ++jj) {
        const int ss = base + (jj - jlo);
        const T x0 = c0 - sm.P[0][ss], x1 = c1 - sm.P[1][ss], x2 = c2 - sm.P[2][ss];
        const T d0 = sm.D[0][ss], d1 = sm.D[1][ss], d2 = sm.D[2][ss];
        T t = (x0 * d0 + x1 * d1 + x2 * d2) * sm.Il2[ss];
        t = t < (T)0 ? (T)0 : (t > (T)1 ? (T)1 : t);
        const T e0 = x0 - t * d0, e1 = x1 - t * d1, e2 = x2 - t * d2;
        const T dd = e0 * e0 + e1 * e1 + e2 * e2;
        if (dd < best) { third = second; second = best; j2 = js; best = dd; js = jj; }
        else if (dd < second) { third = second; second = dd; j2 = jj; }
        else if (dd < third) third = dd;
    }
    const T band = Tr<T>::grr(best);
    if (!(second - best > band)) {
        int r = -1;
        if (sizeof(T) == 4 && third - best > band && abs(js - j2) == 1 && n >= 3) {
            const int k = max(js, j2);                  // decide d_k < d_{k-1}
            r = ff_later_closer((const float *)sc.uhi, sc.ulo, (long long)p.np, first + k, B0, B1, B2,
                                (float)c0, (float)c1, (float)c2);
            if (r >= 0) js = r ? k : k - 1;
        }
        if (r < 0) js = nl_argmin(g, p, first + jlo, first + jhi, n, ci, cj, ck, status) - first;
    }
    return js;
}

// float-float arithmetic for the near-tie decisions of FP32 instances
__device__ __forceinline__ void ff_norm(float &h, float &l) { fast_two_sum(h, l, h, l); }
__device__ __forceinline__ void ffs_sub(float ah, float al, float bh, float bl, float &rh, float &rl) {
    float s, e;
    two_sum(ah, -bh, s, e);
    e = __fadd_rn(e, __fsub_rn(al, bl));
    fast_two_sum(s, e, rh, rl);
}
__device__ __forceinline__ void ffs_mul(float ah, float al, float bh, float bl, float &rh, float &rl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    fast_two_sum(p, e, rh, rl);
}
__device__ __forceinline__ void ffs_add(float ah, float al, float bh, float bl, float &rh, float &rl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    fast_two_sum(s, e, rh, rl);
}
__device__ __forceinline__ void ffs_dot3(const float xh[3], const float xl[3], const float yh[3], const float yl[3],
                                         float &rh, float &rl) {
    ffs_mul(xh[0], xl[0], yh[0], yl[0], rh, rl);
    for (int a = 1; a < 3; ++a) {
        float ph, pl;
        ffs_mul(xh[a], xl[a], yh[a], yl[a], ph, pl);
        ffs_add(rh, rl, ph, pl, rh, rl);
    }
}

// "segment k closer to C than segment k-1" for a cell near the bisector
// plane of node k, from the float-float node positions (about 44 bits).
// With a = C - P_k, A = a . D_k and B = a . D_{k-1}: the foot on segment k
// lies past P_k iff A > 0, the foot on segment k-1 lies before P_k iff
// B < 0, and when both are interior d_{k-1}^2 - d_k^2 has the sign of
// A^2 |D_{k-1}|^2 - B^2 |D_k|^2.  When both feet sit on P_k the distances
// are equal and either segment gives the same contribution (the lower index
// is kept).  Returns 1 / 0, or -1 where the float-float margin does not
// decide (the FP64 evaluation then decides).
static __device__ __noinline__ int ff_later_closer(const float *uhi, const float *ulo, long long np, int k, int B0, int B1,
                                            int B2, float cx, float cy, float cz) {
    const int Bv[3] = {B0, B1, B2};
    const float C[3] = {cx, cy, cz};
    float ph[3][3], pl[3][3];                       // nodes k-1, k, k+1 relative to the brick origin
    for (int n = 0; n < 3; ++n)
        for (int a = 0; a < 3; ++a) {
            float h = __fsub_rn(uhi[a * np + k - 1 + n], (float)Bv[a]);   // exact: |uh| < 2^24, B integer
            float l = ulo[a * np + k - 1 + n];
            ff_norm(h, l);
            ph[n][a] = h;
            pl[n][a] = l;
        }
    float ah[3], al[3], kh[3], kl[3], mh[3], ml[3];
    for (int a = 0; a < 3; ++a) {
        ffs_sub(C[a], 0.0f, ph[1][a], pl[1][a], ah[a], al[a]);
        ffs_sub(ph[2][a], pl[2][a], ph[1][a], pl[1][a], kh[a], kl[a]);    // D_k
        ffs_sub(ph[1][a], pl[1][a], ph[0][a], pl[0][a], mh[a], ml[a]);    // D_{k-1}
    }
    float Ah, Al, Bh, Bl, L2h, L2l, L1h, L1l;       // a . D_k, a . D_{k-1}, |D_k|^2, |D_{k-1}|^2
    ffs_dot3(ah, al, kh, kl, Ah, Al);
    ffs_dot3(ah, al, mh, ml, Bh, Bl);
    ffs_dot3(kh, kl, kh, kl, L2h, L2l);
    ffs_dot3(mh, ml, mh, ml, L1h, L1l);
    if (!(Ah < L2h) || !(-Bh < L1h)) return -1;     // a foot clamped at the far end: not decided here
    if (Ah <= 0.0f && Bh >= 0.0f) return 0;         // both feet on P_k: equal distances
    if (Ah > 0.0f && Bh >= 0.0f) return 1;          // only segment k's foot is interior
    if (Ah <= 0.0f && Bh < 0.0f) return 0;          // only segment k-1's foot is interior
    float t1h, t1l, t2h, t2l, lh, ll, rh, rl, dh, dl;
    ffs_mul(Ah, Al, Ah, Al, t1h, t1l);
    ffs_mul(t1h, t1l, L1h, L1l, lh, ll);
    ffs_mul(Bh, Bl, Bh, Bl, t2h, t2l);
    ffs_mul(t2h, t2l, L2h, L2l, rh, rl);
    ffs_sub(lh, ll, rh, rl, dh, dl);
    if (fabsf(dh) <= 1e-11f * fmaxf(lh, rh)) return -1;
    return dh > 0.0f ? 1 : 0;
}

template <typename T, typename SMT>
__device__ __forceinline__ bool sig_pos(const SMT &sm, int s, const T C[3], const GridC &g,
                                        const StepPtrs<T> &p, const Scratch<T> &sc, int kglob, int B0, int B1,
                                        int B2, int ci, int cj, int ck, int *status) {
    const T x0 = C[0] - sm.P[0][s], x1 = C[1] - sm.P[1][s], x2 = C[2] - sm.P[2][s];
    const T sg = x0 * sm.M[0][s] + x1 * sm.M[1][s] + x2 * sm.M[2][s];
    const T gs = Tr<T>::gsig(tsqrt(x0 * x0 + x1 * x1 + x2 * x2));
    if (sg > gs) return true;
    if (sg < -gs) return false;
    if (sizeof(T) == 4) {
        const int r = ff_later_closer((const float *)sc.uhi, sc.ulo, (long long)p.np, kglob, B0, B1, B2,
                                      (float)C[0], (float)C[1], (float)C[2]);
        if (r >= 0) return r == 1;
    }
    return nl_later_closer(g, p, kglob, ci, cj, ck, status);
}
template <typename T, typename SMT>
__device__ __forceinline__ T node_d2(const SMT &sm, int s, const T C[3]) {
    const T x0 = C[0] - sm.P[0][s], x1 = C[1] - sm.P[1][s], x2 = C[2] - sm.P[2][s];
    return x0 * x0 + x1 * x1 + x2 * x2;
}
// clamped foot parameter and squared distance of C to staged segment ss
template <typename T, typename SMT>
__device__ __forceinline__ void seg_foot(const SMT &sm, int ss, const T C[3], T &s, T &r2) {
    const T x0 = C[0] - sm.P[0][ss], x1 = C[1] - sm.P[1][ss], x2 = C[2] - sm.P[2][ss];
    const T d0 = sm.D[0][ss], d1 = sm.D[1][ss], d2 = sm.D[2][ss];
    s = (x0 * d0 + x1 * d1 + x2 * d2) * sm.Il2[ss];
    s = s < (T)0 ? (T)0 : (s > (T)1 ? (T)1 : s);
    const T e0 = x0 - s * d0, e1 = x1 - s * d1, e2 = x2 - s * d2;
    r2 = e0 * e0 + e1 * e1 + e2 * e2;
}

// seg_foot also returning the unclamped foot parameter
template <typename T, typename SMT>
__device__ __forceinline__ void seg_foot_raw(const SMT &sm, int ss, const T C[3], T &sraw, T &s, T &r2) {
    const T x0 = C[0] - sm.P[0][ss], x1 = C[1] - sm.P[1][ss], x2 = C[2] - sm.P[2][ss];
    const T d0 = sm.D[0][ss], d1 = sm.D[1][ss], d2 = sm.D[2][ss];
    sraw = (x0 * d0 + x1 * d1 + x2 * d2) * sm.Il2[ss];
    s = sraw < (T)0 ? (T)0 : (sraw > (T)1 ? (T)1 : sraw);
    const T e0 = x0 - s * d0, e1 = x1 - s * d1, e2 = x2 - s * d2;
    r2 = e0 * e0 + e1 * e1 + e2 * e2;
}

// One brick of cells and the lines near it.  WP = false: the momentum source
// (Eq. almMomentumSource) of every cell of the brick, written once per cell
// by the thread that owns its column (no atomics), with the deposits of the
// zero-weight nodes inside the brick.  WP = true: the nodal weights w_k
// (Sec. 3.2.4), each (cell, line) pair once, added as fixed-point integers.
// subtract a source from a cell's accumulator: as a fixed-point integer
// (FX) or in the field precision
template <bool FX, typename A, typename T>
__device__ __forceinline__ void acc_sub(A &acc, T v, int fsh) {
    if constexpr (FX) acc -= to_fixed_s(v, fsh);
    else acc -= v;
}

// The mirror images of cell (tx, ty, z) of the brick beyond the reflecting
// faces within reach of it (b.reflect), for line entry e: each image is a
// ghost cell whose pair with the line is found and weighed like a grid
// cell's (exhaustive closest segment, the same in/out decision, the same
// per-pair values in both brick passes), and its share goes to the cell it
// mirrors.  A ghost farther than 3 eps + 1 cell from the face cannot be
// within 3 eps of a line inside the grid.  Returns the pairs within 3 eps.
template <typename T, bool WP, int BZ, bool FX>
__device__ __forceinline__ int d_images(const GridC &g, const BeamsC &b, const Scratch<T> &sc, const StepPtrs<T> &p,
                                     int *status, SpreadSmem<T, BZ, FX> &sm, int e, int z, int tx, int ty, int B0,
                                     int B1, int B2, int fsh) {
    const long long np = b.n_points;
    const int gc[3] = {B0 + tx, B1 + ty, B2 + z}, nn[3] = {g.nx, g.ny, g.nz}, Bv[3] = {B0, B1, B2};
    const int jlo = sm.e_jlo[e], jhi = sm.e_jhi[e], base = sm.e_base[e], first = sm.e_first[e], n = sm.e_n[e];
    const T R2 = sm.e_R2[e], gr = sm.e_gr[e], ie2 = sm.e_ie2[e], e0v = sm.e_eta0[e];
    const int G = (int)ceilf(sqrtf((float)R2)) + 1;
    int opt[3][3], nopt[3];
    for (int a = 0; a < 3; ++a) {
        nopt[a] = 1;
        opt[a][0] = gc[a];
        if (((b.reflect >> (2 * a)) & 1) && gc[a] < G) opt[a][nopt[a]++] = -1 - gc[a];
        if (((b.reflect >> (2 * a + 1)) & 1) && gc[a] > nn[a] - 1 - G) opt[a][nopt[a]++] = 2 * nn[a] - 1 - gc[a];
    }
    if (nopt[0] * nopt[1] * nopt[2] == 1) return 0;
    const int c = ty * BX + tx;
    int ns = 0;
    for (int i0 = 0; i0 < nopt[0]; ++i0)
        for (int i1 = 0; i1 < nopt[1]; ++i1)
            for (int i2 = 0; i2 < nopt[2]; ++i2) {
                if (i0 == 0 && i1 == 0 && i2 == 0) continue;             // the cell itself
                const int gi[3] = {opt[0][i0], opt[1][i1], opt[2][i2]};
                T C[3];
                for (int a = 0; a < 3; ++a) C[a] = (T)(gi[a] - Bv[a]) + (T)0.5;
                int js;
                T s, r2;
                if (base >= 0) {
                    js = nl_exhaustive_staged(sm, g, p, sc, base, first, n, jlo, jhi, C[0], C[1], C[2], B0, B1, B2,
                                              gi[0], gi[1], gi[2], status);
                    seg_foot(sm, base + (js - jlo), C, s, r2);
                } else {
                    js = nl_exhaustive(g, sc, p, first, n, jlo, jhi, C[0], C[1], C[2], B0, B1, B2, gi[0], gi[1],
                                       gi[2], status);
                    const int ka = first + js;
                    T x[3], Dj[3];
                    for (int a = 0; a < 3; ++a) {
                        x[a] = C[a] - rel(sc.uhi[a * np + ka], sc.ulo[a * np + ka], Bv[a]);
                        Dj[a] = sc.segD[a * np + ka];
                    }
                    s = (x[0] * Dj[0] + x[1] * Dj[1] + x[2] * Dj[2]) * sc.segIl2[ka];
                    s = s < (T)0 ? (T)0 : (s > (T)1 ? (T)1 : s);
                    const T f0 = x[0] - s * Dj[0], f1 = x[1] - s * Dj[1], f2 = x[2] - s * Dj[2];
                    r2 = f0 * f0 + f1 * f1 + f2 * f2;
                }
                bool in;
                if (r2 < R2 - gr) in = true;
                else if (r2 > R2 + gr) in = false;
                else in = nl_within(g, p, b.eps[sm.e_line[e]], first + js, n, gi[0], gi[1], gi[2], status);
                if (!in) continue;
                ++ns;
                const T q = Tr<T>::ex2(-r2 * ie2);
                const int ka = first + js, kb = seg_end(ka, n);
                if constexpr (!WP) {
                    T fa[3], fb[3];
                    if (base >= 0) {
                        const int ss = base + (js - jlo), sb = (n == 1) ? ss : ss + 1;
                        for (int a = 0; a < 3; ++a) { fa[a] = sm.u.s.Fh[a][ss]; fb[a] = sm.u.s.Fh[a][sb]; }
                    } else {
                        for (int a = 0; a < 3; ++a) { fa[a] = sc.fhat[a * np + ka]; fb[a] = sc.fhat[a * np + kb]; }
                    }
                    T wa, wb;
                    pair_w(e0v * q, s, wa, wb);
                    for (int a = 0; a < 3; ++a) acc_sub<FX>(sm.u.s.acc[z][a][c], pair_src(wa, wb, fa[a], fb[a]), fsh);
                } else {
                    const int sh = (int)e0v;
                    const unsigned long long va = to_fixed(q * ((T)1 - s), sh), vb = to_fixed(q * s, sh);
                    if (base >= 0) {
                        const int na = base + (js - jlo), nb2 = (n == 1) ? na : na + 1;
                        if (va) atomicAdd(&sm.u.wq[na], va);
                        if (vb) atomicAdd(&sm.u.wq[nb2], vb);
                    } else {
                        atomicAdd(&sc.wfix[ka], va);
                        atomicAdd(&sc.wfix[kb], vb);
                    }
                }
            }
    return ns;
}

// The mirror-image phase of a batch (reflecting faces within reach of the
// brick): the cells the gather visited, with the same layer and row-pair
// ownership, so each cell is still updated by one warp only.  Kept out of
// line so the gather's cell loop is compiled as without it.
template <typename T, bool WP, int BZ, bool FX>
__device__ __forceinline__ int d_images_phase(const GridC &g, const BeamsC &b, const Scratch<T> &sc,
                                           const StepPtrs<T> &p, int *status, SpreadSmem<T, BZ, FX> &sm, int ne,
                                           int B0, int B1, int B2, int fsh) {
    constexpr int NW = SPREAD_THREADS / 32, WPL = (BZ < NW) ? NW / BZ : 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, zpart = warp % WPL;
    const int nzb = min(BZ, g.nz - B2), nxb = min(BX, g.nx - B0), nyb = min(BY, g.ny - B1);
    const int Bv[3] = {B0, B1, B2}, bs[3] = {BX, BY, BZ}, nn[3] = {g.nx, g.ny, g.nz};
    int ns = 0;
    for (int z = warp / WPL; z < nzb; z += NW / WPL) {
        const float czf = z + 0.5f;
        for (int e = 0; e < ne; ++e) {
            const int jlo = sm.e_jlo[e], jhi = sm.e_jhi[e];
            if (jhi < jlo || czf < sm.e_lo[e][2] || czf > sm.e_hi[e][2]) continue;
            // no cell of the brick within 3 eps + 1 cell of a reflecting face: no images
            const int G = (int)ceilf(sqrtf((float)sm.e_R2[e])) + 1;
            bool near = false;
            for (int a = 0; a < 3; ++a)
                near = near || (((b.reflect >> (2 * a)) & 1) && Bv[a] < G) ||
                       (((b.reflect >> (2 * a + 1)) & 1) && Bv[a] + bs[a] > nn[a] - G);
            if (!near) continue;
            float xlo = sm.e_lo[e][0], xhi = sm.e_hi[e][0], ylo = sm.e_lo[e][1], yhi = sm.e_hi[e][1];
            const float rh2 = sm.l_rh2[e][z], xc = sm.l_xc[e][z], yc = sm.l_yc[e][z];
            if (rh2 < 1e30f) {
                const float rh = sqrtf(rh2);
                xlo = fmaxf(xlo, xc - rh); xhi = fminf(xhi, xc + rh);
                ylo = fmaxf(ylo, yc - rh); yhi = fminf(yhi, yc + rh);
            }
            const int ix0 = max(0, (int)ceilf(fmaxf(xlo, -1.0f) - 0.5f));
            const int ix1 = min(nxb - 1, (int)floorf(fminf(xhi, (float)BX + 1.0f) - 0.5f));
            const int iy0 = max(0, (int)ceilf(fmaxf(ylo, -1.0f) - 0.5f));
            const int iy1 = min(nyb - 1, (int)floorf(fminf(yhi, (float)BY + 1.0f) - 0.5f));
            if (ix0 > ix1 || iy0 > iy1) continue;
            const int w = ix1 - ix0 + 1, ncell = w * (iy1 - iy0 + 1);
            for (int q = lane; q < ncell; q += 32) {
                const int tx = ix0 + q % w, ty = iy0 + q / w;
                if (WPL > 1 && ((ty >> 1) % WPL) != zpart) continue;
                const float dx = (tx + 0.5f) - xc, dy = (ty + 0.5f) - yc;
                if (dx * dx + dy * dy <= rh2) ns += d_images<T, WP, BZ, FX>(g, b, sc, p, status, sm, e, z, tx, ty, B0, B1, B2, fsh);
            }
        }
    }
    return ns;
}

template <typename T, bool WP, int BZ, bool FX, bool REFL = false>
__device__ void d_brick(const GridC &g, const BeamsC &b, const Scratch<T> &sc, const StepPtrs<T> &p, int *status,
                        const int br, SpreadSmem<T, BZ, FX> &sm) {
    using SM = SpreadSmem<T, BZ, FX>;
    const long long np = b.n_points;
    const int nbxy = g.nbx * g.nby;
    const int bzi = br / nbxy, rem = br - bzi * nbxy;
    const int byi = rem / g.nbx, bxi = rem - byi * g.nbx;
    const int B0 = bxi * BX, B1 = byi * BY, B2 = bzi * BZ;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (WP && g.wmode != 0 && *sc.anyIrr == 0 && !g.cm) return;   // the segment pass took every line
    if (WP && b.proj_mode) return;                           // the integrated projection: segment pass only
    const int nzb = min(BZ, g.nz - B2);              // layers of this brick inside the grid
    const int nxb = min(BX, g.nx - B0), nyb = min(BY, g.ny - B1);
    int nsupp = 0;                                   // (cell, line) pairs within 3 eps
    if (!WP)
        for (int i = threadIdx.x; i < BZ * 3 * BX * BY; i += SPREAD_THREADS) (&sm.u.s.acc[0][0][0])[i] = (typename SM::AccT)0;
    const int fsh = WP ? 0 : spread_shift(*sc.smax, (long long)b.n_points + b.n_lines);
    // replay: the certified lines' pairs of this brick as the segment pass
    // recorded them (complete when they fitted the brick's region), added in
    // fixed point, so in any order and with the bits the gather would give;
    // the gather below then takes only the lines without a certificate.  Not
    // when a node has w_k = 0 (its deposit goes with the gathered lines).
    bool replay = false;
    const int nrec_b = (!WP && g.rmode) ? sc.rcnt[br] : 0;
    if constexpr (FX)
    if (!WP && g.rmode && *sc.anyZero == 0 && sc.rplan[0] == g.bz) {
        const int nrec = nrec_b;
        if (nrec <= sc.rcap[br]) {
            replay = true;
            __syncthreads();                             // accumulators cleared
            const Rec<T> *rr = sc.rec + sc.roff[br];
            // four records per thread per round, their loads issued together
            constexpr int RU = 4;
            for (int r0 = threadIdx.x; r0 < nrec; r0 += RU * SPREAD_THREADS) {
                Rec<T> rc[RU];
                T fa[RU][3], fb[RU][3];
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int r = r0 + u * SPREAD_THREADS;
                    if (r < nrec) rc[u] = rr[r];
                    else { rc[u].cell = -1; rc[u].ka = 0; rc[u].wa = rc[u].wb = (T)0; }
                }
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int ka = rc[u].ka & ~REC_SINGLE, kb = (rc[u].ka & REC_SINGLE) ? ka : ka + 1;
                    const bool ok = rc[u].cell >= 0;
                    for (int a = 0; a < 3; ++a) {
                        fa[u][a] = ok ? sc.fhat[a * np + ka] : (T)0;
                        fb[u][a] = ok ? sc.fhat[a * np + kb] : (T)0;
                    }
                }
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    if (rc[u].cell < 0) continue;
                    const int z = rc[u].cell >> 8, c = rc[u].cell & 255;
                    for (int a = 0; a < 3; ++a) {
                        const long long v = to_fixed_s(pair_src(rc[u].wa, rc[u].wb, fa[u][a], fb[u][a]), fsh);
                        atomicAdd(reinterpret_cast<unsigned long long *>(&sm.u.s.acc[z][a][c]), (unsigned long long)(-v));
                    }
                }
            }
            if (threadIdx.x == 0 && nrec > 0) {
                nsupp += nrec;
                atomicAdd(&status[ST_REPLAYED], 1);
            }
        }
    }

    const int W = b.mask_words;
    uint32_t *mrow = sc.mask + (long long)br * W;
    const float blo[3] = {(float)B0, (float)B1, (float)B2};
    const float bhi[3] = {(float)(B0 + BX), (float)(B1 + BY), (float)(B2 + BZ)};

    // candidate lines in line order, up to LIST per pass: warp 0's lanes each
    // take a contiguous run of mask words, so a prefix over lanes keeps line
    // order; bricks with more than LIST candidates take several passes (the
    // spread clears the words in the last one)
    const bool keep_certified = WP ? (g.wmode == 0) : (g.smode == 0 && !replay);
    const bool keep_none = !WP && replay && b.proj_mode;     // integrated: the records hold every line
    const int wper = (W + 31) / 32;
    for (int pass = 0;; ++pass) {
        __syncthreads();
        if (warp == 0) {
            const int wa = min(W, lane * wper), wb = min(W, wa + wper);
            int cnt = 0;
            for (int w = wa; w < wb; ++w) {
                uint32_t m = keep_none ? 0u : mrow[w];
                if (!keep_certified && m) {              // the segment pass takes certified lines
                    uint32_t keep = 0u, t = m;
                    while (t) {
                        const int bit = __ffs(t) - 1;
                        t &= t - 1;
                        const LineG &lk = sc.lines[(w << 5) + bit];
                        // lines without a certificate, and column-march lines
                        // (neither recorded nor in the segment pass)
                        if (!lk.regular || (g.cm && lk.cm)) keep |= 1u << bit;
                    }
                    m = keep;
                }
                cnt += __popc(m);
            }
            int pre = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                int v = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre += v;
            }
            const int total = __shfl_sync(0xffffffffu, pre, 31);
            const int lo = pass * SM::LIST, hi = lo + SM::LIST;
            int pos = pre - cnt;
            if (pos < hi && pos + cnt > lo) {
                for (int w = wa; w < wb; ++w) {
                    uint32_t m = keep_none ? 0u : mrow[w];
                    while (m) {
                        const int bit = __ffs(m) - 1;
                        m &= m - 1;
                        const int l = (w << 5) + bit;
                        if (!keep_certified && sc.lines[l].regular && !(g.cm && sc.lines[l].cm)) continue;
                        if (pos >= lo && pos < hi) sm.list[pos - lo] = l;
                        ++pos;
                    }
                }
            }
            if (!WP && total <= hi)
                for (int w = wa; w < wb; ++w) mrow[w] = 0u;      // clear for the next step
            if (lane == 0) {
                sm.nlist = max(0, min(total - lo, SM::LIST));
                sm.more = total > hi;
            }
        }
        __syncthreads();
        const int nlist = sm.nlist;
        int li = 0;
        while (li < nlist) {
            // ---- batch: candidate segment ranges, one warp per line --------
            const int nb = min(nlist - li, SM::ENT);
            for (int e = warp; e < nb; e += SPREAD_THREADS / 32) {
                const int l = sm.list[li + e];
                const LineG lg = sc.lines[l];
                const int nseg = lg.n == 1 ? 1 : lg.n - 1;
                int jlo = 0x7fffffff, jhi = -1;
                float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
                float czp = 1.0f, czn = 1.0f;          // min D_z/|D| over up- and down-going candidates
                // the box a candidate's support must meet: the brick's, and with
                // reflecting faces within reach the boxes of its mirror images too
                float olo[3] = {blo[0], blo[1], blo[2]}, ohi[3] = {bhi[0], bhi[1], bhi[2]};
                if (REFL) {
                    const float gd = ceilf(lg.Rc) + 1.0f;
                    const float nnf[3] = {(float)g.nx, (float)g.ny, (float)g.nz};
                    for (int a = 0; a < 3; ++a) {
                        if (((b.reflect >> (2 * a)) & 1) && blo[a] < gd) olo[a] = fminf(olo[a], -bhi[a]);
                        if (((b.reflect >> (2 * a + 1)) & 1) && bhi[a] > nnf[a] - gd)
                            ohi[a] = fmaxf(ohi[a], 2.0f * nnf[a] - blo[a]);
                    }
                }
                for (int j = lane; j < nseg; j += 32) {
                    const int ka = lg.first + j;
                    float sl[3], sh[3];
                    seg_box(sc, np, ka, seg_end(ka, lg.n), lg.Rc, sl, sh);
                    bool ov = true;
                    for (int a = 0; a < 3; ++a) ov = ov && (sh[a] >= olo[a] && sl[a] <= ohi[a]);
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
                // climb rate of every segment of the candidate range [jlo, jhi]
                for (int j = jlo + lane; j <= jhi; j += 32) {
                    const int ka = lg.first + j;
                    const float dx = (float)sc.segD[ka], dy = (float)sc.segD[np + ka], dz = (float)sc.segD[2 * np + ka];
                    const float ln = sqrtf(dx * dx + dy * dy + dz * dz);
                    const float cz = ln > 0.0f ? dz / ln : 0.0f;
                    czp = fminf(czp, cz);
                    czn = fminf(czn, -cz);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    czp = fminf(czp, __shfl_xor_sync(0xffffffffu, czp, o));
                    czn = fminf(czn, __shfl_xor_sync(0xffffffffu, czn, o));
                }
                // candidates all climbing (or all descending) by at least 0.3 of their length:
                // cells within 3 eps of the line lie near where it crosses each layer
                const float czm = fmaxf(czp, czn);
                const float cz_ok = (lg.n >= 2 && czm > 0.3f) ? czm : 0.0f;
                if (lane == 0) {
                    sm.e_line[e] = l;
                    sm.e_jlo[e] = jlo;
                    sm.e_jhi[e] = jhi;
                    sm.e_reg[e] = (lg.regular == 2 && cz_ok <= 0.0f) ? 0 : lg.regular;
                    sm.e_n[e] = lg.n;
                    sm.e_first[e] = lg.first;
                    sm.e_R2[e] = lgc<T>(lg.R2c, lg.R2f);
                    sm.e_gr[e] = Tr<T>::grr(lgc<T>(lg.R2c, lg.R2f));
                    sm.e_ie2[e] = lgc<T>(lg.inv_eps2c_l2, lg.ie2f);
                    sm.e_eta0[e] = WP ? (T)lg.wshift : lgc<T>(lg.eta0, lg.eta0f);
                    sm.e_rho2[e] = lg.rho2;
                    sm.e_canon[e] = (g.wmode != 0 && lg.regular != 0 && !(g.cm && lg.cm)) ? 1 : 0;
                    for (int a = 0; a < 3; ++a) { sm.e_lo[e][a] = lo[a] - blo[a]; sm.e_hi[e][a] = hi[a] - blo[a]; }
                    sm.e_cz[e] = cz_ok;
                    if (cz_ok > 0.0f) {
                        // a cell of a layer within 3 eps of the line is within 3 eps + dev of the
                        // axis of the segment crossing that layer: the foot lies within an arc
                        // lam = 3 eps / cz + L_max of that segment, over which the polyline
                        // departs from the axis by at most lam min(1, (lam / L_min + 1) theta_max)
                        const float lam = lg.Rc / cz_ok + lg.Lmax;
                        const float turn = (lg.n >= 3 && lg.Lmin > 0.0f) ? (lam / lg.Lmin + 1.0f) * lg.thmax : 0.0f;
                        sm.e_rad[e] = lg.Rc + lam * fminf(1.0f, turn) + 0.02f;
                    }
                }
            }
            __syncthreads();
            // node budget: entries [li, li + ne) fit in shared memory
            if (threadIdx.x == 0) {
                int base = 0, e = 0;
                for (; e < nb; ++e) {
                    int cnt = sm.e_jhi[e] >= sm.e_jlo[e] ? sm.e_jhi[e] - sm.e_jlo[e] + 2 : 0;
                    if (base + cnt > SM::NN) break;
                    sm.e_base[e] = base;
                    base += cnt;
                }
                if (e == 0) { e = 1; sm.e_base[0] = -1; }  // one oversized line: global-memory path
                sm.nbatch = e;
                sm.nstaged = base;
            }
            __syncthreads();
            const int ne = sm.nbatch;
            // ---- stage the batch's nodes, all threads over all of them ---------
            // (slot s belongs to the last entry whose base is <= s: entries without
            // nodes share the next entry's base)
            for (int s = threadIdx.x; s < sm.nstaged; s += SPREAD_THREADS) {
                int lo = 0, hi = ne - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sm.e_base[mid] <= s) lo = mid; else hi = mid - 1;
                }
                const int e = lo, t = s - sm.e_base[e];
                const int first = sm.e_first[e], n = sm.e_n[e];
                const int kn = (n == 1) ? first : first + sm.e_jlo[e] + t;   // single-node line: copy the node
                for (int a = 0; a < 3; ++a) {
                    sm.P[a][s] = rel(sc.uhi[a * np + kn], sc.ulo[a * np + kn], (a == 0) ? B0 : (a == 1 ? B1 : B2));
                    sm.M[a][s] = sc.nodeM[a * np + kn];
                    sm.D[a][s] = sc.segD[a * np + kn];
                }
                sm.Il2[s] = sc.segIl2[kn];
                sm.Tau[s] = sc.nodeTau[kn];
                sm.Ls[s] = (T)1 / tsqrt(sc.segIl2[kn]);
                if (WP) {
                    sm.u.wq[s] = 0ull;
                } else {
                    for (int a = 0; a < 3; ++a) sm.u.s.Fh[a][s] = sc.fhat[a * np + kn];
                    sm.u.s.sk[s] = kn;
                    sm.zf[s] = (n != 1 || t == 0) && sc.w[kn] == 0.0;
                }
            }
            __syncthreads();
            // ---- where each line crosses each layer (one warp per line) --------
            for (int e = warp; e < ne; e += SPREAD_THREADS / 32) {
                const int jlo = sm.e_jlo[e], jhi = sm.e_jhi[e], base = sm.e_base[e];
                if (lane >= BZ) continue;
                const float cz = sm.e_cz[e];
                if (jhi < jlo || base < 0 || cz <= 0.0f) {
                    sm.l_rh2[e][lane] = 3.0e38f;               // no crossing test for this line
                    sm.l_xc[e][lane] = sm.l_yc[e][lane] = 0.0f;
                    sm.l_ac[e][lane] = (float)max(jlo, 0);
                    sm.l_gx[e][lane] = sm.l_gy[e][lane] = 0.0f;
                    sm.l_jc[e][lane] = max(jlo, 0);
                    continue;
                }
                const float zc = lane + 0.5f;
                // the candidate segment containing the height zc, else the end one nearest
                // to it: the candidates all climb (or all descend), so node heights are
                // monotone and a bisection finds it
                const float z0 = (float)sm.P[2][base], z1 = (float)sm.P[2][base + (jhi - jlo + 1)];
                const float sgn = z1 >= z0 ? 1.0f : -1.0f;
                int jc;
                if (sgn * (zc - z0) <= 0.0f) {
                    jc = jlo;
                } else if (sgn * (zc - z1) >= 0.0f) {
                    jc = jhi;
                } else {
                    int lo = jlo, hi = jhi;                    // largest j with sgn (z_j - zc) <= 0
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sgn * ((float)sm.P[2][base + (mid - jlo)] - zc) <= 0.0f) lo = mid; else hi = mid - 1;
                    }
                    jc = lo;
                }
                const int ss = base + (jc - jlo);
                const float d0 = (float)sm.D[0][ss], d1 = (float)sm.D[1][ss], dz = (float)sm.D[2][ss];
                const float t = (zc - (float)sm.P[2][ss]) / dz;      // |dz| >= 0.3 |D| > 0
                sm.l_xc[e][lane] = (float)sm.P[0][ss] + t * d0;
                sm.l_yc[e][lane] = (float)sm.P[1][ss] + t * d1;
                const float rh = sm.e_rad[e] / cz + 0.02f;
                sm.l_rh2[e][lane] = rh * rh;
                sm.l_jc[e][lane] = jc;
                // foot of a cell (dx, dy) away from the crossing, in segment units
                const float il2 = (float)sm.Il2[ss];
                sm.l_ac[e][lane] = (float)jc + t;
                sm.l_gx[e][lane] = d0 * il2;
                sm.l_gy[e][lane] = d1 * il2;
            }
            __syncthreads();
            // ---- gather: warp w takes layer w; for each line in order its lanes take
            //      the cells of the layer near the line, 32 at a time, so no two lanes
            //      share a cell and every cell sums its lines in line order ----
            // WPL warps share a layer (bricks lower than the warp count), taking
            // alternate row pairs; taller bricks give each warp several layers
            constexpr int NW = SPREAD_THREADS / 32, WPL = (BZ < NW) ? NW / BZ : 1;
            static_assert(BY <= 32 && (BY & (BY - 1)) == 0, "one lane per row, a power of two");
            const int zpart = warp % WPL;
            for (int z = warp / WPL; z < nzb; z += NW / WPL) {
                const float czf = z + 0.5f;
                const int gz = B2 + z;
                for (int e = 0; e < ne; ++e) {
                    const int jlo = sm.e_jlo[e], jhi = sm.e_jhi[e];
                    if (jhi < jlo || czf < sm.e_lo[e][2] || czf > sm.e_hi[e][2]) continue;
                    float xlo = sm.e_lo[e][0], xhi = sm.e_hi[e][0], ylo = sm.e_lo[e][1], yhi = sm.e_hi[e][1];
                    const float rh2 = sm.l_rh2[e][z], xc = sm.l_xc[e][z], yc = sm.l_yc[e][z];
                    if (rh2 < 1e30f) {
                        const float rh = sqrtf(rh2);
                        xlo = fmaxf(xlo, xc - rh); xhi = fminf(xhi, xc + rh);
                        ylo = fmaxf(ylo, yc - rh); yhi = fminf(yhi, yc + rh);
                    }
                    // columns whose centre i + 1/2 lies in [lo, hi], inside brick and grid
                    const int ix0 = max(0, (int)ceilf(fmaxf(xlo, -1.0f) - 0.5f));
                    const int ix1 = min(nxb - 1, (int)floorf(fminf(xhi, (float)BX + 1.0f) - 0.5f));
                    const int iy0 = max(0, (int)ceilf(fmaxf(ylo, -1.0f) - 0.5f));
                    const int iy1 = min(nyb - 1, (int)floorf(fminf(yhi, (float)BY + 1.0f) - 0.5f));
                    if (ix0 > ix1 || iy0 > iy1) continue;
                    const int base = sm.e_base[e], first = sm.e_first[e], n = sm.e_n[e], reg = sm.e_reg[e];
                    const T R2 = sm.e_R2[e], gr = sm.e_gr[e], ie2 = sm.e_ie2[e], e0v = sm.e_eta0[e];
                    const float rho2 = sm.e_rho2[e];
                    const float ac = sm.l_ac[e][z], gxv = sm.l_gx[e][z], gyv = sm.l_gy[e][z];
                    const int jcz = sm.l_jc[e][z];
                    // weights pass: per-lane sums for the four nodes around the crossing
                    // (slots w0s .. w0s + 3), reduced over the warp once per line and layer
                    unsigned long long wacc0 = 0ull, wacc1 = 0ull, wacc2 = 0ull, wacc3 = 0ull;
                    const int w0s = (base >= 0) ? base + (jcz - jlo) - 1 : 0;
                    // the cells to test, packed over the lanes: lane r takes row iy0 + r's
                    // run of columns (the disc around the crossing widened by a column on
                    // each side, so it holds every cell the disc test below passes), a
                    // scan places the runs end to end, and the lanes take cells q, q + 32,
                    // ... of that order.  Row pairs (2p, 2p + 1) belong to warp p % WPL of
                    // the layer, the same warp for every line, so a cell is only ever
                    // updated by one warp, once per line, in line order.
                    int rcnt = 0, rx0 = 0;
                    {
                        const int ry = iy0 + lane;
                        if (ry <= iy1 && (WPL == 1 || ((ry >> 1) % WPL) == zpart)) {
                            int xa = ix0, xb = ix1;
                            if (rh2 < 1e30f) {
                                const float dyr = (ry + 0.5f) - yc;
                                const float hw = sqrtf(fmaxf(rh2 - dyr * dyr, 0.0f));
                                xa = max(ix0, (int)ceilf(xc - hw - 0.5f) - 1);
                                xb = min(ix1, (int)floorf(xc + hw - 0.5f) + 1);
                            }
                            rcnt = max(0, xb - xa + 1);
                            rx0 = xa;
                        }
                    }
                    int rinc = rcnt;                 // inclusive scan over the (at most BY) rows
                    for (int o = 1; o < BY; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, rinc, o);
                        if (lane >= o) rinc += v;
                    }
                    const int ncell = __shfl_sync(0xffffffffu, rinc, BY - 1);
                    for (int q0 = 0; q0 < ncell; q0 += 32) {
                        const int qc = q0 + lane;
                        int r = 0;                   // rows whose runs end at or before qc
#pragma unroll
                        for (int st = BY / 2; st > 0; st >>= 1) {
                            const int v = __shfl_sync(0xffffffffu, rinc, r + st - 1);
                            if (v <= qc) r += st;
                        }
                        const int rb = __shfl_sync(0xffffffffu, rinc - rcnt, r);
                        const int rx = __shfl_sync(0xffffffffu, rx0, r);
                        const int tx = qc < ncell ? rx + (qc - rb) : ix1 + 1;
                        const int ty = iy0 + r;
                        const float cx = tx + 0.5f, cy = ty + 0.5f;
                        const float dx = cx - xc, dy = cy - yc;
                        bool in = false;
                        int js = 0;
                        T s = (T)0, r2 = (T)0;
                        if (FX && !WP && b.proj_mode && n >= 2 && tx <= ix1 && ty >= iy0 && ty <= iy1 &&
                            dx * dx + dy * dy <= rh2) {
                            // integrated projection: every candidate segment within 3 eps
                            // adds its integrated kernel, with the segment pass's values
                            const int cgl[3] = {B0 + tx, B1 + ty, gz};
                            const T epsc = (T)(b.eps[sm.e_line[e]] / g.h);
                            const int c = ty * BX + tx;
                            for (int jj = jlo; jj <= jhi; ++jj) {
                                const int ka = first + jj;
                                T s2, r22;
                                pair_sr(sc, np, ka, ka + 1, cgl, s2, r22);
                                bool inj;
                                if (r22 < R2 - gr) inj = true;
                                else if (r22 > R2 + gr) inj = false;
                                else inj = nl_within(g, p, b.eps[sm.e_line[e]], ka, n, cgl[0], cgl[1], cgl[2], status);
                                if (!inj) continue;
                                ++nsupp;
                                T wa, wb;
                                pair_int(sc, np, ka, cgl, epsc, e0v, ie2, wa, wb);
                                T fa3[3], fb3[3];
                                if (base >= 0) {
                                    const int ss = base + (jj - jlo);
                                    for (int a = 0; a < 3; ++a) { fa3[a] = sm.u.s.Fh[a][ss]; fb3[a] = sm.u.s.Fh[a][ss + 1]; }
                                } else {
                                    for (int a = 0; a < 3; ++a) { fa3[a] = sc.fhat[a * np + ka]; fb3[a] = sc.fhat[a * np + ka + 1]; }
                                }
                                for (int a = 0; a < 3; ++a)
                                    acc_sub<FX>(sm.u.s.acc[z][a][c], pair_src(wa, wb, fa3[a], fb3[a]), fsh);
                            }
                        } else if (tx <= ix1 && ty >= iy0 && ty <= iy1 && dx * dx + dy * dy <= rh2) {
                            const int gxc = B0 + tx, gyc = B1 + ty;
                            const T C[3] = {(T)cx, (T)cy, (T)czf};
                            if (base < 0) {
                                js = nl_exhaustive(g, sc, p, first, n, jlo, jhi, C[0], C[1], C[2], B0, B1, B2, gxc, gyc,
                                                   gz, status);
                                const int ka = first + js;
                                T x[3], Dj[3];
                                const int Bv[3] = {B0, B1, B2};
                                for (int a = 0; a < 3; ++a) {
                                    x[a] = C[a] - rel(sc.uhi[a * np + ka], sc.ulo[a * np + ka], Bv[a]);
                                    Dj[a] = sc.segD[a * np + ka];
                                }
                                s = (x[0] * Dj[0] + x[1] * Dj[1] + x[2] * Dj[2]) * sc.segIl2[ka];
                                s = s < (T)0 ? (T)0 : (s > (T)1 ? (T)1 : s);
                                const T f0 = x[0] - s * Dj[0], f1 = x[1] - s * Dj[1], f2 = x[2] - s * Dj[2];
                                r2 = f0 * f0 + f1 * f1 + f2 * f2;
                            } else {
                                bool exh = reg == 0, start_ok = true;
                                js = jlo;
                                if (!exh) {
                                    // start near the foot: the crossing plus the in-layer offset along the segment
                                    int j = (int)floorf(ac + dx * gxv + dy * gyv);
                                    j = min(max(j, jlo), jhi);
                                    if (reg == 2 && node_d2(sm, base + (j - jlo), C) > (T)rho2) {
                                        j = jcz;
                                        start_ok = node_d2(sm, base + (j - jlo), C) <= (T)rho2;
                                    }
                                    // the foot on the start segment lies inside it by more than
                                    // r tan(theta/2) at both ends: both bisector tests are decided
                                    // (sigma = a cos(theta/2) + ... >= a cos(theta/2) - r sin(theta/2))
                                    bool fast = false;
                                    if (start_ok) {
                                        const int sl = base + (j - jlo);
                                        T sr, sc0, rr;
                                        seg_foot_raw(sm, sl, C, sr, sc0, rr);
                                        // distances along the segment in cells (its length staged
                                        // per node, so no root or division per pair)
                                        const T L = sm.Ls[sl], r = tsqrt(rr);
                                        const T band = Tr<T>::gsig(r + L);
                                        const bool lo_ok = j == jlo || sr * L > r * (T)sm.Tau[sl] + band;
                                        const bool hi_ok = j == jhi || ((T)1 - sr) * L > r * (T)sm.Tau[sl + 1] + band;
                                        if (lo_ok && hi_ok) { fast = true; s = sc0; r2 = rr; }
                                    }
                                    if (!fast) {
                                        while (j > jlo && !sig_pos(sm, base + (j - jlo), C, g, p, sc, first + j, B0, B1,
                                                                   B2, gxc, gyc, gz, status)) --j;
                                        while (j < jhi && sig_pos(sm, base + (j + 1 - jlo), C, g, p, sc, first + j + 1,
                                                                  B0, B1, B2, gxc, gyc, gz, status)) ++j;
                                        seg_foot(sm, base + (j - jlo), C, s, r2);
                                    }
                                    js = j;
                                } else {
                                    seg_foot(sm, base + (js - jlo), C, s, r2);
                                }
                                // a walk from outside the certified radius is exact only when it ends within R
                                if (exh || (!start_ok && !(r2 < R2 - gr))) {
                                    js = nl_exhaustive_staged(sm, g, p, sc, base, first, n, jlo, jhi, C[0], C[1], C[2],
                                                              B0, B1, B2, gxc, gyc, gz, status);
                                    seg_foot(sm, base + (js - jlo), C, s, r2);
                                }
                            }
                            if (r2 < R2 - gr) in = true;
                            else if (r2 > R2 + gr) in = false;
                            else in = nl_within(g, p, b.eps[sm.e_line[e]], first + js, n, gxc, gyc, gz, status);
                        }
                        T q = (T)0;
                        if (in) {
                            ++nsupp;
                            q = Tr<T>::ex2(-r2 * ie2);
                        }
                        if (!WP) {
                            if (in) {
                                T fa0, fa1, fa2, fb0, fb1, fb2;
                                if (base >= 0) {
                                    const int ss = base + (js - jlo), sb = (n == 1) ? ss : ss + 1;
                                    fa0 = sm.u.s.Fh[0][ss]; fa1 = sm.u.s.Fh[1][ss]; fa2 = sm.u.s.Fh[2][ss];
                                    fb0 = sm.u.s.Fh[0][sb]; fb1 = sm.u.s.Fh[1][sb]; fb2 = sm.u.s.Fh[2][sb];
                                } else {
                                    const int ka = first + js, kb = seg_end(ka, n);
                                    fa0 = sc.fhat[ka]; fa1 = sc.fhat[np + ka]; fa2 = sc.fhat[2 * np + ka];
                                    fb0 = sc.fhat[kb]; fb1 = sc.fhat[np + kb]; fb2 = sc.fhat[2 * np + kb];
                                }
                                // the pair's values as the pass that summed the line's
                                // weights computed them (a node whose weight is small
                                // keeps its load only if the two agree): the segment
                                // pass's for certified lines under segment weights,
                                // this pass's own otherwise
                                T wa, wb;
                                if (FX && sm.e_canon[e]) {
                                    const int cgl[3] = {B0 + tx, B1 + ty, gz};
                                    T s2, r22;
                                    pair_sr(sc, np, first + js, (n == 1) ? first + js : first + js + 1, cgl, s2, r22);
                                    pair_w(e0v * Tr<T>::ex2(-r22 * ie2), s2, wa, wb);
                                } else {
                                    pair_w(e0v * q, s, wa, wb);
                                }
                                const int c = ty * BX + tx;
                                acc_sub<FX>(sm.u.s.acc[z][0][c], pair_src(wa, wb, fa0, fb0), fsh);
                                acc_sub<FX>(sm.u.s.acc[z][1][c], pair_src(wa, wb, fa1, fb1), fsh);
                                acc_sub<FX>(sm.u.s.acc[z][2][c], pair_src(wa, wb, fa2, fb2), fsh);
                            }
                        } else {
                            // omega eta / eta0 into the two nodes of the closest segment, as
                            // fixed-point integers summed over the warp per node (exact)
                            const int sh = (int)e0v;
                            unsigned long long va = 0ull, vb = 0ull;
                            int na = -1, nb2 = -1;
                            if (in) {
                                va = to_fixed(q * ((T)1 - s), sh);
                                vb = to_fixed(q * s, sh);
                                if (base >= 0) {
                                    na = base + (js - jlo);
                                    nb2 = (n == 1) ? na : na + 1;
                                } else {
                                    const int ka = first + js;
                                    atomicAdd(&sc.wfix[ka], va);
                                    atomicAdd(&sc.wfix[seg_end(ka, n)], vb);
                                }
                            }
                            // exact integer sums: near the crossing into the lane's counters,
                            // elsewhere straight into the shared node sums
                            if (na >= 0) {
                                const int oa = na - w0s, ob = nb2 - w0s;
                                wacc0 += (oa == 0 ? va : 0ull) + (ob == 0 ? vb : 0ull);
                                wacc1 += (oa == 1 ? va : 0ull) + (ob == 1 ? vb : 0ull);
                                wacc2 += (oa == 2 ? va : 0ull) + (ob == 2 ? vb : 0ull);
                                wacc3 += (oa == 3 ? va : 0ull) + (ob == 3 ? vb : 0ull);
                                if ((unsigned)oa > 3u && va) atomicAdd(&sm.u.wq[na], va);
                                if ((unsigned)ob > 3u && vb) atomicAdd(&sm.u.wq[nb2], vb);
                            }
                        }
                    }
                    if (WP && base >= 0) {
                        unsigned long long wv[4] = {wacc0, wacc1, wacc2, wacc3};
                        for (int q4 = 0; q4 < 4; ++q4) {
                            unsigned long long v = wv[q4];
                            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                            const int slot = w0s + q4;
                            if (lane == 0 && v && slot >= base && slot < base + (jhi - jlo + 2))
                                atomicAdd(&sm.u.wq[slot], v);
                        }
                    }
                }
            }
            // mirror images beyond reflecting faces within reach of this brick
            if constexpr (REFL) nsupp += d_images_phase<T, WP, BZ, FX>(g, b, sc, p, status, sm, ne, B0, B1, B2, fsh);
            __syncthreads();
            if (WP) {
                for (int e = 0; e < ne; ++e) {
                    const int jlo = sm.e_jlo[e], jhi = sm.e_jhi[e], base = sm.e_base[e];
                    if (jhi < jlo || base < 0) continue;
                    const int first = sm.e_first[e], n = sm.e_n[e];
                    const int cnt = (n == 1) ? 1 : jhi - jlo + 2;
                    for (int t = threadIdx.x; t < cnt; t += SPREAD_THREADS) {
                        unsigned long long v = sm.u.wq[base + t];
                        if (n == 1) v += sm.u.wq[base + 1];
                        if (v) atomicAdd(&sc.wfix[first + jlo + t], v);
                    }
                }
            } else if (warp == 0) {
                // ---- deposits of the zero-weight nodes inside this brick, in line and node order
                const int tot = sm.nstaged;
                for (int s0 = 0; s0 < tot; s0 += 32) {
                    const int sl = s0 + lane;
                    int c3[3] = {0, 0, 0};
                    bool f = sl < tot && sm.zf[sl];
                    int k = 0;
                    if (f) {
                        k = sm.u.s.sk[sl];
                        const int Bv[3] = {B0, B1, B2}, bs[3] = {BX, BY, BZ}, nn[3] = {g.nx, g.ny, g.nz};
                        for (int a = 0; a < 3; ++a) {
                            const T uh = sc.uhi[a * np + k];
                            const float ul = sc.ulo[a * np + k];
                            const int c = ffloor(uh, ul);
                            f = f && inside_axis(uh, ul, nn[a]) && c >= Bv[a] && c < Bv[a] + bs[a];
                            c3[a] = c - Bv[a];
                        }
                    }
                    uint32_t bal = __ballot_sync(0xffffffffu, f);
                    while (bal) {
                        const int src = __ffs(bal) - 1;
                        bal &= bal - 1;
                        if (lane == src)
                            for (int a = 0; a < 3; ++a)
                                acc_sub<FX>(sm.u.s.acc[c3[2]][a][c3[1] * BX + c3[0]], p.F[a][k] / (T)g.V, fsh);
                        __syncwarp();
                    }
                }
            }
            li += ne;
            __syncthreads();
        }
        if (!sm.more) break;
    }
    if (WP) return;
    if (g.rmode && threadIdx.x == 0) {
        // this brick's region of the next step: its count plus an eighth and
        // 16, taken from the arena by one atomic (placement does not affect
        // results; a brick that finds the arena full gathers next step)
        const long long want = nrec_b > 0 ? (long long)nrec_b + (nrec_b >> 3) + 16 : 0;
        long long off = 0;
        if (want > 0) off = (long long)atomicAdd(sc.rused, (unsigned long long)want);
        const bool fits = want > 0 && off + want <= g.rec_total;
        sc.rcap[br] = fits ? (int)want : 0;
        sc.roff[br] = fits ? off : 0;
        sc.rcnt[br] = 0;
        if (br == 0) sc.rplan[1] = g.bz;
    }
    // ---- write every cell of the brick once; brick sums of S -----------------
    T cs0 = (T)0, cs1 = (T)0, cs2 = (T)0;
    {
        const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
        if (tx < nxb && ty < nyb) {
            const long long layer = (long long)g.nx * g.ny;
            const long long col = (B0 + tx) + (long long)g.nx * (B1 + ty) + layer * B2;
            for (int z = 0; z < nzb; ++z) {
                const long long idx = col + layer * z;
                T v0, v1, v2;
                if constexpr (FX) {
                    from_fixed(sm.u.s.acc[z][0][threadIdx.x], fsh, v0);
                    from_fixed(sm.u.s.acc[z][1][threadIdx.x], fsh, v1);
                    from_fixed(sm.u.s.acc[z][2][threadIdx.x], fsh, v2);
                } else {
                    v0 = sm.u.s.acc[z][0][threadIdx.x];
                    v1 = sm.u.s.acc[z][1][threadIdx.x];
                    v2 = sm.u.s.acc[z][2][threadIdx.x];
                }
                p.S[0][idx] = v0; p.S[1][idx] = v1; p.S[2][idx] = v2;
                cs0 += v0; cs1 += v1; cs2 += v2;
            }
        }
    }
    // brick sums of S: compensated within the warp in the field precision,
    // one FP64 combination per brick
    {
        Acc<T> a3[3];
        a3[0].add(cs0); a3[1].add(cs1); a3[2].add(cs2);
        for (int a = 0; a < 3; ++a) w_store(&sm.red[a][warp], a3[a]);
    }
    for (int o = 16; o > 0; o >>= 1) nsupp += __shfl_down_sync(0xffffffffu, nsupp, o);
    if (lane == 0) sm.redi[warp] = nsupp;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ns = 0;
        for (int a = 0; a < 3; ++a) {
            double t = 0.0;
            for (int w = 0; w < SPREAD_THREADS / 32; ++w) t += w_load<T>(&sm.red[a][w]);
            sc.brickSum[a * g.nbrick + br] = t;
        }
        for (int w = 0; w < SPREAD_THREADS / 32; ++w) ns += sm.redi[w];
        if (ns) atomicAdd(&status[ST_SUPPORT], ns);
    }
}

// ---------------------------------------------------------------------------
// k_totals: FP64 sum F and sum S V, fixed reduction order
// ---------------------------------------------------------------------------
// Conservation totals (sum F per line, sum S per brick, in FP64): TOT_PARTS
// fixed slices of the lines and bricks, each summed by one CTA
// (d_totals_part), then the slices added in order (d_totals_fin); the same
// two steps in the batched kernels, so the bits match.
constexpr int TOT_PARTS = 32;
template <typename T>
__device__ void d_totals_part(const GridC &g, const BeamsC &b, const Scratch<T> &sc, int part, double (*red)[256]) {
    double v[6] = {0, 0, 0, 0, 0, 0};
    const long long l0 = (long long)b.n_lines * part / TOT_PARTS, l1 = (long long)b.n_lines * (part + 1) / TOT_PARTS;
    const long long r0 = g.nbrick * part / TOT_PARTS, r1 = g.nbrick * (part + 1) / TOT_PARTS;
    for (long long l = l0 + threadIdx.x; l < l1; l += 256)
        for (int a = 0; a < 3; ++a) v[a] += sc.lineF[3 * l + a];
    for (long long r = r0 + threadIdx.x; r < r1; r += 256)
        for (int a = 0; a < 3; ++a) v[3 + a] += sc.brickSum[a * g.nbrick + r];
    for (int a = 0; a < 6; ++a) red[a][threadIdx.x] = v[a];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int a = 0; a < 6; ++a) red[a][threadIdx.x] += red[a][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 6) sc.totPart[part * 6 + threadIdx.x] = red[threadIdx.x][0];
}
template <typename T>
__device__ void d_totals_fin(const GridC &g, const Scratch<T> &sc, double *totals) {
    if (threadIdx.x < 6) {
        const int a = threadIdx.x;
        double t = 0.0;
        for (int q = 0; q < TOT_PARTS; ++q) t += __ldcg(&sc.totPart[q * 6 + a]);
        if (a < 3) totals[a] = t;
        else totals[a] = (t + (g.smode ? sc.scatSum[a - 3] : 0.0)) * g.V;
    }
    if (threadIdx.x == 0) *sc.hasPrev = 1;                 // the next step relaxes against this one
}


// ---------------------------------------------------------------------------
// k_beam_qs: quasi-static reconstruction (Sec. 7), one warp per line: node
// i's displacement is the sum over the line's nodes k of the normal part of
// F_k times the cantilever's influence g(a_i, a_k) / EI
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T cantilever_g(T x, T a) {
    return x <= a ? x * x * ((T)3 * a - x) / (T)6 : a * a * ((T)3 * x - a) / (T)6;
}
template <typename T>
__global__ void __launch_bounds__(256) k_beam_qs(BeamsC b, const double *EI, T ax0, T ax1, T ax2,
                                                 StepPtrs<T> p) {
    // p.P: rest positions P0, p.F: loads, p.S[0..2]: output positions
    // each warp stages its line's stations and normal loads in shared memory
    // (lines of up to QS_N nodes; longer lines read them from global memory)
    constexpr int QS_N = 128;
    __shared__ T st_a[8][QS_N], st_f[8][3][QS_N];
    const int wib = threadIdx.x >> 5;
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (l >= b.n_lines) return;
    const int off = b.line_off[l], n = b.line_off[l + 1] - off;
    const T ax[3] = {ax0, ax1, ax2};
    const T r0[3] = {p.P[0][off], p.P[1][off], p.P[2][off]};
    const T iEI = (T)(1.0 / EI[l]);
    auto node = [&](int k, T &ak, T fp[3]) {
        T fa = (T)0, f[3];
        ak = (T)0;
        for (int a = 0; a < 3; ++a) {
            f[a] = p.F[a][k];
            ak += (p.P[a][k] - r0[a]) * ax[a];
            fa += f[a] * ax[a];
        }
        for (int a = 0; a < 3; ++a) fp[a] = f[a] - fa * ax[a];
    };
    const bool staged = n <= QS_N;
    if (staged) {
        for (int q = lane; q < n; q += 32) {
            T ak, fp[3];
            node(off + q, ak, fp);
            st_a[wib][q] = ak;
            for (int a = 0; a < 3; ++a) st_f[wib][a][q] = fp[a];
        }
        __syncwarp();
    }
    for (int q = lane; q < n; q += 32) {
        const int i = off + q;
        T xi = (T)0;
        for (int a = 0; a < 3; ++a) xi += (p.P[a][i] - r0[a]) * ax[a];
        T w[3] = {(T)0, (T)0, (T)0};
        for (int r = 0; r < n; ++r) {
            T ak, fp[3];
            if (staged) {
                ak = st_a[wib][r];
                for (int a = 0; a < 3; ++a) fp[a] = st_f[wib][a][r];
            } else {
                node(off + r, ak, fp);
            }
            const T gk = cantilever_g(xi, ak);
            for (int a = 0; a < 3; ++a) w[a] += fp[a] * gk;
        }
        for (int a = 0; a < 3; ++a) p.S[a][i] = p.P[a][i] + w[a] * iEI;
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

// One compiled body per form (a thread or a warp per point), called by the
// single-instance and the batched kernels alike, so an instance's forces
// have the same bits alone and in a batch.
template <typename T, int LANES>
__device__ __noinline__ void d_points_nl(const GridC &g, const BeamsC &b, const StepPtrs<T> &p,
                                         const Scratch<T> &sc, int *status, int i) {
    d_points<T, LANES>(g, b, p, sc, status, i);
}
template <typename T>
__global__ void __launch_bounds__(256) k_points(GridC g, BeamsC b, StepPtrs<T> p, Scratch<T> sc, int *status) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < b.n_points) d_points_nl<T, 1>(g, b, p, sc, status, i);
}
// one warp per point (volume-average sampler)
template <typename T>
__global__ void __launch_bounds__(256) k_points_w(GridC g, BeamsC b, StepPtrs<T> p, Scratch<T> sc, int *status) {
    pdl_enter();
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i < b.n_points) d_points_nl<T, 32>(g, b, p, sc, status, i);
}
template <typename T>
__global__ void __launch_bounds__(256) k_segments(BeamsC b, Scratch<T> sc) {
    pdl_enter();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < b.n_points) d_segments(b, sc, k);
}
template <typename T>
__global__ void __launch_bounds__(256) k_lines(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p, int *status) {
    pdl_enter();
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if constexpr (std::is_same<T, float>::value) {
        // per warp: its line's node heights and line-local positions, for the
        // column march's layer records
        __shared__ float sZ[8][CM_LN];
        __shared__ float4 sP[8][CM_LN];
        if (w < b.n_lines) d_lines(g, b, sc, p, status, w, threadIdx.x & 31, sZ[threadIdx.x >> 5], sP[threadIdx.x >> 5]);
    } else {
        if (w < b.n_lines) d_lines(g, b, sc, p, status, w, threadIdx.x & 31);
    }
}
template <typename T>
__global__ void __launch_bounds__(256) k_mask(GridC g, BeamsC b, Scratch<T> sc) {
    pdl_enter();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < b.n_points) d_mask(g, b, sc, k);
}
template <typename T>
__global__ void __launch_bounds__(128, 4) k_weights(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p, int *status) {
    pdl_enter();
    __shared__ RecStage<T> st;
    const bool stage = g.rmode != 0;
    if (stage) rec_init(st);
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k < b.n_points) d_weights<T, false>(g, b, sc, p, status, k, threadIdx.x & 31, stage ? &st : nullptr, 0);
    if (stage) rec_flush(st, [&](int) -> const Scratch<T> & { return sc; });
}
// scatter form of the projection: one warp per segment of a certified line
template <typename T>
__global__ void __launch_bounds__(128) k_scatter(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p, int *status) {
    pdl_enter();
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k < b.n_points) d_weights<T, true>(g, b, sc, p, status, k, threadIdx.x & 31);
}
template <typename T>
__global__ void __launch_bounds__(256) k_normalise(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p, int *status) {
    pdl_enter();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int m = k < b.n_points ? d_normalise(g, b, sc, p, status, k) : 0u;
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(sc.smax, m);
}
template <typename T, int BZ, bool FX>
__global__ void __launch_bounds__(SPREAD_THREADS) k_spread(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p,
                                                           int *status) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<T, BZ, FX> &sm = *reinterpret_cast<SpreadSmem<T, BZ, FX> *>(smem_raw);
    if (!brick_owned(g, blockIdx.x)) {                 // another slab's cells: no sources, no sum
        if (threadIdx.x < 3) sc.brickSum[threadIdx.x * g.nbrick + blockIdx.x] = 0.0;
        return;
    }
    d_brick<T, false, BZ, FX>(g, b, sc, p, status, (int)blockIdx.x, sm);
}
template <typename T, int BZ>
__global__ void __launch_bounds__(SPREAD_THREADS) k_bweights(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p,
                                                             int *status) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<T, BZ, false> &sm = *reinterpret_cast<SpreadSmem<T, BZ, false> *>(smem_raw);
    if (!brick_owned(g, blockIdx.x)) return;           // another slab's cells add nothing to the weights
    d_brick<T, true, BZ, false>(g, b, sc, p, status, (int)blockIdx.x, sm);
}

// the two brick passes with the kernel reflected at grid faces (ghost cells)
template <typename T, int BZ>
__global__ void __launch_bounds__(SPREAD_THREADS) k_spread_refl(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p,
                                                                int *status) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<T, BZ, false> &sm = *reinterpret_cast<SpreadSmem<T, BZ, false> *>(smem_raw);
    d_brick<T, false, BZ, false, true>(g, b, sc, p, status, (int)blockIdx.x, sm);
}
template <typename T, int BZ>
__global__ void __launch_bounds__(SPREAD_THREADS) k_bweights_refl(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p,
                                                                  int *status) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<T, BZ, false> &sm = *reinterpret_cast<SpreadSmem<T, BZ, false> *>(smem_raw);
    d_brick<T, true, BZ, false, true>(g, b, sc, p, status, (int)blockIdx.x, sm);
}
// the TOT_PARTS parts, one per CTA; the CTA that finishes last adds them
template <typename T>
__global__ void __launch_bounds__(256) k_totals(GridC g, BeamsC b, Scratch<T> sc, double *totals) {
    pdl_enter();
    __shared__ double red[6][256];
    __shared__ int last;
    d_totals_part(g, b, sc, (int)blockIdx.x, red);
    __threadfence();                                     // this part, before the count that publishes it
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(sc.totDone, 1) == TOT_PARTS - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        d_totals_fin(g, sc, totals);
        if (threadIdx.x == 0) *sc.totDone = 0;           // for the next step
    }
}

// ---- batched -------------------------------------------------------------
// pre: prefix sums of the per-instance item counts (n + 1 entries) of the n
// selected instances; sel: instance index of each selected slot (NULL: slot q
// is instance q)
#define AL_SEL(q) (sel ? sel[q] : (q))
// skip_gauss: the volume-average instances are left to kb_points_w
template <typename T>
__global__ void __launch_bounds__(256) kb_points(const Inst<T> *I, const int *sel, const long long *pre, int n,
                                                 int skip_gauss) {
    const long long total = pre[n];
    for (long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
         gid += (long long)gridDim.x * blockDim.x) {
        const int q = owner(pre, n, gid);
        const Inst<T> &x = I[AL_SEL(q)];
        if (skip_gauss && x.b.sample_mode == 2) continue;
        d_points_nl<T, 1>(x.g, x.b, x.p, x.sc, x.status, (int)(gid - pre[q]));
    }
}
// one warp per point, for the batch's instances with the volume-average sampler
template <typename T>
__global__ void __launch_bounds__(256) kb_points_w(const Inst<T> *I, const int *sel, const long long *pre, int n) {
    const long long total = pre[n];
    const long long nw = (long long)gridDim.x * blockDim.x / 32;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
        const int q = owner(pre, n, w);
        const Inst<T> &x = I[AL_SEL(q)];
        if (x.b.sample_mode != 2) continue;                 // kb_points takes the others
        d_points_nl<T, 32>(x.g, x.b, x.p, x.sc, x.status, (int)(w - pre[q]));
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
__global__ void __launch_bounds__(128, 4) kb_weights(const Inst<T> *I, const int *sel, const long long *pre, int n) {
    __shared__ RecStage<T> st;
    rec_init(st);
    const long long total = pre[n];
    const int nwb = blockDim.x / 32;
    // rounds of one segment per warp, the whole CTA together (the staged
    // records are flushed after each round)
    for (long long w0 = (long long)blockIdx.x * nwb; w0 < total; w0 += (long long)gridDim.x * nwb) {
        const long long w = w0 + (threadIdx.x >> 5);
        if (w < total) {
            const int q = owner(pre, n, w);
            const Inst<T> &x = I[AL_SEL(q)];
            d_weights<T, false>(x.g, x.b, x.sc, x.p, x.status, (int)(w - pre[q]), threadIdx.x & 31,
                                x.g.rmode ? &st : nullptr, q);
        }
        rec_flush(st, [&](int q) -> const Scratch<T> & { return I[AL_SEL(q)].sc; });
    }
}
template <typename T>
__global__ void __launch_bounds__(256) kb_normalise(const Inst<T> *I, const int *sel, const long long *pre, int n) {
    const long long total = pre[n];
    // the whole warp steps together so the bounds reduce per instance
    for (long long g0 = (long long)blockIdx.x * blockDim.x; g0 < total; g0 += (long long)gridDim.x * blockDim.x) {
        const long long gid = g0 + threadIdx.x;
        int q = -1;
        unsigned int m = 0u;
        if (gid < total) {
            q = owner(pre, n, gid);
            const Inst<T> &x = I[AL_SEL(q)];
            m = d_normalise(x.g, x.b, x.sc, x.p, x.status, (int)(gid - pre[q]));
        }
        const unsigned int grp = __match_any_sync(0xffffffffu, q);
        m = __reduce_max_sync(grp, m);
        if (q >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1 && m) atomicMax(I[AL_SEL(q)].sc.smax, m);
    }
}
// the next brick item of a persistent batched pass, taken by the CTA from a
// counter of the run (every thread has read the previous one first)
__device__ __forceinline__ long long kb_take(unsigned long long *ctr, long long *slot) {
    __syncthreads();
    if (threadIdx.x == 0) *slot = (long long)atomicAdd(ctr, 1ull);
    __syncthreads();
    return *slot;
}
// persistent: a fixed grid of CTAs takes the bricks of every instance from a counter
template <typename T, int BZ>
__global__ void __launch_bounds__(SPREAD_THREADS) kb_spread(const Inst<T> *I, const int *sel, const long long *pre, int n,
                                                            unsigned long long *ctr) {
    __shared__ long long s_item;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // each instance in the accumulation form it has alone (the shared memory
    // is sized for the larger, fixed-point form)
    const long long total = pre[n];
    for (long long item = kb_take(ctr + 2, &s_item); item < total; item = kb_take(ctr + 2, &s_item)) {
        const int q = owner(pre, n, item);
        const Inst<T> &x = I[AL_SEL(q)];
        if (x.b.reflect) continue;                   // kb_spread_refl takes these
        if (x.g.fx)
            d_brick<T, false, BZ, true>(x.g, x.b, x.sc, x.p, x.status, (int)(item - pre[q]),
                                        *reinterpret_cast<SpreadSmem<T, BZ, true> *>(smem_raw));
        else
            d_brick<T, false, BZ, false>(x.g, x.b, x.sc, x.p, x.status, (int)(item - pre[q]),
                                         *reinterpret_cast<SpreadSmem<T, BZ, false> *>(smem_raw));
        __syncthreads();
    }
}
template <typename T, int BZ>
__global__ void __launch_bounds__(SPREAD_THREADS) kb_spread_refl(const Inst<T> *I, const int *sel,
                                                                 const long long *pre, int n,
                                                                 unsigned long long *ctr) {
    __shared__ long long s_item;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<T, BZ, false> &sm = *reinterpret_cast<SpreadSmem<T, BZ, false> *>(smem_raw);
    const long long total = pre[n];
    for (long long item = kb_take(ctr + 3, &s_item); item < total; item = kb_take(ctr + 3, &s_item)) {
        const int q = owner(pre, n, item);
        const Inst<T> &x = I[AL_SEL(q)];
        if (!x.b.reflect) continue;
        d_brick<T, false, BZ, false, true>(x.g, x.b, x.sc, x.p, x.status, (int)(item - pre[q]), sm);
        __syncthreads();
    }
}
template <typename T, int BZ>
__global__ void __launch_bounds__(SPREAD_THREADS) kb_bweights(const Inst<T> *I, const int *sel, const long long *pre,
                                                              int n, unsigned long long *ctr) {
    __shared__ long long s_item;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<T, BZ, false> &sm = *reinterpret_cast<SpreadSmem<T, BZ, false> *>(smem_raw);
    const long long total = pre[n];
    for (long long item = kb_take(ctr + 0, &s_item); item < total; item = kb_take(ctr + 0, &s_item)) {
        const int q = owner(pre, n, item);
        const Inst<T> &x = I[AL_SEL(q)];
        if (x.b.reflect) continue;                   // kb_bweights_refl takes these
        d_brick<T, true, BZ, false>(x.g, x.b, x.sc, x.p, x.status, (int)(item - pre[q]), sm);
        __syncthreads();
    }
}
// the same for the instances whose kernel is reflected at grid faces
template <typename T, int BZ>
__global__ void __launch_bounds__(SPREAD_THREADS) kb_bweights_refl(const Inst<T> *I, const int *sel,
                                                                   const long long *pre, int n,
                                                                   unsigned long long *ctr) {
    __shared__ long long s_item;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<T, BZ, false> &sm = *reinterpret_cast<SpreadSmem<T, BZ, false> *>(smem_raw);
    const long long total = pre[n];
    for (long long item = kb_take(ctr + 1, &s_item); item < total; item = kb_take(ctr + 1, &s_item)) {
        const int q = owner(pre, n, item);
        const Inst<T> &x = I[AL_SEL(q)];
        if (!x.b.reflect) continue;
        d_brick<T, true, BZ, false, true>(x.g, x.b, x.sc, x.p, x.status, (int)(item - pre[q]), sm);
        __syncthreads();
    }
}
template <typename T>
__global__ void __launch_bounds__(256) kb_totals(const Inst<T> *I, const int *sel, int n) {
    __shared__ double red[6][256];
    for (long long w = blockIdx.x; w < (long long)n * TOT_PARTS; w += gridDim.x) {
        const Inst<T> &x = I[AL_SEL((int)(w / TOT_PARTS))];
        d_totals_part(x.g, x.b, x.sc, (int)(w % TOT_PARTS), red);
        __syncthreads();
    }
}
template <typename T>
__global__ void __launch_bounds__(32) kb_totals_fin(const Inst<T> *I, const int *sel, int n) {
    for (int q = blockIdx.x; q < n; q += gridDim.x) {
        const Inst<T> &x = I[AL_SEL(q)];
        d_totals_fin(x.g, x.sc, x.totals);
    }
}
#undef AL_SEL

}  // namespace al

#include "al_cm.cuh"
