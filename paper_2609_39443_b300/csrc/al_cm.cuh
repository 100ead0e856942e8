// al_cm.cuh -- the column march: both projection passes (Sec. 3.2.4) for a
// brick whose candidate lines all climb and carry the column-march
// certificate (LineG::cm, set by k_lines for FP32 instances).
//
// Geometry.  For a cell C and an interior node k let sigma_k(C) =
// (C - P_k) . m_k, m_k the unit bisector of the two segment directions.  On
// a line whose segments all climb (D_z / |D| >= 0.8), every m_k has a
// positive z component, so along a column of cells (fixed x, y, rising z)
// each sigma_k increases.  The certificate makes the signs of sigma_k over a
// brick's candidate segments monotone (+ ... + - ... -) for every cell within
// 3 eps of the line, where the last positive sign is the closest segment
// (Eq. almProjectionPoint; the node shared by the two segments is within
// reach of both feet).  Hence, walking up a column, the closest segment only
// ever moves up the line: each layer costs one test of the next bisector,
// which is linear in z, instead of a search.  A column starts with a walk
// from the segment containing its first layer's height.  Cells farther than
// 3 eps from every candidate get a segment whose distance exceeds 3 eps too
// and receive nothing, as Eq. almGaussian truncates.
//
// Decisions.  A bisector sign or the cut-off r <= 3 eps is taken in FP32
// only outside a band around zero that bounds the FP32 error; inside the
// band the float-float test of "segment k closer than k-1" decides, then an
// FP64 evaluation of the paper's distances in the oracle's operation order,
// exactly as in the brick passes, so every (cell, line) pair inside 3 eps is
// the oracle's.  Those exact decisions are rare and out of line: the march
// leaves its inner loop when a value falls inside a band, takes the decision
// and resumes, so the inner loop holds no call.
//
// Coordinates.  Node positions are stored relative to the integer origin of
// their line's first node (float, lines shorter than 250 cells: within
// 8e-6 cells), and a column works in those line-local coordinates.
//
// A march keeps the next segment's records in registers, loaded one
// advance ahead.
//
// Passes (one step):
//   k_cm_entries  one warp per brick: the brick goes to the column march
//                 when all its candidate lines take it (list 0), else to the
//                 brick passes (list 1); for a column-march brick each
//                 candidate line gets an entry (segment range, layer range,
//                 2-D reach of its columns, start segment), stored in line
//                 order per brick
//   k_cm_weights  one warp per entry: its lanes take the brick's columns in
//                 reach of the line, 32 at a time; each lane adds
//                 omega eta / eta0 of its pairs per node into its own column
//                 of a per-warp buffer, whose rows are summed in a fixed
//                 order and added to the node's fixed-point weight (exact
//                 integer sums, independent of the order of the entries)
//   k_cm_spread   one CTA per brick: each thread marches whole columns
//                 through their entries, subtracting eta (f^_a + s (f^_b -
//                 f^_a)) from the column's sources in registers; the brick's
//                 sources are then written once per cell, with no atomics
// Both passes run the same march (cm_start, cm_march) with the same
// explicitly rounded operations on the same node records, so they take the
// same decisions and the same (s, eta) bits for every pair.
#pragma once

#include <cuda.h>                 // CUtensorMap (the descriptors of the S tile stores)

namespace al {

constexpr int CM_ENT = 32;       // entries per batch of a brick
constexpr int CM_EN = 32;        // nodes of one entry in a warp's weight buffer
// node records, four float4 per node k at cmN[4 k + ...]
constexpr int CM_P = 0;          // position (line-local) and 1/|D_k|^2
constexpr int CM_D = 1;          // D_k (segment k)
constexpr int CM_M = 2;          // bisector m_k (interior nodes, else 0)
constexpr int CM_F = 3;          // f^_k and 1 where w_k = 0

// one candidate line of one column-march brick (96 bytes)
struct alignas(16) CmEnt {
    int br, line, kfirst, nseg;  // brick, line, global index of its first candidate node, candidate segments
    int zf, zl, j0, wsh;         // layer range within the brick; segment containing the height of layer zf;
                                 // the line's fixed-point weight shift
    float ox, oy, oz, gs;        // brick corner minus the line's origin (cells); bisector band
    float ux, uy, iuu, reach2;   // 2-D chord of the candidate nodes: vector, 1/|u|^2; squared reach of a
                                 // column (-1: no column)
    float bx, by, R2lo, R2hi;    // the chord's start relative to the brick corner; cut-off band on r^2
    float ie2, eta0, pad0, pad1; // log2(e) / eps^2 (cells), 1 / (pi eps^2)
};

// one brick layer of a certified line (k_lines): what its entries in that
// layer share; an entry adds the brick's corner
struct alignas(16) CmLay {
    int kfirst, nseg, zf, zl;     // first candidate node (global), candidate segments (0: none), layer range
    int j0, O0, O1, pad;          // segment containing the height of layer zf; the line's origin cell (x, y)
    float oz, gs, ux, uy;         // layer corner minus the origin (z); bisector band; 2-D chord vector
    float iuu, reach2, ax, ay;    // 1/|u|^2; squared reach (-1: no column); chord start (line-local)
};

// ---- node records (per step, FP32 instances with the column march) ---------
__device__ __forceinline__ void cm_line_origin(const Scratch<float> &sc, long long np, int first, int O[3]) {
    for (int a = 0; a < 3; ++a) O[a] = ifloor(sc.uhi[a * np + first]);
}
__device__ __forceinline__ void cm_write_node(const Scratch<float> &sc, long long np, int k, int first) {
    if (!sc.cmN) return;
    int O[3];
    cm_line_origin(sc, np, first, O);
    float p[3];
    for (int a = 0; a < 3; ++a) p[a] = rel(sc.uhi[a * np + k], sc.ulo[a * np + k], O[a]);
    float4 *r = sc.cmN + 4 * (long long)k;
    r[CM_P] = make_float4(p[0], p[1], p[2], sc.segIl2[k]);
    r[CM_D] = make_float4(sc.segD[k], sc.segD[np + k], sc.segD[2 * np + k], 0.0f);
    r[CM_M] = make_float4(sc.nodeM[k], sc.nodeM[np + k], sc.nodeM[2 * np + k], 0.0f);
}
__device__ __forceinline__ void cm_write_node(const Scratch<double> &, long long, int, int) {}
__device__ __forceinline__ void cm_write_fhat(const Scratch<float> &sc, long long np, int k, double w) {
    if (!sc.cmN) return;
    sc.cmN[4 * (long long)k + CM_F] =
        make_float4(sc.fhat[k], sc.fhat[np + k], sc.fhat[2 * np + k], w == 0.0 ? 1.0f : 0.0f);
}
__device__ __forceinline__ void cm_write_fhat(const Scratch<double> &, long long, int, double) {}

// ---- slow paths (rare, out of line): exact decisions ----------------------------
// what the exact decisions read (shared memory): the caller's projection
// positions, the float-float cell coordinates, the grid's origin and cell
// size, the lines' eps
struct CmExact {
    const float *P0, *P1, *P2;
    const float *uhi, *ulo;
    const double *eps;
    long long np;
    double ox, oy, oz, h;
    int *status;
};
// sigma of the bisector at node k for the cell (X, Y, Z) relative to the
// brick corner (B0, B1, B2), d = the cell minus the node: the FP32 value sg
// outside the band of its error at the cell's distance from the node, else
// the float-float test of "segment k closer than k-1", else FP64 in the
// oracle's operation order
static __device__ __noinline__ bool cm_sig_slow(const CmExact *x, int k, int B0, int B1, int B2, float X, float Y,
                                                float Z, float sg, float d0, float d1, float d2) {
    const float gsx = Tr<float>::gsig(sqrtf(d0 * d0 + d1 * d1 + d2 * d2));
    if (sg > gsx) return true;
    if (sg < -gsx) return false;
    const int r = ff_later_closer(x->uhi, x->ulo, x->np, k, B0, B1, B2, X, Y, Z);
    if (r >= 0) return r == 1;
    atomicAdd(&x->status[ST_REFINED], 1);
    const int ci = B0 + (int)X, cj = B1 + (int)Y, ck = B2 + (int)Z;
    const double e1 = dist2_f64_raw(x->P0, x->P1, x->P2, x->ox, x->oy, x->oz, x->h, k, k + 1, ci, cj, ck);
    const double e0 = dist2_f64_raw(x->P0, x->P1, x->P2, x->ox, x->oy, x->oz, x->h, k - 1, k, ci, cj, ck);
    return __dsqrt_rn(e1) < __dsqrt_rn(e0);
}
// r <= 3 eps in FP64 for segment (k, k + 1) of line l
static __device__ __noinline__ bool cm_in_slow(const CmExact *x, int l, int k, int ci, int cj, int ck) {
    atomicAdd(&x->status[ST_REFINED], 1);
    const double d2 = dist2_f64_raw(x->P0, x->P1, x->P2, x->ox, x->oy, x->oz, x->h, k, k + 1, ci, cj, ck);
    return __dsqrt_rn(d2) <= __dmul_rn(3.0, x->eps[l]);
}

// ---- the march of one column against one entry --------------------------------
struct CmCtx {                    // one item's constants (registers)
    const float4 *N;              // node records of candidate 0 onwards
    const CmExact *x;             // for the exact decisions (shared memory)
    int B0, B1, B2;
    int kfirst, nseg, line;       // global node index of candidate 0, candidate segments, line
    float ox, oy, oz, gs;         // brick corner minus the line origin; bisector band
    float R2lo, R2hi, ie2;        // cut-off band on r^2, log2(e) / eps^2 (cells)
};

struct CmWalk {
    int j;                        // current segment (candidate index)
    float xx, xy, pz, il2;        // Xl - P_j.x, Yl - P_j.y, P_j.z, 1/|D_j|^2
    float dx, dy, dz, dxy;        // D_j; (Xl - P_j.x) D_x + (Yl - P_j.y) D_y
    float b1, m1z;                // sigma_{j+1} at height Zl: fma(Zl, m1z, b1); no next bisector: -inf
    float4 nP, nD, n2P, n2M;      // node j + 1 (position, segment vector); node j + 2 (position, bisector)
};

// record f of candidate node j (c.N: the records of candidate 0, in global
// or shared memory)
__device__ __forceinline__ float4 cm_rec(const CmCtx &c, int j, int f) { return c.N[4 * j + f]; }
// the bisector of node (P, M) for the column: sigma(Zl) = fma(Zl, M.z, b1)
__device__ __forceinline__ float cm_b1(float Xl, float Yl, const float4 &P, const float4 &M) {
    return __fmaf_rn(-P.z, M.z, __fmaf_rn(__fsub_rn(Yl, P.y), M.y, __fmul_rn(__fsub_rn(Xl, P.x), M.x)));
}
// segment j's column constants from its start node (P) and vector (D)
__device__ __forceinline__ void cm_seg(CmWalk &w, const float4 &P, const float4 &D, float Xl, float Yl) {
    w.xx = __fsub_rn(Xl, P.x);
    w.xy = __fsub_rn(Yl, P.y);
    w.pz = P.z;
    w.il2 = P.w;
    w.dx = D.x; w.dy = D.y; w.dz = D.z;
    w.dxy = __fmaf_rn(w.xy, D.y, __fmul_rn(w.xx, D.x));
}
// one step up the line (j -> j + 1, j + 1 < nseg) from the prefetched
// records; the records of the next step are loaded for later
__device__ __forceinline__ void cm_adv(const CmCtx &c, CmWalk &w, float Xl, float Yl) {
    const int j = ++w.j;
    cm_seg(w, w.nP, w.nD, Xl, Yl);
    if (j + 1 < c.nseg) {
        w.b1 = cm_b1(Xl, Yl, w.n2P, w.n2M);
        w.m1z = w.n2M.z;
    } else {
        w.b1 = -INFINITY;
        w.m1z = 0.0f;
    }
    w.nP = w.n2P;
    w.nD = cm_rec(c, min(j + 1, c.nseg), CM_D);
    const int j2 = min(j + 2, c.nseg);
    w.n2P = cm_rec(c, j2, CM_P);
    w.n2M = cm_rec(c, j2, CM_M);
}

// sigma of candidate node jn (> 0: the cell's closest segment is at or after it)
__device__ __forceinline__ bool cm_pos(const CmCtx &c, int jn, float Xl, float Yl, float Zl) {
    const float4 a = cm_rec(c, jn, CM_P), m = cm_rec(c, jn, CM_M);
    const float d0 = __fsub_rn(Xl, a.x), d1 = __fsub_rn(Yl, a.y), d2 = __fsub_rn(Zl, a.z);
    const float sg = __fmaf_rn(d2, m.z, __fmaf_rn(d1, m.y, __fmul_rn(d0, m.x)));
    if (sg >= c.gs) return true;
    if (sg <= -c.gs) return false;
    return cm_sig_slow(c.x, c.kfirst + jn, c.B0, c.B1, c.B2, Xl - c.ox, Yl - c.oy, Zl - c.oz, sg, d0, d1, d2);
}

// the walk at the column's first layer: from j0 (the segment containing that
// height) down while the bisector at j is not positive, then up while the
// next one is; loads the segment's constants and the records ahead
__device__ __forceinline__ void cm_start(const CmCtx &c, CmWalk &w, int j0, float Xl, float Yl, float Zl0) {
    int j = j0;
    while (j > 0 && !cm_pos(c, j, Xl, Yl, Zl0)) --j;
    while (j < c.nseg - 1 && cm_pos(c, j + 1, Xl, Yl, Zl0)) ++j;
    w.j = j;
    cm_seg(w, cm_rec(c, j, CM_P), cm_rec(c, j, CM_D), Xl, Yl);
    w.nP = cm_rec(c, j + 1, CM_P);
    w.nD = cm_rec(c, j + 1, CM_D);
    if (j + 1 < c.nseg) {
        const float4 m = cm_rec(c, j + 1, CM_M);
        w.b1 = cm_b1(Xl, Yl, w.nP, m);
        w.m1z = m.z;
    } else {
        w.b1 = -INFINITY;
        w.m1z = 0.0f;
    }
    const int j2 = min(j + 2, c.nseg);
    w.n2P = cm_rec(c, j2, CM_P);
    w.n2M = cm_rec(c, j2, CM_M);
}

// cm_start's walk without the exact decisions: false when a bisector at
// the first layer falls inside its band (cm_start_slow then walks with them)
__device__ __forceinline__ bool cm_start_fast(const CmCtx &c, int j0, float Xl, float Yl, float Zl0, int &jout) {
    int j = j0;
    for (; j > 0; --j) {
        const float4 a = cm_rec(c, j, CM_P), m = cm_rec(c, j, CM_M);
        const float sg = __fmaf_rn(__fsub_rn(Zl0, a.z), m.z,
                                   __fmaf_rn(__fsub_rn(Yl, a.y), m.y, __fmul_rn(__fsub_rn(Xl, a.x), m.x)));
        if (sg >= c.gs) break;
        if (sg > -c.gs) return false;
    }
    for (; j < c.nseg - 1; ++j) {
        const float4 a = cm_rec(c, j + 1, CM_P), m = cm_rec(c, j + 1, CM_M);
        const float sg = __fmaf_rn(__fsub_rn(Zl0, a.z), m.z,
                                   __fmaf_rn(__fsub_rn(Yl, a.y), m.y, __fmul_rn(__fsub_rn(Xl, a.x), m.x)));
        if (sg <= -c.gs) break;
        if (sg < c.gs) return false;
    }
    jout = j;
    return true;
}
static __device__ __noinline__ int cm_start_slow(const CmCtx *c, int j0, float Xl, float Yl, float Zl0) {
    int j = j0;
    while (j > 0 && !cm_pos(*c, j, Xl, Yl, Zl0)) --j;
    while (j < c->nseg - 1 && cm_pos(*c, j + 1, Xl, Yl, Zl0)) ++j;
    return j;
}
// the walk's state at segment j
__device__ __forceinline__ void cm_walk_at(const CmCtx &c, CmWalk &w, int j, float Xl, float Yl) {
    w.j = j;
    cm_seg(w, cm_rec(c, j, CM_P), cm_rec(c, j, CM_D), Xl, Yl);
    w.nP = cm_rec(c, j + 1, CM_P);
    w.nD = cm_rec(c, j + 1, CM_D);
    if (j + 1 < c.nseg) {
        const float4 m = cm_rec(c, j + 1, CM_M);
        w.b1 = cm_b1(Xl, Yl, w.nP, m);
        w.m1z = m.z;
    } else {
        w.b1 = -INFINITY;
        w.m1z = 0.0f;
    }
    const int j2 = min(j + 2, c.nseg);
    w.n2P = cm_rec(c, j2, CM_P);
    w.n2M = cm_rec(c, j2, CM_M);
}

// The walk without records held ahead (for records in shared memory, where
// a load at the advance is cheap): the same state, from the same operations
// on the same records, as CmWalk's.
struct CmWalkL {
    int j;
    float xx, xy, pz, il2, dx, dy, dz, dxy, b1, m1z;
};
__device__ __forceinline__ void cm_walkl_at(const CmCtx &c, CmWalkL &w, int j, float Xl, float Yl) {
    const float4 P = cm_rec(c, j, CM_P), D = cm_rec(c, j, CM_D);
    w.j = j;
    w.xx = __fsub_rn(Xl, P.x);
    w.xy = __fsub_rn(Yl, P.y);
    w.pz = P.z;
    w.il2 = P.w;
    w.dx = D.x; w.dy = D.y; w.dz = D.z;
    w.dxy = __fmaf_rn(w.xy, D.y, __fmul_rn(w.xx, D.x));
    if (j + 1 < c.nseg) {
        const float4 P1 = cm_rec(c, j + 1, CM_P), M1 = cm_rec(c, j + 1, CM_M);
        w.b1 = cm_b1(Xl, Yl, P1, M1);
        w.m1z = M1.z;
    } else {
        w.b1 = -INFINITY;
        w.m1z = 0.0f;
    }
}
__device__ __forceinline__ void cm_geoml(const CmWalkL &w, float Zl, float &s, float &r2) {
    const float xz = __fsub_rn(Zl, w.pz);
    const float dot = __fmaf_rn(xz, w.dz, w.dxy);
    s = __saturatef(__fmul_rn(dot, w.il2));
    const float ex = __fmaf_rn(-s, w.dx, w.xx), ey = __fmaf_rn(-s, w.dy, w.xy), ez = __fmaf_rn(-s, w.dz, xz);
    r2 = __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
}

// foot s (clamped) and r^2 of the cell at height Zl and the current segment
__device__ __forceinline__ void cm_geom(const CmWalk &w, float Zl, float &s, float &r2) {
    const float xz = __fsub_rn(Zl, w.pz);
    const float dot = __fmaf_rn(xz, w.dz, w.dxy);
    s = __saturatef(__fmul_rn(dot, w.il2));
    const float ex = __fmaf_rn(-s, w.dx, w.xx), ey = __fmaf_rn(-s, w.dy, w.xy), ez = __fmaf_rn(-s, w.dz, xz);
    r2 = __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
}

// March layers zf .. zl of the column (Xl, Yl) (line-local): per layer the
// walk advances while the next bisector is positive (sink.adv(c, jp) after
// each advance), then the pair (clamped foot s, r^2) of the cell and the
// current segment; sink.pair(c, z, s, q) for each pair inside 3 eps with
// q = exp(-(r / eps)^2).  A bisector or cut-off value inside its band leaves
// the inner loop; the exact decision is taken out of line and the march
// resumes where it stopped.
template <typename SINK>
__device__ __forceinline__ void cm_march(const CmCtx &c, CmWalk &w, float Xl, float Yl, int zf, int zl, SINK &sink) {
    int z = zf;
    float Zl = __fadd_rn((float)zf + 0.5f, c.oz);
    for (;;) {
        int pend = 0;             // 1: a bisector inside its band; 2: a cut-off inside its band
        float pv = 0.0f;
        for (; z <= zl; ++z, Zl = __fadd_rn(Zl, 1.0f)) {
            float sg = __fmaf_rn(Zl, w.m1z, w.b1);
            while (sg >= c.gs) {
                cm_adv(c, w, Xl, Yl);
                sink.adv(c, w.j - 1);
                sg = __fmaf_rn(Zl, w.m1z, w.b1);
            }
            if (sg > -c.gs) { pend = 1; pv = sg; break; }
            float s, r2;
            cm_geom(w, Zl, s, r2);
            if (r2 < c.R2lo) sink.pair(c, z, s, Tr<float>::ex2(__fmul_rn(-r2, c.ie2)));
            else if (!(r2 > c.R2hi)) { pend = 2; break; }
        }
        if (!pend) return;
        if (pend == 1) {
            const float4 n = w.nP;
            if (cm_sig_slow(c.x, c.kfirst + w.j + 1, c.B0, c.B1, c.B2, Xl - c.ox, Yl - c.oy, Zl - c.oz, pv,
                            __fsub_rn(Xl, n.x), __fsub_rn(Yl, n.y), __fsub_rn(Zl, n.z))) {
                cm_adv(c, w, Xl, Yl);
                sink.adv(c, w.j - 1);
                continue;         // the same layer, from its next bisector
            }
        }
        // this layer's pair with the current segment, its cut-off decided
        // exactly inside the band
        float s, r2;
        cm_geom(w, Zl, s, r2);
        if (r2 < c.R2lo || (!(r2 > c.R2hi) && cm_in_slow(c.x, c.line, c.kfirst + w.j, c.B0 + (int)(Xl - c.ox),
                                                          c.B1 + (int)(Yl - c.oy), c.B2 + z)))
            sink.pair(c, z, s, Tr<float>::ex2(__fmul_rn(-r2, c.ie2)));
        ++z;
        Zl = __fadd_rn(Zl, 1.0f);
    }
}

// is the column (X, Y) (brick-relative) within reach of the entry: within
// 3 eps + the arc's deviation of the 2-D chord of its candidate nodes (every
// cell within 3 eps of the arc projects within that distance of the chord)
__device__ __forceinline__ bool cm_reach(const CmEnt &e, float X, float Y) {
    const float4 u = reinterpret_cast<const float4 *>(&e)[3], b = reinterpret_cast<const float4 *>(&e)[4];
    const float qx = X - b.x, qy = Y - b.y;
    const float t = __saturatef((qx * u.x + qy * u.y) * u.z);
    const float ex = qx - t * u.x, ey = qy - t * u.y;
    return ex * ex + ey * ey <= u.w;
}

__device__ __forceinline__ void cm_brick_origin(const GridC &g, int br, int bz, int &B0, int &B1, int &B2) {
    const int nbxy = g.nbx * g.nby;
    const int bzi = br / nbxy, rem = br - bzi * nbxy;
    const int byi = rem / g.nbx, bxi = rem - byi * g.nbx;
    B0 = bxi * BX; B1 = byi * BY; B2 = bzi * bz;
}

__device__ __forceinline__ CmCtx cm_ctx(const float4 *N, const CmExact *x, const CmEnt &e, int B0, int B1, int B2) {
    CmCtx c;
    c.N = N;
    c.x = x;
    c.B0 = B0; c.B1 = B1; c.B2 = B2;
    c.kfirst = e.kfirst; c.nseg = e.nseg; c.line = e.line;
    c.ox = e.ox; c.oy = e.oy; c.oz = e.oz; c.gs = e.gs;
    c.R2lo = e.R2lo; c.R2hi = e.R2hi; c.ie2 = e.ie2;
    return c;
}
__device__ __forceinline__ void cm_exact_init(CmExact &x, const GridC &g, const BeamsC &b, const Scratch<float> &sc,
                                              const StepPtrs<float> &p, int *status) {
    x = CmExact{p.Ps[0], p.Ps[1], p.Ps[2], sc.uhi, sc.ulo, b.eps, (long long)p.np,
                g.o[0], g.o[1], g.o[2], g.h, status};
}

// ---- entries ---------------------------------------------------------------------
// entry of line l in the brick at (B0, B1, B2) with nzb layers inside the
// grid: the candidate segments are those whose height range meets the
// layer centres widened by 3 eps + 0.02 (node heights increase along the
// line, so they form a range), and at least the brick's own height range,
// so that a node inside the brick is a candidate node for its zero-weight
// deposit
// per brick layer of a certified line (one warp, k_lines, a lane per
// layer): the candidate segments [jlo, jhi] (node heights increase along a
// climbing line, so they form a range), the layers within 3 eps (+0.02) of
// their height range, the start segment, the 2-D chord of the candidate
// nodes with its reach (3 eps + their largest departure from it + 0.02) and
// the bisector band; index guards flag status[ST_GUARD] and leave the layer
// without candidates
static __device__ void cm_layer_records(const GridC &g, const Scratch<float> &sc, long long np, int l, int off,
                                        int n, float Rc, float Lmax, int lane, int *status, float *sZ, float4 *sP) {
    const int nbz_max = (g.nz + 3) / 4;
    const float *uz = sc.uhi + 2 * np + off;
    int O[3];
    cm_line_origin(sc, np, off, O);
    // the line's node heights and positions (records) in the warp's shared
    // memory when they fit: the searches below then wait on no global load
    const bool st = sZ != nullptr && sP != nullptr && n <= CM_LN && off >= 0 && off + n <= np;
    if (st) {
        for (int q = lane; q < n; q += 32) {
            sZ[q] = uz[q];
            sP[q] = sc.cmN[4 * (long long)(off + q) + CM_P];
        }
        __syncwarp();
    }
    const float *Z = st ? sZ : uz;
    for (int bzi = lane; bzi < g.nbz; bzi += 32) {
        const int B2 = bzi * g.bz, nzb = min(g.bz, g.nz - B2);
        const float zlo = (float)B2 + fminf(0.5f - Rc, 0.0f) - 0.02f;
        const float zhi = (float)B2 + (float)nzb + fmaxf(Rc - 0.5f, 0.0f) + 0.02f;
        int lo = 1, hi = n;                      // first node q >= 1 with z_q >= zlo (n: none)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Z[mid] >= zlo) hi = mid; else lo = mid + 1;
        }
        const int jlo = lo - 1;
        lo = -1; hi = n - 2;                     // last node q <= n - 2 with z_q <= zhi (-1: none)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (Z[mid] <= zhi) lo = mid; else hi = mid - 1;
        }
        const int jhi = lo;
        CmLay r;
        r.kfirst = off + jlo;
        r.nseg = jhi >= jlo ? jhi - jlo + 1 : 0;
        r.zf = 1; r.zl = 0; r.j0 = 0;
        r.O0 = O[0]; r.O1 = O[1]; r.pad = 0;
        r.oz = (float)(B2 - O[2]);
        r.gs = 0.0f;
        r.ux = r.uy = r.iuu = 0.0f;
        r.reach2 = -1.0f;
        r.ax = r.ay = 0.0f;
        if (!(jlo >= 0 && jlo <= n - 1 && jhi <= n - 2 && off >= 0 && off + n <= np)) {
            atomicOr(&status[ST_GUARD], 128);
            r.nseg = 0;
        }
        if (r.nseg > 0) {
            const float4 *N = sc.cmN + 4 * (long long)r.kfirst;
            auto PN = [&](int t) { return st ? sP[jlo + t] : N[4 * t + CM_P]; };   // candidate t's position
            const float4 a0 = PN(0), a1 = PN(r.nseg);
            const float ux = a1.x - a0.x, uy = a1.y - a0.y, uu = ux * ux + uy * uy;
            const float iuu = uu > 0.0f ? 1.0f / uu : 0.0f;
            // layers: cell centres z + 1/2 (brick-relative) within 3 eps (+0.02)
            // of the candidate nodes' height range
            r.zf = max(0, (int)ceilf(a0.z - r.oz - Rc - 0.02f - 0.5f));
            r.zl = min(nzb - 1, (int)floorf(a1.z - r.oz + Rc + 0.02f - 0.5f));
            const float Zf = (float)r.zf + 0.5f + r.oz;
            float dev2 = 0.0f;                   // the largest squared departure (sqrt is monotone)
            int j0 = 0;                          // last segment starting at or below the height of layer zf
#pragma unroll 4
            for (int t = 0; t <= r.nseg; ++t) {
                const float4 a = PN(t);
                const float qx = a.x - a0.x, qy = a.y - a0.y;
                const float tt = __saturatef((qx * ux + qy * uy) * iuu);
                const float ex = qx - tt * ux, ey = qy - tt * uy;
                dev2 = fmaxf(dev2, ex * ex + ey * ey);
                if (t <= r.nseg - 1 && a.z <= Zf) j0 = t;
            }
            const float dev = sqrtf(dev2);
            r.j0 = j0;
            const float reach = Rc + dev + 0.02f;
            r.ux = ux; r.uy = uy; r.iuu = iuu;
            r.ax = a0.x; r.ay = a0.y;
            r.reach2 = r.zf <= r.zl ? reach * reach : -1.0f;
            // every tested cell is within reach + dev + |chord| of a node
            // horizontally and within the brick height + 3 eps + L_max + 1
            // vertically: the band of the FP32 bisector error there
            r.gs = Tr<float>::gsig(reach + dev + sqrtf(uu) + (float)g.bz + Rc + Lmax + 1.0f);
        }
        sc.cmlay[(long long)l * nbz_max + bzi] = r;
    }
}

// the entry of line l in brick br: the layer's record and the brick's corner
static __device__ void cm_make_entry(const GridC &g, const Scratch<float> &sc, int br, int l, int B0, int B1,
                                     int B2, int bz, CmEnt &e) {
    const LineG &lg = sc.lines[l];
    const CmLay r = sc.cmlay[(long long)l * ((g.nz + 3) / 4) + B2 / bz];
    e.br = br;
    e.line = l;
    e.kfirst = r.kfirst;
    e.nseg = r.nseg;
    e.zf = r.zf; e.zl = r.zl; e.j0 = r.j0;
    e.wsh = lg.wshift;
    e.ox = (float)(B0 - r.O0); e.oy = (float)(B1 - r.O1); e.oz = r.oz;
    e.gs = r.gs;
    e.ux = r.ux; e.uy = r.uy; e.iuu = r.iuu;
    e.reach2 = r.reach2;
    e.bx = r.nseg > 0 ? __fsub_rn(r.ax, e.ox) : 0.0f;     // exact: a node within reach of the brick
    e.by = r.nseg > 0 ? __fsub_rn(r.ay, e.oy) : 0.0f;
    {
        const float gr = Tr<float>::grr(lg.R2f);
        e.R2lo = lg.R2f - gr;
        e.R2hi = lg.R2f + gr;
    }
    e.ie2 = lg.ie2f;
    e.eta0 = lg.eta0f;
    e.pad0 = e.pad1 = 0.0f;
}

// one warp per brick: which passes take it, and the entries of a
// column-march brick (candidates in line order, CM_LIST per pass over the
// mask words; the words of a column-march brick are cleared here, as no
// other pass reads them).  Index guards flag status[ST_GUARD] and skip.
constexpr int CM_LIST = 256;
template <typename T>
__global__ void __launch_bounds__(256) k_cm_entries(GridC g, BeamsC b, Scratch<T> sc, int *status) {
    pdl_enter();
#define CHK(c, bit) if (!(c)) { atomicOr(&status[ST_GUARD], bit); } else
    __shared__ int lst[8][CM_LIST];
    const long long brl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (brl >= g.nbrick) return;
    const int br = (int)brl;
    const int W = b.mask_words, wper = (W + 31) / 32;
    uint32_t *mrow = sc.mask + (long long)br * W;
    const int wa = min(W, lane * wper), wb = min(W, wa + wper);
    if (!brick_owned(g, br)) {                         // another slab's cells: neither pass visits them
        if (lane < 3) sc.brickSum[lane * g.nbrick + br] = 0.0;
        if (lane == 0) { CHK(br < g.nbrick_max, 8) { sc.bent_off[br] = 0; sc.bent_n[br] = 0; } }
        for (int w = wa; w < wb; ++w) mrow[w] = 0u;
        return;
    }
    int cnt = 0, bad = 0;
    for (int w = wa; w < wb; ++w) {
        uint32_t m = mrow[w];
        cnt += __popc(m);
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            CHK((w << 5) + bit < b.n_lines, 1) if (!sc.lines[(w << 5) + bit].cm) bad = 1;
        }
    }
    int pre = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    bad = __any_sync(0xffffffffu, bad);
    int off = 0;
    if (!bad && total > 0) {
        if (lane == 0) off = atomicAdd(sc.cment_n, total);
        off = __shfl_sync(0xffffffffu, off, 0);
        if ((long long)off + total > sc.cment_cap) {
            // no room: the brick passes take the brick; its reserved slots
            // below the capacity become empty entries
            bad = 1;
            for (int i = lane; i < total; i += 32)
                if ((long long)off + i < sc.cment_cap) { CHK(off + i >= 0, 2) sc.cment[off + i].nseg = 0; }
        }
    }
    if (lane == 0) {
        // list 0: bricks with candidate lines from the front, bricks without
        // from the back (the spread takes the costly ones first)
        const int t = bad ? 1 : 0;
        const bool back = !bad && total == 0;
        const int pos = atomicAdd(&sc.cmcnt[back ? 4 : t], 1);
        CHK(pos >= 0 && pos < g.nbrick_max, 4) sc.cmlist[back ? g.nbrick_max - 1 - pos : t * g.nbrick_max + pos] = br;
        CHK(br >= 0 && br < g.nbrick_max, 8) { sc.bent_off[br] = bad ? 0 : off; sc.bent_n[br] = bad ? 0 : total; }
    }
    if (bad) return;
    int B0, B1, B2;
    cm_brick_origin(g, br, g.bz, B0, B1, B2);
    const int nzb = min(g.bz, g.nz - B2);
    for (int p0 = 0; p0 < total; p0 += CM_LIST) {
        // the lines of this pass in line order, then one entry per lane
        int pos = pre - cnt;
        if (pos < p0 + CM_LIST && pos + cnt > p0) {
            for (int w = wa; w < wb; ++w) {
                uint32_t m = mrow[w];
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    if (pos >= p0 && pos < p0 + CM_LIST) {
                        CHK(pos - p0 >= 0 && pos - p0 < CM_LIST && wib < 8, 16) lst[wib][pos - p0] = (w << 5) + bit;
                    }
                    ++pos;
                }
            }
        }
        __syncwarp();
        const int nl = min(CM_LIST, total - p0);
        for (int i = lane; i < nl; i += 32) {
            CmEnt e;
            const int l = lst[wib][i];
            CHK(l >= 0 && l < b.n_lines, 32) {
                if constexpr (std::is_same<T, float>::value) cm_make_entry(g, sc, br, l, B0, B1, B2, g.bz, e);
                CHK((long long)off + p0 + i < sc.cment_cap && off + p0 + i >= 0, 64) sc.cment[off + p0 + i] = e;
            }
        }
        __syncwarp();
    }
    for (int w = wa; w < wb; ++w) mrow[w] = 0u;        // read once per step
#undef CHK
}

// ---- weights pass: one warp per entry ------------------------------------------------
struct CmWarpBuf {
    float E[CM_EN][33];              // node row, lane column (padded)
    float4 nodes[CM_EN * 4];         // the entry's node records (entries of at most CM_EN nodes)
    unsigned char cols[BX * BY];     // columns in reach of the entry's line
};
constexpr int CM_WTHREADS = 256;
struct CmWeightSmem {
    CmExact x;
    CmWarpBuf wb[CM_WTHREADS / 32];
};

// the weights pass's per-lane sums: omega eta / eta0 of the current segment's
// two nodes; a node passed by the walk goes to the lane's column of the
// warp's buffer (or, for an entry of more nodes than the buffer holds, to the
// node's weight)
struct CmWeightSink {
    float ra, rb;
    float *col;                      // &E[0][lane]
    bool buf;
    int wsh;
    unsigned long long *wfix;
    __device__ __forceinline__ void emit(const CmCtx &c, int t, float v) {
        if (buf) col[t * 33] += v;
        else if (v > 0.0f) atomicAdd(&wfix[c.kfirst + t], to_fixed(v, wsh));
    }
    __device__ __forceinline__ void adv(const CmCtx &c, int jp) {
        emit(c, jp, ra);
        ra = rb;
        rb = 0.0f;
    }
    __device__ __forceinline__ void pair(const CmCtx &, int, float s, float q) {
        const float qb = __fmul_rn(q, s);
        ra = __fadd_rn(ra, __fsub_rn(q, qb));
        rb = __fadd_rn(rb, qb);
    }
};

// cm_march without a call inside: a value inside a band stops it at its
// layer, which is returned (zl + 1: none); cm_tail_w continues from there
template <typename SINK>
__device__ __forceinline__ int cm_march_fast(const CmCtx &c, CmWalk &w, float Xl, float Yl, int zf, int zl,
                                             SINK &sink) {
    float Zl = __fadd_rn((float)zf + 0.5f, c.oz);
    for (int z = zf; z <= zl; ++z, Zl = __fadd_rn(Zl, 1.0f)) {
        float sg = __fmaf_rn(Zl, w.m1z, w.b1);
        while (sg >= c.gs) {
            cm_adv(c, w, Xl, Yl);
            sink.adv(c, w.j - 1);
            sg = __fmaf_rn(Zl, w.m1z, w.b1);
        }
        if (sg > -c.gs) return z;
        float s, r2;
        cm_geom(w, Zl, s, r2);
        if (r2 < c.R2lo) sink.pair(c, z, s, Tr<float>::ex2(__fmul_rn(-r2, c.ie2)));
        else if (!(r2 > c.R2hi)) return z;
    }
    return zl + 1;
}
static __device__ __noinline__ void cm_tail_w(const CmCtx *c, CmWalk *w, float Xl, float Yl, int z, int zl,
                                              CmWeightSink *sk) {
    cm_march(*c, *w, Xl, Yl, z, zl, *sk);
}

// 16-byte copies global -> shared that complete in the background (cp.async),
// and the wait for a thread's copies
__device__ __forceinline__ void cm_cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src));
}
__device__ __forceinline__ void cm_cp_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

static __device__ __forceinline__ void d_cm_weights_entry(const GridC &g, const Scratch<float> &sc,
                                                          const CmExact *x, const CmEnt &e, CmWarpBuf &wb) {
    const int lane = threadIdx.x & 31;
    if (e.nseg <= 0 || e.zf > e.zl) return;
    int B0, B1, B2;
    cm_brick_origin(g, e.br, g.bz, B0, B1, B2);
    const int nxb = min(BX, g.nx - B0), nyb = min(BY, g.ny - B1);
    const int nseg = e.nseg, zf = e.zf, zl = e.zl, j0 = e.j0;
    const bool buf = nseg + 1 <= CM_EN;
    const float4 *src = sc.cmN + 4 * (long long)e.kfirst;
    if (buf) {                                   // the records arrive while the columns are listed
        for (int r = lane; r < 4 * (nseg + 1); r += 32) cm_cp16(&wb.nodes[r], &src[r]);
        for (int t = 0; t <= nseg; ++t) wb.E[t][lane] = 0.0f;
    }
    const CmCtx c = cm_ctx(buf ? wb.nodes : src, x, e, B0, B1, B2);
    CmWeightSink sk;
    sk.col = &wb.E[0][lane];
    sk.buf = buf;
    sk.wsh = e.wsh;
    sk.wfix = sc.wfix;
    int nc = 0;                                  // the brick's columns in reach, packed over the lanes
    for (int c0 = 0; c0 < BX * BY; c0 += 32) {
        const int col = c0 + lane, tx = col & (BX - 1), ty = col / BX;
        const bool ok = tx < nxb && ty < nyb && cm_reach(e, tx + 0.5f, ty + 0.5f);
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (ok) wb.cols[nc + __popc(bal & ((1u << lane) - 1u))] = (unsigned char)col;
        nc += __popc(bal);
    }
    cm_cp_wait();
    __syncwarp();
    const float Zl0 = __fadd_rn((float)zf + 0.5f, c.oz);
    for (int r0 = 0; r0 < nc; r0 += 32) {
        if (r0 + lane < nc) {
            const int col = wb.cols[r0 + lane];
            const float Xl = (float)(col & (BX - 1)) + 0.5f + c.ox, Yl = (float)(col / BX) + 0.5f + c.oy;
            int j;
            if (!cm_start_fast(c, j0, Xl, Yl, Zl0, j)) {
                const CmCtx cc = c;
                j = cm_start_slow(&cc, j0, Xl, Yl, Zl0);
            }
            CmWalk w;
            cm_walk_at(c, w, j, Xl, Yl);
            sk.ra = 0.0f;
            sk.rb = 0.0f;
            const int zs = cm_march_fast(c, w, Xl, Yl, zf, zl, sk);
            if (zs <= zl) {
                const CmCtx cc = c;
                CmWalk wc = w;
                CmWeightSink skc = sk;
                cm_tail_w(&cc, &wc, Xl, Yl, zs, zl, &skc);
                w.j = wc.j;
                sk.ra = skc.ra;
                sk.rb = skc.rb;
            }
            sk.emit(c, w.j, sk.ra);
            sk.emit(c, w.j + 1, sk.rb);
        }
    }
    __syncwarp();
    if (buf)
        for (int t = lane; t <= nseg; t += 32) {
            float v = 0.0f;
            for (int l2 = 0; l2 < 32; ++l2) v = __fadd_rn(v, wb.E[t][l2]);
            if (v > 0.0f) atomicAdd(&sc.wfix[e.kfirst + t], to_fixed(v, sk.wsh));
        }
    __syncwarp();
}

template <typename T>
__global__ void __launch_bounds__(CM_WTHREADS, 3) k_cm_weights(GridC g, BeamsC b, Scratch<T> sc, StepPtrs<T> p,
                                                               int *status) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CmWeightSmem &sm = *reinterpret_cast<CmWeightSmem *>(smem_raw);
    if (threadIdx.x == 0) cm_exact_init(sm.x, g, b, sc, p, status);
    __syncthreads();
    CmWarpBuf &wb = sm.wb[threadIdx.x >> 5];
    const int n = (int)min((long long)*sc.cment_n, sc.cment_cap);
    // the warps take the entries one at a time from a counter, so the last
    // entries end together
    for (;;) {
        int i = 0;
        if ((threadIdx.x & 31) == 0) i = atomicAdd(&sc.cmcnt[3], 1);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= n) break;
        const CmEnt e = sc.cment[i];
        d_cm_weights_entry(g, sc, &sm.x, e, wb);
    }
}

// ---- spread: one CTA per brick, two columns per thread --------------------------------
// Per batch of up to CM_SB entries, every column of the brick gets the mask
// of the entries in reach of it; the columns are sorted by their number of
// entries and dealt in snake order (thread t takes the t-th and the
// (255 - t)-th), so the threads carry nearly equal work.  A thread marches
// each of its columns through its entries in line order with the layers
// unrolled, the column's sources in registers, and adds them once to the
// brick's sources in shared memory: every column's sum is formed by one
// thread in a fixed order, so S has the same bits whatever thread takes it.
constexpr int CM_STHREADS = 128;      // threads per brick
constexpr int CM_SB = 64;             // entries per batch (one bit each in a column's mask)
constexpr int CM_SNODES = 256;        // node records of a batch kept in shared memory (more: read from global)

// the S tile of a brick goes out by three TMA stores (one per component)
// when the host could describe S as 3-D tensors (16-byte aligned, rows a
// multiple of 16 bytes): on = 1
struct CmStore {
    CUtensorMap m[3];
    int on;
};

template <int BZ> struct alignas(128) CmSpreadSmem {
    float out[3][BZ][BX * BY];        // S of the brick's cells (component, layer, column)
    float4 nodes[CM_SNODES * 4];      // the batch's candidate nodes' records
    CmEnt ent[CM_SB];
    unsigned long long mask[BX * BY]; // per column: the entries in reach
    unsigned short order[BX * BY];    // columns by decreasing number of entries
    int hist[CM_SB + 2];
    int npre[CM_SB + 1];              // candidate nodes before each entry
    int next;                         // next column to take
    int nnz;                          // columns with at least one entry
    int brick;                        // the brick this CTA takes next (list 0 index)
    CmExact x;
    double red[3][CM_STHREADS / 32];
    int redi[CM_STHREADS / 32];
};

// the rest of a column's march (rare): layers z .. zl with the exact
// decisions, the sources added straight to the column in shared memory
struct CmOutSink {
    float *col;                      // &out[0][0][column]
    int cs;                          // the tile's component stride (layers x columns)
    float eta0;
    float4 fa, fb, nF;
    int nsupp;
    __device__ __forceinline__ void adv(const CmCtx &c, int jp) {
        fa = fb;
        fb = nF;
        nF = cm_rec(c, min(jp + 3, c.nseg), CM_F);
    }
    __device__ __forceinline__ void pair(const CmCtx &, int z, float s, float q) {
        ++nsupp;
        const float meq = -__fmul_rn(eta0, q);
        float *o = col + z * (BX * BY);
        o[0] = __fmaf_rn(meq, __fmaf_rn(s, __fsub_rn(fb.x, fa.x), fa.x), o[0]);
        o[cs] = __fmaf_rn(meq, __fmaf_rn(s, __fsub_rn(fb.y, fa.y), fa.y), o[cs]);
        o[2 * cs] = __fmaf_rn(meq, __fmaf_rn(s, __fsub_rn(fb.z, fa.z), fa.z), o[2 * cs]);
    }
};
static __device__ __noinline__ int cm_tail(const CmCtx *c, CmWalk *w, const float4 *f, float Xl, float Yl, int z,
                                           int zl, float eta0, float *col, int cs) {
    CmOutSink sk;
    sk.col = col;
    sk.cs = cs;
    sk.eta0 = eta0;
    sk.fa = f[0]; sk.fb = f[1]; sk.nF = f[2];
    sk.nsupp = 0;
    cm_march(*c, *w, Xl, Yl, z, zl, sk);
    return sk.nsupp;
}

// one column against one entry, the layers unrolled and no call inside:
// the column's sources acc[z][a] -= eta (f^_a + s (f^_b - f^_a)) for its
// pairs inside 3 eps, with cm_march's decisions (the same operations on the
// same values).  A value inside a band stops the march at its layer, which
// is returned (BZ: none); cm_tail continues from there.
template <int BZ>
__device__ __forceinline__ int cm_march_acc(const CmCtx &c, CmWalkL &w, float Xl, float Yl, int zf, int zl, float eta0,
                                            float3 &fa, float3 &fb, float (&acc)[BZ][3], int &nsupp) {
    const float Z0 = __fadd_rn(0.5f, c.oz);
    int stop = BZ;
#pragma unroll
    for (int z = 0; z < BZ; ++z) {
        if (z < zf || z > zl || stop < BZ) continue;
        const float Zl = __fadd_rn(Z0, (float)z);
        float sg = __fmaf_rn(Zl, w.m1z, w.b1);
        while (sg >= c.gs) {
            cm_walkl_at(c, w, w.j + 1, Xl, Yl);
            fa = fb;
            const float4 f = cm_rec(c, w.j + 1, CM_F);
            fb = make_float3(f.x, f.y, f.z);
            sg = __fmaf_rn(Zl, w.m1z, w.b1);
        }
        if (sg > -c.gs) { stop = z; continue; }
        float s, r2;
        cm_geoml(w, Zl, s, r2);
        if (r2 < c.R2lo) {
            ++nsupp;
            const float meq = -__fmul_rn(eta0, Tr<float>::ex2(__fmul_rn(-r2, c.ie2)));
            acc[z][0] = __fmaf_rn(meq, __fmaf_rn(s, __fsub_rn(fb.x, fa.x), fa.x), acc[z][0]);
            acc[z][1] = __fmaf_rn(meq, __fmaf_rn(s, __fsub_rn(fb.y, fa.y), fa.y), acc[z][1]);
            acc[z][2] = __fmaf_rn(meq, __fmaf_rn(s, __fsub_rn(fb.z, fa.z), fa.z), acc[z][2]);
        } else if (!(r2 > c.R2hi)) {
            stop = z;
        }
    }
    return stop;
}

template <int BZ>
__device__ __forceinline__ void d_cm_spread(const GridC &g, const BeamsC &b, const Scratch<float> &sc,
                                            const StepPtrs<float> &p, int *status, const int br, CmSpreadSmem<BZ> &sm,
                                            const CmStore &tma) {
    int B0, B1, B2;
    cm_brick_origin(g, br, BZ, B0, B1, B2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    constexpr int NT = CM_STHREADS, NW = CM_STHREADS / 32;
    const int nzb = min(BZ, g.nz - B2), nxb = min(BX, g.nx - B0), nyb = min(BY, g.ny - B1);
    const long long np = b.n_points;
    {
        float4 *o = reinterpret_cast<float4 *>(&sm.out[0][0][0]);
        for (int i = tid; i < BZ * 3 * BX * BY / 4; i += NT) o[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    int nsupp = 0;
    const int nent = sc.bent_n[br], off = sc.bent_off[br];
    for (int e0 = 0; e0 < nent; e0 += CM_SB) {
        const int ne = min(CM_SB, nent - e0);
        __syncthreads();
        {
            const int4 *src = reinterpret_cast<const int4 *>(sc.cment + off + e0);
            int4 *dst = reinterpret_cast<int4 *>(sm.ent);
            constexpr int Q = sizeof(CmEnt) / 16;
            for (int i = tid; i < ne * Q; i += NT) dst[i] = src[i];
        }
        if (tid < CM_SB + 2) sm.hist[tid] = 0;
        if (tid == 0) sm.next = 0;
        __syncthreads();
        // candidate nodes before each entry (every warp scans the counts), then
        // each warp starts the copies of its entries' node records
        int c0 = lane < ne ? max(sm.ent[lane].nseg, 0) + 1 : 0;
        int c1 = lane + 32 < ne ? max(sm.ent[lane + 32].nseg, 0) + 1 : 0;
        int s0 = c0, s1 = c1;
        for (int o = 1; o < 32; o <<= 1) {
            const int v0 = __shfl_up_sync(0xffffffffu, s0, o), v1 = __shfl_up_sync(0xffffffffu, s1, o);
            if (lane >= o) { s0 += v0; s1 += v1; }
        }
        s1 += __shfl_sync(0xffffffffu, s0, 31);
        const int ntot = __shfl_sync(0xffffffffu, s1, 31);
        if (warp == 0) {
            sm.npre[lane] = s0 - c0;
            sm.npre[lane + 32] = s1 - c1;
            if (lane == 0) sm.npre[CM_SB] = ntot;
        }
        // an entry's records are staged when they fit after the entries before it
        for (int i = warp; i < ne; i += NW) {
            const int pi = __shfl_sync(0xffffffffu, i < 32 ? s0 - c0 : s1 - c1, i & 31);
            const int nn = max(sm.ent[i].nseg, 0) + 1;
            if (pi + nn <= CM_SNODES) {
                const int nr = 4 * nn;
                const float4 *src = sc.cmN + 4 * (long long)sm.ent[i].kfirst;
                for (int r = lane; r < nr; r += 32) cm_cp16(&sm.nodes[4 * pi + r], &src[r]);
            }
        }
        // the entries in reach of each column
        for (int cc = tid; cc < BX * BY; cc += NT) {
            const int tx = cc & (BX - 1), ty = cc / BX;
            unsigned long long m = 0ull;
            if (tx < nxb && ty < nyb)
                for (int i = 0; i < ne; ++i)
                    if (cm_reach(sm.ent[i], tx + 0.5f, ty + 0.5f)) m |= 1ull << i;
            sm.mask[cc] = m;
            atomicAdd(&sm.hist[__popcll(m)], 1);
        }
        cm_cp_wait();
        __syncthreads();
        if (warp == 0) {                               // start of each count, decreasing counts first
            int run = 0;
            for (int k0 = ne; k0 >= 0; k0 -= 32) {
                const int k = k0 - lane;
                const int v = k >= 0 ? sm.hist[k] : 0;
                int inc = v;
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += t;
                }
                if (k >= 0) sm.hist[k] = run + inc - v;
                run += __shfl_sync(0xffffffffu, inc, 31);
            }
            __syncwarp();
            if (lane == 0) sm.nnz = sm.hist[0];        // columns with at least one entry
        }
        __syncthreads();
        const int nnz = sm.nnz;
        for (int cc = tid; cc < BX * BY; cc += NT) sm.order[atomicAdd(&sm.hist[__popcll(sm.mask[cc])], 1)] = (unsigned short)cc;
        __syncthreads();
        // the columns, most entries first, each taken whole by one thread
        for (;;) {
            const int k = atomicAdd(&sm.next, 1);
            if (k >= nnz) break;
            const int cc_col = sm.order[k];
            unsigned long long m = sm.mask[cc_col];
            float acc[BZ][3];
#pragma unroll
            for (int z = 0; z < BZ; ++z) acc[z][0] = acc[z][1] = acc[z][2] = 0.0f;
            const float X = (float)(cc_col & (BX - 1)) + 0.5f, Y = (float)(cc_col / BX) + 0.5f;
            while (m) {
                const int i = __ffsll((long long)m) - 1;
                m &= m - 1;
                const CmEnt &e = sm.ent[i];
                const bool staged = sm.npre[i + 1] <= CM_SNODES;
                const CmCtx c = cm_ctx(staged ? &sm.nodes[4 * sm.npre[i]] : sc.cmN + 4 * (long long)e.kfirst, &sm.x,
                                       e, B0, B1, B2);
                const float Xl = X + c.ox, Yl = Y + c.oy;
                const float Zl0 = __fadd_rn((float)e.zf + 0.5f, c.oz);
                int j;
                if (!cm_start_fast(c, e.j0, Xl, Yl, Zl0, j)) {
                    const CmCtx cc = c;
                    j = cm_start_slow(&cc, e.j0, Xl, Yl, Zl0);
                }
                CmWalkL w;
                cm_walkl_at(c, w, j, Xl, Yl);
                const float4 f0 = cm_rec(c, j, CM_F), f1 = cm_rec(c, j + 1, CM_F);
                float3 fa = make_float3(f0.x, f0.y, f0.z), fb = make_float3(f1.x, f1.y, f1.z);
                const int zs = cm_march_acc<BZ>(c, w, Xl, Yl, e.zf, e.zl, e.eta0, fa, fb, acc, nsupp);
                if (zs <= e.zl) {
                    // the rest of the column out of line, from a walk rebuilt at
                    // the same segment (the same state from the same records)
                    const CmEnt &e2 = sm.ent[i];
                    const CmCtx cc = cm_ctx(sm.npre[i + 1] <= CM_SNODES ? &sm.nodes[4 * sm.npre[i]]
                                                                         : sc.cmN + 4 * (long long)e2.kfirst,
                                            &sm.x, e2, B0, B1, B2);
                    CmWalk wc;
                    cm_walk_at(cc, wc, w.j, Xl, Yl);
                    const float4 fc[3] = {cm_rec(cc, w.j, CM_F), cm_rec(cc, w.j + 1, CM_F),
                                          cm_rec(cc, min(w.j + 2, cc.nseg), CM_F)};
                    nsupp += cm_tail(&cc, &wc, fc, Xl, Yl, zs, e2.zl, e2.eta0, &sm.out[0][0][cc_col], BZ * BX * BY);
                }
            }
#pragma unroll
            for (int z = 0; z < BZ; ++z) {
                sm.out[0][z][cc_col] = __fadd_rn(sm.out[0][z][cc_col], acc[z][0]);
                sm.out[1][z][cc_col] = __fadd_rn(sm.out[1][z][cc_col], acc[z][1]);
                sm.out[2][z][cc_col] = __fadd_rn(sm.out[2][z][cc_col], acc[z][2]);
            }
        }
        // deposits of the zero-weight nodes inside this brick, in line and node order
        if (*sc.anyZero) {
            __syncthreads();
            if (warp == 0)
                for (int i = 0; i < ne; ++i) {
                    const CmEnt &e = sm.ent[i];
                    if (e.nseg <= 0) continue;
                    for (int t0 = 0; t0 <= e.nseg; t0 += 32) {
                        const int t = t0 + lane;
                        int c3[3] = {0, 0, 0};
                        const int k = e.kfirst + t;
                        bool f = t <= e.nseg && __ldg(&sc.cmN[4 * (long long)k + CM_F]).w != 0.0f;
                        if (f) {
                            const int Bv[3] = {B0, B1, B2}, bs[3] = {BX, BY, BZ}, nn[3] = {g.nx, g.ny, g.nz};
                            for (int a = 0; a < 3; ++a) {
                                const float uh = sc.uhi[a * np + k], ul = sc.ulo[a * np + k];
                                const int cc = ffloor(uh, ul);
                                f = f && inside_axis(uh, ul, nn[a]) && cc >= Bv[a] && cc < Bv[a] + bs[a];
                                c3[a] = cc - Bv[a];
                            }
                        }
                        uint32_t bal = __ballot_sync(0xffffffffu, f);
                        while (bal) {
                            const int src = __ffs(bal) - 1;
                            bal &= bal - 1;
                            if (lane == src)
                                for (int a = 0; a < 3; ++a) {
                                    float &o = sm.out[a][c3[2]][c3[1] * BX + c3[0]];
                                    o = __fsub_rn(o, p.F[a][k] / (float)g.V);
                                }
                            __syncwarp();
                        }
                    }
                }
        }
    }
    if (g.rmode && tid == 0) {                       // no recorded pairs in this brick next step
        sc.rcap[br] = 0;
        sc.roff[br] = 0;
        sc.rcnt[br] = 0;
        if (br == 0) sc.rplan[1] = g.bz;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the tile's writes, to the TMA
    __syncthreads();
    // ---- write every cell of the brick once; brick sums of S -----------------
    // one TMA store of the tile per component where S allows it (the brick's
    // cells outside the grid are clipped), else four cells along x per store
    // where the rows allow it, else one
    float cs0 = 0.0f, cs1 = 0.0f, cs2 = 0.0f;
    const long long layer = (long long)g.nx * g.ny;
    const long long base = B0 + (long long)g.nx * B1 + layer * B2;
    const bool use_tma = tma.on != 0;
    const bool vec = (g.nx & 3) == 0 && (nxb & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(p.S[0]) | reinterpret_cast<uintptr_t>(p.S[1]) |
                       reinterpret_cast<uintptr_t>(p.S[2])) & 15) == 0;
    if (use_tma && tid == 0) {
        for (int a = 0; a < 3; ++a)
            asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                         :: "l"(reinterpret_cast<unsigned long long>(&tma.m[a])), "r"(B0), "r"(B1), "r"(B2),
                            "r"((unsigned)__cvta_generic_to_shared(&sm.out[a][0][0]))
                         : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    if (use_tma || vec) {
        for (int q = tid; q < BZ * 3 * (BX * BY / 4); q += NT) {
            const int za = q / (BX * BY / 4), quad = q - za * (BX * BY / 4);
            const int z = za / 3, a = za - 3 * z;
            const int ty = quad / (BX / 4), tx = (quad - ty * (BX / 4)) * 4;
            if (z < nzb && ty < nyb && tx < nxb) {
                const float4 v = *reinterpret_cast<const float4 *>(&sm.out[a][z][ty * BX + tx]);
                if (!use_tma) *reinterpret_cast<float4 *>(p.S[a] + base + tx + (long long)g.nx * ty + layer * z) = v;
                const float t = (v.x + v.y) + (v.z + v.w);
                if (a == 0) cs0 += t; else if (a == 1) cs1 += t; else cs2 += t;
            }
        }
    } else {
        for (int cc = tid; cc < BX * BY; cc += NT) {
            const int tx = cc & (BX - 1), ty = cc / BX;
            if (tx < nxb && ty < nyb) {
                const long long col = base + tx + (long long)g.nx * ty;
                float *S0 = p.S[0] + col, *S1 = p.S[1] + col, *S2 = p.S[2] + col;
                for (int z = 0; z < nzb; ++z) {
                    const float v0 = sm.out[0][z][cc], v1 = sm.out[1][z][cc], v2 = sm.out[2][z][cc];
                    S0[layer * z] = v0; S1[layer * z] = v1; S2[layer * z] = v2;
                    cs0 += v0; cs1 += v1; cs2 += v2;
                }
            }
        }
    }
    // the brick's sums: float-float over the warp (the three components
    // interleaved), then the warps' pairs in FP64, one lane per component
    {
        float h[3] = {cs0, cs1, cs2}, l[3] = {0.0f, 0.0f, 0.0f};
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float oh = __shfl_xor_sync(0xffffffffu, h[a], o), ol = __shfl_xor_sync(0xffffffffu, l[a], o);
                float su, er;
                two_sum(h[a], oh, su, er);
                er = __fadd_rn(er, __fadd_rn(l[a], ol));
                fast_two_sum(su, er, h[a], l[a]);
            }
        }
        if (lane == 0)
            for (int a = 0; a < 3; ++a) *reinterpret_cast<float2 *>(&sm.red[a][warp]) = make_float2(h[a], l[a]);
    }
    for (int o = 16; o > 0; o >>= 1) nsupp += __shfl_down_sync(0xffffffffu, nsupp, o);
    if (lane == 0) sm.redi[warp] = nsupp;
    __syncthreads();
    if (warp == 0 && lane < 3) {
        double t = 0.0;
        for (int w2 = 0; w2 < NW; ++w2) t += w_load<float>(&sm.red[lane][w2]);
        sc.brickSum[lane * g.nbrick + br] = t;
    } else if (warp == 0 && lane == 3) {
        int ns = 0;
        for (int w2 = 0; w2 < NW; ++w2) ns += sm.redi[w2];
        if (ns) atomicAdd(&status[ST_SUPPORT], ns);
        atomicAdd(&status[ST_COLUMN], 1);
    }
}

// persistent: the CTAs take the bricks of list 0 one at a time from a
// counter, so the last bricks end together
template <int BZ>
__global__ void __launch_bounds__(CM_STHREADS, 4) k_cm_spread(GridC g, BeamsC b, Scratch<float> sc, StepPtrs<float> p,
                                                              int *status, const __grid_constant__ CmStore tma) {
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CmSpreadSmem<BZ> &sm = *reinterpret_cast<CmSpreadSmem<BZ> *>(smem_raw);
    if (threadIdx.x == 0) cm_exact_init(sm.x, g, b, sc, p, status);
    const int n0 = sc.cmcnt[0], n = n0 + sc.cmcnt[4];
    for (;;) {
        if (threadIdx.x == 0) sm.brick = atomicAdd(&sc.cmcnt[2], 1);
        __syncthreads();
        const int i = sm.brick;
        if (i >= n) break;
        d_cm_spread<BZ>(g, b, sc, p, status, sc.cmlist[i < n0 ? i : g.nbrick_max - 1 - (i - n0)], sm, tma);
        // the tile's stores have read it before the next brick writes it
        if (threadIdx.x == 0 && tma.on) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncthreads();
    }
    if (threadIdx.x == 0 && tma.on) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // written
}
// the brick passes over the bricks of list 1
template <int BZ, bool FX>
__global__ void __launch_bounds__(SPREAD_THREADS) k_spread_ls(GridC g, BeamsC b, Scratch<float> sc,
                                                              StepPtrs<float> p, int *status) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<float, BZ, FX> &sm = *reinterpret_cast<SpreadSmem<float, BZ, FX> *>(smem_raw);
    const int n = sc.cmcnt[1];
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        d_brick<float, false, BZ, FX>(g, b, sc, p, status, sc.cmlist[g.nbrick_max + i], sm);
        __syncthreads();
    }
}
template <int BZ>
__global__ void __launch_bounds__(SPREAD_THREADS) k_bweights_ls(GridC g, BeamsC b, Scratch<float> sc,
                                                                StepPtrs<float> p, int *status) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<float, BZ, false> &sm = *reinterpret_cast<SpreadSmem<float, BZ, false> *>(smem_raw);
    const int n = sc.cmcnt[1];
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        d_brick<float, true, BZ, false>(g, b, sc, p, status, sc.cmlist[g.nbrick_max + i], sm);
        __syncthreads();
    }
}

}  // namespace al
