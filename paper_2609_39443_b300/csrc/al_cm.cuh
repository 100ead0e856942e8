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
// only outside a band around zero that bounds the FP32 error (positions are
// staged relative to the brick corner); inside the band the float-float test
// of "segment k closer than k-1" decides, then an FP64 evaluation of the
// paper's distances in the oracle's operation order, exactly as in the brick
// passes, so every (cell, line) pair inside 3 eps is the oracle's.
//
// Passes.  Both passes run the same walk (cm_start, cm_advance, cm_pair) with the same
// explicitly rounded operations on the same staged values, so they take the
// same decisions and the same (s, eta) bits for every pair:
//   k_cm_weights  one warp per candidate line; its lanes take the brick's
//                 columns in reach of the line, 32 at a time, and march the
//                 layers together; each lane adds omega eta / eta0 of its
//                 pairs per node into its own column of a per-warp buffer,
//                 whose rows are summed in a fixed order and added to the
//                 node's fixed-point weight (exact integer sums, so the
//                 result does not depend on the order of the bricks)
//   k_cm_spread   one thread per column of the brick; it marches each line in
//                 reach of its column in line order and subtracts
//                 eta (f^_a + s (f^_b - f^_a)) from its cells' sources in
//                 shared memory; every cell of S is written once, with no
//                 atomics, and the zero-weight deposits follow in line and
//                 node order as in the brick passes
// k_cm_classify sends each brick to these passes or to the brick passes.
#pragma once

namespace al {

constexpr int CM_ENT = 32;       // lines per batch (one bit each in a column's reach mask)
constexpr int CM_LIST = 512;     // candidate lines per pass over a brick's mask words
constexpr int CM_EN = 48;        // nodes of one line in a warp's weight buffer
constexpr int CM_WARPS = SPREAD_THREADS / 32;

struct CmEntries {
    int line[CM_ENT], first[CM_ENT], n[CM_ENT], jlo[CM_ENT], nseg[CM_ENT], base[CM_ENT];
    int zf[CM_ENT], zl[CM_ENT], wsh[CM_ENT];
    float ax[CM_ENT], ay[CM_ENT], ux[CM_ENT], uy[CM_ENT], iuu[CM_ENT], reach2[CM_ENT];   // 2-D chord
    float R2lo[CM_ENT], R2hi[CM_ENT], ie2[CM_ENT], eta0[CM_ENT], gs[CM_ENT];
    double eps[CM_ENT];
};

template <int BZ> struct CmSpreadBuf { float acc[BZ][3][BX * BY]; };          // S of the brick's cells
struct CmWeightBuf {
    float E[CM_WARPS][CM_EN][33];                 // per warp: node row, lane column (padded)
    unsigned char cols[CM_WARPS][BX * BY];        // per warp: columns in reach of its line
};

template <int BZ, bool WP> struct CmSmem {
    float4 A[CM_NN];      // node position relative to the brick corner; w: 1/|D|^2 of the segment it starts
    float4 M[CM_NN];      // bisector unit normal at the node (interior nodes)
    float4 D[CM_NN];      // vector of the segment the node starts
    float4 F[CM_NN];      // spread: f^ at the node; w = 1 when w_k = 0 (its load is deposited)
    int sk[CM_NN];        // global node index
    int list[CM_LIST];
    int nlist, more, nbatch, nstaged;
    CmEntries e;
    unsigned short jz[CM_ENT][BZ];                // segment containing each layer's height
    typename std::conditional<WP, CmWeightBuf, CmSpreadBuf<BZ>>::type u;
    double red[3][CM_WARPS];
    int redi[CM_WARPS];
};

// ---- slow paths (rare): exact decisions --------------------------------------
// sigma of the bisector at node k (staged position a) for the cell (X, Y, Z)
// relative to the brick corner: the FP32 value sg outside the band of its
// error at the cell's distance from the node, else the float-float test of
// "segment k closer than k-1", else FP64
static __device__ __noinline__ bool cm_sig_slow(const GridC &g, const Scratch<float> &sc, const StepPtrs<float> &p,
                                         int k, int B0, int B1, int B2, float X, float Y, float Z, float sg,
                                         float4 a, int *status) {
    const float x0 = X - a.x, x1 = Y - a.y, x2 = Z - a.z;
    const float gsx = Tr<float>::gsig(sqrtf(x0 * x0 + x1 * x1 + x2 * x2));
    if (sg > gsx) return true;
    if (sg < -gsx) return false;
    const int r = ff_later_closer((const float *)sc.uhi, sc.ulo, (long long)p.np, k, B0, B1, B2, X, Y, Z);
    if (r >= 0) return r == 1;
    atomicAdd(&status[ST_REFINED], 1);
    return later_closer_f64(g, p, k, B0 + (int)X, B1 + (int)Y, B2 + (int)Z);
}
// r <= 3 eps in FP64 for segment k of a line of n nodes
static __device__ __noinline__ bool cm_in_slow(const GridC &g, const StepPtrs<float> &p, double eps, int k, int n, int ci,
                                        int cj, int ck, int *status) {
    atomicAdd(&status[ST_REFINED], 1);
    return within_f64(g, p, eps, k, n, ci, cj, ck);
}

// ---- the walk of one column against one staged line ---------------------------
struct CmWalk {
    int j;                        // current segment (index within the line's staged range)
    float xx, xy, pz;             // X - P_j.x, Y - P_j.y, P_j.z
    float dx, dy, dz, il2;        // D_j and 1/|D_j|^2
    float dbase;                  // (X - P_j.x) D_x + (Y - P_j.y) D_y - P_j.z D_z
    float b1, m1z;                // sigma_{j+1}(Z) = b1 + Z m1z; no next bisector: b1 = -inf
};

struct CmCtx {                    // the brick and the line, for the slow paths
    const GridC *g;
    const Scratch<float> *sc;
    const StepPtrs<float> *p;
    int *status;
    int B0, B1, B2;
    int kfirst;                   // global index of the line's staged node 0
    int n;                        // nodes of the line
    double eps;
};

__device__ __forceinline__ void cm_seg(CmWalk &w, const float4 *A, const float4 *D, const float4 *M, int s,
                                       bool has_next, float X, float Y) {
    const float4 a = A[s], d = D[s];
    w.xx = __fsub_rn(X, a.x);
    w.xy = __fsub_rn(Y, a.y);
    w.pz = a.z;
    w.il2 = a.w;
    w.dx = d.x; w.dy = d.y; w.dz = d.z;
    w.dbase = __fmaf_rn(-a.z, d.z, __fmaf_rn(w.xy, d.y, __fmul_rn(w.xx, d.x)));
    if (has_next) {
        const float4 a1 = A[s + 1], m = M[s + 1];
        w.b1 = __fmaf_rn(-a1.z, m.z, __fmaf_rn(__fsub_rn(Y, a1.y), m.y, __fmul_rn(__fsub_rn(X, a1.x), m.x)));
        w.m1z = m.z;
    } else {
        w.b1 = -INFINITY;
        w.m1z = 0.0f;
    }
}

// sigma of staged node s (> 0: the cell's closest segment is at or after it)
__device__ __forceinline__ bool cm_pos(const CmCtx &c, const float4 *A, const float4 *M, int s, int jn, float X,
                                       float Y, float Z, float gs) {
    const float4 a = A[s], m = M[s];
    const float sg = __fmaf_rn(__fsub_rn(Z, a.z), m.z,
                               __fmaf_rn(__fsub_rn(Y, a.y), m.y, __fmul_rn(__fsub_rn(X, a.x), m.x)));
    if (sg >= gs) return true;
    if (sg <= -gs) return false;
    return cm_sig_slow(*c.g, *c.sc, *c.p, c.kfirst + jn, c.B0, c.B1, c.B2, X, Y, Z, sg, a, c.status);
}

// closest segment of the column's cell at height Z0: a walk from j0 (the
// segment containing that height), down while the bisector at j is not
// positive, then up while the next one is
__device__ __forceinline__ int cm_start(const CmCtx &c, const float4 *A, const float4 *M, int base, int nseg, int j0,
                                        float X, float Y, float Z0, float gs) {
    int j = j0;
    while (j > 0 && !cm_pos(c, A, M, base + j, j, X, Y, Z0, gs)) --j;
    while (j < nseg - 1 && cm_pos(c, A, M, base + j + 1, j + 1, X, Y, Z0, gs)) ++j;
    return j;
}

// the next bisector test at height Z: advance the walk while it is positive
// (ADV is called after each advance with the previous segment index)
template <typename ADV>
__device__ __forceinline__ void cm_advance(const CmCtx &c, CmWalk &w, const float4 *A, const float4 *D,
                                           const float4 *M, int base, int nseg, float X, float Y, float Z, float gs,
                                           ADV &&adv) {
    for (;;) {
        const float sg = __fmaf_rn(Z, w.m1z, w.b1);
        if (!(sg > -gs)) break;
        if (!(sg >= gs) &&
            !cm_sig_slow(*c.g, *c.sc, *c.p, c.kfirst + w.j + 1, c.B0, c.B1, c.B2, X, Y, Z, sg, A[base + w.j + 1],
                         c.status))
            break;
        const int jp = w.j;
        ++w.j;
        cm_seg(w, A, D, M, base + w.j, w.j + 1 < nseg, X, Y);
        adv(jp);
    }
}

// the pair (cell at height Z, segment w.j): clamped foot s and whether r <= 3 eps;
// q = exp(-(r / eps)^2) (eta / eta0) when inside, else 0
__device__ __forceinline__ bool cm_pair(const CmCtx &c, const CmWalk &w, float Z, float R2lo, float R2hi, float ie2,
                                        int ci, int cj, int ck, float &s, float &q) {
    const float xz = __fsub_rn(Z, w.pz);
    const float dot = __fmaf_rn(Z, w.dz, w.dbase);      // (X - P) . D
    s = __saturatef(__fmul_rn(dot, w.il2));
    const float ex = __fmaf_rn(-s, w.dx, w.xx), ey = __fmaf_rn(-s, w.dy, w.xy), ez = __fmaf_rn(-s, w.dz, xz);
    const float r2 = __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
    bool in;
    if (r2 < R2lo) in = true;
    else if (r2 > R2hi) in = false;
    else in = cm_in_slow(*c.g, *c.p, c.eps, c.kfirst + w.j, c.n, ci, cj, ck, c.status);
    q = in ? Tr<float>::ex2(__fmul_rn(-r2, ie2)) : 0.0f;
    return in;
}

// is the column (X, Y) within reach of entry e: within 3 eps + the arc's
// deviation of the 2-D chord of its staged nodes (every cell within 3 eps of
// the arc projects within that distance of the chord)
template <typename SMT>
__device__ __forceinline__ bool cm_reach(const SMT &sm, int e, float X, float Y) {
    const float qx = X - sm.e.ax[e], qy = Y - sm.e.ay[e];
    const float ux = sm.e.ux[e], uy = sm.e.uy[e];
    const float t = __saturatef((qx * ux + qy * uy) * sm.e.iuu[e]);
    const float ex = qx - t * ux, ey = qy - t * uy;
    return ex * ex + ey * ey <= sm.e.reach2[e];
}

// ---- per brick: candidate lines, entries, staging ------------------------------
__device__ __forceinline__ void cm_brick_origin(const GridC &g, int br, int bz, int &B0, int &B1, int &B2) {
    const int nbxy = g.nbx * g.nby;
    const int bzi = br / nbxy, rem = br - bzi * nbxy;
    const int byi = rem / g.nbx, bxi = rem - byi * g.nbx;
    B0 = bxi * BX; B1 = byi * BY; B2 = bzi * bz;
}

// candidate lines of the brick (line order), pass `pass` of CM_LIST; warp 0.
// clear: the spread clears the mask words in the last pass
template <typename SMT>
__device__ void cm_candidates(const BeamsC &b, const Scratch<float> &sc, int br, int pass, bool clear, SMT &sm) {
    const int lane = threadIdx.x & 31;
    const int W = b.mask_words, wper = (W + 31) / 32;
    uint32_t *mrow = sc.mask + (long long)br * W;
    const int wa = min(W, lane * wper), wb = min(W, wa + wper);
    int cnt = 0;
    for (int w = wa; w < wb; ++w) cnt += __popc(mrow[w]);
    int pre = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    const int lo = pass * CM_LIST, hi = lo + CM_LIST;
    int pos = pre - cnt;
    if (pos < hi && pos + cnt > lo) {
        for (int w = wa; w < wb; ++w) {
            uint32_t m = mrow[w];
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                if (pos >= lo && pos < hi) sm.list[pos - lo] = (w << 5) + bit;
                ++pos;
            }
        }
    }
    __syncwarp();
    if (clear && total <= hi)
        for (int w = wa; w < wb; ++w) mrow[w] = 0u;
    if (lane == 0) {
        sm.nlist = max(0, min(total - lo, CM_LIST));
        sm.more = total > hi;
    }
}

// entry e of the batch for line l (one warp): the candidate segments are those
// whose height range meets the brick's layer centres widened by 3 eps + 0.02
// (node heights increase along the line, so they form a range [jlo, jhi])
template <typename SMT>
__device__ void cm_entry(const GridC &g, const BeamsC &b, const Scratch<float> &sc, int e, int l, int B2, int nzb,
                         SMT &sm) {
    const int lane = threadIdx.x & 31;
    const long long np = b.n_points;
    const LineG &lg = sc.lines[l];
    const int first = lg.first, n = lg.n;
    const float zlo = (float)B2 + 0.5f - lg.Rc - 0.02f, zhi = (float)B2 + (float)nzb - 0.5f + lg.Rc + 0.02f;
    int jlo = n, jhi = -1;
    for (int q = lane; q < n; q += 32) {
        const float z = sc.uhi[2 * np + first + q];
        if (q >= 1 && z >= zlo) jlo = min(jlo, q - 1);
        if (q <= n - 2 && z <= zhi) jhi = max(jhi, q);
    }
    jlo = __reduce_min_sync(0xffffffffu, jlo);
    jhi = __reduce_max_sync(0xffffffffu, jhi);
    if (lane == 0) {
        sm.e.line[e] = l;
        sm.e.first[e] = first;
        sm.e.n[e] = n;
        sm.e.jlo[e] = jlo;
        sm.e.nseg[e] = jhi >= jlo ? jhi - jlo + 1 : 0;
        sm.e.wsh[e] = lg.wshift;
        const float gr = Tr<float>::grr(lg.R2f);
        sm.e.R2lo[e] = lg.R2f - gr;
        sm.e.R2hi[e] = lg.R2f + gr;
        sm.e.ie2[e] = lg.ie2f;
        sm.e.eta0[e] = lg.eta0f;
        sm.e.eps[e] = b.eps[l];
    }
}

// after staging: the 2-D chord and its deviation, the layer range, the
// bisector band, and the segment containing each layer's height (one warp
// per entry)
template <int BZ, typename SMT>
__device__ void cm_entry_geometry(const Scratch<float> &sc, int e, int nzb, SMT &sm) {
    const int lane = threadIdx.x & 31;
    const int nseg = sm.e.nseg[e], base = sm.e.base[e];
    if (nseg <= 0) return;
    const LineG &lg = sc.lines[sm.e.line[e]];
    const float4 a0 = sm.A[base], a1 = sm.A[base + nseg];
    const float ux = a1.x - a0.x, uy = a1.y - a0.y, uu = ux * ux + uy * uy;
    const float iuu = uu > 0.0f ? 1.0f / uu : 0.0f;
    float dev = 0.0f;
    for (int t = lane; t <= nseg; t += 32) {
        const float4 a = sm.A[base + t];
        const float qx = a.x - a0.x, qy = a.y - a0.y;
        const float tt = __saturatef((qx * ux + qy * uy) * iuu);
        const float ex = qx - tt * ux, ey = qy - tt * uy;
        dev = fmaxf(dev, sqrtf(ex * ex + ey * ey));
    }
    for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    const float Rc = lg.Rc;
    const int zf = max(0, (int)ceilf(a0.z - Rc - 0.02f - 0.5f));
    const int zl = min(nzb - 1, (int)floorf(a1.z + Rc + 0.02f - 0.5f));
    if (lane == 0) {
        const float reach = Rc + dev + 0.02f;
        sm.e.ax[e] = a0.x; sm.e.ay[e] = a0.y; sm.e.ux[e] = ux; sm.e.uy[e] = uy; sm.e.iuu[e] = iuu;
        sm.e.reach2[e] = reach * reach;
        sm.e.zf[e] = zf;
        sm.e.zl[e] = zl;
        // every tested cell is within reach + dev + |chord| of a node horizontally and
        // within the brick height + 3 eps + L_max + 1 vertically: the bisector error band there
        const float xmax = reach + dev + sqrtf(uu) + (float)BZ + Rc + lg.Lmax + 1.0f;
        sm.e.gs[e] = Tr<float>::gsig(xmax);
    }
    if (lane < BZ) {
        const float Z = lane + 0.5f;
        int lo = 0, hi = nseg - 1;                   // last segment starting at or below Z
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sm.A[base + mid].z <= Z) lo = mid; else hi = mid - 1;
        }
        sm.jz[e][lane] = (unsigned short)lo;
    }
}

// one batch of the candidate list starting at li: entries, node budget,
// staging, geometry.  Returns the number of entries.
template <int BZ, bool WP, typename SMT>
__device__ int cm_batch(const GridC &g, const BeamsC &b, const Scratch<float> &sc, int li, int B0, int B1, int B2,
                        int nzb, SMT &sm) {
    const int warp = threadIdx.x >> 5;
    const long long np = b.n_points;
    const int nb = min(sm.nlist - li, CM_ENT);
    for (int e = warp; e < nb; e += CM_WARPS) cm_entry(g, b, sc, e, sm.list[li + e], B2, nzb, sm);
    __syncthreads();
    if (threadIdx.x == 0) {
        int base = 0, e = 0;
        for (; e < nb; ++e) {
            const int cnt = sm.e.nseg[e] > 0 ? sm.e.nseg[e] + 1 : 0;
            if (base + cnt > CM_NN) break;
            sm.e.base[e] = base;
            base += cnt;
        }
        if (e == 0) {                                // never: k_lines bounds a line's range below CM_NN
            sm.e.nseg[0] = 0;                        // (guard: the line is dropped rather than looping)
            sm.e.base[0] = 0;
            e = 1;
        }
        sm.nbatch = e;
        sm.nstaged = base;
    }
    __syncthreads();
    const int ne = sm.nbatch;
    for (int s = threadIdx.x; s < sm.nstaged; s += SPREAD_THREADS) {
        // the last entry whose base is <= s holds slot s (an entry without
        // nodes shares the next entry's base)
        int lo = 0, hi = ne - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sm.e.base[mid] <= s) lo = mid; else hi = mid - 1;
        }
        const int e = lo;
        const int k = sm.e.first[e] + sm.e.jlo[e] + (s - sm.e.base[e]);
        sm.A[s] = make_float4(rel(sc.uhi[k], sc.ulo[k], B0), rel(sc.uhi[np + k], sc.ulo[np + k], B1),
                              rel(sc.uhi[2 * np + k], sc.ulo[2 * np + k], B2), sc.segIl2[k]);
        sm.M[s] = make_float4(sc.nodeM[k], sc.nodeM[np + k], sc.nodeM[2 * np + k], 0.0f);
        sm.D[s] = make_float4(sc.segD[k], sc.segD[np + k], sc.segD[2 * np + k], 0.0f);
        sm.sk[s] = k;
        if (!WP) sm.F[s] = make_float4(sc.fhat[k], sc.fhat[np + k], sc.fhat[2 * np + k], sc.w[k] == 0.0 ? 1.0f : 0.0f);
    }
    __syncthreads();
    for (int e = warp; e < ne; e += CM_WARPS) cm_entry_geometry<BZ>(sc, e, nzb, sm);
    __syncthreads();
    return ne;
}

// ---- weights pass -----------------------------------------------------------------
template <int BZ>
__device__ void d_cm_weights(const GridC &g, const BeamsC &b, const Scratch<float> &sc, const StepPtrs<float> &p,
                             int *status, const int br, CmSmem<BZ, true> &sm) {
    int B0, B1, B2;
    cm_brick_origin(g, br, BZ, B0, B1, B2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nzb = min(BZ, g.nz - B2), nxb = min(BX, g.nx - B0), nyb = min(BY, g.ny - B1);
    float (*E)[33] = sm.u.E[warp];
    unsigned char *cols = sm.u.cols[warp];
    for (int pass = 0;; ++pass) {
        __syncthreads();
        if (warp == 0) cm_candidates(b, sc, br, pass, false, sm);
        __syncthreads();
        for (int li = 0; li < sm.nlist;) {
            const int ne = cm_batch<BZ, true>(g, b, sc, li, B0, B1, B2, nzb, sm);
            for (int e = warp; e < ne; e += CM_WARPS) {
                const int nseg = sm.e.nseg[e];
                if (nseg <= 0) continue;
                const int base = sm.e.base[e], zf = sm.e.zf[e], zl = sm.e.zl[e];
                if (zf > zl) continue;
                CmCtx c{&g, &sc, &p, status, B0, B1, B2, sm.e.first[e] + sm.e.jlo[e], sm.e.n[e], sm.e.eps[e]};
                const float gs = sm.e.gs[e], R2lo = sm.e.R2lo[e], R2hi = sm.e.R2hi[e], ie2 = sm.e.ie2[e];
                const int wsh = sm.e.wsh[e];
                const bool buf = nseg + 1 <= CM_EN;     // else each lane adds its sums to the nodes directly
                if (buf)
                    for (int t = 0; t <= nseg; ++t) E[t][lane] = 0.0f;
                // the brick's columns in reach of the line, packed over the lanes
                int nc = 0;
                for (int c0 = 0; c0 < BX * BY; c0 += 32) {
                    const int col = c0 + lane, tx = col & (BX - 1), ty = col / BX;
                    const bool ok = tx < nxb && ty < nyb && cm_reach(sm, e, tx + 0.5f, ty + 0.5f);
                    const unsigned bal = __ballot_sync(0xffffffffu, ok);
                    if (ok) cols[nc + __popc(bal & ((1u << lane) - 1u))] = (unsigned char)col;
                    nc += __popc(bal);
                }
                __syncwarp();
                auto emit = [&](int t, float v) {
                    if (buf) E[t][lane] += v;
                    else if (v > 0.0f) atomicAdd(&sc.wfix[c.kfirst + t], to_fixed(v, wsh));
                };
                for (int r0 = 0; r0 < nc; r0 += 32) {
                    if (r0 + lane >= nc) continue;
                    const int col = cols[r0 + lane], tx = col & (BX - 1), ty = col / BX;
                    const float X = tx + 0.5f, Y = ty + 0.5f;
                    CmWalk w;
                    w.j = cm_start(c, sm.A, sm.M, base, nseg, sm.jz[e][zf], X, Y, zf + 0.5f, gs);
                    cm_seg(w, sm.A, sm.D, sm.M, base + w.j, w.j + 1 < nseg, X, Y);
                    float ra = 0.0f, rb = 0.0f;
                    for (int z = zf; z <= zl; ++z) {
                        const float Z = z + 0.5f;
                        cm_advance(c, w, sm.A, sm.D, sm.M, base, nseg, X, Y, Z, gs, [&](int jp) {
                            emit(jp, ra);
                            ra = rb;
                            rb = 0.0f;
                        });
                        float s, q;
                        cm_pair(c, w, Z, R2lo, R2hi, ie2, B0 + tx, B1 + ty, B2 + z, s, q);
                        const float wb = __fmul_rn(q, s);
                        ra = __fadd_rn(ra, __fsub_rn(q, wb));
                        rb = __fadd_rn(rb, wb);
                    }
                    emit(w.j, ra);
                    emit(w.j + 1, rb);
                }
                __syncwarp();
                if (buf)
                    for (int t = lane; t <= nseg; t += 32) {
                        float v = 0.0f;
                        for (int l2 = 0; l2 < 32; ++l2) v = __fadd_rn(v, E[t][l2]);
                        if (v > 0.0f) atomicAdd(&sc.wfix[c.kfirst + t], to_fixed(v, wsh));
                    }
                __syncwarp();
            }
            li += ne;
            __syncthreads();
        }
        if (!sm.more) break;
    }
}

// ---- spread -----------------------------------------------------------------------
template <int BZ>
__device__ void d_cm_spread(const GridC &g, const BeamsC &b, const Scratch<float> &sc, const StepPtrs<float> &p,
                            int *status, const int br, CmSmem<BZ, false> &sm) {
    int B0, B1, B2;
    cm_brick_origin(g, br, BZ, B0, B1, B2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int nzb = min(BZ, g.nz - B2), nxb = min(BX, g.nx - B0), nyb = min(BY, g.ny - B1);
    const int tx = tid % BX, ty = tid / BX;
    const bool mine = tx < nxb && ty < nyb;
    const float X = tx + 0.5f, Y = ty + 0.5f;
    const long long np = b.n_points;
    for (int z = 0; z < BZ; ++z)
        for (int a = 0; a < 3; ++a) sm.u.acc[z][a][tid] = 0.0f;
    int nsupp = 0;
    for (int pass = 0;; ++pass) {
        __syncthreads();
        if (warp == 0) cm_candidates(b, sc, br, pass, true, sm);
        __syncthreads();
        for (int li = 0; li < sm.nlist;) {
            const int ne = cm_batch<BZ, false>(g, b, sc, li, B0, B1, B2, nzb, sm);
            // the lines in reach of this column, in line order
            unsigned int mask = 0u;
            if (mine)
                for (int e = 0; e < ne; ++e)
                    if (sm.e.nseg[e] > 0 && sm.e.zf[e] <= sm.e.zl[e] && cm_reach(sm, e, X, Y)) mask |= 1u << e;
            while (mask) {
                const int e = __ffs(mask) - 1;
                mask &= mask - 1;
                const int nseg = sm.e.nseg[e], base = sm.e.base[e], zf = sm.e.zf[e], zl = sm.e.zl[e];
                CmCtx c{&g, &sc, &p, status, B0, B1, B2, sm.e.first[e] + sm.e.jlo[e], sm.e.n[e], sm.e.eps[e]};
                const float gs = sm.e.gs[e], R2lo = sm.e.R2lo[e], R2hi = sm.e.R2hi[e], ie2 = sm.e.ie2[e];
                const float eta0 = sm.e.eta0[e];
                CmWalk w;
                w.j = cm_start(c, sm.A, sm.M, base, nseg, sm.jz[e][zf], X, Y, zf + 0.5f, gs);
                cm_seg(w, sm.A, sm.D, sm.M, base + w.j, w.j + 1 < nseg, X, Y);
                float4 fa = sm.F[base + w.j], fb = sm.F[base + w.j + 1];
                float df0 = __fsub_rn(fb.x, fa.x), df1 = __fsub_rn(fb.y, fa.y), df2 = __fsub_rn(fb.z, fa.z);
                for (int z = zf; z <= zl; ++z) {
                    const float Z = z + 0.5f;
                    cm_advance(c, w, sm.A, sm.D, sm.M, base, nseg, X, Y, Z, gs, [&](int) {
                        fa = fb;
                        fb = sm.F[base + w.j + 1];
                        df0 = __fsub_rn(fb.x, fa.x); df1 = __fsub_rn(fb.y, fa.y); df2 = __fsub_rn(fb.z, fa.z);
                    });
                    float s, q;
                    if (cm_pair(c, w, Z, R2lo, R2hi, ie2, B0 + tx, B1 + ty, B2 + z, s, q)) {
                        ++nsupp;
                        const float eq = __fmul_rn(eta0, q);
                        float *acc = &sm.u.acc[z][0][tid];
                        acc[0] = __fmaf_rn(-eq, __fmaf_rn(s, df0, fa.x), acc[0]);
                        acc[BX * BY] = __fmaf_rn(-eq, __fmaf_rn(s, df1, fa.y), acc[BX * BY]);
                        acc[2 * BX * BY] = __fmaf_rn(-eq, __fmaf_rn(s, df2, fa.z), acc[2 * BX * BY]);
                    }
                }
            }
            __syncthreads();
            // deposits of the zero-weight nodes inside this brick, in line and node order
            if (warp == 0 && *sc.anyZero) {
                const int tot = sm.nstaged;
                for (int s0 = 0; s0 < tot; s0 += 32) {
                    const int sl = s0 + lane;
                    int c3[3] = {0, 0, 0};
                    bool f = sl < tot && sm.F[sl].w != 0.0f;
                    int k = 0;
                    if (f) {
                        k = sm.sk[sl];
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
                                float &acc = sm.u.acc[c3[2]][a][c3[1] * BX + c3[0]];
                                acc = __fsub_rn(acc, p.F[a][k] / (float)g.V);
                            }
                        __syncwarp();
                    }
                }
            }
            li += ne;
            __syncthreads();
        }
        if (!sm.more) break;
    }
    if (g.rmode && tid == 0) {                       // no recorded pairs in this brick next step
        sc.rcap[br] = 0;
        sc.roff[br] = 0;
        sc.rcnt[br] = 0;
        if (br == 0) sc.rplan[1] = g.bz;
    }
    // ---- write every cell of the brick once; brick sums of S -----------------
    float cs0 = 0.0f, cs1 = 0.0f, cs2 = 0.0f;
    if (mine) {
        const long long layer = (long long)g.nx * g.ny;
        const long long col = (B0 + tx) + (long long)g.nx * (B1 + ty) + layer * B2;
        for (int z = 0; z < nzb; ++z) {
            const long long idx = col + layer * z;
            const float v0 = sm.u.acc[z][0][tid], v1 = sm.u.acc[z][1][tid], v2 = sm.u.acc[z][2][tid];
            p.S[0][idx] = v0; p.S[1][idx] = v1; p.S[2][idx] = v2;
            cs0 += v0; cs1 += v1; cs2 += v2;
        }
    }
    {
        Acc<float> a3[3];
        a3[0].add(cs0); a3[1].add(cs1); a3[2].add(cs2);
        for (int a = 0; a < 3; ++a) w_store(&sm.red[a][warp], a3[a]);
    }
    for (int o = 16; o > 0; o >>= 1) nsupp += __shfl_down_sync(0xffffffffu, nsupp, o);
    if (lane == 0) sm.redi[warp] = nsupp;
    __syncthreads();
    if (tid == 0) {
        int ns = 0;
        for (int a = 0; a < 3; ++a) {
            double t = 0.0;
            for (int w2 = 0; w2 < CM_WARPS; ++w2) t += w_load<float>(&sm.red[a][w2]);
            sc.brickSum[a * g.nbrick + br] = t;
        }
        for (int w2 = 0; w2 < CM_WARPS; ++w2) ns += sm.redi[w2];
        if (ns) atomicAdd(&status[ST_SUPPORT], ns);
        atomicAdd(&status[ST_COLUMN], 1);
    }
}

// ---- kernels ------------------------------------------------------------------------
// one warp per brick: to the column-march passes when every candidate line
// takes the column march (list 0), else to the brick passes (list 1)
template <typename T>
__global__ void __launch_bounds__(256) k_cm_classify(GridC g, BeamsC b, Scratch<T> sc) {
    const long long br = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (br >= g.nbrick) return;
    const int W = b.mask_words;
    const uint32_t *mrow = sc.mask + br * W;
    int bad = 0;
    for (int w = lane; w < W; w += 32) {
        uint32_t m = mrow[w];
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            if (!sc.lines[(w << 5) + bit].cm) bad = 1;
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        const int t = bad ? 1 : 0;
        const int pos = atomicAdd(&sc.cmcnt[t], 1);
        sc.cmlist[t * g.nbrick_max + pos] = (int)br;
    }
}

// persistent: the CTAs walk the bricks of one list
template <int BZ>
__global__ void __launch_bounds__(SPREAD_THREADS, 2) k_cm_weights(GridC g, BeamsC b, Scratch<float> sc,
                                                                  StepPtrs<float> p, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CmSmem<BZ, true> &sm = *reinterpret_cast<CmSmem<BZ, true> *>(smem_raw);
    const int n = sc.cmcnt[0];
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        d_cm_weights<BZ>(g, b, sc, p, status, sc.cmlist[i], sm);
        __syncthreads();
    }
}
template <int BZ>
__global__ void __launch_bounds__(SPREAD_THREADS, 2) k_cm_spread(GridC g, BeamsC b, Scratch<float> sc,
                                                                 StepPtrs<float> p, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CmSmem<BZ, false> &sm = *reinterpret_cast<CmSmem<BZ, false> *>(smem_raw);
    const int n = sc.cmcnt[0];
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        d_cm_spread<BZ>(g, b, sc, p, status, sc.cmlist[i], sm);
        __syncthreads();
    }
}
// the brick passes over the bricks of list 1
template <int BZ, bool FX>
__global__ void __launch_bounds__(SPREAD_THREADS) k_spread_ls(GridC g, BeamsC b, Scratch<float> sc,
                                                              StepPtrs<float> p, int *status) {
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
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<float, BZ, false> &sm = *reinterpret_cast<SpreadSmem<float, BZ, false> *>(smem_raw);
    const int n = sc.cmcnt[1];
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        d_brick<float, true, BZ, false>(g, b, sc, p, status, sc.cmlist[g.nbrick_max + i], sm);
        __syncthreads();
    }
}

}  // namespace al
