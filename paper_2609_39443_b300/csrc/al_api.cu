// al_api.cu -- host side of the C ABI declared in include/al.h.
//
// Owns the per-instance device scratch, validates descriptors on the host,
// and enqueues the kernels of al_kernels.cuh on the caller's stream.  No
// allocation, no host synchronisation and no CPU arithmetic of the method
// happens inside al_sample_drag_spread.
#include "al.h"
#include "al_kernels.cuh"

#include <cudaTypedefs.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <utility>
#include <vector>

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char *what) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? AL_ERR_OOM : AL_ERR_CUDA;
}

#define AL_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// One device allocation carved into an instance's arrays, 256-byte aligned:
// the same sequence of take() calls first sizes it (base == nullptr), then
// hands out the pointers.  A few allocations per instance instead of one per
// array: admission is cheaper and the memory it holds is exactly the slabs.
struct Slab {
    size_t off = 0;
    char *base = nullptr;
    void *take_bytes(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? base + off : nullptr;
        off += bytes ? bytes : 1;
        return p;
    }
    template <typename P> void take(P **p, size_t n) { *p = static_cast<P *>(take_bytes((n ? n : 1) * sizeof(P))); }
};
// device bytes the driver commits for an allocation: whole 2 MiB pages
static size_t page_round(size_t bytes) { return bytes ? (bytes + (2u << 20) - 1) & ~(size_t)((2u << 20) - 1) : 0; }

// brick decomposition of the projection for brick height bz
void set_brick_z(al::GridC &c, int bz) {
    c.bz = bz;
    c.nbz = (c.nz + bz - 1) / bz;
    c.nbrick = (long long)c.nbx * c.nby * c.nbz;
}

void split_ff(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

}  // namespace

struct al_grid_s {
    al_grid_desc d{};
    int device = 0;
    al::GridC gc{};
    size_t esize = 4;                 // bytes per field element
    long long nbrick_max = 0;         // bricks at the lowest brick height (sizes the masks)

    // lines
    bool loaded = false;
    int n_lines = 0, n_points = 0, mask_words = 0;
    int *d_line_off = nullptr, *d_line_of = nullptr;
    double *d_d = nullptr, *d_cdn = nullptr, *d_cdt = nullptr, *d_eps = nullptr, *d_ell = nullptr,
           *d_af = nullptr, *d_cvl = nullptr, *d_cmn = nullptr, *d_cmt = nullptr, *d_EI = nullptr;
    std::vector<double> h_EI;         // the stiffnesses last copied to d_EI
    al_beam_desc bd{};                // scalars of the loaded descriptor (its array pointers are not kept)
    std::vector<int> h_line_off;      // host copies of the line table that size the record arena
    std::vector<double> h_eps, h_cv_len;

    // per-point scratch (element type per precision)
    void *fprev = nullptr, *uhi = nullptr, *segD = nullptr, *segIl2 = nullptr, *nodeM = nullptr,
         *fhat = nullptr;
    float *ulo = nullptr, *nodeTau = nullptr;
    double *segWa = nullptr, *segWb = nullptr, *w = nullptr, *lineF = nullptr;
    unsigned long long *wfix = nullptr;
    al::LineG *lines = nullptr;
    uint32_t *mask = nullptr;

    // per-grid scratch
    double *brickSum = nullptr;
    double *scatSum = nullptr;
    double *totPart = nullptr;        // [TOT_PARTS][6] partial totals
    int *totDone = nullptr;           // parts of the totals done in a step
    int *statusInt = nullptr;
    double *totalsInt = nullptr;
    int *hasPrev = nullptr;           // device flag: f_prev is valid
    int *anyIrr = nullptr;            // device flag: some line without a walk certificate
    unsigned int *smax = nullptr;     // device: bound on one spread contribution (float bits)
    int *anyZero = nullptr;           // device flag: some node with w_k = 0
    int *rcnt = nullptr, *rcap = nullptr;   // per brick: records found / region capacity
    long long *roff = nullptr;        // per brick: region start
    int *rplan = nullptr;             // [2] brick height of this / the next step's regions
    int *cmcnt = nullptr;             // [5] bricks of a step on the column-march (with candidate lines) /
                                      // the brick passes; the next column-march brick of the spread / entry
                                      // of the weights pass; column-march bricks without candidate lines
    int *cmlist = nullptr;            // [2][nbrick_max] those bricks
    int opt_column = 1;               // AL_OPT_COLUMN
    int own_x0 = 0, own_x1 = -1;      // AL_OPT_OWN_X0 / X1: owned cells along x (-1: to the end)
    long long launches = 0;           // kernels launched by this instance's steps (al_launches)
    cudaEvent_t host_ev = nullptr;    // end of the last al_step_host step (orders steps across streams)
    bool host_ev_set = false;
    // column march (FP32, nearest-segment projection, no reflection): node
    // records, entries of the column-march bricks
    float4 *cmN = nullptr;            // [np][4] node records
    al::CmLay *cmlay = nullptr;       // [n_lines][(nz + 3) / 4] per line and brick layer
    al::CmEnt *cment = nullptr;
    int *cment_n = nullptr, *bent_off = nullptr, *bent_n = nullptr;
    long long cment_cap = 0;
    unsigned long long *rused = nullptr;    // arena taken by the next step's regions
    void *rec = nullptr;              // record arena (rec_total records), allocated only while records are used
    long long rec_total = 0;
    int opt_record = 1;

    // device bytes this instance holds (al_footprint): per-grid scratch,
    // per-point scratch of the loaded lines, record arena
    size_t grid_bytes = 0, beam_bytes = 0, rec_bytes = 0;
    void *grid_slab = nullptr, *beam_slab = nullptr;   // the allocations the per-grid / per-line arrays live in

    // tracing
    bool trace = false;
    cudaEvent_t ev[AL_TRACE_N + 1] = {};
};

static void trace_mark(al_grid g, int i, cudaStream_t st) {
    if (g->trace) cudaEventRecord(g->ev[i], st);
}

static void free_beams(al_grid g) {
    if (g->beam_slab) cudaFree(g->beam_slab);
    if (g->rec) cudaFree(g->rec);
    g->beam_slab = nullptr;
    g->d_line_off = g->d_line_of = nullptr;
    g->d_d = g->d_cdn = g->d_cdt = g->d_eps = g->d_ell = g->d_af = g->d_cvl = g->d_cmn = g->d_cmt = nullptr;
    g->d_EI = nullptr;
    g->h_EI.clear();
    g->fprev = g->uhi = g->segD = g->segIl2 = g->nodeM = g->fhat = nullptr;
    g->ulo = g->nodeTau = nullptr;
    g->segWa = g->segWb = g->w = g->lineF = nullptr;
    g->wfix = nullptr;
    g->lines = nullptr;
    g->mask = nullptr;
    g->rec = nullptr;
    g->rec_total = 0;
    g->cmN = nullptr;
    g->cmlay = nullptr;
    g->cment = nullptr;
    g->cment_n = g->bent_off = g->bent_n = nullptr;
    g->cment_cap = 0;
    g->beam_bytes = g->rec_bytes = 0;
    g->loaded = false;
    g->n_lines = g->n_points = g->mask_words = 0;
}

extern "C" const char *al_error_string(int code) {
    switch (code) {
    case AL_OK: return "ok";
    case AL_ERR_ARG: return "invalid argument";
    case AL_ERR_CUDA: return "CUDA runtime error";
    case AL_ERR_OOM: return "out of device memory";
    case AL_ERR_STATE: return "call out of order";
    case AL_ERR_TIMEOUT: return "bounded wait expired";
    case AL_ERR_CAPACITY: return "request exceeds a fixed capacity";
    default: return "unknown status";
    }
}

extern "C" const char *al_last_cuda_error(void) { return g_cuda_err; }

extern "C" int al_create_grid(const al_grid_desc *desc, al_grid *out) {
    if (!desc || !out) return AL_ERR_ARG;
    *out = nullptr;
    const al_grid_desc &d = *desc;
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return AL_ERR_ARG;
    if (!(d.dx > 0.0) || !std::isfinite(d.dx)) return AL_ERR_ARG;
    if (d.precision != AL_FP32 && d.precision != AL_FP64) return AL_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(d.origin[a])) return AL_ERR_ARG;
    if (d.has_alpha && (!(d.rho1 > 0.0) || !(d.rho2 > 0.0))) return AL_ERR_ARG;
    if (!d.has_alpha && !(d.rho_const > 0.0)) return AL_ERR_ARG;
    const long long ncell = (long long)d.nx * d.ny * d.nz;
    if (ncell > (1LL << 40)) return AL_ERR_ARG;

    al_grid g = new (std::nothrow) al_grid_s();
    if (!g) return AL_ERR_OOM;
    g->d = d;
    cudaGetDevice(&g->device);
    g->esize = d.precision == AL_FP64 ? 8 : 4;
    al::GridC &c = g->gc;
    c.nx = d.nx; c.ny = d.ny; c.nz = d.nz;
    c.ncell = ncell;
    c.nbx = (d.nx + al::BX - 1) / al::BX;
    c.nby = (d.ny + al::BY - 1) / al::BY;
    set_brick_z(c, al::BZ_MIN);
    g->nbrick_max = c.nbrick;
    set_brick_z(c, 8);
    c.h = d.dx;
    c.V = d.dx * d.dx * d.dx;
    for (int a = 0; a < 3; ++a) {
        c.o[a] = d.origin[a];
        split_ff(d.origin[a], c.o_hi[a], c.o_lo[a]);
    }
    split_ff(1.0 / d.dx, c.ih_hi, c.ih_lo);
    c.has_alpha = d.has_alpha ? 1 : 0;
    c.rho1 = d.rho1; c.rho2 = d.rho2; c.rho_const = d.rho_const;

    auto carve = [&](Slab &sl) {
        sl.take(&g->brickSum, 3 * (size_t)g->nbrick_max);
        sl.take(&g->scatSum, 3);
        sl.take(&g->totPart, 6 * (size_t)al::TOT_PARTS);
        sl.take(&g->totDone, 1);
        sl.take(&g->statusInt, AL_STATUS_N); sl.take(&g->totalsInt, 6);
        sl.take(&g->hasPrev, 1); sl.take(&g->anyIrr, 1); sl.take(&g->smax, 1); sl.take(&g->anyZero, 1);
        sl.take(&g->rcnt, (size_t)g->nbrick_max); sl.take(&g->rcap, (size_t)g->nbrick_max);
        sl.take(&g->roff, (size_t)g->nbrick_max);
        sl.take(&g->rplan, 2); sl.take(&g->rused, 1);
        sl.take(&g->cmcnt, 5); sl.take(&g->cmlist, 2 * (size_t)g->nbrick_max);
    };
    Slab size;
    carve(size);
    Slab sl;
    const cudaError_t e = cudaMalloc((void **)&sl.base, size.off);
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "cudaMalloc");
        al_destroy(g);
        return rc;
    }
    carve(sl);
    g->grid_slab = sl.base;
    g->grid_bytes = size.off;
    *out = g;
    return AL_OK;
}

// The record arena of the replayed gather is held only while an instance
// can use it: segment weights with records on (AL_OPT_WEIGHTS = SEGMENT,
// AL_OPT_RECORD = 1), or the integrated projection with records on; never
// with a reflected kernel.  Sized from the lines: the cells within
// R_c = 3 eps / h of a line of length L_c (cells) number about
// pi R_c^2 L_c + 4/3 pi R_c^3 plus half the surface; a quarter more, and
// 4096.  A failed allocation leaves no arena (every brick is then gathered).
static bool arena_wanted(al_grid g) {
    if (!g->loaded || g->n_lines == 0 || g->bd.wall_reflect || g->opt_record != 1) return false;
    return g->bd.proj_mode == AL_PROJ_INTEGRATED || g->gc.wmode == AL_WEIGHTS_SEGMENT;
}
static int arena_sync(al_grid g) {
    const bool want_arena = arena_wanted(g);
    if (want_arena == (g->rec != nullptr)) return AL_OK;
    AL_CUDA(cudaDeviceSynchronize());                  // no step may still use the regions
    if (!want_arena) {
        cudaFree(g->rec);
        g->rec = nullptr;
        g->rec_total = 0;
        g->rec_bytes = 0;
    } else {
        const al_beam_desc &b = g->bd;
        double est = 0.0;
        for (int l = 0; l < b.n_lines; ++l) {
            double L = 0.0;
            for (int i = g->h_line_off[l]; i < g->h_line_off[l + 1]; ++i) L += g->h_cv_len[i];
            const double Rc = 3.0 * g->h_eps[l] / g->d.dx, Lc = L / g->d.dx, pi = 3.14159265358979323846;
            double pairs = pi * Rc * Rc * Lc + 4.0 / 3.0 * pi * Rc * Rc * Rc + pi * Rc * Lc + 2.0 * pi * Rc * Rc + 64.0;
            const int nl_pts = g->h_line_off[l + 1] - g->h_line_off[l];
            if (b.proj_mode == AL_PROJ_INTEGRATED && nl_pts >= 2)   // a cell pairs with every segment within 3 eps
                pairs *= 2.0 * Rc / std::max(Lc / (nl_pts - 1), 0.25) + 2.0;
            est += pairs;
        }
        const size_t rsz = g->d.precision == AL_FP64 ? sizeof(al::Rec<double>) : sizeof(al::Rec<float>);
        long long want = (long long)(1.25 * est) + 4096;
        want = std::min<long long>(want, (8ll << 30) / (long long)rsz);       // at most 8 GiB
        if (cudaMalloc(&g->rec, (size_t)want * rsz) == cudaSuccess) {
            g->rec_total = want;
            g->rec_bytes = (size_t)want * rsz;
        } else {
            (void)cudaGetLastError();
            g->rec = nullptr;
            g->rec_total = 0;
        }
    }
    // regions planned in another arena are void: the next step gathers
    AL_CUDA(cudaMemset(g->rcap, 0, (size_t)g->nbrick_max * sizeof(int)));
    AL_CUDA(cudaMemset(g->rplan, 0, 2 * sizeof(int)));
    return AL_OK;
}

// Host-side checks of a beam descriptor against a grid (the rules of
// al_load_beams, shared with al_line_forces_noalloc).  *np_out receives the
// number of actuator points.
int al_detail_check_beams(const al_beam_desc &b, const al_grid_desc &gd, int *np_out) {
    *np_out = 0;
    if (b.n_lines < 0) return AL_ERR_ARG;
    if (b.n_lines > 0 && (!b.line_off || !b.d || !b.cdn || !b.cdt || !b.eps || !b.ell_s || !b.alpha_f))
        return AL_ERR_ARG;
    if ((b.cm_n == nullptr) != (b.cm_t == nullptr)) return AL_ERR_ARG;      // both or neither
    if (b.sample_mode != AL_SAMPLE_TRILINEAR && b.sample_mode != AL_SAMPLE_CELL && b.sample_mode != AL_SAMPLE_GAUSS)
        return AL_ERR_ARG;
    if (b.drag_mode != AL_DRAG_DISCRETE && b.drag_mode != AL_DRAG_SPLIT) return AL_ERR_ARG;
    if (b.proj_mode != AL_PROJ_NEAREST && b.proj_mode != AL_PROJ_INTEGRATED) return AL_ERR_ARG;
    if (b.wall_reflect < 0 || b.wall_reflect > 63) return AL_ERR_ARG;
    if (b.wall_reflect && b.proj_mode != AL_PROJ_NEAREST) return AL_ERR_ARG;
    if (!(b.tau >= 0.0)) return AL_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(b.n_p[a]) || !std::isfinite(b.g_up[a])) return AL_ERR_ARG;
    const double npn = std::sqrt(b.n_p[0] * b.n_p[0] + b.n_p[1] * b.n_p[1] + b.n_p[2] * b.n_p[2]);
    if (!(npn == 0.0 || std::fabs(npn - 1.0) < 1e-9)) return AL_ERR_ARG;
    int np = 0;
    if (b.n_lines > 0) {
        if (b.line_off[0] != 0) return AL_ERR_ARG;
        for (int l = 0; l < b.n_lines; ++l) {
            if (b.line_off[l + 1] < b.line_off[l]) return AL_ERR_ARG;
            if (!(b.eps[l] > 0.0) || !(b.ell_s[l] >= 0.0) || !(b.alpha_f[l] > 0.0 && b.alpha_f[l] <= 1.0) ||
                !(b.d[l] >= 0.0) || !std::isfinite(b.cdn[l]) || !std::isfinite(b.cdt[l]) ||
                !std::isfinite(b.d[l]) || !std::isfinite(b.ell_s[l]) || !std::isfinite(b.eps[l]))
                return AL_ERR_ARG;
            // the kernel support 3 eps must span fewer than 2^20 cells
            if (3.0 * b.eps[l] / gd.dx > 1048576.0) return AL_ERR_ARG;
            if (b.cm_n && (!std::isfinite(b.cm_n[l]) || !std::isfinite(b.cm_t[l]))) return AL_ERR_ARG;
        }
        np = b.line_off[b.n_lines];
        if (np > 0 && !b.cv_len) return AL_ERR_ARG;
        if (b.wall_reflect) {                            // one reflection per face: ghosts <= n deep
            double emax = 0.0;
            for (int l = 0; l < b.n_lines; ++l) emax = std::max(emax, b.eps[l]);
            const double gdep = std::ceil(3.0 * emax / gd.dx) + 1.0;
            const int nn[3] = {gd.nx, gd.ny, gd.nz};
            for (int a = 0; a < 3; ++a)
                if (((b.wall_reflect >> (2 * a)) & 3) && gdep > (double)nn[a]) return AL_ERR_ARG;
        }
        for (int i = 0; i < np; ++i)
            if (!(b.cv_len[i] >= 0.0) || !std::isfinite(b.cv_len[i])) return AL_ERR_ARG;
    }
    *np_out = np;
    return AL_OK;
}

// CUDA failure recorded in the text al_last_cuda_error returns (shared with
// al_line_forces_noalloc)
int al_detail_cuda_fail(cudaError_t e, const char *what) { return cuda_fail(e, what); }

extern "C" int al_load_beams(al_grid g, const al_beam_desc *bp) {
    if (!g || !bp) return AL_ERR_ARG;
    const al_beam_desc &b = *bp;
    int np = 0;
    {
        const int rc = al_detail_check_beams(b, g->d, &np);
        if (rc != AL_OK) return rc;
    }
    AL_CUDA(cudaDeviceSynchronize());
    free_beams(g);
    g->n_lines = b.n_lines;
    g->n_points = np;
    g->mask_words = (b.n_lines + 31) / 32;
    g->bd = b;
    const size_t es = g->esize, n3 = 3 * (size_t)np;
    const size_t nl = (size_t)b.n_lines;
    g->cment_cap = 0;
    auto carve = [&](Slab &sl) {
        auto A = [&](auto **p, size_t n) { sl.take(p, n); };
        auto AB = [&](void **p, size_t n) { *p = sl.take_bytes((n ? n : 1) * es); };
        A(&g->d_line_off, nl + 1);
        A(&g->d_line_of, (size_t)np);
        A(&g->d_d, nl); A(&g->d_cdn, nl); A(&g->d_cdt, nl); A(&g->d_eps, nl); A(&g->d_ell, nl); A(&g->d_af, nl);
        A(&g->d_cvl, (size_t)np);
        if (b.cm_n) { A(&g->d_cmn, nl); A(&g->d_cmt, nl); }
        A(&g->d_EI, nl);
        AB(&g->fprev, n3); AB(&g->uhi, n3); AB(&g->segD, n3); AB(&g->segIl2, (size_t)np); AB(&g->nodeM, n3);
        AB(&g->fhat, n3);
        A(&g->ulo, n3); A(&g->nodeTau, (size_t)np);
        A(&g->segWa, (size_t)np); A(&g->segWb, (size_t)np);
        A(&g->wfix, (size_t)np); A(&g->w, (size_t)np); A(&g->lineF, 3 * nl);
        A(&g->lines, nl);
        A(&g->mask, (size_t)g->nbrick_max * g->mask_words);
        if (g->d.precision == AL_FP32 && b.proj_mode == AL_PROJ_NEAREST && !b.wall_reflect && np > 0) {
            // the column march: four float4 records per node, and an entry pool of
            // 16 entries per brick at the lowest brick height (bricks beyond it in
            // a step take the brick passes)
            A(&g->cmN, 4 * (size_t)np);
            A(&g->cmlay, nl * (size_t)((g->d.nz + 3) / 4));
            g->cment_cap = 16 * g->nbrick_max;
            A(&g->cment, (size_t)g->cment_cap);
            A(&g->cment_n, 1);
            A(&g->bent_off, (size_t)g->nbrick_max);
            A(&g->bent_n, (size_t)g->nbrick_max);
        }
    };
    Slab size;
    carve(size);
    Slab sl;
    const cudaError_t e = cudaMalloc((void **)&sl.base, size.off);
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "cudaMalloc");
        free_beams(g);
        return rc;
    }
    carve(sl);
    g->beam_slab = sl.base;
    g->beam_bytes = size.off;
    std::vector<int> off(nl + 1, 0), of((size_t)np);
    if (b.n_lines > 0) {
        for (size_t l = 0; l <= nl; ++l) off[l] = b.line_off[l];
        for (size_t l = 0; l < nl; ++l)
            for (int i = off[l]; i < off[l + 1]; ++i) of[i] = (int)l;
    }
    g->h_line_off = off;
    g->h_eps.assign(b.eps, b.eps + nl);
    g->h_cv_len.assign(b.cv_len, b.cv_len + np);
    AL_CUDA(cudaMemcpy(g->d_line_off, off.data(), (nl + 1) * sizeof(int), cudaMemcpyHostToDevice));
    if (np) {
        AL_CUDA(cudaMemcpy(g->d_line_of, of.data(), np * sizeof(int), cudaMemcpyHostToDevice));
        AL_CUDA(cudaMemcpy(g->d_cvl, b.cv_len, np * sizeof(double), cudaMemcpyHostToDevice));
        AL_CUDA(cudaMemset(g->fprev, 0, n3 * es));
        AL_CUDA(cudaMemset(g->ulo, 0, n3 * sizeof(float)));
    }
    if (nl) {
        AL_CUDA(cudaMemcpy(g->d_d, b.d, nl * sizeof(double), cudaMemcpyHostToDevice));
        AL_CUDA(cudaMemcpy(g->d_cdn, b.cdn, nl * sizeof(double), cudaMemcpyHostToDevice));
        AL_CUDA(cudaMemcpy(g->d_cdt, b.cdt, nl * sizeof(double), cudaMemcpyHostToDevice));
        AL_CUDA(cudaMemcpy(g->d_eps, b.eps, nl * sizeof(double), cudaMemcpyHostToDevice));
        AL_CUDA(cudaMemcpy(g->d_ell, b.ell_s, nl * sizeof(double), cudaMemcpyHostToDevice));
        AL_CUDA(cudaMemcpy(g->d_af, b.alpha_f, nl * sizeof(double), cudaMemcpyHostToDevice));
        if (b.cm_n) {
            AL_CUDA(cudaMemcpy(g->d_cmn, b.cm_n, nl * sizeof(double), cudaMemcpyHostToDevice));
            AL_CUDA(cudaMemcpy(g->d_cmt, b.cm_t, nl * sizeof(double), cudaMemcpyHostToDevice));
        }
    }
    AL_CUDA(cudaMemset(g->mask, 0, ((size_t)g->nbrick_max * g->mask_words ? (size_t)g->nbrick_max * g->mask_words : 1) * sizeof(uint32_t)));
    AL_CUDA(cudaMemset(g->hasPrev, 0, sizeof(int)));
    AL_CUDA(cudaMemset(g->totDone, 0, sizeof(int)));
    AL_CUDA(cudaMemset(g->anyIrr, 0, sizeof(int)));
    AL_CUDA(cudaMemset(g->smax, 0, sizeof(unsigned int)));
    AL_CUDA(cudaMemset(g->anyZero, 0, sizeof(int)));
    AL_CUDA(cudaMemset(g->rcnt, 0, (size_t)g->nbrick_max * sizeof(int)));
    AL_CUDA(cudaMemset(g->rcap, 0, (size_t)g->nbrick_max * sizeof(int)));
    AL_CUDA(cudaMemset(g->roff, 0, (size_t)g->nbrick_max * sizeof(long long)));
    AL_CUDA(cudaMemset(g->rplan, 0, 2 * sizeof(int)));
    AL_CUDA(cudaMemset(g->rused, 0, sizeof(unsigned long long)));
    g->loaded = true;
    return arena_sync(g);
}

// The projection kernels use more than 48 KB of dynamic shared memory, and
// prefer shared memory over L1 so that several bricks share an SM.
template <typename T, int BZ>
static cudaError_t brick_attrs() {
    const int fx = (int)sizeof(al::SpreadSmem<T, BZ, true>), fl = (int)sizeof(al::SpreadSmem<T, BZ, false>);
    const void *fns[9] = {(const void *)al::k_spread<T, BZ, true>, (const void *)al::k_spread<T, BZ, false>,
                          (const void *)al::kb_spread<T, BZ>, (const void *)al::k_bweights<T, BZ>,
                          (const void *)al::kb_bweights<T, BZ>, (const void *)al::k_spread_refl<T, BZ>,
                          (const void *)al::k_bweights_refl<T, BZ>, (const void *)al::kb_spread_refl<T, BZ>,
                          (const void *)al::kb_bweights_refl<T, BZ>};
    const int bytes_of[9] = {fx, fl, fx, fl, fl, fl, fl, fl, fl};
    for (int i = 0; i < 9; ++i) {
        const void *f = fns[i];
        const int bytes = bytes_of[i];
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
// the column-march kernels and the list-driven brick passes (FP32 only)
template <int BZ>
static cudaError_t cm_attrs() {
    const void *fns[5] = {(const void *)al::k_cm_weights<float>, (const void *)al::k_cm_spread<BZ>,
                          (const void *)al::k_spread_ls<BZ, true>, (const void *)al::k_spread_ls<BZ, false>,
                          (const void *)al::k_bweights_ls<BZ>};
    const int bytes_of[5] = {(int)(sizeof(al::CmWeightSmem)), (int)sizeof(al::CmSpreadSmem<BZ>),
                             (int)sizeof(al::SpreadSmem<float, BZ, true>), (int)sizeof(al::SpreadSmem<float, BZ, false>),
                             (int)sizeof(al::SpreadSmem<float, BZ, false>)};
    for (int i = 0; i < 5; ++i) {
        cudaError_t e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes_of[i]);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fns[i], cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
// persistent grids of the column-march and list-driven kernels: SMs x
// resident CTAs, per kernel (queried once per process, device and height)
struct CmGrids { int cw, cs, sl_fx, sl, bw; };
template <int BZ>
static cudaError_t cm_grids(CmGrids &gr) {
    static int dev_done = -1;
    static CmGrids cache{};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev_done == dev) { gr = cache; return cudaSuccess; }
    e = cm_attrs<BZ>();
    if (e != cudaSuccess) return e;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int o[5] = {0, 0, 0, 0, 0};
    using namespace al;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[0], k_cm_weights<float>, CM_WTHREADS, sizeof(CmWeightSmem));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[1], k_cm_spread<BZ>, CM_STHREADS, sizeof(CmSpreadSmem<BZ>));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[2], k_spread_ls<BZ, true>, SPREAD_THREADS, sizeof(SpreadSmem<float, BZ, true>));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[3], k_spread_ls<BZ, false>, SPREAD_THREADS, sizeof(SpreadSmem<float, BZ, false>));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[4], k_bweights_ls<BZ>, SPREAD_THREADS, sizeof(SpreadSmem<float, BZ, false>));
    if (e != cudaSuccess) return e;
    for (int i = 0; i < 5; ++i) o[i] = nsm * std::max(o[i], 1);
    cache = CmGrids{o[0], o[1], o[2], o[3], o[4]};
    dev_done = dev;
    gr = cache;
    return cudaSuccess;
}

template <typename T>
static cudaError_t spread_smem_attr() {
    static cudaError_t done = cudaErrorNotReady;
    if (done != cudaSuccess) {
        done = brick_attrs<T, 4>();
        if (done == cudaSuccess) done = brick_attrs<T, 8>();
        if (done == cudaSuccess) done = brick_attrs<T, 16>();
    }
    return done;
}

// A kernel of the step after its first, launched with programmatic
// dependent launch: it is set up while the previous kernel of the stream
// runs and starts as that one ends (about 1 us between two kernels instead
// of about 3 on a B300).  Every kernel launched so begins with pdl_enter(),
// which waits for that kernel to complete and its writes to be visible
// (errors are seen by cudaGetLastError, as for a plain launch).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                              Args &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// the two brick passes of one instance at brick height BZ
template <typename T, int BZ>
static void launch_bricks(const al::Inst<T> &I, bool weights, cudaStream_t st) {
    using namespace al;
    if (weights && I.b.reflect)
        launch_pdl(k_bweights_refl<T, BZ>, (unsigned)I.g.nbrick, SPREAD_THREADS, sizeof(SpreadSmem<T, BZ, false>), st,
            I.g, I.b, I.sc, I.p, I.status);
    else if (weights)
        launch_pdl(k_bweights<T, BZ>, (unsigned)I.g.nbrick, SPREAD_THREADS, sizeof(SpreadSmem<T, BZ, false>), st,
            I.g, I.b, I.sc, I.p, I.status);
    else if (I.b.reflect)
        launch_pdl(k_spread_refl<T, BZ>, (unsigned)I.g.nbrick, SPREAD_THREADS, sizeof(SpreadSmem<T, BZ, false>), st,
            I.g, I.b, I.sc, I.p, I.status);
    else if (I.g.fx)
        launch_pdl(k_spread<T, BZ, true>, (unsigned)I.g.nbrick, SPREAD_THREADS, sizeof(SpreadSmem<T, BZ, true>), st,
            I.g, I.b, I.sc, I.p, I.status);
    else
        launch_pdl(k_spread<T, BZ, false>, (unsigned)I.g.nbrick, SPREAD_THREADS, sizeof(SpreadSmem<T, BZ, false>), st,
            I.g, I.b, I.sc, I.p, I.status);
}
template <typename T>
static void launch_bricks_bz(const al::Inst<T> &I, bool weights, cudaStream_t st) {
    switch (I.g.bz) {
    case 4: launch_bricks<T, 4>(I, weights, st); break;
    case 16: launch_bricks<T, 16>(I, weights, st); break;
    default: launch_bricks<T, 8>(I, weights, st); break;
    }
}

// the descriptors of S for the spread's tile stores: a 3-D tensor per
// component (x fastest), boxes of a brick; off when the driver's encoder is
// missing or refuses (S not 16-byte aligned, rows not a multiple of 16 bytes)
template <int BZ>
static al::CmStore cm_store(const al::Inst<float> &I) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        else
            (void)cudaGetLastError();
    }
    al::CmStore tm;
    memset(&tm, 0, sizeof(tm));
    const int nx = I.g.nx, ny = I.g.ny, nz = I.g.nz;
    bool ok = enc != nullptr && (nx % 4) == 0;
    for (int a = 0; a < 3 && ok; ++a) ok = (reinterpret_cast<uintptr_t>(I.p.S[a]) & 15) == 0;
    if (ok) {
        const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
        const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
        const cuuint32_t box[3] = {(cuuint32_t)al::BX, (cuuint32_t)al::BY, (cuuint32_t)BZ};
        const cuuint32_t es[3] = {1, 1, 1};
        for (int a = 0; a < 3 && ok; ++a)
            ok = enc(&tm.m[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)I.p.S[a], dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    tm.on = ok ? 1 : 0;
    return tm;
}

// the projection of one FP32 instance with the column march: bricks whose
// lines all take it run the column-march passes, the others the brick
// passes, each brick with one of the two for both its weights and its spread
template <int BZ>
static int cm_launch(const al::Inst<float> &I, bool weights, long long nbrick, cudaStream_t st) {
    using namespace al;
    CmGrids gr;
    AL_CUDA(cm_grids<BZ>(gr));
    auto cap = [&](int gsz) { return (unsigned)std::max(1LL, std::min((long long)gsz, nbrick)); };
    if (weights) {
        // one warp per entry of the bricks of list 0, then the brick passes over list 1
        launch_pdl(k_cm_weights<float>, (unsigned)gr.cw, CM_WTHREADS, sizeof(CmWeightSmem), st, I.g, I.b, I.sc, I.p, I.status);
        launch_pdl(k_bweights_ls<BZ>, cap(gr.bw), SPREAD_THREADS, sizeof(SpreadSmem<float, BZ, false>), st, I.g, I.b, I.sc, I.p, I.status);
    } else {
        const CmStore tm = cm_store<BZ>(I);
        launch_pdl(k_cm_spread<BZ>, cap(gr.cs), CM_STHREADS, sizeof(CmSpreadSmem<BZ>), st, I.g, I.b, I.sc, I.p, I.status, tm);
        if (I.g.fx)
            launch_pdl(k_spread_ls<BZ, true>, cap(gr.sl_fx), SPREAD_THREADS, sizeof(SpreadSmem<float, BZ, true>), st, I.g, I.b, I.sc, I.p, I.status);
        else
            launch_pdl(k_spread_ls<BZ, false>, cap(gr.sl), SPREAD_THREADS, sizeof(SpreadSmem<float, BZ, false>), st, I.g, I.b, I.sc, I.p, I.status);
    }
    return AL_OK;
}
static int cm_launch_bz(const al::Inst<float> &I, bool weights, cudaStream_t st) {
    switch (I.g.bz) {
    case 4: return cm_launch<4>(I, weights, I.g.nbrick, st);
    case 16: return cm_launch<16>(I, weights, I.g.nbrick, st);
    default: return cm_launch<8>(I, weights, I.g.nbrick, st);
    }
}

// the instance owns only part of its grid's cells along x
static bool owns_part(const al_grid_s *g) { return g->own_x0 > 0 || (g->own_x1 >= 0 && g->own_x1 < g->d.nx); }

template <typename T>
static al::Inst<T> make_inst(al_grid g, const al_step_in *in, const al_step_out *out) {
    using namespace al;
    const int np = g->n_points;
    Inst<T> I{};
    StepPtrs<T> &p = I.p;
    for (int a = 0; a < 3; ++a) {
        p.U[a] = (const T *)in->U[a];
        p.P[a] = (const T *)in->P[a];
        p.Pdot[a] = (const T *)in->Pdot[a];
        p.Ps[a] = (const T *)(in->P_spread[a] ? in->P_spread[a] : in->P[a]);
        p.tan[a] = (const T *)in->tangent[a];
        p.S[a] = (T *)out->S[a];
        p.F[a] = (T *)out->F[a];
    }
    p.alpha = (const T *)in->alpha;
    p.np = np;
    const bool inert = g->d_cmn != nullptr;
    for (int a = 0; a < 3; ++a) {
        p.Uprev[a] = inert ? (const T *)in->U_prev[a] : nullptr;
        p.Pdd[a] = inert ? (const T *)in->Pddot[a] : nullptr;
    }
    p.dt = in->dt;
    Scratch<T> &sc = I.sc;
    sc.fprev = (T *)g->fprev; sc.uhi = (T *)g->uhi; sc.ulo = g->ulo; sc.segD = (T *)g->segD;
    sc.segIl2 = (T *)g->segIl2; sc.nodeM = (T *)g->nodeM; sc.nodeTau = g->nodeTau;
    sc.segWa = g->segWa; sc.segWb = g->segWb; sc.wfix = g->wfix; sc.w = g->w; sc.fhat = (T *)g->fhat; sc.lineF = g->lineF;
    sc.lines = g->lines; sc.mask = g->mask; sc.brickSum = g->brickSum; sc.scatSum = g->scatSum;
    sc.totPart = g->totPart;
    sc.totDone = g->totDone;
    sc.hasPrev = g->hasPrev; sc.anyIrr = g->anyIrr; sc.smax = g->smax; sc.anyZero = g->anyZero;
    sc.rec = (Rec<T> *)g->rec; sc.rcnt = g->rcnt; sc.rcap = g->rcap; sc.roff = g->roff;
    sc.rplan = g->rplan; sc.rused = g->rused;
    sc.cmcnt = g->cmcnt; sc.cmlist = g->cmlist;
    BeamsC &bc = I.b;
    bc.n_lines = g->n_lines; bc.n_points = np; bc.mask_words = g->mask_words;
    bc.line_off = g->d_line_off; bc.line_of = g->d_line_of;
    bc.d = g->d_d; bc.cdn = g->d_cdn; bc.cdt = g->d_cdt; bc.eps = g->d_eps; bc.ell_s = g->d_ell;
    bc.alpha_f = g->d_af; bc.cv_len = g->d_cvl;
    for (int a = 0; a < 3; ++a) { bc.n_p[a] = g->bd.n_p[a]; bc.g_up[a] = g->bd.g_up[a]; }
    bc.tau = g->bd.tau; bc.sample_mode = g->bd.sample_mode; bc.drag_mode = g->bd.drag_mode;
    bc.tangents_given = g->bd.tangents_given;
    bc.cm_n = g->d_cmn; bc.cm_t = g->d_cmt;
    bc.proj_mode = g->bd.proj_mode;
    bc.reflect = g->bd.wall_reflect;
    bc.inertia = (g->d_cmn != nullptr && g->n_lines > 0) ? 1 : 0;
    I.g = g->gc;
    I.g.rec_total = g->rec_total;
    I.g.nbrick_max = g->nbrick_max;
    if (g->bd.proj_mode == AL_PROJ_INTEGRATED) {        // segment pass and gather for every line
        I.g.wmode = AL_WEIGHTS_SEGMENT;
        I.g.smode = AL_SPREAD_GATHER;
    }
    if (g->bd.wall_reflect) {                           // ghost cells: the brick passes for every line
        I.g.wmode = AL_WEIGHTS_BRICK;
        I.g.smode = AL_SPREAD_GATHER;
    }
    I.g.rmode = (g->opt_record == 1 && I.g.wmode != 0 && I.g.smode == 0 && g->rec_total > 0) ? 1 : 0;
    // the column-march passes: FP32, the paper's nearest-segment projection,
    // no reflecting face, the gather
    I.g.cm = (g->opt_column && g->cmN && I.g.smode == AL_SPREAD_GATHER) ? 1 : 0;
    sc.cmN = I.g.cm ? g->cmN : nullptr;
    sc.cmlay = I.g.cm ? g->cmlay : nullptr;
    sc.cment = g->cment; sc.cment_n = I.g.cm ? g->cment_n : nullptr; sc.cment_cap = g->cment_cap;
    sc.bent_off = g->bent_off; sc.bent_n = g->bent_n;
    I.g.fx = (I.g.rmode || g->opt_record == 2 || g->bd.proj_mode == AL_PROJ_INTEGRATED) ? 1 : 0;
    if (g->bd.wall_reflect) I.g.fx = 0;                 // the reflected passes gather in line order
    // a slab of a decomposition along x: the brick passes (or the column
    // march) on the owned brick columns, weights as fixed-point partial sums
    I.g.own_bx0 = g->own_x0 / al::BX;
    I.g.own_bx1 = g->own_x1 < 0 ? I.g.nbx : (g->own_x1 + al::BX - 1) / al::BX;
    if (owns_part(g)) {
        I.g.wmode = AL_WEIGHTS_BRICK;
        I.g.smode = AL_SPREAD_GATHER;
        I.g.rmode = 0;
        I.g.fx = 0;
    }
    I.status = out->status ? out->status : g->statusInt;
    I.totals = out->totals ? out->totals : g->totalsInt;
    return I;
}

// phases: 1 = points, line geometry, bins and weights (up to the weights'
// partial sums); 2 = normalisation, spread and totals; 3 = the whole step
template <typename T>
static int step_impl(al_grid g, const al_step_in *in, const al_step_out *out, cudaStream_t st, int phases = 3) {
    using namespace al;
    const al::Inst<T> I = make_inst<T>(g, in, out);
    const GridC &gc = I.g;
    const BeamsC &bc = I.b;
    const Scratch<T> &sc = I.sc;
    const StepPtrs<T> &p = I.p;
    int *status = I.status;
    const int np = g->n_points;

    AL_CUDA(spread_smem_attr<T>());
    const int nb = (np + 255) / 256;
    long long nl = 0;                                        // kernels launched by this step
    const bool cm = std::is_same<T, float>::value && gc.cm;
    if (phases & 1) {
    trace_mark(g, 0, st);
    if (np > 0) {
        nl += 2;
        if (bc.sample_mode == AL_SAMPLE_GAUSS)               // one warp per point
            k_points_w<T><<<(unsigned)(((long long)np * 32 + 255) / 256), 256, 0, st>>>(gc, bc, p, sc, status);
        else
            k_points<T><<<nb, 256, 0, st>>>(gc, bc, p, sc, status);
        launch_pdl(k_segments<T>, nb, 256, 0, st, bc, sc);
    }
    if (g->n_lines > 0) { launch_pdl(k_lines<T>, (g->n_lines + 7) / 8, 256, 0, st, gc, bc, sc, p, status); ++nl; }
    trace_mark(g, 1, st);
    if (np > 0) { launch_pdl(k_mask<T>, nb, 256, 0, st, gc, bc, sc); ++nl; }
    if constexpr (std::is_same<T, float>::value) {
        if (gc.cm) {
            if (np == 0) AL_CUDA(cudaMemsetAsync(g->cmcnt, 0, 5 * sizeof(int), st));   // (k_points resets them)
            launch_pdl(k_cm_entries<float>, (unsigned)((gc.nbrick * 32 + 255) / 256), 256, 0, st, gc, bc, sc, status);
            ++nl;
        }
    }
    trace_mark(g, 2, st);
    if (np > 0) {
        if (gc.wmode != 0) {
            launch_pdl(k_weights<T>, (unsigned)(((long long)np * 32 + 127) / 128), 128, 0, st, gc, bc, sc, p, status);
            ++nl;
        }
        nl += cm ? 2 : 1;
        if constexpr (std::is_same<T, float>::value) {
            if (cm) {
                const int rc = cm_launch_bz(I, true, st);
                if (rc != AL_OK) return rc;
            } else {
                launch_bricks_bz<T>(I, true, st);
            }
        } else {
            launch_bricks_bz<T>(I, true, st);
        }
    }
    trace_mark(g, 3, st);
    }
    if (!(phases & 2)) {
        g->launches += nl;
        AL_CUDA(cudaGetLastError());
        return AL_OK;
    }
    if (np > 0) { launch_pdl(k_normalise<T>, nb, 256, 0, st, gc, bc, sc, p, status); ++nl; }
    trace_mark(g, 4, st);
    nl += cm ? 2 : 1;
    if constexpr (std::is_same<T, float>::value) {
        if (cm) {
            const int rc = cm_launch_bz(I, false, st);
            if (rc != AL_OK) return rc;
        } else {
            launch_bricks_bz<T>(I, false, st);
        }
    } else {
        launch_bricks_bz<T>(I, false, st);
    }
    if (gc.smode != 0 && np > 0) {
        // scatter form: certified lines add their sources with atomics after the
        // gather has written every cell (uncertified lines and deposits)
        AL_CUDA(cudaMemsetAsync(g->scatSum, 0, 3 * sizeof(double), st));
        launch_pdl(k_scatter<T>, (unsigned)(((long long)np * 32 + 127) / 128), 128, 0, st, gc, bc, sc, p, status);
        ++nl;
    }
    trace_mark(g, 5, st);
    launch_pdl(k_totals<T>, TOT_PARTS, 256, 0, st, gc, bc, sc, I.totals);
    ++nl;
    g->launches += nl;
    trace_mark(g, 6, st);
    AL_CUDA(cudaGetLastError());
    return AL_OK;
}

static int check_step(al_grid g, const al_step_in *in, const al_step_out *out);

extern "C" int al_sample_drag_spread(al_grid g, const al_step_in *in, const al_step_out *out, void *stream) {
    const int rc = check_step(g, in, out);
    if (rc != AL_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    return g->d.precision == AL_FP64 ? step_impl<double>(g, in, out, st) : step_impl<float>(g, in, out, st);
}

// one step with host inputs and results: the copies in, the step (after the
// previous al_step_host step of the instance, whatever its stream), the
// copies out, all on `stream`
extern "C" int al_step_host(al_grid g, const al_step_in *host_in, const al_step_out *host_out,
                            const al_step_in *dev_in, const al_step_out *dev_out, void *stream) {
    if (!g || !host_in || !host_out) return AL_ERR_ARG;
    int rc = check_step(g, dev_in, dev_out);
    if (rc != AL_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = g->d.precision == AL_FP64 ? sizeof(double) : sizeof(float);
    const size_t bc = es * (size_t)g->d.nx * g->d.ny * g->d.nz, bp = es * (size_t)g->n_points;
    auto h2d = [&](const void *dst, const void *src, size_t bytes) -> int {
        if (!src || !dst || bytes == 0) return AL_OK;
        AL_CUDA(cudaMemcpyAsync(const_cast<void *>(dst), src, bytes, cudaMemcpyHostToDevice, st));
        return AL_OK;
    };
    for (int a = 0; a < 3 && rc == AL_OK; ++a) rc = h2d(dev_in->U[a], host_in->U[a], bc);
    if (rc == AL_OK && g->d.has_alpha) rc = h2d(dev_in->alpha, host_in->alpha, bc);
    for (int a = 0; a < 3 && rc == AL_OK; ++a) {
        rc = h2d(dev_in->P[a], host_in->P[a], bp);
        if (rc == AL_OK) rc = h2d(dev_in->Pdot[a], host_in->Pdot[a], bp);
        if (rc == AL_OK && dev_in->P_spread[a]) rc = h2d(dev_in->P_spread[a], host_in->P_spread[a], bp);
        if (rc == AL_OK && g->bd.tangents_given) rc = h2d(dev_in->tangent[a], host_in->tangent[a], bp);
        if (rc == AL_OK && g->d_cmn && dev_in->U_prev[a]) rc = h2d(dev_in->U_prev[a], host_in->U_prev[a], bc);
        if (rc == AL_OK && g->d_cmn && dev_in->Pddot[a]) rc = h2d(dev_in->Pddot[a], host_in->Pddot[a], bp);
    }
    if (rc != AL_OK) return rc;
    if (!g->host_ev) AL_CUDA(cudaEventCreateWithFlags(&g->host_ev, cudaEventDisableTiming));
    if (g->host_ev_set) AL_CUDA(cudaStreamWaitEvent(st, g->host_ev, 0));
    rc = g->d.precision == AL_FP64 ? step_impl<double>(g, dev_in, dev_out, st) : step_impl<float>(g, dev_in, dev_out, st);
    if (rc != AL_OK) return rc;
    AL_CUDA(cudaEventRecord(g->host_ev, st));
    g->host_ev_set = true;
    for (int a = 0; a < 3; ++a) {
        if (host_out->S[a]) AL_CUDA(cudaMemcpyAsync(host_out->S[a], dev_out->S[a], bc, cudaMemcpyDeviceToHost, st));
        if (host_out->F[a] && bp) AL_CUDA(cudaMemcpyAsync(host_out->F[a], dev_out->F[a], bp, cudaMemcpyDeviceToHost, st));
    }
    return AL_OK;
}

extern "C" int al_step_begin(al_grid g, const al_step_in *in, const al_step_out *out, void *stream) {
    const int rc = check_step(g, in, out);
    if (rc != AL_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    return g->d.precision == AL_FP64 ? step_impl<double>(g, in, out, st, 1) : step_impl<float>(g, in, out, st, 1);
}

extern "C" int al_step_end(al_grid g, const al_step_in *in, const al_step_out *out, void *stream) {
    const int rc = check_step(g, in, out);
    if (rc != AL_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    return g->d.precision == AL_FP64 ? step_impl<double>(g, in, out, st, 2) : step_impl<float>(g, in, out, st, 2);
}

extern "C" int al_weights_get(al_grid g, void *dst, void *stream) {
    if (!g || (!dst && g->n_points > 0)) return AL_ERR_ARG;
    if (!g->loaded) return AL_ERR_STATE;
    if (!owns_part(g) && g->gc.wmode != AL_WEIGHTS_BRICK) return AL_ERR_STATE;
    if (g->n_points > 0)
        AL_CUDA(cudaMemcpyAsync(dst, g->wfix, (size_t)g->n_points * sizeof(unsigned long long),
                                cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return AL_OK;
}

extern "C" int al_weights_set(al_grid g, const void *src, void *stream) {
    if (!g || (!src && g->n_points > 0)) return AL_ERR_ARG;
    if (!g->loaded) return AL_ERR_STATE;
    if (!owns_part(g) && g->gc.wmode != AL_WEIGHTS_BRICK) return AL_ERR_STATE;
    if (g->n_points > 0)
        AL_CUDA(cudaMemcpyAsync(g->wfix, src, (size_t)g->n_points * sizeof(unsigned long long),
                                cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return AL_OK;
}

static int check_step(al_grid g, const al_step_in *in, const al_step_out *out) {
    if (!g || !in || !out) return AL_ERR_ARG;
    if (!g->loaded) return AL_ERR_STATE;
    for (int a = 0; a < 3; ++a)
        if (!in->U[a] || !out->S[a]) return AL_ERR_ARG;
    if (g->d.has_alpha && !in->alpha) return AL_ERR_ARG;
    if (g->n_points > 0) {
        for (int a = 0; a < 3; ++a) {
            if (!in->P[a] || !in->Pdot[a] || !out->F[a]) return AL_ERR_ARG;
            if (g->bd.tangents_given && !in->tangent[a]) return AL_ERR_ARG;
        }
        const bool sp = in->P_spread[0] != nullptr;
        if ((in->P_spread[1] != nullptr) != sp || (in->P_spread[2] != nullptr) != sp) return AL_ERR_ARG;
        if (g->d_cmn) {                                   // inertia term: all three or none of each
            const bool up = in->U_prev[0] != nullptr, pa = in->Pddot[0] != nullptr;
            for (int a = 1; a < 3; ++a)
                if ((in->U_prev[a] != nullptr) != up || (in->Pddot[a] != nullptr) != pa) return AL_ERR_ARG;
            if (up && !(in->dt > 0.0 && std::isfinite(in->dt))) return AL_ERR_ARG;
        }
    }
    // a slab: no reflecting face and the paper's nearest-segment projection
    if (owns_part(g) && (g->bd.wall_reflect || g->bd.proj_mode != AL_PROJ_NEAREST)) return AL_ERR_STATE;
    return AL_OK;
}

extern "C" int al_set_option(al_grid g, int option, int value) {
    if (!g) return AL_ERR_ARG;
    switch (option) {
    case AL_OPT_WEIGHTS:
        if (value != AL_WEIGHTS_BRICK && value != AL_WEIGHTS_SEGMENT) return AL_ERR_ARG;
        g->gc.wmode = value;
        return arena_sync(g);
    case AL_OPT_BRICK_Z:
        if (value != 4 && value != 8 && value != 16) return AL_ERR_ARG;
        set_brick_z(g->gc, value);
        return AL_OK;
    case AL_OPT_SPREAD:
        if (value != AL_SPREAD_GATHER && value != AL_SPREAD_SCATTER) return AL_ERR_ARG;
        g->gc.smode = value;
        return AL_OK;
    case AL_OPT_RECORD:
        if (value < 0 || value > 2) return AL_ERR_ARG;
        g->opt_record = value;
        return arena_sync(g);
    case AL_OPT_COLUMN:
        if (value != 0 && value != 1) return AL_ERR_ARG;
        g->opt_column = value;
        return AL_OK;
    case AL_OPT_OWN_X0:
        if (value < 0 || value % al::BX != 0 || value >= g->d.nx) return AL_ERR_ARG;
        g->own_x0 = value;
        return AL_OK;
    case AL_OPT_OWN_X1:
        if (value != -1 && (value <= 0 || value > g->d.nx || (value % al::BX != 0 && value != g->d.nx)))
            return AL_ERR_ARG;
        g->own_x1 = value;
        return AL_OK;
    default:
        return AL_ERR_ARG;
    }
}

extern "C" int al_trace_enable(al_grid g, int on) {
    if (!g) return AL_ERR_ARG;
    if (on && !g->trace) {
        for (int i = 0; i <= AL_TRACE_N; ++i) AL_CUDA(cudaEventCreate(&g->ev[i]));
        g->trace = true;
    } else if (!on && g->trace) {
        cudaDeviceSynchronize();
        for (int i = 0; i <= AL_TRACE_N; ++i) cudaEventDestroy(g->ev[i]);
        g->trace = false;
    }
    return AL_OK;
}

extern "C" int al_trace_last(al_grid g, float *ms) {
    if (!g || !ms) return AL_ERR_ARG;
    if (!g->trace) return AL_ERR_STATE;
    AL_CUDA(cudaEventSynchronize(g->ev[AL_TRACE_N]));
    for (int i = 0; i < AL_TRACE_N; ++i) AL_CUDA(cudaEventElapsedTime(&ms[i], g->ev[i], g->ev[i + 1]));
    return AL_OK;
}

extern "C" int al_destroy(al_grid g) {
    if (!g) return AL_ERR_ARG;
    cudaDeviceSynchronize();
    if (g->trace) al_trace_enable(g, 0);
    free_beams(g);
    if (g->grid_slab) cudaFree(g->grid_slab);
    if (g->host_ev) cudaEventDestroy(g->host_ev);
    delete g;
    return AL_OK;
}

extern "C" int al_get_state(al_grid g, void *f_prev_dev, int *has_prev, void *stream) {
    if (!g || !has_prev) return AL_ERR_ARG;
    if (!g->loaded) return AL_ERR_STATE;
    if (g->n_points > 0 && !f_prev_dev) return AL_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (g->n_points > 0)
        AL_CUDA(cudaMemcpyAsync(f_prev_dev, g->fprev, 3 * (size_t)g->n_points * g->esize, cudaMemcpyDeviceToDevice, st));
    int hp = 0;
    AL_CUDA(cudaMemcpyAsync(&hp, g->hasPrev, sizeof(int), cudaMemcpyDeviceToHost, st));
    AL_CUDA(cudaStreamSynchronize(st));
    *has_prev = hp;
    return AL_OK;
}

extern "C" int al_set_state(al_grid g, const void *f_prev_dev, int has_prev, void *stream) {
    if (!g) return AL_ERR_ARG;
    if (!g->loaded) return AL_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    if (g->n_points > 0 && has_prev) {
        if (!f_prev_dev) return AL_ERR_ARG;
        AL_CUDA(cudaMemcpyAsync(g->fprev, f_prev_dev, 3 * (size_t)g->n_points * g->esize,
                                cudaMemcpyDeviceToDevice, st));
    }
    AL_CUDA(cudaMemsetAsync(g->hasPrev, has_prev ? 0x01 : 0, 1, st));
    AL_CUDA(cudaMemsetAsync((char *)g->hasPrev + 1, 0, sizeof(int) - 1, st));
    return AL_OK;
}

template <typename T>
static int beam_qs_t(al_grid g, const double *EI, const double axis[3], const void *const P0[3],
                     const void *const F[3], void *const P_out[3], cudaStream_t st) {
    using namespace al;
    StepPtrs<T> p{};
    for (int a = 0; a < 3; ++a) {
        p.P[a] = (const T *)P0[a];
        p.F[a] = (T *)F[a];
        p.S[a] = (T *)P_out[a];
    }
    BeamsC bc{};
    bc.n_lines = g->n_lines; bc.n_points = g->n_points; bc.line_off = g->d_line_off;
    // the stiffnesses go to the device only when they change
    if (g->h_EI.size() != (size_t)g->n_lines || !std::equal(EI, EI + g->n_lines, g->h_EI.begin())) {
        g->h_EI.assign(EI, EI + g->n_lines);
        AL_CUDA(cudaMemcpyAsync(g->d_EI, g->h_EI.data(), (size_t)g->n_lines * sizeof(double),
                                cudaMemcpyHostToDevice, st));
    }
    k_beam_qs<T><<<(unsigned)((g->n_lines + 7) / 8), 256, 0, st>>>(bc, g->d_EI, (T)axis[0], (T)axis[1],
                                                                     (T)axis[2], p);
    AL_CUDA(cudaGetLastError());
    return AL_OK;
}

extern "C" int al_beam_quasistatic(al_grid g, const double *EI, const double axis[3], const void *const P0[3],
                                   const void *const F[3], void *const P_out[3], void *stream) {
    if (!g || !axis || !P0 || !F || !P_out) return AL_ERR_ARG;
    if (!g->loaded) return AL_ERR_STATE;
    if (g->n_lines == 0) return AL_OK;
    if (!EI) return AL_ERR_ARG;
    for (int l = 0; l < g->n_lines; ++l)
        if (!(EI[l] > 0.0) || !std::isfinite(EI[l])) return AL_ERR_ARG;
    const double an = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    if (!(std::fabs(an - 1.0) < 1e-9)) return AL_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        if (!P0[a] || !F[a] || !P_out[a]) return AL_ERR_ARG;
        if (P_out[a] == P0[a] || P_out[a] == F[a]) return AL_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return g->d.precision == AL_FP64 ? beam_qs_t<double>(g, EI, axis, P0, F, P_out, st)
                                     : beam_qs_t<float>(g, EI, axis, P0, F, P_out, st);
}

extern "C" int al_sizes(al_grid g, long long *n_cells, long long *n_points, int *n_lines) {
    if (!g) return AL_ERR_ARG;
    if (n_cells) *n_cells = g->gc.ncell;
    if (n_points) *n_points = g->n_points;
    if (n_lines) *n_lines = g->n_lines;
    return AL_OK;
}

extern "C" int al_footprint(al_grid g, unsigned long long *bytes) {
    if (!g || !bytes) return AL_ERR_ARG;
    *bytes = (unsigned long long)(page_round(g->grid_bytes) + page_round(g->beam_bytes) + page_round(g->rec_bytes));
    return AL_OK;
}

// ---------------------------------------------------------------------------
// batched form
// ---------------------------------------------------------------------------

struct al_batch_s {
    std::vector<al_grid> grids;
    std::vector<al_step_in> ins;
    std::vector<al_step_out> outs;
    int precision = -1;
    int capacity = 0;                          // slots (>= added instances)
    bool committed = false;
    void *h_inst = nullptr;                    // pinned staging of slot descriptors
    std::vector<cudaEvent_t> slot_ev;
    bool use_graph = false;
    int n = 0;
    void *d_inst = nullptr;                   // Inst<T>[n]
    long long *d_pre = nullptr;               // 4 prefix arrays of n + 1: points, lines, bricks, points(warps)
    unsigned long long *d_ctr = nullptr;      // [4] brick counters of the persistent passes (al_batch_run)
    long long tot_pts = 0, tot_lines = 0, tot_bricks = 0;
    int spread_grid = 0, pt_grid = 0;
    int bz = 8;                               // brick height of the batch's projection
    int ctas = 0;                             // persistent CTAs per SM (0: as many as fit)
    int occ = 1;                              // CTAs per SM that fit at this brick height
    bool any_segment_weights = false;         // some instance sums weights per segment
    bool any_gauss = false;                   // some instance samples by volume average (warp per point)
    bool any_reflect = false;                 // some instance reflects its kernel at grid faces
    // subset runs: a ring of pinned host / device work lists
    static constexpr int RING = 8;
    int maxn = 0;
    void *h_ring = nullptr;                   // pinned: RING x (sel[maxn] + pre[3 (maxn+1)])
    void *d_ring = nullptr;
    cudaEvent_t ring_ev[RING] = {};
    int ring_pos = 0;
    std::vector<long long> cnt_pts, cnt_lines, cnt_bricks;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    long long launches = 0;                   // kernels the batch's runs launched (al_batch_launches)
    int last_nl = 0;                          // kernels of the last enqueue
    int graph_nl = 0;                         // kernels in the captured graph

    // a subset run's slot: selection, 3 prefix arrays, 4 brick counters
    static size_t slot_bytes(int n) {
        size_t a = ((size_t)n * sizeof(int) + 15) & ~(size_t)15;
        return a + 3 * (size_t)(n + 1) * sizeof(long long) + 4 * sizeof(unsigned long long);
    }
};

extern "C" int al_batch_create(al_batch *out) {
    if (!out) return AL_ERR_ARG;
    *out = new (std::nothrow) al_batch_s();
    return *out ? AL_OK : AL_ERR_OOM;
}

extern "C" int al_batch_add(al_batch b, al_grid g, const al_step_in *in, const al_step_out *out) {
    if (!b || !g || !in || !out) return AL_ERR_ARG;
    if (b->committed) return AL_ERR_STATE;
    if (!g->loaded || owns_part(g)) return AL_ERR_STATE;
    if (b->precision >= 0 && b->precision != g->d.precision) return AL_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!in->U[a] || !out->S[a]) return AL_ERR_ARG;
    if (g->d.has_alpha && !in->alpha) return AL_ERR_ARG;
    if (g->n_points > 0)
        for (int a = 0; a < 3; ++a)
            if (!in->P[a] || !in->Pdot[a] || !out->F[a] || (g->bd.tangents_given && !in->tangent[a]))
                return AL_ERR_ARG;
    b->precision = g->d.precision;
    b->grids.push_back(g);
    b->ins.push_back(*in);
    b->outs.push_back(*out);
    return AL_OK;
}

// (Re)build the device instance table and work-list prefixes for the
// batch's brick height and persistent grid size; a captured graph is dropped
// (it is captured again at the next run).
template <typename T>
static int batch_rebuild_t(al_batch b) {
    using namespace al;
    AL_CUDA(cudaDeviceSynchronize());                    // no step or slot update in flight
    const int n = b->n;
    Inst<T> *h = (Inst<T> *)b->h_inst;
    std::vector<long long> pre(4 * (size_t)(n + 1), 0);
    b->any_segment_weights = false;
    b->any_gauss = false;
    b->any_reflect = false;
    b->cnt_pts.assign(n, 0); b->cnt_lines.assign(n, 0); b->cnt_bricks.assign(n, 0);
    for (int q = 0; q < n; ++q) {
        const bool used = b->grids[q] != nullptr;
        if (used) {
            h[q] = make_inst<T>(b->grids[q], &b->ins[q], &b->outs[q]);
            set_brick_z(h[q].g, b->bz);
            h[q].g.smode = 0;                                // batches always gather
            h[q].g.cm = 0;                                   // and take the brick passes
            h[q].sc.cmN = nullptr;
            h[q].sc.cmlay = nullptr;
            h[q].sc.cment_n = nullptr;
            if (h[q].g.wmode != 0) b->any_segment_weights = true;
            if (h[q].b.sample_mode == AL_SAMPLE_GAUSS) b->any_gauss = true;
            if (h[q].b.reflect) b->any_reflect = true;
            b->cnt_pts[q] = b->grids[q]->n_points;
            b->cnt_lines[q] = b->grids[q]->n_lines;
            b->cnt_bricks[q] = h[q].g.nbrick;
        } else {
            memset((void *)&h[q], 0, sizeof(Inst<T>));
        }
        pre[0 * (n + 1) + q + 1] = pre[0 * (n + 1) + q] + b->cnt_pts[q];
        pre[1 * (n + 1) + q + 1] = pre[1 * (n + 1) + q] + b->cnt_lines[q];
        pre[2 * (n + 1) + q + 1] = pre[2 * (n + 1) + q] + b->cnt_bricks[q];
    }
    b->tot_pts = pre[n];
    b->tot_lines = pre[(n + 1) + n];
    b->tot_bricks = pre[2 * (n + 1) + n];
    AL_CUDA(cudaMemcpy(b->d_inst, h, sizeof(Inst<T>) * n, cudaMemcpyHostToDevice));
    AL_CUDA(cudaMemcpy(b->d_pre, pre.data(), sizeof(long long) * pre.size(), cudaMemcpyHostToDevice));
    AL_CUDA(spread_smem_attr<T>());
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    switch (b->bz) {
    case 4: AL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_spread<T, 4>, SPREAD_THREADS, sizeof(SpreadSmem<T, 4, true>))); break;
    case 16: AL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_spread<T, 16>, SPREAD_THREADS, sizeof(SpreadSmem<T, 16, true>))); break;
    default: AL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_spread<T, 8>, SPREAD_THREADS, sizeof(SpreadSmem<T, 8, true>))); break;
    }
    if (occ < 1) occ = 1;
    b->occ = occ;
    const int per = b->ctas > 0 ? std::min(b->ctas, occ) : occ;
    b->spread_grid = nsm * per;                          // capped by each run's brick count at launch
    b->pt_grid = nsm * 8;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    return AL_OK;
}

template <typename T>
static int batch_commit_t(al_batch b) {
    using namespace al;
    const int added = (int)b->grids.size();
    const int n = std::max(added, b->capacity);
    b->grids.resize(n, nullptr);
    b->ins.resize(n, al_step_in{});
    b->outs.resize(n, al_step_out{});
    AL_CUDA(cudaMallocHost(&b->h_inst, sizeof(Inst<T>) * (n ? n : 1)));
    b->slot_ev.assign(n, nullptr);
    for (int q = 0; q < n; ++q) AL_CUDA(cudaEventCreateWithFlags(&b->slot_ev[q], cudaEventDisableTiming));
    b->maxn = n;
    const size_t slot = al_batch_s::slot_bytes(n);
    AL_CUDA(cudaMallocHost(&b->h_ring, slot * al_batch_s::RING));
    AL_CUDA(cudaMalloc(&b->d_ring, slot * al_batch_s::RING));
    for (int r = 0; r < al_batch_s::RING; ++r) AL_CUDA(cudaEventCreateWithFlags(&b->ring_ev[r], cudaEventDisableTiming));
    AL_CUDA(cudaMalloc(&b->d_inst, sizeof(Inst<T>) * (n ? n : 1)));
    AL_CUDA(cudaMalloc(&b->d_pre, sizeof(long long) * 4 * (size_t)(n + 1)));
    AL_CUDA(cudaMalloc(&b->d_ctr, 4 * sizeof(unsigned long long)));
    return batch_rebuild_t<T>(b);
}

// enqueue one step of n selected instances (sel NULL: all); pre: device
// prefix arrays (points, lines, bricks) of the selection; totals: host copies
template <typename T>
static int batch_enqueue_t(al_batch b, cudaStream_t st, const int *sel, const long long *pre, int n,
                           long long tot_pts, long long tot_lines, long long tot_bricks, unsigned long long *ctr) {
    using namespace al;
    AL_CUDA(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned long long), st));
    const Inst<T> *I = (const Inst<T> *)b->d_inst;
    const long long *pp = pre, *pl = pre + (n + 1), *pb = pre + 2 * (n + 1);
    auto grid_for = [&](long long items, int per_block) {
        long long g = (items + per_block - 1) / per_block;
        return (unsigned)std::max<long long>(1, std::min<long long>(g, (long long)b->pt_grid * 4));
    };
    int nl = 0;
    if (tot_pts > 0) {
        // each instance in the same form as alone: a warp per point for the
        // volume-average sampler, a thread per point otherwise
        kb_points<T><<<grid_for(tot_pts, 256), 256, 0, st>>>(I, sel, pp, n, b->any_gauss ? 1 : 0);
        if (b->any_gauss) kb_points_w<T><<<grid_for(tot_pts, 8), 256, 0, st>>>(I, sel, pp, n);
        kb_segments<T><<<grid_for(tot_pts, 256), 256, 0, st>>>(I, sel, pp, n);
        nl += b->any_gauss ? 3 : 2;
    }
    if (tot_lines > 0) { kb_lines<T><<<grid_for(tot_lines, 8), 256, 0, st>>>(I, sel, pl, n); ++nl; }
    if (tot_pts > 0) {
        kb_mask<T><<<grid_for(tot_pts, 256), 256, 0, st>>>(I, sel, pp, n);
        ++nl;
        if (b->any_segment_weights) { kb_weights<T><<<grid_for(tot_pts, 4), 128, 0, st>>>(I, sel, pp, n); ++nl; }
        if (tot_bricks > 0) {
            const int gs = (int)std::min<long long>(b->spread_grid, tot_bricks);
            switch (b->bz) {
            case 4: kb_bweights<T, 4><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 4, false>), st>>>(I, sel, pb, n, ctr); break;
            case 16: kb_bweights<T, 16><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 16, false>), st>>>(I, sel, pb, n, ctr); break;
            default: kb_bweights<T, 8><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 8, false>), st>>>(I, sel, pb, n, ctr); break;
            }
            if (b->any_reflect) switch (b->bz) {
            case 4: kb_bweights_refl<T, 4><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 4, false>), st>>>(I, sel, pb, n, ctr); break;
            case 16: kb_bweights_refl<T, 16><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 16, false>), st>>>(I, sel, pb, n, ctr); break;
            default: kb_bweights_refl<T, 8><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 8, false>), st>>>(I, sel, pb, n, ctr); break;
            }
            nl += b->any_reflect ? 2 : 1;
        }
        kb_normalise<T><<<grid_for(tot_pts, 256), 256, 0, st>>>(I, sel, pp, n);
        ++nl;
    }
    if (tot_bricks > 0) {
        const int gs = (int)std::min<long long>(b->spread_grid, tot_bricks);
        switch (b->bz) {
        case 4: kb_spread<T, 4><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 4, true>), st>>>(I, sel, pb, n, ctr); break;
        case 16: kb_spread<T, 16><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 16, true>), st>>>(I, sel, pb, n, ctr); break;
        default: kb_spread<T, 8><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 8, true>), st>>>(I, sel, pb, n, ctr); break;
        }
        if (b->any_reflect) switch (b->bz) {
        case 4: kb_spread_refl<T, 4><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 4, false>), st>>>(I, sel, pb, n, ctr); break;
        case 16: kb_spread_refl<T, 16><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 16, false>), st>>>(I, sel, pb, n, ctr); break;
        default: kb_spread_refl<T, 8><<<gs, SPREAD_THREADS, sizeof(SpreadSmem<T, 8, false>), st>>>(I, sel, pb, n, ctr); break;
        }
        nl += b->any_reflect ? 2 : 1;
    }
    kb_totals<T><<<std::max(1, std::min(n * TOT_PARTS, 2048)), 256, 0, st>>>(I, sel, n);
    kb_totals_fin<T><<<std::max(1, std::min(n, 1024)), 32, 0, st>>>(I, sel, n);
    nl += 2;
    b->last_nl = nl;
    AL_CUDA(cudaGetLastError());
    return AL_OK;
}

extern "C" int al_batch_reserve(al_batch b, int n_slots, int precision) {
    if (!b || n_slots < 0 || (precision != AL_FP32 && precision != AL_FP64)) return AL_ERR_ARG;
    if (b->committed) return AL_ERR_STATE;
    if (b->precision >= 0 && b->precision != precision) return AL_ERR_ARG;
    b->precision = precision;
    b->capacity = n_slots;
    return AL_OK;
}

template <typename T>
static int batch_assign_t(al_batch b, int slot, al_grid g, const al_step_in *in, const al_step_out *out,
                          cudaStream_t st) {
    using namespace al;
    AL_CUDA(cudaEventSynchronize(b->slot_ev[slot]));       // staging of this slot is free again
    Inst<T> *h = (Inst<T> *)b->h_inst + slot;
    if (g) {
        *h = make_inst<T>(g, in, out);
        set_brick_z(h->g, b->bz);
        h->g.smode = 0;                                      // batches always gather
        h->g.cm = 0;                                         // and take the brick passes
        h->sc.cmN = nullptr;
        h->sc.cmlay = nullptr;
        h->sc.cment_n = nullptr;
    } else {
        memset((void *)h, 0, sizeof(Inst<T>));
    }
    AL_CUDA(cudaMemcpyAsync((Inst<T> *)b->d_inst + slot, h, sizeof(Inst<T>), cudaMemcpyHostToDevice, st));
    AL_CUDA(cudaEventRecord(b->slot_ev[slot], st));
    b->grids[slot] = g;
    if (g) { b->ins[slot] = *in; b->outs[slot] = *out; }
    if (g && h->g.wmode != 0) b->any_segment_weights = true;
    if (g && g->bd.sample_mode == AL_SAMPLE_GAUSS) b->any_gauss = true;
    if (g && g->bd.wall_reflect) b->any_reflect = true;
    b->cnt_pts[slot] = g ? g->n_points : 0;
    b->cnt_lines[slot] = g ? g->n_lines : 0;
    b->cnt_bricks[slot] = g ? h->g.nbrick : 0;
    return AL_OK;
}

extern "C" int al_batch_assign(al_batch b, int slot, al_grid g, const al_step_in *in, const al_step_out *out,
                               void *stream) {
    if (!b) return AL_ERR_ARG;
    if (!b->committed) return AL_ERR_STATE;
    if (slot < 0 || slot >= b->n) return AL_ERR_ARG;
    if (g) {
        if (!in || !out || !g->loaded || g->d.precision != b->precision) return AL_ERR_ARG;
        if (owns_part(g)) return AL_ERR_STATE;
        for (int a = 0; a < 3; ++a)
            if (!in->U[a] || !out->S[a]) return AL_ERR_ARG;
        if (g->d.has_alpha && !in->alpha) return AL_ERR_ARG;
        if (g->n_points > 0)
            for (int a = 0; a < 3; ++a)
                if (!in->P[a] || !in->Pdot[a] || !out->F[a] || (g->bd.tangents_given && !in->tangent[a]))
                    return AL_ERR_ARG;
    }
    if (b->use_graph && b->exec) return AL_ERR_STATE;         // a captured graph holds the old table
    cudaStream_t st = (cudaStream_t)stream;
    return b->precision == AL_FP64 ? batch_assign_t<double>(b, slot, g, in, out, st)
                                   : batch_assign_t<float>(b, slot, g, in, out, st);
}

extern "C" int al_batch_commit(al_batch b, int use_graph, int spread_ctas_per_sm) {
    if (!b) return AL_ERR_ARG;
    if (b->committed) return AL_ERR_STATE;
    if (b->grids.empty() && b->capacity == 0) return AL_ERR_ARG;
    if (b->precision < 0) return AL_ERR_ARG;
    b->n = std::max((int)b->grids.size(), b->capacity);
    if (spread_ctas_per_sm < 0) return AL_ERR_ARG;
    b->ctas = spread_ctas_per_sm;
    int rc = b->precision == AL_FP64 ? batch_commit_t<double>(b) : batch_commit_t<float>(b);
    if (rc != AL_OK) return rc;
    b->use_graph = use_graph != 0;
    b->committed = true;
    return AL_OK;
}

extern "C" int al_batch_run(al_batch b, void *stream) {
    if (!b) return AL_ERR_ARG;
    if (!b->committed) return AL_ERR_STATE;
    for (int q = 0; q < b->n; ++q)
        if (!b->grids[q]) return AL_ERR_STATE;                // every slot must be bound
    cudaStream_t st = (cudaStream_t)stream;
    auto enqueue = [&](cudaStream_t s) {
        return b->precision == AL_FP64
                   ? batch_enqueue_t<double>(b, s, nullptr, b->d_pre, b->n, b->tot_pts, b->tot_lines, b->tot_bricks,
                                             b->d_ctr)
                   : batch_enqueue_t<float>(b, s, nullptr, b->d_pre, b->n, b->tot_pts, b->tot_lines, b->tot_bricks,
                                            b->d_ctr);
    };
    if (!b->use_graph) {
        int rc = enqueue(st);
        if (rc == AL_OK) b->launches += b->last_nl;
        return rc;
    }
    if (!b->exec) {
        if (!b->cap) AL_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        AL_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue(b->cap);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
        if (rc != AL_OK) return rc;
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        b->graph = graph;
        b->graph_nl = b->last_nl;
        AL_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    AL_CUDA(cudaGraphLaunch(b->exec, st));
    b->launches += b->graph_nl;
    return AL_OK;
}

extern "C" int al_batch_run_subset(al_batch b, const int *idx, int n_idx, void *stream) {
    if (!b || (n_idx > 0 && !idx) || n_idx < 0) return AL_ERR_ARG;
    if (!b->committed) return AL_ERR_STATE;
    if (n_idx > b->maxn) return AL_ERR_CAPACITY;
    if (n_idx == 0) return AL_OK;
    for (int k = 0; k < n_idx; ++k) {
        if (idx[k] < 0 || idx[k] >= b->n || !b->grids[idx[k]]) return AL_ERR_ARG;
        for (int j = 0; j < k; ++j)
            if (idx[j] == idx[k]) return AL_ERR_ARG;     // one step per instance per run
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int r = b->ring_pos;
    b->ring_pos = (b->ring_pos + 1) % al_batch_s::RING;
    // the slot's previous work list must have been consumed
    AL_CUDA(cudaEventSynchronize(b->ring_ev[r]));
    const size_t slot = al_batch_s::slot_bytes(b->maxn);
    char *h = (char *)b->h_ring + r * slot, *d = (char *)b->d_ring + r * slot;
    const size_t off_pre = ((size_t)b->maxn * sizeof(int) + 15) & ~(size_t)15;
    int *hs = (int *)h;
    long long *hp = (long long *)(h + off_pre);
    long long tp = 0, tl = 0, tb = 0;
    hp[0] = hp[n_idx + 1] = hp[2 * (n_idx + 1)] = 0;
    for (int k = 0; k < n_idx; ++k) {
        hs[k] = idx[k];
        tp += b->cnt_pts[idx[k]]; tl += b->cnt_lines[idx[k]]; tb += b->cnt_bricks[idx[k]];
        hp[k + 1] = tp; hp[(n_idx + 1) + k + 1] = tl; hp[2 * (n_idx + 1) + k + 1] = tb;
    }
    AL_CUDA(cudaMemcpyAsync(d, h, off_pre + 3 * (size_t)(n_idx + 1) * sizeof(long long), cudaMemcpyHostToDevice, st));
    const int *ds = (const int *)d;
    const long long *dp = (const long long *)(d + off_pre);
    unsigned long long *dc =
        reinterpret_cast<unsigned long long *>(d + off_pre + 3 * (size_t)(n_idx + 1) * sizeof(long long));
    int rc = b->precision == AL_FP64 ? batch_enqueue_t<double>(b, st, ds, dp, n_idx, tp, tl, tb, dc)
                                     : batch_enqueue_t<float>(b, st, ds, dp, n_idx, tp, tl, tb, dc);
    if (rc != AL_OK) return rc;
    b->launches += b->last_nl;
    AL_CUDA(cudaEventRecord(b->ring_ev[r], st));
    return AL_OK;
}

extern "C" int al_batch_destroy(al_batch b) {
    if (!b) return AL_ERR_ARG;
    cudaDeviceSynchronize();
    for (int r = 0; r < al_batch_s::RING; ++r)
        if (b->ring_ev[r]) cudaEventDestroy(b->ring_ev[r]);
    if (b->h_ring) cudaFreeHost(b->h_ring);
    if (b->h_inst) cudaFreeHost(b->h_inst);
    for (cudaEvent_t e : b->slot_ev)
        if (e) cudaEventDestroy(e);
    if (b->d_ring) cudaFree(b->d_ring);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_pre) cudaFree(b->d_pre);
    if (b->d_ctr) cudaFree(b->d_ctr);
    delete b;
    return AL_OK;
}

// ---------------------------------------------------------------------------
// autotuning: time every execution choice on the caller's own step and keep
// the fastest.  The relaxation state and the status counters are restored,
// so tuning leaves the instance as it found it (S, F and totals hold the
// last trial's outputs).
// ---------------------------------------------------------------------------
namespace {
struct saved_state {
    void *fprev = nullptr;
    int has_prev = 0;
    int status[AL_STATUS_N] = {};
};
int save_state(al_grid g, const al_step_out *out, saved_state &sv, cudaStream_t st) {
    if (g->n_points > 0) AL_CUDA(cudaMalloc(&sv.fprev, 3 * (size_t)g->n_points * g->esize));
    int rc = al_get_state(g, sv.fprev, &sv.has_prev, st);
    if (rc != AL_OK) return rc;
    if (out && out->status)
        AL_CUDA(cudaMemcpyAsync(sv.status, out->status, sizeof(sv.status), cudaMemcpyDeviceToHost, st));
    AL_CUDA(cudaStreamSynchronize(st));
    return AL_OK;
}
int restore_state(al_grid g, const al_step_out *out, const saved_state &sv, cudaStream_t st) {
    int rc = al_set_state(g, sv.fprev, sv.has_prev, st);
    if (rc != AL_OK) return rc;
    if (out && out->status)
        AL_CUDA(cudaMemcpyAsync(out->status, sv.status, sizeof(sv.status), cudaMemcpyHostToDevice, st));
    AL_CUDA(cudaStreamSynchronize(st));
    return AL_OK;
}
struct event_pair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~event_pair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};
}  // namespace

extern "C" int al_autotune(al_grid g, const al_step_in *in, const al_step_out *out, int trials, void *stream,
                           int *choice) {
    if (!g || !in || !out || trials < 1 || trials > 1000) return AL_ERR_ARG;
    if (!g->loaded) return AL_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    saved_state sv;
    int rc = save_state(g, out, sv, st);
    event_pair ev;
    if (rc == AL_OK && (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess))
        rc = AL_ERR_CUDA;
    // every timed step starts with the L2 cold, as a coupled solver leaves it
    // between two calls: a write of twice the L2 before it (none where that
    // buffer cannot be had; the trials are then back to back)
    void *flush = nullptr;
    size_t flush_bytes = 0;
    {
        int dev = 0, l2 = 0;
        if (rc == AL_OK && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess && l2 > 0) {
            flush_bytes = 2 * (size_t)l2;
            if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
                cudaGetLastError();
                flush = nullptr;
            }
        }
    }
    // weights pass and records: brick; segment without records; segment with
    // records (the warm-up step sizes the record regions the timed steps use);
    // the column march on and off where the instance can take it
    const int wms[3] = {AL_WEIGHTS_BRICK, AL_WEIGHTS_SEGMENT, AL_WEIGHTS_SEGMENT}, recs[3] = {0, 0, 1};
    const int bzs[3] = {4, 8, 16};
    const int ncol = g->cmN ? 2 : 1;
    float best = INFINITY;
    int best_w = g->gc.wmode, best_z = g->gc.bz, best_r = g->opt_record, best_c = g->opt_column;
    for (int ci = 0; ci < ncol && rc == AL_OK; ++ci)
        for (int wi = 0; wi < 3 && rc == AL_OK; ++wi)
            for (int zi = 0; zi < 3 && rc == AL_OK; ++zi) {
                g->opt_column = ncol == 2 ? 1 - ci : g->opt_column;
                g->gc.wmode = wms[wi];
                g->opt_record = recs[wi];
                set_brick_z(g->gc, bzs[zi]);
                if ((rc = arena_sync(g)) != AL_OK) break;
                if ((rc = restore_state(g, out, sv, st)) != AL_OK) break;
                if ((rc = al_sample_drag_spread(g, in, out, stream)) != AL_OK) break;       // warm-up
                // the candidate's time: its fastest single step (the least disturbed)
                float ms = INFINITY;
                for (int t = 0; t < trials && rc == AL_OK; ++t) {
                    if (flush && cudaMemsetAsync(flush, t & 0xff, flush_bytes, st) != cudaSuccess) { rc = AL_ERR_CUDA; break; }
                    if (cudaEventRecord(ev.a, st) != cudaSuccess) { rc = AL_ERR_CUDA; break; }
                    if ((rc = al_sample_drag_spread(g, in, out, stream)) != AL_OK) break;
                    if (cudaEventRecord(ev.b, st) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess) {
                        rc = AL_ERR_CUDA;
                        break;
                    }
                    float mt = 0.0f;
                    cudaEventElapsedTime(&mt, ev.a, ev.b);
                    ms = std::min(ms, mt);
                }
                if (rc != AL_OK) break;
                if (ms < best) { best = ms; best_w = wms[wi]; best_z = bzs[zi]; best_r = recs[wi]; best_c = g->opt_column; }
            }
    g->opt_column = best_c;
    g->gc.wmode = best_w;
    g->opt_record = best_r;
    set_brick_z(g->gc, best_z);
    int rc2 = arena_sync(g);                          // the arena only if the choice records
    if (rc2 == AL_OK) rc2 = restore_state(g, out, sv, st);
    if (sv.fprev) cudaFree(sv.fprev);
    if (flush) cudaFree(flush);
    if (rc == AL_OK) rc = rc2;
    if (rc == AL_OK && choice) *choice = 10000 * best_c + 1000 * best_r + 100 * best_w + best_z;
    return rc;
}

extern "C" int al_batch_set_option(al_batch b, int option, int value) {
    if (!b) return AL_ERR_ARG;
    if (!b->committed) return AL_ERR_STATE;
    switch (option) {
    case AL_OPT_BRICK_Z:
        if (value != 4 && value != 8 && value != 16) return AL_ERR_ARG;
        b->bz = value;
        break;
    case AL_OPT_SPREAD_CTAS:
        if (value < 0 || value > 32) return AL_ERR_ARG;
        b->ctas = value;
        break;
    default:
        return AL_ERR_ARG;
    }
    return b->precision == AL_FP64 ? batch_rebuild_t<double>(b) : batch_rebuild_t<float>(b);
}

extern "C" int al_batch_autotune(al_batch b, int trials, void *stream, int *choice) {
    if (!b || trials < 1 || trials > 1000) return AL_ERR_ARG;
    if (!b->committed) return AL_ERR_STATE;
    for (int q = 0; q < b->n; ++q)
        if (!b->grids[q]) return AL_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<saved_state> sv(b->n);
    int rc = AL_OK;
    for (int q = 0; q < b->n && rc == AL_OK; ++q) rc = save_state(b->grids[q], &b->outs[q], sv[q], st);
    event_pair ev;
    if (rc == AL_OK && (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess))
        rc = AL_ERR_CUDA;
    const int bzs[3] = {4, 8, 16}, ctas[2] = {0, 1};
    float best = INFINITY;
    int best_z = b->bz, best_c = b->ctas;
    for (int zi = 0; zi < 3 && rc == AL_OK; ++zi)
        for (int ci = 0; ci < 2 && rc == AL_OK; ++ci) {
            b->bz = bzs[zi];
            b->ctas = ctas[ci];
            rc = b->precision == AL_FP64 ? batch_rebuild_t<double>(b) : batch_rebuild_t<float>(b);
            if (rc != AL_OK) break;
            if (ctas[ci] == 1 && b->occ == 1) continue;       // the same launch as "as many as fit"
            for (int q = 0; q < b->n && rc == AL_OK; ++q) rc = restore_state(b->grids[q], &b->outs[q], sv[q], st);
            if (rc != AL_OK || (rc = al_batch_run(b, stream)) != AL_OK) break;        // warm-up (and capture)
            if (cudaEventRecord(ev.a, st) != cudaSuccess) { rc = AL_ERR_CUDA; break; }
            for (int t = 0; t < trials && rc == AL_OK; ++t) rc = al_batch_run(b, stream);
            if (rc != AL_OK) break;
            if (cudaEventRecord(ev.b, st) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess) {
                rc = AL_ERR_CUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, ev.a, ev.b);
            if (ms < best) { best = ms; best_z = bzs[zi]; best_c = ctas[ci]; }
        }
    b->bz = best_z;
    b->ctas = best_c;
    int rc2 = b->precision == AL_FP64 ? batch_rebuild_t<double>(b) : batch_rebuild_t<float>(b);
    for (int q = 0; q < b->n; ++q) {
        const int r = restore_state(b->grids[q], &b->outs[q], sv[q], st);
        if (rc2 == AL_OK) rc2 = r;
        if (sv[q].fprev) cudaFree(sv[q].fprev);
    }
    if (rc == AL_OK) rc = rc2;
    if (rc == AL_OK && choice) *choice = 10 * best_z + best_c;
    return rc;
}

extern "C" int al_batch_launches(al_batch b, long long *n) {
    if (!b || !n) return AL_ERR_ARG;
    *n = b->launches;
    return AL_OK;
}

extern "C" int al_launches(al_grid g, long long *n) {
    if (!g || !n) return AL_ERR_ARG;
    *n = g->launches;
    return AL_OK;
}

// ---------------------------------------------------------------------------
// slab plan of a decomposition along x (host logic)
// ---------------------------------------------------------------------------
extern "C" int al_slab_plan(const al_grid_desc *grid, const al_beam_desc *beams, const double *P_host, int n_ranks,
                            int rank, al_slab *out, int *lines, int *owner) {
    if (!grid || !beams || !out || n_ranks < 1 || rank < 0 || rank >= n_ranks) return AL_ERR_ARG;
    if (grid->nx < 1 || !(grid->dx > 0.0) || beams->n_lines < 0) return AL_ERR_ARG;
    int np = 0;
    const int rc = al_detail_check_beams(*beams, *grid, &np);
    if (rc != AL_OK) return rc;
    if (np > 0 && !P_host) return AL_ERR_ARG;
    const double h = grid->dx, ox = grid->origin[0];
    const int nbx = (grid->nx + al::BX - 1) / al::BX;
    const int bx0 = (int)((long long)rank * nbx / n_ranks), bx1 = (int)((long long)(rank + 1) * nbx / n_ranks);
    out->x0 = std::min(bx0 * al::BX, grid->nx);
    out->x1 = std::min(bx1 * al::BX, grid->nx);
    // per line: x range of its points and its reach 3 eps + L (longest segment)
    double need = 0.0;
    std::vector<double> lo(beams->n_lines), hi(beams->n_lines), reach(beams->n_lines);
    for (int l = 0; l < beams->n_lines; ++l) {
        const int a = beams->line_off[l], b = beams->line_off[l + 1];
        double mn = INFINITY, mx = -INFINITY, L = 0.0;
        for (int i = a; i < b; ++i) {
            mn = std::min(mn, P_host[i]);
            mx = std::max(mx, P_host[i]);
            if (i + 1 < b) {
                double d2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    const double d = P_host[(size_t)c * np + i + 1] - P_host[(size_t)c * np + i];
                    d2 += d * d;
                }
                L = std::max(L, std::sqrt(d2));
            }
        }
        lo[l] = mn; hi[l] = mx;
        reach[l] = 3.0 * beams->eps[l] + L;
        need = std::max(need, beams->ell_s[l] + reach[l]);
    }
    int halo = (int)std::ceil(need / h) + 2;
    halo = (halo + al::BX - 1) / al::BX * al::BX;
    out->halo = halo;
    out->lx0 = std::max(0, out->x0 - halo);
    out->lx1 = std::min(grid->nx, out->x1 + halo);
    const double X0 = ox + out->x0 * h, X1 = ox + out->x1 * h;
    int n = 0;
    for (int l = 0; l < beams->n_lines; ++l) {
        if (beams->line_off[l + 1] == beams->line_off[l]) continue;
        const double r = reach[l] + h;
        if (hi[l] + r >= X0 && lo[l] - r < X1 && out->x1 > out->x0) {
            if (lines) lines[n] = l;
            ++n;
        }
    }
    out->n_lines = n;
    if (owner)
        for (int i = 0; i < np; ++i) {
            long long c = (long long)std::floor((P_host[i] - ox) / h);
            c = std::max(0ll, std::min((long long)grid->nx - 1, c));
            int r = 0;
            while (r + 1 < n_ranks && c >= std::min((long long)((long long)(r + 1) * nbx / n_ranks) * al::BX,
                                                    (long long)grid->nx))
                ++r;
            owner[i] = r;
        }
    return AL_OK;
}
