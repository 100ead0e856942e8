// al_noalloc.cu -- line forces without any device allocation.
//
// al_line_forces_noalloc evaluates the per-CV line loads F = f L of every
// actuator point (sampling, upstream direction, Morison drag with the
// optional inertia term, optional relaxation against a caller-supplied
// previous force) with the same point evaluation as al_sample_drag_spread,
// but needs no al_grid and allocates nothing.  It serves callers that cannot
// call cudaMalloc where they need the forces: code running under an
// allocator that forbids device allocation after start-up (a fixed,
// pre-reserved memory pool, a real-time loop where an allocation's latency
// and possible implicit synchronisation are not acceptable), or a plug-in
// whose host application owns all device memory and hands it only buffers.
// Those callers pass every input and output buffer themselves; the line
// table the kernel reads on the device is copied into one file-scope
// __device__ array of fixed size (below), so the only device memory the call
// touches besides the caller's buffers is that array.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Calls whose work overlaps on the GPU (different streams without
// ordering between them) race on it; callers serialise them.
#include "al.h"
#include "al_kernels.cuh"

#include <cmath>
#include <cstdio>
#include <mutex>

// shared with al_api.cu: descriptor checks of al_load_beams, and the CUDA
// error text that al_last_cuda_error returns
int al_detail_check_beams(const al_beam_desc &b, const al_grid_desc &gd, int *np_out);
int al_detail_cuda_fail(cudaError_t e, const char *what);

namespace {

using namespace al;

// ---- the static scratch: line table, per-line coefficients, counters ----
constexpr size_t al_align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t NA_OFF_LINE_OFF = 0;
constexpr size_t NA_OFF_LINE_OF = al_align256(NA_OFF_LINE_OFF + (AL_NOALLOC_MAX_LINES + 1) * sizeof(int));
constexpr size_t NA_OFF_COEF = al_align256(NA_OFF_LINE_OF + AL_NOALLOC_MAX_POINTS * sizeof(int));
constexpr int NA_NCOEF = 8;   // d, cdn, cdt, eps, ell_s, alpha_f, cm_n, cm_t per line
constexpr size_t NA_OFF_CVLEN = al_align256(NA_OFF_COEF + NA_NCOEF * AL_NOALLOC_MAX_LINES * sizeof(double));
constexpr size_t NA_OFF_STATUS = al_align256(NA_OFF_CVLEN + AL_NOALLOC_MAX_POINTS * sizeof(double));
constexpr size_t NA_BYTES = al_align256(NA_OFF_STATUS + AL_STATUS_N * sizeof(int));

static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

// Device address of g_na_scratch, looked up once per device with that device
// current.  In host code the name g_na_scratch is only a host-side stand-in
// for the symbol, never a device address.
std::mutex g_na_mu;
constexpr int NA_MAX_DEVICES = 64;
void *g_na_addr[NA_MAX_DEVICES] = {};

int na_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return al_detail_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= NA_MAX_DEVICES) return AL_ERR_CAPACITY;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return al_detail_cuda_fail(e, "cudaGetSymbolAddress");
        if (!p) return al_detail_cuda_fail(cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
        g_na_addr[dev] = p;
    }
    *out = g_na_addr[dev];
    return AL_OK;
}

// line id of every point (one thread per line)
__global__ void k_na_line_of(const int *line_off, int n_lines, int *line_of) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_lines) return;
    for (int i = line_off[l]; i < line_off[l + 1]; ++i) line_of[i] = l;
}

// the point kernel's force evaluation, with the previous force supplied by
// the caller (or none) instead of the instance state
template <typename T>
__global__ void __launch_bounds__(256) k_na_points(GridC g, BeamsC b, StepPtrs<T> p, const T *fp0, const T *fp1,
                                                   const T *fp2, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n_points) return;
    const int l = b.line_of[i];
    const int off = b.line_off[l], n = b.line_off[l + 1] - off, q = i - off;
    T Pa[3], Pd[3], t[3];
    for (int a = 0; a < 3; ++a) { Pa[a] = p.P[a][i]; Pd[a] = p.Pdot[a][i]; }
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
    T ab[3] = {(T)0, (T)0, (T)0};                  // beam acceleration of the inertia term
    if (b.inertia && p.Pdd[0])
        for (int a = 0; a < 3; ++a) ab[a] = p.Pdd[a][i];
    if (point_fstar<T, T>(g, b, p, l, Pa, Pd, t, fstar, status, sizeof(T) == 4, ab)) {
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
        point_fstar<T, double>(g, b, p, l, Pa64, Pd64, t64, f64, status, false, ab64);
        for (int a = 0; a < 3; ++a) fstar[a] = (T)f64[a];
        atomicAdd(&status[ST_REFINED], 1);
    }
    const T af = (T)b.alpha_f[l];
    const T L = (T)b.cv_len[i];
    const T *fp[3] = {fp0, fp1, fp2};
    for (int a = 0; a < 3; ++a) {
        T f = fp0 ? af * fstar[a] + ((T)1 - af) * fp[a][i] : fstar[a];
        p.F[a][i] = f * L;
    }
}

template <typename T>
int na_launch(const al_grid_desc &d, const al_beam_desc &bd, const al_step_in &in, const void *const *f_prev,
              void *const *F, int *status, unsigned char *scr, cudaStream_t st) {
    GridC g{};
    g.nx = d.nx; g.ny = d.ny; g.nz = d.nz;
    g.ncell = (long long)d.nx * d.ny * d.nz;
    g.h = d.dx;
    g.V = d.dx * d.dx * d.dx;
    for (int a = 0; a < 3; ++a) {
        g.o[a] = d.origin[a];
        g.o_hi[a] = (float)d.origin[a];
        g.o_lo[a] = (float)(d.origin[a] - (double)g.o_hi[a]);
    }
    g.ih_hi = (float)(1.0 / d.dx);
    g.ih_lo = (float)(1.0 / d.dx - (double)g.ih_hi);
    g.has_alpha = d.has_alpha ? 1 : 0;
    g.rho1 = d.rho1; g.rho2 = d.rho2; g.rho_const = d.rho_const;

    const int nl = bd.n_lines, np = nl > 0 ? bd.line_off[nl] : 0;
    int *line_off = (int *)(scr + NA_OFF_LINE_OFF);
    int *line_of = (int *)(scr + NA_OFF_LINE_OF);
    double *coef = (double *)(scr + NA_OFF_COEF);
    double *cvl = (double *)(scr + NA_OFF_CVLEN);
    int *st_int = (int *)(scr + NA_OFF_STATUS);
    cudaError_t e;
#define NA_CHECK(call)                                                                         \
    if ((e = (call)) != cudaSuccess) return al_detail_cuda_fail(e, #call);
    if (!status) {                                // the shared counters start at zero every call
        NA_CHECK(cudaMemsetAsync(st_int, 0, AL_STATUS_N * sizeof(int), st));
        status = st_int;
    }
    if (np == 0) return AL_OK;                    // nothing to evaluate (no lines, or lines of no points)
    const bool inertia = bd.cm_n != nullptr;
    NA_CHECK(cudaMemcpyAsync(line_off, bd.line_off, (nl + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    const double *src[NA_NCOEF] = {bd.d, bd.cdn, bd.cdt, bd.eps, bd.ell_s, bd.alpha_f, bd.cm_n, bd.cm_t};
    for (int c = 0; c < NA_NCOEF; ++c)
        if (src[c])
            NA_CHECK(cudaMemcpyAsync(coef + (size_t)c * AL_NOALLOC_MAX_LINES, src[c], nl * sizeof(double),
                                     cudaMemcpyHostToDevice, st));
    NA_CHECK(cudaMemcpyAsync(cvl, bd.cv_len, np * sizeof(double), cudaMemcpyHostToDevice, st));
    k_na_line_of<<<(nl + 255) / 256, 256, 0, st>>>(line_off, nl, line_of);

    BeamsC b{};
    b.n_lines = nl; b.n_points = np; b.mask_words = 0;
    b.line_off = line_off; b.line_of = line_of;
    b.d = coef; b.cdn = coef + AL_NOALLOC_MAX_LINES; b.cdt = coef + 2 * AL_NOALLOC_MAX_LINES;
    b.eps = coef + 3 * AL_NOALLOC_MAX_LINES; b.ell_s = coef + 4 * AL_NOALLOC_MAX_LINES;
    b.alpha_f = coef + 5 * AL_NOALLOC_MAX_LINES; b.cv_len = cvl;
    b.cm_n = inertia ? coef + 6 * AL_NOALLOC_MAX_LINES : nullptr;
    b.cm_t = inertia ? coef + 7 * AL_NOALLOC_MAX_LINES : nullptr;
    b.inertia = inertia ? 1 : 0;
    for (int a = 0; a < 3; ++a) { b.n_p[a] = bd.n_p[a]; b.g_up[a] = bd.g_up[a]; }
    b.tau = bd.tau; b.sample_mode = bd.sample_mode; b.drag_mode = bd.drag_mode;
    b.tangents_given = bd.tangents_given;

    StepPtrs<T> p{};
    for (int a = 0; a < 3; ++a) {
        p.U[a] = (const T *)in.U[a];
        p.P[a] = (const T *)in.P[a];
        p.Pdot[a] = (const T *)in.Pdot[a];
        p.Ps[a] = p.P[a];
        p.tan[a] = (const T *)in.tangent[a];
        p.F[a] = (T *)F[a];
    }
    p.alpha = (const T *)in.alpha;
    p.np = np;
    for (int a = 0; a < 3; ++a) {                 // the inertia term's inputs (ignored without it)
        p.Uprev[a] = inertia ? (const T *)in.U_prev[a] : nullptr;
        p.Pdd[a] = inertia ? (const T *)in.Pddot[a] : nullptr;
    }
    p.dt = in.dt;
    const T *fp[3] = {nullptr, nullptr, nullptr};
    if (f_prev)
        for (int a = 0; a < 3; ++a) fp[a] = (const T *)f_prev[a];
    k_na_points<T><<<(np + 255) / 256, 256, 0, st>>>(g, b, p, fp[0], fp[1], fp[2], status);
    NA_CHECK(cudaGetLastError());
#undef NA_CHECK
    return AL_OK;
}

}  // namespace

extern "C" int al_line_forces_noalloc(const al_grid_desc *grid, const al_beam_desc *beams, const al_step_in *in,
                                      const void *const f_prev[3], void *const F[3], int *status, void *stream) {
    if (!grid || !beams || !in || !F) return AL_ERR_ARG;
    const al_grid_desc &d = *grid;
    const al_beam_desc &b = *beams;
    // host-side validation: the grid rules of al_create_grid, the descriptor
    // rules of al_load_beams, the capacity of the fixed array
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || !(d.dx > 0.0) || !std::isfinite(d.dx)) return AL_ERR_ARG;
    if ((long long)d.nx * d.ny * d.nz > (1LL << 40)) return AL_ERR_ARG;
    if (d.precision != AL_FP32 && d.precision != AL_FP64) return AL_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(d.origin[a])) return AL_ERR_ARG;
    if (d.has_alpha ? (!(d.rho1 > 0.0) || !(d.rho2 > 0.0) || !in->alpha) : !(d.rho_const > 0.0)) return AL_ERR_ARG;
    if (b.n_lines > AL_NOALLOC_MAX_LINES) return AL_ERR_CAPACITY;
    int np = 0;
    {
        const int rc = al_detail_check_beams(b, d, &np);
        if (rc != AL_OK) return rc;
    }
    // the volume-average sampler reads the kernel widths of an al_grid's
    // line table per cell; this entry point offers the two local samplers
    if (b.sample_mode == AL_SAMPLE_GAUSS) return AL_ERR_ARG;
    if (np > AL_NOALLOC_MAX_POINTS) return AL_ERR_CAPACITY;
    if (np > 0) {
        for (int a = 0; a < 3; ++a) {
            if (!in->U[a] || !in->P[a] || !in->Pdot[a] || !F[a]) return AL_ERR_ARG;
            if (b.tangents_given && !in->tangent[a]) return AL_ERR_ARG;
            if (f_prev && !f_prev[a]) return AL_ERR_ARG;
        }
        if (b.cm_n) {                              // inertia term: all three or none of each
            const bool up = in->U_prev[0] != nullptr, pa = in->Pddot[0] != nullptr;
            for (int a = 1; a < 3; ++a)
                if ((in->U_prev[a] != nullptr) != up || (in->Pddot[a] != nullptr) != pa) return AL_ERR_ARG;
            if (up && !(in->dt > 0.0 && std::isfinite(in->dt))) return AL_ERR_ARG;
        }
    }
    void *scr = nullptr;
    int rc = na_scratch(&scr);
    if (rc != AL_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    return d.precision == AL_FP64
               ? na_launch<double>(d, b, *in, f_prev, F, status, (unsigned char *)scr, st)
               : na_launch<float>(d, b, *in, f_prev, F, status, (unsigned char *)scr, st);
}
