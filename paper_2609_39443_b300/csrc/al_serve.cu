// al_serve.cu -- continuous batching of coupling-step requests (al_server_*).
//
// Many simulations send coupling-step requests (the actuator-point positions
// of their next step) as they arrive.  The server keeps each admitted
// simulation resident: its instance (library scratch: line table, relaxation
// state, geometry, masks) bound to a slot of one batch, with the caller's
// device fields and outputs.  Simulations are admitted while their device
// bytes (al_footprint of the instance plus the bytes the caller declares for
// its own buffers) fit the budget and a slot is free.  Every poll retires
// the waves that completed and launches one wave: every resident simulation
// with a queued request and no step in flight, advanced together by one
// batched launch sequence (al_batch_run_subset).  Waves alternate between
// two streams, so a wave forms and launches while the previous one runs; a
// simulation's requests run in submission order, one at a time.
//
// Copies per wave: the requests' positions are packed on the host into one
// pinned staging buffer, copied to the device in one transfer and scattered
// into each simulation's position arrays by one kernel; the line forces are
// gathered by one kernel into a device staging buffer and copied back in one
// transfer, then unpacked into each request's host buffer when the wave is
// retired.  The paper's counterpart is the per-step call of Algorithm 1; the
// server adds nothing to the arithmetic of a step (a served step has the
// bits of the same step run alone).
#include "al.h"
#include "al_kernels.cuh"

#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <thread>
#include <vector>

int al_detail_cuda_fail(cudaError_t e, const char *what);

namespace {

#define SV_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return al_detail_cuda_fail(e_, #call);   \
    } while (0)

// one simulation's segment of a wave's staging buffer
struct WaveItem {
    void *P[3];           // the simulation's device positions
    const void *F[3];     // its device line forces
    long long off;        // element offset of its 3 x n values in the staging buffers
    int n;                // actuator points
    int pad;
};

// staging buffers -> the simulations' positions (one CTA row per item)
template <typename T>
__global__ void __launch_bounds__(256) k_sv_scatter(const WaveItem *items, int n_items, const T *src) {
    const int it = blockIdx.y;
    if (it >= n_items) return;
    const WaveItem w = items[it];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * w.n; i += gridDim.x * blockDim.x) {
        const int a = i / w.n, k = i - a * w.n;
        static_cast<T *>(w.P[a])[k] = src[w.off + i];
    }
}
// the simulations' line forces -> staging buffer
template <typename T>
__global__ void __launch_bounds__(256) k_sv_gather(const WaveItem *items, int n_items, T *dst) {
    const int it = blockIdx.y;
    if (it >= n_items) return;
    const WaveItem w = items[it];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * w.n; i += gridDim.x * blockDim.x) {
        const int a = i / w.n, k = i - a * w.n;
        dst[w.off + i] = static_cast<const T *>(w.F[a])[k];
    }
}

struct Req {
    const void *P_host;
    void *F_host;
    long long tag;
};

struct Sim {
    bool used = false;
    al_grid g = nullptr;
    al_step_in in{};
    al_step_out out{};
    int n_points = 0;
    unsigned long long bytes = 0;     // footprint + caller bytes
    std::deque<Req> queue;
    bool busy = false;                // a step in flight
    bool releasing = false;
};

struct Wave {
    bool live = false;
    cudaEvent_t ev = nullptr;
    std::vector<int> sims;
    std::vector<Req> reqs;
    std::vector<long long> offs;
};

}  // namespace

struct al_server_s {
    al_server_desc d{};
    size_t es = 4;
    al_batch batch = nullptr;
    std::vector<Sim> sims;
    unsigned long long used = 0;
    cudaStream_t st[2] = {nullptr, nullptr};
    // per stream: pinned host staging (positions in, forces out, wave items) and device staging
    void *hP[2] = {nullptr, nullptr}, *hF[2] = {nullptr, nullptr}, *hI[2] = {nullptr, nullptr};
    void *dP[2] = {nullptr, nullptr}, *dF[2] = {nullptr, nullptr}, *dI[2] = {nullptr, nullptr};
    Wave wave[2];
    int next_stream = 0;
    int rr = 0;                       // round-robin start of wave formation
    std::vector<long long> done;      // tags completed, not yet reported
    long long n_waves = 0, n_wave_steps = 0;   // waves launched, steps they carried
    double wait_s = 10.0;             // limit of a wait for a wave (al_server_set_timeout)
};

// wait for a wave's event, polling, for at most limit_s seconds: AL_ERR_TIMEOUT
// when it runs out (the wave stays in flight)
static int sv_wait(cudaEvent_t ev, double limit_s) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess) return AL_OK;
        if (q != cudaErrorNotReady) return al_detail_cuda_fail(q, "cudaEventQuery");
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >= limit_s)
            return AL_ERR_TIMEOUT;
        std::this_thread::yield();
    }
}

static size_t sv_stage_elems(const al_server_desc &d) { return 3 * (size_t)d.max_points; }

extern "C" int al_server_create(const al_server_desc *d, al_server *out) {
    if (!d || !out) return AL_ERR_ARG;
    *out = nullptr;
    if (d->max_sims < 1 || d->max_sims > 65536 || d->max_wave < 1 || d->max_wave > d->max_sims ||
        d->max_points < 1 || (d->precision != AL_FP32 && d->precision != AL_FP64))
        return AL_ERR_ARG;
    al_server s = new (std::nothrow) al_server_s();
    if (!s) return AL_ERR_OOM;
    s->d = *d;
    s->es = d->precision == AL_FP64 ? 8 : 4;
    s->sims.resize(d->max_sims);
    int rc = al_batch_create(&s->batch);
    if (rc == AL_OK) rc = al_batch_reserve(s->batch, d->max_sims, d->precision);
    if (rc == AL_OK) rc = al_batch_commit(s->batch, 0, 0);
    const size_t bytes = sv_stage_elems(*d) * s->es;
    const size_t ibytes = (size_t)d->max_wave * sizeof(WaveItem);
    for (int k = 0; k < 2 && rc == AL_OK; ++k) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->st[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->wave[k].ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&s->hP[k], bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&s->hF[k], bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&s->hI[k], ibytes);
        if (e == cudaSuccess) e = cudaMalloc(&s->dP[k], bytes);
        if (e == cudaSuccess) e = cudaMalloc(&s->dF[k], bytes);
        if (e == cudaSuccess) e = cudaMalloc(&s->dI[k], ibytes);
        if (e != cudaSuccess) rc = al_detail_cuda_fail(e, "al_server_create");
    }
    if (rc != AL_OK) {
        al_server_destroy(s);
        return rc;
    }
    *out = s;
    return AL_OK;
}

extern "C" int al_server_admit(al_server s, const al_grid_desc *grid, const al_beam_desc *beams, const al_step_in *in,
                               const al_step_out *out, unsigned long long caller_bytes, int *sim) {
    if (!s || !grid || !beams || !in || !out || !sim) return AL_ERR_ARG;
    if (grid->precision != s->d.precision) return AL_ERR_ARG;
    int slot = -1;
    for (int k = 0; k < (int)s->sims.size(); ++k)
        if (!s->sims[k].used) { slot = k; break; }
    if (slot < 0) return AL_ERR_CAPACITY;
    if (s->used + caller_bytes > s->d.hbm_budget) return AL_ERR_CAPACITY;
    al_grid g = nullptr;
    int rc = al_create_grid(grid, &g);
    if (rc != AL_OK) return rc;
    rc = al_load_beams(g, beams);
    long long nc = 0, np = 0;
    int nl = 0;
    unsigned long long fp = 0;
    if (rc == AL_OK) rc = al_sizes(g, &nc, &np, &nl);
    if (rc == AL_OK) rc = al_footprint(g, &fp);
    if (rc == AL_OK && np > s->d.max_points) rc = AL_ERR_CAPACITY;
    if (rc == AL_OK && s->used + fp + caller_bytes > s->d.hbm_budget) rc = AL_ERR_CAPACITY;
    if (rc == AL_OK) rc = al_batch_assign(s->batch, slot, g, in, out, s->st[0]);
    if (rc == AL_OK) SV_CUDA(cudaStreamSynchronize(s->st[0]));      // every stream sees the slot's descriptor
    if (rc != AL_OK) {
        al_destroy(g);
        return rc;
    }
    Sim &m = s->sims[slot];
    m.used = true;
    m.g = g;
    m.in = *in;
    m.out = *out;
    m.n_points = (int)np;
    m.bytes = fp + caller_bytes;
    m.busy = false;
    m.releasing = false;
    m.queue.clear();
    s->used += m.bytes;
    *sim = slot;
    return AL_OK;
}

extern "C" int al_server_submit(al_server s, int sim, const void *P_host, void *F_host, long long tag) {
    if (!s || sim < 0 || sim >= (int)s->sims.size() || !s->sims[sim].used || s->sims[sim].releasing) return AL_ERR_ARG;
    Sim &m = s->sims[sim];
    if (m.n_points > 0 && (!P_host || !F_host)) return AL_ERR_ARG;
    m.queue.push_back(Req{P_host, F_host, tag});
    return AL_OK;
}

// retire wave k if it completed (or wait for it): unpack the forces
static int sv_retire(al_server s, int k, bool wait) {
    Wave &w = s->wave[k];
    if (!w.live) return AL_OK;
    if (wait) {
        const int rc = sv_wait(w.ev, s->wait_s);
        if (rc != AL_OK) return rc;
    } else {
        const cudaError_t q = cudaEventQuery(w.ev);
        if (q == cudaErrorNotReady) return AL_OK;
        if (q != cudaSuccess) return al_detail_cuda_fail(q, "cudaEventQuery");
    }
    const char *src = (const char *)s->hF[k];
    for (size_t i = 0; i < w.sims.size(); ++i) {
        Sim &m = s->sims[w.sims[i]];
        if (m.n_points > 0)
            std::memcpy(w.reqs[i].F_host, src + (size_t)w.offs[i] * s->es, 3 * (size_t)m.n_points * s->es);
        m.busy = false;
        s->done.push_back(w.reqs[i].tag);
    }
    w.live = false;
    w.sims.clear();
    w.reqs.clear();
    w.offs.clear();
    return AL_OK;
}

template <typename T>
static int sv_launch(al_server s, int k) {
    Wave &w = s->wave[k];
    const int n = (int)w.sims.size();
    cudaStream_t st = s->st[k];
    WaveItem *hi = (WaveItem *)s->hI[k];
    T *hp = (T *)s->hP[k];
    std::vector<int> slots(n);
    int nmax = 1;
    for (int i = 0; i < n; ++i) {
        const Sim &m = s->sims[w.sims[i]];
        slots[i] = w.sims[i];
        WaveItem it{};
        for (int a = 0; a < 3; ++a) {
            it.P[a] = const_cast<void *>(m.in.P[a]);
            it.F[a] = m.out.F[a];
        }
        it.off = w.offs[i];
        it.n = m.n_points;
        hi[i] = it;
        if (m.n_points > 0) std::memcpy(hp + w.offs[i], w.reqs[i].P_host, 3 * (size_t)m.n_points * sizeof(T));
        nmax = std::max(nmax, m.n_points);
    }
    const long long tot = n > 0 ? w.offs[n - 1] + 3 * (long long)s->sims[w.sims[n - 1]].n_points : 0;
    SV_CUDA(cudaMemcpyAsync(s->dI[k], hi, (size_t)n * sizeof(WaveItem), cudaMemcpyHostToDevice, st));
    if (tot > 0) SV_CUDA(cudaMemcpyAsync(s->dP[k], hp, (size_t)tot * sizeof(T), cudaMemcpyHostToDevice, st));
    const dim3 grid((unsigned)std::min(64, (3 * nmax + 255) / 256), (unsigned)n);
    k_sv_scatter<T><<<grid, 256, 0, st>>>((const WaveItem *)s->dI[k], n, (const T *)s->dP[k]);
    int rc = al_batch_run_subset(s->batch, slots.data(), n, st);
    if (rc != AL_OK) return rc;
    k_sv_gather<T><<<grid, 256, 0, st>>>((const WaveItem *)s->dI[k], n, (T *)s->dF[k]);
    if (tot > 0) SV_CUDA(cudaMemcpyAsync(s->hF[k], s->dF[k], (size_t)tot * sizeof(T), cudaMemcpyDeviceToHost, st));
    SV_CUDA(cudaGetLastError());
    SV_CUDA(cudaEventRecord(w.ev, st));
    w.live = true;
    return AL_OK;
}

extern "C" int al_server_poll(al_server s, long long *done_tags, int max_done, int *n_done, int wait) {
    if (!s || !n_done || max_done < 0 || (max_done > 0 && !done_tags)) return AL_ERR_ARG;
    *n_done = 0;
    // retire completed waves (waiting for the oldest when asked and nothing else can happen)
    for (int k = 0; k < 2; ++k) {
        const int rc = sv_retire(s, k, false);
        if (rc != AL_OK) return rc;
    }
    // a wave on each free stream: each resident simulation with a queued
    // request and none in flight (the second wave takes what the first left)
    const int k0 = s->next_stream;
    for (int t = 0; t < 2; ++t) {
        const int k = (k0 + t) & 1;
        if (s->wave[k].live) continue;
        Wave &w = s->wave[k];
        const int ns = (int)s->sims.size();
        long long off = 0;
        for (int u = 0; u < ns && (int)w.sims.size() < s->d.max_wave; ++u) {
            const int q = (s->rr + u) % ns;
            Sim &m = s->sims[q];
            if (!m.used || m.busy || m.queue.empty()) continue;
            if (off + 3 * (long long)m.n_points > 3 * (long long)s->d.max_points) continue;   // staging full
            w.sims.push_back(q);
            w.reqs.push_back(m.queue.front());
            w.offs.push_back(off);
            m.queue.pop_front();
            m.busy = true;
            off += 3 * (long long)m.n_points;
        }
        if (w.sims.empty()) break;
        s->rr = (w.sims.back() + 1) % ns;
        const int rc = s->d.precision == AL_FP64 ? sv_launch<double>(s, k) : sv_launch<float>(s, k);
        if (rc != AL_OK) return rc;
        ++s->n_waves;
        s->n_wave_steps += (long long)w.sims.size();
        s->next_stream = k ^ 1;
    }
    if (wait && s->done.empty()) {
        // nothing completed yet: wait for the oldest wave in flight
        const int first = s->next_stream;          // launched before the newest
        for (int t = 0; t < 2 && s->done.empty(); ++t) {
            const int rc = sv_retire(s, (first + t) & 1, true);
            if (rc != AL_OK) return rc;
        }
    }
    const int m = std::min<int>(max_done, (int)s->done.size());
    for (int i = 0; i < m; ++i) done_tags[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + m);
    *n_done = m;
    return AL_OK;
}

extern "C" int al_server_release(al_server s, int sim) {
    if (!s || sim < 0 || sim >= (int)s->sims.size() || !s->sims[sim].used) return AL_ERR_ARG;
    Sim &m = s->sims[sim];
    m.releasing = true;
    for (int k = 0; k < 2; ++k) {                   // its step in flight, and its results
        bool mine = false;
        for (int q : s->wave[k].sims) mine = mine || q == sim;
        if (mine) {
            const int rc = sv_retire(s, k, true);
            if (rc != AL_OK) {
                m.releasing = false;                // still resident; the caller may retry
                return rc;
            }
        }
    }
    if (!m.queue.empty()) {
        m.releasing = false;
        return AL_ERR_STATE;                        // queued requests would be lost
    }
    int rc = al_batch_assign(s->batch, sim, nullptr, nullptr, nullptr, s->st[0]);
    if (rc == AL_OK) SV_CUDA(cudaStreamSynchronize(s->st[0]));
    if (rc != AL_OK) return rc;
    rc = al_destroy(m.g);
    s->used -= m.bytes;
    m = Sim();
    return rc;
}

extern "C" int al_server_footprint(al_server s, unsigned long long *bytes, int *resident) {
    if (!s || !bytes) return AL_ERR_ARG;
    *bytes = s->used;
    if (resident) {
        int r = 0;
        for (const Sim &m : s->sims) r += m.used ? 1 : 0;
        *resident = r;
    }
    return AL_OK;
}

extern "C" int al_server_stats(al_server s, long long *waves, long long *steps) {
    if (!s || !waves || !steps) return AL_ERR_ARG;
    *waves = s->n_waves;
    *steps = s->n_wave_steps;
    return AL_OK;
}

extern "C" int al_server_set_timeout(al_server s, double seconds) {
    if (!s || !(seconds >= 0.0) || !(seconds <= 1e6)) return AL_ERR_ARG;
    s->wait_s = seconds;
    return AL_OK;
}

extern "C" int al_server_destroy(al_server s) {
    if (!s) return AL_ERR_ARG;
    cudaDeviceSynchronize();
    for (Sim &m : s->sims)
        if (m.used && m.g) al_destroy(m.g);
    if (s->batch) al_batch_destroy(s->batch);
    for (int k = 0; k < 2; ++k) {
        if (s->wave[k].ev) cudaEventDestroy(s->wave[k].ev);
        if (s->st[k]) cudaStreamDestroy(s->st[k]);
        if (s->hP[k]) cudaFreeHost(s->hP[k]);
        if (s->hF[k]) cudaFreeHost(s->hF[k]);
        if (s->hI[k]) cudaFreeHost(s->hI[k]);
        if (s->dP[k]) cudaFree(s->dP[k]);
        if (s->dF[k]) cudaFree(s->dF[k]);
        if (s->dI[k]) cudaFree(s->dI[k]);
    }
    delete s;
    return AL_OK;
}
