// server.cu -- continuous-batching request loop for many concurrent Langevin
// trajectories (different N, density, temperature) on one GPU.
//
// A trajectory is a qmc_system handle (its walkers stay resident in HBM between
// MD steps) plus its own CUDA stream and pinned host buffers.  A request is one
// MD step of one trajectory: an energy/force/covariance evaluation at the
// trajectory's current nuclei followed by the accelerated Langevin step.
//   * Requests of a trajectory run in submission order, one at a time.
//   * Up to max_active requests run at once, each on its trajectory's stream,
//     so their kernels overlap on the device; a request that arrives while
//     others run is admitted as soon as a slot and memory are free
//     (qmc_server_progress, called by the host loop, never blocks).
//   * Admission is by device-memory footprint against a budget.  To make room,
//     idle resident trajectories are evicted least-recently-used first: their
//     sampler and MD state go to host memory (qmc_checkpoint_save) and come back
//     on re-admission, so a result does not depend on evictions or on which
//     other requests ran alongside it.
//   * The budget is one device arena allocated when the server is created; a
//     trajectory's handle is carved from one block of it (first fit), so
//     admission and eviction call no cudaMalloc / cudaFree (which may
//     synchronise the device and stall the requests in flight).  Streams and
//     pinned buffers are made when a trajectory is added, events when a
//     request is submitted; qmc_server_progress itself only launches, queries
//     events and moves checkpoints.
//   * Every request records a start and an end event on its stream, so the
//     device-side interval of each request is reported (qmc_served) and the
//     overlap of requests on the GPU can be checked.
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/qmcmd.h"
#include "pool.h"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit arena over one device allocation; offsets and sizes are multiples
// of qmc::kPoolAlign, free blocks are coalesced.
struct Arena {
    unsigned char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes
    static size_t round(size_t b) { return (b + qmc::kPoolAlign - 1) & ~(qmc::kPoolAlign - 1); }
    bool fits(size_t bytes) const {
        bytes = round(bytes);
        for (const auto& kv : free_)
            if (kv.second >= bytes) return true;
        return false;
    }
    bool take(size_t bytes, size_t* off) {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, roff = it->first + bytes;
            free_.erase(it);
            if (rest) free_[roff] = rest;
            return true;
        }
        return false;
    }
    void give(size_t off, size_t bytes) {
        bytes = round(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }
};

struct Traj {
    qmc_params p;
    std::vector<double> zeta, coeff, twist;   // the parameter arrays, owned (twist: [K][3] or empty)
    int N = 0;
    size_t footprint = 0;             // handle + d_R + d_out, the arena block's size
    size_t handle_bytes = 0;          // the handle's part of the block
    size_t block_off = 0;             // offset of the block in the arena (resident only)
    double T_kelvin = 0, delta = 0;
    int s_mode = QMC_S_COV;
    std::vector<double> R;            // current nuclei [3N]
    qmc_system* h = nullptr;          // resident handle, or nullptr
    cudaStream_t stream = nullptr;
    double* d_R = nullptr;            // [3N]
    double* d_out = nullptr;          // [4 + 3N + 9N^2]
    double* h_out = nullptr;          // pinned copies
    double* h_R = nullptr;
    std::vector<unsigned char> ckpt;  // state of an evicted trajectory
    bool has_ckpt = false;
    bool busy = false;
    long long last_used = 0;
    size_t out_len() const { return 4 + 3 * (size_t)N + 9 * (size_t)N * N; }
};

struct Req {
    long long ticket = 0;
    int traj = 0;
    int status = QMC_OK;
    bool done = false;
    double t_submit = 0, t_start = 0, t_done = 0;
    cudaEvent_t ev = nullptr;          // end of the request's work on its stream
    cudaEvent_t ev0 = nullptr;         // start of it
    double gpu_start = -1, gpu_end = -1;
    std::vector<double> out, R_next;
};

}  // namespace

struct qmc_server {
    size_t budget = 0, used = 0;
    Arena arena;
    cudaEvent_t ref = nullptr;             // device time origin of the served intervals
    int max_active = 1;
    std::vector<Traj> trajs;
    std::deque<long long> queue;           // submitted, not started (FIFO)
    std::vector<long long> active;         // started, not completed
    std::map<long long, Req> reqs;
    long long next_ticket = 1, tick = 0;
    long long n_evict = 0, n_done = 0, n_admit = 0;
};

namespace {

// Give a resident trajectory's block back to the arena (its stream stays).
void release_device(qmc_server* s, Traj& t) {
    if (!t.h) return;
    qmc_destroy(t.h);    // waits for the stream; frees nothing carved from the block
    t.h = nullptr;
    t.d_R = t.d_out = nullptr;
    s->arena.give(t.block_off, t.footprint);
    s->used -= t.footprint;
}

int evict(qmc_server* s, Traj& t) {
    t.ckpt.resize(qmc_checkpoint_size(t.h));
    int rc = qmc_checkpoint_save(t.h, t.ckpt.data());
    if (rc != QMC_OK) return rc;
    t.has_ckpt = true;
    release_device(s, t);
    ++s->n_evict;
    return QMC_OK;
}

int make_resident(qmc_server* s, Traj& t) {
    size_t off = 0;
    if (!s->arena.take(t.footprint, &off)) return QMC_ERR_OOM;
    unsigned char* blk = s->arena.base + off;
    t.block_off = off;
    s->used += t.footprint;
    int rc = qmc::init_handle(&t.p, t.R.data(), blk, t.handle_bytes, t.stream, false, &t.h);
    if (rc != QMC_OK) {
        t.h = nullptr;
        s->arena.give(off, t.footprint);
        s->used -= t.footprint;
        return rc;
    }
    t.d_R = (double*)(blk + t.handle_bytes);
    t.d_out = t.d_R + Arena::round(sizeof(double) * 3 * t.N) / sizeof(double);
    if (t.has_ckpt) {
        rc = qmc_checkpoint_load(t.h, t.ckpt.data());
        if (rc != QMC_OK) { release_device(s, t); return rc; }
    }
    ++s->n_admit;
    return QMC_OK;
}

// Make room for `need` bytes by evicting idle resident trajectories, LRU first,
// until the budget allows it and one free block of the arena holds it.
bool make_room(qmc_server* s, size_t need, int keep) {
    while (s->used + need > s->budget || !s->arena.fits(need)) {
        int victim = -1;
        for (int k = 0; k < (int)s->trajs.size(); ++k) {
            const Traj& t = s->trajs[k];
            if (k == keep || !t.h || t.busy) continue;
            if (victim < 0 || t.last_used < s->trajs[victim].last_used) victim = k;
        }
        if (victim < 0) return false;
        if (evict(s, s->trajs[victim]) != QMC_OK) return false;
    }
    return true;
}

int launch(qmc_server* s, Req& r) {
    Traj& t = s->trajs[r.traj];
    const int N3 = 3 * t.N;
    if (cudaEventRecord(r.ev0, t.stream) != cudaSuccess) return QMC_ERR_CUDA;
    std::memcpy(t.h_R, t.R.data(), sizeof(double) * N3);
    cudaMemcpyAsync(t.d_R, t.h_R, sizeof(double) * N3, cudaMemcpyHostToDevice, t.stream);
    int rc = qmc_energy_forces_device(t.h, t.d_R, t.d_out);
    if (rc == QMC_OK)
        rc = langevin_step_device(t.h, t.d_R, t.d_out + 4, t.d_out + 4 + N3, t.T_kelvin, t.delta, t.s_mode, 0.0);
    if (rc != QMC_OK) return rc;
    cudaMemcpyAsync(t.h_out, t.d_out, sizeof(double) * t.out_len(), cudaMemcpyDeviceToHost, t.stream);
    cudaMemcpyAsync(t.h_R, t.d_R, sizeof(double) * N3, cudaMemcpyDeviceToHost, t.stream);
    if (cudaEventRecord(r.ev, t.stream) != cudaSuccess) return QMC_ERR_CUDA;
    t.busy = true;
    r.t_start = now_ms();
    return QMC_OK;
}

}  // namespace

extern "C" {

int qmc_server_create(size_t hbm_budget_bytes, int max_active, qmc_server** out) {
    if (!out || max_active < 1 || hbm_budget_bytes == 0) return QMC_ERR_INVALID;
    qmc_server* s = new (std::nothrow) qmc_server();
    if (!s) return QMC_ERR_OOM;
    s->budget = Arena::round(hbm_budget_bytes);
    s->max_active = max_active;
    if (cudaMalloc(&s->arena.base, s->budget) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return QMC_ERR_OOM;
    }
    s->arena.size = s->budget;
    s->arena.free_[0] = s->budget;
    if (cudaEventCreate(&s->ref) != cudaSuccess || cudaEventRecord(s->ref, 0) != cudaSuccess ||
        cudaEventSynchronize(s->ref) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->arena.base);
        delete s;
        return QMC_ERR_CUDA;
    }
    *out = s;
    return QMC_OK;
}

void qmc_server_destroy(qmc_server* s) {
    if (!s) return;
    for (auto& t : s->trajs) {
        if (t.stream) cudaStreamSynchronize(t.stream);
        release_device(s, t);
        if (t.stream) cudaStreamDestroy(t.stream);
        if (t.h_out) cudaFreeHost(t.h_out);
        if (t.h_R) cudaFreeHost(t.h_R);
    }
    for (auto& kv : s->reqs) {
        if (kv.second.ev) cudaEventDestroy(kv.second.ev);
        if (kv.second.ev0) cudaEventDestroy(kv.second.ev0);
    }
    if (s->ref) cudaEventDestroy(s->ref);
    if (s->arena.base) cudaFree(s->arena.base);
    delete s;
}

int qmc_server_add_trajectory(qmc_server* s, const qmc_params* p, const double* R0, double T_kelvin, double delta,
                              int s_mode, int* traj) {
    if (!s || !p || !R0 || !traj || !p->zeta || !p->coeff) return QMC_ERR_INVALID;
    if (p->fj) return QMC_ERR_INVALID;   // the served form carries no e-e-n-n Jastrow term
    if (s_mode != QMC_S_IDENTITY && s_mode != QMC_S_COV) return QMC_ERR_INVALID;
    const size_t fp = qmc_footprint_bytes(p);
    if (fp == 0) return QMC_ERR_INVALID;
    Traj t;
    t.p = *p;
    t.N = p->n_protons;
    t.zeta.assign(p->zeta, p->zeta + p->n_gauss);
    t.coeff.assign(p->coeff, p->coeff + (size_t)t.N * p->n_gauss * (t.N / 2));
    if (p->n_twist > 0) t.twist.assign(p->twist, p->twist + 3 * (size_t)p->n_twist);
    t.handle_bytes = Arena::round(fp);
    t.footprint = t.handle_bytes + Arena::round(sizeof(double) * 3 * (size_t)t.N) +
                  Arena::round(sizeof(double) * t.out_len());
    if (t.footprint > s->budget) return QMC_ERR_OOM;
    t.T_kelvin = T_kelvin;
    t.delta = delta;
    t.s_mode = s_mode;
    t.R.assign(R0, R0 + 3 * t.N);
    if (cudaHostAlloc((void**)&t.h_out, sizeof(double) * t.out_len(), cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&t.h_R, sizeof(double) * 3 * t.N, cudaHostAllocDefault) != cudaSuccess ||
        cudaStreamCreateWithFlags(&t.stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (t.h_out) cudaFreeHost(t.h_out);
        if (t.h_R) cudaFreeHost(t.h_R);
        return QMC_ERR_CUDA;
    }
    s->trajs.push_back(std::move(t));
    Traj& tt = s->trajs.back();
    tt.p.zeta = tt.zeta.data();
    tt.p.coeff = tt.coeff.data();
    tt.p.twist = tt.twist.empty() ? nullptr : tt.twist.data();
    *traj = (int)s->trajs.size() - 1;
    return QMC_OK;
}

int qmc_server_submit(qmc_server* s, int traj, long long* ticket) {
    if (!s || !ticket || traj < 0 || traj >= (int)s->trajs.size()) return QMC_ERR_INVALID;
    Req r;
    if (cudaEventCreate(&r.ev0) != cudaSuccess || cudaEventCreate(&r.ev) != cudaSuccess) {
        cudaGetLastError();
        if (r.ev0) cudaEventDestroy(r.ev0);
        return QMC_ERR_CUDA;
    }
    r.ticket = s->next_ticket++;
    r.traj = traj;
    r.t_submit = now_ms();
    s->reqs[r.ticket] = std::move(r);
    s->queue.push_back(s->next_ticket - 1);
    *ticket = s->next_ticket - 1;
    return QMC_OK;
}

int qmc_server_progress(qmc_server* s) {
    if (!s) return QMC_ERR_INVALID;
    int completed = 0;
    ++s->tick;
    // 1. completions
    for (size_t k = 0; k < s->active.size();) {
        Req& r = s->reqs[s->active[k]];
        const cudaError_t q = cudaEventQuery(r.ev);
        if (q == cudaErrorNotReady) { ++k; continue; }
        Traj& t = s->trajs[r.traj];
        r.status = (q == cudaSuccess) ? qmc_sync(t.h) : QMC_ERR_CUDA;
        if (q != cudaSuccess) cudaGetLastError();
        r.out.assign(t.h_out, t.h_out + t.out_len());
        r.R_next.assign(t.h_R, t.h_R + 3 * t.N);
        if (r.status == QMC_OK) t.R = r.R_next;
        r.t_done = now_ms();
        r.done = true;
        float a = 0.f, b = 0.f;
        if (q == cudaSuccess && cudaEventElapsedTime(&a, s->ref, r.ev0) == cudaSuccess &&
            cudaEventElapsedTime(&b, s->ref, r.ev) == cudaSuccess) {
            r.gpu_start = a;
            r.gpu_end = b;
        }
        cudaGetLastError();
        cudaEventDestroy(r.ev);
        cudaEventDestroy(r.ev0);
        r.ev = r.ev0 = nullptr;
        t.busy = false;
        t.last_used = s->tick;
        s->active.erase(s->active.begin() + k);
        ++completed;
        ++s->n_done;
    }
    // 2. admissions, FIFO; a trajectory's later requests wait behind its earlier ones
    std::vector<char> blocked(s->trajs.size(), 0);
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)s->active.size() < s->max_active;) {
        Req& r = s->reqs[*it];
        Traj& t = s->trajs[r.traj];
        if (t.busy || blocked[r.traj]) { blocked[r.traj] = 1; ++it; continue; }
        if (!t.h) {
            if (!make_room(s, t.footprint, r.traj)) { blocked[r.traj] = 1; ++it; continue; }
            const int rc = make_resident(s, t);
            if (rc != QMC_OK) {
                r.status = rc; r.done = true; r.t_done = now_ms();
                it = s->queue.erase(it);
                ++completed;
                continue;
            }
        }
        const int rc = launch(s, r);
        if (rc != QMC_OK) {
            r.status = rc; r.done = true; r.t_done = now_ms();
            t.busy = false;
            it = s->queue.erase(it);
            ++completed;
            continue;
        }
        t.last_used = s->tick;
        s->active.push_back(r.ticket);
        it = s->queue.erase(it);
    }
    return completed;
}

int qmc_server_fetch(qmc_server* s, long long ticket, qmc_served* out) {
    if (!s || !out) return QMC_ERR_INVALID;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return QMC_ERR_INVALID;
    Req& r = it->second;
    if (!r.done) return 0;
    const Traj& t = s->trajs[r.traj];
    const int N3 = 3 * t.N;
    out->traj = r.traj;
    out->status = r.status;
    out->latency_ms = r.t_done - r.t_submit;
    out->wait_ms = (r.t_start > 0 ? r.t_start : r.t_done) - r.t_submit;
    out->run_ms = r.t_start > 0 ? r.t_done - r.t_start : 0.0;
    out->gpu_start_ms = r.gpu_start;
    out->gpu_end_ms = r.gpu_end;
    if (!r.out.empty()) {
        out->E = r.out[0]; out->E_err = r.out[1]; out->n_samples = r.out[2]; out->accept = r.out[3];
        if (out->f) std::memcpy(out->f, r.out.data() + 4, sizeof(double) * N3);
        if (out->cov) std::memcpy(out->cov, r.out.data() + 4 + N3, sizeof(double) * N3 * N3);
        if (out->R_next) std::memcpy(out->R_next, r.R_next.data(), sizeof(double) * N3);
    }
    s->reqs.erase(it);
    return 1;
}

int qmc_server_stats(qmc_server* s, long long* st) {
    if (!s || !st) return QMC_ERR_INVALID;
    long long resident = 0;
    for (const auto& t : s->trajs) resident += t.h != nullptr;
    st[0] = (long long)s->used; st[1] = resident; st[2] = (long long)s->active.size();
    st[3] = (long long)s->queue.size(); st[4] = s->n_evict; st[5] = s->n_done; st[6] = s->n_admit;
    st[7] = (long long)s->budget;
    return QMC_OK;
}

}  // extern "C"
