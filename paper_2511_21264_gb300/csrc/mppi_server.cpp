// Replan server with continuous batching (see include/mppi.h).
//
// Scenes are registered once: their model, controller settings, simulator
// state, warm-started nominal sequence and Philox counter stay resident on
// the device (receding horizon, paper §III-A: warm start from nu_M).  A
// request asks for one replan of one scene: M MPPI iterations.  A scheduler
// thread works in iteration steps: at every boundary it admits waiting
// requests while active slots and the device-memory budget allow, runs one
// batched iteration of every active request (one persistent rollout launch
// plus one update launch), and retires requests that reached M iterations:
// their scene's state advances one simulator step under u_nom[0], u_nom is
// shifted by one step, the plan is copied out and the latency recorded.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <random>
#include <thread>
#include <vector>

#include "../../include/mppi.h"
#include "mppi_internal.h"

using namespace mppi;

namespace {

using Clock = std::chrono::steady_clock;

struct Scene {
    const mppi_model* model = nullptr;
    int K = 0, H = 0, nu = 0, nx = 0;
    float lambda = 1.0f;
    uint64_t seed = 0;
    float* d_state = nullptr;
    float* d_u = nullptr;
    float* d_params = nullptr;  // sigma, u_lo, u_hi (3 x 16)
    unsigned long long* d_iter = nullptr;
    unsigned int* d_done = nullptr;
    int* d_err = nullptr;
    float* d_best = nullptr;
    bool busy = false;  // a request of this scene is active
};

struct Request {
    uint64_t ticket = 0;
    int scene = 0;
    Clock::time_point arrival;
    int iters_done = 0;
    size_t arena_off = 0;
    bool done = false, cancelled = false;
    int status = MPPI_OK;
    double latency_ms = 0.0;
    std::vector<float> plan;
};

// First-fit allocator over one device buffer (the admission budget).
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    void init(size_t n) {
        size = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    bool alloc(size_t n, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, o = it->first + n;
                free_.erase(it);
                if (rest) free_[o] = rest;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t n) {
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

size_t request_bytes(int K) { return ((size_t)K * sizeof(float) + 255) / 256 * 256; }

}  // namespace

struct mppi_server {
    mppi_server_config cfg{};
    int na = 0;
    std::vector<Scene> scenes;
    unsigned char* d_arena = nullptr;
    Arena arena;
    BatchInst* d_insts = nullptr;
    BatchInst* h_insts = nullptr;  // pinned
    BatchCtl* d_ctl = nullptr;
    BatchLaunch L;
    cudaStream_t stream = nullptr;
    int device = 0;
    // queues
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<uint64_t> waiting;
    std::vector<uint64_t> active;
    std::map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    std::thread th;
    std::atomic<bool> running{false}, stop{false};
    Clock::time_point t0;
    // statistics
    std::vector<double> lat;
    long long completed = 0, iterations = 0, sum_active = 0, admission_waits = 0;
    double sample_steps = 0.0;
    Clock::time_point first_arrival, last_done;
    bool have_first = false;
    int error = MPPI_OK;
};

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? MPPI_OK : (e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA); }

// One scheduler step: admit, run one batched iteration, retire.  The queue
// lock is held only while the queues change; GPU work runs unlocked (map
// nodes of active requests are stable: only the scheduler retires them).
// Returns false when there was nothing to do.
bool scheduler_step(mppi_server* S) {
    std::vector<Request*> act;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        // admission, FIFO: a request waits for a free slot, its scene (one
        // request per scene at a time) and budget; later requests may pass a
        // blocked one
        for (auto it = S->waiting.begin(); it != S->waiting.end();) {
            if ((int)S->active.size() >= S->cfg.max_active) break;
            Request& r = S->reqs.at(*it);
            Scene& sc = S->scenes[r.scene];
            if (sc.busy) {
                ++it;
                continue;
            }
            size_t off = 0;
            if (!S->arena.alloc(request_bytes(sc.K), &off)) {
                ++S->admission_waits;
                ++it;
                continue;
            }
            r.arena_off = off;
            sc.busy = true;
            S->active.push_back(r.ticket);
            it = S->waiting.erase(it);
        }
        for (uint64_t tk : S->active) act.push_back(&S->reqs.at(tk));
    }
    if (act.empty()) return false;
    NvtxRange range("srv_iteration");
    // descriptor table: longest (K H) first, tile and row prefixes
    std::stable_sort(act.begin(), act.end(), [&](const Request* a, const Request* b) {
        const Scene& x = S->scenes[a->scene];
        const Scene& y = S->scenes[b->scene];
        return (long long)x.K * x.H > (long long)y.K * y.H;
    });
    int t = 0, row = 0;
    const int n = (int)act.size();
    for (int e = 0; e < n; ++e) {
        const Request& r = *act[e];
        const Scene& sc = S->scenes[r.scene];
        BatchInst& I = S->h_insts[e];
        std::memset(&I, 0, sizeof I);
        I.model = model_device(sc.model);
        I.state = sc.d_state;
        I.u = sc.d_u;
        I.costs = reinterpret_cast<float*>(S->d_arena + r.arena_off);
        I.sigma = sc.d_params;
        I.u_lo = sc.d_params + 16;
        I.u_hi = sc.d_params + 32;
        I.iter = sc.d_iter;
        I.done = sc.d_done;
        I.err = sc.d_err;
        I.best = sc.d_best;
        I.seed = sc.seed;
        I.K = sc.K;
        I.H = sc.H;
        I.lambda = sc.lambda;
        I.stage_unom = sc.H * sc.nu <= 2048;
        I.tile0 = t;
        I.row0 = row;
        t += (sc.K + S->L.spc - 1) / S->L.spc;
        row += sc.H;
    }
    int rc = cuda_rc(cudaMemcpyAsync(S->d_insts, S->h_insts, n * sizeof(BatchInst), cudaMemcpyHostToDevice,
                                     S->stream));
    if (rc == MPPI_OK) rc = launch_batch_iteration(S->d_insts, n, t, row, S->d_ctl, S->L, S->stream);
    if (rc == MPPI_OK) rc = cuda_rc(cudaStreamSynchronize(S->stream));
    if (rc != MPPI_OK) S->error = rc;
    ++S->iterations;
    S->sum_active += n;
    std::vector<Request*> fin;
    for (Request* r : act)
        if (++r->iters_done >= S->cfg.iters_per_request) fin.push_back(r);
    if (fin.empty()) return true;
    // retire: copy the plan out, execute u_nom[0] on the resident state,
    // shift the warm start by one step
    for (Request* r : fin) {
        Scene& sc = S->scenes[r->scene];
        r->plan.resize((size_t)sc.H * sc.nu);
        cudaMemcpyAsync(r->plan.data(), sc.d_u, r->plan.size() * sizeof(float), cudaMemcpyDeviceToHost, S->stream);
        RolloutArgs a{};
        a.model = model_device(sc.model);
        a.n = 1;
        a.H = 1;
        a.states = sc.d_state;
        a.state_stride = sc.nx;
        a.U = sc.d_u;
        a.costs = reinterpret_cast<float*>(S->d_arena + r->arena_off);
        a.states_out = sc.d_state;
        a.err = sc.d_err;
        rc = launch_rollout(S->na, 0, a, 1, S->stream);
        if (rc == MPPI_OK) rc = launch_shift(sc.d_u, sc.H, sc.nu, S->stream);
        if (rc != MPPI_OK) S->error = rc;
    }
    rc = cuda_rc(cudaStreamSynchronize(S->stream));
    if (rc != MPPI_OK) S->error = rc;
    std::vector<int> errs(fin.size(), 0);
    for (size_t q = 0; q < fin.size(); ++q) {
        Scene& sc = S->scenes[fin[q]->scene];
        cudaMemcpy(&errs[q], sc.d_err, sizeof(int), cudaMemcpyDeviceToHost);
        cudaMemset(sc.d_err, 0, sizeof(int));
    }
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (size_t q = 0; q < fin.size(); ++q) {
            Request& r = *fin[q];
            Scene& sc = S->scenes[r.scene];
            const int err = errs[q];
            r.status = (err & ERRB_CHOLESKY) ? MPPI_ERR_CHOLESKY : (err & ERRB_NONFINITE) ? MPPI_ERR_NONFINITE : S->error;
            r.latency_ms = std::chrono::duration<double, std::milli>(now - r.arrival).count();
            S->arena.release(r.arena_off, request_bytes(sc.K));
            sc.busy = false;
            S->lat.push_back(r.latency_ms);
            S->completed++;
            S->sample_steps += (double)sc.K * sc.H * S->cfg.iters_per_request;
            S->last_done = now;
            S->active.erase(std::find(S->active.begin(), S->active.end(), r.ticket));
            r.done = true;
        }
    }
    S->done_cv.notify_all();
    return true;
}

void scheduler_main(mppi_server* S) {
    cudaSetDevice(S->device);
    while (!S->stop.load()) {
        if (!scheduler_step(S)) {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait_for(lk, std::chrono::microseconds(200),
                           [&] { return S->stop.load() || !S->waiting.empty(); });
        }
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double idx = p * (double)(v.size() - 1);
    const size_t lo = (size_t)idx, hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (idx - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace

extern "C" {

int srv_create(const mppi_server_config* cfg, mppi_server** out) {
    if (!cfg || !out || cfg->max_active < 1 || cfg->max_active > 4096 || cfg->iters_per_request < 1 ||
        cfg->mem_budget_bytes < 256)
        return MPPI_ERR_INVALID_ARG;
    *out = nullptr;
    mppi_server* S = new (std::nothrow) mppi_server();
    if (!S) return MPPI_ERR_OOM;
    S->cfg = *cfg;
    if (S->cfg.samples_per_cta <= 0) S->cfg.samples_per_cta = 4;
    cudaGetDevice(&S->device);
    cudaError_t e = cudaMalloc(&S->d_arena, cfg->mem_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_insts, cfg->max_active * sizeof(BatchInst));
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_insts, cfg->max_active * sizeof(BatchInst));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_ctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMemset(S->d_ctl, 0, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        srv_destroy(S);
        return cuda_rc(e);
    }
    S->arena.init(cfg->mem_budget_bytes);
    S->t0 = Clock::now();
    *out = S;
    return MPPI_OK;
}

int srv_add_scene(mppi_server* S, const mppi_model* m, int K, int H, float lambda, const float* sigma, uint64_t seed,
                  const float* x0, int* scene_id) {
    if (!S || !m || !sigma || !scene_id || K < 1 || K > (1 << 20) || H < 1 || H > 1024 || !(lambda > 0.0f) ||
        S->running.load())
        return MPPI_ERR_INVALID_ARG;
    int nq = 0, nv = 0, nu = 0;
    mppi_model_dims(m, &nq, &nv, &nu, nullptr);
    const int na = nu / 2;
    if (na != 3 && na != 7) return MPPI_ERR_UNSUPPORTED;
    if (S->na && S->na != na) return MPPI_ERR_INVALID_ARG;
    if (request_bytes(K) > S->cfg.mem_budget_bytes) return MPPI_ERR_ADMISSION;
    S->na = na;
    Scene sc;
    sc.model = m;
    sc.K = K;
    sc.H = H;
    sc.nu = nu;
    sc.nx = nq + nv;
    sc.lambda = lambda;
    sc.seed = seed;
    std::vector<float> x(sc.nx), params(48, 0.0f), zeros((size_t)H * nu, 0.0f);
    if (x0) std::memcpy(x.data(), x0, sc.nx * sizeof(float));
    else mppi_model_home(m, x.data());
    for (int j = 0; j < nu; ++j) {
        params[j] = sigma[j];
        model_bounds(m, j, &params[16 + j], &params[32 + j]);
    }
    cudaError_t e = cudaMalloc(&sc.d_state, sc.nx * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&sc.d_u, zeros.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&sc.d_params, 48 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&sc.d_iter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&sc.d_done, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&sc.d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&sc.d_best, 2 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(sc.d_state, x.data(), sc.nx * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sc.d_u, zeros.data(), zeros.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sc.d_params, params.data(), 48 * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(sc.d_iter, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(sc.d_done, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(sc.d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(sc.d_state);
        cudaFree(sc.d_u);
        cudaFree(sc.d_params);
        cudaFree(sc.d_iter);
        cudaFree(sc.d_done);
        cudaFree(sc.d_err);
        cudaFree(sc.d_best);
        return cuda_rc(e);
    }
    *scene_id = (int)S->scenes.size();
    S->scenes.push_back(sc);
    return MPPI_OK;
}

int srv_start(mppi_server* S) {
    if (!S || S->running.load() || S->scenes.empty()) return MPPI_ERR_INVALID_ARG;
    int max_h = 0;
    for (const Scene& sc : S->scenes) max_h = std::max(max_h, sc.H);
    int rc = batch_shape(S->na, S->cfg.samples_per_cta, 0, 0, max_h, &S->L);
    if (rc != MPPI_OK) return rc;
    S->stop = false;
    S->running = true;
    S->th = std::thread(scheduler_main, S);
    return MPPI_OK;
}

int srv_stop(mppi_server* S) {
    if (!S) return MPPI_ERR_INVALID_ARG;
    if (S->running.load()) {
        S->stop = true;
        S->cv.notify_all();
        S->th.join();
        S->running = false;
    }
    return S->error;
}

int srv_destroy(mppi_server* S) {
    if (!S) return MPPI_OK;
    srv_stop(S);
    for (Scene& sc : S->scenes) {
        cudaFree(sc.d_state);
        cudaFree(sc.d_u);
        cudaFree(sc.d_params);
        cudaFree(sc.d_iter);
        cudaFree(sc.d_done);
        cudaFree(sc.d_err);
        cudaFree(sc.d_best);
    }
    if (S->stream) cudaStreamDestroy(S->stream);
    cudaFree(S->d_arena);
    cudaFree(S->d_insts);
    cudaFreeHost(S->h_insts);
    cudaFree(S->d_ctl);
    delete S;
    return MPPI_OK;
}

int srv_submit(mppi_server* S, int scene_id, uint64_t* ticket) {
    if (!S || !ticket || scene_id < 0 || scene_id >= (int)S->scenes.size()) return MPPI_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        Request r;
        r.ticket = S->next_ticket++;
        r.scene = scene_id;
        r.arrival = Clock::now();
        if (!S->have_first) {
            S->first_arrival = r.arrival;
            S->have_first = true;
        }
        *ticket = r.ticket;
        S->waiting.push_back(r.ticket);
        S->reqs.emplace(r.ticket, std::move(r));
    }
    S->cv.notify_all();
    return MPPI_OK;
}

int srv_cancel(mppi_server* S, uint64_t ticket) {
    if (!S) return MPPI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return MPPI_ERR_INVALID_ARG;
    auto w = std::find(S->waiting.begin(), S->waiting.end(), ticket);
    if (w == S->waiting.end()) return MPPI_ERR_INVALID_ARG;  // already admitted or done
    it->second.cancelled = true;
    S->waiting.erase(w);
    S->reqs.erase(it);
    return MPPI_OK;
}

int srv_poll(mppi_server* S, uint64_t ticket, float* u_out, int u_len, double* latency_ms, int* done, int wait_ms) {
    if (!S || !done) return MPPI_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return MPPI_ERR_INVALID_ARG;
    if (!it->second.done && wait_ms > 0)
        S->done_cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return it->second.done; });
    *done = it->second.done ? 1 : 0;
    if (!*done) return MPPI_OK;
    const Request& r = it->second;
    if (u_out) std::memcpy(u_out, r.plan.data(), std::min<size_t>(r.plan.size(), (size_t)std::max(u_len, 0)) * sizeof(float));
    if (latency_ms) *latency_ms = r.latency_ms;
    const int st = r.status;
    S->reqs.erase(it);
    return st;
}

int srv_get_state(mppi_server* S, int scene_id, float* x_host) {
    if (!S || !x_host || scene_id < 0 || scene_id >= (int)S->scenes.size()) return MPPI_ERR_INVALID_ARG;
    const Scene& sc = S->scenes[scene_id];
    std::lock_guard<std::mutex> lk(S->mu);
    if (sc.busy) return MPPI_ERR_INVALID_ARG;
    return cuda_rc(cudaMemcpy(x_host, sc.d_state, sc.nx * sizeof(float), cudaMemcpyDeviceToHost));
}

int srv_stats(mppi_server* S, srv_stats_t* st) {
    if (!S || !st) return MPPI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof *st);
    st->completed = S->completed;
    st->iterations = S->iterations;
    st->waiting = (long long)S->waiting.size();
    st->active = (long long)S->active.size();
    st->admission_waits = S->admission_waits;
    st->p50_ms = percentile(S->lat, 0.50);
    st->p99_ms = percentile(S->lat, 0.99);
    st->mean_ms = S->lat.empty() ? 0.0 : std::accumulate(S->lat.begin(), S->lat.end(), 0.0) / S->lat.size();
    st->mean_active = S->iterations ? (double)S->sum_active / S->iterations : 0.0;
    const double span = S->have_first && S->completed
                            ? std::chrono::duration<double>(S->last_done - S->first_arrival).count()
                            : 0.0;
    st->sample_steps_per_s = span > 0 ? S->sample_steps / span : 0.0;
    return MPPI_OK;
}

// Poisson arrivals at rate_hz for duration_s over the registered scenes
// (uniform), then wait for every request; statistics via srv_stats.
int srv_run_load(mppi_server* S, double rate_hz, double duration_s, uint64_t seed, int drain_ms) {
    if (!S || !(rate_hz > 0) || !(duration_s > 0) || !S->running.load()) return MPPI_ERR_INVALID_ARG;
    std::mt19937_64 rng(seed);
    std::exponential_distribution<double> gap(rate_hz);
    std::uniform_int_distribution<int> pick(0, (int)S->scenes.size() - 1);
    const Clock::time_point start = Clock::now();
    double t = gap(rng);
    std::vector<uint64_t> tickets;
    while (t < duration_s) {
        std::this_thread::sleep_until(start + std::chrono::duration_cast<Clock::duration>(
                                                  std::chrono::duration<double>(t)));
        uint64_t tk = 0;
        int rc = srv_submit(S, pick(rng), &tk);
        if (rc != MPPI_OK) return rc;
        tickets.push_back(tk);
        t += gap(rng);
    }
    const Clock::time_point deadline = Clock::now() + std::chrono::milliseconds(drain_ms);
    for (uint64_t tk : tickets) {
        int done = 0;
        while (!done) {
            const int left = (int)std::chrono::duration_cast<std::chrono::milliseconds>(deadline - Clock::now()).count();
            if (left <= 0) return MPPI_ERR_TIMEOUT;
            srv_poll(S, tk, nullptr, 0, nullptr, &done, std::min(left, 100));
        }
    }
    return S->error;
}

}  // extern "C"
