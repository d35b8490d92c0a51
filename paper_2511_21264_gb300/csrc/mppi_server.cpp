// Replan server with continuous batching (see include/mppi.h).
//
// Scenes are registered once: their model, controller settings, simulator
// state, warm-started nominal sequence and Philox counter stay resident on
// the device (receding horizon, paper §III-A: warm start from nu_M).  A
// request asks for one replan of one scene: M MPPI iterations.  Active
// requests are grouped into size classes by their work per iteration
// (K x H, powers of two); each class runs on a stream of its own, one
// batched iteration of all its requests at a time (one persistent rollout
// launch plus one update launch), so classes overlap on the device and a
// short request never waits for a long one.  A scheduler thread polls the
// classes' completion events: it retires the requests that reached M
// iterations (the plan is copied out, the scene's state advances one
// simulator step under u_nom[0] and u_nom shifts by one step), admits
// waiting requests while active slots and the device-memory budget allow,
// and launches the next iteration of every idle class at once.
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
    // the full Eq. 8 (elite != 0); the covariance blocks stay resident and
    // warm-start the scene's next request
    int elite = 0, n_elite = 0, update_cov = 0, cov_sampling = 0;
    float eta = 1.0f, cov_floor = 0.0f;
    float* d_eq8 = nullptr;              // Sigma, L (H x nu x nu each), elite indices (K)
    unsigned long long* d_sel = nullptr;
    void* d_qp = nullptr;                // projection classes and factors (server-wide projection)
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

// A request's device workspace: its K sample costs and, with the
// projection on, its H x K x nu projected samples.
size_t request_bytes(int K, int H = 0, int nu = 0) {
    return ((size_t)K * sizeof(float) + 255) / 256 * 256 + ((size_t)H * K * nu * sizeof(float) + 255) / 256 * 256;
}

}  // namespace

// One size class: its requests and the resources of their iterations.
struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    BatchInst* h_insts = nullptr;  // pinned descriptor table (max_active)
    BatchInst* d_insts = nullptr;
    BatchCtl* d_ctl = nullptr;
    float* h_plans = nullptr;      // pinned, one plan slot per retiring request
    int* h_err = nullptr;          // pinned, one error word per retiring request
    std::vector<Request*> act;        // admitted requests of this class
    std::vector<Request*> inflight;   // requests of the launched iteration
    std::vector<Request*> retiring;   // of those, the ones that finish with it
    bool busy = false;
};

constexpr int MAX_CLASSES = 8;

struct mppi_server {
    mppi_server_config cfg{};
    int na = 0;
    int nclass = 1;     // size classes (1: one batch for every request)
    int plan_max = 0;   // floats of the longest plan (H x nu)
    std::vector<Scene> scenes;
    unsigned char* d_arena = nullptr;
    Arena arena;
    Lane lanes[MAX_CLASSES];
    BatchLaunch L;
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

// Size class of a scene: log2 of its work per iteration over 8192
// sample-steps, clamped to the classes in use.
int class_of(const mppi_server* S, const Scene& sc) {
    if (S->nclass == 1) return 0;
    long long w = (long long)sc.K * sc.H / 8192;
    int c = 0;
    while (w > 1 && c < S->nclass - 1) {
        w >>= 1;
        ++c;
    }
    return c;
}

// A class's iteration has finished on the device: count it, retire the
// requests that reached M iterations.
void complete_lane(mppi_server* S, Lane& ln, cudaError_t e) {
    if (e != cudaSuccess) S->error = cuda_rc(e);
    for (Request* r : ln.inflight) ++r->iters_done;
    const Clock::time_point now = Clock::now();
    if (!ln.retiring.empty()) {
        std::lock_guard<std::mutex> lk(S->mu);
        for (size_t q = 0; q < ln.retiring.size(); ++q) {
            Request& r = *ln.retiring[q];
            Scene& sc = S->scenes[r.scene];
            r.plan.assign(ln.h_plans + q * S->plan_max, ln.h_plans + q * S->plan_max + (size_t)sc.H * sc.nu);
            const int err = ln.h_err[q];
            r.status = (err & ERRB_CHOLESKY) ? MPPI_ERR_CHOLESKY : (err & ERRB_NONFINITE) ? MPPI_ERR_NONFINITE : S->error;
            r.latency_ms = std::chrono::duration<double, std::milli>(now - r.arrival).count();
            S->arena.release(r.arena_off, request_bytes(sc.K, S->cfg.qp_iters ? sc.H : 0, sc.nu));
            sc.busy = false;
            S->lat.push_back(r.latency_ms);
            S->completed++;
            S->sample_steps += (double)sc.K * sc.H * S->cfg.iters_per_request;
            S->last_done = now;
            S->active.erase(std::find(S->active.begin(), S->active.end(), r.ticket));
            ln.act.erase(std::find(ln.act.begin(), ln.act.end(), &r));
            r.done = true;
        }
    }
    ln.inflight.clear();
    ln.retiring.clear();
    ln.busy = false;
    S->done_cv.notify_all();
}

// Enqueue one batched iteration of a class on its stream: the descriptor
// table (longest first), the persistent rollout and the update; for the
// requests that finish with it, the plan copy, the executed step of the
// resident state, the warm-start shift and the error word; then the event.
int launch_lane(mppi_server* S, Lane& ln) {
    std::vector<Request*>& act = ln.act;
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
        BatchInst& I = ln.h_insts[e];
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
        if (sc.d_eq8) {
            const size_t blk = (size_t)sc.H * sc.nu * sc.nu;
            I.elite = sc.elite;
            I.n_elite = sc.n_elite;
            I.update_cov = sc.update_cov;
            I.cov_sampling = sc.cov_sampling;
            I.eta = sc.eta;
            I.cov_floor = sc.cov_floor;
            I.Sigma = sc.d_eq8;
            I.Lfac = sc.d_eq8 + blk;
            I.eidx = reinterpret_cast<int*>(sc.d_eq8 + 2 * blk);
            I.sel = sc.d_sel;
        }
        if (S->cfg.qp_iters)  // the projected samples follow the costs in the request's workspace
            I.U = reinterpret_cast<float*>(S->d_arena + r.arena_off + ((size_t)sc.K * sizeof(float) + 255) / 256 * 256);
        t += (sc.K + S->L.spc - 1) / S->L.spc;
        row += sc.H;
    }
    ln.inflight = act;
    ln.retiring.clear();
    for (Request* r : act)
        if (r->iters_done + 1 >= S->cfg.iters_per_request) ln.retiring.push_back(r);
    NvtxRange range("srv_iteration");
    BatchLaunch L = S->L;
    L.grid = std::min(L.grid, t);  // CTAs past the work would only exit
    L.mode = S->cfg.qp_iters ? 0 : 1;
    L.sel_P = 0;
    for (int e = 0; e < n; ++e)
        if (ln.h_insts[e].elite) {
            int p = 1;
            while (p < ln.h_insts[e].K) p <<= 1;
            L.sel_P = std::max(L.sel_P, p);
        }
    int rc = cuda_rc(cudaMemcpyAsync(ln.d_insts, ln.h_insts, n * sizeof(BatchInst), cudaMemcpyHostToDevice, ln.stream));
    for (int e = 0; e < n && rc == MPPI_OK && S->cfg.qp_iters; ++e) {  // sample and project (Eq. 5)
        const BatchInst& I = ln.h_insts[e];
        const Scene& sc = S->scenes[act[e]->scene];
        const QPArgs q = qp_controller_args(sc.nu, 2 * S->na + 7, sc.K, sc.H, S->cfg.qp_iters, model_dt(sc.model),
                                            sc.d_qp, I.state, I.u, I.sigma, I.cov_sampling ? I.Lfac : nullptr, I.seed,
                                            I.iter, I.U);
        rc = launch_qp(q, ln.stream);
    }
    if (rc == MPPI_OK) rc = launch_batch_iteration(ln.d_insts, n, t, row, ln.d_ctl, L, ln.stream);
    for (size_t q = 0; q < ln.retiring.size() && rc == MPPI_OK; ++q) {
        Request& r = *ln.retiring[q];
        Scene& sc = S->scenes[r.scene];
        rc = cuda_rc(cudaMemcpyAsync(ln.h_plans + q * S->plan_max, sc.d_u, (size_t)sc.H * sc.nu * sizeof(float),
                                     cudaMemcpyDeviceToHost, ln.stream));
        RolloutArgs a{};
        a.model = model_device(sc.model);
        a.n = 1;
        a.H = 1;
        a.states = sc.d_state;
        a.state_stride = sc.nx;
        a.U = sc.d_u;
        a.costs = reinterpret_cast<float*>(S->d_arena + r.arena_off);
        a.states_out = sc.d_state;
        a.err = sc.d_err;
        if (rc == MPPI_OK) rc = launch_rollout(S->na, 0, a, 1, ln.stream);
        if (rc == MPPI_OK) rc = launch_shift(sc.d_u, sc.H, sc.nu, ln.stream);
        if (rc == MPPI_OK)
            rc = cuda_rc(cudaMemcpyAsync(ln.h_err + q, sc.d_err, sizeof(int), cudaMemcpyDeviceToHost, ln.stream));
        if (rc == MPPI_OK) rc = cuda_rc(cudaMemsetAsync(sc.d_err, 0, sizeof(int), ln.stream));
    }
    if (rc == MPPI_OK) rc = cuda_rc(cudaEventRecord(ln.ev, ln.stream));
    if (rc != MPPI_OK) {
        S->error = rc;
        cudaStreamSynchronize(ln.stream);
        complete_lane(S, ln, cudaSuccess);
        return rc;
    }
    ++S->iterations;
    S->sum_active += n;
    ln.busy = true;
    return MPPI_OK;
}

// One scheduler pass: finish the classes whose iteration is done, admit,
// launch every idle class that has requests.  The queue lock is held only
// while the queues change; GPU work is enqueued unlocked (map nodes of
// active requests are stable: only the scheduler retires them).  Returns
// false when there was nothing to do.
bool scheduler_step(mppi_server* S) {
    bool did = false;
    for (int c = 0; c < S->nclass; ++c) {
        Lane& ln = S->lanes[c];
        if (!ln.busy) continue;
        const cudaError_t e = cudaEventQuery(ln.ev);
        if (e == cudaErrorNotReady) continue;
        complete_lane(S, ln, e);
        did = true;
    }
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
            if (!S->arena.alloc(request_bytes(sc.K, S->cfg.qp_iters ? sc.H : 0, sc.nu), &off)) {
                ++S->admission_waits;
                ++it;
                continue;
            }
            r.arena_off = off;
            sc.busy = true;
            S->active.push_back(r.ticket);
            S->lanes[class_of(S, sc)].act.push_back(&r);
            it = S->waiting.erase(it);
            did = true;
        }
    }
    for (int c = 0; c < S->nclass; ++c) {
        Lane& ln = S->lanes[c];
        if (ln.busy || ln.act.empty()) continue;
        launch_lane(S, ln);
        did = true;
    }
    return did;
}

void scheduler_main(mppi_server* S) {
    cudaSetDevice(S->device);
    while (!S->stop.load()) {
        if (scheduler_step(S)) continue;
        bool inflight = false;
        for (int c = 0; c < S->nclass; ++c) inflight = inflight || S->lanes[c].busy;
        if (inflight) {
            std::this_thread::yield();  // GPU work in flight: poll its events again
            continue;
        }
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv.wait_for(lk, std::chrono::microseconds(200), [&] { return S->stop.load() || !S->waiting.empty(); });
    }
    for (int c = 0; c < S->nclass; ++c)  // drain before the stream objects go
        if (S->lanes[c].stream) cudaStreamSynchronize(S->lanes[c].stream);
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
    if (cfg->size_classes < 0 || cfg->size_classes > MAX_CLASSES || cfg->qp_iters < 0) {
        delete S;
        return MPPI_ERR_INVALID_ARG;
    }
    S->nclass = cfg->size_classes == 0 ? 6 : cfg->size_classes;
    // larger classes get higher stream priority: the longest requests set
    // the latency tail, and their CTAs then go first when SMs free up
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_arena, cfg->mem_budget_bytes);
    for (int c = 0; c < S->nclass && e == cudaSuccess; ++c) {
        Lane& ln = S->lanes[c];
        e = cudaMalloc(&ln.d_insts, cfg->max_active * sizeof(BatchInst));
        if (e == cudaSuccess) e = cudaMallocHost(&ln.h_insts, cfg->max_active * sizeof(BatchInst));
        if (e == cudaSuccess) e = cudaMalloc(&ln.d_ctl, sizeof(BatchCtl));
        if (e == cudaSuccess) e = cudaMemset(ln.d_ctl, 0, sizeof(BatchCtl));
        if (e == cudaSuccess) e = cudaMallocHost(&ln.h_err, cfg->max_active * sizeof(int));
        const int prio = S->nclass == 1 ? least : least - (least - greatest) * c / (S->nclass - 1);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ln.stream, cudaStreamNonBlocking, prio);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ln.ev, cudaEventDisableTiming);
    }
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
    if (request_bytes(K, S->cfg.qp_iters ? H : 0, 2 * ((nq - 7) / 2)) > S->cfg.mem_budget_bytes)
        return MPPI_ERR_ADMISSION;
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
    if (S->cfg.qp_iters)
        for (const Scene& sc : S->scenes)
            if (!sc.d_qp) return MPPI_ERR_INVALID_ARG;  // every scene needs its projection bounds
    int max_h = 0;
    for (const Scene& sc : S->scenes) max_h = std::max(max_h, sc.H);
    // 16 lanes per sample for 7-link arms unless set: the mixes hold large K,
    // whose rollouts run faster two to a warp (p99 at 200 req/s over the
    // served pool: 10.2 ms against 15.7 with 32 lanes)
    const int lps = S->cfg.lanes_per_sample ? S->cfg.lanes_per_sample : (S->na == 7 ? 16 : 32);
    int rc = batch_shape(S->na, S->cfg.samples_per_cta, lps, 0, max_h, &S->L);
    if (rc != MPPI_OK) return rc;
    // pinned plan slots for the retiring requests of each class
    S->plan_max = 0;
    for (const Scene& sc : S->scenes) S->plan_max = std::max(S->plan_max, sc.H * sc.nu);
    for (int c = 0; c < S->nclass; ++c) {
        Lane& ln = S->lanes[c];
        cudaFreeHost(ln.h_plans);
        ln.h_plans = nullptr;
        const cudaError_t e = cudaMallocHost(&ln.h_plans, (size_t)S->cfg.max_active * S->plan_max * sizeof(float));
        if (e != cudaSuccess) return cuda_rc(e);
    }
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
        cudaFree(sc.d_eq8);
        cudaFree(sc.d_sel);
        cudaFree(sc.d_qp);
    }
    for (int c = 0; c < MAX_CLASSES; ++c) {
        Lane& ln = S->lanes[c];
        if (ln.stream) cudaStreamDestroy(ln.stream);
        if (ln.ev) cudaEventDestroy(ln.ev);
        cudaFree(ln.d_insts);
        cudaFreeHost(ln.h_insts);
        cudaFree(ln.d_ctl);
        cudaFreeHost(ln.h_plans);
        cudaFreeHost(ln.h_err);
    }
    cudaFree(S->d_arena);
    delete S;
    return MPPI_OK;
}

int srv_set_scene_update(mppi_server* S, int scene_id, int n_elite, float eta, int update_cov, float cov_floor) {
    if (!S || scene_id < 0 || scene_id >= (int)S->scenes.size() || S->running.load()) return MPPI_ERR_INVALID_ARG;
    Scene& sc = S->scenes[scene_id];
    if (n_elite == 0) n_elite = sc.K;
    if (n_elite < 1 || n_elite > sc.K || !(eta > 0.0f && eta <= 1.0f) || update_cov < 0 || update_cov > 1 ||
        !(cov_floor >= 0.0f))
        return MPPI_ERR_INVALID_ARG;
    if (n_elite < sc.K && sc.K > 8192) return MPPI_ERR_UNSUPPORTED;  // the elite sort holds 8192 keys
    const size_t blk = (size_t)sc.H * sc.nu * sc.nu;
    if (!sc.d_eq8) {
        cudaError_t e = cudaMalloc(&sc.d_eq8, (2 * blk + (size_t)sc.K) * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&sc.d_sel, 3 * sizeof(unsigned long long));
        std::vector<float> sig(sc.nu), B(2 * blk, 0.0f);  // Sigma_0 = diag(sigma^2), its factor diag(sigma)
        if (e == cudaSuccess) e = cudaMemcpy(sig.data(), sc.d_params, sc.nu * sizeof(float), cudaMemcpyDeviceToHost);
        for (int h = 0; h < sc.H; ++h)
            for (int j = 0; j < sc.nu; ++j) {
                B[((size_t)h * sc.nu + j) * sc.nu + j] = sig[j] * sig[j];
                B[blk + ((size_t)h * sc.nu + j) * sc.nu + j] = sig[j];
            }
        if (e == cudaSuccess) e = cudaMemcpy(sc.d_eq8, B.data(), 2 * blk * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(sc.d_eq8);
            cudaFree(sc.d_sel);
            sc.d_eq8 = nullptr;
            sc.d_sel = nullptr;
            return cuda_rc(e);
        }
    }
    sc.n_elite = n_elite;
    sc.eta = eta;
    sc.update_cov = update_cov;
    sc.cov_floor = cov_floor;
    if (update_cov) sc.cov_sampling = 1;
    sc.elite = (n_elite != sc.K || eta != 1.0f || update_cov || sc.cov_sampling) ? 1 : 0;
    return MPPI_OK;
}

int srv_set_scene_projection(mppi_server* S, int scene_id, const float* bounds, float rho, const float* scales) {
    if (!S || !bounds || scene_id < 0 || scene_id >= (int)S->scenes.size() || S->running.load())
        return MPPI_ERR_INVALID_ARG;
    Scene& sc = S->scenes[scene_id];
    std::vector<unsigned char> host;
    const int rc = qp_build(sc.nu, sc.H, bounds, rho, scales, host);
    if (rc != MPPI_OK) return rc;
    cudaFree(sc.d_qp);
    sc.d_qp = nullptr;
    cudaError_t e = cudaMalloc(&sc.d_qp, host.size());
    if (e == cudaSuccess) e = cudaMemcpy(sc.d_qp, host.data(), host.size(), cudaMemcpyHostToDevice);
    return cuda_rc(e);
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
