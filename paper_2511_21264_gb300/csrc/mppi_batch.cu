// Batched MPPI: many independent controllers (uneven K, H and obstacle
// counts, same arm model size) advanced by one persistent rollout launch and
// one update launch per iteration, optionally replayed from a CUDA graph,
// with an autotuner for the launch shape (see include/mppi.h).
#include <cuda_runtime.h>
#include <sys/stat.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/mppi.h"
#include "mppi_device.cuh"
#include "mppi_internal.h"
#include "mppi_kernels.cuh"
#include "mppi_rollout.cuh"

using namespace mppi;

namespace mppi {

// Persistent rollout: each CTA takes (instance, tile of samples-per-CTA
// samples) work items from a counter until none are left.  The model and
// u_nom of the tile's instance are staged when the instance changes.  The
// last CTA out resets the counters for the next launch (no CTA waits).
// instance owning work item t: the last instance whose first item is <= t
__device__ __forceinline__ int owner(const BatchInst* insts, int n, int t, bool rows) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int first = rows ? insts[mid].row0 : insts[mid].tile0;
        if (first <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int NA, int LPS, int PLACE, int MODE>
__global__ void __launch_bounds__(256, 2) batch_rollout_kernel(const BatchInst* insts, int n, int ntiles, BatchCtl* ctl,
                                                             int max_unom) {
    using d = Dims<NA>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_tile;
    DevModel& M = *reinterpret_cast<DevModel*>(smem);
    float* unom_s = reinterpret_cast<float*>(smem + sizeof(DevModel));
    unsigned char* wsb = smem + sizeof(DevModel) + ((size_t)max_unom * sizeof(float) + 15) / 16 * 16;
    const int spc = blockDim.x / LPS, gi = threadIdx.x / LPS;
    const Lanes<LPS> g(threadIdx.x & 31);
    WarpWS<NA>& w = *reinterpret_cast<WarpWS<NA>*>(wsb + (size_t)gi * ws_stride<NA, LPS>());
    int staged = -1;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&ctl->next, 1u);
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        const int inst = owner(insts, n, t, false);
        const BatchInst& I = insts[inst];
        const int unom_n = (MODE == 1 && I.stage_unom) ? I.H * d::NU : 0;
        if (inst != staged) {
            stage_model(smem, I.model, unom_s, I.u, unom_n);
            staged = inst;
        }
        __syncthreads();
        const int k = (t - I.tile0) * spc + gi;
        if (k < I.K) {
            SampleIO io{};
            io.x = I.state;
            io.k = k;
            io.H = I.H;
            io.err = I.err;
            if (MODE == 1) {
                io.unom = unom_n ? unom_s : I.u;
                io.iter = (uint32_t)(*I.iter);
                io.key = make_uint2((uint32_t)I.seed, (uint32_t)(I.seed >> 32));
                io.Lfac = I.cov_sampling ? I.Lfac : nullptr;
                if (g.sl < d::NU) {
                    io.sig = I.sigma[g.sl];
                    io.lo = I.u_lo[g.sl];
                    io.hi = I.u_hi[g.sl];
                }
            } else {  // the instance's projected samples, h-major
                io.U = I.U + (size_t)k * d::NU;
                io.u_stride = (long long)I.K * d::NU;
                io.u_ext = (long long)I.H * I.K * d::NU - (long long)k * d::NU;
            }
            // drawn samples: the covariance-capable draw (instances may mix)
            const float cost = rollout_sample<NA, LPS, MODE == 1 ? 2 : 0, false, PLACE>(M, w, g, io);
            if (g.sl == 0) I.costs[k] = cost;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned e = atomicAdd(&ctl->exited, 1u);
        if (e == gridDim.x - 1) {
            ctl->next = 0u;
            ctl->exited = 0u;
            __threadfence();
        }
    }
}

// Elite threshold of every instance that uses the full Eq. 8 (one CTA per
// instance in execution order; the others exit).
__global__ void __launch_bounds__(1024) batch_select_kernel(const BatchInst* insts, int n) {
    extern __shared__ unsigned long long keys[];
    __shared__ int nfin;
    const BatchInst& I = insts[blockIdx.x];
    if (!I.elite) return;
    int P = 1;
    while (P < I.K) P <<= 1;
    elite_select_block(I.costs, I.K, P, I.n_elite, I.sel, I.eidx, keys, nfin);
}

// One CTA per (instance, horizon step): the plain update (Eq. 8a/8d with
// eta = 1 over every sample) or the full Eq. 8 (elite set, learning rate,
// covariance block) as the instance asks; each instance's last CTA
// advances its iteration counter.
template <int NU>
__global__ void __launch_bounds__(256) batch_update_kernel(const BatchInst* insts, int n) {
    __shared__ union {
        UpdateSmem<NU> u;
        EliteSmem<NU> e;
    } sm;
    const int inst = owner(insts, n, blockIdx.x, true);
    const BatchInst& I = insts[inst];
    const int h = blockIdx.x - I.row0;
    if (I.elite) {
        EliteArgs a{};
        a.K = I.K;
        a.H = I.H;
        a.n_elite = I.n_elite;
        a.update_cov = I.update_cov;
        a.beta = I.lambda;
        a.eta = I.eta;
        a.cov_floor = I.cov_floor;
        a.costs = I.costs;
        a.u_nom = I.u;
        a.u_out = I.u;
        a.sigma = I.sigma;
        a.Lfac = I.cov_sampling ? I.Lfac : nullptr;
        a.u_lo = I.u_lo;
        a.u_hi = I.u_hi;
        a.Sigma = I.Sigma;
        a.Lout = I.Lfac;
        a.seed = I.seed;
        a.iter_ptr = I.iter;
        a.U_stored = I.U;
        a.sel = I.sel;
        a.eidx = I.eidx;
        a.best_U = nullptr;
        a.err = I.err;
        elite_update_step<NU>(a, h, sm.e);
        __syncthreads();
        if (threadIdx.x == 0) {  // the last CTA of the instance advances its counter (no waiting)
            __threadfence();
            const unsigned t = atomicAdd(I.done, 1u);
            sm.e.is_last = (t == (unsigned)I.H - 1u);
        }
        __syncthreads();
        if (sm.e.is_last && threadIdx.x == 0) {
            *I.done = 0u;
            *I.iter += 1ull;
            __threadfence();
        }
        return;
    }
    UpdateArgs a{};
    a.K = I.K;
    a.H = I.H;
    a.costs = I.costs;
    a.u_nom = I.u;
    a.u_out = I.u;
    a.sigma = I.sigma;
    a.u_lo = I.u_lo;
    a.u_hi = I.u_hi;
    a.lambda = I.lambda;
    a.seed = I.seed;
    a.iter_ptr = I.iter;
    a.err = I.err;
    a.best = I.best;
    a.advance = 1;
    a.done = I.done;
    a.U_stored = I.U;
    update_step<NU>(a, h, sm.u);
    update_finish<NU>(a, I.H, sm.u);
}

// Shift a nominal sequence one step: u[h] <- u[h+1], the last step kept.
__global__ void shift_kernel(float* u, int H, int nu) {
    for (int j = threadIdx.x; j < nu; j += blockDim.x) {
        for (int h = 0; h + 1 < H; ++h) u[h * nu + j] = u[(h + 1) * nu + j];
    }
}

using BatchFn = void (*)(const BatchInst*, int, int, BatchCtl*, int);

// The persistent rollout of a layout: samples drawn in-kernel (mode 1, both
// placements) or the instances' projected samples (mode 0, fused placement).
template <int NA>
BatchFn batch_fn(int lps, int place, int mode = 1) {
    if (mode == 0) {
        if (lps == 32) return batch_rollout_kernel<NA, 32, 0, 0>;
        if (lps == 16) return batch_rollout_kernel<NA, 16, 0, 0>;
        if constexpr (Lanes<8>::SEG > NA) {
            if (lps == 8) return batch_rollout_kernel<NA, 8, 0, 0>;
        }
        return nullptr;
    }
    if (lps == 32) return place ? batch_rollout_kernel<NA, 32, 1, 1> : batch_rollout_kernel<NA, 32, 0, 1>;
    if (lps == 16) return place ? batch_rollout_kernel<NA, 16, 1, 1> : batch_rollout_kernel<NA, 16, 0, 1>;
    if constexpr (Lanes<8>::SEG > NA) {
        if (lps == 8) return place ? batch_rollout_kernel<NA, 8, 1, 1> : batch_rollout_kernel<NA, 8, 0, 1>;
    }
    return nullptr;
}

template <int NA>
size_t batch_ws_stride(int lps) {
    if (lps == 16) return ws_stride<NA, 16>();
    if (lps == 8) return ws_stride<NA, 8>();
    return ws_stride<NA, 32>();
}

template <int NA>
int batch_shape_t(int spc, int lps, int place, int max_h, BatchLaunch* L) {
    BatchFn fn = batch_fn<NA>(lps, place);
    if (!fn) return MPPI_ERR_UNSUPPORTED;
    const int spw = 32 / lps;
    spc = (spc + spw - 1) / spw * spw;
    if (spc * lps > 256) return MPPI_ERR_INVALID_ARG;
    const int max_unom = max_h * Dims<NA>::NU <= 2048 ? max_h * Dims<NA>::NU : 0;
    L->max_unom = max_unom;
    L->smem = sizeof(DevModel) + ((size_t)max_unom * sizeof(float) + 15) / 16 * 16 + (size_t)spc * batch_ws_stride<NA>(lps);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L->smem);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    int per_sm = 0, dev = 0, sms = 0;
    BatchFn fn0 = batch_fn<NA>(lps, 0, 0);  // the projected-sample form of the layout
    if (fn0) e = cudaFuncSetAttribute(fn0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L->smem);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, spc * lps, L->smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    L->grid = (per_sm > 0 ? per_sm : 1) * sms;
    L->spc = spc;
    L->lps = lps;
    L->place = place;
    L->na = NA;
    return MPPI_OK;
}

int batch_shape(int na, int spc, int lps, int place, int max_h, BatchLaunch* L) {
    if (lps == 0) lps = 32;
    if (lps != 8 && lps != 16 && lps != 32) return MPPI_ERR_INVALID_ARG;
    if (place < 0 || place > 1) return MPPI_ERR_INVALID_ARG;
    if (na == 3) return batch_shape_t<3>(spc, lps, place, max_h, L);
    if (na == 7) return batch_shape_t<7>(spc, lps, place, max_h, L);
    return MPPI_ERR_UNSUPPORTED;
}

// One batched iteration: persistent rollout over all tiles, then the update
// CTAs.  insts (device) are in execution order with tile0/row0 prefixes.
int launch_batch_iteration(const BatchInst* insts, int n, int ntiles, int nrows, BatchCtl* ctl, const BatchLaunch& L,
                           cudaStream_t s) {
    if (n <= 0) return MPPI_OK;
    BatchFn fn = L.na == 3 ? batch_fn<3>(L.lps, L.place, L.mode) : batch_fn<7>(L.lps, L.place, L.mode);
    if (!fn) return MPPI_ERR_UNSUPPORTED;
    fn<<<L.grid, L.spc * L.lps, L.smem, s>>>(insts, n, ntiles, ctl, L.max_unom);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    if (L.sel_P > 0) {  // elite thresholds of the instances that use them
        const size_t sm = (size_t)(L.sel_P <= 1024 ? 2048 : L.sel_P) * sizeof(unsigned long long);
        if (sm > 48 * 1024) {
            e = cudaFuncSetAttribute(batch_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return MPPI_ERR_CUDA;
        }
        batch_select_kernel<<<n, 1024, sm, s>>>(insts, n);
        e = cudaGetLastError();
        if (e != cudaSuccess) return MPPI_ERR_CUDA;
    }
    if (L.na == 3) batch_update_kernel<6><<<nrows, 256, 0, s>>>(insts, n);
    else batch_update_kernel<14><<<nrows, 256, 0, s>>>(insts, n);
    return cudaGetLastError() == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

MPPI_BOUNDS_READER(bounds_word_batch)

int launch_shift(float* u, int H, int nu, cudaStream_t s) {
    shift_kernel<<<1, 32, 0, s>>>(u, H, nu);
    return cudaGetLastError() == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

}  // namespace mppi

// ---------------------------------------------------------------------------
// autotuner table: "key spc order lps place ms" lines in a text file
// ---------------------------------------------------------------------------
namespace {

std::mutex g_tune_mu;

std::string tune_path() {
    const char* p = std::getenv("MPPI_TUNE_FILE");
    if (p && *p) return p;
    const char* home = std::getenv("HOME");
    return std::string(home && *home ? home : "/tmp") + "/.cache/mppi_tune.txt";
}

}  // namespace

extern "C" int mppi_tune_lookup(const char* key, int* spc, int* order, int* lps, int* place) {
    if (!key || !spc || !order || !lps || !place) return MPPI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    FILE* f = std::fopen(tune_path().c_str(), "r");
    if (!f) return MPPI_ERR_INVALID_ARG;
    char k[256];
    int s = 0, o = 0, l = 0, pl = 0;
    float ms = 0.0f;
    int found = MPPI_ERR_INVALID_ARG;
    while (std::fscanf(f, "%255s %d %d %d %d %f", k, &s, &o, &l, &pl, &ms) == 6) {
        if (std::strcmp(k, key) == 0) {  // the last entry for a key wins
            *spc = s;
            *order = o;
            *lps = l;
            *place = pl;
            found = MPPI_OK;
        }
    }
    std::fclose(f);
    return found;
}

extern "C" int mppi_tune_store(const char* key, int spc, int order, int lps, int place, float ms) {
    if (!key || !*key || std::strlen(key) > 255 || std::strchr(key, ' ') || spc < 1 || spc > 32 || order < 0 ||
        order > 1 || (lps != 8 && lps != 16 && lps != 32) || place < 0 || place > 1)
        return MPPI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const std::string path = tune_path();
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos) {
        const std::string dir = path.substr(0, slash);  // create it without a shell
        for (size_t i = 1; i <= dir.size(); ++i)
            if (i == dir.size() || dir[i] == '/') {
                std::string part = dir.substr(0, i);
                FILE* probe = std::fopen((part + "/.").c_str(), "r");
                if (probe) std::fclose(probe);
                else mkdir(part.c_str(), 0755);
            }
    }
    FILE* f = std::fopen(path.c_str(), "a");
    if (!f) return MPPI_ERR_INVALID_ARG;
    std::fprintf(f, "%s %d %d %d %d %.6f\n", key, spc, order, lps, place, ms);
    std::fclose(f);
    return MPPI_OK;
}

// ---------------------------------------------------------------------------
// batch handle
// ---------------------------------------------------------------------------
struct mppi_batch {
    int n = 0, na = 0, nu = 0, max_h = 0, spc = 4, order = 1, lps = 32, place = 0;
    std::vector<mppi_batch_desc> desc;
    std::vector<BatchInst> inst;  // per user instance
    std::vector<int> perm;        // execution order -> user instance
    std::vector<BatchInst> host;  // descriptor table in execution order
    BatchInst* h_pinned = nullptr;
    BatchInst* d_insts = nullptr;
    int ntiles = 0;
    int nrows = 0;
    BatchLaunch L;
    BatchCtl* d_ctl = nullptr;
    float* d_pool = nullptr;  // costs, sigma, bounds, best (per instance)
    unsigned long long* d_iter = nullptr;
    unsigned int* d_done = nullptr;
    int* d_err = nullptr;
    std::string key;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t gstream = nullptr;
    // full Eq. 8 and the projection, per instance (user order)
    std::vector<float*> d_eq8;       // Sigma, L (H x nu x nu each), then the elite indices
    std::vector<unsigned long long*> d_sel;
    std::vector<float*> d_Ubuf;      // H x K x nu projected samples
    std::vector<void*> d_qp;         // projection classes and factors
    int qp_iters = 0;
    float qp_dt = 0.0f;
};

namespace {

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return MPPI_OK;
    if (e == cudaErrorMemoryAllocation) return MPPI_ERR_OOM;
    return MPPI_ERR_CUDA;
}

// Execution order (as given, or longest first: estimated work
// H x (1 + boxes/4) x K, largest first) and the tile/row prefixes.
void build_order(mppi_batch* b) {
    b->perm.resize(b->n);
    std::iota(b->perm.begin(), b->perm.end(), 0);
    if (b->order == 1) {
        std::vector<double> work(b->n);
        for (int i = 0; i < b->n; ++i) {
            int nb = 0;
            mppi_model_dims(b->desc[i].model, nullptr, nullptr, nullptr, &nb);
            work[i] = (double)b->desc[i].H * (1.0 + nb / 4.0) * b->desc[i].K;
        }
        std::stable_sort(b->perm.begin(), b->perm.end(), [&](int x, int y) { return work[x] > work[y]; });
    }
    b->host.resize(b->n);
    int t = 0, r = 0;
    for (int e = 0; e < b->n; ++e) {
        BatchInst I = b->inst[b->perm[e]];
        I.tile0 = t;
        I.row0 = r;
        t += (I.K + b->spc - 1) / b->spc;
        r += I.H;
        b->host[e] = I;
    }
    b->ntiles = t;
    b->nrows = r;
}

int reshape(mppi_batch* b) {
    int rc = batch_shape(b->na, b->spc, b->lps, b->place, b->max_h, &b->L);
    if (rc != MPPI_OK) return rc;
    b->spc = b->L.spc;  // rounded up to whole warps
    build_order(b);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    return MPPI_OK;
}

int enqueue_batch(mppi_batch* b, cudaStream_t s) {
    if (b->qp_iters > 0) {  // sample and project every instance's sequences (Eq. 5) into its buffer
        const int nq = 2 * b->na + 7;
        for (int i = 0; i < b->n; ++i) {
            const BatchInst& I = b->inst[i];
            const QPArgs q = qp_controller_args(b->nu, nq, I.K, I.H, b->qp_iters, b->qp_dt, b->d_qp[i], I.state, I.u,
                                                I.sigma, I.cov_sampling ? I.Lfac : nullptr, I.seed, I.iter, I.U);
            const int rc = launch_qp(q, s);
            if (rc != MPPI_OK) return rc;
        }
    }
    return launch_batch_iteration(b->d_insts, b->n, b->ntiles, b->nrows, b->d_ctl, b->L, s);
}

// The elite sort's key count for the instances that use the elite set.
void update_flags(mppi_batch* b) {
    int P = 0;
    for (const BatchInst& I : b->inst)
        if (I.elite) {
            int p = 1;
            while (p < I.K) p <<= 1;
            P = std::max(P, p);
        }
    b->L.sel_P = P;
    b->L.mode = b->qp_iters > 0 ? 0 : 1;
}

// Write the caller's state and control pointers into the execution-order
// descriptor table.
void stage_pointers(mppi_batch* b, const float* const* states, float* const* u) {
    for (int e = 0; e < b->n; ++e) {
        const int i = b->perm[e];
        b->inst[i].state = states[i];
        b->inst[i].u = u[i];
        b->host[e].state = states[i];
        b->host[e].u = u[i];
    }
}

}  // namespace

extern "C" {

int mppi_batch_destroy(mppi_batch* b) {
    if (!b) return MPPI_OK;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (float* p : b->d_eq8) cudaFree(p);
    for (unsigned long long* p : b->d_sel) cudaFree(p);
    for (float* p : b->d_Ubuf) cudaFree(p);
    for (void* p : b->d_qp) cudaFree(p);
    cudaFreeHost(b->h_pinned);
    cudaFree(b->d_insts);
    cudaFree(b->d_ctl);
    cudaFree(b->d_pool);
    cudaFree(b->d_iter);
    cudaFree(b->d_done);
    cudaFree(b->d_err);
    delete b;
    return MPPI_OK;
}

int mppi_batch_create(const mppi_batch_desc* desc, int n, mppi_batch** out) {
    if (!desc || !out || n < 1 || n > 65536) return MPPI_ERR_INVALID_ARG;
    *out = nullptr;
    int nq0 = 0;
    mppi_model_dims(desc[0].model, &nq0, nullptr, nullptr, nullptr);
    const int na = (nq0 - 7) / 2;
    if (na != 3 && na != 7) return MPPI_ERR_UNSUPPORTED;
    for (int i = 0; i < n; ++i) {
        int nq = 0;
        if (!desc[i].model || !desc[i].sigma || desc[i].K < 1 || desc[i].K > (1 << 20) || desc[i].H < 1 ||
            desc[i].H > 1024 || !(desc[i].lambda > 0.0f))
            return MPPI_ERR_INVALID_ARG;
        mppi_model_dims(desc[i].model, &nq, nullptr, nullptr, nullptr);
        if (nq != nq0) return MPPI_ERR_INVALID_ARG;
    }
    mppi_batch* b = new (std::nothrow) mppi_batch();
    if (!b) return MPPI_ERR_OOM;
    b->n = n;
    b->na = na;
    b->nu = 2 * na;
    b->desc.assign(desc, desc + n);
    for (int i = 0; i < n; ++i) b->max_h = std::max(b->max_h, desc[i].H);
    // per instance: costs K, sigma/lo/hi 3 x 16, best 2 (floats)
    std::vector<size_t> off(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        off[i] = total;
        total += ((size_t)desc[i].K + 48 + 2 + 63) / 64 * 64;
    }
    cudaError_t e = cudaMalloc(&b->d_pool, total * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_iter, n * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_done, n * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_insts, n * sizeof(BatchInst));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_pinned, n * sizeof(BatchInst));
    if (e == cudaSuccess) e = cudaMemset(b->d_iter, 0, n * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b->d_done, 0, n * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_ctl, 0, sizeof(BatchCtl));
    if (e != cudaSuccess) {
        mppi_batch_destroy(b);
        return cuda_rc(e);
    }
    std::vector<float> params(48);
    b->inst.resize(n);
    for (int i = 0; i < n; ++i) {
        const mppi_batch_desc& dsc = desc[i];
        float* base = b->d_pool + off[i];
        BatchInst& I = b->inst[i];
        std::memset(&I, 0, sizeof I);
        I.model = model_device(dsc.model);
        I.costs = base;
        I.sigma = base + dsc.K;
        I.u_lo = base + dsc.K + 16;
        I.u_hi = base + dsc.K + 32;
        I.best = base + dsc.K + 48;
        I.iter = b->d_iter + i;
        I.done = b->d_done + i;
        I.err = b->d_err + i;
        I.seed = dsc.seed;
        I.K = dsc.K;
        I.H = dsc.H;
        I.lambda = dsc.lambda;
        I.stage_unom = dsc.H * b->nu <= 2048;
        std::fill(params.begin(), params.end(), 0.0f);
        for (int j = 0; j < b->nu; ++j) {
            params[j] = dsc.sigma[j];
            model_bounds(dsc.model, j, &params[16 + j], &params[32 + j]);
        }
        e = cudaMemcpy(base + dsc.K, params.data(), 48 * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            mppi_batch_destroy(b);
            return cuda_rc(e);
        }
    }
    // autotuner key: arm size, box-count bucket, total samples, longest horizon
    int boxes = 0;
    long long ksum = 0;
    for (int i = 0; i < n; ++i) {
        int nb = 0;
        mppi_model_dims(desc[i].model, nullptr, nullptr, nullptr, &nb);
        boxes = std::max(boxes, nb);
        ksum += desc[i].K;
    }
    char key[128];
    std::snprintf(key, sizeof key, "nv%d_nb%d_n%d_K%lld_H%d", 2 * na + 6, boxes <= 0 ? 0 : (boxes <= 8 ? 8 : 16), n,
                  ksum, b->max_h);
    b->key = key;
    int spc = 0, order = 0, lps = 0, place = 0;
    if (mppi_tune_lookup(key, &spc, &order, &lps, &place) == MPPI_OK) {
        b->spc = spc;
        b->order = order;
        b->lps = lps;
        b->place = place;
    }
    b->d_eq8.assign(n, nullptr);
    b->d_sel.assign(n, nullptr);
    b->d_Ubuf.assign(n, nullptr);
    b->d_qp.assign(n, nullptr);
    int rc = reshape(b);
    if (rc != MPPI_OK) {
        mppi_batch_destroy(b);
        return rc;
    }
    *out = b;
    return MPPI_OK;
}

int mppi_batch_set_update(mppi_batch* b, int i, int n_elite, float eta, int update_cov, float cov_floor) {
    if (!b || i < -1 || i >= b->n) return MPPI_ERR_INVALID_ARG;
    if (i < 0) {
        for (int q = 0; q < b->n; ++q) {
            const int rc = mppi_batch_set_update(b, q, n_elite, eta, update_cov, cov_floor);
            if (rc != MPPI_OK) return rc;
        }
        return MPPI_OK;
    }
    BatchInst& I = b->inst[i];
    if (n_elite == 0) n_elite = I.K;
    if (n_elite < 1 || n_elite > I.K || !(eta > 0.0f && eta <= 1.0f) || update_cov < 0 || update_cov > 1 ||
        !(cov_floor >= 0.0f))
        return MPPI_ERR_INVALID_ARG;
    if (n_elite < I.K && I.K > 8192) return MPPI_ERR_UNSUPPORTED;  // the elite sort holds 8192 keys
    const int nu = b->nu;
    const size_t blk = (size_t)I.H * nu * nu;
    if (!b->d_eq8[i]) {
        float* p = nullptr;
        unsigned long long* sp = nullptr;
        cudaError_t e = cudaMalloc(&p, (2 * blk + (size_t)I.K) * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&sp, 3 * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            cudaFree(p);
            return cuda_rc(e);
        }
        // Sigma_0 = diag(sigma^2), its factor diag(sigma)
        std::vector<float> sig(nu), S(2 * blk, 0.0f);
        e = cudaMemcpy(sig.data(), I.sigma, nu * sizeof(float), cudaMemcpyDeviceToHost);
        for (int h = 0; h < I.H; ++h)
            for (int j = 0; j < nu; ++j) {
                S[((size_t)h * nu + j) * nu + j] = sig[j] * sig[j];
                S[blk + ((size_t)h * nu + j) * nu + j] = sig[j];
            }
        if (e == cudaSuccess) e = cudaMemcpy(p, S.data(), 2 * blk * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(p);
            cudaFree(sp);
            return cuda_rc(e);
        }
        b->d_eq8[i] = p;
        b->d_sel[i] = sp;
    }
    I.Sigma = b->d_eq8[i];
    I.Lfac = b->d_eq8[i] + blk;
    I.eidx = reinterpret_cast<int*>(b->d_eq8[i] + 2 * blk);
    I.sel = b->d_sel[i];
    I.n_elite = n_elite;
    I.eta = eta;
    I.update_cov = update_cov;
    I.cov_floor = cov_floor;
    if (update_cov) I.cov_sampling = 1;
    I.elite = (n_elite != I.K || eta != 1.0f || update_cov || I.cov_sampling) ? 1 : 0;
    update_flags(b);
    return reshape(b);
}

int mppi_batch_set_projection(mppi_batch* b, const float* bounds, int iters, float rho, const float* scales) {
    if (!b || iters < 0) return MPPI_ERR_INVALID_ARG;
    if (iters == 0) {
        b->qp_iters = 0;
        for (BatchInst& I : b->inst) I.U = nullptr;
        update_flags(b);
        return reshape(b);
    }
    if (!bounds) return MPPI_ERR_INVALID_ARG;
    const int nu = b->nu;
    std::vector<std::vector<unsigned char>> host(b->n);
    for (int i = 0; i < b->n; ++i) {
        const int rc = qp_build(nu, b->inst[i].H, bounds + (size_t)i * nu * 8, rho, scales, host[i]);
        if (rc != MPPI_OK) return rc;
    }
    float dt = 0.0f;
    for (int i = 0; i < b->n; ++i) {
        const float dti = model_dt(b->desc[i].model);
        if (i > 0 && dti != dt) return MPPI_ERR_INVALID_ARG;  // one time step across the batch
        dt = dti;
    }
    for (int i = 0; i < b->n; ++i) {
        BatchInst& I = b->inst[i];
        cudaFree(b->d_qp[i]);
        b->d_qp[i] = nullptr;
        cudaError_t e = cudaMalloc(&b->d_qp[i], host[i].size());
        if (e == cudaSuccess) e = cudaMemcpy(b->d_qp[i], host[i].data(), host[i].size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !b->d_Ubuf[i])
            e = cudaMalloc(&b->d_Ubuf[i], (size_t)I.H * I.K * nu * sizeof(float));
        if (e != cudaSuccess) return cuda_rc(e);
        I.U = b->d_Ubuf[i];
    }
    b->qp_iters = iters;
    b->qp_dt = dt;
    update_flags(b);
    return reshape(b);
}

int mppi_batch_set_launch(mppi_batch* b, int spc, int order) {
    if (!b || spc < 1 || spc > 32 || order < 0 || order > 1) return MPPI_ERR_INVALID_ARG;
    const int os = b->spc, oo = b->order;
    b->spc = spc;
    b->order = order;
    const int rc = reshape(b);
    if (rc != MPPI_OK) {
        b->spc = os;
        b->order = oo;
        reshape(b);
    }
    return rc;
}

int mppi_batch_get_launch(const mppi_batch* b, int* spc, int* order) {
    if (!b) return MPPI_ERR_INVALID_ARG;
    if (spc) *spc = b->spc;
    if (order) *order = b->order;
    return MPPI_OK;
}

int mppi_batch_set_layout(mppi_batch* b, int lps, int place) {
    if (!b) return MPPI_ERR_INVALID_ARG;
    if (lps == 0) lps = 32;
    if ((lps != 8 && lps != 16 && lps != 32) || place < 0 || place > 1) return MPPI_ERR_INVALID_ARG;
    const int ol = b->lps, op = b->place, os = b->spc;
    b->lps = lps;
    b->place = place;
    const int rc = reshape(b);
    if (rc != MPPI_OK) {
        b->lps = ol;
        b->place = op;
        b->spc = os;
        reshape(b);
    }
    return rc;
}

int mppi_batch_get_layout(const mppi_batch* b, int* lps, int* place) {
    if (!b) return MPPI_ERR_INVALID_ARG;
    if (lps) *lps = b->lps;
    if (place) *place = b->place;
    return MPPI_OK;
}

int mppi_batch_step(mppi_batch* b, const float* const* states, float* const* u, void* stream) {
    if (!b || !states || !u) return MPPI_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i)
        if (!states[i] || !u[i]) return MPPI_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    NvtxRange r("mppi_batch_step");
    stage_pointers(b, states, u);
    cudaError_t e = cudaMemcpyAsync(b->d_insts, b->host.data(), b->n * sizeof(BatchInst), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_rc(e);
    return enqueue_batch(b, s);
}

int mppi_batch_step_graph(mppi_batch* b, const float* const* states, float* const* u, void* stream) {
    if (!b || !states || !u || !stream) return MPPI_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i)
        if (!states[i] || !u[i]) return MPPI_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    NvtxRange r("mppi_batch_step_graph");
    stage_pointers(b, states, u);
    // the graph's copy node reads the pinned table when it executes: rewrite
    // it only when its content changes, after any launch in flight is done
    const bool changed = std::memcmp(b->h_pinned, b->host.data(), b->n * sizeof(BatchInst)) != 0;
    if (changed) {
        if (b->gexec) {
            cudaError_t e = cudaStreamSynchronize(b->gstream);
            if (e != cudaSuccess) return cuda_rc(e);
        }
        std::memcpy(b->h_pinned, b->host.data(), b->n * sizeof(BatchInst));
    }
    if (!b->gexec || b->gstream != s) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->gexec = nullptr;
        b->graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_rc(e);
        e = cudaMemcpyAsync(b->d_insts, b->h_pinned, b->n * sizeof(BatchInst), cudaMemcpyHostToDevice, s);
        int rc = e == cudaSuccess ? enqueue_batch(b, s) : cuda_rc(e);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s, &g);
        if (rc != MPPI_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc != MPPI_OK ? rc : cuda_rc(e);
        }
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_rc(e);
        }
        b->graph = g;
        b->gstream = s;
    }
    return cuda_rc(cudaGraphLaunch(b->gexec, s));
}

int mppi_batch_sync(mppi_batch* b, int* errors, void* stream) {
    if (!b) return MPPI_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_rc(e);
    std::vector<int> err(b->n);
    e = cudaMemcpy(err.data(), b->d_err, b->n * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, b->n * sizeof(int));
    if (e != cudaSuccess) return cuda_rc(e);
    int worst = MPPI_OK;
    for (int i = 0; i < b->n; ++i) {
        const int c = (err[i] & ERRB_TIMEOUT) ? MPPI_ERR_TIMEOUT
                      : (err[i] & ERRB_CHOLESKY) ? MPPI_ERR_CHOLESKY
                      : (err[i] & ERRB_NONFINITE) ? MPPI_ERR_NONFINITE
                                                  : MPPI_OK;
        if (errors) errors[i] = c;
        if (c != MPPI_OK && worst == MPPI_OK) worst = c;
    }
    return worst;
}

int mppi_batch_iteration(mppi_batch* b, int i, uint64_t* it, void* stream) {
    if (!b || i < 0 || i >= b->n || !it) return MPPI_ERR_INVALID_ARG;
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, b->d_iter + i, sizeof v, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_rc(e);
    *it = v;
    return MPPI_OK;
}

int mppi_batch_set_iteration(mppi_batch* b, int i, uint64_t it, void* stream) {
    if (!b || i < -1 || i >= b->n) return MPPI_ERR_INVALID_ARG;
    std::vector<unsigned long long> v(b->n, (unsigned long long)it);
    cudaError_t e;
    if (i < 0)
        e = cudaMemcpyAsync(b->d_iter, v.data(), b->n * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream);
    else
        e = cudaMemcpyAsync(b->d_iter + i, v.data(), sizeof(unsigned long long), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return cuda_rc(e);
}

const float* mppi_batch_costs(const mppi_batch* b, int i) {
    if (!b || i < 0 || i >= b->n) return nullptr;
    return b->inst[i].costs;
}

int mppi_batch_autotune(mppi_batch* b, const float* const* states, float* const* u, int reps, void* stream,
                        float* best_ms) {
    if (!b || !states || !u || reps < 1 || !stream) return MPPI_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<unsigned long long> iters(b->n);
    cudaError_t e = cudaMemcpyAsync(iters.data(), b->d_iter, b->n * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_rc(e);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bs = b->spc, bo = b->order, bl = b->lps, bp = b->place;
    // lanes per sample (8 only for the 3-link arms) x placement of the lone
    // ball contact's solve x samples per CTA (whole warps, <= 256 threads)
    // x instance order
    const int lpss[3] = {32, 16, 8};
    int rc = MPPI_OK;
    for (int li = 0; li < 3 && rc == MPPI_OK; ++li) {
        const int lps = lpss[li];
        if (lps == 8 && b->na != 3) continue;
        const int spw = 32 / lps;
        for (int pl = 0; pl < 2 && rc == MPPI_OK; ++pl)
            for (int sm = 1; sm <= 8 && rc == MPPI_OK; sm <<= 1)
                for (int o = 0; o < 2 && rc == MPPI_OK; ++o) {
                    const int spc = sm * spw;
                    b->spc = spc;
                    b->order = o;
                    b->lps = lps;
                    b->place = pl;
                    rc = reshape(b);
                    if (rc != MPPI_OK) break;
                    rc = mppi_batch_step(b, states, u, stream);  // warm-up
                    if (rc != MPPI_OK) break;
                    cudaEventRecord(e0, s);
                    for (int r = 0; r < reps && rc == MPPI_OK; ++r) rc = mppi_batch_step(b, states, u, stream);
                    cudaEventRecord(e1, s);
                    e = cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e != cudaSuccess) rc = cuda_rc(e);
                    ms /= reps;
                    if (ms < best) {
                        best = ms;
                        bs = spc;
                        bo = o;
                        bl = lps;
                        bp = pl;
                    }
                }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->spc = bs;
    b->order = bo;
    b->lps = bl;
    b->place = bp;
    if (rc == MPPI_OK) rc = reshape(b);
    // the tuning iterations do not count: restore the counters
    if (rc == MPPI_OK) {
        e = cudaMemcpyAsync(b->d_iter, iters.data(), b->n * sizeof(unsigned long long), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_rc(e);
    }
    if (rc == MPPI_OK) mppi_tune_store(b->key.c_str(), bs, bo, bl, bp, best);
    if (best_ms) *best_ms = best;
    return rc;
}

}  // extern "C"
