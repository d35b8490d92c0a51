// Kernels and C ABI of libmppi (see include/mppi.h).
//
// Kernels
//   rollout_kernel            (mppi_rollout.cuh) one lane group per sample: H
//                             simulator steps with the state resident in
//                             shared memory, stage costs, cost[k].
//   update_kernel<NU>         one CTA per horizon step h: min cost, weights
//                             exp(-(c - c_min)/lambda), sum_k w_k U_k[h,:]
//                             with the samples regenerated from Philox,
//                             fixed-order tree reductions (Eq. 8a, 8d).
//   noise_kernel<NU>          materialises the Philox noise (tests).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/mppi.h"
#include "mppi_device.cuh"
#include "mppi_internal.h"
#include "mppi_kernels.cuh"
#include "mppi_rollout.cuh"
#include "mppi_task.cuh"

using namespace mppi;

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
namespace mppi {

template <int NU>
__global__ void __launch_bounds__(256) update_kernel(UpdateArgs a) {
    cudaGridDependencySynchronize();  // the rollout's costs and samples
    cudaTriggerProgrammaticLaunchCompletion();
    __shared__ UpdateSmem<NU> sm;
    update_step<NU>(a, blockIdx.x, sm);
    update_finish<NU>(a, gridDim.x, sm);
}

template <int NU>
__global__ void noise_kernel(NoiseArgs a) {
    const size_t n = (size_t)a.K * a.H * NU;
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % NU);
        const int h = (int)((i / NU) % a.H);
        const int k = (int)(i / ((size_t)NU * a.H));
        const uint4 wv = philox4x32_10(make_uint4((uint32_t)(j >> 2), (uint32_t)h, (uint32_t)k, (uint32_t)a.iter), key);
        a.eps[i] = __fmul_rn(a.sigma[j], block_normal(wv, j & 3));
    }
}

// Elite threshold of one controller (one CTA of 1024 threads; the sort in
// mppi_kernels.cuh).
__global__ void __launch_bounds__(1024) elite_select_kernel(const float* costs, int K, int P, int n_elite,
                                                            unsigned long long* sel, int* eidx) {
    extern __shared__ unsigned long long keys[];
    __shared__ int nfin;
    elite_select_block(costs, K, P, n_elite, sel, eidx, keys, nfin);
}

template <int NU>
__global__ void __launch_bounds__(256) elite_update_kernel(EliteArgs a) {
    __shared__ EliteSmem<NU> sm;
    elite_update_step<NU>(a, blockIdx.x, sm);
    if (a.advance) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned t = atomicAdd(a.done, 1u);
            sm.is_last = (t == gridDim.x - 1);
        }
        __syncthreads();
        if (sm.is_last && threadIdx.x == 0) {
            *a.done = 0u;
            *const_cast<unsigned long long*>(a.iter_ptr) += 1ull;
            __threadfence();
        }
    }
}

__global__ void philox_kernel(int n, const uint4* ctr, uint2 key, uint4* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

}  // namespace mppi

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
namespace {

int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return MPPI_OK;
    if (e == cudaErrorMemoryAllocation) return MPPI_ERR_OOM;
    return MPPI_ERR_CUDA;
}

// Kernel launch, optionally as a programmatic dependent of the stream's
// previous kernel (its launch overlaps that kernel's tail; the kernel waits
// in cudaGridDependencySynchronize before reading what that kernel wrote).
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                          Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace

namespace mppi {

int launch_rollout(int na, int mode, const RolloutArgs& a, int spc, cudaStream_t s) {
    if (a.n <= 0) return MPPI_OK;
    if (na == 3) return launch_rollout_na3(mode, a, spc, s);
    if (na == 7) return launch_rollout_na7(mode, a, spc, s);
    return MPPI_ERR_UNSUPPORTED;
}

int launch_update(int nu, const UpdateArgs& a_in, int H, cudaStream_t s) {
    UpdateArgs a = a_in;
    a.H = H;
    cudaError_t e;
    if (nu == 6) e = launch_kernel(update_kernel<6>, dim3(H), dim3(256), 0, s, a.pdl != 0, a);
    else if (nu == 14) e = launch_kernel(update_kernel<14>, dim3(H), dim3(256), 0, s, a.pdl != 0, a);
    else return MPPI_ERR_UNSUPPORTED;
    return cuda_fail(e != cudaSuccess ? e : cudaGetLastError());
}

int launch_noise(int nu, const NoiseArgs& a, cudaStream_t s) {
    const size_t n = (size_t)a.K * a.H * nu;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
    if (nu == 6) noise_kernel<6><<<grid, 256, 0, s>>>(a);
    else if (nu == 14) noise_kernel<14><<<grid, 256, 0, s>>>(a);
    else return MPPI_ERR_UNSUPPORTED;
    return cuda_fail(cudaGetLastError());
}



// Parse the scene blob into the device representation.
int parse_model_blob(const void* blob, size_t len, DevModel* out, HostModelInfo* info) {
    // Values are read one at a time with memcpy (the blob need not be
    // 8-byte aligned) and nothing is allocated unless `info` is given.
    if (!blob || !out || len < 16) return MPPI_ERR_INVALID_ARG;
    const unsigned char* raw = static_cast<const unsigned char*>(blob);
    uint32_t h[4];
    std::memcpy(h, raw, 16);
    if (h[0] != 0x4950504Du || h[1] != 1u) return MPPI_ERR_INVALID_ARG;
    const size_t n = h[2];
    if (n < 23 || len < 16 + 8 * n) return MPPI_ERR_INVALID_ARG;
    auto v = [raw](size_t i) {
        double x;
        std::memcpy(&x, raw + 16 + 8 * i, 8);
        return x;
    };
    const int na = (int)v(0), nb = (int)v(1), maxc = (int)v(2);
    if (na < 1 || na > MAXL || nb < 0 || nb > MAXB || maxc < 1 || maxc > 16) return MPPI_ERR_INVALID_ARG;
    if (maxc > MAXC) return MPPI_ERR_UNSUPPORTED;  // more contacts than the device solver keeps
    const int nq = 2 * na + 7, nv = 2 * na + 6;
    if (n != 23 + 2 * (12 + 39 * (size_t)na) + 6 * (size_t)nb + (size_t)(nq + nv)) return MPPI_ERR_INVALID_ARG;
    DevModel M;
    std::memset(&M, 0, sizeof M);
    M.na = na;
    M.nb = nb;
    M.maxc = maxc;
    M.dt = (float)v(3);
    M.sweeps = (int)v(4);
    M.mu = (float)v(5);
    M.imp = (float)v(6);
    M.erp = (float)v(7);
    for (int k = 0; k < 3; ++k) M.g[k] = (float)v(8 + k);
    M.floor_z = (float)v(11);
    M.rb = (float)v(12);
    M.mb = (float)v(13);
    M.Ib = (float)v(14);
    for (int k = 0; k < 3; ++k) M.goal[k] = (float)v(15 + k);
    M.w_goal = (float)v(18);
    M.w_u = (float)v(19);
    M.w_pen = (float)v(20);
    M.w_obst = (float)v(21);
    M.w_grasp = (float)v(22);
    if (!(M.dt > 0) || M.sweeps < 0 || M.sweeps > 1000 || !(M.imp > 0 && M.imp <= 1) || !(M.mb > 0) || !(M.Ib > 0))
        return MPPI_ERR_INVALID_ARG;
    size_t o = 23;
    for (int a = 0; a < 2; ++a) {
        for (int k = 0; k < 9; ++k) M.baseR[a][k] = (float)v(o++);
        for (int k = 0; k < 3; ++k) M.basep[a][k] = (float)v(o++);
        for (int i = 0; i < na; ++i) {
            DevLink& L = M.link[a][i];
            for (int k = 0; k < 9; ++k) L.FR[k] = (float)v(o++);
            for (int k = 0; k < 3; ++k) L.Fp[k] = (float)v(o++);
            L.mass = (float)v(o++);
            for (int k = 0; k < 3; ++k) L.com[k] = (float)v(o++);
            double I[9];
            for (int k = 0; k < 9; ++k) I[k] = v(o++);
            L.I[0] = (float)I[0];
            L.I[1] = (float)I[4];
            L.I[2] = (float)I[8];
            L.I[3] = (float)(0.5 * (I[1] + I[3]));
            L.I[4] = (float)(0.5 * (I[2] + I[6]));
            L.I[5] = (float)(0.5 * (I[5] + I[7]));
            for (int k = 0; k < 3; ++k) L.s0[k] = (float)v(o++);
            for (int k = 0; k < 3; ++k) L.s1[k] = (float)v(o++);
            L.rcap = (float)v(o++);
            const double damping = v(o++), kv = v(o++);
            L.D = (float)(damping + kv);
            L.gear = (float)v(o++);
            L.tau_max = (float)v(o++);
            L.u_lo = (float)v(o++);
            L.u_hi = (float)v(o++);
            L.gravcomp = (float)v(o++);
            if (!(L.mass > 0)) return MPPI_ERR_INVALID_ARG;
        }
    }
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < 6; ++k) M.box[b][k] = (float)v(o++);
    if (info) {
        info->na = na;
        info->nb = nb;
        info->x0.assign(nq + nv, 0.0f);
        for (int k = 0; k < nq + nv; ++k) info->x0[k] = (float)v(o + k);
    }
    *out = M;
    return MPPI_OK;
}

MPPI_BOUNDS_READER(bounds_word_api)

}  // namespace mppi

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
struct mppi_model {
    DevModel host;
    DevModel* dev = nullptr;
    HostModelInfo info;
    int device = 0;
};

struct mppi_ctx {
    const mppi_model* m = nullptr;
    int K = 0, H = 0, spc = 4;
    int lps = 32, place = 0;  // lanes per sample, placement of the lone ball contact's solve
    bool spc_auto = true;     // spc is the library's choice for the layout
    int spc_alt = 0, spc_alt_lps = 0;  // the default shape of another layout (the task suite's)
    float lambda = 1.0f;
    uint64_t seed = 0;
    float* d_sigma = nullptr;
    float* h_stage = nullptr;  // pinned staging of mppi_step_host: state, u_nom, u_nom_out
    float* d_stage = nullptr;  // its device copy: state, u_nom (updated in place)
    float* d_ulo = nullptr;
    float* d_uhi = nullptr;
    float* d_costs = nullptr;
    float* d_best = nullptr;
    int* d_err = nullptr;
    unsigned long long* d_iter = nullptr;
    unsigned int* d_done = nullptr;
    // captured solve
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    const float* g_state = nullptr;
    float* g_u = nullptr;
    float* g_best = nullptr;
    int g_iters = 0;
    cudaStream_t g_stream = nullptr;
    // profiling
    int prof_cap = 0, prof_n = 0;
    std::vector<cudaEvent_t> prof_ev;  // 4 per recorded iteration: start, projected, rolled out, updated
    unsigned long long* d_stats = nullptr;
    float* d_U = nullptr;  // sampled controls of the last rollout (H x K x nu), when it fits
    // full Eq. 8 (elite set, learning rate, covariance blocks)
    int n_elite = 0;
    float eta = 1.0f, cov_floor = 0.0f;
    int update_cov = 0, cov_sampling = 0;
    float* d_Sigma = nullptr;  // H x nu x nu
    float* d_L = nullptr;      // H x nu x nu factors used for sampling
    unsigned long long* d_sel = nullptr;
    int* d_eidx = nullptr;     // elite indices (K)
    float* d_bestU = nullptr;  // H x nu
    // QP smoothing projection (Eq. 5)
    int qp_iters = 0;
    float qp_dt = 0.0f;
    void* d_qp = nullptr;  // nu QPClass records, then per joint the inverse (H <= 32) or 2H band rows
    size_t qp_bytes = 0;
    // ball-task cost suite (Sec. IV-B)
    DevTask* d_task = nullptr;
    int task_on = 0;
};

namespace mppi {
const DevModel* model_device(const mppi_model* m) { return m ? m->dev : nullptr; }
float model_dt(const mppi_model* m) { return m->host.dt; }
void model_bounds(const mppi_model* m, int j, float* lo, float* hi) {
    const int na = m->info.na;
    *lo = m->host.link[j / na][j % na].u_lo;
    *hi = m->host.link[j / na][j % na].u_hi;
}
}  // namespace mppi

extern "C" {

const char* mppi_strerror(int code) {
    switch (code) {
        case MPPI_OK: return "ok";
        case MPPI_ERR_INVALID_ARG: return "invalid argument";
        case MPPI_ERR_OOM: return "out of memory";
        case MPPI_ERR_CUDA: return "CUDA error";
        case MPPI_ERR_NONFINITE: return "non-finite costs or state";
        case MPPI_ERR_TIMEOUT: return "bounded device wait timed out";
        case MPPI_ERR_ADMISSION: return "request does not fit the admission budget";
        case MPPI_ERR_CHOLESKY: return "mass matrix lost positive definiteness";
        case MPPI_ERR_UNSUPPORTED: return "model outside the compiled variants";
        default: return "unknown error";
    }
}

int mppi_model_load(const void* blob, size_t len, mppi_model** out) {
    if (!out) return MPPI_ERR_INVALID_ARG;
    *out = nullptr;
    mppi_model* m = new (std::nothrow) mppi_model();
    if (!m) return MPPI_ERR_OOM;
    int rc = parse_model_blob(blob, len, &m->host, &m->info);
    if (rc != MPPI_OK) {
        delete m;
        return rc;
    }
    cudaGetDevice(&m->device);
    cudaError_t e = cudaMalloc(&m->dev, sizeof(DevModel));
    if (e == cudaSuccess) e = cudaMemcpy(m->dev, &m->host, sizeof(DevModel), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (m->dev) cudaFree(m->dev);
        delete m;
        return cuda_fail(e);
    }
    *out = m;
    return MPPI_OK;
}

void mppi_model_free(mppi_model* m) {
    if (!m) return;
    if (m->dev) cudaFree(m->dev);
    delete m;
}

int mppi_model_dims(const mppi_model* m, int* nq, int* nv, int* nu, int* n_boxes) {
    if (!m) return MPPI_ERR_INVALID_ARG;
    const int na = m->info.na;
    if (nq) *nq = 2 * na + 7;
    if (nv) *nv = 2 * na + 6;
    if (nu) *nu = 2 * na;
    if (n_boxes) *n_boxes = m->info.nb;
    return MPPI_OK;
}

int mppi_model_home(const mppi_model* m, float* x0) {
    if (!m || !x0) return MPPI_ERR_INVALID_ARG;
    std::memcpy(x0, m->info.x0.data(), m->info.x0.size() * sizeof(float));
    return MPPI_OK;
}

int mppi_destroy(mppi_ctx* c) {
    if (!c) return MPPI_OK;
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    cudaFree(c->d_stats);
    cudaFree(c->d_U);
    cudaFree(c->d_Sigma);
    cudaFree(c->d_L);
    cudaFree(c->d_sel);
    cudaFree(c->d_eidx);
    cudaFree(c->d_qp);
    cudaFree(c->d_task);
    cudaFree(c->d_bestU);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    cudaFree(c->d_sigma);
    cudaFreeHost(c->h_stage);
    cudaFree(c->d_stage);
    cudaFree(c->d_ulo);
    cudaFree(c->d_uhi);
    cudaFree(c->d_costs);
    cudaFree(c->d_best);
    cudaFree(c->d_err);
    cudaFree(c->d_iter);
    cudaFree(c->d_done);
    delete c;
    return MPPI_OK;
}

// Samples per rollout CTA when the caller sets none: the shape that puts
// the K samples on the SMs in the fewest waves with the least load on the
// busiest SM (occupancy of the sampling rollout kernel of the layout).
static int default_spc_for(const mppi_ctx* c, int lps) {
    const int unom = c->H * 2 * c->m->info.na <= 2048 ? c->H * 2 * c->m->info.na : 0;
    return c->m->info.na == 3 ? choose_spc_na3(lps, c->K, unom) : choose_spc_na7(lps, c->K, unom);
}
static int default_spc(const mppi_ctx* c) { return default_spc_for(c, c->lps); }

// Samples per CTA for a launch in layout lps: the handle's shape when lps is
// its layout, else (the ball-task suite runs on 32 lanes per sample) the
// default shape for lps, or the handle's shape capped at 512 threads when
// the caller chose it.
static int launch_spc(mppi_ctx* c, int lps) {
    if (lps == c->lps) return c->spc;
    if (c->spc_auto) {
        if (c->spc_alt_lps != lps) {
            c->spc_alt = default_spc_for(c, lps);
            c->spc_alt_lps = lps;
        }
        return c->spc_alt;
    }
    return std::min(c->spc, 512 / lps);
}

int mppi_create(const mppi_model* m, int K, int H, float lambda, const float* sigma, uint64_t seed, mppi_ctx** out) {
    if (!m || !out || !sigma || K < 1 || K > (1 << 20) || H < 1 || H > 1024 || !(lambda > 0.0f))
        return MPPI_ERR_INVALID_ARG;
    *out = nullptr;
    if (m->info.na != 3 && m->info.na != 7) return MPPI_ERR_UNSUPPORTED;
    mppi_ctx* c = new (std::nothrow) mppi_ctx();
    if (!c) return MPPI_ERR_OOM;
    c->m = m;
    c->K = K;
    c->H = H;
    c->lambda = lambda;
    c->seed = seed;
    c->n_elite = K;
    c->lps = default_lps(K);
    c->spc = default_spc(c);
    const int nu = 2 * m->info.na;
    std::vector<float> lo(nu), hi(nu);
    for (int j = 0; j < nu; ++j) {
        lo[j] = m->host.link[j / m->info.na][j % m->info.na].u_lo;
        hi[j] = m->host.link[j / m->info.na][j % m->info.na].u_hi;
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&c->d_sigma, nu * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ulo, nu * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_uhi, nu * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_costs, (size_t)K * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_best, 2 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_iter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_done, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_sigma, sigma, nu * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_ulo, lo.data(), nu * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_uhi, hi.data(), nu * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_iter, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->d_done, 0, sizeof(unsigned int));
    // the update reads the rollout's samples instead of regenerating them
    // when the buffer is modest
    const size_t ubytes = (size_t)K * H * nu * sizeof(float);
    if (e == cudaSuccess && ubytes <= ((size_t)256 << 20)) e = cudaMalloc(&c->d_U, ubytes);
    if (e != cudaSuccess) {
        mppi_destroy(c);
        return cuda_fail(e);
    }
    *out = c;
    return MPPI_OK;
}

int mppi_profile(mppi_ctx* c, int n) {
    if (!c || n < 0 || n > (1 << 20)) return MPPI_ERR_INVALID_ARG;
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->prof_cap = 0;
    c->prof_n = 0;
    if (n == 0) return MPPI_OK;
    cudaError_t e = cudaSuccess;
    if (!c->d_stats) e = cudaMalloc(&c->d_stats, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->d_stats, 0, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e);
    c->prof_ev.resize(4 * (size_t)n);
    for (auto& ev : c->prof_ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    c->prof_cap = n;
    return MPPI_OK;
}

int mppi_profile_read(mppi_ctx* c, int* n, float* rollout_ms, float* update_ms, double* contacts_per_step,
                      double* box_tests_per_step) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    float tr = 0.0f, tu = 0.0f;
    for (int i = 0; i < c->prof_n; ++i) {
        cudaError_t e = cudaEventSynchronize(c->prof_ev[4 * i + 3]);
        float a = 0.0f, b = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, c->prof_ev[4 * i + 1], c->prof_ev[4 * i + 2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, c->prof_ev[4 * i + 2], c->prof_ev[4 * i + 3]);
        if (e != cudaSuccess) return cuda_fail(e);
        tr += a;
        tu += b;
    }
    unsigned long long st[4] = {0, 0, 0, 0};
    if (c->d_stats) {
        cudaError_t e = cudaMemcpy(st, c->d_stats, sizeof st, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (n) *n = c->prof_n;
    if (rollout_ms) *rollout_ms = tr;
    if (update_ms) *update_ms = tu;
    if (contacts_per_step) *contacts_per_step = st[0] ? (double)st[1] / (double)st[0] : 0.0;
    if (box_tests_per_step) *box_tests_per_step = st[0] ? (double)st[2] / (double)st[0] : 0.0;
    return MPPI_OK;
}

int mppi_profile_lone_contacts(mppi_ctx* c, double* lone_per_step) {
    if (!c || !lone_per_step) return MPPI_ERR_INVALID_ARG;
    unsigned long long st[4] = {0, 0, 0, 0};
    if (c->d_stats) {
        cudaError_t e = cudaMemcpy(st, c->d_stats, sizeof st, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    *lone_per_step = st[0] ? (double)st[3] / (double)st[0] : 0.0;
    return MPPI_OK;
}

int mppi_profile_projection(mppi_ctx* c, float* qp_ms) {
    if (!c || !qp_ms) return MPPI_ERR_INVALID_ARG;
    float tq = 0.0f;
    for (int i = 0; i < c->prof_n; ++i) {
        cudaError_t e = cudaEventSynchronize(c->prof_ev[4 * i + 3]);
        float a = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, c->prof_ev[4 * i], c->prof_ev[4 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e);
        tq += a;
    }
    *qp_ms = tq;
    return MPPI_OK;
}

int mppi_set_update(mppi_ctx* c, int n_elite, float eta, int update_cov, float cov_floor) {
    if (!c || n_elite < 1 || n_elite > c->K || !(eta > 0.0f && eta <= 1.0f) || update_cov < 0 || update_cov > 1 ||
        !(cov_floor >= 0.0f))
        return MPPI_ERR_INVALID_ARG;
    if (n_elite < c->K && c->K > 8192) return MPPI_ERR_UNSUPPORTED;  // the elite sort holds 8192 keys
    const int nu = 2 * c->m->info.na;
    if (update_cov && !c->d_U) return MPPI_ERR_UNSUPPORTED;  // needs the stored samples
    cudaError_t e = cudaSuccess;
    const size_t blk = (size_t)c->H * nu * nu;
    if (!c->d_Sigma) {
        e = cudaMalloc(&c->d_Sigma, blk * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&c->d_L, blk * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&c->d_sel, 3 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&c->d_eidx, (size_t)c->K * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&c->d_bestU, (size_t)c->H * nu * sizeof(float));
        if (e != cudaSuccess) return cuda_fail(e);
        // Sigma_0 = diag(sigma^2), its factor diag(sigma)
        std::vector<float> sig(nu), S(blk, 0.0f), Lh(blk, 0.0f);
        e = cudaMemcpy(sig.data(), c->d_sigma, nu * sizeof(float), cudaMemcpyDeviceToHost);
        for (int h = 0; h < c->H; ++h)
            for (int j = 0; j < nu; ++j) {
                S[((size_t)h * nu + j) * nu + j] = sig[j] * sig[j];
                Lh[((size_t)h * nu + j) * nu + j] = sig[j];
            }
        if (e == cudaSuccess) e = cudaMemcpy(c->d_Sigma, S.data(), blk * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->d_L, Lh.data(), blk * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    c->n_elite = n_elite;
    c->eta = eta;
    c->update_cov = update_cov;
    c->cov_floor = cov_floor;
    if (update_cov) c->cov_sampling = 1;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    return MPPI_OK;
}

int mppi_get_covariance(mppi_ctx* c, float* Sigma, void* stream) {
    if (!c || !Sigma) return MPPI_ERR_INVALID_ARG;
    const int nu = 2 * c->m->info.na;
    const size_t blk = (size_t)c->H * nu * nu;
    if (!c->d_Sigma) {  // fixed diagonal Sigma = diag(sigma^2)
        std::vector<float> sig(nu), S(blk, 0.0f);
        cudaError_t e = cudaMemcpy(sig.data(), c->d_sigma, nu * sizeof(float), cudaMemcpyDeviceToHost);
        for (int h = 0; h < c->H; ++h)
            for (int j = 0; j < nu; ++j) S[((size_t)h * nu + j) * nu + j] = sig[j] * sig[j];
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(Sigma, S.data(), blk * sizeof(float), cudaMemcpyHostToDevice, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        return cuda_fail(e);
    }
    return cuda_fail(cudaMemcpyAsync(Sigma, c->d_Sigma, blk * sizeof(float), cudaMemcpyDeviceToDevice,
                                     (cudaStream_t)stream));
}

int mppi_set_covariance(mppi_ctx* c, const float* Sigma, void* stream) {
    if (!c || !Sigma) return MPPI_ERR_INVALID_ARG;
    if (!c->d_Sigma) {
        int rc = mppi_set_update(c, c->n_elite, c->eta, c->update_cov, c->cov_floor);
        if (rc != MPPI_OK) return rc;
    }
    const int nu = 2 * c->m->info.na;
    const size_t blk = (size_t)c->H * nu * nu;
    std::vector<float> S(blk), Lh(blk, 0.0f);
    cudaError_t e = cudaMemcpyAsync(S.data(), Sigma, blk * sizeof(float), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int h = 0; h < c->H; ++h) {  // factor on the host (FP64), once
        const float* A = &S[(size_t)h * nu * nu];
        std::vector<double> L(nu * nu, 0.0);
        for (int j = 0; j < nu; ++j) {
            double d = A[j * nu + j];
            for (int k = 0; k < j; ++k) d -= L[j * nu + k] * L[j * nu + k];
            if (!(d > 0.0)) return MPPI_ERR_INVALID_ARG;  // not positive definite
            d = std::sqrt(d);
            L[j * nu + j] = d;
            for (int r = j + 1; r < nu; ++r) {
                double t = A[r * nu + j];
                for (int k = 0; k < j; ++k) t -= L[r * nu + k] * L[j * nu + k];
                L[r * nu + j] = t / d;
            }
        }
        for (int q = 0; q < nu * nu; ++q) Lh[(size_t)h * nu * nu + q] = (float)L[q];
    }
    e = cudaMemcpy(c->d_Sigma, S.data(), blk * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_L, Lh.data(), blk * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e);
    c->cov_sampling = 1;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    return MPPI_OK;
}

int mppi_best_controls(mppi_ctx* c, float* U_best, void* stream) {
    if (!c || !U_best || !c->d_bestU) return MPPI_ERR_INVALID_ARG;
    const int nu = 2 * c->m->info.na;
    return cuda_fail(cudaMemcpyAsync(U_best, c->d_bestU, (size_t)c->H * nu * sizeof(float), cudaMemcpyDeviceToDevice,
                                     (cudaStream_t)stream));
}

static void drop_graph(mppi_ctx* c);

int mppi_set_launch(mppi_ctx* c, int spc) {
    if (!c || spc < 0 || spc > 32) return MPPI_ERR_INVALID_ARG;
    const int v = spc == 0 ? default_spc(c) : spc;
    if (v * c->lps > 512) return MPPI_ERR_INVALID_ARG;
    if (v != c->spc) drop_graph(c);  // a captured solve holds the old launch shape
    c->spc = v;
    c->spc_auto = spc == 0;
    return MPPI_OK;
}

int mppi_set_layout(mppi_ctx* c, int lps, int place) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    if (lps == 0) lps = 32;
    if ((lps != 8 && lps != 16 && lps != 32) || place < 0 || place > 1) return MPPI_ERR_INVALID_ARG;
    if (lps == 8 && c->m->info.na != 3) return MPPI_ERR_UNSUPPORTED;  // a 7-link arm needs 8 lanes per arm
    if (!c->spc_auto && c->spc * lps > 512) return MPPI_ERR_INVALID_ARG;
    if (lps != c->lps || place != c->place) drop_graph(c);
    c->lps = lps;
    c->place = place;
    if (c->spc_auto) c->spc = default_spc(c);  // the default shape follows the layout
    return MPPI_OK;
}

int mppi_get_layout(const mppi_ctx* c, int* lps, int* place, int* spc) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    if (lps) *lps = c->lps;
    if (place) *place = c->place;
    if (spc) *spc = c->spc;
    return MPPI_OK;
}

static RolloutArgs philox_args(mppi_ctx* c, const float* state, const float* u_nom) {
    RolloutArgs a{};
    a.model = c->m->dev;
    a.n = c->K;
    a.H = c->H;
    a.states = state;
    a.state_stride = 0;
    a.u_nom = u_nom;
    a.sigma = c->d_sigma;
    a.seed = c->seed;
    a.iter_ptr = c->d_iter;
    a.costs = c->d_costs;
    a.err = c->d_err;
    a.stage_unom = c->H * 2 * c->m->info.na <= 2048;
    a.U_store = c->d_U;
    a.Lfac = c->cov_sampling ? c->d_L : nullptr;
    a.task = c->task_on ? c->d_task : nullptr;
    a.lps = a.task ? 32 : c->lps;  // the ball-task suite runs on 32 lanes per sample
    a.place = a.task ? 0 : c->place;
    return a;
}

static void drop_graph(mppi_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
}

// Projection launch: sequence i = j * K + k (a warp's sequences share a
// joint, hence a band factor); output U[h][k][j] (h-major sample buffer).
static int launch_projection(mppi_ctx* c, const float* state, const float* u_nom, cudaStream_t s) {
    const int na = c->m->info.na, nu = 2 * na, nq = 2 * na + 7;
    const QPArgs q = qp_controller_args(nu, nq, c->K, c->H, c->qp_iters, c->qp_dt, c->d_qp, state, u_nom, c->d_sigma,
                                        c->cov_sampling ? c->d_L : nullptr, c->seed, c->d_iter, c->d_U);
    return launch_qp(q, s);
}

}  // extern "C"

namespace mppi {
// Per-joint projection data of one controller: nu class records, then per
// joint the dense inverse (H <= 32, warp kernel) or the band factor rows.
int qp_build(int nu, int H, const float* bounds, float rho, const float* scales, std::vector<unsigned char>& host) {
    static const float kDefault[4] = {MPPI_QP_SCALE_POSITION, MPPI_QP_SCALE_VELOCITY, MPPI_QP_SCALE_ACCELERATION,
                                      MPPI_QP_SCALE_JERK};
    const float* sc = scales ? scales : kDefault;
    for (int j = 0; j < nu; ++j) {
        const int rc = qp_validate(bounds + 8 * j, sc, rho);
        if (rc != MPPI_OK) return rc;
    }
    if (H > MPPI_QP_MAX_H) return MPPI_ERR_UNSUPPORTED;
    const bool warp = H <= QP_WARP_MAX_H;
    const size_t per = warp ? 32 * 32 * sizeof(float) : 2 * (size_t)H * sizeof(float4);
    host.assign((size_t)nu * sizeof(QPClass) + (size_t)nu * per, 0);
    QPClass* cls = reinterpret_cast<QPClass*>(host.data());
    unsigned char* fac = host.data() + (size_t)nu * sizeof(QPClass);
    for (int j = 0; j < nu; ++j) {
        qp_make_class(bounds + 8 * j, sc, rho, &cls[j]);
        const double scd[4] = {cls[j].s[0], cls[j].s[1], cls[j].s[2], cls[j].s[3]};
        const int rc = warp ? qp_dense_inverse(H, rho, scd, reinterpret_cast<float*>(fac + j * per))
                            : qp_band_factor(H, rho, scd, reinterpret_cast<float4*>(fac + j * per));
        if (rc != MPPI_OK) return rc;
    }
    return MPPI_OK;
}

// Projection of the K x nu sampled sequences of one controller into its
// h-major sample buffer U (Eq. 5).
QPArgs qp_controller_args(int nu, int nq, int K, int H, int iters, float dt, const void* d_qp, const float* state,
                          const float* u_nom, const float* sigma, const float* Lfac, uint64_t seed,
                          const unsigned long long* iter_ptr, float* U) {
    QPArgs q{};
    q.n = K * nu;
    q.H = H;
    q.iters = iters;
    q.per_cls = K;
    q.dt = dt;
    q.cls = static_cast<const QPClass*>(d_qp);
    const unsigned char* fac = static_cast<const unsigned char*>(d_qp) + (size_t)nu * sizeof(QPClass);
    if (H <= QP_WARP_MAX_H) q.minv = reinterpret_cast<const float*>(fac);
    else q.band = reinterpret_cast<const float4*>(fac);
    q.q0 = state;
    q.qd0 = state + nq;
    q.q_per_seq = 0;
    q.vin = nullptr;
    q.nu = nu;
    q.u_nom = u_nom;
    q.sigma = sigma;
    q.Lfac = Lfac;
    q.seed = seed;
    q.iter_ptr = iter_ptr;
    q.out = U;
    q.o_a = nu;                  // member k
    q.o_b = 1;                   // class j
    q.o_h = (long long)K * nu;   // step h
    q.n_cls = nu;
    q.in_n = 0;
    q.out_n = (long long)H * K * nu;
    return q;
}
}  // namespace mppi

extern "C" {

int mppi_set_projection(mppi_ctx* c, const float* bounds, int iters, float rho, const float* scales) {
    if (!c || iters < 0) return MPPI_ERR_INVALID_ARG;
    if (iters == 0) {
        if (c->qp_iters) drop_graph(c);
        c->qp_iters = 0;
        return MPPI_OK;
    }
    if (!bounds) return MPPI_ERR_INVALID_ARG;
    const int nu = 2 * c->m->info.na;
    std::vector<unsigned char> host;
    const int brc = qp_build(nu, c->H, bounds, rho, scales, host);
    if (brc != MPPI_OK) return brc;
    if (!c->d_U) return MPPI_ERR_UNSUPPORTED;
    const float dt = c->m->host.dt;
    const size_t bytes = host.size();
    if (c->d_qp && c->qp_bytes != bytes) {
        cudaFree(c->d_qp);
        c->d_qp = nullptr;
    }
    if (!c->d_qp) {
        cudaError_t e = cudaMalloc(&c->d_qp, bytes);
        if (e != cudaSuccess) return cuda_fail(e);
        c->qp_bytes = bytes;
    }
    cudaError_t e = cudaMemcpy(c->d_qp, host.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e);
    c->qp_iters = iters;
    c->qp_dt = dt;
    drop_graph(c);  // a captured solve holds the old launches
    return MPPI_OK;
}

int mppi_set_task_cost(mppi_ctx* c, const float* p, int n) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    if (!p) {
        if (c->task_on) drop_graph(c);
        c->task_on = 0;
        return MPPI_OK;
    }
    const int nu = 2 * c->m->info.na;
    if (n != MPPI_TASK_N + nu) return MPPI_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return MPPI_ERR_INVALID_ARG;
    if (!(p[0] == 0.0f || p[0] == 1.0f) || !(p[2] >= 0.0f && p[2] < 1.0f) || !(p[8] >= 0.0f)) return MPPI_ERR_INVALID_ARG;
    for (int q = 18; q <= 22; q += 4) {
        const float nn = p[q] * p[q] + p[q + 1] * p[q + 1] + p[q + 2] * p[q + 2] + p[q + 3] * p[q + 3];
        if (std::fabs(nn - 1.0f) > 1e-3f) return MPPI_ERR_INVALID_ARG;
    }
    DevTask t{};
    t.phase = (int)p[0];
    t.w_c = p[1];
    t.gamma = p[2];
    t.w_theta = p[3];
    t.w_yz = p[4];
    t.w_v = p[5];
    t.w_r = p[6];
    t.w_l = p[7];
    t.l_ball = p[8];
    t.w_eo = p[9];
    t.w_ot = p[10];
    t.eps = p[11];
    for (int k = 0; k < 3; ++k) {
        t.pb0[k] = p[12 + k];
        t.ptg[k] = p[15 + k];
    }
    for (int k = 0; k < 4; ++k) {
        t.q1s[k] = p[18 + k];
        t.q2s[k] = p[22 + k];
    }
    for (int j = 0; j < nu; ++j) t.home[j] = p[MPPI_TASK_N + j];
    if (!c->d_task) {
        cudaError_t e = cudaMalloc(&c->d_task, sizeof(DevTask));
        if (e != cudaSuccess) return cuda_fail(e);
    }
    cudaError_t e = cudaMemcpy(c->d_task, &t, sizeof t, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e);
    c->task_on = 1;
    drop_graph(c);
    return MPPI_OK;
}

int mppi_get_samples(mppi_ctx* c, float* U, void* stream) {
    if (!c || !U) return MPPI_ERR_INVALID_ARG;
    if (!c->d_U) return MPPI_ERR_UNSUPPORTED;
    const size_t n = (size_t)c->H * c->K * 2 * c->m->info.na;
    return cuda_fail(cudaMemcpyAsync(U, c->d_U, n * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
}

static bool elite_mode(const mppi_ctx* c) {
    return c->n_elite != c->K || c->eta != 1.0f || c->update_cov || c->cov_sampling;
}

static int launch_elite(mppi_ctx* c, const float* costs, const float* u_nom, float* u_out, int advance,
                        const float* U_stored, cudaStream_t s) {
    const int nu = 2 * c->m->info.na;
    int P = 1;
    while (P < c->K) P <<= 1;
    // keys in shared memory: all P of them, or the two 1024-key buffers of
    // the register network (P <= 1024)
    const size_t sm = (size_t)(P <= 1024 ? 2048 : P) * sizeof(unsigned long long);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(elite_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    elite_select_kernel<<<1, 1024, sm, s>>>(costs, c->K, P, c->n_elite, c->d_sel, c->d_eidx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    EliteArgs a{};
    a.K = c->K;
    a.H = c->H;
    a.n_elite = c->n_elite;
    a.update_cov = c->update_cov;
    a.beta = c->lambda;
    a.eta = c->eta;
    a.cov_floor = c->cov_floor;
    a.costs = costs;
    a.u_nom = u_nom;
    a.u_out = u_out;
    a.sigma = c->d_sigma;
    a.Lfac = c->cov_sampling ? c->d_L : nullptr;
    a.u_lo = c->d_ulo;
    a.u_hi = c->d_uhi;
    a.Sigma = c->d_Sigma;
    a.Lout = c->d_L;
    a.seed = c->seed;
    a.iter_ptr = c->d_iter;
    a.U_stored = U_stored;
    a.sel = c->d_sel;
    a.eidx = c->d_eidx;
    a.best_U = c->d_bestU;
    a.err = c->d_err;
    a.advance = advance;
    a.done = c->d_done;
    if (nu == 6) elite_update_kernel<6><<<c->H, 256, 0, s>>>(a);
    else elite_update_kernel<14><<<c->H, 256, 0, s>>>(a);
    return cuda_fail(cudaGetLastError());
}

static UpdateArgs update_args(mppi_ctx* c, const float* costs, const float* u_nom, float* u_out, int advance,
                              float* best) {
    UpdateArgs u{};
    u.K = c->K;
    u.costs = costs;
    u.u_nom = u_nom;
    u.u_out = u_out;
    u.sigma = c->d_sigma;
    u.u_lo = c->d_ulo;
    u.u_hi = c->d_uhi;
    u.lambda = c->lambda;
    u.seed = c->seed;
    u.iter_ptr = c->d_iter;
    u.err = c->d_err;
    u.best = best;
    u.advance = advance;
    u.done = c->d_done;
    return u;
}

static int enqueue_step(mppi_ctx* c, const float* state, const float* u_nom, float* u_out, float* best,
                        cudaStream_t s, bool capturing = false) {
    RolloutArgs a = philox_args(c, state, u_nom);
    const bool prof = !capturing && c->prof_n < c->prof_cap;
    cudaEvent_t* ev = prof ? &c->prof_ev[4 * c->prof_n] : nullptr;
    if (prof) {
        a.stats = c->d_stats;
        cudaEventRecord(ev[0], s);
    }
    int rc = MPPI_OK;
    int mode = 1;
    if (c->qp_iters > 0) {  // sample, project (Eq. 5), then roll the projected sequences out
        rc = launch_projection(c, state, u_nom, s);
        if (rc != MPPI_OK) return rc;
        a.U = c->d_U;
        a.U_hmajor = 1;
        a.U_store = nullptr;
        a.Lfac = nullptr;
        mode = 0;
    }
    if (prof) cudaEventRecord(ev[1], s);
    // Programmatic dependent launches overlap a kernel's launch with its
    // predecessor's tail.  With one-warp CTAs (small K) the early-placed
    // dependent CTAs cost more than the overlap saves (lift, K = 1024: 0.146
    // ms per iteration without, 0.168 with), so they are used with wider CTAs
    // only; event records between the kernels would break the overlap anyway.
    const bool pdl = !prof && launch_spc(c, a.lps) * a.lps > 32;
    a.pdl = pdl;
    rc = launch_rollout(c->m->info.na, mode, a, launch_spc(c, a.lps), s);
    if (rc != MPPI_OK) return rc;
    if (prof) cudaEventRecord(ev[2], s);
    if (elite_mode(c)) {
        rc = launch_elite(c, c->d_costs, u_nom, u_out, 1, c->d_U, s);
    } else {
        UpdateArgs u = update_args(c, c->d_costs, u_nom, u_out, 1, best);
        u.U_stored = c->d_U;
        u.pdl = pdl;
        rc = launch_update(2 * c->m->info.na, u, c->H, s);
    }
    if (prof) {
        cudaEventRecord(ev[3], s);
        c->prof_n++;
    }
    return rc;
}

int mppi_step(mppi_ctx* c, const float* state, const float* u_nom, float* u_nom_out, void* stream) {
    if (!c || !state || !u_nom || !u_nom_out) return MPPI_ERR_INVALID_ARG;
    NvtxRange r("mppi_step");
    return enqueue_step(c, state, u_nom, u_nom_out, c->d_best, (cudaStream_t)stream);
}

int mppi_step_host(mppi_ctx* c, const float* state, const float* u_nom, float* u_nom_out, void* stream) {
    if (!c || !state || !u_nom || !u_nom_out) return MPPI_ERR_INVALID_ARG;
    NvtxRange r("mppi_step_host");
    const int na = c->m->info.na, nx = 4 * na + 13, nu_h = c->H * 2 * na;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!c->h_stage) {
        e = cudaMallocHost(&c->h_stage, (size_t)(nx + 2 * nu_h) * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&c->d_stage, (size_t)(nx + nu_h) * sizeof(float));
        if (e != cudaSuccess) {
            cudaFreeHost(c->h_stage);
            c->h_stage = nullptr;
            return e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : cuda_fail(e);
        }
    }
    // one H2D copy of (state, u_nom), the iteration in place, one D2H copy
    std::memcpy(c->h_stage, state, (size_t)nx * sizeof(float));
    std::memcpy(c->h_stage + nx, u_nom, (size_t)nu_h * sizeof(float));
    e = cudaMemcpyAsync(c->d_stage, c->h_stage, (size_t)(nx + nu_h) * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e);
    int rc = enqueue_step(c, c->d_stage, c->d_stage + nx, c->d_stage + nx, c->d_best, s);
    if (rc != MPPI_OK) return rc;
    e = cudaMemcpyAsync(c->h_stage + nx + nu_h, c->d_stage + nx, (size_t)nu_h * sizeof(float), cudaMemcpyDeviceToHost,
                        s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    std::memcpy(u_nom_out, c->h_stage + nx + nu_h, (size_t)nu_h * sizeof(float));
    return MPPI_OK;
}

int mppi_solve(mppi_ctx* c, const float* state, float* u, int iters, float* best_out, void* stream) {
    if (!c || !state || !u || iters < 1) return MPPI_ERR_INVALID_ARG;
    NvtxRange r("mppi_solve");
    cudaStream_t s = (cudaStream_t)stream;
    float* best = best_out ? best_out : c->d_best;
    if (s == nullptr) {  // the legacy stream cannot be captured: run eagerly
        for (int it = 0; it < iters; ++it) {
            int rc = enqueue_step(c, state, u, u, best, s);
            if (rc != MPPI_OK) return rc;
        }
        return MPPI_OK;
    }
    const bool hit = c->gexec && c->g_state == state && c->g_u == u && c->g_iters == iters && c->g_stream == s &&
                     c->g_best == best;
    if (!hit) {
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        if (c->graph) cudaGraphDestroy(c->graph);
        c->gexec = nullptr;
        c->graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e);
        int rc = MPPI_OK;
        for (int it = 0; it < iters && rc == MPPI_OK; ++it) rc = enqueue_step(c, state, u, u, best, s, true);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s, &g);
        if (rc != MPPI_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e);
        }
        c->graph = g;
        c->g_state = state;
        c->g_u = u;
        c->g_iters = iters;
        c->g_stream = s;
        c->g_best = best;
    }
    return cuda_fail(cudaGraphLaunch(c->gexec, s));
}

int mppi_update(mppi_ctx* c, const float* costs, const float* u_nom, float* u_out, void* stream) {
    if (!c || !costs || !u_nom || !u_out) return MPPI_ERR_INVALID_ARG;
    if (elite_mode(c)) return launch_elite(c, costs, u_nom, u_out, 0, nullptr, (cudaStream_t)stream);
    UpdateArgs u = update_args(c, costs, u_nom, u_out, 0, c->d_best);
    return launch_update(2 * c->m->info.na, u, c->H, (cudaStream_t)stream);
}

int rollout_batch(mppi_ctx* c, int n, const float* states, const float* U, float* costs, float* states_out,
                  void* stream) {
    if (!c || n < 0 || n > c->K || (n > 0 && (!states || !U || !costs))) return MPPI_ERR_INVALID_ARG;
    NvtxRange r("rollout_batch");
    RolloutArgs a{};
    a.model = c->m->dev;
    a.n = n;
    a.H = c->H;
    a.states = states;
    a.state_stride = 4 * c->m->info.na + 13;
    a.U = U;
    a.costs = costs;
    a.states_out = states_out;
    a.err = c->d_err;
    a.task = c->task_on ? c->d_task : nullptr;
    a.lps = a.task ? 32 : c->lps;
    return launch_rollout(c->m->info.na, 0, a, launch_spc(c, a.lps), (cudaStream_t)stream);
}

int sim_step(mppi_ctx* c, int n, float* states, const float* U1, void* stream) {
    if (!c || n < 0 || n > c->K || (n > 0 && (!states || !U1))) return MPPI_ERR_INVALID_ARG;
    RolloutArgs a{};
    a.model = c->m->dev;
    a.n = n;
    a.H = 1;
    a.states = states;
    a.state_stride = 4 * c->m->info.na + 13;
    a.U = U1;
    a.costs = c->d_costs;
    a.states_out = states;  // each lane group reads its state before writing it back
    a.err = c->d_err;
    a.lps = c->lps;
    return launch_rollout(c->m->info.na, 0, a, launch_spc(c, a.lps), (cudaStream_t)stream);
}

int mppi_debug_noise(mppi_ctx* c, uint64_t iteration, float* eps, void* stream) {
    if (!c || !eps) return MPPI_ERR_INVALID_ARG;
    NoiseArgs a{};
    a.K = c->K;
    a.H = c->H;
    a.sigma = c->d_sigma;
    a.seed = c->seed;
    a.iter = iteration;
    a.eps = eps;
    return launch_noise(2 * c->m->info.na, a, (cudaStream_t)stream);
}

int mppi_debug_philox(int n, const uint32_t* ctr, uint64_t key, uint32_t* out, void* stream) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return MPPI_ERR_INVALID_ARG;
    if (n == 0) return MPPI_OK;
    philox_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        n, reinterpret_cast<const uint4*>(ctr), make_uint2((uint32_t)key, (uint32_t)(key >> 32)),
        reinterpret_cast<uint4*>(out));
    return cuda_fail(cudaGetLastError());
}

int mppi_get_iteration(mppi_ctx* c, uint64_t* it, void* stream) {
    if (!c || !it) return MPPI_ERR_INVALID_ARG;
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, c->d_iter, sizeof v, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    *it = v;
    return MPPI_OK;
}

int mppi_set_iteration(mppi_ctx* c, uint64_t it, void* stream) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    unsigned long long v = it;
    cudaError_t e = cudaMemcpyAsync(c->d_iter, &v, sizeof v, cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return cuda_fail(e);
}

int mppi_sync(mppi_ctx* c, void* stream) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int err = 0;
    e = cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e);
    if (err & ERRB_TIMEOUT) return MPPI_ERR_TIMEOUT;
    if (err & ERRB_CHOLESKY) return MPPI_ERR_CHOLESKY;
    if (err & ERRB_NONFINITE) return MPPI_ERR_NONFINITE;
    return MPPI_OK;
}

int mppi_debug_bounds(unsigned* word, int* checked) {
    unsigned w = bounds_word_api() | bounds_word_batch() | bounds_word_qp() | bounds_word_loop() |
                 bounds_word_rollout7() | bounds_word_rollout3();
    if (word) *word = w;
    if (checked) *checked = kBoundsCheck ? 1 : 0;
    return w == ~0u ? MPPI_ERR_CUDA : MPPI_OK;
}

}  // extern "C"

int mppi_run_episode(mppi_ctx* c, const float* x0, float* u, const mppi_episode_config* cfg, float* traj,
                     float* u_exec, float* comp_ms, mppi_episode_result* res, void* stream) {
    if (!c || !x0 || !u || !cfg || !res) return MPPI_ERR_INVALID_ARG;
    if (cfg->iters < 1 || cfg->n_avg < 1 || cfg->n_avg > c->H || cfg->max_steps < 1 || !(cfg->goal_tol > 0.0f) ||
        !(cfg->lift_dz >= 0.0f) || !(cfg->drop_dz > 0.0f) || !(cfg->pick_tol >= 0.0f))
        return MPPI_ERR_INVALID_ARG;
    const bool elite = elite_mode(c);
    if (!elite && !c->d_U) return MPPI_ERR_UNSUPPORTED;  // the best sample is read from the sample buffer
    NvtxRange r("mppi_run_episode");
    cudaStream_t s = (cudaStream_t)stream;
    const int na = c->m->info.na, nu = 2 * na, nq = 2 * na + 7, nx = nq + 2 * na + 6;
    float* d_world = nullptr;  // world state (nx), executed control (nu), probe (8)
    cudaError_t e = cudaMalloc(&d_world, (size_t)(nx + nu + 8) * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e);
    float* d_u1 = d_world + nx;
    float* d_probe = d_u1 + nu;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    int rc = cuda_fail(cudaMemcpyAsync(d_world, x0, (size_t)nx * sizeof(float), cudaMemcpyHostToDevice, s));
    DevTask task{};
    bool switching = false;
    float goal[3] = {c->m->host.goal[0], c->m->host.goal[1], c->m->host.goal[2]};
    if (rc == MPPI_OK && c->task_on) {
        rc = cuda_fail(cudaMemcpy(&task, c->d_task, sizeof task, cudaMemcpyDeviceToHost));
        for (int k = 0; k < 3; ++k) goal[k] = task.ptg[k];
        switching = task.phase == 0 && cfg->pick_tol > 0.0f;
    }
    if (traj) std::memcpy(traj, x0, (size_t)nx * sizeof(float));
    mppi_episode_result out{};
    out.outcome = MPPI_EP_TIMEOUT;
    out.switch_step = -1;
    const float z0 = x0[2 * na + 2];
    float zmax = z0;
    bool lifted = false;
    float arm0 = 0.0f;  // left-right link distance at the start: arms already crossing are exempt
    double sum = 0.0, sum2 = 0.0;
    float probe[8];
    if (rc == MPPI_OK) rc = launch_probe(na, c->m->dev, d_world, d_probe, s);
    if (rc == MPPI_OK) rc = cuda_fail(cudaMemcpyAsync(probe, d_probe, sizeof probe, cudaMemcpyDeviceToHost, s));
    if (rc == MPPI_OK) rc = cuda_fail(cudaStreamSynchronize(s));
    arm0 = probe[1];
    bool done = false;
    while (rc == MPPI_OK && !done && out.steps < cfg->max_steps) {
        cudaEventRecord(ev[0], s);
        rc = mppi_solve(c, d_world, u, cfg->iters, c->d_best, s);
        if (rc == MPPI_OK)
            rc = launch_best_average(c->d_U, c->d_best, elite ? c->d_bestU : nullptr, c->K, nu, cfg->n_avg, d_u1, s);
        cudaEventRecord(ev[1], s);
        if (rc != MPPI_OK) break;
        for (int i = 0; i < cfg->n_avg && out.steps < cfg->max_steps && rc == MPPI_OK; ++i) {
            rc = sim_step(c, 1, d_world, d_u1, s);
            if (rc == MPPI_OK) rc = launch_probe(na, c->m->dev, d_world, d_probe, s);
            if (rc == MPPI_OK) rc = cuda_fail(cudaMemcpyAsync(probe, d_probe, sizeof probe, cudaMemcpyDeviceToHost, s));
            if (rc == MPPI_OK && (traj || u_exec)) {
                if (traj)
                    rc = cuda_fail(cudaMemcpyAsync(traj + (size_t)(out.steps + 1) * nx, d_world, (size_t)nx * sizeof(float),
                                                   cudaMemcpyDeviceToHost, s));
                if (rc == MPPI_OK && u_exec)
                    rc = cuda_fail(cudaMemcpyAsync(u_exec + (size_t)out.steps * nu, d_u1, (size_t)nu * sizeof(float),
                                                   cudaMemcpyDeviceToHost, s));
            }
            if (rc == MPPI_OK) rc = cuda_fail(cudaStreamSynchronize(s));
            if (rc != MPPI_OK) break;
            ++out.steps;
            const float bz = probe[4];
            if (!lifted && bz > z0 + cfg->lift_dz) lifted = true;
            zmax = fmaxf(zmax, bz);
            const float g0 = probe[2] - goal[0], g1 = probe[3] - goal[1], g2 = probe[4] - goal[2];
            if (probe[0] < 0.0f || (arm0 >= 0.0f && probe[1] < 0.0f)) {
                out.outcome = MPPI_EP_COLLISION;
                done = true;
            } else if (std::sqrt(g0 * g0 + g1 * g1 + g2 * g2) < cfg->goal_tol) {
                out.outcome = MPPI_EP_SUCCESS;
                done = true;
            } else if (lifted && bz < zmax - cfg->drop_dz) {
                out.outcome = MPPI_EP_DROPPED;
                done = true;
            }
            if (done) break;
            if (switching) {  // pick -> move once the end effectors reach the pick point
                const float m0 = probe[5] - task.pb0[0], m1 = probe[6] - task.pb0[1],
                            m2 = probe[7] - (task.pb0[2] - task.eps);
                if (std::sqrt(m0 * m0 + m1 * m1 + m2 * m2) < cfg->pick_tol) {
                    std::vector<float> p(MPPI_TASK_N + nu);
                    p[0] = 1.0f;
                    p[1] = task.w_c; p[2] = task.gamma; p[3] = task.w_theta; p[4] = task.w_yz; p[5] = task.w_v;
                    p[6] = task.w_r; p[7] = task.w_l; p[8] = task.l_ball; p[9] = task.w_eo; p[10] = task.w_ot;
                    p[11] = task.eps;
                    for (int k = 0; k < 3; ++k) {
                        p[12 + k] = task.pb0[k];
                        p[15 + k] = task.ptg[k];
                    }
                    for (int k = 0; k < 4; ++k) {
                        p[18 + k] = task.q1s[k];
                        p[22 + k] = task.q2s[k];
                    }
                    for (int j = 0; j < nu; ++j) p[MPPI_TASK_N + j] = task.home[j];
                    rc = mppi_set_task_cost(c, p.data(), (int)p.size());
                    switching = false;
                    out.switch_step = out.steps;
                }
            }
        }
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) {
            if (comp_ms && out.plans < cfg->max_steps) comp_ms[out.plans] = ms;
            sum += ms;
            sum2 += (double)ms * ms;
        }
        ++out.plans;
        if (done || rc != MPPI_OK) break;
        // warm start: shift the nominal sequence and the covariance blocks
        rc = launch_shift_rows(u, c->H, nu, cfg->n_avg, s);
        if (rc == MPPI_OK && c->update_cov) {
            rc = launch_shift_rows(c->d_Sigma, c->H, nu * nu, cfg->n_avg, s);
            if (rc == MPPI_OK) rc = launch_shift_rows(c->d_L, c->H, nu * nu, cfg->n_avg, s);
        }
    }
    if (rc == MPPI_OK) rc = cuda_fail(cudaStreamSynchronize(s));
    out.task_time_s = out.steps * (double)c->m->host.dt;
    if (out.plans > 0) {
        out.comp_mean_ms = sum / out.plans;
        const double var = sum2 / out.plans - out.comp_mean_ms * out.comp_mean_ms;
        out.comp_std_ms = var > 0.0 ? std::sqrt(var) : 0.0;
    }
    *res = out;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaFree(d_world);
    return rc;
}
