// mppi_step_noalloc: one MPPI iteration that allocates nothing.
//
// Some callers cannot allocate device memory when they want to plan: a
// real-time control loop may not call cudaMalloc/cudaFree once it runs (those
// calls can synchronise the device and take unbounded time), and a host
// framework that owns the GPU's memory budget may forbid allocation inside
// its callbacks.  This entry point runs the same kernels as mppi_step, but
// its scratch (the scene model, sigma and control bounds, the error word and
// the K sample costs) lives in one file-scope static device array that every
// GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/mppi.h"
#include "mppi_device.cuh"
#include "mppi_internal.h"

using namespace mppi;

namespace {

constexpr int NOALLOC_MAX_K = MPPI_NOALLOC_MAX_K;
constexpr int NOALLOC_MAX_H = 1024;
// scratch layout (byte offsets, each region 256-byte aligned)
constexpr size_t OFF_MODEL = 0;
constexpr size_t OFF_PARAMS = 3072;              // sigma, u_lo, u_hi: 3 x 16 floats
constexpr size_t OFF_WORDS = OFF_PARAMS + 256;   // error word
constexpr size_t OFF_COSTS = OFF_WORDS + 256;    // K sample costs
constexpr size_t SCRATCH_BYTES = OFF_COSTS + (size_t)NOALLOC_MAX_K * sizeof(float);
static_assert(sizeof(DevModel) <= OFF_PARAMS, "model region too small");

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[MAX_DEVICES] = {nullptr};

}  // namespace

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return MPPI_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return MPPI_ERR_CUDA;
        g_dev_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_dev_ptr[dev];
    return MPPI_OK;
}

double blob_value(const unsigned char* b, size_t i) {
    double v;
    std::memcpy(&v, b + 16 + 8 * i, 8);
    return v;
}

// Blob -> device model representation without any heap allocation (the same
// format mppi_model_load reads).
int parse_blob_noalloc(const void* blob, size_t len, DevModel* M) {
    if (!blob || len < 16) return MPPI_ERR_INVALID_ARG;
    const unsigned char* b = static_cast<const unsigned char*>(blob);
    uint32_t h[4];
    std::memcpy(h, b, 16);
    if (h[0] != 0x4950504Du || h[1] != 1u) return MPPI_ERR_INVALID_ARG;
    const size_t n = h[2];
    if (n < 23 || len < 16 + 8 * n) return MPPI_ERR_INVALID_ARG;
    const int na = (int)blob_value(b, 0), nb = (int)blob_value(b, 1), maxc = (int)blob_value(b, 2);
    if (na < 1 || na > MAXL || nb < 0 || nb > MAXB || maxc < 1 || maxc > 16) return MPPI_ERR_INVALID_ARG;
    if (maxc > MAXC) return MPPI_ERR_UNSUPPORTED;  // more contacts than the device solver keeps
    const int nq = 2 * na + 7, nv = 2 * na + 6;
    if (n != 23 + 2 * (12 + 39 * (size_t)na) + 6 * (size_t)nb + (size_t)(nq + nv)) return MPPI_ERR_INVALID_ARG;
    std::memset(M, 0, sizeof *M);
    M->na = na;
    M->nb = nb;
    M->maxc = maxc;
    M->dt = (float)blob_value(b, 3);
    M->sweeps = (int)blob_value(b, 4);
    M->mu = (float)blob_value(b, 5);
    M->imp = (float)blob_value(b, 6);
    M->erp = (float)blob_value(b, 7);
    for (int k = 0; k < 3; ++k) M->g[k] = (float)blob_value(b, 8 + k);
    M->floor_z = (float)blob_value(b, 11);
    M->rb = (float)blob_value(b, 12);
    M->mb = (float)blob_value(b, 13);
    M->Ib = (float)blob_value(b, 14);
    for (int k = 0; k < 3; ++k) M->goal[k] = (float)blob_value(b, 15 + k);
    M->w_goal = (float)blob_value(b, 18);
    M->w_u = (float)blob_value(b, 19);
    M->w_pen = (float)blob_value(b, 20);
    M->w_obst = (float)blob_value(b, 21);
    M->w_grasp = (float)blob_value(b, 22);
    if (!(M->dt > 0) || M->sweeps < 0 || M->sweeps > 1000 || !(M->imp > 0 && M->imp <= 1) || !(M->mb > 0) ||
        !(M->Ib > 0))
        return MPPI_ERR_INVALID_ARG;
    size_t o = 23;
    for (int a = 0; a < 2; ++a) {
        for (int k = 0; k < 9; ++k) M->baseR[a][k] = (float)blob_value(b, o++);
        for (int k = 0; k < 3; ++k) M->basep[a][k] = (float)blob_value(b, o++);
        for (int i = 0; i < na; ++i) {
            DevLink& L = M->link[a][i];
            for (int k = 0; k < 9; ++k) L.FR[k] = (float)blob_value(b, o++);
            for (int k = 0; k < 3; ++k) L.Fp[k] = (float)blob_value(b, o++);
            L.mass = (float)blob_value(b, o++);
            for (int k = 0; k < 3; ++k) L.com[k] = (float)blob_value(b, o++);
            double I[9];
            for (int k = 0; k < 9; ++k) I[k] = blob_value(b, o++);
            L.I[0] = (float)I[0];
            L.I[1] = (float)I[4];
            L.I[2] = (float)I[8];
            L.I[3] = (float)(0.5 * (I[1] + I[3]));
            L.I[4] = (float)(0.5 * (I[2] + I[6]));
            L.I[5] = (float)(0.5 * (I[5] + I[7]));
            for (int k = 0; k < 3; ++k) L.s0[k] = (float)blob_value(b, o++);
            for (int k = 0; k < 3; ++k) L.s1[k] = (float)blob_value(b, o++);
            L.rcap = (float)blob_value(b, o++);
            const double damping = blob_value(b, o++), kv = blob_value(b, o++);
            L.D = (float)(damping + kv);
            L.gear = (float)blob_value(b, o++);
            L.tau_max = (float)blob_value(b, o++);
            L.u_lo = (float)blob_value(b, o++);
            L.u_hi = (float)blob_value(b, o++);
            L.gravcomp = (float)blob_value(b, o++);
            if (!(L.mass > 0)) return MPPI_ERR_INVALID_ARG;
        }
    }
    for (int bi = 0; bi < nb; ++bi)
        for (int k = 0; k < 6; ++k) M->box[bi][k] = (float)blob_value(b, o++);
    return MPPI_OK;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return MPPI_OK;
    return MPPI_ERR_CUDA;
}

}  // namespace

extern "C" int mppi_step_noalloc(const void* blob, size_t len, int K, int H, float lambda, const float* sigma,
                                 uint64_t seed, uint64_t iteration, const float* state, const float* u_nom,
                                 float* u_nom_out, int* status_out, void* stream) {
    if (!blob || !sigma || !state || !u_nom || !u_nom_out || !(lambda > 0.0f)) return MPPI_ERR_INVALID_ARG;
    if (K < 1 || K > NOALLOC_MAX_K || H < 1 || H > NOALLOC_MAX_H) return MPPI_ERR_INVALID_ARG;
    DevModel M;
    int rc = parse_blob_noalloc(blob, len, &M);
    if (rc != MPPI_OK) return rc;
    if (M.na != 3 && M.na != 7) return MPPI_ERR_UNSUPPORTED;
    const int nu = 2 * M.na;
    unsigned char* base = nullptr;
    rc = scratch_address(&base);
    if (rc != MPPI_OK) return rc;
    float params[48];
    std::memset(params, 0, sizeof params);
    for (int j = 0; j < nu; ++j) {
        params[j] = sigma[j];
        params[16 + j] = M.link[j / M.na][j % M.na].u_lo;
        params[32 + j] = M.link[j / M.na][j % M.na].u_hi;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // host buffers are pageable: each copy returns once the data are staged
    cudaError_t e = cudaMemcpyAsync(base + OFF_MODEL, &M, sizeof M, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + OFF_PARAMS, params, sizeof params, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + OFF_WORDS, 0, 256, s);  // error word starts at zero
    if (e != cudaSuccess) return cuda_status(e);
    const float* d_params = reinterpret_cast<const float*>(base + OFF_PARAMS);
    int* d_err = reinterpret_cast<int*>(base + OFF_WORDS);
    float* d_costs = reinterpret_cast<float*>(base + OFF_COSTS);

    RolloutArgs a{};
    a.model = reinterpret_cast<const DevModel*>(base + OFF_MODEL);
    a.n = K;
    a.H = H;
    a.states = state;
    a.state_stride = 0;
    a.u_nom = u_nom;
    a.sigma = d_params;
    a.seed = seed;
    a.iter_ptr = nullptr;
    a.iter_val = iteration;
    a.costs = d_costs;
    a.err = d_err;
    a.stage_unom = H * nu <= 2048;
    rc = launch_rollout(M.na, 1, a, 4, s);
    if (rc != MPPI_OK) return rc;
    UpdateArgs u{};
    u.K = K;
    u.costs = d_costs;
    u.u_nom = u_nom;
    u.u_out = u_nom_out;
    u.sigma = d_params;
    u.u_lo = d_params + 16;
    u.u_hi = d_params + 32;
    u.lambda = lambda;
    u.seed = seed;
    u.iter_ptr = nullptr;
    u.iter_val = iteration;
    u.err = d_err;
    u.best = nullptr;
    u.advance = 0;
    u.done = nullptr;
    rc = launch_update(nu, u, H, s);
    if (rc != MPPI_OK) return rc;
    if (status_out) {
        int err = 0;
        e = cudaMemcpyAsync(&err, d_err, sizeof err, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        *status_out = (err & ERRB_TIMEOUT) ? MPPI_ERR_TIMEOUT
                      : (err & ERRB_CHOLESKY) ? MPPI_ERR_CHOLESKY
                      : (err & ERRB_NONFINITE) ? MPPI_ERR_NONFINITE
                                               : MPPI_OK;
    }
    return MPPI_OK;
}
