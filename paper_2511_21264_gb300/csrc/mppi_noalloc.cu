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

// What one call uploads, passed by value as a kernel parameter: the launch
// copies it, so the call never reads host memory after it returns and needs
// no host-to-device copy (a copy from pageable memory would first wait for
// the stream).
struct NoallocUpload {
    DevModel model;
    float params[48];  // sigma, u_lo, u_hi at 0, 16, 32
};
static_assert(sizeof(NoallocUpload) <= 4000, "kernel parameter block too large");

}  // namespace

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

// Writes the call's model and parameters into the scratch array and clears
// the error word; one CTA, word by word.
__global__ void noalloc_upload_kernel(NoallocUpload up, unsigned char* base) {
    const int t = threadIdx.x;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&up.model);
    uint32_t* dst = reinterpret_cast<uint32_t*>(base + OFF_MODEL);
    for (int i = t; i < (int)(sizeof(DevModel) / 4); i += blockDim.x) dst[i] = src[i];
    float* p = reinterpret_cast<float*>(base + OFF_PARAMS);
    for (int i = t; i < 48; i += blockDim.x) p[i] = up.params[i];
    if (t == 0) *reinterpret_cast<int*>(base + OFF_WORDS) = 0;
}

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached for the life of the
// process.
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
    NoallocUpload up;
    std::memset(&up, 0, sizeof up);
    // the same parser as mppi_model_load; without the host info it allocates nothing
    int rc = parse_model_blob(blob, len, &up.model, nullptr);
    if (rc != MPPI_OK) return rc;
    const DevModel& M = up.model;
    if (M.na != 3 && M.na != 7) return MPPI_ERR_UNSUPPORTED;
    const int nu = 2 * M.na;
    unsigned char* base = nullptr;
    rc = scratch_address(&base);
    if (rc != MPPI_OK) return rc;
    for (int j = 0; j < nu; ++j) {
        up.params[j] = sigma[j];
        up.params[16 + j] = M.link[j / M.na][j % M.na].u_lo;
        up.params[32 + j] = M.link[j / M.na][j % M.na].u_hi;
    }
    cudaStream_t s = (cudaStream_t)stream;
    noalloc_upload_kernel<<<1, 256, 0, s>>>(up, base);
    cudaError_t e = cudaGetLastError();
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
        // device -> pageable host copy, then wait: this branch synchronises the stream
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
