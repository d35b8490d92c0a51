// The rollout kernel (sampling + H-step contact rollout + stage cost of K
// samples, Alg. 1) and its launch: template over the arm size NA, the lanes
// per sample LPS (32, 16 or 8 -- one, two or four samples per warp), the
// control source MODE (0 explicit, 1 Philox with the diagonal sigma, 2
// Philox through the covariance factors when they are given: the draw's
// covariance branch stays out of the plain kernel), the ball-task cost suite and
// the placement of the lone ball contact's solve.  Each arm size is
// instantiated in a translation unit of its own (mppi_rollout_dh7.cu,
// mppi_rollout_planar3.cu) so that they compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "../../include/mppi.h"
#include "mppi_device.cuh"
#include "mppi_internal.h"
#include "mppi_kernels.cuh"
#include "mppi_task.cuh"

namespace mppi {

// Byte stride between the workspaces of consecutive samples of a CTA.  With
// several samples per warp the workspaces of a warp's samples start
// 128 / (samples per warp) bytes apart modulo 128, so that the groups'
// lane-indexed shared-memory accesses fall in different banks.
template <int NA, int LPS>
__host__ __device__ constexpr size_t ws_stride() {
    size_t s = (sizeof(WarpWS<NA>) + 31) / 32 * 32;
    if (LPS == 32) return s;
    const size_t want = 128 / (32 / LPS);
    while (s % 128 != want) s += 32;
    return s;
}

template <int NA, int LPS>
size_t rollout_smem(int spc, int unom_floats, bool task) {
    return sizeof(DevModel) + (task ? sizeof(DevTask) : 0) + ((size_t)unom_floats * sizeof(float) + 15) / 16 * 16 +
           (size_t)spc * ws_stride<NA, LPS>();
}

template <int NA, int LPS, int MODE, bool TASK, int PLACE>
__global__ void __launch_bounds__(512) rollout_kernel(RolloutArgs args) {
    using d = Dims<NA>;
    // launched as a programmatic dependent: wait for the previous kernel's
    // results (u_nom, the counter), then let the next kernel launch early
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();
    extern __shared__ __align__(16) unsigned char smem[];
    DevModel& M = *reinterpret_cast<DevModel*>(smem);
    constexpr size_t task_b = TASK ? sizeof(DevTask) : 0;
    DevTask* task_s = reinterpret_cast<DevTask*>(smem + sizeof(DevModel));
    float* unom_s = reinterpret_cast<float*>(smem + sizeof(DevModel) + task_b);
    const int unom_n = (MODE >= 1 && args.stage_unom) ? args.H * d::NU : 0;
    const size_t ws_off = sizeof(DevModel) + task_b + ((size_t)unom_n * sizeof(float) + 15) / 16 * 16;
    stage_model(smem, args.model, unom_s, args.u_nom, unom_n);
    if constexpr (TASK) {
        const float4* src = reinterpret_cast<const float4*>(args.task);
        float4* dst = reinterpret_cast<float4*>(task_s);
        for (int t = threadIdx.x; t < (int)(sizeof(DevTask) / 16); t += blockDim.x) dst[t] = src[t];
    }
    __syncthreads();

    const int spc = blockDim.x / LPS, gi = threadIdx.x / LPS;
    const Lanes<LPS> g(threadIdx.x & 31);
    const int k = blockIdx.x * spc + gi;
    if (k >= args.n) return;
    WarpWS<NA>& w = *reinterpret_cast<WarpWS<NA>*>(smem + ws_off + (size_t)gi * ws_stride<NA, LPS>());
    SampleIO io{};
    io.x = args.states + (size_t)k * args.state_stride;
    io.k = k;
    io.H = args.H;
    io.err = args.err;
    io.stats = args.stats;
    io.task = TASK ? task_s : nullptr;
    io.x_out = args.states_out ? args.states_out + (size_t)k * d::NX : nullptr;
    io.U_store = MODE >= 1 ? args.U_store : nullptr;
    io.Kn = args.n;
    io.Lfac = MODE == 2 ? args.Lfac : nullptr;
    if (MODE >= 1) {
        io.unom = unom_n ? unom_s : args.u_nom;
        io.iter = (uint32_t)(args.iter_ptr ? *args.iter_ptr : args.iter_val);
        io.key = make_uint2((uint32_t)args.seed, (uint32_t)(args.seed >> 32));
        if (g.sl < d::NU) {
            io.sig = ld_checked(args.sigma, g.sl, d::NU);
            io.lo = M.link[g.sl / NA][g.sl % NA].u_lo;
            io.hi = M.link[g.sl / NA][g.sl % NA].u_hi;
        }
    } else {
        const long long total = (long long)args.n * args.H * d::NU;
        if (args.U_hmajor) {
            io.U = args.U + (size_t)k * d::NU;
            io.u_stride = (long long)args.n * d::NU;
            io.u_ext = total - (long long)k * d::NU;
        } else {
            io.U = args.U + (size_t)k * args.H * d::NU;
            io.u_stride = d::NU;
            io.u_ext = total - (long long)k * args.H * d::NU;
        }
    }
    const float cost = rollout_sample<NA, LPS, MODE, TASK, PLACE>(M, w, g, io);
    if (g.sl == 0 && MPPI_IN_RANGE(k, args.n)) args.costs[k] = cost;
}

namespace rollout_launch {

inline int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return MPPI_OK;
    if (e == cudaErrorMemoryAllocation) return MPPI_ERR_OOM;
    return MPPI_ERR_CUDA;
}

template <int NA, int LPS, int MODE, bool TASK, int PLACE>
int launch_t(const RolloutArgs& a, int spc, cudaStream_t s) {
    const int unom = (MODE >= 1 && a.stage_unom) ? a.H * Dims<NA>::NU : 0;
    const size_t sm = rollout_smem<NA, LPS>(spc, unom, TASK);
    auto fn = rollout_kernel<NA, LPS, MODE, TASK, PLACE>;
    int dev = 0, max_sm = 0;
    cudaError_t q = cudaGetDevice(&dev);
    if (q == cudaSuccess) q = cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (q != cudaSuccess) return cuda_fail(q);
    if (sm > (size_t)max_sm) return MPPI_ERR_INVALID_ARG;  // too many samples per CTA for shared memory
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    const int grid = (a.n + spc - 1) / spc;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(spc * LPS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = a.pdl ? at : nullptr;
    cfg.numAttrs = a.pdl ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, fn, a);
    return cuda_fail(e != cudaSuccess ? e : cudaGetLastError());
}

template <int NA, int LPS>
int launch_lps(int mode, const RolloutArgs& a, int spc, cudaStream_t s) {
    if (mode == 0) return launch_t<NA, LPS, 0, false, 0>(a, spc, s);
    if (a.Lfac) return a.place ? launch_t<NA, LPS, 2, false, 1>(a, spc, s) : launch_t<NA, LPS, 2, false, 0>(a, spc, s);
    return a.place ? launch_t<NA, LPS, 1, false, 1>(a, spc, s) : launch_t<NA, LPS, 1, false, 0>(a, spc, s);
}

}  // namespace rollout_launch

// Launch for one arm size.  a.lps (0 = 32) and a.place select the layout;
// spc is rounded up to whole warps.  The ball-task suite runs on 32 lanes
// per sample with the fused placement only.  A shape whose workspaces do not
// fit one CTA's shared memory is refused with MPPI_ERR_INVALID_ARG.
template <int NA>
int dispatch_rollout(int mode, const RolloutArgs& a, int spc, cudaStream_t s) {
    using namespace rollout_launch;
    const int lps = a.lps ? a.lps : 32;
    if (lps != 8 && lps != 16 && lps != 32) return MPPI_ERR_INVALID_ARG;
    if (a.place < 0 || a.place > 1) return MPPI_ERR_INVALID_ARG;
    const int spw = 32 / lps;
    spc = (spc + spw - 1) / spw * spw;
    if (spc * lps > 512) return MPPI_ERR_INVALID_ARG;
    if (a.task) {
        if (lps != 32 || a.place != 0) return MPPI_ERR_UNSUPPORTED;
        if (mode == 0) return launch_t<NA, 32, 0, true, 0>(a, spc, s);
        return a.Lfac ? launch_t<NA, 32, 2, true, 0>(a, spc, s) : launch_t<NA, 32, 1, true, 0>(a, spc, s);
    }
    if (lps == 32) return launch_lps<NA, 32>(mode, a, spc, s);
    if (lps == 16) return launch_lps<NA, 16>(mode, a, spc, s);
    if constexpr (Lanes<8>::SEG > NA) return launch_lps<NA, 8>(mode, a, spc, s);
    return MPPI_ERR_UNSUPPORTED;
}

// Samples per CTA for K samples in layout LPS (sampling rollout, fused
// placement).  One wave matters most: every sample runs the same H steps, so
// a partial second wave doubles the time of the samples in it.  So: the
// fewest waves of CTAs over the SMs; within one wave the fewest samples on
// the busiest SM, then the larger CTA (fewer model copies to stage; on
// GB300 a 28-sample CTA per SM beat two 14-sample CTAs by 5%); past one wave
// the most samples resident per SM, then the smaller CTA.
template <int NA>
int choose_spc(int lps, int K, int unom_floats) {
    int dev = 0, nsm = 0, max_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || nsm <= 0)
        return 4;
    const int spw = 32 / lps;
    long best_w = 1L << 40, best_key = 1L << 40;
    int best = spw;
    for (int spc = spw; spc * lps <= 512; spc += spw) {
        size_t sm = 0;
        int per_sm = 0;
        cudaError_t e = cudaSuccess;
        if (lps == 32) {
            sm = rollout_smem<NA, 32>(spc, unom_floats, false);
            if (sm <= (size_t)max_sm) {
                e = cudaFuncSetAttribute(rollout_kernel<NA, 32, 1, false, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rollout_kernel<NA, 32, 1, false, 0>,
                                                                      spc * 32, sm);
            }
        } else if (lps == 16) {
            sm = rollout_smem<NA, 16>(spc, unom_floats, false);
            if (sm <= (size_t)max_sm) {
                e = cudaFuncSetAttribute(rollout_kernel<NA, 16, 1, false, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rollout_kernel<NA, 16, 1, false, 0>,
                                                                      spc * 16, sm);
            }
        } else if constexpr (Lanes<8>::SEG > NA) {
            sm = rollout_smem<NA, 8>(spc, unom_floats, false);
            if (sm <= (size_t)max_sm) {
                e = cudaFuncSetAttribute(rollout_kernel<NA, 8, 1, false, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rollout_kernel<NA, 8, 1, false, 0>,
                                                                      spc * 8, sm);
            }
        }
        if (e != cudaSuccess || per_sm <= 0) continue;
        const long blocks = (K + spc - 1) / spc;
        const long cap = (long)per_sm * nsm;
        const long waves = (blocks + cap - 1) / cap;
        // lower is better: one wave -> load on the busiest SM (ties to the
        // larger CTA below); more -> minus the samples resident per SM
        const long key = waves == 1 ? (blocks + nsm - 1) / nsm * spc : -(long)per_sm * spc;
        const bool tie_larger = waves == 1;
        if (waves < best_w || (waves == best_w && (key < best_key || (key == best_key && tie_larger)))) {
            best_w = waves;
            best_key = key;
            best = spc;
        }
    }
    return best;
}

// Default layout for K samples: 16 lanes per sample once 32-lane groups
// cannot hold all K samples in one wave (their registers allow 16 warps per
// SM), else 32 (the shorter per-step chain of one sample per warp).
inline int default_lps(int K) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return 32;
    return K > 16 * nsm ? 16 : 32;
}

int launch_rollout_na7(int mode, const RolloutArgs& a, int spc, cudaStream_t s);
int launch_rollout_na3(int mode, const RolloutArgs& a, int spc, cudaStream_t s);
int choose_spc_na7(int lps, int K, int unom_floats);
int choose_spc_na3(int lps, int K, int unom_floats);

}  // namespace mppi
