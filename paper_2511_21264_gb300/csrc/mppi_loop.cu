// Device helpers of the closed-loop episode (mppi_run_episode): the
// executed control (the average of the best sequence's first steps), the
// warm-start shift by several steps, and the per-step probe of the world
// state (collision distances, ball, end effectors).
#include <cuda_runtime.h>

#include "../../include/mppi.h"
#include "mppi_device.cuh"
#include "mppi_internal.h"
#include "mppi_task.cuh"

namespace mppi {

namespace {

// u1[j] = mean over h < n of the best sequence's row h: the elite update's
// stored best sequence (H x nu) if given, else sample best[1] of the h-major
// sample buffer U (H x K x nu).
__global__ void best_average_kernel(const float* U, const float* best, const float* bestU, int K, int nu, int n,
                                    float* u1) {
    const int j = threadIdx.x;
    if (j >= nu) return;
    const int k = bestU ? 0 : (int)best[1];
    float s = 0.0f;
    for (int h = 0; h < n; ++h) s += bestU ? bestU[h * nu + j] : U[((size_t)h * K + k) * nu + j];
    u1[j] = s / (float)n;
}

// Row h <- row min(h + n, H - 1) for H rows of `row` floats.
__global__ void shift_rows_kernel(float* u, int H, int row, int n) {
    for (int i = threadIdx.x; i < row; i += blockDim.x)
        for (int h = 0; h < H; ++h) u[(size_t)h * row + i] = u[(size_t)(h + n < H ? h + n : H - 1) * row + i];
}

// One warp: out = [min link-box distance, min left-right link distance,
// ball x y z, end-effector midpoint x y z].
template <int NA>
__global__ void __launch_bounds__(32) probe_kernel(const DevModel* model, const float* x, float* out) {
    using d = Dims<NA>;
    __shared__ __align__(16) unsigned char smem[sizeof(DevModel) + sizeof(WarpWS<NA>)];
    DevModel& M = *reinterpret_cast<DevModel*>(smem);
    WarpWS<NA>& w = *reinterpret_cast<WarpWS<NA>*>(smem + sizeof(DevModel));
    const int lane = threadIdx.x;
    const float4* src = reinterpret_cast<const float4*>(model);
    float4* dst = reinterpret_cast<float4*>(smem);
    for (int t = lane; t < (int)(sizeof(DevModel) / 16); t += 32) dst[t] = src[t];
    __syncwarp();
    if (lane < d::NQ) w.q[lane] = x[lane];
    if (lane < d::NV) w.qd[lane] = x[d::NQ + lane];
    __syncwarp();
    float Rl[9], cl[3];
    forward_kinematics<NA>(M, w, Lanes<32>(lane), Rl, cl);
    __syncwarp();
    const int nlb = 2 * NA * M.nb, np = nlb + NA * NA;
    float mb = INFINITY, ma = INFINITY;
    for (int b = lane; b < np; b += 32) {
        if (b < nlb) {
            const int l = b / M.nb, bx = b - l * M.nb;
            mb = fminf(mb, capsule_box_distance(w.a0[l], w.a1[l], M.link[l / NA][l % NA].rcap, M.box[bx]));
        } else {
            const int r = b - nlb, i = r / NA, j = r - i * NA;
            ma = fminf(ma, capsule_capsule_distance(w.a0[i], w.a1[i], M.link[0][i].rcap, w.a0[NA + j], w.a1[NA + j],
                                                    M.link[1][j].rcap));
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mb = fminf(mb, __shfl_xor_sync(FULL, mb, off));
        ma = fminf(ma, __shfl_xor_sync(FULL, ma, off));
    }
    if (lane == 0) {
        out[0] = mb;
        out[1] = ma;
        for (int k = 0; k < 3; ++k) {
            out[2 + k] = w.q[d::B + k];
            out[5 + k] = 0.5f * (w.a1[NA - 1][k] + w.a1[2 * NA - 1][k]);
        }
    }
}

}  // namespace

int launch_best_average(const float* U, const float* best, const float* bestU, int K, int nu, int n, float* u1,
                        cudaStream_t s) {
    best_average_kernel<<<1, 32, 0, s>>>(U, best, bestU, K, nu, n, u1);
    return cudaGetLastError() == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

int launch_shift_rows(float* u, int H, int row, int n, cudaStream_t s) {
    if (n <= 0) return MPPI_OK;
    shift_rows_kernel<<<1, 256, 0, s>>>(u, H, row, n);
    return cudaGetLastError() == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

int launch_probe(int na, const DevModel* model, const float* x, float* out, cudaStream_t s) {
    if (na == 3) probe_kernel<3><<<1, 32, 0, s>>>(model, x, out);
    else if (na == 7) probe_kernel<7><<<1, 32, 0, s>>>(model, x, out);
    else return MPPI_ERR_UNSUPPORTED;
    return cudaGetLastError() == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

MPPI_BOUNDS_READER(bounds_word_loop)

}  // namespace mppi
