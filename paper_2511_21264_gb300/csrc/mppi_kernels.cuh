// Per-sample rollout and per-horizon-step update, shared by the single-
// controller kernels and the batched persistent kernels.
#pragma once
#include "mppi_device.cuh"
#include "mppi_internal.h"

namespace mppi {

// Inputs of one sample's rollout (one warp).
struct SampleIO {
    const float* x;            // start state (nx)
    const float* U;            // explicit controls of this sample (H x nu), MODE 0
    const float* unom;         // nominal controls (H x nu, shared or global), MODE 1
    float sig, lo, hi;         // this lane's sigma and control bounds (lane < nu), MODE 1
    uint2 key;                 // Philox key, MODE 1
    uint32_t iter;             // Philox iteration word, MODE 1
    int k, H;                  // sample index, horizon
    float* x_out;              // optional final state (nx)
    float* U_store;            // optional: sampled controls out, H x Kn x nu (h-major)
    int Kn;                    // sample count of U_store
    int* err;                  // error word
    unsigned long long* stats; // optional [sample-steps, contacts, exact box tests]
};

// Copy the scene model (and optionally u_nom) into shared memory.
__device__ __forceinline__ void stage_model(unsigned char* smem, const DevModel* model, float* unom_s,
                                            const float* u_nom, int unom_n) {
    const float4* src = reinterpret_cast<const float4*>(model);
    float4* dst = reinterpret_cast<float4*>(smem);
    for (int t = threadIdx.x; t < (int)(sizeof(DevModel) / 16); t += blockDim.x) dst[t] = src[t];
    for (int t = threadIdx.x; t < unom_n; t += blockDim.x) unom_s[t] = u_nom[t];
}

// H simulator steps of one sample with its stage costs; the warp's state
// stays in shared memory throughout.  Returns the summed cost on every lane.
template <int NA, int MODE>
__device__ __forceinline__ float rollout_sample(const DevModel& M, WarpWS<NA>& w, int lane, const SampleIO& io) {
    using d = Dims<NA>;
    const int k = io.k;
    if (lane < d::NQ) w.q[lane] = io.x[lane];
    if (lane < d::NV) w.qd[lane] = io.x[d::NQ + lane];
    __syncwarp();
    float cost = 0.0f;
    const float* gb = M.goal;
    unsigned n_exact = 0, n_con = 0;
    for (int h = 0; h < io.H; ++h) {
        if (MODE == 1) {
            // every 8 steps the 32 lanes draw one Philox block each: 8 steps x
            // 16 controls of standard normals (the same values sample_control
            // draws one at a time)
            if ((h & 7) == 0) {
                const int jb = lane & 3, hs = h + (lane >> 2);
                if (4 * jb < d::NU && hs < io.H) {
                    const uint4 wv = philox4x32_10(make_uint4((uint32_t)jb, (uint32_t)hs, (uint32_t)k, io.iter), io.key);
#pragma unroll
                    for (int t = 0; t < 4; ++t) w.zn[lane >> 2][4 * jb + t] = block_normal(wv, t);
                }
                __syncwarp();
            }
            if (lane < d::NU) {
                w.u[lane] = fminf(fmaxf(__fmaf_rn(io.sig, w.zn[h & 7][lane], io.unom[h * d::NU + lane]), io.lo), io.hi);
                if (io.U_store) io.U_store[((size_t)h * io.Kn + k) * d::NU + lane] = w.u[lane];
            }
        } else if (lane < d::NU) {
            w.u[lane] = io.U[(size_t)h * d::NU + lane];
        }
        float Rl[9], cl[3];  // this lane's link rotation and COM, kept for the dynamics
        forward_kinematics<NA>(M, w, lane, Rl, cl);
        __syncwarp();
        if (h > 0 && lane == 0 && M.w_grasp != 0.0f) cost += M.w_grasp * grasp_term<NA>(w);
        n_exact += collide<NA>(M, w, lane);
        __syncwarp();
        n_con += w.ncon;
        dynamics<NA>(M, w, lane, io.err, Rl, cl);
        contacts<NA>(M, w, lane);
        integrate<NA>(M, w, lane);
        if (lane == 0) {
            const float* pb = &w.q[d::B];
            const float e0 = pb[0] - gb[0], e1 = pb[1] - gb[1], e2 = pb[2] - gb[2];
            float uu = 0.0f;
#pragma unroll
            for (int j = 0; j < d::NU; ++j) uu += w.u[j] * w.u[j];
            cost += M.w_goal * (e0 * e0 + e1 * e1 + e2 * e2) + M.w_u * uu + M.w_pen * w.pen_all +
                    M.w_obst * w.pen_box;
        }
        __syncwarp();
    }
    if (M.w_grasp != 0.0f) {
        float Rl[9], cl[3];
        forward_kinematics<NA>(M, w, lane, Rl, cl);
        __syncwarp();
        if (lane == 0) cost += M.w_grasp * grasp_term<NA>(w);
    }
    // a non-finite state poisons the sample's cost (weight 0 in the update)
    const bool bad = (lane < d::NQ && !isfinite(w.q[lane])) || (lane < d::NV && !isfinite(w.qd[lane]));
    if (__any_sync(FULL, bad)) cost = __int_as_float(0x7fc00000);
    cost = __shfl_sync(FULL, cost, 0);
    if (lane == 0 && !isfinite(cost)) atomicOr(io.err, ERRB_NONFINITE);
    if (io.stats && lane == 0) {
        atomicAdd(&io.stats[0], (unsigned long long)io.H);
        atomicAdd(&io.stats[1], (unsigned long long)n_con);
        atomicAdd(&io.stats[2], (unsigned long long)n_exact);
    }
    if (io.x_out) {
        if (lane < d::NQ) io.x_out[lane] = w.q[lane];
        if (lane < d::NV) io.x_out[d::NQ + lane] = w.qd[lane];
    }
    return cost;
}

// Shared memory of one update CTA.
template <int NU>
struct UpdateSmem {
    float red[NU + 1][256];
    float rmin[256];
    int ridx[256];
    int is_last;
};

// Weighted-mean update of horizon step h for one controller (256 threads):
// lowest finite cost, weights exp(-(c - c_min)/lambda), sum_k w_k U_k[h,:]
// with the samples regenerated from Philox, fixed-order trees (Eq. 8a, 8d).
// The result depends only on this controller's costs, not on the launch.
template <int NU>
__device__ __forceinline__ void update_step(const UpdateArgs& a, int h, UpdateSmem<NU>& sm) {
    constexpr int T = 256;
    const int tid = threadIdx.x;
    const uint32_t iter = (uint32_t)(a.iter_ptr ? *a.iter_ptr : a.iter_val);
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    float cm = INFINITY;
    int ci = 0x7fffffff;
    for (int k = tid; k < a.K; k += T) {
        const float c = a.costs[k];
        if (isfinite(c) && (c < cm)) {
            cm = c;
            ci = k;
        }
    }
    sm.rmin[tid] = cm;
    sm.ridx[tid] = ci;
    __syncthreads();
    for (int st = T / 2; st > 0; st >>= 1) {
        if (tid < st) {
            const float o = sm.rmin[tid + st];
            const int oi = sm.ridx[tid + st];
            if (o < sm.rmin[tid] || (o == sm.rmin[tid] && oi < sm.ridx[tid])) {
                sm.rmin[tid] = o;
                sm.ridx[tid] = oi;
            }
        }
        __syncthreads();
    }
    const float cmin = sm.rmin[0];
    const int cidx = sm.ridx[0];
    __syncthreads();
    const bool any = isfinite(cmin);
    float acc[NU];
#pragma unroll
    for (int j = 0; j < NU; ++j) acc[j] = 0.0f;
    float Z = 0.0f;
    float un[NU], sg[NU], lo[NU], hi[NU];
#pragma unroll
    for (int j = 0; j < NU; ++j) {
        un[j] = a.u_nom[h * NU + j];
        sg[j] = a.sigma[j];
        lo[j] = a.u_lo[j];
        hi[j] = a.u_hi[j];
    }
    if (any) {
        const float inv_lam = 1.0f / a.lambda;
        for (int k = tid; k < a.K; k += T) {
            const float c = a.costs[k];
            const float wk = isfinite(c) ? expf(-(c - cmin) * inv_lam) : 0.0f;
            Z += wk;
            if (a.U_stored) {
                // the rollout's own samples (bit-identical to regenerating them)
                const float* uk = a.U_stored + ((size_t)h * a.K + k) * NU;
#pragma unroll
                for (int j = 0; j < NU; ++j) acc[j] += wk * uk[j];
            } else {
#pragma unroll
                for (int jb = 0; jb < (NU + 3) / 4; ++jb) {
                    const uint4 wv = philox4x32_10(make_uint4((uint32_t)jb, (uint32_t)h, (uint32_t)k, iter), key);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int j = 4 * jb + t;
                        if (j < NU) {
                            const float z = block_normal(wv, t);
                            const float u = fminf(fmaxf(__fmaf_rn(sg[j], z, un[j]), lo[j]), hi[j]);
                            acc[j] += wk * u;
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NU; ++j) sm.red[j][tid] = acc[j];
    sm.red[NU][tid] = Z;
    __syncthreads();
    for (int st = T / 2; st > 0; st >>= 1) {
        if (tid < st) {
#pragma unroll
            for (int j = 0; j <= NU; ++j) sm.red[j][tid] += sm.red[j][tid + st];
        }
        __syncthreads();
    }
    if (tid < NU) a.u_out[h * NU + tid] = any ? sm.red[tid][0] / sm.red[NU][0] : un[tid];
    if (h == 0 && tid == 0) {
        if (!any) atomicOr(a.err, ERRB_NONFINITE);
        if (a.best) {
            a.best[0] = cmin;
            a.best[1] = (float)cidx;
        }
    }
}

// After a controller's H update CTAs: the last one to finish advances its
// iteration counter (counting, no waiting).  `ncta` = H.
template <int NU>
__device__ __forceinline__ void update_finish(const UpdateArgs& a, int ncta, UpdateSmem<NU>& sm) {
    if (!a.advance) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(a.done, 1u);
        sm.is_last = (t == (unsigned)ncta - 1u);
    }
    __syncthreads();
    if (sm.is_last && threadIdx.x == 0) {
        *a.done = 0u;
        *a.iter_ptr += 1ull;
        __threadfence();
    }
}

}  // namespace mppi
