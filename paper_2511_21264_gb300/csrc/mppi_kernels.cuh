// Per-sample rollout and per-horizon-step update, shared by the single-
// controller kernels and the batched persistent kernels.
#pragma once
#include "mppi_device.cuh"
#include "mppi_internal.h"
#include "mppi_task.cuh"

namespace mppi {

// Inputs of one sample's rollout (one lane group).
struct SampleIO {
    const float* x;            // start state (nx)
    const float* U;            // explicit controls of this sample, row h at U + h * u_stride, MODE 0
    long long u_stride;
    long long u_ext;           // floats from U to the end of the caller's control buffer, MODE 0
    const float* unom;         // nominal controls (H x nu, shared or global), MODE 1 and 2
    float sig, lo, hi;         // this lane's sigma and control bounds (group lane < nu), MODE 1 and 2
    uint2 key;                 // Philox key, MODE 1 and 2
    uint32_t iter;             // Philox iteration word, MODE 1 and 2
    int k, H;                  // sample index, horizon
    float* x_out;              // optional final state (nx)
    float* U_store;            // optional: sampled controls out, H x Kn x nu (h-major)
    int Kn;                    // sample count of U_store
    const float* Lfac;         // optional (MODE 2): H x nu x nu factors of the sampling covariance blocks
    int* err;                  // error word
    unsigned long long* stats; // optional [sample-steps, contacts, exact box tests]
    const DevTask* task;       // ball-task cost suite (TASK rollouts), in place of the stage cost
};

// Copy the scene model (and optionally u_nom) into shared memory.
__device__ __forceinline__ void stage_model(unsigned char* smem, const DevModel* model, float* unom_s,
                                            const float* u_nom, int unom_n) {
    const float4* src = reinterpret_cast<const float4*>(model);
    float4* dst = reinterpret_cast<float4*>(smem);
    for (int t = threadIdx.x; t < (int)(sizeof(DevModel) / 16); t += blockDim.x) dst[t] = src[t];
    for (int t = threadIdx.x; t < unom_n; t += blockDim.x) unom_s[t] = u_nom[t];
}

// H simulator steps of one sample with its stage costs (TASK: the ball-task
// cost suite instead, 32 lanes per sample only); the group's state stays in
// shared memory throughout.  PLACE selects where the lone ball contact's
// solve runs: 0 fused with the arms' factorisation (every lane runs both
// chains), 1 after it (the factor on one lane per arm, then the sweeps);
// both give the same bits.  Returns the summed cost on every lane.
template <int NA, int LPS, int MODE, bool TASK = false, int PLACE = 0>
__device__ __forceinline__ float rollout_sample(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g,
                                                const SampleIO& io) {
    using d = Dims<NA>;
    static_assert(!TASK || LPS == 32, "the ball-task cost suite runs on 32 lanes per sample");
    static_assert(d::NU <= LPS, "one lane per control");
    constexpr int PS = 32 / LPS;  // pair slots per lane
    constexpr int DS = LPS / 4;   // steps of normals per Philox draw (one block of 4 per lane)
    const int k = io.k;
    const int sl = g.sl;
#pragma unroll
    for (int c0 = 0; c0 < d::NX; c0 += LPS) {
        const int c = c0 + sl;
        if (c < d::NQ) w.q[c] = ld_checked(io.x, c, d::NX);
        else if (c < d::NX) w.qd[c - d::NQ] = ld_checked(io.x, c, d::NX);
    }
    g.sync();
    float cost = 0.0f;
    const float* gb = M.goal;
    unsigned n_exact = 0, n_con = 0, n_lone = 0;
    float uacc = 0.0f;  // this lane's control's sum of squares over the horizon
    float pacc[PS], pbacc[PS];  // this lane's contacts' depths (all, against boxes) over the horizon, per slot
#pragma unroll
    for (int t = 0; t < PS; ++t) pacc[t] = pbacc[t] = 0.0f;
    float gacc = 0.0f;  // squared goal error of this lane's ball coordinate over the horizon
    float kacc = 0.0f;  // squared grasp error (p_L + p_R - 2 p_ball) of this lane's coordinate
    TaskAcc<NA> tacc;
    if constexpr (TASK) {
#pragma unroll
        for (int s = 0; s < TaskDims<NA>::CB; ++s) tacc.prevb[s] = 0.0f;
#pragma unroll
        for (int s = 0; s < TaskDims<NA>::CC; ++s) tacc.prevc[s] = 0.0f;
        tacc.c = tacc.th = tacc.yz = tacc.v2 = tacc.r = tacc.l = tacc.eo = tacc.ot = 0.0f;
    }
    float upre = 0.0f;  // explicit controls: the next step's value
    if (MODE == 0 && sl < d::NU) upre = ld_checked(io.U, sl, io.u_ext);
    for (int h = 0; h < io.H; ++h) {
        if (MODE >= 1) {
            // every DS steps the group's lanes draw one Philox block each: DS
            // steps x 16 controls of standard normals, counter (j/4, h, k,
            // iteration), Box-Muller on the word pairs (the values sample_row
            // and the debug draw give)
            if ((h & (DS - 1)) == 0) {
                const int jb = sl & 3, hs = h + (sl >> 2);
                if (4 * jb < d::NU && hs < io.H) {
                    const uint4 wv = philox4x32_10(make_uint4((uint32_t)jb, (uint32_t)hs, (uint32_t)k, io.iter), io.key);
                    float z4[4];
                    block_normals4(wv, z4);
#pragma unroll
                    for (int t = 0; t < 4; ++t) w.zn[sl >> 2][4 * jb + t] = z4[t];
                }
                g.sync();
            }
            {  // every lane computes (past the controls on the last one), the controls' lanes store
                const int jc = sl < d::NU ? sl : d::NU - 1;
                const float* zr = w.zn[h & (DS - 1)];
                float acc = ld_checked(io.unom, h * d::NU + jc, (long long)io.H * d::NU);
                if (MODE == 2 && io.Lfac) {  // u = nu + L_h z, FMAs in the order sample_row uses
                    // (unrolled over the row so that its loads are issued together)
                    const long long r0 = ((long long)h * d::NU + jc) * d::NU, n_l = (long long)io.H * d::NU * d::NU;
#pragma unroll
                    for (int i = 0; i < d::NU; ++i)
                        if (i <= jc) acc = __fmaf_rn(ld_checked(io.Lfac, r0 + i, n_l), zr[i], acc);
                } else {
                    acc = __fmaf_rn(io.sig, zr[jc], acc);
                }
                const float uv = fminf(fmaxf(acc, io.lo), io.hi);
                if (sl < d::NU) {
                    w.u[sl] = uv;
                    uacc = __fmaf_rn(uv, uv, uacc);
                    const long long si = ((long long)h * io.Kn + k) * d::NU + sl;
                    if (io.U_store && MPPI_IN_RANGE(si, (long long)io.H * io.Kn * d::NU)) io.U_store[si] = uv;
                }
            }
        } else if (sl < d::NU) {
            const float uv = upre;  // read one step ahead: its latency overlaps the step
            if (h + 1 < io.H) upre = ld_checked(io.U, (h + 1) * io.u_stride + sl, io.u_ext);
            w.u[sl] = uv;
            uacc = __fmaf_rn(uv, uv, uacc);
        }
        float Rl[9], cl[3];  // this lane's link rotation and COM, kept for the dynamics
        forward_kinematics<NA>(M, w, g, Rl, cl);
        g.sync();
        if constexpr (TASK) {
            task_state<NA>(M, *io.task, w, sl, Rl, h == 0, tacc);
        } else {
            if (h > 0 && sl < 3 && M.w_grasp != 0.0f) kacc += grasp_coord<NA>(w, sl);
        }
        // the mass matrix and bias forces do not depend on the contacts:
        // formed before the collision phase, so that the link frames kept
        // from the kinematics are no longer live across it
        dynamics<NA>(M, w, g, io.err, Rl, cl, 0, false);
        int ncon, tb;
        n_exact += collide<NA>(M, w, g, pacc, pbacc, ncon, tb);
        g.sync();
        n_con += ncon;
        // one ball contact with static geometry (the lift's common case)
        const bool lone = tb == 4 && ncon == 1;
        n_lone += lone ? 1u : 0u;
        if (PLACE == 0) {
            // the arms' solve and the contact solve side by side
            if (lone) {
                solve_ball_contacts<NA, 1, 0>(M, w, g, io.err);
            } else {
                arm_factor_step<NA, LPS>(M, w, g, io.err, tb);
                contacts<NA>(M, w, g, ncon, tb);
            }
        } else {
            arm_factor_step<NA, LPS>(M, w, g, io.err, tb);
            contacts<NA>(M, w, g, ncon, tb);
        }
        integrate<NA>(M, w, g);
        if (!TASK && sl < 3) {  // the goal error of ball coordinate sl
            const float e = w.q[d::B + sl] - gb[sl];
            gacc = __fmaf_rn(e, e, gacc);
        }
        g.sync();
    }
    if constexpr (TASK) {
        float Rl[9], cl[3];
        forward_kinematics<NA>(M, w, g, Rl, cl);
        g.sync();
        task_state<NA>(M, *io.task, w, sl, Rl, false, tacc);
        cost = task_total<NA>(*io.task, tacc);
    } else if (M.w_grasp != 0.0f) {
        float Rl[9], cl[3];
        forward_kinematics<NA>(M, w, g, Rl, cl);
        g.sync();
        if (sl < 3) kacc += grasp_coord<NA>(w, sl);
    }
    if constexpr (!TASK) {
        // w_goal sum_h |p_ball - goal|^2 + w_u sum_h |u_h|^2 + w_pen sum_h pen_h
        // + w_obst sum_h pen_box_h + w_grasp sum_h |p_L + p_R - 2 p_ball|^2
        // from the lanes' sums, each reduced in the order of a 32-slot butterfly
        gacc = group_sum(g, gacc);
        uacc = group_sum(g, uacc);
        const float ps = slot_sum(g, pacc);
        const float pbs = slot_sum(g, pbacc);
        kacc = group_sum(g, kacc);
        cost += M.w_goal * gacc + M.w_u * uacc + M.w_pen * ps + M.w_obst * pbs + M.w_grasp * kacc;
    }
    // a non-finite state poisons the sample's cost (weight 0 in the update)
    bool bad = false;
#pragma unroll
    for (int c0 = 0; c0 < d::NQ; c0 += LPS) {
        const int c = c0 + sl;
        bad = bad || (c < d::NQ && !isfinite(w.q[c])) || (c < d::NV && !isfinite(w.qd[c]));
    }
    if (g.any(bad)) cost = __int_as_float(0x7fc00000);
    cost = g.shfl(cost, 0);
    if (sl == 0 && !isfinite(cost)) atomicOr(io.err, ERRB_NONFINITE);
    if (io.stats && sl == 0) {
        atomicAdd(&io.stats[0], (unsigned long long)io.H);
        atomicAdd(&io.stats[1], (unsigned long long)n_con);
        atomicAdd(&io.stats[2], (unsigned long long)n_exact);
        atomicAdd(&io.stats[3], (unsigned long long)n_lone);
    }
    if (io.x_out) {
#pragma unroll
        for (int c0 = 0; c0 < d::NX; c0 += LPS) {
            const int c = c0 + sl;
            if (c < d::NQ && MPPI_IN_RANGE(c, d::NX)) io.x_out[c] = w.q[c];
            else if (c < d::NX && MPPI_IN_RANGE(c, d::NX)) io.x_out[c] = w.qd[c - d::NQ];
        }
    }
    return cost;
}

// Shared memory of one update CTA.
template <int NU>
struct UpdateSmem {
    CArr<CArr<float, 256>, NU + 1> red;
    CArr<float, 256> rmin;
    CArr<int, 256> ridx;
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
        const float c = ld_checked(a.costs, k, a.K);
        if (isfinite(c) && (c < cm)) {
            cm = c;
            ci = k;
        }
    }
    // lowest (cost, index): butterfly within each warp, then the 8 warp
    // results in order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float o = __shfl_xor_sync(0xffffffffu, cm, off);
        const int oi = __shfl_xor_sync(0xffffffffu, ci, off);
        if (o < cm || (o == cm && oi < ci)) {
            cm = o;
            ci = oi;
        }
    }
    if ((tid & 31) == 0) {
        sm.rmin[tid >> 5] = cm;
        sm.ridx[tid >> 5] = ci;
    }
    __syncthreads();
    if (tid == 0) {
        for (int q = 1; q < T / 32; ++q)
            if (sm.rmin[q] < sm.rmin[0] || (sm.rmin[q] == sm.rmin[0] && sm.ridx[q] < sm.ridx[0])) {
                sm.rmin[0] = sm.rmin[q];
                sm.ridx[0] = sm.ridx[q];
            }
    }
    __syncthreads();
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
        un[j] = ld_checked(a.u_nom, h * NU + j, (long long)a.H * NU);
        sg[j] = ld_checked(a.sigma, j, NU);
        lo[j] = ld_checked(a.u_lo, j, NU);
        hi[j] = ld_checked(a.u_hi, j, NU);
    }
    if (any) {
        const float inv_lam = 1.0f / a.lambda;
        for (int k = tid; k < a.K; k += T) {
            const float c = ld_checked(a.costs, k, a.K);
            const float wk = isfinite(c) ? expf(-(c - cmin) * inv_lam) : 0.0f;
            Z += wk;
            if (a.U_stored) {
                // the rollout's own samples (bit-identical to regenerating them)
                const long long u0 = ((long long)h * a.K + k) * NU, n_u = (long long)a.H * a.K * NU;
#pragma unroll
                for (int j = 0; j < NU; ++j) acc[j] = __fmaf_rn(wk, ld_checked(a.U_stored, u0 + j, n_u), acc[j]);
            } else {
#pragma unroll
                for (int jb = 0; jb < (NU + 3) / 4; ++jb) {
                    const uint4 wv = philox4x32_10(make_uint4((uint32_t)jb, (uint32_t)h, (uint32_t)k, iter), key);
                    float z4[4];
                    block_normals4(wv, z4);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int j = 4 * jb + t;
                        if (j < NU) {
                            const float z = z4[t];
                            const float u = fminf(fmaxf(__fmaf_rn(sg[j], z, un[j]), lo[j]), hi[j]);
                            acc[j] = __fmaf_rn(wk, u, acc[j]);
                        }
                    }
                }
            }
        }
    }
    // fixed-order sums: butterfly within each warp, then the warps in order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int j = 0; j < NU; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], off);
        Z += __shfl_xor_sync(0xffffffffu, Z, off);
    }
    if ((tid & 31) == 0) {
#pragma unroll
        for (int j = 0; j < NU; ++j) sm.red[j][tid >> 5] = acc[j];
        sm.red[NU][tid >> 5] = Z;
    }
    __syncthreads();
    if (tid <= NU) {
        float t = sm.red[tid][0];
        for (int q = 1; q < T / 32; ++q) t += sm.red[tid][q];
        sm.red[tid][0] = t;
    }
    __syncthreads();
    if (tid < NU && MPPI_IN_RANGE(h * NU + tid, (long long)a.H * NU))
        a.u_out[h * NU + tid] = any ? sm.red[tid][0] / sm.red[NU][0] : un[tid];
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

namespace mppi {

// ---------------------------------------------------------------------------
// Eq. 8 in full: elite set, learning rate, per-step covariance blocks
// ---------------------------------------------------------------------------
// Sample row h of sample k: u_j = clamp(nu_j + sum_{i<=j} L_h[j][i] z_i)
// (FMAs in the order i = 0..j, as the rollout computes it), or with a
// diagonal sigma u_j = clamp(nu_j + sigma_j z_j).
template <int NU>
__device__ __forceinline__ void sample_row(uint2 key, uint32_t iter, int k, int h, const float* unom_h,
                                           const float* sigma, const float* L_h, const float* lo, const float* hi,
                                           float (&u)[NU]) {
    float z[NU];
#pragma unroll
    for (int jb = 0; jb < (NU + 3) / 4; ++jb) {
        const uint4 wv = philox4x32_10(make_uint4((uint32_t)jb, (uint32_t)h, (uint32_t)k, iter), key);
        float z4[4];
        block_normals4(wv, z4);
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (4 * jb + t < NU) z[4 * jb + t] = z4[t];
    }
#pragma unroll
    for (int j = 0; j < NU; ++j) {
        float acc = unom_h[j];
        if (L_h) {
#pragma unroll
            for (int i = 0; i <= j; ++i) acc = __fmaf_rn(L_h[j * NU + i], z[i], acc);
        } else {
            acc = __fmaf_rn(sigma[j], z[j], acc);
        }
        u[j] = fminf(fmaxf(acc, lo[j]), hi[j]);
    }
}

// Orderable 64-bit key of (cost, index): lower cost first, then lower index;
// non-finite costs sort last.
__device__ __forceinline__ unsigned long long cost_key(float c, int k) {
    unsigned u = isfinite(c) ? __float_as_uint(c) : 0xFFFFFFFFu;
    if (isfinite(c)) u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned)k;
}

struct EliteArgs {
    int K, H, n_elite, update_cov;
    float beta, eta, cov_floor;
    const float* costs;
    const float* u_nom;
    float* u_out;
    const float* sigma;
    const float* Lfac;  // H x NU x NU factors of the sampling blocks, or null (diagonal sigma)
    const float* u_lo;
    const float* u_hi;
    float* Sigma;       // H x NU x NU, updated in place when update_cov
    float* Lout;        // H x NU x NU, new factors when update_cov
    uint64_t seed;
    const unsigned long long* iter_ptr;
    unsigned long long iter_val;
    const float* U_stored;  // H x K x NU, or null (regenerate)
    const unsigned long long* sel;  // [threshold key, best key, finite count]
    const int* eidx;    // elite sample indices, lowest cost first
    float* best_U;      // optional H x NU: controls of the lowest-cost sample
    int* err;
    int advance;
    unsigned int* done;
};

template <int NU>
struct EliteSmem {
    CArr<CArr<float, 256>, NU + 1> red;
    CArr<CArr<float, NU + 1>, 64> d;  // a chunk of weighted deviations
    CArr<CArr<float, NU>, NU> cov;
    CArr<float, NU> mean;
    int is_last;
};

template <int NU>
__device__ __forceinline__ void elite_row(const EliteArgs& a, int h, int k, uint2 key, uint32_t iter,
                                          const float* unom_h, float (&u)[NU]) {
    if (a.U_stored) {
        const long long u0 = ((long long)h * a.K + k) * NU, n_u = (long long)a.H * a.K * NU;
#pragma unroll
        for (int j = 0; j < NU; ++j) u[j] = ld_checked(a.U_stored, u0 + j, n_u);
    } else {
        sample_row<NU>(key, iter, k, h, unom_h, a.sigma, a.Lfac ? a.Lfac + (size_t)h * NU * NU : nullptr, a.u_lo,
                       a.u_hi, u);
    }
}

// One CTA per horizon step h (256 threads).
template <int NU>
__device__ __forceinline__ void elite_update_step(const EliteArgs& a, int h, EliteSmem<NU>& sm) {
    constexpr int T = 256;
    const int tid = threadIdx.x;
    const uint32_t iter = (uint32_t)(a.iter_ptr ? *a.iter_ptr : a.iter_val);
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    const unsigned long long bestk = a.sel[1];
    const bool any = a.sel[2] > 0;
    const float cmin = any ? ld_checked(a.costs, (long long)(bestk & 0xFFFFFFFFull), a.K) : 0.0f;
    float unom_h[NU];
#pragma unroll
    for (int j = 0; j < NU; ++j) unom_h[j] = ld_checked(a.u_nom, h * NU + j, (long long)a.H * NU);
    const float inv_beta = 1.0f / a.beta;
    // (1) weighted elite mean over the elite list
    const int nfin = (int)a.sel[2];
    const int ne = nfin < a.n_elite ? nfin : a.n_elite;
    float acc[NU];
#pragma unroll
    for (int j = 0; j < NU; ++j) acc[j] = 0.0f;
    float Z = 0.0f;
    const bool cached = ne <= 64;  // the covariance pass then reuses the rows kept here
    for (int e = tid; e < ne; e += T) {
        const int k = ld_checked(a.eidx, e, a.K);
        const float wk = expf(-(ld_checked(a.costs, k, a.K) - cmin) * inv_beta);
        float u[NU];
        elite_row<NU>(a, h, k, key, iter, unom_h, u);
        Z += wk;
        // products and sums with their rounding written out (explicit FMAs):
        // every kernel that inlines this step computes the same bits
#pragma unroll
        for (int j = 0; j < NU; ++j) acc[j] = __fmaf_rn(wk, u[j], acc[j]);
        if (cached) {
#pragma unroll
            for (int j = 0; j < NU; ++j) sm.d[e][j] = u[j];
            sm.d[e][NU] = wk;
        }
    }
    // fixed-order sums: butterfly within each warp, then the warps in order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int j = 0; j < NU; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], off);
        Z += __shfl_xor_sync(0xffffffffu, Z, off);
    }
    if ((tid & 31) == 0) {
#pragma unroll
        for (int j = 0; j < NU; ++j) sm.red[j][tid >> 5] = acc[j];
        sm.red[NU][tid >> 5] = Z;
    }
    __syncthreads();
    if (tid <= NU) {
        float t = sm.red[tid][0];
        for (int q = 1; q < T / 32; ++q) t += sm.red[tid][q];
        sm.red[tid][0] = t;
    }
    __syncthreads();
    const float Zs = sm.red[NU][0];
    if (tid < NU) {
        const float m = any ? sm.red[tid][0] / Zs : unom_h[tid];
        sm.mean[tid] = any ? __fmaf_rn(a.eta, m, __fmul_rn(1.0f - a.eta, unom_h[tid])) : unom_h[tid];
    }
    // the lowest-cost sample's row, read before this CTA rewrites the block's
    // factor (regeneration samples through the current factor)
    if (a.best_U && any && tid == 0) {
        float u[NU];
        elite_row<NU>(a, h, (int)(bestk & 0xFFFFFFFFull), key, iter, unom_h, u);
#pragma unroll
        for (int j = 0; j < NU; ++j)
            if (MPPI_IN_RANGE(h * NU + j, (long long)a.H * NU)) a.best_U[h * NU + j] = u[j];
    }
    __syncthreads();
    // (2) weighted covariance about the new mean, one block per step
    if (a.update_cov && any) {
        constexpr int NE = NU * (NU + 1) / 2;
        float cv = 0.0f;
        int ci = 0, cj = 0;
        if (tid < NE) {  // entry (ci, cj), cj <= ci
            int rem = tid;
            while (rem > ci) {
                rem -= ci + 1;
                ++ci;
            }
            cj = rem;
        }
        for (int e0 = 0; e0 < ne; e0 += 64) {
            if (tid < 64) {
                const int e = e0 + tid;
                float wk = 0.0f;
                float u[NU];
#pragma unroll
                for (int j = 0; j < NU; ++j) u[j] = sm.mean[j];
                if (e < ne) {
                    if (cached) {  // this thread's own row from the mean pass
#pragma unroll
                        for (int j = 0; j < NU; ++j) u[j] = sm.d[tid][j];
                        wk = sm.d[tid][NU];
                    } else {
                        const int k = ld_checked(a.eidx, e, a.K);
                        wk = expf(-(ld_checked(a.costs, k, a.K) - cmin) * inv_beta);
                        elite_row<NU>(a, h, k, key, iter, unom_h, u);
                    }
                }
#pragma unroll
                for (int j = 0; j < NU; ++j) sm.d[tid][j] = u[j] - sm.mean[j];
                sm.d[tid][NU] = wk;
            }
            __syncthreads();
            if (tid < NE) {
                const int nt = ne - e0 < 64 ? ne - e0 : 64;
#pragma unroll 4
                for (int t = 0; t < nt; ++t) cv = __fmaf_rn(__fmul_rn(sm.d[t][NU], sm.d[t][ci]), sm.d[t][cj], cv);
            }
            __syncthreads();
        }
        if (tid < NE) {
            const long long n_s = (long long)a.H * NU * NU;
            float v = __fmaf_rn(a.eta, cv / Zs,
                                __fmul_rn(1.0f - a.eta, ld_checked(a.Sigma, (long long)h * NU * NU + ci * NU + cj, n_s)));
            if (ci == cj) v += a.cov_floor;
            sm.cov[ci][cj] = v;
            sm.cov[cj][ci] = v;
        }
        __syncthreads();
        if (tid < NU * NU && MPPI_IN_RANGE((long long)h * NU * NU + tid, (long long)a.H * NU * NU))
            a.Sigma[(size_t)h * NU * NU + tid] = sm.cov[tid / NU][tid % NU];
        __syncthreads();
        if (tid < 32) {  // factor the new block in place (one warp, right-looking) for the next sampling
            bool ok = true;
            for (int j = 0; j < NU; ++j) {
                const float s = sm.cov[j][j];
                ok = ok && s > 0.0f;
                const float dj = sqrtf(fmaxf(s, 1e-30f)), inv = 1.0f / dj;
                __syncwarp();
                for (int r = j + 1 + tid; r < NU; r += 32) sm.cov[r][j] *= inv;
                if (tid == 0) sm.cov[j][j] = dj;
                __syncwarp();
                const int n = NU - j - 1;
                for (int t = tid; t < n * n; t += 32) {
                    const int r = j + 1 + t / n, q = j + 1 + t % n;
                    if (q <= r) sm.cov[r][q] = __fmaf_rn(-sm.cov[r][j], sm.cov[q][j], sm.cov[r][q]);
                }
                __syncwarp();
            }
            if (ok) {
                float* Lo = a.Lout + (size_t)h * NU * NU;
                for (int t = tid; t < NU * NU; t += 32)
                    if (MPPI_IN_RANGE((long long)h * NU * NU + t, (long long)a.H * NU * NU))
                        Lo[t] = (t % NU) <= (t / NU) ? sm.cov[t / NU][t % NU] : 0.0f;
            } else if (tid == 0) {
                atomicOr(a.err, ERRB_CHOLESKY);
            }
        }
    }
    // (3) outputs (u_out may alias u_nom: this CTA read its row above)
    if (tid < NU && MPPI_IN_RANGE(h * NU + tid, (long long)a.H * NU)) a.u_out[h * NU + tid] = sm.mean[tid];
    if (h == 0 && tid == 0 && !any) atomicOr(a.err, ERRB_NONFINITE);
}

// Elite threshold: bitonic sort of (cost, index) keys in shared memory (one
// CTA of 1024 threads, P = power of two >= K; keys holds 2048 keys when
// P <= 1024, else P); sel = [key of the n_e-th elite, lowest key, finite
// count], eidx = the elite indices in cost order.
__device__ __forceinline__ void elite_select_block(const float* costs, int K, int P, int n_elite,
                                                  unsigned long long* sel, int* eidx, unsigned long long* keys,
                                                  int& nfin) {
    if (P <= 1024) {
        // one key per thread (padding keys sort last): the same bitonic
        // network in registers, partners by shuffles below stride 32 and
        // through a double-buffered shared array above
        const int t = threadIdx.x;
        unsigned long long x = ~0ull;
        bool fin = false;
        if (t < K) {
            const float c = ld_checked(costs, t, K);
            x = cost_key(c, t);
            fin = isfinite(c);
        }
        const int nf = __syncthreads_count(fin);
        int buf = 0;
        for (int size = 2; size <= 1024; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                unsigned long long y;
                if (stride >= 32) {
                    if (MPPI_IN_RANGE(buf * 1024 + t, 2048)) keys[buf * 1024 + t] = x;
                    __syncthreads();
                    y = MPPI_IN_RANGE(buf * 1024 + (t ^ stride), 2048) ? keys[buf * 1024 + (t ^ stride)] : x;
                    buf ^= 1;
                } else {
                    y = __shfl_xor_sync(0xffffffffu, x, stride);
                }
                const bool asc = (t & size) == 0, lower = (t & stride) == 0;
                x = (lower == asc) ? (x < y ? x : y) : (x < y ? y : x);
            }
        const int ne = nf == 0 ? 0 : (n_elite < nf ? n_elite : nf);
        if (t < ne && MPPI_IN_RANGE(t, K)) eidx[t] = (int)(x & 0xFFFFFFFFull);
        if (t == 0) {
            sel[1] = x;
            sel[2] = (unsigned long long)nf;
            if (ne == 0) sel[0] = 0ull;
        }
        if (ne > 0 && t == ne - 1) sel[0] = x;
        return;
    }
    if (threadIdx.x == 0) nfin = 0;
    __syncthreads();
    int mine = 0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const float c = i < K ? ld_checked(costs, i, K) : 0.0f;
        if (MPPI_IN_RANGE(i, P)) keys[i] = i < K ? cost_key(c, i) : ~0ull;
        mine += (i < K && isfinite(c)) ? 1 : 0;
    }
    atomicAdd(&nfin, mine);
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i && MPPI_IN_RANGE(j, P)) {
                    const bool asc = (i & size) == 0;
                    const unsigned long long x = keys[i], y = keys[j];
                    if ((x > y) == asc) {
                        keys[i] = y;
                        keys[j] = x;
                    }
                }
            }
            __syncthreads();
        }
    const int nf = nfin;
    const int ne = nf == 0 ? 0 : (n_elite < nf ? n_elite : nf);
    for (int e = threadIdx.x; e < ne; e += blockDim.x)
        if (MPPI_IN_RANGE(e, K)) eidx[e] = (int)(keys[e] & 0xFFFFFFFFull);
    if (threadIdx.x == 0) {
        sel[0] = ne > 0 ? keys[ne - 1] : 0ull;
        sel[1] = keys[0];
        sel[2] = (unsigned long long)nf;
    }
}

}  // namespace mppi
