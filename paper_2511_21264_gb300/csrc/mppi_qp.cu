// QP smoothing projection (Eq. 5): each sampled joint-velocity sequence is
// moved to the nearest sequence (in the 2-norm) whose position, velocity,
// acceleration and jerk (r = 0..3, Sec. III) stay within their bounds.
//
// Solver: a fixed number of ADMM iterations (the paper names none).  Two
// kernels run the same iteration:
//
// H <= 32: one warp per sequence, lane t = horizon step, in the velocity
// coordinates themselves.  The rows come from warp scans and neighbour
// shuffles (position = prefix sum, acceleration and jerk = differences),
// their transposes from a suffix scan and two shuffles, and the linear
// solve is a product with the precomputed inverse of I + rho D^T D (shared
// by every sequence of a class), whose row t each lane keeps in registers.
// Many warps per SM hide the shuffle and FMA latencies.
//
// Longer horizons: one thread per sequence.  The iteration is run in the coordinates
//   x_i = sum_{t<i} v_t   (i = 1..H, the position offset over dt),
// where every constraint row touches at most four consecutive x_i and the
// ADMM linear system  N x = B^T vt + rho D^T (w - y),  N = B^T B + rho D^T D
// (B: first differences, D: the scaled rows) is banded with bandwidth 3.
// N depends only on H, rho and the group scales, so its band Cholesky factor
// is computed once on the host in FP64 and shared by every sequence of a
// class (one class per joint).  Changing coordinates leaves the ADMM
// iterates unchanged in exact arithmetic; only the rounding differs.
//
// Per iteration a thread makes one forward sweep over t that evaluates the
// four rows at t, updates their scaled duals y (w = clip(D x + y),
// y = D x + y - w), accumulates the right-hand side D^T (w - y) and runs
// the forward substitution three indices behind, then one backward
// substitution sweep.  The per-thread vectors live in shared memory, laid
// out [t][thread] so that a warp's accesses are conflict-free; the band
// factors are read through the read-only cache, uniform across a warp when
// its sequences share a class.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/mppi.h"
#include "mppi_device.cuh"
#include "mppi_internal.h"

namespace mppi {

namespace {

constexpr int QP_THREADS = 64;

// x-coordinate form of one scaled row group: value at t is
// s * (x_{t+1} + c1 x_t + c2 x_{t-1} + c3 x_{t-2})
void add_group(std::vector<double>& N, int H, double w, const double* c, int t0) {
    for (int t = t0; t < H; ++t) {
        int idx[4];
        double co[4];
        int m = 0;
        for (int d = 0; d < 4; ++d) {
            const int i = t + 1 - d;  // x index (1-based); i <= 0 are fixed at zero
            if (i >= 1 && c[d] != 0.0) {
                idx[m] = i - 1;
                co[m] = c[d];
                ++m;
            }
        }
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b) N[(size_t)idx[a] * H + idx[b]] += w * co[a] * co[b];
    }
}

}  // namespace

// Band factor of N for one class: 2H float4, forward rows then backward rows.
int qp_band_factor(int H, double rho, const double sc[4], float4* band) {
    std::vector<double> N((size_t)H * H, 0.0);
    static const double cB[4] = {1, -1, 0, 0}, cP[4] = {1, 0, 0, 0}, cA[4] = {1, -2, 1, 0}, cJ[4] = {1, -3, 3, -1};
    add_group(N, H, 1.0, cB, 0);                       // objective 1/2 |B x - vt|^2
    add_group(N, H, rho * sc[0] * sc[0], cP, 0);       // position rows
    add_group(N, H, rho * sc[1] * sc[1], cB, 0);       // velocity rows
    add_group(N, H, rho * sc[2] * sc[2], cA, 0);       // acceleration rows
    add_group(N, H, rho * sc[3] * sc[3], cJ, 1);       // jerk rows, t >= 1
    // dense Cholesky (N is SPD); the factor keeps the band of N
    for (int j = 0; j < H; ++j) {
        double s = N[(size_t)j * H + j];
        for (int k = 0; k < j; ++k) s -= N[(size_t)j * H + k] * N[(size_t)j * H + k];
        if (!(s > 0.0)) return MPPI_ERR_CHOLESKY;
        const double d = std::sqrt(s);
        N[(size_t)j * H + j] = d;
        for (int i = j + 1; i < H; ++i) {
            double t = N[(size_t)i * H + j];
            for (int k = 0; k < j; ++k) t -= N[(size_t)i * H + k] * N[(size_t)j * H + k];
            N[(size_t)i * H + j] = t / d;
        }
    }
    auto L = [&](int i, int j) { return (i >= 0 && i < H && j >= 0 && j <= i && i - j <= 3) ? N[(size_t)i * H + j] : 0.0; };
    for (int i = 0; i < H; ++i) {
        const double dinv = 1.0 / L(i, i);
        band[i] = make_float4((float)dinv, (float)L(i, i - 1), (float)L(i, i - 2), (float)L(i, i - 3));
        band[H + i] = make_float4((float)dinv, (float)L(i + 1, i), (float)L(i + 2, i), (float)L(i + 3, i));
    }
    return MPPI_OK;
}

// Inverse of I + rho D^T D in velocity coordinates (H <= 32), rows padded to
// 32 columns, rows >= H zero.  D's rows: position (prefix sums), velocity,
// acceleration (first differences), jerk (second differences, t >= 1), each
// group times its scale.
int qp_dense_inverse(int H, double rho, const double sc[4], float* minv) {
    if (H < 1 || H > QP_WARP_MAX_H) return MPPI_ERR_INVALID_ARG;
    std::vector<double> A((size_t)H * H, 0.0), row(H);
    auto add_row = [&](double w) {
        for (int a = 0; a < H; ++a)
            if (row[a] != 0.0)
                for (int b = 0; b < H; ++b) A[(size_t)a * H + b] += w * row[a] * row[b];
    };
    for (int t = 0; t < H; ++t) {
        std::fill(row.begin(), row.end(), 0.0);
        for (int i = 0; i <= t; ++i) row[i] = 1.0;
        add_row(rho * sc[0] * sc[0]);
        std::fill(row.begin(), row.end(), 0.0);
        row[t] = 1.0;
        add_row(rho * sc[1] * sc[1]);
        if (t >= 1) row[t - 1] = -1.0;
        add_row(rho * sc[2] * sc[2]);
        if (t >= 1) {
            std::fill(row.begin(), row.end(), 0.0);
            row[t] = 1.0;
            row[t - 1] = -2.0;
            if (t >= 2) row[t - 2] = 1.0;
            add_row(rho * sc[3] * sc[3]);
        }
    }
    for (int i = 0; i < H; ++i) A[(size_t)i * H + i] += 1.0;
    // Cholesky, then the inverse column by column
    for (int j = 0; j < H; ++j) {
        double s = A[(size_t)j * H + j];
        for (int k = 0; k < j; ++k) s -= A[(size_t)j * H + k] * A[(size_t)j * H + k];
        if (!(s > 0.0)) return MPPI_ERR_CHOLESKY;
        const double d = std::sqrt(s);
        A[(size_t)j * H + j] = d;
        for (int i = j + 1; i < H; ++i) {
            double t = A[(size_t)i * H + j];
            for (int k = 0; k < j; ++k) t -= A[(size_t)i * H + k] * A[(size_t)j * H + k];
            A[(size_t)i * H + j] = t / d;
        }
    }
    std::fill(minv, minv + 32 * 32, 0.0f);
    std::vector<double> x(H);
    for (int c = 0; c < H; ++c) {
        for (int i = 0; i < H; ++i) {  // L y = e_c
            double t = i == c ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= A[(size_t)i * H + k] * x[k];
            x[i] = t / A[(size_t)i * H + i];
        }
        for (int i = H - 1; i >= 0; --i) {  // L^T x = y
            double t = x[i];
            for (int k = i + 1; k < H; ++k) t -= A[(size_t)k * H + i] * x[k];
            x[i] = t / A[(size_t)i * H + i];
        }
        for (int i = 0; i < H; ++i) minv[i * 32 + c] = (float)x[i];
    }
    return MPPI_OK;
}

// Class record from 8 physical bounds: free groups get scale 0.
void qp_make_class(const float b[8], const float sc[4], float rho, QPClass* c) {
    std::memset(c, 0, sizeof *c);
    for (int g = 0; g < 4; ++g) {
        c->lo[g] = b[2 * g];
        c->hi[g] = b[2 * g + 1];
        const bool free_g = std::isinf(b[2 * g]) && b[2 * g] < 0 && std::isinf(b[2 * g + 1]) && b[2 * g + 1] > 0;
        c->s[g] = free_g ? 0.0f : sc[g];
    }
    c->rho = rho;
}

int qp_validate(const float b[8], const float sc[4], float rho) {
    if (!(rho > 0.0f) || !std::isfinite(rho)) return MPPI_ERR_INVALID_ARG;
    for (int g = 0; g < 4; ++g) {
        if (std::isnan(b[2 * g]) || std::isnan(b[2 * g + 1]) || !(b[2 * g] <= b[2 * g + 1])) return MPPI_ERR_INVALID_ARG;
        if (!(sc[g] > 0.0f) || !std::isfinite(sc[g])) return MPPI_ERR_INVALID_ARG;
    }
    return MPPI_OK;
}

// ---------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------

// scaled bounds of one row group: [s lo, s hi], or unbounded for a free group
__device__ __forceinline__ void qp_bound(float s, float lo, float hi, float& blo, float& bhi) {
    if (s == 0.0f) {
        blo = -INFINITY;
        bhi = INFINITY;
    } else {
        blo = s * lo;
        bhi = s * hi;
    }
}

// One row: s = val + y; w = clip(s); y = s - w; returns e = rho s_g (w - y).
__device__ __forceinline__ float qp_row(float val, float& y, float lo, float hi, float rs) {
    const float s = val + y;
    const float w = fminf(fmaxf(s, lo), hi);
    y = s - w;
    return rs * (w - y);
}

// ADMM iterations of one thread's sequence.  xb[t*T] = (x_{t+1}, (B^T vt)_{t+1})
// on entry holds the start point x = prefix sums of vt; y[t*T] = 0.  On exit
// xb[.].x holds the last iterate.
__device__ void qp_admm(const QPClass& c, const float4* __restrict__ band, int H, int iters, float dt, float q,
                        float qd, float2* xb, float4* yv, int T) {
    const float s0 = c.s[0], s1 = c.s[1], s2 = c.s[2], s3 = c.s[3];
    const float rs0 = c.rho * s0, rs1 = c.rho * s1, rs2 = c.rho * s2, rs3 = c.rho * s3;
    float Plo, Phi, Vlo, Vhi, Alo, Ahi, A0lo, A0hi, Jlo, Jhi, J1lo, J1hi;
    const float idt = 1.0f / dt, dt2 = dt * dt;
    qp_bound(s0, (c.lo[0] - q) * idt, (c.hi[0] - q) * idt, Plo, Phi);
    qp_bound(s1, c.lo[1], c.hi[1], Vlo, Vhi);
    qp_bound(s2, c.lo[2] * dt, c.hi[2] * dt, Alo, Ahi);
    qp_bound(s2, c.lo[2] * dt + qd, c.hi[2] * dt + qd, A0lo, A0hi);  // v_{-1} = qd moved into the bounds
    qp_bound(s3, c.lo[3] * dt2, c.hi[3] * dt2, Jlo, Jhi);
    qp_bound(s3, c.lo[3] * dt2 - qd, c.hi[3] * dt2 - qd, J1lo, J1hi);
    const float4* __restrict__ bf = band;      // forward rows
    const float4* __restrict__ bb = band + H;  // backward rows
    // slot index i (0 <= i < H) of this thread's vectors and band rows;
    // checked in the bounds-check build, the identity otherwise
    auto sl = [H](int i) { return MPPI_IN_RANGE(i, H) ? i : 0; };

    for (int it = 0; it < iters; ++it) {
        // forward sweep: rows at t, right-hand side, forward substitution
        float x0 = 0.0f;                         // x_t (x_0 and earlier are zero)
        float d1p = 0.0f, d2p = 0.0f;            // first and second differences at t-1
        float r0 = 0.0f, r1 = 0.0f, r2 = 0.0f;   // rhs of x_{t-2}, x_{t-1}, x_t
        float z1 = 0.0f, z2 = 0.0f, z3 = 0.0f;   // z_{i-1}, z_{i-2}, z_{i-3} of the substitution
        // unrolled so that the next steps' loads are in flight during the
        // substitution chain (the operations and their order are unchanged)
#pragma unroll 4
        for (int t = 0; t < H; ++t) {
            const float2 xv = xb[(size_t)sl(t) * T];
            float4 y = yv[(size_t)sl(t) * T];
            const float xp1 = xv.x;
            const float d1 = xp1 - x0, d2 = d1 - d1p, d3 = d2 - d2p;
            const float eP = qp_row(s0 * xp1, y.x, Plo, Phi, rs0);
            const float eV = qp_row(s1 * d1, y.y, Vlo, Vhi, rs1);
            const float eA = qp_row(s2 * d2, y.z, t == 0 ? A0lo : Alo, t == 0 ? A0hi : Ahi, rs2);
            float eJ = 0.0f;
            if (t >= 1) eJ = qp_row(s3 * d3, y.w, t == 1 ? J1lo : Jlo, t == 1 ? J1hi : Jhi, rs3);
            yv[(size_t)sl(t) * T] = y;
            // row t touches x_{t+1} (+1), x_t (-1, -2, -3), x_{t-1} (+1, +3), x_{t-2} (-1)
            const float r3 = xv.y + eP + eV + eA + eJ;
            r2 = r2 - eV - 2.0f * eA - 3.0f * eJ;
            r1 = r1 + eA + 3.0f * eJ;
            r0 = r0 - eJ;
            if (t >= 3) {  // x_{t-2} is complete: substitute (index i = t-2, slot t-3)
                const float4 L = __ldg(&bf[sl(t - 3)]);
                const float z = (r0 - L.y * z1 - L.z * z2 - L.w * z3) * L.x;
                xb[(size_t)sl(t - 3) * T].x = z;
                z3 = z2;
                z2 = z1;
                z1 = z;
            }
            r0 = r1;
            r1 = r2;
            r2 = r3;
            x0 = xp1;
            d2p = d2;
            d1p = d1;
        }
        // the last (up to) three indices: r0, r1, r2 belong to x_{H-2}, x_{H-1}, x_H
        for (int i = H - 2; i <= H; ++i) {
            const float r = i == H - 2 ? r0 : (i == H - 1 ? r1 : r2);
            if (i < 1) continue;
            const float4 L = __ldg(&bf[sl(i - 1)]);
            const float z = (r - L.y * z1 - L.z * z2 - L.w * z3) * L.x;
            xb[(size_t)sl(i - 1) * T].x = z;
            z3 = z2;
            z2 = z1;
            z1 = z;
        }
        // backward substitution L^T x = z
        float p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;  // x_{i+1}, x_{i+2}, x_{i+3}
#pragma unroll 4
        for (int i = H; i >= 1; --i) {
            const float4 L = __ldg(&bb[sl(i - 1)]);
            float* slot = &xb[(size_t)sl(i - 1) * T].x;
            const float xi = (*slot - L.y * p1 - L.z * p2 - L.w * p3) * L.x;
            *slot = xi;
            p3 = p2;
            p2 = p1;
            p1 = xi;
        }
    }
}

// Raw sample h of member k (sample) in class j (joint): the value the
// rollout's sampler draws, unclamped.
__device__ __forceinline__ float qp_sample(const QPArgs& a, uint2 key, uint32_t iter, int k, int j, int h) {
    float v = ld_checked(a.u_nom, (long long)h * a.nu + j, (long long)a.H * a.nu);
    if (a.Lfac) {
        const long long r0 = ((long long)h * a.nu + j) * a.nu, n_l = (long long)a.H * a.nu * a.nu;
        for (int jb = 0; 4 * jb <= j; ++jb) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)jb, (uint32_t)h, (uint32_t)k, iter), key);
            for (int t = 0; t < 4 && 4 * jb + t <= j; ++t)
                v = __fmaf_rn(ld_checked(a.Lfac, r0 + 4 * jb + t, n_l), block_normal(w, t), v);
        }
    } else {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(j >> 2), (uint32_t)h, (uint32_t)k, iter), key);
        v = __fmaf_rn(ld_checked(a.sigma, j, a.nu), block_normal(w, j & 3), v);
    }
    return v;
}

// ADMM iterations of one sequence held by one warp (lane = step t < H);
// Mi = this lane's row of the inverse, bc = 32 floats of this warp's shared
// memory.  Returns v_t (0 on lanes >= H).
__device__ __forceinline__ float qp_warp_admm(const QPClass& c, const float (&Mi)[32], int H, int iters, float dt,
                                              float q, float qd, float vt, int lane, float* bc) {
    const bool act = lane < H;
    const float s0 = c.s[0], s1 = c.s[1], s2 = c.s[2], s3 = c.s[3];
    const float rs0 = c.rho * s0, rs1 = c.rho * s1, rs2 = c.rho * s2, rs3 = c.rho * s3;
    const float idt = 1.0f / dt, dt2 = dt * dt;
    float Plo, Phi, Vlo, Vhi, Alo, Ahi, Jlo, Jhi;
    qp_bound(s0, (c.lo[0] - q) * idt, (c.hi[0] - q) * idt, Plo, Phi);
    qp_bound(s1, c.lo[1], c.hi[1], Vlo, Vhi);
    // v_{-1} = qd moves into the bounds of the first acceleration and jerk rows
    qp_bound(s2, c.lo[2] * dt + (lane == 0 ? qd : 0.0f), c.hi[2] * dt + (lane == 0 ? qd : 0.0f), Alo, Ahi);
    qp_bound(s3, c.lo[3] * dt2 - (lane == 1 ? qd : 0.0f), c.hi[3] * dt2 - (lane == 1 ? qd : 0.0f), Jlo, Jhi);
    float v = act ? vt : 0.0f;
    const float vt0 = v;
    float yP = 0.0f, yV = 0.0f, yA = 0.0f, yJ = 0.0f;
    const float4* bc4 = reinterpret_cast<const float4*>(bc);
    for (int it = 0; it < iters; ++it) {
        // rows at step t: prefix sum, v, first and second differences
        float pre = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float n = __shfl_up_sync(FULL, pre, d);
            if (lane >= d) pre += n;
        }
        float vm1 = __shfl_up_sync(FULL, v, 1), vm2 = __shfl_up_sync(FULL, v, 2);
        if (lane < 1) vm1 = 0.0f;
        if (lane < 2) vm2 = 0.0f;
        const float d1 = v - vm1, d2 = d1 - (vm1 - vm2);
        float eP = qp_row(s0 * pre, yP, Plo, Phi, rs0);
        float eV = qp_row(s1 * v, yV, Vlo, Vhi, rs1);
        float eA = qp_row(s2 * d1, yA, Alo, Ahi, rs2);
        float eJ = lane >= 1 ? qp_row(s3 * d2, yJ, Jlo, Jhi, rs3) : 0.0f;
        if (!act) eP = eV = eA = eJ = 0.0f;
        // right-hand side vt + D^T e: suffix sum (position), e (velocity),
        // e_t - e_{t+1} (acceleration), e_t - 2 e_{t+1} + e_{t+2} (jerk)
        float suf = eP;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float n = __shfl_down_sync(FULL, suf, d);
            if (lane + d < 32) suf += n;
        }
        float c1 = __shfl_down_sync(FULL, -eA - 2.0f * eJ, 1), c2 = __shfl_down_sync(FULL, eJ, 2);
        if (lane + 1 >= 32) c1 = 0.0f;
        if (lane + 2 >= 32) c2 = 0.0f;
        const float rhs = vt0 + suf + eV + eA + eJ + c1 + c2;
        // v = (I + rho D^T D)^-1 rhs
        bc[lane] = rhs;
        __syncwarp();
        float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, acc3 = 0.0f;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const float4 r = bc4[s];
            acc0 = __fmaf_rn(Mi[4 * s + 0], r.x, acc0);
            acc1 = __fmaf_rn(Mi[4 * s + 1], r.y, acc1);
            acc2 = __fmaf_rn(Mi[4 * s + 2], r.z, acc2);
            acc3 = __fmaf_rn(Mi[4 * s + 3], r.w, acc3);
        }
        __syncwarp();
        v = act ? (acc0 + acc1) + (acc2 + acc3) : 0.0f;
    }
    return v;
}

__device__ __forceinline__ void qp_load_row(const float* minv_cls, int lane, float (&Mi)[32]) {
    const float4* r = reinterpret_cast<const float4*>(minv_cls + (size_t)lane * 32);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const float4 m = __ldg(&r[s]);
        Mi[4 * s + 0] = m.x;
        Mi[4 * s + 1] = m.y;
        Mi[4 * s + 2] = m.z;
        Mi[4 * s + 3] = m.w;
    }
}

// Controller form: CTA = sample k, warp = joint j (nu warps); the CTA's
// projected sequences are staged in shared memory and written to the h-major
// sample buffer as contiguous rows of nu values.
__global__ void __launch_bounds__(14 * 32, 2) qp_warp_sample_kernel(QPArgs a) {
    extern __shared__ __align__(16) float wsm[];
    const int lane = threadIdx.x & 31, j = threadIdx.x >> 5, k = blockIdx.x, nu = a.nu;
    float* bc = wsm + 32 * j;
    float* stage = wsm + 32 * nu;  // H x nu
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    const uint32_t iter = (uint32_t)(a.iter_ptr ? *a.iter_ptr : a.iter_val);
    const QPClass c = a.cls[MPPI_IN_RANGE(j, a.n_cls) ? j : 0];
    float Mi[32];
    qp_load_row(a.minv + (size_t)(MPPI_IN_RANGE(j, a.n_cls) ? j : 0) * 32 * 32, lane, Mi);
    const float vt = lane < a.H ? qp_sample(a, key, iter, k, j, lane) : 0.0f;
    const float v = qp_warp_admm(c, Mi, a.H, a.iters, a.dt, ld_checked(a.q0, j, a.n_cls), ld_checked(a.qd0, j, a.n_cls),
                                 vt, lane, bc);
    // shared memory: nu rows of 32 floats, then the H x nu stage
    if (lane < a.H && MPPI_IN_RANGE(lane * nu + j, a.H * nu)) stage[lane * nu + j] = v;
    __syncthreads();
    for (int i = threadIdx.x; i < a.H * nu; i += blockDim.x) {
        const long long o = ((long long)(i / nu) * a.per_cls + k) * nu + (i % nu);
        if (MPPI_IN_RANGE(o, a.out_n)) a.out[o] = stage[i];
    }
}

// Standalone form: 8 warps per CTA, one sequence (class 0) each.
__global__ void __launch_bounds__(256) qp_warp_kernel(QPArgs a) {
    __shared__ __align__(16) float bcs[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 8 + w;
    if (i >= a.n) return;
    float Mi[32];
    qp_load_row(a.minv, lane, Mi);
    const float vt = lane < a.H ? ld_checked(a.vin, (long long)i * a.H + lane, a.in_n) : 0.0f;
    const float v = qp_warp_admm(a.cls[0], Mi, a.H, a.iters, a.dt, ld_checked(a.q0, i, a.n), ld_checked(a.qd0, i, a.n),
                                 vt, lane, bcs[MPPI_IN_RANGE(w, 8) ? w : 0]);
    if (lane < a.H && MPPI_IN_RANGE((long long)i * a.H + lane, a.out_n)) a.out[(size_t)i * a.H + lane] = v;
}

// Sequence i: class i / per_cls, member i % per_cls.
__global__ void __launch_bounds__(QP_THREADS) qp_project_kernel(QPArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x, tid = threadIdx.x;
    float4* yv = reinterpret_cast<float4*>(smem) + tid;
    float2* xb = reinterpret_cast<float2*>(smem + (size_t)a.H * T * sizeof(float4)) + tid;
    const int i = blockIdx.x * T + tid;
    if (i >= a.n) return;
    const int cls = i / a.per_cls, mem = i % a.per_cls;
    const QPClass c = a.cls[MPPI_IN_RANGE(cls, a.n_cls) ? cls : 0];
    const long long nq = a.q_per_seq ? a.n : a.n_cls;
    const float q = ld_checked(a.q0, a.q_per_seq ? i : cls, nq), qd = ld_checked(a.qd0, a.q_per_seq ? i : cls, nq);
    auto sl = [&a](int h) { return MPPI_IN_RANGE(h, a.H) ? h : 0; };  // this thread's slots
    const long long base_in = (long long)mem * a.i_a + (long long)cls * a.i_b;
    // start point x = prefix sums of vt, and (B^T vt)_i = vt_{i-1} - vt_i (vt_H for i = H)
    uint2 key{};
    uint32_t iter = 0;
    if (!a.vin) {
        key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
        iter = (uint32_t)(a.iter_ptr ? *a.iter_ptr : a.iter_val);
    }
    float prev = 0.0f, acc = 0.0f;
    for (int h = 0; h < a.H; ++h) {
        float vt;
        if (a.vin) {
            vt = ld_checked(a.vin, base_in + (long long)h * a.i_h, a.in_n);
        } else {  // sample k = member, joint j = class
            vt = qp_sample(a, key, iter, mem, cls, h);
        }
        acc += vt;
        if (h > 0) xb[(size_t)sl(h - 1) * T].y = prev - vt;
        xb[(size_t)sl(h) * T].x = acc;
        yv[(size_t)sl(h) * T] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        prev = vt;
    }
    xb[(size_t)sl(a.H - 1) * T].y = prev;
    qp_admm(c, a.band + (size_t)(MPPI_IN_RANGE(cls, a.n_cls) ? cls : 0) * 2 * a.H, a.H, a.iters, a.dt, q, qd, xb, yv, T);
    const long long base_out = (long long)mem * a.o_a + (long long)cls * a.o_b;
    float xp = 0.0f;
    for (int h = 0; h < a.H; ++h) {
        const float x = xb[(size_t)sl(h) * T].x;
        const long long o = base_out + (long long)h * a.o_h;
        if (MPPI_IN_RANGE(o, a.out_n)) a.out[o] = x - xp;
        xp = x;
    }
}

// 24 H bytes of shared memory per thread: 64 threads per CTA while that
// stays within 100 KB (two CTAs per SM), else one warp.
int qp_threads(int H) { return (size_t)H * 64 * (sizeof(float4) + sizeof(float2)) <= 100 * 1024 ? 64 : 32; }
size_t qp_smem_bytes(int H) { return (size_t)H * qp_threads(H) * (sizeof(float4) + sizeof(float2)); }

int launch_qp(const QPArgs& a, cudaStream_t s) {
    if (a.n <= 0) return MPPI_OK;
    if (a.minv && a.H <= QP_WARP_MAX_H) {
        if (a.vin) {  // standalone, one class
            qp_warp_kernel<<<(a.n + 7) / 8, 256, 0, s>>>(a);
        } else {      // controller: CTA = sample, warp = joint
            if (a.nu > 14 || a.n != a.per_cls * a.nu) return MPPI_ERR_UNSUPPORTED;
            const size_t sm = (size_t)(32 * a.nu + a.H * a.nu) * sizeof(float);
            qp_warp_sample_kernel<<<a.per_cls, 32 * a.nu, sm, s>>>(a);
        }
        return cudaGetLastError() == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
    }
    const size_t sm = qp_smem_bytes(a.H);
    if (sm > 227 * 1024) return MPPI_ERR_UNSUPPORTED;
    const int T = qp_threads(a.H);
    static size_t max_set = 0;
    if (sm > 48 * 1024 && sm > max_set) {
        cudaError_t e = cudaFuncSetAttribute(qp_project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return MPPI_ERR_CUDA;
        max_set = sm;
    }
    const int grid = (a.n + T - 1) / T;
    qp_project_kernel<<<grid, T, sm, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

MPPI_BOUNDS_READER(bounds_word_qp)

}  // namespace mppi

using namespace mppi;

extern "C" int mppi_qp_project(int n, int H, float dt, const float* bounds, int iters, float rho, const float* scales,
                               const float* q0, const float* qd0, const float* v_in, float* v_out, void* stream) {
    static const float kDefault[4] = {MPPI_QP_SCALE_POSITION, MPPI_QP_SCALE_VELOCITY, MPPI_QP_SCALE_ACCELERATION,
                                      MPPI_QP_SCALE_JERK};
    const float* sc = scales ? scales : kDefault;
    if (n < 0 || H < 1 || H > MPPI_QP_MAX_H || iters < 0 || !(dt > 0.0f) || !bounds) return MPPI_ERR_INVALID_ARG;
    if (n > 0 && (!q0 || !qd0 || !v_in || !v_out)) return MPPI_ERR_INVALID_ARG;
    int rc = qp_validate(bounds, sc, rho);
    if (rc != MPPI_OK) return rc;
    if (n == 0) return MPPI_OK;
    QPClass c;
    qp_make_class(bounds, sc, rho, &c);
    const bool warp = H <= QP_WARP_MAX_H;
    // band factor rows (thread kernel) or the dense inverse (warp kernel), as float4s
    std::vector<float4> band(warp ? 32 * 32 / 4 : 2 * (size_t)H);
    const double scd[4] = {c.s[0], c.s[1], c.s[2], c.s[3]};
    rc = warp ? qp_dense_inverse(H, rho, scd, reinterpret_cast<float*>(band.data()))
              : qp_band_factor(H, rho, scd, band.data());
    if (rc != MPPI_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the class record and the factor live in one stream-ordered scratch block
    const size_t bytes = sizeof(QPClass) + band.size() * sizeof(float4);
    void* d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, bytes, s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA;
    std::vector<unsigned char> host(bytes);
    std::memcpy(host.data(), &c, sizeof c);
    std::memcpy(host.data() + sizeof c, band.data(), band.size() * sizeof(float4));
    e = cudaMemcpyAsync(d, host.data(), bytes, cudaMemcpyHostToDevice, s);  // pageable: staged before return
    QPArgs a{};
    a.n = n;
    a.H = H;
    a.iters = iters;
    a.dt = dt;
    a.per_cls = n;
    a.cls = static_cast<const QPClass*>(d);
    a.band = reinterpret_cast<const float4*>(static_cast<unsigned char*>(d) + sizeof(QPClass));
    if (warp) a.minv = reinterpret_cast<const float*>(a.band);
    a.q0 = q0;
    a.qd0 = qd0;
    a.q_per_seq = 1;
    a.vin = v_in;
    a.i_a = H;
    a.i_b = 0;
    a.i_h = 1;
    a.out = v_out;
    a.o_a = H;
    a.o_b = 0;
    a.o_h = 1;
    a.n_cls = 1;
    a.in_n = a.out_n = (long long)n * H;
    if (e == cudaSuccess) rc = launch_qp(a, s);
    else rc = MPPI_ERR_CUDA;
    cudaFreeAsync(d, s);
    return rc;
}
