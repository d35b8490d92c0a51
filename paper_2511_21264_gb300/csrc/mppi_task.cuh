// The paper's ball-task cost suite (Sec. IV-B) evaluated inside the rollout:
// per state, the signed distances of the collision pairs (one lane per
// pair), the end effectors' positions, orientations and velocities, and the
// per-state terms; the barrier keeps each pair's previous distance in the
// lane's registers.
#pragma once
#include "mppi_device.cuh"

namespace mppi {

// Parameters (host layout: MPPI_TASK_N + nu floats, see mppi.h).
struct __align__(16) DevTask {
    int phase, pad0, pad1, pad2;
    float w_c, gamma, w_theta, w_yz;
    float w_v, w_r, w_l, l_ball;
    float w_eo, w_ot, eps, pad3;
    float pb0[4], ptg[4];  // ball before the pick, target
    float q1s[4], q2s[4];  // target EE orientations (w, x, y, z)
    float home[16];        // theta_home
};

// pairs: links x boxes (link-major), links x ball (pick), left x right links
template <int NA>
struct TaskDims {
    static constexpr int MAXPAIRS = 2 * NA * MAXB + 2 * NA + NA * NA;
    static constexpr int SLOTS = (MAXPAIRS + 31) / 32;
};

template <int NA>
struct TaskAcc {
    float prev[TaskDims<NA>::SLOTS];  // each slot's pair distance at the previous state (this lane)
    float c;                          // barrier + penetration count (this lane)
    float th, yz, v2, r, l, eo, ot;   // per-state terms (lane 0)
};

// Exact distance between a capsule (segment a0-a1, radius rcap) and a box:
// the minimum over t in [0,1] of the box SDF f(t) at a0 + t (a1 - a0), minus
// the radius.  f is convex; its kinks along the segment are where a
// coordinate crosses a slab plane or the box's mid-plane, plus, inside the
// box, where two face distances cross.  f is evaluated at the nine crossing
// parameters and both ends; by convexity the minimiser lies in one of the
// two pieces next to the best of them.  On a piece outside the box f is the
// root of a quadratic (exceeded slabs and signs fixed), minimised at its
// stationary point; inside, f is the largest of three linear face
// distances, minimised at a pairwise crossing or an end.
__device__ __forceinline__ float capsule_box_distance(const float* a0, const float* a1, float rcap, const float* box) {
    const float dd[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
    float T[11];
    T[0] = 0.0f;
    T[1] = 1.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool mv = dd[k] != 0.0f;
        const float inv = mv ? 1.0f / dd[k] : 0.0f;
        const float t0 = (box[k] - box[3 + k] - a0[k]) * inv, t1 = (box[k] + box[3 + k] - a0[k]) * inv;
        const float tc = (box[k] - a0[k]) * inv;
        T[2 + 3 * k] = mv ? fminf(fmaxf(t0, 0.0f), 1.0f) : 0.0f;
        T[3 + 3 * k] = mv ? fminf(fmaxf(t1, 0.0f), 1.0f) : 0.0f;
        T[4 + 3 * k] = mv ? fminf(fmaxf(tc, 0.0f), 1.0f) : 0.0f;
    }
    float best = INFINITY, tb = 0.0f;
#pragma unroll
    for (int i = 0; i < 11; ++i) {
        const float f = box_sdf_only(a0, dd, T[i], box);
        if (f < best) {
            best = f;
            tb = T[i];
        }
    }
    float tl = 0.0f, tr = 1.0f;
#pragma unroll
    for (int i = 0; i < 11; ++i) {
        if (T[i] < tb) tl = fmaxf(tl, T[i]);
        if (T[i] > tb) tr = fminf(tr, T[i]);
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const float lo = side == 0 ? tl : tb, hi = side == 0 ? tb : tr;
        if (!(hi > lo)) continue;
        const float tm = 0.5f * (lo + hi);
        float al[3], be[3], num = 0.0f, den = 0.0f;
        bool outside = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float xk = a0[k] + tm * dd[k] - box[k];
            const float sg = xk >= 0.0f ? 1.0f : -1.0f;
            al[k] = sg * (a0[k] - box[k]) - box[3 + k];
            be[k] = sg * dd[k];
            if (sg * xk - box[3 + k] > 0.0f) {  // slab k exceeded on this piece
                outside = true;
                num += al[k] * be[k];
                den += be[k] * be[k];
            }
        }
        if (outside) {
            if (den > 0.0f) {
                const float t = fminf(fmaxf(-num / den, lo), hi);
                best = fminf(best, box_sdf_only(a0, dd, t, box));
            }
        } else {
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const int j = p, k = (p + 1) % 3;
                const float dn = be[k] - be[j];
                if (dn != 0.0f) {
                    const float t = fminf(fmaxf((al[j] - al[k]) / dn, lo), hi);
                    best = fminf(best, box_sdf_only(a0, dd, t, box));
                }
            }
        }
    }
    return best - rcap;
}

__device__ __forceinline__ float seg_clamp_t(const float* p0, const float* d, float dd, float x0, float x1, float x2) {
    if (!(dd > 0.0f)) return 0.0f;
    const float t = ((x0 - p0[0]) * d[0] + (x1 - p0[1]) * d[1] + (x2 - p0[2]) * d[2]) / dd;
    return fminf(fmaxf(t, 0.0f), 1.0f);
}

__device__ __forceinline__ float sphere_capsule_distance(const float* c, float r, const float* a0, const float* a1,
                                                         float rcap) {
    const float d[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
    const float t = seg_clamp_t(a0, d, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], c[0], c[1], c[2]);
    const float e0 = c[0] - a0[0] - t * d[0], e1 = c[1] - a0[1] - t * d[1], e2 = c[2] - a0[2] - t * d[2];
    return sqrtf(e0 * e0 + e1 * e1 + e2 * e2) - r - rcap;
}

// Segment-segment distance minus both radii: the squared distance is a
// convex quadratic on [0,1]^2; take the interior stationary point if it lies
// inside, and every edge's clamped minimum.
__device__ __forceinline__ float capsule_capsule_distance(const float* a0, const float* a1, float ra, const float* b0,
                                                          const float* b1, float rb) {
    float u[3], v[3], w0[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u[k] = a1[k] - a0[k];
        v[k] = b1[k] - b0[k];
        w0[k] = a0[k] - b0[k];
    }
    const float A = u[0] * u[0] + u[1] * u[1] + u[2] * u[2], Bq = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
    const float Cq = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const float D = u[0] * w0[0] + u[1] * w0[1] + u[2] * w0[2], E = v[0] * w0[0] + v[1] * w0[1] + v[2] * w0[2];
    auto d2 = [&](float s, float t) {
        float r = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float e = w0[k] + s * u[k] - t * v[k];
            r += e * e;
        }
        return r;
    };
    float best = INFINITY;
    const float den = A * Cq - Bq * Bq;
    if (den > 1e-7f * A * Cq) {
        const float s = (Bq * E - Cq * D) / den, t = (A * E - Bq * D) / den;
        if (s >= 0.0f && s <= 1.0f && t >= 0.0f && t <= 1.0f) best = d2(s, t);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float fe = (float)e;
        const float t = seg_clamp_t(b0, v, Cq, a0[0] + fe * u[0], a0[1] + fe * u[1], a0[2] + fe * u[2]);
        best = fminf(best, d2(fe, t));
        const float s = seg_clamp_t(a0, u, A, b0[0] + fe * v[0], b0[1] + fe * v[1], b0[2] + fe * v[2]);
        best = fminf(best, d2(s, fe));
    }
    return sqrtf(best) - ra - rb;
}

// Unit quaternion (w, x, y, z), w >= 0, of a row-major rotation: the
// largest of 1 + tr, 1 + R00 - R11 - R22, ... fixes one component, the
// off-diagonal sums and differences the others.
__device__ __forceinline__ void rot_to_quat(const float* R, float* q) {
    const float c0 = 1.0f + R[0] + R[4] + R[8], c1 = 1.0f + R[0] - R[4] - R[8];
    const float c2 = 1.0f - R[0] + R[4] - R[8], c3 = 1.0f - R[0] - R[4] + R[8];
    int i = 0;
    float cm = c0;
    if (c1 > cm) { i = 1; cm = c1; }
    if (c2 > cm) { i = 2; cm = c2; }
    if (c3 > cm) { i = 3; cm = c3; }
    const float h = 0.5f * sqrtf(cm), s = 0.25f / h;
    if (i == 0) { q[0] = h; q[1] = (R[7] - R[5]) * s; q[2] = (R[2] - R[6]) * s; q[3] = (R[3] - R[1]) * s; }
    else if (i == 1) { q[1] = h; q[0] = (R[7] - R[5]) * s; q[2] = (R[1] + R[3]) * s; q[3] = (R[2] + R[6]) * s; }
    else if (i == 2) { q[2] = h; q[0] = (R[2] - R[6]) * s; q[1] = (R[1] + R[3]) * s; q[3] = (R[5] + R[7]) * s; }
    else { q[3] = h; q[0] = (R[3] - R[1]) * s; q[1] = (R[2] + R[6]) * s; q[2] = (R[5] + R[7]) * s; }
    if (q[0] < 0.0f) {
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = -q[k];
    }
}

__device__ __forceinline__ float quat_angle(const float* q, const float* qs) {
    const float c = fabsf(q[0] * qs[0] + q[1] * qs[1] + q[2] * qs[2] + q[3] * qs[3]);
    return 2.0f * acosf(fminf(c, 1.0f));
}

// Task terms of the state whose kinematics forward_kinematics just wrote
// (w.a0/a1/z/o, Rl on the lane of each link).  first: the present state
// x_0, which only seeds the barrier's previous distances.
template <int NA>
__device__ __forceinline__ void task_state(const DevModel& M, const DevTask& T, WarpWS<NA>& w, int lane,
                                           const float (&Rl)[9], bool first, TaskAcc<NA>& acc) {
    using d = Dims<NA>;
    const int nlb = 2 * NA * M.nb;
    const int nball = T.phase == 0 ? 2 * NA : 0;
    const int np = nlb + nball + NA * NA;
#pragma unroll
    for (int s = 0; s < TaskDims<NA>::SLOTS; ++s) {
        const int b = lane + 32 * s;
        if (b < np) {
            float dist;
            if (b < nlb) {
                const int l = b / M.nb, bx = b - l * M.nb;
                dist = capsule_box_distance(w.a0[l], w.a1[l], M.link[l / NA][l % NA].rcap, M.box[bx]);
            } else if (b < nlb + nball) {
                const int l = b - nlb;
                dist = sphere_capsule_distance(&w.q[d::B], M.rb, w.a0[l], w.a1[l], M.link[l / NA][l % NA].rcap);
            } else {
                const int r = b - nlb - nball, i = r / NA, j = r - i * NA;
                dist = capsule_capsule_distance(w.a0[i], w.a1[i], M.link[0][i].rcap, w.a0[NA + j], w.a1[NA + j],
                                                M.link[1][j].rcap);
            }
            if (!first) acc.c += fmaxf(-dist + (1.0f - T.gamma) * acc.prev[s], 0.0f) + (dist < 0.0f ? 1.0f : 0.0f);
            acc.prev[s] = dist;
        }
    }
    if (first) return;
    // end effectors: velocity = sum over the arm's joints of (z_j x (p - o_j)) qd_j
    const int a = lane >> 4, i = lane & 15;
    const float* pe = w.a1[a * NA + NA - 1];
    float vx = 0.0f, vy = 0.0f, vz = 0.0f;
    if (i < NA) {
        const float* z = w.z[a * NA + i];
        const float* o = w.o[a * NA + i];
        const float r0 = pe[0] - o[0], r1 = pe[1] - o[1], r2 = pe[2] - o[2], qdj = w.qd[a * NA + i];
        vx = (z[1] * r2 - z[2] * r1) * qdj;
        vy = (z[2] * r0 - z[0] * r2) * qdj;
        vz = (z[0] * r1 - z[1] * r0) * qdj;
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
        vx += __shfl_xor_sync(FULL, vx, off);
        vy += __shfl_xor_sync(FULL, vy, off);
        vz += __shfl_xor_sync(FULL, vz, off);
    }
    if (i == NA - 1) {
        float* e = w.ee[a];
        e[0] = pe[0];
        e[1] = pe[1];
        e[2] = pe[2];
        e[3] = vx;
        e[4] = vy;
        e[5] = vz;
        rot_to_quat(Rl, e + 6);
    }
    float th = 0.0f;
    if (lane < d::NU) {
        const float e = w.q[lane] - T.home[lane];
        th = e * e;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) th += __shfl_xor_sync(FULL, th, off);
    __syncwarp();
    if (lane == 0) {
        const float* e1 = w.ee[0];
        const float* e2 = w.ee[1];
        const float dp0 = e1[0] - e2[0], dp1 = e1[1] - e2[1], dp2 = e1[2] - e2[2];
        const float rv = dp0 * (e1[3] - e2[3]) + dp1 * (e1[4] - e2[4]) + dp2 * (e1[5] - e2[5]);
        const float c0 = 0.5f * (e1[0] + e2[0]), c1 = 0.5f * (e1[1] + e2[1]), c2 = 0.5f * (e1[2] + e2[2]);
        const float lerr = sqrtf(dp0 * dp0 + dp1 * dp1 + dp2 * dp2) - T.l_ball;
        acc.th += sqrtf(th);
        acc.yz += sqrtf(dp1 * dp1 + dp2 * dp2);
        acc.v2 += rv * rv;
        acc.r += 0.5f * (quat_angle(e1 + 6, T.q1s) + quat_angle(e2 + 6, T.q2s));
        acc.l += lerr * lerr;
        const float o0 = c0 - T.pb0[0], o1 = c1 - T.pb0[1], o2 = c2 - (T.pb0[2] - T.eps);
        acc.eo += sqrtf(o0 * o0 + o1 * o1 + o2 * o2);
        const float t0 = c0 - T.ptg[0], t1 = c1 - T.ptg[1], t2 = c2 + T.eps - T.ptg[2];
        acc.ot += sqrtf(t0 * t0 + t1 * t1 + t2 * t2);
    }
    __syncwarp();
}

// Weighted total on lane 0 after the last state (the barrier sums reduced
// over the warp).
template <int NA>
__device__ __forceinline__ float task_total(const DevTask& T, TaskAcc<NA>& acc) {
    float c = acc.c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
    const float pick = T.phase == 0 ? 1.0f : 0.0f, move = 1.0f - pick;
    return pick * (T.w_c * c + T.w_eo * acc.eo) + move * (T.w_c * c + T.w_ot * acc.ot) + T.w_theta * acc.th +
           T.w_yz * acc.yz + T.w_v * sqrtf(acc.v2) + T.w_r * acc.r + T.w_l * acc.l;
}

}  // namespace mppi
