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

// pairs: links x boxes (link-major) in the first lane passes, then links x
// ball (pick) and left x right links, so that every pass evaluates one kind
template <int NA>
struct TaskDims {
    static constexpr int CB = (2 * NA * MAXB + 31) / 32;  // capsule-box passes at most
    static constexpr int CC = (2 * NA + NA * NA + 31) / 32;
};

template <int NA>
struct TaskAcc {
    float prevb[TaskDims<NA>::CB];  // each pass's pair distance at the previous state (this lane)
    float prevc[TaskDims<NA>::CC];
    float c;                        // barrier + penetration count (this lane)
    float r;                        // orientation error (the end-effector lanes)
    float th, yz, v2, l, eo, ot;    // per-state terms (lane 0)
};

// Minimum over t in [0,1] of the box SDF f(t) at a0 + t dd, for any segment
// (the piece walk).  f is convex; its kinks along the segment are where a
// coordinate crosses a slab plane or the box's mid-plane, plus, inside the
// box, where two face distances cross.  f is evaluated at the nine crossing
// parameters and both ends; by convexity the minimiser lies in one of the
// two pieces next to the best of them.  On a piece outside the box f is the
// root of a quadratic (exceeded slabs and signs fixed), minimised at its
// stationary point; inside, f is the largest of three linear face
// distances, minimised at a pairwise crossing or an end.
__device__ __forceinline__ float segment_box_sdf_min(const float* a0, const float (&dd)[3], const float* box) {
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
    return best;
}

// Exact distance between a capsule (segment a0-a1, radius rcap) and a box
// (centre, half extents): the minimum of the box SDF along the segment,
// minus the radius.  A segment that misses the box (the slab intervals of
// the three axes have no common t in [0,1]) stays outside it, where the
// squared distance g(t) = sum_k e_k(t)^2, e_k the excess of coordinate k
// past its slab (zero within it), is a convex piecewise quadratic: g'/2 =
// sum_k e_k d_k is continuous, nondecreasing, and linear between the slab
// crossings.  g' at the six crossings and both ends brackets its zero
// between two candidates with no crossing in between, where one linear
// interpolation gives the minimiser.  A segment that meets the box takes the
// piece walk above.
__device__ __forceinline__ float capsule_box_distance(const float* a0, const float* a1, float rcap, const float* box) {
    float y0[3], dd[3], h[3], tc[6];
    float tin = 0.0f, tout = 1.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        y0[k] = a0[k] - box[k];
        dd[k] = a1[k] - a0[k];
        h[k] = box[3 + k];
        const bool mv = dd[k] != 0.0f;
        const float inv = 1.0f / (mv ? dd[k] : 1.0f);
        const float ta = (-h[k] - y0[k]) * inv, tb = (h[k] - y0[k]) * inv;
        tin = mv ? fmaxf(tin, fminf(ta, tb)) : (fabsf(y0[k]) > h[k] ? 2.0f : tin);
        tout = mv ? fminf(tout, fmaxf(ta, tb)) : tout;
        tc[2 * k] = mv ? fminf(fmaxf(ta, 0.0f), 1.0f) : 0.0f;
        tc[2 * k + 1] = mv ? fminf(fmaxf(tb, 0.0f), 1.0f) : 0.0f;
    }
    if (tin <= tout) return segment_box_sdf_min(a0, dd, box) - rcap;
    auto gp = [&](float t) {
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float y = __fmaf_rn(t, dd[k], y0[k]);
            s = __fmaf_rn(y - fminf(fmaxf(y, -h[k]), h[k]), dd[k], s);
        }
        return s;
    };
    // tl: the last candidate with g' <= 0, tr: the first with g' > 0
    float tl = 0.0f, gl = gp(0.0f), tr = 1.0f, gr = gp(1.0f);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const float v = gp(tc[c]);
        const bool lo = v <= 0.0f && tc[c] > tl, hi = v > 0.0f && tc[c] < tr;
        tl = lo ? tc[c] : tl;
        gl = lo ? v : gl;
        tr = hi ? tc[c] : tr;
        gr = hi ? v : gr;
    }
    const float t = gl >= 0.0f ? tl : (gr <= 0.0f ? tr : tl - gl * (tr - tl) / (gr - gl));
    float g = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float y = __fmaf_rn(t, dd[k], y0[k]);
        const float e = y - fminf(fmaxf(y, -h[k]), h[k]);
        g = __fmaf_rn(e, e, g);
    }
    return sqrtf(g) - rcap;
}

// Segment-segment distance minus both radii: the squared distance is a
// convex quadratic on [0,1]^2; take the interior stationary point if it lies
// inside, and every edge's clamped minimum.  A segment of zero length (a
// sphere) leaves only the projection onto the other segment and its ends.
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
    // the interior candidate (masked unless it lies in the square) and the
    // four edges' clamped minimisers, each edge's projection formed from the
    // dot products above
    const float den = A * Cq - Bq * Bq;
    const bool inner = den > 1e-7f * A * Cq;
    const float idn = inner ? 1.0f / den : 0.0f;
    const float si = (Bq * E - Cq * D) * idn, ti = (A * E - Bq * D) * idn;
    const bool in_sq = inner && si >= 0.0f && si <= 1.0f && ti >= 0.0f && ti <= 1.0f;
    float best = in_sq ? d2(si, ti) : INFINITY;
    const float ia = A > 0.0f ? 1.0f / A : 0.0f, ic = Cq > 0.0f ? 1.0f / Cq : 0.0f;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float fe = (float)e;
        const float t = fminf(fmaxf((E + fe * Bq) * ic, 0.0f), 1.0f);
        best = fminf(best, d2(fe, t));
        const float s = fminf(fmaxf((fe * Bq - D) * ia, 0.0f), 1.0f);
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
    const int ncb = (nlb + 31) >> 5;  // capsule-box passes
    const int nball = T.phase == 0 ? 2 * NA : 0;
    const int ncc = nball + NA * NA;
    const float keep = 1.0f - T.gamma;
    // capsule-box passes: one copy of the code, the pass's previous
    // distance picked out of the register array by selects
#pragma unroll 1
    for (int s = 0; s < ncb; ++s) {
        const int b = lane + 32 * s;
        if (b < nlb) {
            const int l = b / M.nb, bx = b - l * M.nb;
            const float dist = capsule_box_distance(w.a0[l], w.a1[l], M.link[l / NA][l % NA].rcap, M.box[bx]);
            float pv = acc.prevb[0];
#pragma unroll
            for (int k = 1; k < TaskDims<NA>::CB; ++k) pv = s == k ? acc.prevb[k] : pv;
            if (!first) acc.c += fmaxf(-dist + keep * pv, 0.0f) + (dist < 0.0f ? 1.0f : 0.0f);
#pragma unroll
            for (int k = 0; k < TaskDims<NA>::CB; ++k) acc.prevb[k] = s == k ? dist : acc.prevb[k];
        }
    }
    // ball-link and link-link passes (the ball is a capsule of zero length)
#pragma unroll
    for (int s = 0; s < TaskDims<NA>::CC; ++s) {
        const int b = lane + 32 * s;
        if (b < ncc) {
            const bool ball = b < nball;
            const int r = b - nball, i = r / NA, j = r - i * NA;
            const int la = ball ? b : i, lb = ball ? 0 : NA + j;
            const float* c0 = ball ? &w.q[d::B] : w.a0[lb];
            const float* c1 = ball ? &w.q[d::B] : w.a1[lb];
            const float rb = ball ? M.rb : M.link[1][j].rcap;
            const float dist = capsule_capsule_distance(w.a0[la], w.a1[la], M.link[la / NA][la % NA].rcap, c0, c1, rb);
            if (!first) acc.c += fmaxf(-dist + keep * acc.prevc[s], 0.0f) + (dist < 0.0f ? 1.0f : 0.0f);
            acc.prevc[s] = dist;
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
        // orientation error against this arm's target, on this lane
        float qe[4];
        rot_to_quat(Rl, qe);
        acc.r += 0.5f * quat_angle(qe, a == 0 ? T.q1s : T.q2s);
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
        acc.l += lerr * lerr;
        const float o0 = c0 - T.pb0[0], o1 = c1 - T.pb0[1], o2 = c2 - (T.pb0[2] - T.eps);
        acc.eo += sqrtf(o0 * o0 + o1 * o1 + o2 * o2);
        const float t0 = c0 - T.ptg[0], t1 = c1 - T.ptg[1], t2 = c2 + T.eps - T.ptg[2];
        acc.ot += sqrtf(t0 * t0 + t1 * t1 + t2 * t2);
    }
    __syncwarp();
}

// Weighted total after the last state (the barrier and orientation sums
// reduced over the warp; the other terms from lane 0).
template <int NA>
__device__ __forceinline__ float task_total(const DevTask& T, TaskAcc<NA>& acc) {
    float c = acc.c, r = acc.r;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        c += __shfl_xor_sync(FULL, c, off);
        r += __shfl_xor_sync(FULL, r, off);
    }
    const float pick = T.phase == 0 ? 1.0f : 0.0f, move = 1.0f - pick;
    return pick * (T.w_c * c + T.w_eo * acc.eo) + move * (T.w_c * c + T.w_ot * acc.ot) + T.w_theta * acc.th +
           T.w_yz * acc.yz + T.w_v * sqrtf(acc.v2) + T.w_r * r + T.w_l * acc.l;
}

}  // namespace mppi
