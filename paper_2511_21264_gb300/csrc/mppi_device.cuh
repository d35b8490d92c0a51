// Device side of the MPPI + contact-rollout path (sm_103a, FP32, CUDA cores).
//
// A group of LPS lanes of one warp simulates one sample: LPS = 32 (one
// sample per warp), 16 (two) or 8 (four; the planar 3-link arms).  The
// sample's articulated state, link frames, contact set and solver scratch
// live in the group's slice of shared memory for all H steps; the scene
// model is staged once per CTA.  Every synchronisation (shuffle, ballot,
// __syncwarp) names the group's lanes only, so the samples of one warp may
// take different branches.  Lane roles inside a step (SEG = LPS / 2 lanes
// per arm segment):
//   - controls: lane j < nu draws its Gaussian from Philox4x32-10 (or reads
//     the explicit control);
//   - kinematics: one lane per link, prefix product of the link transforms;
//   - collision: one lane per ball pair and per capsule-box cull, each
//     surviving capsule-box pair minimised by the whole group over a closed
//     candidate set, contacts compacted with ballots in canonical order;
//   - dynamics: lane SEG*a + i owns link i of arm a (spatial inertia,
//     composite inertia, mass-matrix column, Newton-Euler bias force), lane
//     SEG*a factors the arm's (M + dt D) block, lane SEG-1 handles the ball;
//   - contact rows: one lane per Jacobian row (half-solved by the Cholesky
//     factor), the Delassus block across lanes, projected Gauss-Seidel in
//     contact space;
//   - integration: one lane per coordinate (strided when nv > LPS).
// Every reduction follows the order of a 32-slot tree whatever LPS is (a
// lane of a narrower group folds its slots in that order), so the result of
// a sample does not depend on the layout it ran in.
// The formulation (world-frame spatial algebra, composite-rigid-body mass
// matrix, recursive bias, half-solved contact rows) is independent of the
// FP64 oracle, which builds the same quantities from Jacobian definitions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mppi_check.cuh"
#include "mppi_internal.h"

namespace mppi {

constexpr int MAXL = 7;    // joints per arm
constexpr int MAXB = 16;   // boxes
constexpr int MAXC = 8;    // contacts kept per step (models with a larger cap are rejected)
constexpr int MAXR = 3 * MAXC;
constexpr unsigned FULL = 0xffffffffu;


// Arrays are CArr (mppi_check.cuh): plain arrays, range-checked in the
// bounds-check build.
struct __align__(16) DevLink {
    CArr<float, 9> FR;
    CArr<float, 3> Fp;
    CArr<float, 3> com;
    float mass;
    CArr<float, 6> I;  // inertia about the COM in link axes: xx yy zz xy xz yz
    CArr<float, 3> s0;
    CArr<float, 3> s1;
    float rcap, D, gear, tau_max;  // D = joint damping + servo gain (implicit)
    float u_lo, u_hi, gravcomp, pad;
};

struct __align__(16) DevModel {
    int na, nb, maxc, sweeps;
    float dt, mu, imp, erp;
    CArr<float, 3> g;
    float floor_z;
    float rb, mb, Ib, pad0;
    CArr<float, 3> goal;
    float w_goal;
    float w_u, w_pen, w_obst, w_grasp;
    CArr<CArr<float, 9>, 2> baseR;
    CArr<CArr<float, 3>, 2> basep;
    CArr<CArr<float, 6>, MAXB> box;  // centre, half-extents
    CArr<CArr<DevLink, MAXL>, 2> link;
};
static_assert(sizeof(DevModel) % 16 == 0, "model must stage with 16-byte copies");

template <int NA>
struct Dims {
    static constexpr int NL = 2 * NA, NV = 2 * NA + 6, NQ = 2 * NA + 7, NU = 2 * NA;
    static constexpr int NX = NQ + NV, B = 2 * NA;
};

// The lanes of one warp that simulate one sample.  Arm a's links sit on
// group lanes SEG*a .. SEG*a + NA - 1; group lane SEG - 1 (past the first
// arm's links) is the ball's lane.
template <int LPS>
struct Lanes {
    static_assert(LPS == 8 || LPS == 16 || LPS == 32, "lanes per sample: 8, 16 or 32");
    static constexpr int SEG = LPS / 2;  // lanes per arm segment
    static constexpr int SPW = 32 / LPS;  // samples per warp
    int sl;       // lane within the group
    int base;     // the group's first lane in the warp
    unsigned gm;  // the group's lanes
    int a, i;     // arm segment, lane within it
    __device__ __forceinline__ explicit Lanes(int lane) {
        sl = lane & (LPS - 1);
        base = lane & ~(LPS - 1);
        gm = LPS == 32 ? FULL : (((1u << (LPS & 31)) - 1u) << base);
        a = sl / SEG;
        i = sl & (SEG - 1);
    }
    __device__ __forceinline__ void sync() const { __syncwarp(gm); }
    // the group's ballot, bit t = group lane t
    __device__ __forceinline__ unsigned ballot(bool p) const {
        const unsigned b = __ballot_sync(gm, p) & gm;
        return LPS == 32 ? b : b >> base;
    }
    __device__ __forceinline__ bool any(bool p) const { return ballot(p) != 0u; }
    __device__ __forceinline__ float shfl(float v, int src) const { return __shfl_sync(gm, v, src, LPS); }
    __device__ __forceinline__ int shfl(int v, int src) const { return __shfl_sync(gm, v, src, LPS); }
    __device__ __forceinline__ float xor_(float v, int off) const { return __shfl_xor_sync(gm, v, off, LPS); }
    __device__ __forceinline__ int xor_(int v, int off) const { return __shfl_xor_sync(gm, v, off, LPS); }
    // within the lane's arm segment
    __device__ __forceinline__ float up_seg(float v, int off) const { return __shfl_up_sync(gm, v, off, SEG); }
    __device__ __forceinline__ float down_seg(float v, int off) const { return __shfl_down_sync(gm, v, off, SEG); }
};

// Sum over the 32 slots of a sample, slot t held by group lane t % LPS as
// element t / LPS of v: the order of a 32-lane xor butterfly with offsets
// 16, 8, 4, 2, 1 (in-lane folds for the offsets >= LPS), on every lane.
template <int LPS, int PS>
__device__ __forceinline__ float slot_sum(const Lanes<LPS>& g, float (&v)[PS]) {
    static_assert(PS * LPS == 32, "32 slots");
#pragma unroll
    for (int n = PS; n > 1; n >>= 1)
#pragma unroll
        for (int t = 0; t < n / 2; ++t) v[t] = v[t] + v[t + n / 2];
    float s = v[0];
#pragma unroll
    for (int off = LPS / 2; off > 0; off >>= 1) s += g.xor_(s, off);
    return s;
}
// The same for a value that only slots < LPS hold (the others are zero).
template <int LPS>
__device__ __forceinline__ float group_sum(const Lanes<LPS>& g, float v) {
#pragma unroll
    for (int off = LPS / 2; off > 0; off >>= 1) v += g.xor_(v, off);
    return v;
}

// Per-sample workspace in shared memory.  Scratch that lives in
// one phase only shares storage: the capsule-box survivor list (collision)
// and the contact rows, Delassus block and impulses (contacts).
template <int NA>
struct __align__(16) WarpWS {
    using d = Dims<NA>;
    CArr<float, d::NQ + 1> q;
    CArr<float, d::NV> qd;
    CArr<float, d::NV> v;
    CArr<float, d::NV> vf;
    CArr<float, d::NV> zz;
    CArr<float, d::NV> rhs;
    CArr<float, d::NU> u;
    CArr<CArr<float, 16>, 8> zn;  // standard normals of the next steps (Philox path)
    // kinematics, per link (read across lanes)
    CArr<CArr<float, 3>, d::NL> z;
    CArr<CArr<float, 3>, d::NL> o;
    CArr<CArr<float, 3>, d::NL> a0;
    CArr<CArr<float, 3>, d::NL> a1;
    // factors of (M + dt D), per arm
    CArr<CArr<CArr<float, NA>, NA>, 2> L;
    CArr<CArr<float, NA>, 2> Ldi;  // reciprocal diagonal of the factors
    // contacts of this step, canonical order
    CArr<CArr<float, 3>, MAXC> cp;
    CArr<CArr<float, 3>, MAXC> cn;
    CArr<float, MAXC> cdep;
    CArr<int, MAXC> cA;
    CArr<int, MAXC> cB;
    CArr<CArr<float, 6>, 2> ee;   // task cost: end-effector position and velocity per arm
    union Phase {
        struct {
            CArr<short, 2 * MAXL * MAXB> surv;  // capsule-box pairs that pass the cull
        } col;
        struct {
            CArr<CArr<float, d::NV>, MAXR> Y;
            CArr<float, MAXR * MAXR> G;  // Delassus block Y Y^T, nr x nr
            CArr<float4, MAXR> rc4;      // per row: b = J v_f, R, 1/(A+R), reference velocity
            CArr<float, MAXR> lam;
            CArr<int, MAXR> tmask;       // blocks a row touches: 1 left arm, 2 right arm, 4 ball
        } con;
    } ph;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and the Gaussian sampler
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Uniform in (0,1) from the top 23 bits: ((x >> 9) + 1/2) 2^-23, exact in FP32.
__device__ __forceinline__ float u01_23(uint32_t x) {
    return __fmul_rn(__fadd_rn((float)(x >> 9), 0.5f), 1.1920928955078125e-07f);
}

// Standard normal number t (0..3) of a Philox block: Box-Muller on the word
// pairs (0,1) and (2,3); even t takes the cosine, odd t the sine.
__device__ __forceinline__ float block_normal(uint4 w, int t) {
    const uint32_t a = (t < 2) ? w.x : w.z;
    const uint32_t b = (t < 2) ? w.y : w.w;
    const float r = sqrtf(__fmul_rn(-2.0f, logf(u01_23(a))));
    float s, c;
    sincospif(__fmul_rn(2.0f, u01_23(b)), &s, &c);
    return __fmul_rn(r, (t & 1) ? s : c);
}

// All four normals of a Philox block, each word pair's radius and angle
// computed once (the values block_normal gives for t = 0..3).
__device__ __forceinline__ void block_normals4(uint4 w, float (&z)[4]) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float r = sqrtf(__fmul_rn(-2.0f, logf(u01_23(p ? w.z : w.x))));
        float s, c;
        sincospif(__fmul_rn(2.0f, u01_23(p ? w.w : w.y)), &s, &c);
        z[2 * p] = __fmul_rn(r, c);
        z[2 * p + 1] = __fmul_rn(r, s);
    }
}

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cross3(const float* a, const float* b, float* o) {
    const float x = a[1] * b[2] - a[2] * b[1];
    const float y = a[2] * b[0] - a[0] * b[2];
    const float z = a[0] * b[1] - a[1] * b[0];
    o[0] = x;
    o[1] = y;
    o[2] = z;
}
__device__ __forceinline__ float dot3(const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// spatial inertia (m, h = m c, J = inertia about the world origin) times a
// motion vector (w, v): (J w + h x v, m v + w x h)
__device__ __forceinline__ void spatial_inertia_apply(const float* I, const float* x, float* out) {
    const float m = I[0];
    const float* h = I + 1;
    const float* J = I + 4;  // xx yy zz xy xz yz
    float hv[3], wh[3];
    cross3(h, x + 3, hv);
    cross3(x, h, wh);
    out[0] = J[0] * x[0] + J[3] * x[1] + J[4] * x[2] + hv[0];
    out[1] = J[3] * x[0] + J[1] * x[1] + J[5] * x[2] + hv[1];
    out[2] = J[4] * x[0] + J[5] * x[1] + J[2] * x[2] + hv[2];
    out[3] = m * x[3] + wh[0];
    out[4] = m * x[4] + wh[1];
    out[5] = m * x[5] + wh[2];
}

// ---------------------------------------------------------------------------
// kinematics: the lanes of arm segment a walk arm a
// ---------------------------------------------------------------------------
template <int NA, int LPS>
__device__ __forceinline__ void forward_kinematics(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g,
                                                   float (&Rl)[9], float (&cl)[3]) {
    // Lane i of segment a owns link i of arm a.  Each lane forms its local
    // transform Rz(q_i) F_i; an inclusive prefix product over the segment
    // (Hillis-Steele, log2(n_a) shuffle rounds) gives the chain to link i;
    // the base transform is applied last.  The joint axis and origin of link
    // i are the previous link's frame (the base for i = 0).
    static_assert(Lanes<LPS>::SEG > NA, "an arm segment holds the arm's links and one spare lane");
    const int a = g.a, i = g.i;
    const bool act = i < NA;
    float R[9], p[3];
    {
        // every lane forms a local transform, with no divergent branch: lanes
        // past the last link use the last link's data (the prefix products of
        // the links' lanes never read theirs)
        const int ic = act ? i : NA - 1;
        const DevLink& L = M.link[a][ic];
        float sn, cs;
        // the hardware sine and cosine: absolute error about 1e-6 for joint
        // angles of a few radians, growing slowly with the angle
        __sincosf(w.q[a * NA + ic], &sn, &cs);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            R[cc] = cs * L.FR[cc] - sn * L.FR[3 + cc];
            R[3 + cc] = sn * L.FR[cc] + cs * L.FR[3 + cc];
            R[6 + cc] = L.FR[6 + cc];
        }
        p[0] = cs * L.Fp[0] - sn * L.Fp[1];
        p[1] = sn * L.Fp[0] + cs * L.Fp[1];
        p[2] = L.Fp[2];
    }
#pragma unroll
    for (int off = 1; off < NA; off <<= 1) {
        float Rp[9], pp[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) Rp[k] = g.up_seg(R[k], off);
#pragma unroll
        for (int k = 0; k < 3; ++k) pp[k] = g.up_seg(p[k], off);
        // every lane forms the product; lanes with no predecessor this far
        // back keep their transform (a select, no divergent branch)
        const bool take = i >= off;
        float Rn[9], pn[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                Rn[3 * r + cc] = Rp[3 * r] * R[cc] + Rp[3 * r + 1] * R[3 + cc] + Rp[3 * r + 2] * R[6 + cc];
            pn[r] = Rp[3 * r] * p[0] + Rp[3 * r + 1] * p[1] + Rp[3 * r + 2] * p[2] + pp[r];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = take ? Rn[k] : R[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) p[k] = take ? pn[k] : p[k];
    }
    // world frame: base * chain
    const float* B = M.baseR[a];
    float Rw[9], pw[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) Rw[3 * r + cc] = B[3 * r] * R[cc] + B[3 * r + 1] * R[3 + cc] + B[3 * r + 2] * R[6 + cc];
        pw[r] = B[3 * r] * p[0] + B[3 * r + 1] * p[1] + B[3 * r + 2] * p[2] + M.basep[a][r];
    }
    float zp[3], op[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        zp[r] = g.up_seg(Rw[3 * r + 2], 1);
        op[r] = g.up_seg(pw[r], 1);
    }
    if (i == 0) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            zp[r] = B[3 * r + 2];
            op[r] = M.basep[a][r];
        }
    }
    {  // every lane computes (lanes past the last link on its data), the links' lanes store
        const int ic = act ? i : NA - 1;
        const DevLink& L = M.link[a][ic];
        const int l = a * NA + ic;
#pragma unroll
        for (int k = 0; k < 9; ++k) Rl[k] = Rw[k];
        float c0[3], c1[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            cl[r] = Rw[3 * r] * L.com[0] + Rw[3 * r + 1] * L.com[1] + Rw[3 * r + 2] * L.com[2] + pw[r];
            c0[r] = Rw[3 * r] * L.s0[0] + Rw[3 * r + 1] * L.s0[1] + Rw[3 * r + 2] * L.s0[2] + pw[r];
            c1[r] = Rw[3 * r] * L.s1[0] + Rw[3 * r + 1] * L.s1[1] + Rw[3 * r + 2] * L.s1[2] + pw[r];
        }
        if (act) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                w.z[l][r] = zp[r];
                w.o[l][r] = op[r];
                w.a0[l][r] = c0[r];
                w.a1[l][r] = c1[r];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// narrow phase
// ---------------------------------------------------------------------------
// signed distance from x to an axis-aligned box, outward normal, closest
// surface point.  Inside: nearest face; faces within FACE_TIE of the nearest
// count as tied (a segment's deepest point inside a box lies where two faces
// are equidistant), ties -> lowest axis, + face before - face.
constexpr float FACE_TIE = 1e-5f;
__device__ __forceinline__ float box_sdf(const float* x, const float* box, float* n, float* surf) {
    float q[3], cl[3];
    bool inside = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = box[k] - box[3 + k], hi = box[k] + box[3 + k];
        cl[k] = fminf(fmaxf(x[k], lo), hi);
        q[k] = x[k] - cl[k];
        inside = inside && (x[k] >= lo) && (x[k] <= hi);
    }
    if (!inside) {
        const float len = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        const float il = 1.0f / len;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            n[k] = q[k] * il;
            surf[k] = cl[k];
        }
        return len;
    }
    float fd[6], best = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        fd[2 * k] = (box[k] + box[3 + k]) - x[k];
        fd[2 * k + 1] = x[k] - (box[k] - box[3 + k]);
        best = fminf(best, fminf(fd[2 * k], fd[2 * k + 1]));
    }
    // faces within FACE_TIE of the nearest are tied: lowest axis, + first
    int f = 5;
#pragma unroll
    for (int t = 5; t >= 0; --t)
        if (fd[t] <= best + FACE_TIE) f = t;
    const int ax = f >> 1;
    const float sg = (f & 1) ? -1.0f : 1.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        n[k] = (k == ax) ? sg : 0.0f;
        surf[k] = (k == ax) ? box[k] + sg * box[3 + k] : x[k];
    }
    return -best;
}

__device__ __forceinline__ float box_sdf_only(const float* a, const float* d, float t, const float* box) {
    float x[3] = {a[0] + t * d[0], a[1] + t * d[1], a[2] + t * d[2]};
    float q2 = 0.0f, mx = -INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float e = fabsf(x[k] - box[k]) - box[3 + k];
        mx = fmaxf(mx, e);
        const float ep = fmaxf(e, 0.0f);
        q2 += ep * ep;
    }
    return sqrtf(q2) + fminf(mx, 0.0f);
}

// Separating-axis test of the segment mid +- hv against the box inflated
// by r on every side (half-extents h + r): the three box axes, then the
// three products hv x e_k, onto which the segment projects to one point.
// A capsule of radius r that touches the box lies in that inflated box, so
// it always passes; the margin eps absorbs FP32 rounding.
__device__ __forceinline__ bool segment_meets_inflated_box(const float* mid, const float* hv, const float* box,
                                                           float r) {
    constexpr float eps = 1e-5f;
    float dc[3], e[3], ah[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dc[k] = mid[k] - box[k];
        e[k] = box[3 + k] + r + eps;
        ah[k] = fabsf(hv[k]);
    }
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) ok = ok && fabsf(dc[k]) <= e[k] + ah[k];
    ok = ok && fabsf(dc[1] * hv[2] - dc[2] * hv[1]) <= e[1] * ah[2] + e[2] * ah[1] + eps;
    ok = ok && fabsf(dc[2] * hv[0] - dc[0] * hv[2]) <= e[0] * ah[2] + e[2] * ah[0] + eps;
    ok = ok && fabsf(dc[0] * hv[1] - dc[1] * hv[0]) <= e[0] * ah[1] + e[1] * ah[0] + eps;
    return ok;
}

// Candidate minimisers of the box SDF along the segment a + t d, t in [0,1].
// The SDF is convex along the segment and piecewise smooth; its minimum lies
// at an end point, at a slab-plane or axis-centre crossing (kinks), at the
// stationary point of the squared distance to an edge or vertex region (for
// every set of >= 2 exceeded slabs and sign pattern), or inside the box where
// two face distances cross.  43 candidates in all; each is clamped to [0,1].
//
// Every candidate is t = num / den with, per axis k and for a sign s_k,
//   al_k = s_k (a_k - c_k) - Z_k h_k,   be_k = s_k d_k,
//   num  = sum_k al_k (b_k - p_k be_k),  den = sum_k be_k (p_k be_k - b_k):
//   - ends (ids 0, 1): no axis terms, t = 0 or 1;
//   - slab planes x_k = c_k + s h_k (ids 2-7) and axis centres x_k = c_k
//     (ids 8-10, Z_k = 0): b_k = -1 on that axis, t = -al_k / be_k;
//   - edge (ids 11-22, two axes) and vertex (ids 23-30, three axes) regions:
//     p_k = 1 on the exceeded slabs, t = -sum al_k be_k / sum be_k^2, the
//     stationary point of the squared distance to that edge or vertex;
//   - two face distances crossing inside the box (ids 31-42): b = -1 on the
//     lower axis j and +1 on the higher one k, t = (al_k - al_j) / (be_j - be_k).
// One arithmetic path for all of them (no branches on the candidate's kind);
// the table holds (s_k, Z_k, p_k, b_k) per candidate and axis.
constexpr int CB_CANDIDATES = 43;
static __device__ const float4 CB_TABLE[CB_CANDIDATES][3] = {
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{-1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {-1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, -1.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {-1.0f, 1.0f, 0.0f, -1.0f}},
    {{1.0f, 0.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 0.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 0.0f, 0.0f, -1.0f}},
    {{1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{-1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{-1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}},
    {{-1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}},
    {{1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}},
    {{-1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}},
    {{1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}},
    {{-1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}},
    {{1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}},
    {{-1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}},
    {{1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}},
    {{-1.0f, 1.0f, 1.0f, 0.0f}, {1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}},
    {{1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}},
    {{-1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}, {-1.0f, 1.0f, 1.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{-1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, -1.0f}, {-1.0f, 1.0f, 0.0f, 1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{-1.0f, 1.0f, 0.0f, -1.0f}, {-1.0f, 1.0f, 0.0f, 1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}},
    {{1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 1.0f}},
    {{-1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, 1.0f}},
    {{1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {-1.0f, 1.0f, 0.0f, 1.0f}},
    {{-1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 0.0f}, {-1.0f, 1.0f, 0.0f, 1.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 1.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {-1.0f, 1.0f, 0.0f, -1.0f}, {1.0f, 1.0f, 0.0f, 1.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {1.0f, 1.0f, 0.0f, -1.0f}, {-1.0f, 1.0f, 0.0f, 1.0f}},
    {{1.0f, 1.0f, 0.0f, 0.0f}, {-1.0f, 1.0f, 0.0f, -1.0f}, {-1.0f, 1.0f, 0.0f, 1.0f}},
};
__device__ __forceinline__ float capsule_box_candidate(int id, const float* a, const float* d, const float* box) {
    float num = id == 1 ? 1.0f : 0.0f, den = id < 2 ? 1.0f : 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 c = __ldg(&CB_TABLE[id][k]);  // s, Z, p, b
        const float al = fmaf(c.x, a[k] - box[k], -(c.y * box[3 + k]));
        const float be = c.x * d[k];
        const float t1 = fmaf(-c.z, be, c.w);
        num = fmaf(al, t1, num);
        den = fmaf(be, -t1, den);
    }
    float t = num / den;
    if (!(t >= 0.0f)) t = 0.0f;  // also maps NaN from degenerate directions
    if (t > 1.0f) t = 1.0f;
    return t;
}

// Ball pairs live in 32 fixed slots: slot 0 the floor, slot 1 + l link l
// (l < 2 n_a <= 14), slot 16 + b box b (b < 16); slot t sits on group lane
// t % LPS as element t / LPS of the lane's depth sums.  One pass covers the
// LPS slots of one element: a pass that holds floor and link slots only runs
// the capsule test, one that holds box slots only runs the box test, and the
// single pass of a 32-lane group (both kinds) runs both tests on every lane
// and keeps the one its slot needs -- no divergent branches.  Contacts are
// compacted with a ballot per pass, in slot order, which is the canonical
// pair order.
template <int NA, int LPS, int S>
__device__ __forceinline__ void ball_pass(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g,
                                          float (&pa)[32 / LPS], float (&pbox)[32 / LPS], int& base,
                                          unsigned& tbits) {
    using d = Dims<NA>;
    static_assert(1 + 2 * MAXL <= 16 && MAXB <= 16, "ball pairs must fit their slot ranges");
    constexpr int lo = S * LPS, hi = lo + LPS;            // the slots of this pass
    constexpr bool has_link = lo < 1 + d::NL, has_box = hi > 16;
    if constexpr (!has_link && !has_box) return;
    const int nb = M.nb;
    if (!has_link && lo >= 16 + nb) return;  // no box slot in use (group-uniform)
    const int slot = lo + g.sl;
    const float* pb = &w.q[d::B];
    const float rb = M.rb;
    const bool isf = slot == 0, isc = slot >= 1 && slot <= d::NL, isb = slot >= 16 && slot < 16 + nb;
    float dist = 1.0f, nn[3] = {0.0f, 0.0f, 1.0f}, cp[3] = {0.0f, 0.0f, 0.0f};
    const int l = min(max(slot - 1, 0), d::NL - 1);
    if constexpr (has_link) {  // ball - capsule, and the floor on slot 0
        const float* a0 = w.a0[l];
        const float* a1 = w.a1[l];
        float dd[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
        float ac[3] = {pb[0] - a0[0], pb[1] - a0[1], pb[2] - a0[2]};
        const float den = dot3(dd, dd);
        float t = den > 0.0f ? dot3(ac, dd) / den : 0.0f;
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        float sp[3] = {a0[0] + t * dd[0], a0[1] + t * dd[1], a0[2] + t * dd[2]};
        float df[3] = {pb[0] - sp[0], pb[1] - sp[1], pb[2] - sp[2]};
        const float len = sqrtf(dot3(df, df));
        const float il = 1.0f / len;
        nn[0] = !isf && len > 0.0f ? df[0] * il : 0.0f;
        nn[1] = !isf && len > 0.0f ? df[1] * il : 0.0f;
        nn[2] = !isf && len > 0.0f ? df[2] * il : 1.0f;
        const float rc = M.link[l / NA][l % NA].rcap;
#pragma unroll
        for (int k = 0; k < 3; ++k) cp[k] = 0.5f * ((pb[k] - rb * nn[k]) + (sp[k] + rc * nn[k]));
        dist = len - rb - rc;
        if (isf) {  // ball - floor
            dist = (pb[2] - M.floor_z) - rb;
            cp[0] = pb[0];
            cp[1] = pb[1];
            cp[2] = 0.5f * ((pb[2] - rb) + M.floor_z);
        }
    }
    if constexpr (has_box) {  // ball - box
        if (nb > 0) {
            const float* box = M.box[min(max(slot - 16, 0), nb - 1)];
            float nb3[3], surf[3];
            const float db = box_sdf(pb, box, nb3, surf) - rb;
            if (isb) {
                dist = db;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    nn[k] = nb3[k];
                    cp[k] = 0.5f * ((pb[k] - rb * nn[k]) + surf[k]);
                }
            }
        }
    }
    const int Bb = isc ? l : -1;
    const bool active = (isf || isc || isb) && dist < 0.0f;
    const unsigned mask = g.ballot(active);
    const int pos = base + __popc(mask & ((1u << g.sl) - 1u));
    const bool keep = active && pos < M.maxc;
    pa[S] += active ? -dist : 0.0f;
    pbox[S] += active && isb ? -dist : 0.0f;
    tbits |= keep ? 4u | (Bb >= 0 ? 1u << (Bb / NA) : 0u) : 0u;
    if (keep) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            w.cp[pos][k] = cp[k];
            w.cn[pos][k] = nn[k];
        }
        w.cdep[pos] = -dist;
        w.cA[pos] = d::B;
        w.cB[pos] = Bb;
    }
    base += __popc(mask);
}

// Narrow phase in canonical pair order (ball-floor, ball-links, ball-boxes,
// links x boxes).  Ball pairs: one lane per pair slot (above), exact,
// compacted with a ballot.  Capsule-box pairs: a conservative
// separating-axis cull per lane (segment_meets_inflated_box), then each
// surviving pair (in pair order) is minimised by the whole group over the
// candidate set above.  Each lane adds
// the depths of the contacts it found to pa (all) and pbox (against boxes),
// per slot element; every lane gets the number of stored contacts (ncon) and
// the blocks they touch (tb: 1 left arm, 2 right arm, 4 ball).  Returns the
// number of exact capsule-box tests on group lane 0 (0 on the other lanes).
template <int NA, int LPS>
__device__ __forceinline__ int collide(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g,
                                      float (&pa)[32 / LPS], float (&pbox)[32 / LPS], int& ncon, int& tb) {
    using d = Dims<NA>;
    const int nb = M.nb;
    int base = 0, nsurv = 0;
    unsigned tbits = 0u;  // blocks the stored contacts touch
    ball_pass<NA, LPS, 0>(M, w, g, pa, pbox, base, tbits);
    if constexpr (LPS <= 16) ball_pass<NA, LPS, 1>(M, w, g, pa, pbox, base, tbits);
    if constexpr (LPS <= 8) {
        ball_pass<NA, LPS, 2>(M, w, g, pa, pbox, base, tbits);
        ball_pass<NA, LPS, 3>(M, w, g, pa, pbox, base, tbits);
    }
    // capsule-box: lane l (and, where a pass over the links fills half the
    // group, lane CL + l) tests link l's capsule against the boxes (or one
    // half of them each): the segment against the box inflated by the
    // capsule radius (separating axes, conservative); the survivors are
    // placed link-major, box-minor by a prefix sum over the links
    if (nb > 0) {
        constexpr int CL = d::NL <= LPS / 2 ? LPS / 2 : LPS;  // lanes of one pass over the links
        constexpr int NH = LPS / CL;                          // box halves
        const int l = g.sl & (CL - 1), half = g.sl / CL;
        const int bsplit = NH == 2 ? (nb + 1) >> 1 : nb;
        const int b0 = half ? bsplit : 0, b1 = half ? nb : bsplit;
        unsigned smask = 0u;
        if (l < d::NL) {
            const float* a0 = w.a0[l];
            const float* a1 = w.a1[l];
            const float rc = M.link[l / NA][l % NA].rcap;
            float mid[3], hv[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                mid[k] = 0.5f * (a0[k] + a1[k]);
                hv[k] = 0.5f * (a1[k] - a0[k]);
            }
#pragma unroll 4
            for (int bi = b0; bi < b1; ++bi)
                if (segment_meets_inflated_box(mid, hv, M.box[bi], rc)) smask |= 1u << bi;
        }
        const int cnt = __popc(smask);
        const int cnt_link = NH == 2 ? cnt + g.xor_(cnt, CL) : cnt;  // both halves of link l
        int pre = cnt_link;  // inclusive prefix over the links (both halves alike)
#pragma unroll
        for (int off = 1; off < CL; off <<= 1) {
            const int o = __shfl_up_sync(g.gm, pre, off, CL);
            if (l >= off) pre += o;
        }
        int pos = pre - cnt_link + (half ? cnt_link - cnt : 0);
        while (smask) {
            const int bi = __ffs(smask) - 1;
            smask &= smask - 1u;
            w.ph.col.surv[pos++] = (short)(l * nb + bi);
        }
        nsurv = g.shfl(pre, CL - 1);
    }
    g.sync();
    for (int si = 0; si < nsurv; ++si) {
        const int idx = w.ph.col.surv[si];
        const int l = idx / nb, bi = idx - l * nb;
        const float* box = M.box[bi];
        const float* a0 = w.a0[l];
        const float rc = M.link[l / NA][l % NA].rcap;
        const float dd[3] = {w.a1[l][0] - a0[0], w.a1[l][1] - a0[1], w.a1[l][2] - a0[2]};
        float bf = INFINITY, bt = 0.0f;
        for (int cid = g.sl; cid < CB_CANDIDATES; cid += LPS) {
            const float t = capsule_box_candidate(cid, a0, dd, box);
            const float f = box_sdf_only(a0, dd, t, box);
            if (f < bf || (f == bf && t < bt)) {
                bf = f;
                bt = t;
            }
        }
        // the lexicographic minimum of (f, t) over all candidates: the same
        // whichever lanes held them
#pragma unroll
        for (int off = LPS / 2; off > 0; off >>= 1) {
            const float of = g.xor_(bf, off);
            const float ot = g.xor_(bt, off);
            if (of < bf || (of == bf && ot < bt)) {
                bf = of;
                bt = ot;
            }
        }
        float x[3] = {a0[0] + bt * dd[0], a0[1] + bt * dd[1], a0[2] + bt * dd[2]};
        float nn[3], surf[3];
        const float dist = box_sdf(x, box, nn, surf) - rc;
        if (dist < 0.0f) {
            if (g.sl == 0) {
                pa[0] += -dist;
                pbox[0] += -dist;
                if (base < M.maxc) {
                    tbits |= 1u << (l / NA);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        w.cp[base][k] = 0.5f * ((x[k] - rc * nn[k]) + surf[k]);
                        w.cn[base][k] = nn[k];
                    }
                    w.cdep[base] = -dist;
                    w.cA[base] = l;
                    w.cB[base] = -1;
                }
            }
            ++base;
        }
    }
    tb = (int)__reduce_or_sync(g.gm, tbits);
    ncon = base < M.maxc ? base : M.maxc;
    return g.sl == 0 ? nsurv : 0;
}

// ---------------------------------------------------------------------------
// dynamics: free velocity vf = qd + dt (M + dt D)^-1 (tau_drive - c - D qd)
// ---------------------------------------------------------------------------
// Inclusive scans over the links of one arm (the lane's arm segment; lanes
// past the last link hold zeros).  Suffix sums run towards the base, prefix
// sums towards the tip.
template <int N, int LPS>
__device__ __forceinline__ void seg_suffix_sum(const Lanes<LPS>& g, float (&v)[N], int i, int nlinks) {
#pragma unroll
    for (int off = 1; off < Lanes<LPS>::SEG; off <<= 1) {
        if (off >= nlinks) break;
#pragma unroll
        for (int t = 0; t < N; ++t) {
            const float o = g.down_seg(v[t], off);
            if (i + off < nlinks) v[t] += o;  // lanes past the last link never enter
        }
    }
}
template <int N, int LPS>
__device__ __forceinline__ void seg_prefix_sum(const Lanes<LPS>& g, float (&v)[N], int i, int nlinks) {
#pragma unroll
    for (int off = 1; off < Lanes<LPS>::SEG; off <<= 1) {
        if (off >= nlinks) break;
#pragma unroll
        for (int t = 0; t < N; ++t) {
            const float o = g.up_seg(v[t], off);
            if (i >= off) v[t] += o;
        }
    }
}

// Cholesky factor of arm a's block of (M + dt D) (lower triangle of w.L[a]
// on entry) and the solution y of (M + dt D) y = rhs for that arm, in
// registers; ok is false on a finite non-positive pivot.
template <int NA>
__device__ __forceinline__ void arm_solve(const WarpWS<NA>& w, int a, float (&A)[NA][NA], float (&di)[NA],
                                          float (&y)[NA], bool& ok) {
#pragma unroll
    for (int r = 0; r < NA; ++r)
#pragma unroll
        for (int cc = 0; cc <= r; ++cc) A[r][cc] = w.L[a][r][cc];
    ok = true;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        float sj = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) sj -= A[j][k] * A[j][k];
        // a NaN pivot comes from a non-finite state (reported through the
        // cost); only a finite non-positive pivot is a loss of positive
        // definiteness
        ok = ok && !(sj <= 0.0f);
        const float inv = rsqrtf(sj);
        A[j][j] = sj * inv;
        di[j] = inv;
#pragma unroll
        for (int r = j + 1; r < NA; ++r) {
            float t = A[r][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= A[r][k] * A[j][k];
            A[r][j] = t * inv;
        }
    }
#pragma unroll
    for (int r = 0; r < NA; ++r) {
        float sr = w.rhs[a * NA + r];
#pragma unroll
        for (int k = 0; k < r; ++k) sr -= A[r][k] * y[k];
        y[r] = sr * di[r];
    }
#pragma unroll
    for (int r = NA - 1; r >= 0; --r) {
        float sr = y[r];
#pragma unroll
        for (int k = r + 1; k < NA; ++k) sr -= A[k][r] * y[k];
        y[r] = sr * di[r];
    }
}

template <int NA, int LPS>
__device__ __forceinline__ void arm_factor_step(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g, int* err,
                                                int tb);

template <int NA, int LPS>
__device__ __forceinline__ void dynamics(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g, int* err,
                                         const float (&R)[9], const float (&cl)[3], int tb, bool solve) {
    const int a = g.a, i = g.i;
    const bool act = i < NA;
    const int l = a * NA + (act ? i : 0);
    // (1) per link (lane i): spatial inertia about the world origin
    //     (m, h = m c, J = R I R^T + m(|c|^2 E - c c^T)), joint motion axis
    //     S = (z, o x z), velocity term S qd
    //     Every lane computes (no divergent branch); lanes past the last
    //     link work on link 0's data, and the scans below never pass their
    //     values to a link's lane.
    float Is[10], S[6], sq[6];
    float qdi;
    {
        const DevLink& L = M.link[a][l - a * NA];
        const float* Ib = L.I;
        const float B9[9] = {Ib[0], Ib[3], Ib[4], Ib[3], Ib[1], Ib[5], Ib[4], Ib[5], Ib[2]};
        float T[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                T[3 * r + cc] = R[3 * r] * B9[cc] + R[3 * r + 1] * B9[3 + cc] + R[3 * r + 2] * B9[6 + cc];
        const float c0 = cl[0], c1 = cl[1], c2 = cl[2];
        const float m = L.mass;
        const float cc2 = c0 * c0 + c1 * c1 + c2 * c2;
        Is[0] = m;
        Is[1] = m * c0;
        Is[2] = m * c1;
        Is[3] = m * c2;
        Is[4] = T[0] * R[0] + T[1] * R[1] + T[2] * R[2] + m * (cc2 - c0 * c0);
        Is[5] = T[3] * R[3] + T[4] * R[4] + T[5] * R[5] + m * (cc2 - c1 * c1);
        Is[6] = T[6] * R[6] + T[7] * R[7] + T[8] * R[8] + m * (cc2 - c2 * c2);
        Is[7] = T[0] * R[3] + T[1] * R[4] + T[2] * R[5] - m * c0 * c1;
        Is[8] = T[0] * R[6] + T[1] * R[7] + T[2] * R[8] - m * c0 * c2;
        Is[9] = T[3] * R[6] + T[4] * R[7] + T[5] * R[8] - m * c1 * c2;
        S[0] = w.z[l][0];
        S[1] = w.z[l][1];
        S[2] = w.z[l][2];
        cross3(w.o[l], w.z[l], S + 3);
        qdi = w.qd[l];
#pragma unroll
        for (int t = 0; t < 6; ++t) sq[t] = S[t] * qdi;
    }
    // (2) composite inertia of the subtree (suffix) and F_i = I^c_i S_i;
    //     spatial velocity V_i = sum_{k<=i} S_k qd_k (prefix)
    float Ic[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) Ic[t] = Is[t];
    seg_suffix_sum<10>(g, Ic, i, NA);
    float F[6];
    spatial_inertia_apply(Ic, S, F);
    float V[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) V[t] = sq[t];
    seg_prefix_sum<6>(g, V, i, NA);
    // (3) velocity-product acceleration A_i = sum_{k<=i} V_{k-1} x (S_k qd_k)
    float Vp[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        Vp[t] = g.up_seg(V[t], 1);
        if (i == 0) Vp[t] = 0.0f;
    }
    float Aa[6];
    {
        float t1[3], t2[3], t3[3];
        cross3(Vp, sq, t1);
        cross3(Vp, sq + 3, t2);
        cross3(Vp + 3, sq, t3);
        Aa[0] = t1[0];
        Aa[1] = t1[1];
        Aa[2] = t1[2];
        Aa[3] = t2[0] + t3[0];
        Aa[4] = t2[1] + t3[1];
        Aa[5] = t2[2] + t3[2];
    }
    seg_prefix_sum<6>(g, Aa, i, NA);
    // bias force of link i: I_i (A_i + a_g) + V_i x* (I_i V_i), gravity as a
    // base acceleration -g on links without compensation
    float f[6];
    {
        const float gw = act ? 1.0f - M.link[a][l - a * NA].gravcomp : 0.0f;
        Aa[3] -= gw * M.g[0];
        Aa[4] -= gw * M.g[1];
        Aa[5] -= gw * M.g[2];
        float IA[6], IV[6];
        spatial_inertia_apply(Is, Aa, IA);
        spatial_inertia_apply(Is, V, IV);
        float n1[3], n2[3], f1[3];
        cross3(V, IV, n1);
        cross3(V + 3, IV + 3, n2);
        cross3(V, IV + 3, f1);
        f[0] = IA[0] + n1[0] + n2[0];
        f[1] = IA[1] + n1[1] + n2[1];
        f[2] = IA[2] + n1[2] + n2[2];
        f[3] = IA[3] + f1[0];
        f[4] = IA[4] + f1[1];
        f[5] = IA[5] + f1[2];
    }
    // (4) bias torque S_i . (subtree force); drive; implicit damping
    seg_suffix_sum<6>(g, f, i, NA);
    {  // every lane computes, the links' lanes store
        const float tb = S[0] * f[0] + S[1] * f[1] + S[2] * f[2] + S[3] * f[3] + S[4] * f[4] + S[5] * f[5];
        const DevLink& L = M.link[a][l - a * NA];
        const float td = fminf(fmaxf(L.gear * w.u[l], -L.tau_max), L.tau_max);
        const float rhs = td - tb - L.D * qdi;
        if (act) w.rhs[l] = rhs;
    }
    // (5) mass-matrix column c = i, M[r][c] = S_r . F_c (r <= c), on lane c
    //     of the arm's segment: S_r comes from lane r by shuffles, F_c is the
    //     lane's own; dt D on the diagonal.  The dot product's rounding is
    //     written out (explicit FMAs) so that every layout forms the same bits.
    {
        const float dtD = M.dt * M.link[a][l - a * NA].D;
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            float sr[6];
#pragma unroll
            for (int t = 0; t < 6; ++t) sr[t] = __shfl_sync(g.gm, S[t], r, Lanes<LPS>::SEG);
            float mv = __fmul_rn(sr[0], F[0]);
#pragma unroll
            for (int t = 1; t < 6; ++t) mv = __fmaf_rn(sr[t], F[t], mv);
            if (r == i) mv = __fadd_rn(mv, dtD);
            if (act && r <= i) w.L[a][i][r] = mv;
        }
    }
    g.sync();
    // (6) Cholesky of each arm block (in registers), the free velocity; ball.
    //     The factor is kept only for arms a contact touches (the contact
    //     solve's rows need it there).  Skipped (solve = false) when the
    //     caller solves the arms together with a ball-only contact problem.
    if (solve) arm_factor_step<NA, LPS>(M, w, g, err, tb);
}

// (6) of dynamics on its own: the Cholesky factor of each arm block (in
// registers) and the free velocity; the ball's free velocity.  The factor is
// kept for the arms a contact touches (tb), whose contact rows need it.
template <int NA, int LPS>
__device__ __forceinline__ void arm_factor_step(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g, int* err,
                                                int tb) {
    using d = Dims<NA>;
    constexpr int SEG = Lanes<LPS>::SEG;
    const int a = g.a, i = g.i;
    const int armc = tb & 3;
    if (i == 0) {
        float A[NA][NA], di[NA], y[NA];
        bool ok;
        arm_solve<NA>(w, a, A, di, y, ok);
#pragma unroll
        for (int r = 0; r < NA; ++r) w.vf[a * NA + r] = w.qd[a * NA + r] + M.dt * y[r];
        if ((armc >> a) & 1) {
#pragma unroll
            for (int r = 0; r < NA; ++r) {
                w.Ldi[a][r] = di[r];
#pragma unroll
                for (int cc = 0; cc <= r; ++cc) w.L[a][r][cc] = A[r][cc];
            }
        }
        if (!ok) atomicOr(err, ERRB_CHOLESKY);
    }
    if (a == 0 && i == SEG - 1) {  // the ball's lane
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            w.vf[d::B + r] = w.qd[d::B + r] + M.dt * M.g[r];
            w.vf[d::B + 3 + r] = w.qd[d::B + 3 + r];
        }
    }
    g.sync();
}

// ---------------------------------------------------------------------------
// contacts: Jacobian rows half-solved by the factor, PGS in z = L^T v
// ---------------------------------------------------------------------------
template <int NA>
__device__ __forceinline__ void contact_frame_row(const float* n, int k, float* e) {
    if (k == 0) {
        e[0] = n[0];
        e[1] = n[1];
        e[2] = n[2];
        return;
    }
    // t1 = normalise(n x e_axis), axis of smallest |n_i| (ties -> lowest)
    const float ax = fabsf(n[0]), ay = fabsf(n[1]), az = fabsf(n[2]);
    int ia = 0;
    float best = ax;
    if (ay < best) {
        best = ay;
        ia = 1;
    }
    if (az < best) ia = 2;
    // n x e_ia, written out per axis (no dynamically indexed local array)
    float t1[3];
    t1[0] = ia == 0 ? 0.0f : (ia == 1 ? -n[2] : n[1]);
    t1[1] = ia == 0 ? n[2] : (ia == 1 ? 0.0f : -n[0]);
    t1[2] = ia == 0 ? -n[1] : (ia == 1 ? n[0] : 0.0f);
    const float il = rsqrtf(dot3(t1, t1));
    t1[0] *= il;
    t1[1] *= il;
    t1[2] *= il;
    if (k == 1) {
        e[0] = t1[0];
        e[1] = t1[1];
        e[2] = t1[2];
        return;
    }
    cross3(n, t1, e);
}


// One or two contacts that touch only the ball (floor, boxes): the rows act
// on the ball's six velocities alone and its mass matrix is diag(m, m, m,
// I, I, I), so every lane forms the whole problem in registers -- row
// directions e (signed by the ball's side) and d = (p - c) x e, Delassus
// G_rs = e_r.e_s / m + d_r.d_s / I, b_r = e_r.v_f + d_r.w_f -- runs the
// sweeps and applies the impulse, with no shared-memory rows or factor.
// The same iteration as the general path, summed in a different order.
template <int NA, int NC, int SW>
__device__ __forceinline__ void ball_contact_dv(const DevModel& M, const WarpWS<NA>& w, const float* vl,
                                                const float* va, float (&dv)[6]) {
    using d = Dims<NA>;
    constexpr int NR = 3 * NC;
    const float im = 1.0f / M.mb, iI = 1.0f / M.Ib, regc = (1.0f - M.imp) / M.imp;
    const float* bc = &w.q[d::B];
    // rows without the side sign s_c (+1 when the ball is body A): it enters
    // b, the cross-contact Delassus entries and the applied impulse
    float E[NR][3], D[NR][3], bb[NR], vs[NR], sg[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float sgn = w.cA[c] == d::B ? 1.0f : -1.0f;
        sg[c] = sgn;
        const float* p = w.cp[c];
        const float dd[3] = {p[0] - bc[0], p[1] - bc[1], p[2] - bc[2]};
        const float nrm[3] = {w.cn[c][0], w.cn[c][1], w.cn[c][2]};
        float fr[3][3];  // n, t1, t2 (the rows contact_frame_row gives)
        contact_frame_row<NA>(nrm, 1, fr[1]);
        cross3(nrm, fr[1], fr[2]);
#pragma unroll
        for (int q = 0; q < 3; ++q) fr[0][q] = nrm[q];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int r = 3 * c + k;
            const float* e = fr[k];
            float de[3];
            cross3(dd, e, de);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                E[r][q] = e[q];
                D[r][q] = de[q];
            }
            bb[r] = sgn * (dot3(E[r], vl) + dot3(D[r], va));
            vs[r] = k == 0 ? (M.erp / M.dt) * w.cdep[c] : 0.0f;
        }
    }
    float G[NR][NR], R[NR], iA[NR], lam[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
#pragma unroll
        for (int q = r; q < NR; ++q) {
            // one contact's frame is orthonormal: e_r . e_q = delta_rq; a
            // lone contact's block is diagonal (below)
            float g;
            if (NC == 1 && r != q) g = 0.0f;
            else if (r / 3 == q / 3) g = (r == q ? im : 0.0f) + iI * dot3(D[r], D[q]);
            else g = sg[r / 3] * sg[q / 3] * (im * dot3(E[r], E[q]) + iI * dot3(D[r], D[q]));
            G[r][q] = g;
            G[q][r] = g;
        }
        R[r] = regc * G[r][r];
        iA[r] = 1.0f / (G[r][r] + R[r]);
        lam[r] = 0.0f;
    }
    auto sweep = [&]() {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int rn = 3 * c;
            float res = bb[rn] + R[rn] * lam[rn] - vs[rn];
#pragma unroll
            for (int q = 0; q < NR; ++q) res += G[rn][q] * lam[q];
            const float ln = fmaxf(lam[rn] - res * iA[rn], 0.0f);
            lam[rn] = ln;
            float r1 = bb[rn + 1] + R[rn + 1] * lam[rn + 1];
            float r2 = bb[rn + 2] + R[rn + 2] * lam[rn + 2];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                r1 += G[rn + 1][q] * lam[q];
                r2 += G[rn + 2][q] * lam[q];
            }
            float l1 = lam[rn + 1] - r1 * iA[rn + 1];
            float l2 = lam[rn + 2] - r2 * iA[rn + 2];
            const float n2 = l1 * l1 + l2 * l2, lim = M.mu * ln;
            if (n2 > lim * lim) {
                const float sc = lim * rsqrtf(n2);
                l1 *= sc;
                l2 *= sc;
            }
            lam[rn + 1] = l1;
            lam[rn + 2] = l2;
        }
    };
    if constexpr (NC == 1) {
        // One contact of the ball with static geometry (floor or box): the
        // contact point lies on the normal through the ball's centre, so the
        // normal row has no angular part and the tangent rows' angular parts
        // are orthogonal -- the Delassus block is diagonal.  The first sweep
        // then puts every row at its own minimiser (the friction disk's
        // scaling depends on lambda_n alone) and later sweeps leave lambda
        // there: the sweeps reduce to this one.
        if (M.sweeps > 0) {
            const float ln = fmaxf((vs[0] - bb[0]) * iA[0], 0.0f);
            float l1 = -bb[1] * iA[1], l2 = -bb[2] * iA[2];
            const float n2 = l1 * l1 + l2 * l2, lim = M.mu * ln;
            if (n2 > lim * lim) {
                const float sc = lim * rsqrtf(n2);
                l1 *= sc;
                l2 *= sc;
            }
            lam[0] = ln;
            lam[1] = l1;
            lam[2] = l2;
        }
    } else if (SW > 0) {  // a sweep count fixed at compile time, unrolled
#pragma unroll
        for (int sw = 0; sw < SW; ++sw) sweep();
    } else if (M.sweeps == 4) {  // the scenes' sweep counts, unrolled
        sweep();
        sweep();
        sweep();
        sweep();
    } else if (M.sweeps == 3) {
        sweep();
        sweep();
        sweep();
    } else {
        for (int sw = 0; sw < M.sweeps; ++sw) sweep();
    }
    // M^-1 J^T lambda on the ball
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float sl = 0.0f, sa = 0.0f;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const float sl_r = sg[r / 3] * lam[r];
            sl += E[r][k] * sl_r;
            sa += D[r][k] * sl_r;
        }
        dv[k] = im * sl;
        dv[3 + k] = iI * sa;
    }
}

// v = v_f + M^-1 J^T lambda on the ball, v_f elsewhere.
template <int NA, int NC, int LPS>
__device__ __forceinline__ void contacts_ball(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g) {
    using d = Dims<NA>;
    float dv[6];
    ball_contact_dv<NA, NC, 0>(M, w, &w.vf[d::B], &w.vf[d::B + 3], dv);
#pragma unroll
    for (int c0 = 0; c0 < d::NV; c0 += LPS) {
        const int c = c0 + g.sl;
        if (c < d::NV) {
            float add = 0.0f;
#pragma unroll
            for (int k = 0; k < 6; ++k)
                if (c == d::B + k) add = dv[k];
            w.v[c] = w.vf[c] + add;
        }
    }
    g.sync();
}

// The free velocity and a ball-only contact solve together (one or two
// contacts of the ball with static geometry; SW sweeps for two).  Every lane of an
// arm's half-warp factors that arm's block and solves for its free velocity
// (the operations of the one-lane factor in dynamics) while every lane runs
// the contact solve: with no divergence between them the two independent
// chains share the issue slots.  Writes v: the arms' free velocities and the
// ball's after the impulses (the values dynamics and contacts_ball give).
template <int NA, int NC, int SW, int LPS>
__device__ __forceinline__ void solve_ball_contacts(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g,
                                                    int* err) {
    using d = Dims<NA>;
    constexpr int SEG = Lanes<LPS>::SEG;
    const int a = g.a, i = g.i;
    float vb[6];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        vb[r] = w.qd[d::B + r] + M.dt * M.g[r];
        vb[3 + r] = w.qd[d::B + 3 + r];
    }
    float A[NA][NA], di[NA], y[NA];
    bool ok;
    arm_solve<NA>(w, a, A, di, y, ok);
    float dv[6];
    ball_contact_dv<NA, NC, SW>(M, w, vb, vb + 3, dv);
    if (i == 0 && !ok) atomicOr(err, ERRB_CHOLESKY);
    // lane i < NA of segment a: the arm's velocity i (formed on every lane,
    // one stored); the ball's lane stores the ball's six
    float yi = y[0];
#pragma unroll
    for (int r = 1; r < NA; ++r)
        if (i == r) yi = y[r];
    const float vf = w.qd[a * NA + (i < NA ? i : 0)] + M.dt * yi;
    if (i < NA) w.v[a * NA + i] = vf;
    if (a == 0 && i == SEG - 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) w.v[d::B + k] = vb[k] + dv[k];
    }
    g.sync();
}

// Projected Gauss-Seidel for one or two contacts with the Delassus block in
// registers: every lane runs the same sweeps (no shuffles, no shared-memory
// round trips), then lane r stores lambda_r.  The same iteration as the
// lane-parallel path below, summed in a different order.
template <int NA, int NC, int LPS>
__device__ __forceinline__ void pgs_small(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g) {
    constexpr int NR = 3 * NC;
    float G[NR][NR], bb[NR], R[NR], iA[NR], vs[NR], lam[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
#pragma unroll
        for (int q = 0; q < NR; ++q) G[r][q] = w.ph.con.G[r * NR + q];
        const float4 c4 = w.ph.con.rc4[r];
        bb[r] = c4.x;
        R[r] = c4.y;
        iA[r] = c4.z;
        vs[r] = c4.w;
        lam[r] = 0.0f;
    }
    for (int sw = 0; sw < M.sweeps; ++sw) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int rn = 3 * c;
            float res = bb[rn] + R[rn] * lam[rn] - vs[rn];
#pragma unroll
            for (int q = 0; q < NR; ++q) res += G[rn][q] * lam[q];
            const float ln = fmaxf(lam[rn] - res * iA[rn], 0.0f);
            lam[rn] = ln;
            float r1 = bb[rn + 1] + R[rn + 1] * lam[rn + 1];
            float r2 = bb[rn + 2] + R[rn + 2] * lam[rn + 2];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                r1 += G[rn + 1][q] * lam[q];
                r2 += G[rn + 2][q] * lam[q];
            }
            float l1 = lam[rn + 1] - r1 * iA[rn + 1];
            float l2 = lam[rn + 2] - r2 * iA[rn + 2];
            const float n2 = l1 * l1 + l2 * l2, lim = M.mu * ln;
            if (n2 > lim * lim) {
                const float sc = lim * rsqrtf(n2);
                l1 *= sc;
                l2 *= sc;
            }
            lam[rn + 1] = l1;
            lam[rn + 2] = l2;
        }
    }
    static_assert(NR <= LPS, "one lane per row");
#pragma unroll
    for (int r = 0; r < NR; ++r)
        if (g.sl == r) w.ph.con.lam[r] = lam[r];
}

// Soft contact by projected Gauss-Seidel in contact space.  With the
// factor L L^T = M + dt D and rows Y_r = L^-1 J_r^T, the Delassus matrix is
// G = Y Y^T and the unconstrained row velocities are b = Y z_f, z_f = L^T
// v_f; after the sweeps v = L^-T (z_f + Y^T lambda).  This is the same
// iteration as updating v row by row (J_r v = b_r + (G lambda)_r).
template <int NA, int LPS>
__device__ __forceinline__ void contacts(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g, int nc, int tb) {
    using d = Dims<NA>;
    constexpr int SEG = Lanes<LPS>::SEG;
    if (nc == 0) {
#pragma unroll
        for (int c0 = 0; c0 < d::NV; c0 += LPS)
            if (c0 + g.sl < d::NV) w.v[c0 + g.sl] = w.vf[c0 + g.sl];
        g.sync();
        return;
    }
    const float ismb = rsqrtf(M.mb), isIb = rsqrtf(M.Ib);
    // tb: the blocks any contact touches (warp-uniform, from the narrow
    // phase).  Untouched blocks keep v = v_f and skip the z-space work.
    if (tb == 4 && nc <= 2) {  // ball against static geometry only
        if (nc == 1) contacts_ball<NA, 1>(M, w, g);
        else contacts_ball<NA, 2>(M, w, g);
        return;
    }
    // z_f = L^T v_f (one lane per arm coordinate; the ball's lane the ball)
    {
        const int a = g.a, i = g.i;
        if (i < NA && ((tb >> a) & 1)) {
            float sz = 0.0f;
#pragma unroll
            for (int k = 0; k < NA; ++k)
                if (k >= i) sz += w.L[a][k][i] * w.vf[a * NA + k];
            w.zz[a * NA + i] = sz;
        }
        if (a == 0 && i == SEG - 1 && (tb & 4)) {
            const float smb = M.mb * ismb, sIb = M.Ib * isIb;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                w.zz[d::B + r] = smb * w.vf[d::B + r];
                w.zz[d::B + 3 + r] = sIb * w.vf[d::B + 3 + r];
            }
        }
    }
    // rows: Jacobian of the touched bodies (in registers), half-solved by
    // the factor, one store per row
    const int nr = 3 * nc;
    for (int r = g.sl; r < nr; r += LPS) {
        const int c = r / 3, k = r - 3 * (r / 3);
        float e[3];
        contact_frame_row<NA>(w.cn[c], k, e);
        const float* p = w.cp[c];
        float ya[2][NA], yb[6];
#pragma unroll
        for (int q = 0; q < NA; ++q) ya[0][q] = ya[1][q] = 0.0f;
#pragma unroll
        for (int q = 0; q < 6; ++q) yb[q] = 0.0f;
        int msk = 0;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int body = side == 0 ? w.cA[c] : w.cB[c];
            const float sgn = side == 0 ? 1.0f : -1.0f;
            if (body == d::B) {
                const float* bc = &w.q[d::B];
                float dd[3] = {p[0] - bc[0], p[1] - bc[1], p[2] - bc[2]};
                float de[3];
                cross3(dd, e, de);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    yb[q] += sgn * e[q];
                    yb[3 + q] += sgn * de[q];
                }
                msk |= 4;
            } else if (body >= 0) {
                const int ab = body >= NA ? 1 : 0;
                const int ib = body - ab * NA;
                float col[NA];
#pragma unroll
                for (int q = 0; q < NA; ++q) {
                    col[q] = 0.0f;
                    if (q <= ib) {
                        const int lq = ab * NA + q;
                        float dd[3] = {p[0] - w.o[lq][0], p[1] - w.o[lq][1], p[2] - w.o[lq][2]};
                        float cz[3];
                        cross3(w.z[lq], dd, cz);
                        col[q] = sgn * dot3(e, cz);
                    }
                }
                if (ab == 0) {
#pragma unroll
                    for (int q = 0; q < NA; ++q) ya[0][q] += col[q];
                } else {
#pragma unroll
                    for (int q = 0; q < NA; ++q) ya[1][q] += col[q];
                }
                msk |= 1 << ab;
            }
        }
#pragma unroll
        for (int ab = 0; ab < 2; ++ab) {
            if (msk & (1 << ab)) {
#pragma unroll
                for (int ii = 0; ii < NA; ++ii) {
                    float sv = ya[ab][ii];
#pragma unroll
                    for (int kk = 0; kk < ii; ++kk) sv -= w.L[ab][ii][kk] * ya[ab][kk];
                    ya[ab][ii] = sv * w.Ldi[ab][ii];
                }
            }
        }
        float* y = w.ph.con.Y[r];
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            y[q] = ya[0][q];
            y[NA + q] = ya[1][q];
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            y[d::B + q] = yb[q] * ismb;
            y[d::B + 3 + q] = yb[3 + q] * isIb;
        }
        w.ph.con.tmask[r] = msk;
        w.ph.con.rc4[r].w = (k == 0) ? (M.erp / M.dt) * w.cdep[c] : 0.0f;
        w.ph.con.lam[r] = 0.0f;
    }
    g.sync();
    // Delassus block G = Y Y^T (nr x nr) and b = Y z_f, over the blocks rows
    // share
    const float regc = (1.0f - M.imp) / M.imp;
    const int npk = nr * (nr + 1) / 2;
    for (int t = g.sl; t < npk + nr; t += LPS) {
        if (t < npk) {
            // decode (r, s), r <= s, from the upper-triangle index
            int r = 0, rem = t;
            while (rem >= nr - r) {
                rem -= nr - r;
                ++r;
            }
            const int sc = r + rem;
            const int m = w.ph.con.tmask[r] & w.ph.con.tmask[sc];
            const float* yr = w.ph.con.Y[r];
            const float* ys = w.ph.con.Y[sc];
            float g = 0.0f;
            if (m & 1) {
#pragma unroll
                for (int q = 0; q < NA; ++q) g += yr[q] * ys[q];
            }
            if (m & 2) {
#pragma unroll
                for (int q = NA; q < 2 * NA; ++q) g += yr[q] * ys[q];
            }
            if (m & 4) {
#pragma unroll
                for (int q = d::B; q < d::NV; ++q) g += yr[q] * ys[q];
            }
            w.ph.con.G[r * nr + sc] = g;
            w.ph.con.G[sc * nr + r] = g;
            if (sc == r) {
                const float R = regc * g;
                w.ph.con.rc4[r].y = R;
                w.ph.con.rc4[r].z = 1.0f / (g + R);
            }
        } else {
            const int r = t - npk;
            const int m = w.ph.con.tmask[r];
            const float* yr = w.ph.con.Y[r];
            float bb = 0.0f;
            if (m & 1) {
#pragma unroll
                for (int q = 0; q < NA; ++q) bb += yr[q] * w.zz[q];
            }
            if (m & 2) {
#pragma unroll
                for (int q = NA; q < 2 * NA; ++q) bb += yr[q] * w.zz[q];
            }
            if (m & 4) {
#pragma unroll
                for (int q = d::B; q < d::NV; ++q) bb += yr[q] * w.zz[q];
            }
            w.ph.con.rc4[r].x = bb;
        }
    }
    g.sync();
    // projected Gauss-Seidel sweeps (normal row, then the tangent pair with
    // the friction disk |lambda_t| <= mu lambda_n).  One or two contacts:
    // registers.  More: row q's lambda sits on group lane q % LPS as element
    // q / LPS; the three residuals of a contact are one butterfly reduction
    // of G_rq lambda_q over the rows (the order of a 32-lane butterfly with
    // offsets 1, 2, 4, ..., in-lane folds past LPS), and the tangent
    // residuals take the normal update through G's normal column.
    if (nc == 1) {
        pgs_small<NA, 1>(M, w, g);
    } else if (nc == 2) {
        pgs_small<NA, 2>(M, w, g);
    } else {
        constexpr int RS = 32 / LPS;  // row slots per lane
        float lamA[RS];
#pragma unroll
        for (int t = 0; t < RS; ++t) lamA[t] = 0.0f;
        int width = 1;
        while (width < nr && width < 32) width <<= 1;
        for (int sw = 0; sw < M.sweeps; ++sw) {
            for (int c = 0; c < nc; ++c) {
                const int rn = 3 * c;
                float p0[RS], p1[RS], p2[RS];
#pragma unroll
                for (int t = 0; t < RS; ++t) {
                    const int q = t * LPS + g.sl;
                    p0[t] = p1[t] = p2[t] = 0.0f;
                    if (q < nr) {
                        p0[t] = w.ph.con.G[rn * nr + q] * lamA[t];
                        p1[t] = w.ph.con.G[(rn + 1) * nr + q] * lamA[t];
                        p2[t] = w.ph.con.G[(rn + 2) * nr + q] * lamA[t];
                    }
                }
                const float4 cN = w.ph.con.rc4[rn], c1 = w.ph.con.rc4[rn + 1], c2 = w.ph.con.rc4[rn + 2];
                const float g1n = w.ph.con.G[(rn + 1) * nr + rn];
                const float g2n = w.ph.con.G[(rn + 2) * nr + rn];
                for (int off = 1; off < width && off < LPS; off <<= 1) {
#pragma unroll
                    for (int t = 0; t < RS; ++t) {
                        p0[t] += g.xor_(p0[t], off);
                        p1[t] += g.xor_(p1[t], off);
                        p2[t] += g.xor_(p2[t], off);
                    }
                }
#pragma unroll
                for (int st = 1; st < RS; st <<= 1) {
                    if (st * LPS >= width) break;
#pragma unroll
                    for (int t = 0; t + st < RS; t += 2 * st) {
                        p0[t] += p0[t + st];
                        p1[t] += p1[t + st];
                        p2[t] += p2[t + st];
                    }
                }
                // lambda of row r: element r / LPS on group lane r % LPS
                auto lam_of = [&](int r) {
                    float v = lamA[0];
#pragma unroll
                    for (int t = 1; t < RS; ++t)
                        if (r / LPS == t) v = lamA[t];
                    return g.shfl(v, r % LPS);
                };
                const float ln0 = lam_of(rn);
                const float l10 = lam_of(rn + 1);
                const float l20 = lam_of(rn + 2);
                const float res = cN.x + p0[0] + cN.y * ln0 - cN.w;
                const float ln = fmaxf(ln0 - res * cN.z, 0.0f);
                const float dn = ln - ln0;
                const float r1 = c1.x + p1[0] + g1n * dn + c1.y * l10;
                const float r2 = c2.x + p2[0] + g2n * dn + c2.y * l20;
                float l1 = l10 - r1 * c1.z;
                float l2 = l20 - r2 * c2.z;
                const float n2 = l1 * l1 + l2 * l2, lim = M.mu * ln;
                if (n2 > lim * lim) {
                    const float sc = lim * rsqrtf(n2);
                    l1 *= sc;
                    l2 *= sc;
                }
#pragma unroll
                for (int t = 0; t < RS; ++t) {
                    const int q = t * LPS + g.sl;
                    if (q == rn) lamA[t] = ln;
                    if (q == rn + 1) lamA[t] = l1;
                    if (q == rn + 2) lamA[t] = l2;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < RS; ++t)
            if (t * LPS + g.sl < nr) w.ph.con.lam[t * LPS + g.sl] = lamA[t];
    }
    g.sync();
    // z = z_f + Y^T lambda, then v = L^-T z on the touched blocks
#pragma unroll
    for (int c0 = 0; c0 < d::NV; c0 += LPS) {
        const int c = c0 + g.sl;
        if (c < d::NV) {
            const int blk = c < NA ? 1 : (c < 2 * NA ? 2 : 4);
            if (tb & blk) {
                float zv = w.zz[c];
                for (int r = 0; r < nr; ++r) zv += w.ph.con.Y[r][c] * w.ph.con.lam[r];
                w.zz[c] = zv;
            } else {
                w.v[c] = w.vf[c];
            }
        }
    }
    g.sync();
    if (g.i == 0 && ((tb >> g.a) & 1)) {
        const int a = g.a;
        float zl[NA], t[NA];
#pragma unroll
        for (int ii = 0; ii < NA; ++ii) zl[ii] = w.zz[a * NA + ii];
#pragma unroll
        for (int ii = NA - 1; ii >= 0; --ii) {
            float sv = zl[ii];
#pragma unroll
            for (int k = ii + 1; k < NA; ++k) sv -= w.L[a][k][ii] * t[k];
            t[ii] = sv * w.Ldi[a][ii];
        }
#pragma unroll
        for (int ii = 0; ii < NA; ++ii) w.v[a * NA + ii] = t[ii];
    }
    if (g.a == 0 && g.i == SEG - 1 && (tb & 4)) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            w.v[d::B + r] = w.zz[d::B + r] * ismb;
            w.v[d::B + 3 + r] = w.zz[d::B + 3 + r] * isIb;
        }
    }
    g.sync();
}

// ---------------------------------------------------------------------------
// semi-implicit Euler
// ---------------------------------------------------------------------------
template <int NA, int LPS>
__device__ __forceinline__ void integrate(const DevModel& M, WarpWS<NA>& w, const Lanes<LPS>& g) {
    using d = Dims<NA>;
    const float dt = M.dt;
    {  // every lane forms the new orientation (no divergent branch); the group's last lane stores it
        const float* om = &w.v[d::B + 3];
        const float th[3] = {om[0] * dt, om[1] * dt, om[2] * dt};
        // dq = (cos x, th sin(x) / (2x)) with x = |th| / 2.  For x < 1/2 both
        // factors are their Taylor series in x^2 to the x^8 term (truncation
        // below 3e-10), which needs neither the square root nor the sine.
        const float a2 = dot3(th, th), x2 = 0.25f * a2;
        float dq0, kq;
        if (x2 < 0.25f) {
            dq0 = 1.0f + x2 * (-0.5f + x2 * (1.0f / 24.0f + x2 * (-1.0f / 720.0f + x2 * (1.0f / 40320.0f))));
            kq = 0.5f + x2 * (-1.0f / 12.0f + x2 * (1.0f / 240.0f + x2 * (-1.0f / 10080.0f + x2 * (1.0f / 725760.0f))));
        } else {
            // the sine and cosine of x from the argument in half-turns,
            // x / pi, whose reduction is exact (no slow path for large
            // arguments); the division by pi adds one rounding of x
            const float ang = sqrtf(a2);
            float s, c;
            sincospif(0.5f * ang * 0.318309886183790672f, &s, &c);
            dq0 = c;
            kq = s / ang;
        }
        const float dq1 = th[0] * kq, dq2 = th[1] * kq, dq3 = th[2] * kq;
        float* qq = &w.q[d::B + 3];
        const float w0 = qq[0], x0 = qq[1], y0 = qq[2], z0 = qq[3];
        float nw = dq0 * w0 - dq1 * x0 - dq2 * y0 - dq3 * z0;
        float nx = dq0 * x0 + dq1 * w0 + dq2 * z0 - dq3 * y0;
        float ny = dq0 * y0 - dq1 * z0 + dq2 * w0 + dq3 * x0;
        float nz = dq0 * z0 + dq1 * y0 - dq2 * x0 + dq3 * w0;
        const float inv = rsqrtf(nw * nw + nx * nx + ny * ny + nz * nz);
        g.sync();  // every lane has read the old orientation
        if (g.sl == LPS - 1) {
            qq[0] = nw * inv;
            qq[1] = nx * inv;
            qq[2] = ny * inv;
            qq[3] = nz * inv;
        }
    }
#pragma unroll
    for (int c0 = 0; c0 < d::NV; c0 += LPS) {
        const int c = c0 + g.sl;
        if (c < d::NV) w.qd[c] = w.v[c];
        if (c < d::B + 3) w.q[c] += dt * w.v[c];
    }
    g.sync();
}

// coordinate k of the grasp-maintenance error p_L + p_R - 2 p_ball, squared,
// on the current FK
template <int NA>
__device__ __forceinline__ float grasp_coord(const WarpWS<NA>& w, int k) {
    using d = Dims<NA>;
    const float e = w.a1[NA - 1][k] + w.a1[2 * NA - 1][k] - 2.0f * w.q[d::B + k];
    return e * e;
}


}  // namespace mppi
