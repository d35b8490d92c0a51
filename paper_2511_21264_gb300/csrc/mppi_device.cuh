// Device side of the MPPI + contact-rollout path (sm_103a, FP32, CUDA cores).
//
// One warp simulates one sample.  The sample's articulated state, link frames,
// contact set and solver scratch live in the warp's slice of shared memory for
// all H steps; the scene model is staged once per CTA.  Lane roles inside a
// step:
//   - controls: lane j < nu draws its Gaussian from Philox4x32-10 (or reads
//     the explicit control);
//   - kinematics: lane 16a walks arm a's chain;
//   - collision: all 32 lanes over the candidate pairs, compacted with a
//     ballot in canonical pair order;
//   - dynamics: lane 16a + i owns link i of arm a (spatial inertia, composite
//     inertia, mass-matrix column, Newton-Euler bias force), lane 16a factors
//     the arm's (M + dt D) block, lane 15 handles the ball;
//   - contact rows: one lane per Jacobian row (half-solved by the Cholesky
//     factor), projected Gauss-Seidel by lane 0 in the factor's coordinates;
//   - integration: one lane per coordinate.
// The formulation (world-frame spatial algebra, composite-rigid-body mass
// matrix, recursive bias, half-solved contact rows) is independent of the
// FP64 oracle, which builds the same quantities from Jacobian definitions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mppi {

constexpr int MAXL = 7;    // joints per arm
constexpr int MAXB = 16;   // boxes
constexpr int MAXC = 16;   // contacts kept per step
constexpr int MAXR = 3 * MAXC;
constexpr unsigned FULL = 0xffffffffu;

// error word bits (device)
constexpr int ERRB_NONFINITE = 1;
constexpr int ERRB_CHOLESKY = 2;
constexpr int ERRB_TIMEOUT = 4;

struct __align__(16) DevLink {
    float FR[9];
    float Fp[3];
    float com[3];
    float mass;
    float I[6];  // inertia about the COM in link axes: xx yy zz xy xz yz
    float s0[3];
    float s1[3];
    float rcap, D, gear, tau_max;  // D = joint damping + servo gain (implicit)
    float u_lo, u_hi, gravcomp, pad;
};

struct __align__(16) DevModel {
    int na, nb, maxc, sweeps;
    float dt, mu, imp, erp;
    float g[3], floor_z;
    float rb, mb, Ib, pad0;
    float goal[3], w_goal;
    float w_u, w_pen, w_obst, w_grasp;
    float baseR[2][9];
    float basep[2][3];
    float box[MAXB][6];  // centre, half-extents
    DevLink link[2][MAXL];
};
static_assert(sizeof(DevModel) % 16 == 0, "model must stage with 16-byte copies");

template <int NA>
struct Dims {
    static constexpr int NL = 2 * NA, NV = 2 * NA + 6, NQ = 2 * NA + 7, NU = 2 * NA;
    static constexpr int NX = NQ + NV, B = 2 * NA;
};

// Per-warp (per-sample) workspace in shared memory.
template <int NA>
struct __align__(16) WarpWS {
    using d = Dims<NA>;
    float q[d::NQ + 1];
    float qd[d::NV];
    float v[d::NV];
    float vf[d::NV];
    float zz[d::NV];
    float rhs[d::NV];
    float u[d::NU];
    // kinematics, per link
    float R[d::NL][9];
    float z[d::NL][3];
    float o[d::NL][3];
    float c[d::NL][3];
    float a0[d::NL][3];
    float a1[d::NL][3];
    // dynamics
    float S[d::NL][6];
    float F[d::NL][6];
    float V[d::NL][6];
    float f[d::NL][6];
    float Isp[d::NL][10];
    float L[2][NA][NA];
    // contacts
    float cp[MAXC][3];
    float cn[MAXC][3];
    float cdep[MAXC];
    int cA[MAXC];
    int cB[MAXC];
    float Y[MAXR][d::NV];
    float lam[MAXR];
    float Rr[MAXR];
    float Ad[MAXR];
    float vs[MAXR];
    int ncon;
    int nact;
    float pen_all;
    float pen_box;
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

// Sampled control U[k,h,j] = clamp(u_nom[h,j] + sigma_j z, lo, hi) with z
// from counter (j/4, h, k, iteration).  Written with explicit rounding so the
// rollout and the update kernels regenerate identical values.
__device__ __forceinline__ float sample_control(uint2 key, uint32_t iter, int k, int h, int j, float unom,
                                                float sigma, float lo, float hi) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(j >> 2), (uint32_t)h, (uint32_t)k, iter), key);
    const float z = block_normal(w, j & 3);
    const float u = __fmaf_rn(sigma, z, unom);
    return fminf(fmaxf(u, lo), hi);
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
// kinematics: lane 16a walks arm a
// ---------------------------------------------------------------------------
template <int NA>
__device__ __forceinline__ void forward_kinematics(const DevModel& M, WarpWS<NA>& w, int lane) {
    if ((lane & 15) != 0) return;
    const int a = lane >> 4;
    float R[9], p[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = M.baseR[a][k];
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = M.basep[a][k];
#pragma unroll
    for (int i = 0; i < NA; ++i) {
        const DevLink& L = M.link[a][i];
        const int l = a * NA + i;
        w.z[l][0] = R[2];
        w.z[l][1] = R[5];
        w.z[l][2] = R[8];
        w.o[l][0] = p[0];
        w.o[l][1] = p[1];
        w.o[l][2] = p[2];
        float s, c;
        sincosf(w.q[a * NA + i], &s, &c);
        float Rj[9];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            Rj[3 * r + 0] = c * R[3 * r + 0] + s * R[3 * r + 1];
            Rj[3 * r + 1] = c * R[3 * r + 1] - s * R[3 * r + 0];
            Rj[3 * r + 2] = R[3 * r + 2];
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) p[r] += Rj[3 * r] * L.Fp[0] + Rj[3 * r + 1] * L.Fp[1] + Rj[3 * r + 2] * L.Fp[2];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                R[3 * r + cc] = Rj[3 * r] * L.FR[cc] + Rj[3 * r + 1] * L.FR[3 + cc] + Rj[3 * r + 2] * L.FR[6 + cc];
#pragma unroll
        for (int k = 0; k < 9; ++k) w.R[l][k] = R[k];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            w.c[l][r] = R[3 * r] * L.com[0] + R[3 * r + 1] * L.com[1] + R[3 * r + 2] * L.com[2] + p[r];
            w.a0[l][r] = R[3 * r] * L.s0[0] + R[3 * r + 1] * L.s0[1] + R[3 * r + 2] * L.s0[2] + p[r];
            w.a1[l][r] = R[3 * r] * L.s1[0] + R[3 * r + 1] * L.s1[1] + R[3 * r + 2] * L.s1[2] + p[r];
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

// Minimum of the box SDF along a capsule axis (convex in t): golden-section
// search over [0,1] with the end points as candidates.
__device__ __forceinline__ float capsule_box_t(const float* a, const float* d, const float* box) {
    const float gr = 0.6180339887498949f;
    float lo = 0.0f, hi = 1.0f;
    float x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
    float f1 = box_sdf_only(a, d, x1, box), f2 = box_sdf_only(a, d, x2, box);
#pragma unroll 1
    for (int it = 0; it < 34; ++it) {
        if (f1 <= f2) {
            hi = x2;
            x2 = x1;
            f2 = f1;
            x1 = hi - gr * (hi - lo);
            f1 = box_sdf_only(a, d, x1, box);
        } else {
            lo = x1;
            x1 = x2;
            f1 = f2;
            x2 = lo + gr * (hi - lo);
            f2 = box_sdf_only(a, d, x2, box);
        }
    }
    float t = 0.5f * (lo + hi);
    float ft = box_sdf_only(a, d, t, box);
    const float f0 = box_sdf_only(a, d, 0.0f, box), fe = box_sdf_only(a, d, 1.0f, box);
    if (f0 < ft) {
        t = 0.0f;
        ft = f0;
    }
    if (fe < ft) t = 1.0f;
    // Near an edge or vertex minimum the function is flat to second order,
    // so the search pins t only to ~sqrt(FP32 eps).  In such a region (two
    // or three slabs exceeded, fixed signs) the squared distance is the
    // quadratic sum_k (alpha_k + beta_k t)^2: take its exact minimiser if it
    // stays in the same region.
    {
        float al[3], be[3];
        int nact = 0;
        unsigned sig = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float xk = a[k] + t * d[k] - box[k];
            const float s = xk >= 0.0f ? 1.0f : -1.0f;
            const bool on = fabsf(xk) - box[3 + k] > 0.0f;
            nact += on;
            sig |= (on ? 1u : 0u) << (2 * k);
            sig |= (s > 0.0f ? 1u : 0u) << (2 * k + 1);
            al[k] = on ? s * (a[k] - box[k]) - box[3 + k] : 0.0f;
            be[k] = on ? s * d[k] : 0.0f;
        }
        if (nact >= 2) {
            const float den = be[0] * be[0] + be[1] * be[1] + be[2] * be[2];
            const float num = al[0] * be[0] + al[1] * be[1] + al[2] * be[2];
            if (den > 0.0f) {
                const float tq = fminf(fmaxf(-num / den, 0.0f), 1.0f);
                unsigned sq = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float xk = a[k] + tq * d[k] - box[k];
                    const bool on = fabsf(xk) - box[3 + k] > 0.0f;
                    sq |= (on ? 1u : 0u) << (2 * k);
                    sq |= (xk >= 0.0f ? 1u : 0u) << (2 * k + 1);
                }
                // compare only the exceeded slabs and their sides
                const unsigned m = ((sig & 0x15u) | ((sig & 0x15u) << 1));
                if ((sq & m) == (sig & m) && (sq & 0x15u) == (sig & 0x15u)) t = tq;
            }
        }
    }
    return t;
}

// All candidate pairs, 32 at a time across the warp, compacted in canonical
// order (ball-floor, ball-links, ball-boxes, links x boxes).
template <int NA>
__device__ __forceinline__ int collide(const DevModel& M, WarpWS<NA>& w, int lane) {
    using d = Dims<NA>;
    const int nb = M.nb;
    const int npairs = 1 + d::NL + nb + d::NL * nb;
    const float* pb = &w.q[d::B];
    const float rb = M.rb;
    int base = 0, exact = 0;
    float pa = 0.0f, pbox = 0.0f;
    for (int p0 = 0; p0 < npairs; p0 += 32) {
        const int p = p0 + lane;
        bool active = false, isbox = false;
        float dist = 1.0f, cp[3] = {0, 0, 0}, nn[3] = {0, 0, 1};
        int A = -1, Bb = -1;
        if (p < npairs) {
            if (p == 0) {  // ball - floor
                dist = (pb[2] - M.floor_z) - rb;
                cp[0] = pb[0];
                cp[1] = pb[1];
                cp[2] = 0.5f * ((pb[2] - rb) + M.floor_z);
                A = d::B;
            } else if (p < 1 + d::NL) {  // ball - link capsule
                const int l = p - 1;
                const float* a0 = w.a0[l];
                const float* a1 = w.a1[l];
                float dd[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
                float ac[3] = {pb[0] - a0[0], pb[1] - a0[1], pb[2] - a0[2]};
                const float den = dot3(dd, dd);
                float t = den > 0.0f ? dot3(ac, dd) / den : 0.0f;
                t = fminf(fmaxf(t, 0.0f), 1.0f);
                float s[3] = {a0[0] + t * dd[0], a0[1] + t * dd[1], a0[2] + t * dd[2]};
                float df[3] = {pb[0] - s[0], pb[1] - s[1], pb[2] - s[2]};
                const float len = sqrtf(dot3(df, df));
                if (len > 0.0f) {
                    const float il = 1.0f / len;
                    nn[0] = df[0] * il;
                    nn[1] = df[1] * il;
                    nn[2] = df[2] * il;
                }
                const float rc = M.link[l / NA][l % NA].rcap;
                dist = len - rb - rc;
#pragma unroll
                for (int k = 0; k < 3; ++k) cp[k] = 0.5f * ((pb[k] - rb * nn[k]) + (s[k] + rc * nn[k]));
                A = d::B;
                Bb = l;
            } else if (p < 1 + d::NL + nb) {  // ball - box
                const float* box = M.box[p - 1 - d::NL];
                float surf[3];
                dist = box_sdf(pb, box, nn, surf) - rb;
#pragma unroll
                for (int k = 0; k < 3; ++k) cp[k] = 0.5f * ((pb[k] - rb * nn[k]) + surf[k]);
                A = d::B;
                isbox = true;
            } else {  // link capsule - box
                const int idx = p - 1 - d::NL - nb;
                const int l = idx / nb, bi = idx - (idx / nb) * nb;
                const float* box = M.box[bi];
                const float* a0 = w.a0[l];
                const float* a1 = w.a1[l];
                const float rc = M.link[l / NA][l % NA].rcap;
                float dd[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
                // bounding-sphere cull (conservative)
                float mid[3] = {a0[0] + 0.5f * dd[0], a0[1] + 0.5f * dd[1], a0[2] + 0.5f * dd[2]};
                const float rad = 0.5f * sqrtf(dot3(dd, dd)) + rc;
                float lb2 = 0.0f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float e = fmaxf(fabsf(mid[k] - box[k]) - box[3 + k], 0.0f);
                    lb2 += e * e;
                }
                if (lb2 < rad * rad) {
                    ++exact;
                    const float t = capsule_box_t(a0, dd, box);
                    float x[3] = {a0[0] + t * dd[0], a0[1] + t * dd[1], a0[2] + t * dd[2]};
                    float surf[3];
                    dist = box_sdf(x, box, nn, surf) - rc;
#pragma unroll
                    for (int k = 0; k < 3; ++k) cp[k] = 0.5f * ((x[k] - rc * nn[k]) + surf[k]);
                    A = l;
                    isbox = true;
                }
            }
            active = dist < 0.0f;
        }
        const unsigned mask = __ballot_sync(FULL, active);
        if (active) {
            const int pos = base + __popc(mask & ((1u << lane) - 1u));
            pa += -dist;
            if (isbox) pbox += -dist;
            if (pos < M.maxc) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    w.cp[pos][k] = cp[k];
                    w.cn[pos][k] = nn[k];
                }
                w.cdep[pos] = -dist;
                w.cA[pos] = A;
                w.cB[pos] = Bb;
            }
        }
        base += __popc(mask);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        pa += __shfl_xor_sync(FULL, pa, off);
        pbox += __shfl_xor_sync(FULL, pbox, off);
    }
    if (lane == 0) {
        w.ncon = base < M.maxc ? base : M.maxc;
        w.nact = base;
        w.pen_all = pa;
        w.pen_box = pbox;
    }
    return exact;
}

// ---------------------------------------------------------------------------
// dynamics: free velocity vf = qd + dt (M + dt D)^-1 (tau_drive - c - D qd)
// ---------------------------------------------------------------------------
template <int NA>
__device__ __forceinline__ void dynamics(const DevModel& M, WarpWS<NA>& w, int lane, int* err) {
    using d = Dims<NA>;
    const int a = lane >> 4, i = lane & 15;
    const bool act = i < NA;
    const int l = a * NA + i;
    // (1) spatial inertia of each link about the world origin; joint axis
    if (act) {
        const DevLink& L = M.link[a][i];
        const float* R = w.R[l];
        const float* Ib = L.I;
        const float B9[9] = {Ib[0], Ib[3], Ib[4], Ib[3], Ib[1], Ib[5], Ib[4], Ib[5], Ib[2]};
        float T[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                T[3 * r + cc] = R[3 * r] * B9[cc] + R[3 * r + 1] * B9[3 + cc] + R[3 * r + 2] * B9[6 + cc];
        const float Ixx = T[0] * R[0] + T[1] * R[1] + T[2] * R[2];
        const float Iyy = T[3] * R[3] + T[4] * R[4] + T[5] * R[5];
        const float Izz = T[6] * R[6] + T[7] * R[7] + T[8] * R[8];
        const float Ixy = T[0] * R[3] + T[1] * R[4] + T[2] * R[5];
        const float Ixz = T[0] * R[6] + T[1] * R[7] + T[2] * R[8];
        const float Iyz = T[3] * R[6] + T[4] * R[7] + T[5] * R[8];
        const float* c = w.c[l];
        const float m = L.mass;
        const float cc2 = dot3(c, c);
        float* Is = w.Isp[l];
        Is[0] = m;
        Is[1] = m * c[0];
        Is[2] = m * c[1];
        Is[3] = m * c[2];
        Is[4] = Ixx + m * (cc2 - c[0] * c[0]);
        Is[5] = Iyy + m * (cc2 - c[1] * c[1]);
        Is[6] = Izz + m * (cc2 - c[2] * c[2]);
        Is[7] = Ixy - m * c[0] * c[1];
        Is[8] = Ixz - m * c[0] * c[2];
        Is[9] = Iyz - m * c[1] * c[2];
        float* S = w.S[l];
        S[0] = w.z[l][0];
        S[1] = w.z[l][1];
        S[2] = w.z[l][2];
        cross3(w.o[l], w.z[l], S + 3);
    }
    __syncwarp();
    // (2) composite inertia of the subtree (suffix sum) -> F_j = I^c_j S_j;
    //     spatial velocity V_i = sum_{k<=i} S_k qd_k
    if (act) {
        float Ic[10];
#pragma unroll
        for (int t = 0; t < 10; ++t) Ic[t] = 0.0f;
        for (int k = i; k < NA; ++k) {
            const float* Is = w.Isp[a * NA + k];
#pragma unroll
            for (int t = 0; t < 10; ++t) Ic[t] += Is[t];
        }
        spatial_inertia_apply(Ic, w.S[l], w.F[l]);
        float V[6] = {0, 0, 0, 0, 0, 0};
        for (int k = 0; k <= i; ++k) {
            const float qdk = w.qd[a * NA + k];
            const float* S = w.S[a * NA + k];
#pragma unroll
            for (int t = 0; t < 6; ++t) V[t] += S[t] * qdk;
        }
#pragma unroll
        for (int t = 0; t < 6; ++t) w.V[l][t] = V[t];
    }
    __syncwarp();
    // (3) mass-matrix column i: M[r][i] = S_r . F_i (r <= i);
    //     bias force f_i = I_i (A_i + a_g) + V_i x* (I_i V_i) with the
    //     velocity-product acceleration A_i = sum_{k<=i} V_{k-1} x (S_k qd_k)
    if (act) {
        const float* F = w.F[l];
        for (int r = 0; r <= i; ++r) {
            const float* S = w.S[a * NA + r];
            const float mv = S[0] * F[0] + S[1] * F[1] + S[2] * F[2] + S[3] * F[3] + S[4] * F[4] + S[5] * F[5];
            w.L[a][r][i] = mv;
            w.L[a][i][r] = mv;
        }
        float Aa[6] = {0, 0, 0, 0, 0, 0};
        for (int k = 1; k <= i; ++k) {
            const float* Vp = w.V[a * NA + k - 1];
            const float qdk = w.qd[a * NA + k];
            const float* Sk = w.S[a * NA + k];
            float s[6];
#pragma unroll
            for (int t = 0; t < 6; ++t) s[t] = Sk[t] * qdk;
            float t1[3], t2[3], t3[3];
            cross3(Vp, s, t1);
            cross3(Vp, s + 3, t2);
            cross3(Vp + 3, s, t3);
            Aa[0] += t1[0];
            Aa[1] += t1[1];
            Aa[2] += t1[2];
            Aa[3] += t2[0] + t3[0];
            Aa[4] += t2[1] + t3[1];
            Aa[5] += t2[2] + t3[2];
        }
        const float gw = 1.0f - M.link[a][i].gravcomp;
        Aa[3] -= gw * M.g[0];
        Aa[4] -= gw * M.g[1];
        Aa[5] -= gw * M.g[2];
        const float* Is = w.Isp[l];
        const float* V = w.V[l];
        float IA[6], IV[6];
        spatial_inertia_apply(Is, Aa, IA);
        spatial_inertia_apply(Is, V, IV);
        float n1[3], n2[3], f1[3];
        cross3(V, IV, n1);
        cross3(V + 3, IV + 3, n2);
        cross3(V, IV + 3, f1);
        float* f = w.f[l];
        f[0] = IA[0] + n1[0] + n2[0];
        f[1] = IA[1] + n1[1] + n2[1];
        f[2] = IA[2] + n1[2] + n2[2];
        f[3] = IA[3] + f1[0];
        f[4] = IA[4] + f1[1];
        f[5] = IA[5] + f1[2];
    }
    __syncwarp();
    // (4) bias torque = S_i . (sum of subtree forces); drive; implicit damping
    if (act) {
        float Ff[6] = {0, 0, 0, 0, 0, 0};
        for (int k = i; k < NA; ++k) {
            const float* f = w.f[a * NA + k];
#pragma unroll
            for (int t = 0; t < 6; ++t) Ff[t] += f[t];
        }
        const float* S = w.S[l];
        const float tb = S[0] * Ff[0] + S[1] * Ff[1] + S[2] * Ff[2] + S[3] * Ff[3] + S[4] * Ff[4] + S[5] * Ff[5];
        const DevLink& L = M.link[a][i];
        const int dof = a * NA + i;
        const float td = fminf(fmaxf(L.gear * w.u[dof], -L.tau_max), L.tau_max);
        w.rhs[dof] = td - tb - L.D * w.qd[dof];
        w.L[a][i][i] += M.dt * L.D;
    }
    __syncwarp();
    // (5) Cholesky of each arm block and the free velocity; ball
    if (i == 0) {
        float (*Lm)[NA] = w.L[a];
        bool ok = true;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            float s = Lm[j][j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= Lm[j][k] * Lm[j][k];
            // a NaN pivot comes from a non-finite state (reported as such
            // through the cost); only a finite non-positive pivot is a loss
            // of positive definiteness
            ok = ok && !(s <= 0.0f);
            const float dj = sqrtf(s);
            const float inv = 1.0f / dj;
            Lm[j][j] = dj;
#pragma unroll
            for (int r = j + 1; r < NA; ++r) {
                float t = Lm[r][j];
#pragma unroll
                for (int k = 0; k < j; ++k) t -= Lm[r][k] * Lm[j][k];
                Lm[r][j] = t * inv;
            }
        }
        float y[NA];
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            float s = w.rhs[a * NA + r];
#pragma unroll
            for (int k = 0; k < r; ++k) s -= Lm[r][k] * y[k];
            y[r] = s / Lm[r][r];
        }
#pragma unroll
        for (int r = NA - 1; r >= 0; --r) {
            float s = y[r];
#pragma unroll
            for (int k = r + 1; k < NA; ++k) s -= Lm[k][r] * y[k];
            y[r] = s / Lm[r][r];
        }
#pragma unroll
        for (int r = 0; r < NA; ++r) w.vf[a * NA + r] = w.qd[a * NA + r] + M.dt * y[r];
        if (!ok) atomicOr(err, ERRB_CHOLESKY);
    }
    if (lane == 15) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            w.vf[d::B + r] = w.qd[d::B + r] + M.dt * M.g[r];
            w.vf[d::B + 3 + r] = w.qd[d::B + 3 + r];
        }
    }
    __syncwarp();
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
    float ev[3] = {0, 0, 0};
    ev[ia] = 1.0f;
    float t1[3];
    cross3(n, ev, t1);
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

template <int NA>
__device__ __forceinline__ void add_body_row(const DevModel& M, const WarpWS<NA>& w, int body, float sgn,
                                             const float* e, const float* p, float* y) {
    using d = Dims<NA>;
    if (body < 0) return;
    if (body == d::B) {
        const float* c = &w.q[d::B];
        float dd[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
        float de[3];
        cross3(dd, e, de);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            y[d::B + r] += sgn * e[r];
            y[d::B + 3 + r] += sgn * de[r];
        }
        return;
    }
    const int a = body / NA, i = body - a * NA;
    for (int k = 0; k <= i; ++k) {
        const int l = a * NA + k;
        float dd[3] = {p[0] - w.o[l][0], p[1] - w.o[l][1], p[2] - w.o[l][2]};
        float col[3];
        cross3(w.z[l], dd, col);
        y[a * NA + k] += sgn * dot3(e, col);
    }
}

template <int NA>
__device__ __forceinline__ void contacts(const DevModel& M, WarpWS<NA>& w, int lane) {
    using d = Dims<NA>;
    const int nc = w.ncon;
    if (nc == 0) {
        if (lane < d::NV) w.v[lane] = w.vf[lane];
        __syncwarp();
        return;
    }
    const float smb = sqrtf(M.mb), sIb = sqrtf(M.Ib);
    // z_f = L^T v_f
    if ((lane & 15) == 0) {
        const int a = lane >> 4;
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            float s = 0.0f;
#pragma unroll
            for (int k = i; k < NA; ++k) s += w.L[a][k][i] * w.vf[a * NA + k];
            w.zz[a * NA + i] = s;
        }
    }
    if (lane == 15) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            w.zz[d::B + r] = smb * w.vf[d::B + r];
            w.zz[d::B + 3 + r] = sIb * w.vf[d::B + 3 + r];
        }
    }
    const int nr = 3 * nc;
    const float regc = (1.0f - M.imp) / M.imp;
    for (int r = lane; r < nr; r += 32) {
        const int c = r / 3, k = r - 3 * (r / 3);
        float e[3];
        contact_frame_row<NA>(w.cn[c], k, e);
        float* y = w.Y[r];
#pragma unroll
        for (int t = 0; t < d::NV; ++t) y[t] = 0.0f;
        add_body_row<NA>(M, w, w.cA[c], 1.0f, e, w.cp[c], y);
        add_body_row<NA>(M, w, w.cB[c], -1.0f, e, w.cp[c], y);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            float t[NA];
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                float s = y[a * NA + i];
#pragma unroll
                for (int kk = 0; kk < i; ++kk) s -= w.L[a][i][kk] * t[kk];
                t[i] = s / w.L[a][i][i];
            }
#pragma unroll
            for (int i = 0; i < NA; ++i) y[a * NA + i] = t[i];
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            y[d::B + t] /= smb;
            y[d::B + 3 + t] /= sIb;
        }
        float A = 0.0f;
#pragma unroll
        for (int t = 0; t < d::NV; ++t) A += y[t] * y[t];
        const float R = regc * A;
        w.Rr[r] = R;
        w.Ad[r] = A + R;
        w.vs[r] = (k == 0) ? (M.erp / M.dt) * w.cdep[c] : 0.0f;
        w.lam[r] = 0.0f;
    }
    __syncwarp();
    if (lane == 0) {
        float z[d::NV];
#pragma unroll
        for (int t = 0; t < d::NV; ++t) z[t] = w.zz[t];
        for (int s = 0; s < M.sweeps; ++s) {
            for (int c = 0; c < nc; ++c) {
                const int rn = 3 * c;
                const float* yn = w.Y[rn];
                float res = w.Rr[rn] * w.lam[rn] - w.vs[rn];
#pragma unroll
                for (int t = 0; t < d::NV; ++t) res += yn[t] * z[t];
                const float ln = fmaxf(w.lam[rn] - res / w.Ad[rn], 0.0f);
                const float dn = ln - w.lam[rn];
                w.lam[rn] = ln;
#pragma unroll
                for (int t = 0; t < d::NV; ++t) z[t] += yn[t] * dn;
                const float* y1 = w.Y[rn + 1];
                const float* y2 = w.Y[rn + 2];
                float r1 = w.Rr[rn + 1] * w.lam[rn + 1], r2 = w.Rr[rn + 2] * w.lam[rn + 2];
#pragma unroll
                for (int t = 0; t < d::NV; ++t) {
                    r1 += y1[t] * z[t];
                    r2 += y2[t] * z[t];
                }
                float l1 = w.lam[rn + 1] - r1 / w.Ad[rn + 1];
                float l2 = w.lam[rn + 2] - r2 / w.Ad[rn + 2];
                const float nrm = sqrtf(l1 * l1 + l2 * l2), lim = M.mu * ln;
                if (nrm > lim) {
                    const float sc = nrm > 0.0f ? lim / nrm : 0.0f;
                    l1 *= sc;
                    l2 *= sc;
                }
                const float d1 = l1 - w.lam[rn + 1], d2 = l2 - w.lam[rn + 2];
                w.lam[rn + 1] = l1;
                w.lam[rn + 2] = l2;
#pragma unroll
                for (int t = 0; t < d::NV; ++t) z[t] += y1[t] * d1 + y2[t] * d2;
            }
        }
#pragma unroll
        for (int t = 0; t < d::NV; ++t) w.zz[t] = z[t];
    }
    __syncwarp();
    // v = L^-T z
    if ((lane & 15) == 0) {
        const int a = lane >> 4;
        float t[NA];
#pragma unroll
        for (int i = NA - 1; i >= 0; --i) {
            float s = w.zz[a * NA + i];
#pragma unroll
            for (int k = i + 1; k < NA; ++k) s -= w.L[a][k][i] * t[k];
            t[i] = s / w.L[a][i][i];
        }
#pragma unroll
        for (int i = 0; i < NA; ++i) w.v[a * NA + i] = t[i];
    }
    if (lane == 15) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            w.v[d::B + r] = w.zz[d::B + r] / smb;
            w.v[d::B + 3 + r] = w.zz[d::B + 3 + r] / sIb;
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// semi-implicit Euler
// ---------------------------------------------------------------------------
template <int NA>
__device__ __forceinline__ void integrate(const DevModel& M, WarpWS<NA>& w, int lane) {
    using d = Dims<NA>;
    const float dt = M.dt;
    if (lane == 31) {
        const float* om = &w.v[d::B + 3];
        const float th[3] = {om[0] * dt, om[1] * dt, om[2] * dt};
        const float ang = sqrtf(dot3(th, th));
        float dq0 = 1.0f, dq1 = 0.0f, dq2 = 0.0f, dq3 = 0.0f;
        if (ang > 0.0f) {
            float s, c;
            sincosf(0.5f * ang, &s, &c);
            const float k = s / ang;
            dq0 = c;
            dq1 = th[0] * k;
            dq2 = th[1] * k;
            dq3 = th[2] * k;
        }
        float* qq = &w.q[d::B + 3];
        const float w0 = qq[0], x0 = qq[1], y0 = qq[2], z0 = qq[3];
        float nw = dq0 * w0 - dq1 * x0 - dq2 * y0 - dq3 * z0;
        float nx = dq0 * x0 + dq1 * w0 + dq2 * z0 - dq3 * y0;
        float ny = dq0 * y0 - dq1 * z0 + dq2 * w0 + dq3 * x0;
        float nz = dq0 * z0 + dq1 * y0 - dq2 * x0 + dq3 * w0;
        const float inv = rsqrtf(nw * nw + nx * nx + ny * ny + nz * nz);
        qq[0] = nw * inv;
        qq[1] = nx * inv;
        qq[2] = ny * inv;
        qq[3] = nz * inv;
    }
    if (lane < d::NV) w.qd[lane] = w.v[lane];
    if (lane < d::B + 3) w.q[lane] += dt * w.v[lane];
    __syncwarp();
}

// grasp-maintenance term || p_L + p_R - 2 p_ball ||^2 on the current FK
template <int NA>
__device__ __forceinline__ float grasp_term(const WarpWS<NA>& w) {
    using d = Dims<NA>;
    const float* pl = w.a1[NA - 1];
    const float* pr = w.a1[2 * NA - 1];
    const float* pb = &w.q[d::B];
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float e = pl[k] + pr[k] - 2.0f * pb[k];
        s += e * e;
    }
    return s;
}

}  // namespace mppi
