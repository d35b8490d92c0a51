// QP smoothing projection (Eq. 5): each sampled joint-velocity sequence is
// moved to the nearest sequence (in the 2-norm) whose position, velocity,
// acceleration and jerk (r = 0..3, Sec. III) stay within their bounds.
//
// Solver: a fixed number of ADMM iterations (the paper names none), one
// thread per sequence.  The iteration is run in the coordinates
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

    for (int it = 0; it < iters; ++it) {
        // forward sweep: rows at t, right-hand side, forward substitution
        float x0 = 0.0f;                         // x_t (x_0 and earlier are zero)
        float d1p = 0.0f, d2p = 0.0f;            // first and second differences at t-1
        float r0 = 0.0f, r1 = 0.0f, r2 = 0.0f;   // rhs of x_{t-2}, x_{t-1}, x_t
        float z1 = 0.0f, z2 = 0.0f, z3 = 0.0f;   // z_{i-1}, z_{i-2}, z_{i-3} of the substitution
        for (int t = 0; t < H; ++t) {
            const float2 xv = xb[(size_t)t * T];
            float4 y = yv[(size_t)t * T];
            const float xp1 = xv.x;
            const float d1 = xp1 - x0, d2 = d1 - d1p, d3 = d2 - d2p;
            const float eP = qp_row(s0 * xp1, y.x, Plo, Phi, rs0);
            const float eV = qp_row(s1 * d1, y.y, Vlo, Vhi, rs1);
            const float eA = qp_row(s2 * d2, y.z, t == 0 ? A0lo : Alo, t == 0 ? A0hi : Ahi, rs2);
            float eJ = 0.0f;
            if (t >= 1) eJ = qp_row(s3 * d3, y.w, t == 1 ? J1lo : Jlo, t == 1 ? J1hi : Jhi, rs3);
            yv[(size_t)t * T] = y;
            // row t touches x_{t+1} (+1), x_t (-1, -2, -3), x_{t-1} (+1, +3), x_{t-2} (-1)
            const float r3 = xv.y + eP + eV + eA + eJ;
            r2 = r2 - eV - 2.0f * eA - 3.0f * eJ;
            r1 = r1 + eA + 3.0f * eJ;
            r0 = r0 - eJ;
            if (t >= 3) {  // x_{t-2} is complete: substitute (index i = t-2, slot t-3)
                const float4 L = __ldg(&bf[t - 3]);
                const float z = (r0 - L.y * z1 - L.z * z2 - L.w * z3) * L.x;
                xb[(size_t)(t - 3) * T].x = z;
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
            const float4 L = __ldg(&bf[i - 1]);
            const float z = (r - L.y * z1 - L.z * z2 - L.w * z3) * L.x;
            xb[(size_t)(i - 1) * T].x = z;
            z3 = z2;
            z2 = z1;
            z1 = z;
        }
        // backward substitution L^T x = z
        float p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;  // x_{i+1}, x_{i+2}, x_{i+3}
        for (int i = H; i >= 1; --i) {
            const float4 L = __ldg(&bb[i - 1]);
            float* slot = &xb[(size_t)(i - 1) * T].x;
            const float xi = (*slot - L.y * p1 - L.z * p2 - L.w * p3) * L.x;
            *slot = xi;
            p3 = p2;
            p2 = p1;
            p1 = xi;
        }
    }
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
    const QPClass c = a.cls[cls];
    const float q = a.q0[a.q_per_seq ? i : cls], qd = a.qd0[a.q_per_seq ? i : cls];
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
            vt = a.vin[base_in + (long long)h * a.i_h];
        } else {  // sample (k = mem, joint j = cls): the values the rollout's sampler draws, unclamped
            const int j = cls, k = mem;
            float v = a.u_nom[h * a.nu + j];
            if (a.Lfac) {
                const float* Lr = a.Lfac + ((size_t)h * a.nu + j) * a.nu;
                for (int jb = 0; 4 * jb <= j; ++jb) {
                    const uint4 w = philox4x32_10(make_uint4((uint32_t)jb, (uint32_t)h, (uint32_t)k, iter), key);
                    for (int t = 0; t < 4 && 4 * jb + t <= j; ++t) v = __fmaf_rn(Lr[4 * jb + t], block_normal(w, t), v);
                }
            } else {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)(j >> 2), (uint32_t)h, (uint32_t)k, iter), key);
                v = __fmaf_rn(a.sigma[j], block_normal(w, j & 3), v);
            }
            vt = v;
        }
        acc += vt;
        if (h > 0) xb[(size_t)(h - 1) * T].y = prev - vt;
        xb[(size_t)h * T].x = acc;
        yv[(size_t)h * T] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        prev = vt;
    }
    xb[(size_t)(a.H - 1) * T].y = prev;
    qp_admm(c, a.band + (size_t)cls * 2 * a.H, a.H, a.iters, a.dt, q, qd, xb, yv, T);
    const long long base_out = (long long)mem * a.o_a + (long long)cls * a.o_b;
    float xp = 0.0f;
    for (int h = 0; h < a.H; ++h) {
        const float x = xb[(size_t)h * T].x;
        a.out[base_out + (long long)h * a.o_h] = x - xp;
        xp = x;
    }
}

// 24 H bytes of shared memory per thread: 64 threads per CTA while that
// stays within 100 KB (two CTAs per SM), else one warp.
int qp_threads(int H) { return (size_t)H * 64 * (sizeof(float4) + sizeof(float2)) <= 100 * 1024 ? 64 : 32; }
size_t qp_smem_bytes(int H) { return (size_t)H * qp_threads(H) * (sizeof(float4) + sizeof(float2)); }

int launch_qp(const QPArgs& a, cudaStream_t s) {
    if (a.n <= 0) return MPPI_OK;
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
    std::vector<float4> band(2 * (size_t)H);
    const double scd[4] = {c.s[0], c.s[1], c.s[2], c.s[3]};
    rc = qp_band_factor(H, rho, scd, band.data());
    if (rc != MPPI_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the class record and band live in one stream-ordered scratch block
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
    if (e == cudaSuccess) rc = launch_qp(a, s);
    else rc = MPPI_ERR_CUDA;
    cudaFreeAsync(d, s);
    return rc;
}
