/*
 * FP64 CPU oracle for the MPPI + contact-rollout path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the GPU path computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg load it.  It shares no code, header,
 * table or constant generator with the CUDA path; both parse the same scene
 * blob (an input) with their own code.
 *
 * What it computes (paper: Alg. 1 and Eq. 8; the simulator is the fixed
 * MuJoCo-style model of two revolute arms, a free ball, boxes and a floor):
 *   - forward kinematics by composing joint transforms link by link;
 *   - the joint-space mass matrix by its definition
 *       M = sum_i m_i Jv_i^T Jv_i + Jw_i^T I_i Jw_i       (no recursion);
 *   - the bias force by its definition, the body accelerations at zero
 *     joint acceleration projected through the body Jacobians
 *       c = sum_i m_i Jv_i^T (dJv_i qd) + Jw_i^T (I_i dJw_i qd + w_i x I_i w_i)
 *           - sum_i (1 - gravcomp_i) m_i Jv_i^T g ;
 *     a textbook recursive Newton-Euler routine is kept as a second route
 *     for the tests only;
 *   - narrow phase: sphere-plane, sphere-capsule, sphere-box and
 *     capsule-box, every pair tested exactly (no culling);
 *   - the step: free velocity from a dense Cholesky solve of
 *     (M + dt D) where D holds the joint damping and the velocity-servo
 *     gain (treated implicitly, as MuJoCo's Euler integrator treats joint
 *     damping), then projected Gauss-Seidel on the contact impulses with
 *     the dense Delassus matrix A = J (M + dt D)^-1 J^T, soft regularisation
 *     R = (1-d)/d diag(A) and reference velocity ERP/dt * depth, then
 *     semi-implicit Euler;
 *   - Philox4x32-10 (Salmon et al., SC'11) and Box-Muller normals;
 *   - the MPPI iteration: sample, roll out, stage costs, softmax weights at
 *     temperature lambda (log-sum-exp), weighted mean of the samples
 *     (Eq. 8a/8d with eta = 1 and the elite set equal to all samples).
 *
 * Parity status: every function here is pinned by the CPU tests (closed
 * forms, invariants, brute force, published Philox answers) except the
 * capsule-box contact point on exactly flat minima (a tie; the oracle takes
 * the midpoint of the minimising interval), whose depth alone is pinned.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXL 7
#define OR_MAXB 16
#define OR_MAXC 16
#define OR_MAXNV 20
#define OR_MAXNQ 21
#define OR_MAXR (3 * OR_MAXC)
#define OR_FACE_TIE 1e-5   /* m: face distances this close count as tied */

typedef struct {
    double FR[9], Fp[3];
    double mass, com[3], I[9];
    double s0[3], s1[3], rcap;
    double damping, kv, gear, tau_max, u_lo, u_hi, gravcomp;
} or_link;

typedef struct {
    int na, nb, maxc, sweeps, nq, nv, nu;
    double dt, mu, imp, erp, g[3], floor_z, rb, mb, Ib, goal[3];
    double w_goal, w_u, w_pen, w_obst, w_grasp;
    double baseR[2][9], basep[2][3];
    or_link L[2][OR_MAXL];
    double bc[OR_MAXB][3], bh[OR_MAXB][3];
    double x0[OR_MAXNQ + OR_MAXNV];
} or_model;

/* --------------------------------------------------------------------- */
/* small vector helpers                                                   */
/* --------------------------------------------------------------------- */
static void v3_cross(const double *a, const double *b, double *o) {
    double t0 = a[1] * b[2] - a[2] * b[1];
    double t1 = a[2] * b[0] - a[0] * b[2];
    double t2 = a[0] * b[1] - a[1] * b[0];
    o[0] = t0; o[1] = t1; o[2] = t2;
}
static double v3_dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void v3_sub(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double v3_norm(const double *a) { return sqrt(v3_dot(a, a)); }
static void m3_mul(const double *A, const double *B, double *C) { /* C = A B, row-major */
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
    memcpy(C, T, sizeof T);
}
static void m3_vec(const double *A, const double *x, double *y) {
    double t[3];
    for (int i = 0; i < 3; i++) t[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
    memcpy(y, t, sizeof t);
}
static void rot_z(double q, double *R) {
    double c = cos(q), s = sin(q);
    double T[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
    memcpy(R, T, sizeof T);
}

/* --------------------------------------------------------------------- */
/* model blob                                                             */
/* --------------------------------------------------------------------- */
int or_model_size(void) { return (int)sizeof(or_model); }

/* Parse a scene blob (layout documented with the scene generator).
 * Returns 0 on success, a negative code on a malformed blob. */
int or_model_parse(const void *blob, size_t len, or_model *m) {
    const unsigned char *b = (const unsigned char *)blob;
    if (!blob || len < 16) return -1;
    uint32_t h[4];
    memcpy(h, b, 16);
    if (h[0] != 0x4950504Du || h[1] != 1u) return -2;
    size_t n = h[2];
    if (len < 16 + 8 * n || n < 23) return -3;
    const double *v = (const double *)(b + 16);
    double tmp[1024];
    if (n > 1024) return -3;
    memcpy(tmp, v, 8 * n);
    v = tmp;
    memset(m, 0, sizeof *m);
    m->na = (int)v[0]; m->nb = (int)v[1]; m->maxc = (int)v[2];
    if (m->na < 1 || m->na > OR_MAXL || m->nb < 0 || m->nb > OR_MAXB || m->maxc < 1 || m->maxc > OR_MAXC) return -4;
    m->dt = v[3]; m->sweeps = (int)v[4]; m->mu = v[5]; m->imp = v[6]; m->erp = v[7];
    m->g[0] = v[8]; m->g[1] = v[9]; m->g[2] = v[10]; m->floor_z = v[11];
    m->rb = v[12]; m->mb = v[13]; m->Ib = v[14];
    m->goal[0] = v[15]; m->goal[1] = v[16]; m->goal[2] = v[17];
    m->w_goal = v[18]; m->w_u = v[19]; m->w_pen = v[20]; m->w_obst = v[21]; m->w_grasp = v[22];
    m->nq = 2 * m->na + 7; m->nv = 2 * m->na + 6; m->nu = 2 * m->na;
    size_t need = 23 + 2 * (12 + 39 * (size_t)m->na) + 6 * (size_t)m->nb + (size_t)(m->nq + m->nv);
    if (n != need) return -5;
    size_t o = 23;
    for (int a = 0; a < 2; a++) {
        memcpy(m->baseR[a], v + o, 9 * 8); o += 9;
        memcpy(m->basep[a], v + o, 3 * 8); o += 3;
        for (int i = 0; i < m->na; i++) {
            or_link *L = &m->L[a][i];
            memcpy(L->FR, v + o, 72); o += 9;
            memcpy(L->Fp, v + o, 24); o += 3;
            L->mass = v[o++];
            memcpy(L->com, v + o, 24); o += 3;
            memcpy(L->I, v + o, 72); o += 9;
            memcpy(L->s0, v + o, 24); o += 3;
            memcpy(L->s1, v + o, 24); o += 3;
            L->rcap = v[o++]; L->damping = v[o++]; L->kv = v[o++]; L->gear = v[o++];
            L->tau_max = v[o++]; L->u_lo = v[o++]; L->u_hi = v[o++]; L->gravcomp = v[o++];
        }
    }
    for (int k = 0; k < m->nb; k++) {
        memcpy(m->bc[k], v + o, 24); o += 3;
        memcpy(m->bh[k], v + o, 24); o += 3;
    }
    memcpy(m->x0, v + o, 8 * (size_t)(m->nq + m->nv));
    return 0;
}

/* --------------------------------------------------------------------- */
/* forward kinematics                                                     */
/* --------------------------------------------------------------------- */
typedef struct {
    double R[2][OR_MAXL][9];   /* link frame rotation (world)            */
    double p[2][OR_MAXL][3];   /* link frame origin (world)              */
    double z[2][OR_MAXL][3];   /* joint axis (world)                     */
    double o[2][OR_MAXL][3];   /* a point on the joint axis (world)      */
    double c[2][OR_MAXL][3];   /* COM (world)                            */
    double a0[2][OR_MAXL][3];  /* capsule end points (world)             */
    double a1[2][OR_MAXL][3];
    double Iw[2][OR_MAXL][9];  /* inertia about COM in world axes        */
} or_fk;

static void xform_point(const double *R, const double *p, const double *x, double *y) {
    m3_vec(R, x, y);
    y[0] += p[0]; y[1] += p[1]; y[2] += p[2];
}

/* Link i frame = T_{i-1} Rz(q_i) F_i; joint i axis = z axis of T_{i-1}. */
void or_forward_kinematics(const or_model *m, const double *q, or_fk *f) {
    for (int a = 0; a < 2; a++) {
        double R[9], p[3];
        memcpy(R, m->baseR[a], sizeof R);
        memcpy(p, m->basep[a], sizeof p);
        for (int i = 0; i < m->na; i++) {
            const or_link *L = &m->L[a][i];
            f->z[a][i][0] = R[2]; f->z[a][i][1] = R[5]; f->z[a][i][2] = R[8];
            memcpy(f->o[a][i], p, sizeof p);
            double Rz[9], Rj[9], t[3];
            rot_z(q[a * m->na + i], Rz);
            m3_mul(R, Rz, Rj);
            m3_vec(Rj, L->Fp, t);
            p[0] += t[0]; p[1] += t[1]; p[2] += t[2];
            m3_mul(Rj, L->FR, R);
            memcpy(f->R[a][i], R, sizeof R);
            memcpy(f->p[a][i], p, sizeof p);
            xform_point(R, p, L->com, f->c[a][i]);
            xform_point(R, p, L->s0, f->a0[a][i]);
            xform_point(R, p, L->s1, f->a1[a][i]);
            double RI[9], Rt[9];
            for (int r = 0; r < 3; r++)
                for (int s = 0; s < 3; s++) Rt[3 * r + s] = R[3 * s + r];
            m3_mul(R, L->I, RI);
            m3_mul(RI, Rt, f->Iw[a][i]);
        }
    }
}

/* Translational Jacobian (3 x nv, row-major) of a world point moving with
 * link i of arm a: column j (j <= i, same arm) = z_j x (p - o_j). */
static void point_jacobian_link(const or_model *m, const or_fk *f, int a, int i, const double *pt, double *J) {
    int nv = m->nv;
    memset(J, 0, sizeof(double) * 3 * nv);
    for (int j = 0; j <= i; j++) {
        double d[3], col[3];
        v3_sub(pt, f->o[a][j], d);
        v3_cross(f->z[a][j], d, col);
        int dof = a * m->na + j;
        J[dof] = col[0]; J[nv + dof] = col[1]; J[2 * nv + dof] = col[2];
    }
}

/* Translational Jacobian of a point fixed on the ball: v + w x (p - c). */
static void point_jacobian_ball(const or_model *m, const double *ball_c, const double *pt, double *J) {
    int nv = m->nv, b0 = 2 * m->na;
    memset(J, 0, sizeof(double) * 3 * nv);
    double d[3];
    v3_sub(pt, ball_c, d);
    for (int r = 0; r < 3; r++) J[r * nv + b0 + r] = 1.0;
    /* w x d = -d x w : rows of -[d]x */
    J[0 * nv + b0 + 3] = 0.0;   J[0 * nv + b0 + 4] = d[2];  J[0 * nv + b0 + 5] = -d[1];
    J[1 * nv + b0 + 3] = -d[2]; J[1 * nv + b0 + 4] = 0.0;   J[1 * nv + b0 + 5] = d[0];
    J[2 * nv + b0 + 3] = d[1];  J[2 * nv + b0 + 4] = -d[0]; J[2 * nv + b0 + 5] = 0.0;
}

/* --------------------------------------------------------------------- */
/* mass matrix and bias by definition                                     */
/* --------------------------------------------------------------------- */
void or_mass_matrix(const or_model *m, const double *q, double *M) {
    int nv = m->nv, na = m->na;
    or_fk f;
    or_forward_kinematics(m, q, &f);
    memset(M, 0, sizeof(double) * nv * nv);
    double Jv[3 * OR_MAXNV], Jw[3 * OR_MAXNV];
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < na; i++) {
            point_jacobian_link(m, &f, a, i, f.c[a][i], Jv);
            memset(Jw, 0, sizeof Jw);
            for (int j = 0; j <= i; j++)
                for (int r = 0; r < 3; r++) Jw[r * nv + a * na + j] = f.z[a][j][r];
            const double *I = f.Iw[a][i];
            double mass = m->L[a][i].mass;
            for (int r = 0; r < nv; r++)
                for (int s = 0; s < nv; s++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += mass * Jv[k * nv + r] * Jv[k * nv + s];
                    for (int k = 0; k < 3; k++)
                        for (int l = 0; l < 3; l++) acc += Jw[k * nv + r] * I[3 * k + l] * Jw[l * nv + s];
                    M[r * nv + s] += acc;
                }
        }
    int b0 = 2 * na;
    for (int r = 0; r < 3; r++) M[(b0 + r) * nv + b0 + r] = m->mb;
    for (int r = 3; r < 6; r++) M[(b0 + r) * nv + b0 + r] = m->Ib;
}

/* Bias c(q, qd): Coriolis/centrifugal plus gravity (links without gravity
 * compensation and the ball).  Uses dJv qd and dJw qd written out from the
 * time derivative of the Jacobian columns:
 *   d/dt [z_j x (p - o_j)] = dz_j x (p - o_j) + z_j x (dp - do_j),
 *   dz_j = w_{j-1} x z_j (axis j is fixed in the body before joint j),
 *   do_j = velocity of o_j as a point of that body. */
void or_bias(const or_model *m, const double *q, const double *qd, double *c) {
    int nv = m->nv, na = m->na;
    or_fk f;
    or_forward_kinematics(m, q, &f);
    memset(c, 0, sizeof(double) * nv);
    double Jv[3 * OR_MAXNV];
    for (int a = 0; a < 2; a++) {
        const double *qda = qd + a * na;
        double wprev[OR_MAXL + 1][3];  /* wprev[j] = angular velocity of body carrying axis j */
        double dz[OR_MAXL][3], doj[OR_MAXL][3];
        memset(wprev, 0, sizeof wprev);
        for (int j = 0; j < na; j++) {
            v3_cross(wprev[j], f.z[a][j], dz[j]);
            /* velocity of o_j: sum over l<j of z_l x (o_j - o_l) qd_l */
            doj[j][0] = doj[j][1] = doj[j][2] = 0.0;
            for (int l = 0; l < j; l++) {
                double d[3], t[3];
                v3_sub(f.o[a][j], f.o[a][l], d);
                v3_cross(f.z[a][l], d, t);
                for (int r = 0; r < 3; r++) doj[j][r] += t[r] * qda[l];
            }
            for (int r = 0; r < 3; r++) wprev[j + 1][r] = wprev[j][r] + f.z[a][j][r] * qda[j];
        }
        for (int i = 0; i < na; i++) {
            const double *ci = f.c[a][i];
            /* COM velocity */
            double dc[3] = {0, 0, 0};
            for (int l = 0; l <= i; l++) {
                double d[3], t[3];
                v3_sub(ci, f.o[a][l], d);
                v3_cross(f.z[a][l], d, t);
                for (int r = 0; r < 3; r++) dc[r] += t[r] * qda[l];
            }
            double accv[3] = {0, 0, 0}, accw[3] = {0, 0, 0};
            for (int j = 0; j <= i; j++) {
                double d[3], t1[3], t2[3], dd[3];
                v3_sub(ci, f.o[a][j], d);
                v3_cross(dz[j], d, t1);
                v3_sub(dc, doj[j], dd);
                v3_cross(f.z[a][j], dd, t2);
                for (int r = 0; r < 3; r++) {
                    accv[r] += qda[j] * (t1[r] + t2[r]);
                    accw[r] += qda[j] * dz[j][r];
                }
            }
            const double *I = f.Iw[a][i];
            const double *w = wprev[i + 1];
            double Iacc[3], Iw_[3], gyro[3], mom[3];
            m3_vec(I, accw, Iacc);
            m3_vec(I, w, Iw_);
            v3_cross(w, Iw_, gyro);
            for (int r = 0; r < 3; r++) mom[r] = Iacc[r] + gyro[r];
            double mass = m->L[a][i].mass;
            double gw = 1.0 - m->L[a][i].gravcomp;
            double force[3];
            for (int r = 0; r < 3; r++) force[r] = mass * accv[r] - gw * mass * m->g[r];
            point_jacobian_link(m, &f, a, i, ci, Jv);
            for (int s = 0; s < nv; s++) {
                c[s] += Jv[s] * force[0] + Jv[nv + s] * force[1] + Jv[2 * nv + s] * force[2];
            }
            /* angular part: Jw column j = z_j */
            for (int j = 0; j <= i; j++) c[a * na + j] += v3_dot(f.z[a][j], mom);
        }
    }
    int b0 = 2 * na;
    for (int r = 0; r < 3; r++) c[b0 + r] = -m->mb * m->g[r];
    /* isotropic ball: w x (I w) = 0 */
}

/* Textbook recursive Newton-Euler (world-frame vectors), second route for
 * the tests: tau = M qdd + c.  Forward pass: angular velocity/acceleration
 * and COM acceleration of each link; backward pass: force and moment about
 * each joint point, projected on the joint axis.  Gravity enters as a base
 * acceleration -g for links without gravity compensation. */
void or_rnea(const or_model *m, const double *q, const double *qd, const double *qdd, double *tau) {
    int na = m->na, nv = m->nv;
    or_fk f;
    or_forward_kinematics(m, q, &f);
    for (int a = 0; a < 2; a++) {
        double w[OR_MAXL][3], dw[OR_MAXL][3], ao[OR_MAXL][3], ac[OR_MAXL][3], ac_nog[OR_MAXL][3];
        double wp[3] = {0, 0, 0}, dwp[3] = {0, 0, 0}, aop[3] = {0, 0, 0}, op[3];
        memcpy(op, f.o[a][0], sizeof op);
        for (int i = 0; i < na; i++) {
            int dof = a * na + i;
            const double *z = f.z[a][i];
            /* acceleration of o_i as a point of the previous body */
            double d[3], t[3], t2[3];
            v3_sub(f.o[a][i], op, d);
            double aoi[3];
            v3_cross(dwp, d, t);
            v3_cross(wp, d, t2);
            double t3[3];
            v3_cross(wp, t2, t3);
            for (int r = 0; r < 3; r++) aoi[r] = aop[r] + t[r] + t3[r];
            double wi[3], dwi[3], wz[3];
            for (int r = 0; r < 3; r++) wi[r] = wp[r] + z[r] * qd[dof];
            v3_cross(wp, z, wz);
            for (int r = 0; r < 3; r++) dwi[r] = dwp[r] + z[r] * qdd[dof] + wz[r] * qd[dof];
            double dc[3];
            v3_sub(f.c[a][i], f.o[a][i], dc);
            double u1[3], u2[3], u3[3];
            v3_cross(dwi, dc, u1);
            v3_cross(wi, dc, u2);
            v3_cross(wi, u2, u3);
            for (int r = 0; r < 3; r++) ac[i][r] = aoi[r] + u1[r] + u3[r];
            memcpy(w[i], wi, sizeof wi);
            memcpy(dw[i], dwi, sizeof dwi);
            memcpy(ao[i], aoi, sizeof aoi);
            memcpy(wp, wi, sizeof wi);
            memcpy(dwp, dwi, sizeof dwi);
            memcpy(aop, aoi, sizeof aoi);
            memcpy(op, f.o[a][i], sizeof op);
            (void)ac_nog;
        }
        double fn[3] = {0, 0, 0}, nn[3] = {0, 0, 0};
        double onext[3] = {0, 0, 0};
        for (int i = na - 1; i >= 0; i--) {
            double mass = m->L[a][i].mass, gw = 1.0 - m->L[a][i].gravcomp;
            double F[3];
            for (int r = 0; r < 3; r++) F[r] = mass * (ac[i][r] - gw * m->g[r]);
            double Iw_[3], Idw[3], gyro[3], N[3];
            m3_vec(f.Iw[a][i], w[i], Iw_);
            m3_vec(f.Iw[a][i], dw[i], Idw);
            v3_cross(w[i], Iw_, gyro);
            for (int r = 0; r < 3; r++) N[r] = Idw[r] + gyro[r];
            /* moment about o_i */
            double dc[3], mF[3], mchild[3] = {0, 0, 0};
            v3_sub(f.c[a][i], f.o[a][i], dc);
            v3_cross(dc, F, mF);
            if (i < na - 1) {
                double d[3];
                v3_sub(onext, f.o[a][i], d);
                v3_cross(d, fn, mchild);
            }
            double ni[3];
            for (int r = 0; r < 3; r++) ni[r] = N[r] + mF[r] + nn[r] + mchild[r];
            double fi[3];
            for (int r = 0; r < 3; r++) fi[r] = F[r] + fn[r];
            tau[a * na + i] = v3_dot(f.z[a][i], ni);
            memcpy(fn, fi, sizeof fi);
            memcpy(nn, ni, sizeof ni);
            memcpy(onext, f.o[a][i], sizeof onext);
        }
    }
    int b0 = 2 * na;
    for (int r = 0; r < 3; r++) tau[b0 + r] = m->mb * (qdd[b0 + r] - m->g[r]);
    for (int r = 3; r < 6; r++) tau[b0 + r] = m->Ib * qdd[b0 + r];
    (void)nv;
}

/* --------------------------------------------------------------------- */
/* narrow phase                                                           */
/* --------------------------------------------------------------------- */
typedef struct {
    double dist;      /* signed distance (negative = penetration)          */
    double p[3];      /* contact point: midpoint of the two witnesses      */
    double n[3];      /* unit normal from body B to body A                 */
    int bodyA, bodyB; /* body ids: arm a link i -> a*na+i, ball -> 2na,
                         static -> -1                                      */
    int box;          /* box index for box pairs, -1 otherwise             */
} or_contact;

static void closest_on_segment(const double *a, const double *b, const double *c, double *s, double *tout) {
    double d[3], ac[3];
    v3_sub(b, a, d);
    v3_sub(c, a, ac);
    double dd = v3_dot(d, d);
    double t = dd > 0.0 ? v3_dot(ac, d) / dd : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    for (int r = 0; r < 3; r++) s[r] = a[r] + t * d[r];
    if (tout) *tout = t;
}

void or_sphere_plane(double cz, double r, double h, double *dist) { *dist = (cz - h) - r; }

/* sphere (centre c, radius r) vs capsule (segment a-b, radius rc).
 * Normal from the capsule to the sphere; degenerate centre-on-axis -> +z. */
void or_sphere_capsule(const double *c, double r, const double *a, const double *b, double rc,
                       double *dist, double *p, double *n) {
    double s[3], d[3];
    closest_on_segment(a, b, c, s, NULL);
    v3_sub(c, s, d);
    double len = v3_norm(d);
    if (len > 0.0) { n[0] = d[0] / len; n[1] = d[1] / len; n[2] = d[2] / len; }
    else { n[0] = 0.0; n[1] = 0.0; n[2] = 1.0; }
    *dist = len - r - rc;
    for (int k = 0; k < 3; k++) p[k] = 0.5 * ((c[k] - r * n[k]) + (s[k] + rc * n[k]));
}

/* Signed distance from point x to an axis-aligned box, its outward normal
 * and the closest surface point.  Inside: nearest face, faces within 1e-5 m
 * of the nearest are tied, ties -> lowest axis, + face before - face. */
void or_box_sdf(const double *x, const double *bc, const double *bh, double *sdf, double *n, double *surf) {
    double q[3], cl[3];
    int inside = 1;
    for (int k = 0; k < 3; k++) {
        double lo = bc[k] - bh[k], hi = bc[k] + bh[k];
        cl[k] = x[k] < lo ? lo : (x[k] > hi ? hi : x[k]);
        q[k] = x[k] - cl[k];
        if (x[k] < lo || x[k] > hi) inside = 0;
    }
    if (!inside) {
        double len = v3_norm(q);
        *sdf = len;
        for (int k = 0; k < 3; k++) n[k] = q[k] / len;
        memcpy(surf, cl, sizeof cl);
        return;
    }
    /* nearest face; faces within OR_FACE_TIE of the nearest count as tied
     * (the deepest point of a segment crossing a box lies where two faces
     * are equidistant), ties -> lowest axis, + face before - face */
    double fd[6], best = INFINITY;
    for (int k = 0; k < 3; k++) {
        fd[2 * k] = (bc[k] + bh[k]) - x[k];      /* distance to + face */
        fd[2 * k + 1] = x[k] - (bc[k] - bh[k]);  /* distance to - face */
        if (fd[2 * k] < best) best = fd[2 * k];
        if (fd[2 * k + 1] < best) best = fd[2 * k + 1];
    }
    int f = 0;
    while (fd[f] > best + OR_FACE_TIE) f++;
    int ax = f / 2, sg = (f % 2) ? -1 : 1;
    *sdf = -best;
    n[0] = n[1] = n[2] = 0.0;
    n[ax] = (double)sg;
    memcpy(surf, x, 3 * sizeof(double));
    surf[ax] = bc[ax] + sg * bh[ax];
}

void or_sphere_box(const double *c, double r, const double *bc, const double *bh,
                   double *dist, double *p, double *n) {
    double sdf, surf[3];
    or_box_sdf(c, bc, bh, &sdf, n, surf);
    *dist = sdf - r;
    for (int k = 0; k < 3; k++) p[k] = 0.5 * ((c[k] - r * n[k]) + surf[k]);
}

static double seg_box_f(const double *a, const double *d, double t, const double *bc, const double *bh) {
    double x[3] = {a[0] + t * d[0], a[1] + t * d[1], a[2] + t * d[2]};
    double sdf, n[3], s[3];
    or_box_sdf(x, bc, bh, &sdf, n, s);
    return sdf;
}

/* capsule (segment a-b, radius rc) vs box: minimise the box's signed
 * distance (a convex function) along the segment by golden-section search,
 * then take the midpoint of the set where it is within 1e-12 of the minimum
 * (found by bisection on each side) so flat minima give a unique point. */
void or_capsule_box(const double *a, const double *b, double rc, const double *bc, const double *bh,
                    double *dist, double *p, double *n, double *tstar) {
    double d[3];
    v3_sub(b, a, d);
    const double gr = (sqrt(5.0) - 1.0) / 2.0;
    double lo = 0.0, hi = 1.0;
    double x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
    double f1 = seg_box_f(a, d, x1, bc, bh), f2 = seg_box_f(a, d, x2, bc, bh);
    for (int it = 0; it < 200 && (hi - lo) > 1e-14; it++) {
        if (f1 <= f2) { hi = x2; x2 = x1; f2 = f1; x1 = hi - gr * (hi - lo); f1 = seg_box_f(a, d, x1, bc, bh); }
        else { lo = x1; x1 = x2; f1 = f2; x2 = lo + gr * (hi - lo); f2 = seg_box_f(a, d, x2, bc, bh); }
    }
    double tm = 0.5 * (lo + hi);
    /* the end points are candidates too (golden section never evaluates them) */
    double fm = seg_box_f(a, d, tm, bc, bh);
    double f0 = seg_box_f(a, d, 0.0, bc, bh), fe = seg_box_f(a, d, 1.0, bc, bh);
    if (f0 < fm) { tm = 0.0; fm = f0; }
    if (fe < fm) { tm = 1.0; fm = fe; }
    const double tol = 1e-12;
    /* left edge of the minimising set */
    double l0 = 0.0, l1 = tm;
    if (seg_box_f(a, d, 0.0, bc, bh) <= fm + tol) l1 = 0.0;
    else for (int it = 0; it < 100; it++) { double mid = 0.5 * (l0 + l1); if (seg_box_f(a, d, mid, bc, bh) <= fm + tol) l1 = mid; else l0 = mid; }
    double r0 = tm, r1 = 1.0;
    if (seg_box_f(a, d, 1.0, bc, bh) <= fm + tol) r0 = 1.0;
    else for (int it = 0; it < 100; it++) { double mid = 0.5 * (r0 + r1); if (seg_box_f(a, d, mid, bc, bh) <= fm + tol) r0 = mid; else r1 = mid; }
    double t = 0.5 * (l1 + r0);
    double x[3] = {a[0] + t * d[0], a[1] + t * d[1], a[2] + t * d[2]};
    double sdf, surf[3];
    or_box_sdf(x, bc, bh, &sdf, n, surf);
    *dist = sdf - rc;
    for (int k = 0; k < 3; k++) p[k] = 0.5 * ((x[k] - rc * n[k]) + surf[k]);
    if (tstar) *tstar = t;
}

/* All pairs in canonical order: ball-floor; ball-link (left links, then
 * right links); ball-box; link-box (link-major, box-minor).  Every pair is
 * written to `all` (with its distance); the active ones (dist < 0) in order
 * are copied to `act` up to the model's contact cap.  Also returns the total
 * penetration over all active pairs and over the box pairs alone. */
int or_collide(const or_model *m, const or_fk *f, const double *ballp, or_contact *all, int *nall,
               or_contact *act, int *nact, double *pen_all, double *pen_box) {
    int na = m->na, k = 0, ballid = 2 * na;
    double pa = 0.0, pb = 0.0;
    /* ball - floor */
    {
        or_contact *c = &all[k++];
        or_sphere_plane(ballp[2], m->rb, m->floor_z, &c->dist);
        c->n[0] = 0; c->n[1] = 0; c->n[2] = 1;
        c->p[0] = ballp[0]; c->p[1] = ballp[1];
        c->p[2] = 0.5 * ((ballp[2] - m->rb) + m->floor_z);
        c->bodyA = ballid; c->bodyB = -1; c->box = -1;
    }
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < na; i++) {
            or_contact *c = &all[k++];
            or_sphere_capsule(ballp, m->rb, f->a0[a][i], f->a1[a][i], m->L[a][i].rcap, &c->dist, c->p, c->n);
            c->bodyA = ballid; c->bodyB = a * na + i; c->box = -1;
        }
    for (int b = 0; b < m->nb; b++) {
        or_contact *c = &all[k++];
        or_sphere_box(ballp, m->rb, m->bc[b], m->bh[b], &c->dist, c->p, c->n);
        c->bodyA = ballid; c->bodyB = -1; c->box = b;
    }
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < na; i++)
            for (int b = 0; b < m->nb; b++) {
                or_contact *c = &all[k++];
                or_capsule_box(f->a0[a][i], f->a1[a][i], m->L[a][i].rcap, m->bc[b], m->bh[b], &c->dist, c->p, c->n, NULL);
                c->bodyA = a * na + i; c->bodyB = -1; c->box = b;
            }
    int na_ = 0;
    for (int j = 0; j < k; j++) {
        if (all[j].dist < 0.0) {
            pa += -all[j].dist;
            if (all[j].box >= 0) pb += -all[j].dist;
            if (na_ < m->maxc) act[na_++] = all[j];
        }
    }
    if (nall) *nall = k;
    *nact = na_;
    *pen_all = pa;
    *pen_box = pb;
    return 0;
}

/* Smallest |signed distance| over all candidate pairs at state x (used to
 * keep parity scenes away from contact activation boundaries). */
double or_min_abs_dist(const or_model *m, const double *x) {
    or_fk f;
    or_forward_kinematics(m, x, &f);
    or_contact all[1 + 2 * OR_MAXL + OR_MAXB + 2 * OR_MAXL * OR_MAXB], act[OR_MAXC];
    int nall, nact;
    double pa, pb;
    or_collide(m, &f, x + 2 * m->na, all, &nall, act, &nact, &pa, &pb);
    double best = INFINITY;
    for (int j = 0; j < nall; j++) if (fabs(all[j].dist) < best) best = fabs(all[j].dist);
    return best;
}

/* Contact frame rows: n, t1 = normalise(n x e) with e the world axis of
 * smallest |n.e| (ties -> lowest index), t2 = n x t1. */
static void contact_frame(const double *n, double *t1, double *t2) {
    int e = 0;
    double best = fabs(n[0]);
    if (fabs(n[1]) < best) { best = fabs(n[1]); e = 1; }
    if (fabs(n[2]) < best) { e = 2; }
    double ev[3] = {0, 0, 0};
    ev[e] = 1.0;
    v3_cross(n, ev, t1);
    double l = v3_norm(t1);
    t1[0] /= l; t1[1] /= l; t1[2] /= l;
    v3_cross(n, t1, t2);
}

/* --------------------------------------------------------------------- */
/* dense linear algebra                                                   */
/* --------------------------------------------------------------------- */
/* In-place Cholesky of an n x n SPD matrix (lower triangle).  Returns 0 or
 * -1 when a pivot is not positive. */
static int cholesky(double *A, int n) {
    for (int j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (int k = 0; k < j; k++) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return -1;
        double d = sqrt(s);
        A[j * n + j] = d;
        for (int i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (int k = 0; k < j; k++) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / d;
        }
    }
    return 0;
}
static void chol_solve(const double *L, int n, double *x) {
    for (int i = 0; i < n; i++) {
        double s = x[i];
        for (int k = 0; k < i; k++) s -= L[i * n + k] * x[k];
        x[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (int k = i + 1; k < n; k++) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

/* --------------------------------------------------------------------- */
/* one simulator step                                                     */
/* --------------------------------------------------------------------- */
typedef struct {
    int ncon;        /* active contacts used (capped)            */
    int nactive;     /* active pairs before the cap              */
    double pen_all;  /* sum of depths over active pairs          */
    double pen_box;  /* ... over box pairs                       */
    int chol_fail;
} or_step_info;

static void quat_mul(const double *a, const double *b, double *o) {
    double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    o[0] = w; o[1] = x; o[2] = y; o[3] = z;
}

/* x = (q, qd) -> x_out after one step of dt with controls u (nu).
 * Optionally returns the impulses (3 per contact) and the contacts. */
int or_step_ex(const or_model *m, const double *x, const double *u, double *xo, or_step_info *info,
               double *lambda_out, or_contact *con_out) {
    int na = m->na, nq = m->nq, nv = m->nv, b0 = 2 * na;
    const double *q = x, *qd = x + nq;
    double dt = m->dt;
    or_fk f;
    or_forward_kinematics(m, q, &f);
    or_contact all[1 + 2 * OR_MAXL + OR_MAXB + 2 * OR_MAXL * OR_MAXB];
    or_contact act[OR_MAXC];
    int nall, nc;
    double pen_all, pen_box;
    or_collide(m, &f, q + b0, all, &nall, act, &nc, &pen_all, &pen_box);

    double M[OR_MAXNV * OR_MAXNV], c[OR_MAXNV];
    or_mass_matrix(m, q, M);
    or_bias(m, q, qd, c);
    /* actuation and implicit damping: tau_drive = clamp(gear*u, +-tau_max),
       D = damping + kv on the arm joints */
    double rhs[OR_MAXNV];
    for (int s = 0; s < nv; s++) rhs[s] = -c[s];
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < na; i++) {
            const or_link *L = &m->L[a][i];
            int dof = a * na + i;
            double td = L->gear * u[dof];
            if (td > L->tau_max) td = L->tau_max;
            if (td < -L->tau_max) td = -L->tau_max;
            double D = L->damping + L->kv;
            rhs[dof] += td - D * qd[dof];
            M[dof * nv + dof] += dt * D;
        }
    if (cholesky(M, nv) != 0) {
        if (info) info->chol_fail = 1;
        return -1;
    }
    double vf[OR_MAXNV];
    memcpy(vf, rhs, sizeof(double) * nv);
    chol_solve(M, nv, vf);
    for (int s = 0; s < nv; s++) vf[s] = qd[s] + dt * vf[s];

    double v[OR_MAXNV];
    memcpy(v, vf, sizeof(double) * nv);
    double lam[OR_MAXR];
    memset(lam, 0, sizeof lam);
    if (nc > 0) {
        int nr = 3 * nc;
        static __thread double J[OR_MAXR * OR_MAXNV], X[OR_MAXNV * OR_MAXR], A[OR_MAXR * OR_MAXR];
        double JA[3 * OR_MAXNV], JB[3 * OR_MAXNV];
        for (int ci = 0; ci < nc; ci++) {
            const or_contact *cc = &act[ci];
            double t1[3], t2[3];
            contact_frame(cc->n, t1, t2);
            const double *rows[3] = {cc->n, t1, t2};
            memset(JA, 0, sizeof JA);
            memset(JB, 0, sizeof JB);
            if (cc->bodyA == b0) point_jacobian_ball(m, q + b0, cc->p, JA);
            else if (cc->bodyA >= 0) point_jacobian_link(m, &f, cc->bodyA / na, cc->bodyA % na, cc->p, JA);
            if (cc->bodyB == b0) point_jacobian_ball(m, q + b0, cc->p, JB);
            else if (cc->bodyB >= 0) point_jacobian_link(m, &f, cc->bodyB / na, cc->bodyB % na, cc->p, JB);
            for (int r = 0; r < 3; r++)
                for (int s = 0; s < nv; s++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += rows[r][k] * (JA[k * nv + s] - JB[k * nv + s]);
                    J[(3 * ci + r) * nv + s] = acc;
                }
        }
        /* X = (M + dt D)^-1 J^T, column by column */
        for (int r = 0; r < nr; r++) {
            double col[OR_MAXNV];
            for (int s = 0; s < nv; s++) col[s] = J[r * nv + s];
            chol_solve(M, nv, col);
            for (int s = 0; s < nv; s++) X[s * nr + r] = col[s];
        }
        for (int r = 0; r < nr; r++)
            for (int s = 0; s < nr; s++) {
                double acc = 0.0;
                for (int k = 0; k < nv; k++) acc += J[r * nv + k] * X[k * nr + s];
                A[r * nr + s] = acc;
            }
        double b[OR_MAXR], R[OR_MAXR], vstar[OR_MAXR];
        for (int r = 0; r < nr; r++) {
            double acc = 0.0;
            for (int k = 0; k < nv; k++) acc += J[r * nv + k] * vf[k];
            b[r] = acc;
            R[r] = (1.0 - m->imp) / m->imp * A[r * nr + r];
            vstar[r] = 0.0;
        }
        for (int ci = 0; ci < nc; ci++) vstar[3 * ci] = m->erp / dt * (-act[ci].dist);
        for (int sw = 0; sw < m->sweeps; sw++) {
            for (int ci = 0; ci < nc; ci++) {
                int in = 3 * ci;
                /* normal row */
                double res = b[in] + R[in] * lam[in] - vstar[in];
                for (int s = 0; s < nr; s++) res += A[in * nr + s] * lam[s];
                double ln = lam[in] - res / (A[in * nr + in] + R[in]);
                lam[in] = ln > 0.0 ? ln : 0.0;
                /* tangent rows, jointly, then the friction disk */
                double rt[2];
                for (int tr = 0; tr < 2; tr++) {
                    int it = in + 1 + tr;
                    double acc = b[it] + R[it] * lam[it];
                    for (int s = 0; s < nr; s++) acc += A[it * nr + s] * lam[s];
                    rt[tr] = acc;
                }
                double l1 = lam[in + 1] - rt[0] / (A[(in + 1) * nr + in + 1] + R[in + 1]);
                double l2 = lam[in + 2] - rt[1] / (A[(in + 2) * nr + in + 2] + R[in + 2]);
                double nrm = sqrt(l1 * l1 + l2 * l2), lim = m->mu * lam[in];
                if (nrm > lim) {
                    double sc = nrm > 0.0 ? lim / nrm : 0.0;
                    l1 *= sc; l2 *= sc;
                }
                lam[in + 1] = l1;
                lam[in + 2] = l2;
            }
        }
        for (int s = 0; s < nv; s++) {
            double acc = 0.0;
            for (int r = 0; r < nr; r++) acc += X[s * nr + r] * lam[r];
            v[s] = vf[s] + acc;
        }
    }
    /* semi-implicit Euler */
    double *qo = xo, *qdo = xo + nq;
    for (int s = 0; s < nv; s++) qdo[s] = v[s];
    for (int j = 0; j < 2 * na; j++) qo[j] = q[j] + dt * v[j];
    for (int r = 0; r < 3; r++) qo[b0 + r] = q[b0 + r] + dt * v[b0 + r];
    const double *w = v + b0 + 3;
    double th[3] = {w[0] * dt, w[1] * dt, w[2] * dt};
    double ang = v3_norm(th);
    double dq[4] = {1.0, 0.0, 0.0, 0.0};
    if (ang > 0.0) {
        double s = sin(0.5 * ang) / ang;
        dq[0] = cos(0.5 * ang); dq[1] = th[0] * s; dq[2] = th[1] * s; dq[3] = th[2] * s;
    }
    double qn[4];
    quat_mul(dq, q + b0 + 3, qn);
    double qnn = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
    for (int r = 0; r < 4; r++) qo[b0 + 3 + r] = qn[r] / qnn;
    if (info) {
        info->ncon = nc; info->pen_all = pen_all; info->pen_box = pen_box; info->chol_fail = 0;
        int cnt = 0;
        for (int j = 0; j < nall; j++) cnt += all[j].dist < 0.0;
        info->nactive = cnt;
    }
    if (lambda_out) memcpy(lambda_out, lam, sizeof(double) * 3 * nc);
    if (con_out) memcpy(con_out, act, sizeof(or_contact) * nc);
    return 0;
}

int or_step(const or_model *m, const double *x, const double *u, double *xo, or_step_info *info) {
    return or_step_ex(m, x, u, xo, info, NULL, NULL);
}

/* Stage cost of step h: position terms on x_{h+1}, control effort on u_h,
 * penetration detected during step h. */
double or_stage_cost(const or_model *m, const double *x_next, const double *u, const or_step_info *info) {
    int na = m->na, b0 = 2 * na;
    const double *pb = x_next + b0;
    double dg = 0.0;
    for (int r = 0; r < 3; r++) dg += (pb[r] - m->goal[r]) * (pb[r] - m->goal[r]);
    double uu = 0.0;
    for (int j = 0; j < m->nu; j++) uu += u[j] * u[j];
    double c = m->w_goal * dg + m->w_u * uu + m->w_pen * info->pen_all + m->w_obst * info->pen_box;
    if (m->w_grasp != 0.0) {
        or_fk f;
        or_forward_kinematics(m, x_next, &f);
        double s = 0.0;
        for (int r = 0; r < 3; r++) {
            double e = f.a1[0][na - 1][r] + f.a1[1][na - 1][r] - 2.0 * pb[r];
            s += e * e;
        }
        c += m->w_grasp * s;
    }
    return c;
}

/* Roll out H steps from x with controls U (H x nu); returns the summed
 * stage cost.  Optionally stores the H+1 states. */
double or_rollout(const or_model *m, const double *x, const double *U, int H, double *traj) {
    int nx = m->nq + m->nv;
    double cur[OR_MAXNQ + OR_MAXNV], nxt[OR_MAXNQ + OR_MAXNV];
    memcpy(cur, x, sizeof(double) * nx);
    if (traj) memcpy(traj, x, sizeof(double) * nx);
    double cost = 0.0;
    for (int h = 0; h < H; h++) {
        or_step_info info;
        if (or_step(m, cur, U + (size_t)h * m->nu, nxt, &info) != 0) return NAN;
        cost += or_stage_cost(m, nxt, U + (size_t)h * m->nu, &info);
        memcpy(cur, nxt, sizeof(double) * nx);
        if (traj) memcpy(traj + (size_t)(h + 1) * nx, cur, sizeof(double) * nx);
    }
    return cost;
}

/* --------------------------------------------------------------------- */
/* Philox4x32-10 and Gaussian samples                                     */
/* --------------------------------------------------------------------- */
/* Ten rounds of the Philox-4x32 bijection (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): each round
 * multiplies words 0 and 2 by the round constants, mixes the high halves
 * with words 1/3 and the key, and the key is bumped by the Weyl constants
 * between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from the top 23 bits: ((x >> 9) + 1/2) 2^-23.  Never 0
 * or 1, and exactly representable in FP32 as well as FP64, so an FP32
 * implementation draws the very same uniforms. */
static double u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Four standard normals from one Philox block by Box-Muller on the word
 * pairs (0,1) and (2,3): z0 = r cos(2 pi u1), z1 = r sin(2 pi u1). */
void or_normals4(const uint32_t w[4], double z[4]) {
    const double two_pi = 6.283185307179586476925286766559;
    double r01 = sqrt(-2.0 * log(u01(w[0]))), a01 = two_pi * u01(w[1]);
    double r23 = sqrt(-2.0 * log(u01(w[2]))), a23 = two_pi * u01(w[3]);
    z[0] = r01 * cos(a01); z[1] = r01 * sin(a01);
    z[2] = r23 * cos(a23); z[3] = r23 * sin(a23);
}

/* Noise eps[k][h][j] = sigma_j z with z from Philox(key = seed, counter =
 * (j / 4, h, k, iteration)), word j % 4. */
void or_noise(uint64_t seed, uint64_t iteration, int K, int H, int nu, const double *sigma, double *eps) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int k = 0; k < K; k++)
        for (int h = 0; h < H; h++)
            for (int jb = 0; jb < (nu + 3) / 4; jb++) {
                uint32_t ctr[4] = {(uint32_t)jb, (uint32_t)h, (uint32_t)k, (uint32_t)iteration};
                uint32_t w[4];
                double z[4];
                or_philox4x32_10(ctr, key, w);
                or_normals4(w, z);
                for (int t = 0; t < 4; t++) {
                    int j = 4 * jb + t;
                    if (j < nu) eps[((size_t)k * H + h) * nu + j] = sigma[j] * z[t];
                }
            }
}

/* --------------------------------------------------------------------- */
/* MPPI                                                                   */
/* --------------------------------------------------------------------- */
/* Eq. 8a/8d with eta = 1, all samples as the elite set and beta = lambda:
 * s_k = exp(-(c_k - c_min)/lambda) (the shift cancels in the ratio; it is
 * the log-sum-exp form), non-finite costs get weight 0.  Returns 0, or 1
 * when no cost is finite (u_out = u_nom). */
int or_mppi_update(int K, int H, int nu, const double *costs, const double *U, double lambda,
                   const double *u_nom, double *u_out, double *weights_out) {
    double cmin = INFINITY;
    for (int k = 0; k < K; k++) if (isfinite(costs[k]) && costs[k] < cmin) cmin = costs[k];
    if (!isfinite(cmin)) {
        memcpy(u_out, u_nom, sizeof(double) * H * nu);
        return 1;
    }
    double Z = 0.0;
    double *w = (double *)malloc(sizeof(double) * K);
    for (int k = 0; k < K; k++) {
        w[k] = isfinite(costs[k]) ? exp(-(costs[k] - cmin) / lambda) : 0.0;
        Z += w[k];
    }
    for (int i = 0; i < H * nu; i++) {
        double acc = 0.0;
        for (int k = 0; k < K; k++) acc += w[k] * U[(size_t)k * H * nu + i];
        u_out[i] = acc / Z;
    }
    if (weights_out) for (int k = 0; k < K; k++) weights_out[k] = w[k] / Z;
    free(w);
    return 0;
}

double or_rollout_task(const or_model *m, const double *task, const double *x, const double *U, int H,
                       double *traj_out, double *terms);

typedef struct {
    const or_model *m;
    const double *task; /* NULL: the scene's stage cost; else the ball-task suite */
    const double *x;
    const double *U;
    int H, k0, k1;
    double *costs;
} rollout_job;

static void *rollout_worker(void *arg) {
    rollout_job *j = (rollout_job *)arg;
    size_t stride = (size_t)j->H * j->m->nu;
    for (int k = j->k0; k < j->k1; k++) {
        const double *Uk = j->U + (size_t)k * stride;
        j->costs[k] = j->task ? or_rollout_task(j->m, j->task, j->x, Uk, j->H, NULL, NULL)
                              : or_rollout(j->m, j->x, Uk, j->H, NULL);
    }
    return NULL;
}

/* K rollouts from one state, samples split into contiguous chunks over
 * `nthreads` host threads (each cost is computed alone, so the split does
 * not change any result). */
static void rollout_many_from(const or_model *m, const double *task, const double *x, const double *U, int K,
                              int H, double *costs, int nthreads) {
    pthread_t th[256];
    rollout_job jobs[256];
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    int per = (K + nthreads - 1) / nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; t++) {
        jobs[t].m = m; jobs[t].task = task; jobs[t].x = x; jobs[t].U = U; jobs[t].H = H;
        jobs[t].k0 = t * per; jobs[t].k1 = (t + 1) * per < K ? (t + 1) * per : K;
        jobs[t].costs = costs;
        if (jobs[t].k0 >= jobs[t].k1) break;
        if (nthreads == 1) { rollout_worker(&jobs[t]); started = 0; break; }
        pthread_create(&th[t], NULL, rollout_worker, &jobs[t]);
        started++;
    }
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
}

/* Roll out K control sequences from one state (or from K states when
 * per_sample_state != 0) on `nthreads` host threads. */
void or_rollout_many(const or_model *m, const double *x, int per_sample_state, const double *U, int K, int H,
                     double *costs, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (per_sample_state) {
        /* per-sample start states: run serially over samples in chunks */
        int nx = m->nq + m->nv;
        for (int k = 0; k < K; k++) costs[k] = or_rollout(m, x + (size_t)k * nx, U + (size_t)k * H * m->nu, H, NULL);
        return;
    }
    rollout_many_from(m, NULL, x, U, K, H, costs, nthreads);
}

/* The same K rollouts costed by the ball-task suite (Sec. IV-B) instead of
 * the scene's stage cost. */
void or_rollout_task_many(const or_model *m, const double *task, const double *x, const double *U, int K, int H,
                          double *costs, int nthreads) {
    rollout_many_from(m, task, x, U, K, H, costs, nthreads);
}

/* One MPPI iteration (Alg. 1, one pass of the loop without the QP and with
 * the full sample set as elite set): samples U_k = clamp(u_nom + eps_k),
 * roll out, cost, update.  Writes the K costs, the new nominal sequence and
 * optionally the samples.  Returns the update's status. */
static int mppi_iteration_with(const or_model *m, const double *task, const double *x, const double *u_nom, int K,
                               int H, double lambda, const double *sigma, uint64_t seed, uint64_t iteration,
                               double *u_out, double *costs, double *U_out, int nthreads) {
    int nu = m->nu;
    size_t n = (size_t)K * H * nu;
    double *eps = (double *)malloc(sizeof(double) * n);
    double *U = U_out ? U_out : (double *)malloc(sizeof(double) * n);
    or_noise(seed, iteration, K, H, nu, sigma, eps);
    for (int k = 0; k < K; k++)
        for (int h = 0; h < H; h++)
            for (int j = 0; j < nu; j++) {
                size_t i = ((size_t)k * H + h) * nu + j;
                const or_link *L = &m->L[j / m->na][j % m->na];
                double val = u_nom[h * nu + j] + eps[i];
                if (val < L->u_lo) val = L->u_lo;
                if (val > L->u_hi) val = L->u_hi;
                U[i] = val;
            }
    rollout_many_from(m, task, x, U, K, H, costs, nthreads);
    int st = or_mppi_update(K, H, nu, costs, U, lambda, u_nom, u_out, NULL);
    free(eps);
    if (!U_out) free(U);
    return st;
}

int or_mppi_iteration(const or_model *m, const double *x, const double *u_nom, int K, int H, double lambda,
                      const double *sigma, uint64_t seed, uint64_t iteration, double *u_out, double *costs,
                      double *U_out, int nthreads) {
    return mppi_iteration_with(m, NULL, x, u_nom, K, H, lambda, sigma, seed, iteration, u_out, costs, U_out,
                               nthreads);
}

/* The same iteration with every sample costed by the ball-task suite
 * (Sec. IV-B): the optimiser step of the closed-loop task runs. */
int or_mppi_iteration_task(const or_model *m, const double *task, const double *x, const double *u_nom, int K,
                           int H, double lambda, const double *sigma, uint64_t seed, uint64_t iteration,
                           double *u_out, double *costs, double *U_out, int nthreads) {
    return mppi_iteration_with(m, task, x, u_nom, K, H, lambda, sigma, seed, iteration, u_out, costs, U_out,
                               nthreads);
}

/* --------------------------------------------------------------------- */
/* Eq. 8 in full: elite set, learning rate, covariance                    */
/* --------------------------------------------------------------------- */
/* Per horizon step h the sampling covariance is a full nu x nu block
 * Sigma_h (a reading: the paper does not fix the covariance structure);
 * samples are U_k[h] = clamp(nu_h + L_h z_k[h]) with L_h the Cholesky factor
 * of Sigma_h and z the standard normals of or_noise.
 *
 * One update (Eq. 8a-8d):
 *   EliteSet = the n_e samples of lowest cost (ties -> lower index);
 *   s_j = exp(-(c_j - c_min)/beta) over the elite set (the shift cancels);
 *   nu'      = (1 - eta) nu + eta sum_j s_j U_j / sum_j s_j;
 *   dSigma_h = sum_j s_j (U_j[h] - nu'_h)(U_j[h] - nu'_h)^T / sum_j s_j;
 *   Sigma'_h = (1 - eta) Sigma_h + eta dSigma_h + floor I.
 * Returns 0, or 1 when no cost is finite (everything unchanged). */
typedef struct { double c; int k; } or_key;
static int or_key_cmp(const void *a, const void *b) {
    const or_key *x = (const or_key *)a, *y = (const or_key *)b;
    if (x->c < y->c) return -1;
    if (x->c > y->c) return 1;
    return (x->k > y->k) - (x->k < y->k);
}

int or_elite_update(int K, int H, int nu, const double *costs, const double *U, int n_elite, double beta, double eta,
                    int update_cov, double cov_floor, const double *nu_in, const double *Sigma_in, double *nu_out,
                    double *Sigma_out, int *elite_out) {
    or_key *keys = (or_key *)malloc(sizeof(or_key) * K);
    int nf = 0;
    for (int k = 0; k < K; k++) {
        keys[k].c = isfinite(costs[k]) ? costs[k] : INFINITY;
        keys[k].k = k;
        nf += isfinite(costs[k]) ? 1 : 0;
    }
    if (nf == 0) {
        memcpy(nu_out, nu_in, sizeof(double) * H * nu);
        if (Sigma_out) memcpy(Sigma_out, Sigma_in, sizeof(double) * H * nu * nu);
        free(keys);
        return 1;
    }
    qsort(keys, K, sizeof(or_key), or_key_cmp);
    int ne = n_elite < nf ? n_elite : nf;
    if (ne < 1) ne = 1;
    double cmin = keys[0].c, Z = 0.0;
    double *s = (double *)malloc(sizeof(double) * ne);
    for (int e = 0; e < ne; e++) {
        s[e] = exp(-(keys[e].c - cmin) / beta);
        Z += s[e];
        if (elite_out) elite_out[e] = keys[e].k;
    }
    for (int i = 0; i < H * nu; i++) {
        double acc = 0.0;
        for (int e = 0; e < ne; e++) acc += s[e] * U[(size_t)keys[e].k * H * nu + i];
        nu_out[i] = (1.0 - eta) * nu_in[i] + eta * acc / Z;
    }
    if (Sigma_out) {
        for (int h = 0; h < H; h++)
            for (int a = 0; a < nu; a++)
                for (int b = 0; b < nu; b++) {
                    double acc = 0.0;
                    if (update_cov) {
                        for (int e = 0; e < ne; e++) {
                            const double *u = U + (size_t)keys[e].k * H * nu + (size_t)h * nu;
                            acc += s[e] * (u[a] - nu_out[h * nu + a]) * (u[b] - nu_out[h * nu + b]);
                        }
                        acc /= Z;
                    }
                    size_t idx = ((size_t)h * nu + a) * nu + b;
                    double v = update_cov ? (1.0 - eta) * Sigma_in[idx] + eta * acc : Sigma_in[idx];
                    if (update_cov && a == b) v += cov_floor;
                    Sigma_out[idx] = v;
                }
    }
    free(s);
    free(keys);
    return 0;
}

/* Samples from per-step covariance blocks: U_k[h] = clamp(nu_h + L_h z)
 * with L_h = chol(Sigma_h) (dense Cholesky) and z the unit normals of
 * (seed, iteration).  Returns -1 if a block is not positive definite. */
int or_sample_cov(const or_model *m, uint64_t seed, uint64_t iteration, int K, int H, const double *nu_in,
                  const double *Sigma, double *U) {
    int nu = m->nu;
    double *z = (double *)malloc(sizeof(double) * (size_t)K * H * nu);
    double *ones = (double *)malloc(sizeof(double) * nu);
    for (int j = 0; j < nu; j++) ones[j] = 1.0;
    or_noise(seed, iteration, K, H, nu, ones, z);
    double L[OR_MAXNV * OR_MAXNV];
    int rc = 0;
    for (int h = 0; h < H && rc == 0; h++) {
        memcpy(L, Sigma + (size_t)h * nu * nu, sizeof(double) * nu * nu);
        if (cholesky(L, nu) != 0) { rc = -1; break; }
        for (int k = 0; k < K; k++) {
            const double *zk = z + ((size_t)k * H + h) * nu;
            for (int j = 0; j < nu; j++) {
                double acc = nu_in[h * nu + j];
                for (int i = 0; i <= j; i++) acc += L[j * nu + i] * zk[i];
                const or_link *Lk = &m->L[j / m->na][j % m->na];
                if (acc < Lk->u_lo) acc = Lk->u_lo;
                if (acc > Lk->u_hi) acc = Lk->u_hi;
                U[((size_t)k * H + h) * nu + j] = acc;
            }
        }
    }
    free(z);
    free(ones);
    return rc;
}

/* --------------------------------------------------------------------- */
/* QP smoothing projection (Eq. 5)                                        */
/* --------------------------------------------------------------------- */
/* One joint's H commanded velocities v are projected onto the bounds of
 * Eq. 5b, r = 0..3 (the set of r is stated in Sec. III): minimise
 * 1/2 |v - vt|^2 subject to
 *   r=0  theta_{t+1} = q + dt sum_{i<=t} v_i              in [b0, b1], t = 0..H-1
 *   r=1  v_t                                             in [b2, b3], t = 0..H-1
 *   r=2  (v_t - v_{t-1}) / dt,             v_{-1} = qd   in [b4, b5], t = 0..H-1
 *   r=3  (v_t - 2 v_{t-1} + v_{t-2}) / dt^2, v_{-1} = qd in [b6, b7], t = 1..H-1
 * (qd, the joint's present velocity, fixes the first differences; the jerk at
 * t = 0 would need the velocity before it and is not bounded).
 *
 * The paper does not name its solver.  Read here as a fixed number of ADMM
 * iterations on the equilibrated rows
 *   D v = [s0 sum_{i<=t} v_i ; s1 v_t ; s2 (v_t - v_{t-1}) ; s3 (v_t - 2 v_{t-1} + v_{t-2})]
 * (position / dt, velocity, acceleration * dt, jerk * dt^2, times the group
 * scales s0..s3; the terms in qd move into the bounds lo, hi; a group whose
 * bounds are both infinite bounds nothing and takes no rows), in scaled
 * form with penalty rho, from v = vt and y = 0.  Each iteration:
 *   s = D v + y,  w = clip(s, lo, hi),  y = s - w,
 *   v = (I + rho D^T D)^{-1} (vt + rho D^T (w - y)).
 * A feasible vt is a fixed point.  The matrix is formed densely and factored
 * by Cholesky.  Returns the largest bound violation of the returned v in the
 * scaled rows; y_out (optional, 4H - 1 values in row order P, V, A, J) holds
 * the scaled duals (rho y are the multipliers at convergence). */
static void qp_rows(int H, double dt, const double *sc_in, const double *b, double q, double qd, double *D,
                    double *lo, double *hi) {
    int m = 4 * H - 1;
    double sc[4];
    for (int g = 0; g < 4; g++) sc[g] = (isinf(b[2 * g]) && b[2 * g] < 0 && isinf(b[2 * g + 1]) && b[2 * g + 1] > 0)
                                            ? 0.0 : sc_in[g];
    memset(D, 0, sizeof(double) * (size_t)m * H);
    for (int t = 0; t < H; t++) {
        for (int i = 0; i <= t; i++) D[(size_t)t * H + i] = sc[0];
        lo[t] = sc[0] * (b[0] - q) / dt;
        hi[t] = sc[0] * (b[1] - q) / dt;
        D[(size_t)(H + t) * H + t] = sc[1];
        lo[H + t] = sc[1] * b[2];
        hi[H + t] = sc[1] * b[3];
        D[(size_t)(2 * H + t) * H + t] = sc[2];
        if (t > 0) D[(size_t)(2 * H + t) * H + t - 1] = -sc[2];
        lo[2 * H + t] = sc[2] * (b[4] * dt + (t == 0 ? qd : 0.0));
        hi[2 * H + t] = sc[2] * (b[5] * dt + (t == 0 ? qd : 0.0));
    }
    for (int t = 1; t < H; t++) {
        int r = 3 * H + t - 1;
        D[(size_t)r * H + t] = sc[3];
        D[(size_t)r * H + t - 1] = -2.0 * sc[3];
        if (t >= 2) D[(size_t)r * H + t - 2] = sc[3];
        lo[r] = sc[3] * (b[6] * dt * dt - (t == 1 ? qd : 0.0));
        hi[r] = sc[3] * (b[7] * dt * dt - (t == 1 ? qd : 0.0));
    }
    for (int g = 0; g < 4; g++) /* rows of a free group stay zero, unbounded */
        if (sc[g] == 0.0)
            for (int r = g * H; r < (g == 3 ? 4 * H - 1 : (g + 1) * H); r++) {
                lo[r] = -INFINITY;
                hi[r] = INFINITY;
            }
}

double or_qp_project(int H, double dt, double rho, const double *sc, int iters, const double *b, double q, double qd,
                     const double *vt, double *v_out, double *y_out) {
    int m = 4 * H - 1;
    double *D = (double *)malloc(sizeof(double) * (size_t)m * H);
    double *lo = (double *)malloc(sizeof(double) * m), *hi = (double *)malloc(sizeof(double) * m);
    qp_rows(H, dt, sc, b, q, qd, D, lo, hi);
    double *A = (double *)calloc((size_t)H * H, sizeof(double));
    for (int i = 0; i < H; i++)
        for (int j = 0; j < H; j++) {
            double s = 0.0;
            for (int r = 0; r < m; r++) s += D[(size_t)r * H + i] * D[(size_t)r * H + j];
            A[i * H + j] = (i == j ? 1.0 : 0.0) + rho * s;
        }
    cholesky(A, H);
    double *y = (double *)calloc(m, sizeof(double)), *g = (double *)malloc(sizeof(double) * m);
    double *rhs = (double *)malloc(sizeof(double) * H);
    memcpy(v_out, vt, sizeof(double) * H);
    for (int it = 0; it < iters; it++) {
        for (int r = 0; r < m; r++) {
            double s = y[r];
            for (int i = 0; i < H; i++) s += D[(size_t)r * H + i] * v_out[i];
            double w = s < lo[r] ? lo[r] : (s > hi[r] ? hi[r] : s);
            y[r] = s - w;
            g[r] = w - y[r];
        }
        for (int i = 0; i < H; i++) {
            double s = 0.0;
            for (int r = 0; r < m; r++) s += D[(size_t)r * H + i] * g[r];
            rhs[i] = vt[i] + rho * s;
        }
        chol_solve(A, H, rhs);
        memcpy(v_out, rhs, sizeof(double) * H);
    }
    double viol = 0.0;
    for (int r = 0; r < m; r++) {
        double s = 0.0;
        for (int i = 0; i < H; i++) s += D[(size_t)r * H + i] * v_out[i];
        double e = s < lo[r] ? lo[r] - s : (s > hi[r] ? s - hi[r] : 0.0);
        if (e > viol) viol = e;
    }
    if (y_out) memcpy(y_out, y, sizeof(double) * m);
    free(D); free(lo); free(hi); free(A); free(y); free(g); free(rhs);
    return viol;
}

/* --------------------------------------------------------------------- */
/* Ball-task cost suite (Sec. IV-B)                                       */
/* --------------------------------------------------------------------- */
/* Task parameters: a flat array of OR_TASK_N + nu values
 *   [0] phase (0 pick, 1 move)  [1] w_c  [2] gamma  [3] w_theta  [4] w_yz
 *   [5] w_v  [6] w_r  [7] w_l  [8] l_ball  [9] w_eef_obj  [10] w_obj_targ
 *   [11] eps  [12..14] ball position before the pick  [15..17] target
 *   [18..21] q1*  [22..25] q2* (unit quaternions, w first)
 *   [26..26+nu) theta_home. */
#define OR_TASK_N 26
#define OR_MAXPAIRS (2 * OR_MAXL * OR_MAXB + 2 * OR_MAXL + OR_MAXL * OR_MAXL)

/* Distance between two capsules: the minimum over s, t in [0, 1] of
 * |a0 + s (a1 - a0) - b0 - t (b1 - b0)|, minus both radii.  The squared
 * distance is a convex quadratic on the unit square, so its minimum is the
 * interior stationary point when that lies inside, else the best of the
 * four edge minima (each a clamped 1-D quadratic). */
static double seg_point_t(const double *p0, const double *d, double dd, const double *x) {
    if (dd <= 0.0) return 0.0;
    double t = ((x[0] - p0[0]) * d[0] + (x[1] - p0[1]) * d[1] + (x[2] - p0[2]) * d[2]) / dd;
    return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
}
static double seg_seg_d2(const double *a0, const double *u, const double *b0, const double *v, double s, double t) {
    double e[3];
    for (int k = 0; k < 3; k++) e[k] = a0[k] + s * u[k] - b0[k] - t * v[k];
    return v3_dot(e, e);
}
void or_capsule_capsule(const double *a0, const double *a1, double ra, const double *b0, const double *b1, double rb,
                        double *dist) {
    double u[3], v[3], w[3];
    v3_sub(a1, a0, u);
    v3_sub(b1, b0, v);
    v3_sub(a0, b0, w);
    double A = v3_dot(u, u), B = v3_dot(u, v), C = v3_dot(v, v), D = v3_dot(u, w), E = v3_dot(v, w);
    double best = INFINITY;
    double den = A * C - B * B;
    if (den > 1e-14 * (A * C + 1e-300)) { /* interior stationary point */
        double s = (B * E - C * D) / den, t = (A * E - B * D) / den;
        if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) best = seg_seg_d2(a0, u, b0, v, s, t);
    }
    double pts[3];
    /* edges s = 0, s = 1 (closest t to a point), t = 0, t = 1 (closest s) */
    for (int e = 0; e < 2; e++) {
        for (int k = 0; k < 3; k++) pts[k] = a0[k] + e * u[k];
        double t = seg_point_t(b0, v, C, pts);
        double d2 = seg_seg_d2(a0, u, b0, v, (double)e, t);
        if (d2 < best) best = d2;
        for (int k = 0; k < 3; k++) pts[k] = b0[k] + e * v[k];
        double s = seg_point_t(a0, u, A, pts);
        d2 = seg_seg_d2(a0, u, b0, v, s, (double)e);
        if (d2 < best) best = d2;
    }
    *dist = sqrt(best) - ra - rb;
}

/* Unit quaternion (w, x, y, z) of a rotation matrix (row-major): the
 * largest of 4w^2 = 1 + tr, 4x^2 = 1 + R00 - R11 - R22, ... is taken
 * from the diagonal and the other three components from the off-diagonal
 * sums and differences; w >= 0. */
void or_rot_to_quat(const double *R, double *q) {
    double tr = R[0] + R[4] + R[8];
    double c[4] = {1.0 + tr, 1.0 + R[0] - R[4] - R[8], 1.0 - R[0] + R[4] - R[8], 1.0 - R[0] - R[4] + R[8]};
    int i = 0;
    for (int k = 1; k < 4; k++)
        if (c[k] > c[i]) i = k;
    double s = 0.5 / sqrt(c[i]);
    if (i == 0) { q[0] = 0.5 * sqrt(c[0]); q[1] = (R[7] - R[5]) * s; q[2] = (R[2] - R[6]) * s; q[3] = (R[3] - R[1]) * s; }
    else if (i == 1) { q[1] = 0.5 * sqrt(c[1]); q[0] = (R[7] - R[5]) * s; q[2] = (R[1] + R[3]) * s; q[3] = (R[2] + R[6]) * s; }
    else if (i == 2) { q[2] = 0.5 * sqrt(c[2]); q[0] = (R[2] - R[6]) * s; q[1] = (R[1] + R[3]) * s; q[3] = (R[5] + R[7]) * s; }
    else { q[3] = 0.5 * sqrt(c[3]); q[0] = (R[3] - R[1]) * s; q[1] = (R[2] + R[6]) * s; q[2] = (R[5] + R[7]) * s; }
    if (q[0] < 0.0) for (int k = 0; k < 4; k++) q[k] = -q[k];
}

/* End-effector state of both arms: position = distal end of the last
 * capsule, orientation = the last link frame as a quaternion, linear
 * velocity = J(q) qdot of that point.  ee = 20 values:
 * p1[3] p2[3] v1[3] v2[3] q1[4] q2[4]. */
void or_ee_state(const or_model *m, const double *x, double *ee) {
    or_fk f;
    or_forward_kinematics(m, x, &f);
    int na = m->na, nv = m->nv;
    const double *qd = x + m->nq;
    double J[3 * OR_MAXNV];
    for (int a = 0; a < 2; a++) {
        const double *p = f.a1[a][na - 1];
        memcpy(ee + 3 * a, p, 3 * sizeof(double));
        point_jacobian_link(m, &f, a, na - 1, p, J);
        for (int r = 0; r < 3; r++) {
            double s = 0.0;
            for (int j = 0; j < nv; j++) s += J[r * nv + j] * qd[j];
            ee[6 + 3 * a + r] = s;
        }
        or_rot_to_quat(f.R[a][na - 1], ee + 12 + 4 * a);
    }
}

/* Signed distances of the collision cost's pairs at state x: every link
 * against every box (link-major), every link against the ball (pick phase
 * only), every left link against every right link.  Returns the count. */
int or_pair_distances(const or_model *m, const double *x, int phase, double *d) {
    or_fk f;
    or_forward_kinematics(m, x, &f);
    int na = m->na, n = 0;
    double tmp[3], tmp2[3];
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < na; i++)
            for (int b = 0; b < m->nb; b++)
                or_capsule_box(f.a0[a][i], f.a1[a][i], m->L[a][i].rcap, m->bc[b], m->bh[b], &d[n++], tmp, tmp2, NULL);
    if (phase == 0) {
        const double *c = x + 2 * na;
        for (int a = 0; a < 2; a++)
            for (int i = 0; i < na; i++)
                or_sphere_capsule(c, m->rb, f.a0[a][i], f.a1[a][i], m->L[a][i].rcap, &d[n++], tmp, tmp2);
    }
    for (int i = 0; i < na; i++)
        for (int j = 0; j < na; j++)
            or_capsule_capsule(f.a0[0][i], f.a1[0][i], m->L[0][i].rcap, f.a0[1][j], f.a1[1][j], m->L[1][j].rcap,
                               &d[n++]);
    return n;
}

static double qdist(const double *q, const double *qs) {
    double c = fabs(q[0] * qs[0] + q[1] * qs[1] + q[2] * qs[2] + q[3] * qs[3]);
    return 2.0 * acos(c > 1.0 ? 1.0 : c);
}

/* The task cost from per-state features of x_0..x_H: D ((H+1) x B pair
 * distances), TH ((H+1) x nu joint positions), EE ((H+1) x 20 as
 * or_ee_state writes).  Every state term sums over the states x_1..x_H that
 * the H controls produce; the barrier sums over the H transitions
 * x_k -> x_{k+1}, k = 0..H-1, and the penetration indicator over x_1..x_H.
 * terms (optional, 8): C_c, C_theta, C_yz, C_v, C_r, C_l, C_eef_obj,
 * C_obj_targ.  Returns the weighted total. */
double or_task_cost_features(const double *task, int nu, int B, int H, const double *D, const double *TH,
                             const double *EE, double *terms) {
    const int phase = (int)task[0];
    const double gamma = task[2];
    double Cc = 0.0, Cth = 0.0, Cyz = 0.0, Cv2 = 0.0, Cr = 0.0, Cl = 0.0, Ceo = 0.0, Cot = 0.0;
    for (int k = 0; k < H; k++)
        for (int b = 0; b < B; b++) {
            double g = -D[(size_t)(k + 1) * B + b] + (1.0 - gamma) * D[(size_t)k * B + b];
            if (g > 0.0) Cc += g;
        }
    for (int k = 1; k <= H; k++) {
        for (int b = 0; b < B; b++)
            if (D[(size_t)k * B + b] < 0.0) Cc += 1.0;
        const double *th = TH + (size_t)k * nu, *e = EE + (size_t)k * 20;
        const double *p1 = e, *p2 = e + 3, *v1 = e + 6, *v2 = e + 9, *q1 = e + 12, *q2 = e + 16;
        double s = 0.0;
        for (int j = 0; j < nu; j++) s += (th[j] - task[OR_TASK_N + j]) * (th[j] - task[OR_TASK_N + j]);
        Cth += sqrt(s);
        Cyz += sqrt((p1[1] - p2[1]) * (p1[1] - p2[1]) + (p1[2] - p2[2]) * (p1[2] - p2[2]));
        double dp[3], dv[3];
        v3_sub(p1, p2, dp);
        v3_sub(v1, v2, dv);
        double rv = v3_dot(dp, dv);
        Cv2 += rv * rv;
        Cr += 0.5 * (qdist(q1, task + 18) + qdist(q2, task + 22));
        double l = v3_norm(dp) - task[8];
        Cl += l * l;
        double c[3] = {0.5 * (p1[0] + p2[0]), 0.5 * (p1[1] + p2[1]), 0.5 * (p1[2] + p2[2])};
        double eo[3] = {c[0] - task[12], c[1] - task[13], c[2] - (task[14] - task[11])};
        Ceo += v3_norm(eo);
        double ot[3] = {c[0] - task[15], c[1] - task[16], c[2] + task[11] - task[17]};
        Cot += v3_norm(ot);
    }
    double Cv = sqrt(Cv2);
    double wpick = phase == 0 ? 1.0 : 0.0, wmove = phase == 0 ? 0.0 : 1.0;
    if (terms) {
        terms[0] = Cc; terms[1] = Cth; terms[2] = Cyz; terms[3] = Cv;
        terms[4] = Cr; terms[5] = Cl; terms[6] = Ceo; terms[7] = Cot;
    }
    return wpick * (task[1] * Cc + task[9] * Ceo) + wmove * (task[1] * Cc + task[10] * Cot) + task[3] * Cth +
           task[4] * Cyz + task[5] * Cv + task[6] * Cr + task[7] * Cl;
}

/* Task cost of a trajectory x_0..x_H ((H+1) x nx). */
double or_task_cost(const or_model *m, const double *task, const double *traj, int H, double *terms) {
    int nx = m->nq + m->nv, nu = m->nu, phase = (int)task[0];
    double *D = (double *)malloc(sizeof(double) * (size_t)(H + 1) * OR_MAXPAIRS);
    double *TH = (double *)malloc(sizeof(double) * (size_t)(H + 1) * nu);
    double *EE = (double *)malloc(sizeof(double) * (size_t)(H + 1) * 20);
    int B = 0;
    for (int k = 0; k <= H; k++) {
        const double *x = traj + (size_t)k * nx;
        double d[OR_MAXPAIRS];
        B = or_pair_distances(m, x, phase, d);
        for (int b = 0; b < B; b++) D[(size_t)k * B + b] = d[b];
        memcpy(TH + (size_t)k * nu, x, sizeof(double) * nu);
        or_ee_state(m, x, EE + (size_t)k * 20);
    }
    double c = or_task_cost_features(task, nu, B, H, D, TH, EE, terms);
    free(D); free(TH); free(EE);
    return c;
}

/* Roll out H steps from x with controls U and score the trajectory with
 * the task cost (in place of the stage cost).  traj (optional) receives
 * the H+1 states. */
double or_rollout_task(const or_model *m, const double *task, const double *x, const double *U, int H,
                       double *traj_out, double *terms) {
    int nx = m->nq + m->nv;
    double *traj = (double *)malloc(sizeof(double) * (size_t)(H + 1) * nx);
    memcpy(traj, x, sizeof(double) * nx);
    for (int h = 0; h < H; h++) {
        or_step_info info;
        if (or_step(m, traj + (size_t)h * nx, U + (size_t)h * m->nu, traj + (size_t)(h + 1) * nx, &info) != 0) {
            free(traj);
            return NAN;
        }
    }
    double c = or_task_cost(m, task, traj, H, terms);
    if (traj_out) memcpy(traj_out, traj, sizeof(double) * (size_t)(H + 1) * nx);
    free(traj);
    return c;
}
