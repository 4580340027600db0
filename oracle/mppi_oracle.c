/*
 * FP64 CPU oracle of the torque-sampling MPPI update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path (the
 * CUDA library and its Python binding) never links, imports or calls it, and
 * it shares no code, header, table or constant generator with that path.
 *
 * It restates the method step by step in double precision, in the paper's
 * order and notation:
 *   - stochastic control model and noisy input, Eq. 1-2;
 *   - trajectory cost S = phi(x_T) + sum_t l(x_t, v_t), Eq. 3;
 *   - min-shifted importance weights and weighted noise update, Eq. 4a-4b,
 *     and the receding-horizon warm start (Sec. II, last paragraph);
 *   - torque sampling u_{k,t} = tau_t + dtau_{k,t} (Sec. III-A);
 *   - rigid-body dynamics M qdd + h = tau + tau_ext, Eq. 5, solved for qdd,
 *     Eq. 6, and the Euler update of Eq. 7 (the new velocity moves q);
 *   - the inertia matrix by Jacobian accumulation, Eq. 8, kept as a third,
 *     independent way to build M;
 *   - running cost l = C_task + C_constraint with C_motion, C_force and
 *     C_joint, Eq. 9-12 and Eq. 14.
 * Where the paper is silent (contact law, joint-cost hinges, terminal cost,
 * noise generator) the reading used is written beside the function.
 *
 * The dynamics come in three independent forms so that each pins the others:
 * Featherstone's RNEA + CRBA with a Cholesky solve, Featherstone's articulated
 * body algorithm (ABA), and Eq. 8 built from world-frame link Jacobians.  RNEA,
 * CRBA and ABA use explicit 6x6 spatial matrices in link coordinates (slow and
 * plain on purpose).
 *
 * Noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11), key = (seed_lo, seed_hi), counter =
 * (k, 2t + c, iter_lo, iter_hi) for call c in {0, 1}; each 32-bit word x maps
 * to u = ((x >> 8) + 0.5) / 2^24 and pairs of u go through Box-Muller
 * (z0 = r cos(2 pi u2), z1 = r sin(2 pi u2), r = sqrt(-2 ln u1)).  Call 0 gives
 * the normals of joints 0-3, call 1 those of joints 4-7 (the eighth is unused
 * for a 7-joint arm).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NMAX 7
#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Parameter records (mirrored field by field by the oracle's ctypes wrapper) */

typedef struct {
  int n;                        /* number of revolute joints, 1..7            */
  double joint_xyz[NMAX][3];    /* joint i origin in the parent link frame    */
  double joint_rpy[NMAX][3];    /* fixed parent->joint rotation, R=Rz Ry Rx   */
  double axis[NMAX][3];         /* unit rotation axis in the joint frame      */
  double com[NMAX][3];          /* centre of mass of link i, link frame       */
  double mass[NMAX];            /* m_i                                         */
  double inertia[NMAX][6];      /* I^G_i about the CoM: xx yy zz xy xz yz     */
  double armature[NMAX];        /* a_i of Eq. 8                                */
  double damping[NMAX];         /* viscous joint damping b_i                   */
  double ee_xyz[3];             /* end-effector point in the last link frame  */
  double q_min[NMAX], q_max[NMAX], qd_max[NMAX], tau_max[NMAX];
  double gravity[3];            /* world gravity vector                        */
} orc_robot;

typedef struct {
  double w_pos[3], w_ori[3];    /* diagonal W_pos, W_ori of Eq. 11            */
  double w_force, f_des, w_reg; /* Eq. 12 on the contact normal force          */
  double w_qlim, w_qdlim, w_tau, w_posture;
  double q_posture[NMAX];
  double w_terminal;            /* phi(x_T) = w_terminal * C_motion(x_T)       */
  int contact;                  /* 0: free space, 1: plane spring-damper      */
  double k_contact, d_contact;  /* N/m, N s/m                                  */
  /* Eq. 12-13 with the wrench estimate F_ee = Jbar^T (v - g(q)): when set,
   * C_force uses these diagonal 6-axis weights on F_ee = (force; moment)
   * instead of the contact normal force.                                    */
  int force_estimate;
  double w_force6[6], f_des6[6], w_reg6[6];
  /* Eq. 15 collision cost over link capsules: link i is the segment from
   * joint i's origin to joint i+1's (the last ends at the end-effector
   * point) with radius link_radius[i]; obstacles are capsules
   * (a xyz, b xyz, radius); pairs are links at least two apart and every
   * link with every obstacle.  collision: 0 off, 1 indicator (Eq. 15),
   * 2 squared hinge w * max(0, d_th - d)^2 (a smooth reading).          */
  int collision;
  double w_collision, d_th_self, d_th_obs;
  double link_radius[NMAX];
  int n_obs;
  double obs[8][7];
  /* Eq. 5-6 as the paper states them: tau_ext = J(q)^T F_ext with F_ext the
   * external wrench (force xyz; moment about the end-effector point xyz,
   * world frame), "assumed to be constant over the prediction horizon": it
   * is projected once, at the update's initial state q_0, and the same
   * tau_ext enters every step of every rollout (in addition to the plane
   * contact's, when that is on). */
  int ext_wrench;
  double f_ext[6];
} orc_cost;

/* ------------------------------------------------------------------------ */
/* 3-vector and 3x3 helpers                                                  */

static void v3_cross(const double a[3], const double b[3], double o[3]) {
  double t0 = a[1] * b[2] - a[2] * b[1];
  double t1 = a[2] * b[0] - a[0] * b[2];
  double t2 = a[0] * b[1] - a[1] * b[0];
  o[0] = t0; o[1] = t1; o[2] = t2;
}
static double v3_dot(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void m3_mul(const double A[3][3], const double B[3][3], double C[3][3]) {
  double T[3][3];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double s = 0;
      for (int k = 0; k < 3; k++) s += A[i][k] * B[k][j];
      T[i][j] = s;
    }
  memcpy(C, T, sizeof T);
}
static void m3_vec(const double A[3][3], const double x[3], double y[3]) {
  double t[3];
  for (int i = 0; i < 3; i++) t[i] = A[i][0] * x[0] + A[i][1] * x[1] + A[i][2] * x[2];
  memcpy(y, t, sizeof t);
}
static void m3_tvec(const double A[3][3], const double x[3], double y[3]) {
  double t[3];
  for (int i = 0; i < 3; i++) t[i] = A[0][i] * x[0] + A[1][i] * x[1] + A[2][i] * x[2];
  memcpy(y, t, sizeof t);
}
static void m3_transpose(const double A[3][3], double B[3][3]) {
  double T[3][3];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) T[i][j] = A[j][i];
  memcpy(B, T, sizeof T);
}
static void m3_skew(const double v[3], double S[3][3]) {
  S[0][0] = 0;     S[0][1] = -v[2]; S[0][2] = v[1];
  S[1][0] = v[2];  S[1][1] = 0;     S[1][2] = -v[0];
  S[2][0] = -v[1]; S[2][1] = v[0];  S[2][2] = 0;
}

/* R = Rz(yaw) Ry(pitch) Rx(roll) */
void orc_rpy_matrix(const double rpy[3], double R[3][3]) {
  double cr = cos(rpy[0]), sr = sin(rpy[0]);
  double cp = cos(rpy[1]), sp = sin(rpy[1]);
  double cy = cos(rpy[2]), sy = sin(rpy[2]);
  double Rx[3][3] = {{1, 0, 0}, {0, cr, -sr}, {0, sr, cr}};
  double Ry[3][3] = {{cp, 0, sp}, {0, 1, 0}, {-sp, 0, cp}};
  double Rz[3][3] = {{cy, -sy, 0}, {sy, cy, 0}, {0, 0, 1}};
  double T[3][3];
  m3_mul(Ry, Rx, T);
  m3_mul(Rz, T, R);
}

/* Rodrigues: rotation by angle q about unit axis a */
void orc_axis_angle(const double a[3], double q, double R[3][3]) {
  double c = cos(q), s = sin(q), C = 1.0 - c;
  double K[3][3];
  m3_skew(a, K);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      R[i][j] = (i == j ? c : 0.0) + s * K[i][j] + C * a[i] * a[j];
}

/* unit quaternion (w, x, y, z) -> rotation matrix; normalised first */
void orc_quat_matrix(const double qt[4], double R[3][3]) {
  double nrm = sqrt(qt[0] * qt[0] + qt[1] * qt[1] + qt[2] * qt[2] + qt[3] * qt[3]);
  double w = qt[0] / nrm, x = qt[1] / nrm, y = qt[2] / nrm, z = qt[3] / nrm;
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 and Box-Muller normals                                      */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)pb;
    uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)pa;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u24(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

/* eight standard normals for (sample k, step t) of update `iter`, Eq. 2 */
void orc_normals(uint64_t seed, uint64_t iter, uint32_t k, uint32_t t, double z[8]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t c = 0; c < 2; c++) {
    uint32_t ctr[4] = {k, 2u * t + c, (uint32_t)iter, (uint32_t)(iter >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    for (int p = 0; p < 2; p++) {
      double u1 = u24(w[2 * p]), u2 = u24(w[2 * p + 1]);
      double r = sqrt(-2.0 * log(u1));
      z[4 * c + 2 * p + 0] = r * cos(2.0 * PI * u2);
      z[4 * c + 2 * p + 1] = r * sin(2.0 * PI * u2);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Kinematics (Fig. 1: per-rollout FK, link Jacobians, end-effector pose)     */

/* rotation parent->link i and joint origin, for joint angle qi */
static void joint_transform(const orc_robot* rb, int i, double qi, double E[3][3], double r[3]) {
  double F[3][3], A[3][3];
  orc_rpy_matrix(rb->joint_rpy[i], F);
  orc_axis_angle(rb->axis[i], qi, A);
  m3_mul(F, A, E);
  r[0] = rb->joint_xyz[i][0]; r[1] = rb->joint_xyz[i][1]; r[2] = rb->joint_xyz[i][2];
}

/* World pose of every link frame (R[i], p[i]) and of the end-effector. */
void orc_fk(const orc_robot* rb, const double* q, double R[][3][3], double p[][3],
            double R_ee[3][3], double p_ee[3]) {
  double Rp[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double pp[3] = {0, 0, 0};
  for (int i = 0; i < rb->n; i++) {
    double E[3][3], r[3], d[3];
    joint_transform(rb, i, q[i], E, r);
    m3_vec(Rp, r, d);
    for (int a = 0; a < 3; a++) pp[a] += d[a];
    m3_mul(Rp, E, Rp);
    memcpy(R[i], Rp, sizeof Rp);
    memcpy(p[i], pp, sizeof pp);
  }
  double d[3];
  m3_vec(Rp, rb->ee_xyz, d);
  for (int a = 0; a < 3; a++) p_ee[a] = pp[a] + d[a];
  memcpy(R_ee, Rp, sizeof Rp);
}

/* World positions of the link centres of mass (for potential energy). */
void orc_com_positions(const orc_robot* rb, const double* q, double c[][3]) {
  double R[NMAX][3][3], p[NMAX][3], Re[3][3], pe[3];
  orc_fk(rb, q, R, p, Re, pe);
  for (int i = 0; i < rb->n; i++) {
    double d[3];
    m3_vec(R[i], rb->com[i], d);
    for (int a = 0; a < 3; a++) c[i][a] = p[i][a] + d[a];
  }
}

/* Geometric end-effector Jacobian in the world frame, row-major 6 x n:
 * rows 0-2 linear velocity of the end-effector point, rows 3-5 angular. */
void orc_jacobian(const orc_robot* rb, const double* q, double* J) {
  int n = rb->n;
  double R[NMAX][3][3], p[NMAX][3], Re[3][3], pe[3];
  orc_fk(rb, q, R, p, Re, pe);
  for (int j = 0; j < n; j++) {
    double z[3], d[3], v[3];
    m3_vec(R[j], rb->axis[j], z);
    for (int a = 0; a < 3; a++) d[a] = pe[a] - p[j][a];
    v3_cross(z, d, v);
    for (int a = 0; a < 3; a++) {
      J[a * n + j] = v[a];
      J[(3 + a) * n + j] = z[a];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Spatial algebra (Featherstone, Rigid Body Dynamics Algorithms, 2008):      */
/* 6-vectors are (angular; linear), 6x6 matrices are explicit.               */

typedef double m6[6][6];

static void m6_zero(m6 A) { memset(A, 0, sizeof(m6)); }
static void m6_vec(const m6 A, const double x[6], double y[6]) {
  double t[6];
  for (int i = 0; i < 6; i++) {
    double s = 0;
    for (int k = 0; k < 6; k++) s += A[i][k] * x[k];
    t[i] = s;
  }
  memcpy(y, t, sizeof t);
}
static void m6_tvec(const m6 A, const double x[6], double y[6]) {
  double t[6];
  for (int i = 0; i < 6; i++) {
    double s = 0;
    for (int k = 0; k < 6; k++) s += A[k][i] * x[k];
    t[i] = s;
  }
  memcpy(y, t, sizeof t);
}
/* C += A^T B A */
static void m6_add_congruence(const m6 A, const m6 B, m6 C) {
  m6 BA;
  for (int i = 0; i < 6; i++)
    for (int j = 0; j < 6; j++) {
      double s = 0;
      for (int k = 0; k < 6; k++) s += B[i][k] * A[k][j];
      BA[i][j] = s;
    }
  for (int i = 0; i < 6; i++)
    for (int j = 0; j < 6; j++) {
      double s = 0;
      for (int k = 0; k < 6; k++) s += A[k][i] * BA[k][j];
      C[i][j] += s;
    }
}

/* Plucker transform from parent coordinates to child coordinates, for a child
 * frame with rotation E (child axes in parent coordinates) at origin r. */
static void plucker_xform(const double E[3][3], const double r[3], m6 X) {
  double Et[3][3], S[3][3];
  m3_transpose(E, Et);
  m3_skew(r, S);
  m6_zero(X);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double ets = 0;
      for (int k = 0; k < 3; k++) ets += Et[i][k] * S[k][j];
      X[i][j] = Et[i][j];
      X[3 + i][3 + j] = Et[i][j];
      X[3 + i][j] = -ets;
    }
}

/* motion cross product v x m */
static void crm(const double v[6], const double m[6], double o[6]) {
  double a[3], b[3], c[3];
  v3_cross(v, m, a);
  v3_cross(v, m + 3, b);
  v3_cross(v + 3, m, c);
  o[0] = a[0]; o[1] = a[1]; o[2] = a[2];
  o[3] = b[0] + c[0]; o[4] = b[1] + c[1]; o[5] = b[2] + c[2];
}
/* force cross product v x* f */
static void crf(const double v[6], const double f[6], double o[6]) {
  double a[3], b[3], c[3];
  v3_cross(v, f, a);
  v3_cross(v + 3, f + 3, b);
  v3_cross(v, f + 3, c);
  o[0] = a[0] + b[0]; o[1] = a[1] + b[1]; o[2] = a[2] + b[2];
  o[3] = c[0]; o[4] = c[1]; o[5] = c[2];
}

/* spatial inertia of link i about its frame origin, link coordinates */
static void link_inertia(const orc_robot* rb, int i, m6 I) {
  const double* t = rb->inertia[i];
  double Ic[3][3] = {{t[0], t[3], t[4]}, {t[3], t[1], t[5]}, {t[4], t[5], t[2]}};
  double m = rb->mass[i];
  double C[3][3];
  m3_skew(rb->com[i], C);
  m6_zero(I);
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double cct = 0; /* C C^T */
      for (int k = 0; k < 3; k++) cct += C[a][k] * C[b][k];
      I[a][b] = Ic[a][b] + m * cct;
      I[a][3 + b] = m * C[a][b];
      I[3 + a][b] = m * C[b][a];
      I[3 + a][3 + b] = (a == b) ? m : 0.0;
    }
}

static void joint_xform(const orc_robot* rb, int i, double qi, m6 X, double S[6]) {
  double E[3][3], r[3];
  joint_transform(rb, i, qi, E, r);
  plucker_xform(E, r, X);
  S[0] = rb->axis[i][0]; S[1] = rb->axis[i][1]; S[2] = rb->axis[i][2];
  S[3] = S[4] = S[5] = 0.0;
}

/* Recursive Newton-Euler: tau = M(q) qdd + C(q, qd) qd + g(q).  Rigid bodies
 * only: the armature and damping of Eq. 5/8 are added by the callers. */
void orc_rnea(const orc_robot* rb, const double* q, const double* qd, const double* qdd,
              double* tau) {
  int n = rb->n;
  double v[NMAX][6], a[NMAX][6], f[NMAX][6], S[NMAX][6];
  m6 X[NMAX];
  double v0[6] = {0, 0, 0, 0, 0, 0};
  double a0[6] = {0, 0, 0, -rb->gravity[0], -rb->gravity[1], -rb->gravity[2]};
  for (int i = 0; i < n; i++) {
    joint_xform(rb, i, q[i], X[i], S[i]);
    const double* vp = (i == 0) ? v0 : v[i - 1];
    const double* ap = (i == 0) ? a0 : a[i - 1];
    double t[6], vJ[6], c[6];
    m6_vec(X[i], vp, t);
    for (int k = 0; k < 6; k++) vJ[k] = S[i][k] * qd[i];
    for (int k = 0; k < 6; k++) v[i][k] = t[k] + vJ[k];
    m6_vec(X[i], ap, t);
    crm(v[i], vJ, c);
    for (int k = 0; k < 6; k++) a[i][k] = t[k] + S[i][k] * qdd[i] + c[k];
    m6 I;
    double Iv[6], Ia[6], g[6];
    link_inertia(rb, i, I);
    m6_vec(I, a[i], Ia);
    m6_vec(I, v[i], Iv);
    crf(v[i], Iv, g);
    for (int k = 0; k < 6; k++) f[i][k] = Ia[k] + g[k];
  }
  for (int i = n - 1; i >= 0; i--) {
    double s = 0;
    for (int k = 0; k < 6; k++) s += S[i][k] * f[i][k];
    tau[i] = s;
    if (i > 0) {
      double t[6];
      m6_tvec(X[i], f[i], t);
      for (int k = 0; k < 6; k++) f[i - 1][k] += t[k];
    }
  }
}

/* Composite rigid body algorithm: joint-space inertia of the rigid links,
 * row-major n x n, without the armature. */
void orc_crba(const orc_robot* rb, const double* q, double* M) {
  int n = rb->n;
  m6 X[NMAX], Ic[NMAX];
  double S[NMAX][6];
  for (int i = 0; i < n; i++) {
    joint_xform(rb, i, q[i], X[i], S[i]);
    link_inertia(rb, i, Ic[i]);
  }
  for (int i = n - 1; i > 0; i--) m6_add_congruence(X[i], Ic[i], Ic[i - 1]);
  for (int i = 0; i < n; i++) {
    double F[6];
    m6_vec(Ic[i], S[i], F);
    double s = 0;
    for (int k = 0; k < 6; k++) s += S[i][k] * F[k];
    M[i * n + i] = s;
    int j = i;
    while (j > 0) {
      m6_tvec(X[j], F, F);
      j -= 1;
      s = 0;
      for (int k = 0; k < 6; k++) s += S[j][k] * F[k];
      M[i * n + j] = s;
      M[j * n + i] = s;
    }
  }
}

/* Articulated body algorithm with the armature a_i folded into the joint's
 * articulated inertia (D_i + a_i); tau already holds every generalised force. */
void orc_aba(const orc_robot* rb, const double* q, const double* qd, const double* tau,
             double* qdd) {
  int n = rb->n;
  m6 X[NMAX], IA[NMAX];
  double S[NMAX][6], v[NMAX][6], c[NMAX][6], pA[NMAX][6];
  double U[NMAX][6], D[NMAX], u[NMAX];
  double v0[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < n; i++) {
    joint_xform(rb, i, q[i], X[i], S[i]);
    const double* vp = (i == 0) ? v0 : v[i - 1];
    double t[6], vJ[6], Iv[6];
    m6_vec(X[i], vp, t);
    for (int k = 0; k < 6; k++) vJ[k] = S[i][k] * qd[i];
    for (int k = 0; k < 6; k++) v[i][k] = t[k] + vJ[k];
    crm(v[i], vJ, c[i]);
    link_inertia(rb, i, IA[i]);
    m6_vec(IA[i], v[i], Iv);
    crf(v[i], Iv, pA[i]);
  }
  for (int i = n - 1; i >= 0; i--) {
    m6_vec(IA[i], S[i], U[i]);
    double sU = 0, sp = 0;
    for (int k = 0; k < 6; k++) {
      sU += S[i][k] * U[i][k];
      sp += S[i][k] * pA[i][k];
    }
    D[i] = sU + rb->armature[i];
    u[i] = tau[i] - sp;
    if (i > 0) {
      m6 Ia;
      double pa[6], Ic[6];
      for (int r = 0; r < 6; r++)
        for (int s = 0; s < 6; s++) Ia[r][s] = IA[i][r][s] - U[i][r] * U[i][s] / D[i];
      m6_vec(Ia, c[i], Ic);
      for (int k = 0; k < 6; k++) pa[k] = pA[i][k] + Ic[k] + U[i][k] * u[i] / D[i];
      m6_add_congruence(X[i], Ia, IA[i - 1]);
      double t[6];
      m6_tvec(X[i], pa, t);
      for (int k = 0; k < 6; k++) pA[i - 1][k] += t[k];
    }
  }
  double a[NMAX][6];
  double a0[6] = {0, 0, 0, -rb->gravity[0], -rb->gravity[1], -rb->gravity[2]};
  for (int i = 0; i < n; i++) {
    const double* ap = (i == 0) ? a0 : a[i - 1];
    double ai[6];
    m6_vec(X[i], ap, ai);
    for (int k = 0; k < 6; k++) ai[k] += c[i][k];
    double Ua = 0;
    for (int k = 0; k < 6; k++) Ua += U[i][k] * ai[k];
    qdd[i] = (u[i] - Ua) / D[i];
    for (int k = 0; k < 6; k++) a[i][k] = ai[k] + S[i][k] * qdd[i];
  }
}

/* Eq. 8: M = sum_i (J_r,i^T Ibar_i J_r,i + m_i J_c,i^T J_c,i) + diag(a), with
 * Ibar_i = R_i I^G_i R_i^T and the link Jacobians taken in the world frame. */
void orc_mass_eq8(const orc_robot* rb, const double* q, double* M) {
  int n = rb->n;
  double R[NMAX][3][3], p[NMAX][3], Re[3][3], pe[3], z[NMAX][3];
  orc_fk(rb, q, R, p, Re, pe);
  for (int j = 0; j < n; j++) m3_vec(R[j], rb->axis[j], z[j]);
  for (int a = 0; a < n * n; a++) M[a] = 0.0;
  for (int i = 0; i < n; i++) {
    const double* t = rb->inertia[i];
    double IG[3][3] = {{t[0], t[3], t[4]}, {t[3], t[1], t[5]}, {t[4], t[5], t[2]}};
    double Rt[3][3], Ib[3][3], tmp[3][3];
    m3_transpose(R[i], Rt);
    m3_mul(R[i], IG, tmp);
    m3_mul(tmp, Rt, Ib);
    double ci[3], d[3];
    m3_vec(R[i], rb->com[i], d);
    for (int a = 0; a < 3; a++) ci[a] = p[i][a] + d[a];
    double Jr[3][NMAX], Jc[3][NMAX];
    for (int j = 0; j < n; j++) {
      double e[3], w[3];
      for (int a = 0; a < 3; a++) e[a] = ci[a] - p[j][a];
      v3_cross(z[j], e, w);
      for (int a = 0; a < 3; a++) {
        Jr[a][j] = (j <= i) ? z[j][a] : 0.0;
        Jc[a][j] = (j <= i) ? w[a] : 0.0;
      }
    }
    for (int r = 0; r < n; r++)
      for (int s = 0; s < n; s++) {
        double acc = 0;
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) acc += Jr[a][r] * Ib[a][b] * Jr[b][s];
        for (int a = 0; a < 3; a++) acc += rb->mass[i] * Jc[a][r] * Jc[a][s];
        M[r * n + s] += acc;
      }
  }
  for (int j = 0; j < n; j++) M[j * n + j] += rb->armature[j];
}

/* Cholesky factorisation A = L L^T and solve A x = b; returns -1 if A is not
 * positive definite. */
int orc_cholesky_solve(int n, const double* A, const double* b, double* x) {
  double L[NMAX * NMAX];
  for (int i = 0; i < n * n; i++) L[i] = 0.0;
  for (int j = 0; j < n; j++) {
    double s = A[j * n + j];
    for (int k = 0; k < j; k++) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return -1;
    L[j * n + j] = sqrt(s);
    for (int i = j + 1; i < n; i++) {
      double t = A[i * n + j];
      for (int k = 0; k < j; k++) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / L[j * n + j];
    }
  }
  double y[NMAX];
  for (int i = 0; i < n; i++) {
    double t = b[i];
    for (int k = 0; k < i; k++) t -= L[i * n + k] * y[k];
    y[i] = t / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; i--) {
    double t = y[i];
    for (int k = i + 1; k < n; k++) t -= L[k * n + i] * x[k];
    x[i] = t / L[i * n + i];
  }
  return 0;
}

/* Eq. 6: qdd = M^-1 (tau_in - h) with M = M_rb + diag(a) and
 * h = C qd + g + b qd; tau_in already includes tau_ext.
 * method 0: RNEA + CRBA + Cholesky; 1: ABA; 2: Eq. 8 mass + RNEA + Cholesky. */
int orc_forward_dynamics(const orc_robot* rb, const double* q, const double* qd,
                         const double* tau_in, int method, double* qdd) {
  int n = rb->n;
  double rhs[NMAX];
  if (method == 1) {
    for (int j = 0; j < n; j++) rhs[j] = tau_in[j] - rb->damping[j] * qd[j];
    orc_aba(rb, q, qd, rhs, qdd);
    return 0;
  }
  double zero[NMAX] = {0}, h[NMAX], M[NMAX * NMAX];
  orc_rnea(rb, q, qd, zero, h);
  for (int j = 0; j < n; j++) rhs[j] = tau_in[j] - h[j] - rb->damping[j] * qd[j];
  if (method == 2) {
    orc_mass_eq8(rb, q, M);
  } else {
    orc_crba(rb, q, M);
    for (int j = 0; j < n; j++) M[j * n + j] += rb->armature[j];
  }
  return orc_cholesky_solve(n, M, rhs, qdd);
}

/* ------------------------------------------------------------------------ */
/* Contact and costs                                                          */

/* Unilateral plane contact (n . p >= d is free space).  Penetration
 * delta = d - n . p_ee; normal velocity v_n = n . (J_v qd); normal force
 * f = max(0, k delta - c v_n) when delta > 0, else 0.  The wrench (f n, 0)
 * maps to joint torques through J^T (Eq. 5, tau_ext = J^T F_ext).
 * Returns f; writes tau_ext when the pointer is not NULL. */
double orc_contact(const orc_robot* rb, const orc_cost* c, const double plane[4],
                   const double* q, const double* qd, double* tau_ext) {
  int n = rb->n;
  double J[6 * NMAX];
  orc_jacobian(rb, q, J);
  double R[NMAX][3][3], p[NMAX][3], Re[3][3], pe[3];
  orc_fk(rb, q, R, p, Re, pe);
  double delta = plane[3] - v3_dot(plane, pe);
  double f = 0.0;
  if (delta > 0.0) {
    double vee[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++)
      for (int j = 0; j < n; j++) vee[a] += J[a * n + j] * qd[j];
    double vn = v3_dot(plane, vee);
    f = c->k_contact * delta - c->d_contact * vn;
    if (f < 0.0) f = 0.0;
  }
  if (tau_ext)
    for (int j = 0; j < n; j++) {
      double s = 0;
      for (int a = 0; a < 3; a++) s += J[a * n + j] * f * plane[a];
      tau_ext[j] = s;
    }
  return f;
}

/* The paper's constant external torque (Eq. 5): tau_ext = J(q0)^T F_ext,
 * with J the geometric Jacobian of the end-effector point (rows: linear
 * velocity, angular velocity), so tau_j = J_v,j . force + J_w,j . moment.
 * Zero when ext_wrench is off. */
void orc_ext_torque(const orc_robot* rb, const orc_cost* c, const double* q0, double* tau_ext) {
  int n = rb->n;
  for (int j = 0; j < n; j++) tau_ext[j] = 0.0;
  if (!c->ext_wrench) return;
  double J[6 * NMAX];
  orc_jacobian(rb, q0, J);
  for (int j = 0; j < n; j++) {
    double s = 0.0;
    for (int a = 0; a < 6; a++) s += J[a * n + j] * c->f_ext[a];
    tau_ext[j] = s;
  }
}

/* Rotation vector of R (matrix logarithm of Eq. 11), theta in [0, pi]. */
void orc_so3_log(const double R[3][3], double r[3]) {
  double vx = R[2][1] - R[1][2], vy = R[0][2] - R[2][0], vz = R[1][0] - R[0][1];
  double s = 0.5 * sqrt(vx * vx + vy * vy + vz * vz);
  double c = 0.5 * (R[0][0] + R[1][1] + R[2][2] - 1.0);
  double th = atan2(s, c);
  if (s > 1e-7) {
    double k = th / (2.0 * s);
    r[0] = k * vx; r[1] = k * vy; r[2] = k * vz;
  } else if (c > 0.0) {
    /* theta ~ 0: log R ~ vee(R - R^T)/2 */
    r[0] = 0.5 * vx; r[1] = 0.5 * vy; r[2] = 0.5 * vz;
  } else {
    /* theta ~ pi: axis from the symmetric part R + R^T = 2 c I + 2 (1 - c) a a^T */
    double B[3][3];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) B[i][j] = (R[i][j] + R[j][i]) * 0.5 - (i == j ? c : 0.0);
    int m = 0;
    if (B[1][1] > B[m][m]) m = 1;
    if (B[2][2] > B[m][m]) m = 2;
    double a[3];
    double dm = sqrt(B[m][m] / (1.0 - c));
    for (int i = 0; i < 3; i++) a[i] = B[i][m] / ((1.0 - c) * dm);
    double vv[3] = {vx, vy, vz};
    if (v3_dot(a, vv) < 0.0) { a[0] = -a[0]; a[1] = -a[1]; a[2] = -a[2]; }
    r[0] = th * a[0]; r[1] = th * a[1]; r[2] = th * a[2];
  }
}

/* C_motion of Eq. 11 with diagonal weights: goal = (p_des xyz, quat wxyz). */
double orc_motion_cost(const orc_cost* c, const double goal[7], const double p_ee[3],
                       const double R_ee[3][3]) {
  double Rd[3][3], Rdt[3][3], Rerr[3][3], r[3];
  orc_quat_matrix(goal + 3, Rd);
  m3_transpose(Rd, Rdt);
  m3_mul(Rdt, R_ee, Rerr);
  orc_so3_log(Rerr, r);
  double s = 0;
  for (int a = 0; a < 3; a++) {
    double e = goal[a] - p_ee[a];
    s += c->w_pos[a] * e * e + c->w_ori[a] * r[a] * r[a];
  }
  return s;
}

static double hinge2(double x) { return x > 0.0 ? x * x : 0.0; }

/* C_joint: position-limit and velocity-limit hinges plus posture regulariser
 * (the paper defers the formulas; this reading uses smooth quadratic hinges),
 * plus the torque-limit hinge on the sampled input v. */
double orc_joint_cost(const orc_robot* rb, const orc_cost* c, const double* q, const double* qd,
                      const double* v) {
  double s = 0;
  for (int j = 0; j < rb->n; j++) {
    s += c->w_qlim * (hinge2(q[j] - rb->q_max[j]) + hinge2(rb->q_min[j] - q[j]));
    s += c->w_qdlim * hinge2(fabs(qd[j]) - rb->qd_max[j]);
    double e = q[j] - c->q_posture[j];
    s += c->w_posture * e * e;
    s += c->w_tau * hinge2(fabs(v[j]) - rb->tau_max[j]);
  }
  return s;
}

/* End-effector wrench estimate of Eq. 12-13: F_ee = Jbar^T tau with the
 * dynamically consistent generalised inverse Jbar = M^-1 J^T (J M^-1 J^T)^-1
 * (Khatib 1987), so F_ee = Lambda J M^-1 tau with Lambda = (J M^-1 J^T)^-1.
 * Reading of the torque: tau = v - g(q), the input net of the gravity torque
 * g(q) = RNEA(q, 0, 0); M = CRBA + diag(armature); J is the world-frame
 * geometric Jacobian of the end-effector point, so F = (force xyz; moment
 * about the end-effector point xyz) in the world frame.  Each step is the
 * definition written out: the columns of M^-1 J^T and M^-1 tau by Cholesky
 * solves, then the 6x6 solve.  Returns -1 when M or J M^-1 J^T is not
 * positive definite (a kinematic singularity), with F set to NaN. */
int orc_force_estimate(const orc_robot* rb, const double* q, const double* v, double F[6]) {
  int n = rb->n;
  double M[NMAX * NMAX], J[6 * NMAX], g[NMAX], zero[NMAX] = {0}, tau[NMAX];
  for (int a = 0; a < 6; a++) F[a] = NAN;
  orc_crba(rb, q, M);
  for (int j = 0; j < n; j++) M[j * n + j] += rb->armature[j];
  orc_jacobian(rb, q, J);
  orc_rnea(rb, q, zero, zero, g);
  for (int j = 0; j < n; j++) tau[j] = v[j] - g[j];
  /* X = M^-1 J^T, column by column (column a is M^-1 times row a of J) */
  double X[NMAX][6], col[NMAX], x[NMAX];
  for (int a = 0; a < 6; a++) {
    for (int j = 0; j < n; j++) col[j] = J[a * n + j];
    if (orc_cholesky_solve(n, M, col, x) != 0) return -1;
    for (int j = 0; j < n; j++) X[j][a] = x[j];
  }
  /* Lambda^-1 = J M^-1 J^T and the task acceleration J M^-1 tau */
  double A[36], b[6], y[NMAX];
  for (int a = 0; a < 6; a++)
    for (int c2 = 0; c2 < 6; c2++) {
      double s = 0.0;
      for (int j = 0; j < n; j++) s += J[a * n + j] * X[j][c2];
      A[a * 6 + c2] = s;
    }
  if (orc_cholesky_solve(n, M, tau, y) != 0) return -1;
  for (int a = 0; a < 6; a++) {
    double s = 0.0;
    for (int j = 0; j < n; j++) s += J[a * n + j] * y[j];
    b[a] = s;
  }
  double Fx[6];
  if (orc_cholesky_solve(6, A, b, Fx) != 0) return -1;
  for (int a = 0; a < 6; a++) F[a] = Fx[a];
  return 0;
}

/* C_force of Eq. 12 on the wrench estimate: diagonal W_force and W_reg over
 * the six axes, sum_a w_force6[a] (f_des6[a] - F[a])^2 + w_reg6[a] F[a]^2,
 * charged at the configuration q_t where the input v_t acts.  NaN at a
 * kinematic singularity. */
double orc_force_estimate_cost(const orc_robot* rb, const orc_cost* c, const double* q,
                               const double* v) {
  double F[6];
  if (orc_force_estimate(rb, q, v, F) != 0) return NAN;
  double s = 0.0;
  for (int a = 0; a < 6; a++) {
    double e = c->f_des6[a] - F[a];
    s += c->w_force6[a] * e * e + c->w_reg6[a] * F[a] * F[a];
  }
  return s;
}

/* Minimum distance between the segments [p1, q1] and [p2, q2] (the
 * quantity Lumelsky's method computes for Eq. 15).  Written as the
 * definition: the squared distance |p1 + s d1 - p2 - t d2|^2 is a convex
 * quadratic on the square (s, t) in [0, 1]^2, so its minimum is either the
 * stationary point, when that lies inside the square, or on one of the four
 * edges, each of which is an endpoint against the other segment (a clamped
 * projection).  Every candidate is evaluated; the least is returned. */
static double point_segment_dist2(const double x[3], const double a[3], const double b[3]) {
  double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double w[3] = {x[0] - a[0], x[1] - a[1], x[2] - a[2]};
  double dd = v3_dot(d, d);
  double u = dd > 0.0 ? v3_dot(w, d) / dd : 0.0;
  if (u < 0.0) u = 0.0;
  if (u > 1.0) u = 1.0;
  double e[3] = {w[0] - u * d[0], w[1] - u * d[1], w[2] - u * d[2]};
  return v3_dot(e, e);
}

double orc_segment_distance(const double p1[3], const double q1[3], const double p2[3],
                            const double q2[3]) {
  double best = point_segment_dist2(p1, p2, q2);
  double c;
  if ((c = point_segment_dist2(q1, p2, q2)) < best) best = c;
  if ((c = point_segment_dist2(p2, p1, q1)) < best) best = c;
  if ((c = point_segment_dist2(q2, p1, q1)) < best) best = c;
  double d1[3] = {q1[0] - p1[0], q1[1] - p1[1], q1[2] - p1[2]};
  double d2[3] = {q2[0] - p2[0], q2[1] - p2[1], q2[2] - p2[2]};
  double r[3] = {p1[0] - p2[0], p1[1] - p2[1], p1[2] - p2[2]};
  double a = v3_dot(d1, d1), b = v3_dot(d1, d2), e = v3_dot(d2, d2);
  double det = a * e - b * b;
  if (det > 1e-14 * a * e) {
    /* stationary point: a s - b t = -d1.r, b s - e t = -d2.r */
    double f1 = -v3_dot(d1, r), f2 = -v3_dot(d2, r);
    double det2 = b * b - a * e; /* determinant of [[a, -b], [b, -e]] */
    double s_ = (b * f2 - e * f1) / det2;
    double t_ = (a * f2 - b * f1) / det2;
    if (s_ >= 0.0 && s_ <= 1.0 && t_ >= 0.0 && t_ <= 1.0) {
      double g[3];
      for (int k = 0; k < 3; k++) g[k] = r[k] + s_ * d1[k] - t_ * d2[k];
      if ((c = v3_dot(g, g)) < best) best = c;
    }
  }
  return sqrt(best);
}

/* End points of the link segments at q: P[i] = origin of joint i for
 * i < n, P[n] = the end-effector point; link i spans P[i] .. P[i+1]. */
void orc_link_points(const orc_robot* rb, const double* q, double P[][3]) {
  double R[NMAX][3][3], p[NMAX][3], Re[3][3], pe[3];
  orc_fk(rb, q, R, p, Re, pe);
  for (int i = 0; i < rb->n; i++) memcpy(P[i], p[i], sizeof(double) * 3);
  memcpy(P[rb->n], pe, sizeof(double) * 3);
}

/* Signed clearances d_i (segment distance minus both radii) of the
 * collision pairs in a fixed order: self pairs (i, j), j >= i + 2, by i then
 * j, then link i against obstacle o, by i then o.  Returns the count. */
int orc_collision_distances(const orc_robot* rb, const orc_cost* c, const double* q, double* d) {
  int n = rb->n, m = 0;
  double P[NMAX + 1][3];
  orc_link_points(rb, q, P);
  for (int i = 0; i < n; i++)
    for (int j = i + 2; j < n; j++)
      d[m++] = orc_segment_distance(P[i], P[i + 1], P[j], P[j + 1]) - c->link_radius[i] -
               c->link_radius[j];
  for (int i = 0; i < n; i++)
    for (int o = 0; o < c->n_obs; o++)
      d[m++] = orc_segment_distance(P[i], P[i + 1], c->obs[o], c->obs[o] + 3) -
               c->link_radius[i] - c->obs[o][6];
  return m;
}

/* C_collision of Eq. 15 at configuration q. */
double orc_collision_cost(const orc_robot* rb, const orc_cost* c, const double* q) {
  double d[NMAX * NMAX + NMAX * 8];
  int n = rb->n, m = orc_collision_distances(rb, c, q, d);
  int n_self = 0;
  for (int i = 0; i < n; i++)
    for (int j = i + 2; j < n; j++) n_self++;
  double s = 0.0;
  for (int k = 0; k < m; k++) {
    double th = k < n_self ? c->d_th_self : c->d_th_obs;
    if (c->collision == 1)
      s += d[k] < th ? 1.0 : 0.0;
    else
      s += d[k] < th ? (th - d[k]) * (th - d[k]) : 0.0;
  }
  return c->w_collision * s;
}

/* Running cost l(x_{t+1}, v_t) = C_motion + C_force + C_joint + C_collision
 * (Eq. 9-12, 14-15).  With force_estimate set, C_force is the wrench-estimate term, which
 * orc_rollout adds at (q_t, v_t); this function then leaves C_force out. */
double orc_stage_cost(const orc_robot* rb, const orc_cost* c, const double goal[7],
                      const double plane[4], const double* q, const double* qd,
                      const double* v) {
  double R[NMAX][3][3], p[NMAX][3], Re[3][3], pe[3];
  orc_fk(rb, q, R, p, Re, pe);
  double s = orc_motion_cost(c, goal, pe, Re);
  if (c->contact && !c->force_estimate) {
    double f = orc_contact(rb, c, plane, q, qd, NULL);
    double e = c->f_des - f;
    s += c->w_force * e * e + c->w_reg * f * f;
  }
  s += orc_joint_cost(rb, c, q, qd, v);
  if (c->collision) s += orc_collision_cost(rb, c, q);
  return s;
}

/* ------------------------------------------------------------------------ */
/* Rollout, update, step                                                      */

/* One rollout k (Eq. 1-3 with Eq. 5-7): for t = 0..T-1 the noisy torque
 * v_t = u_t + dtau_{k,t} acts on x_t and gives x_{t+1}; l is charged on
 * (x_{t+1}, v_t), the wrench-estimate C_force (when set) on (q_t, v_t); the
 * terminal cost is w_terminal * C_motion(x_T).
 * noise_out (T*n, [t][j]) receives dtau when not NULL.  Returns S_k. */
double orc_rollout(const orc_robot* rb, const orc_cost* c, double dt, int T, const double* sigma,
                   uint64_t seed, uint64_t iter, uint32_t k, const double* q0, const double* qd0,
                   const double goal[7], const double plane[4], const double* plan, int method,
                   double* noise_out) {
  int n = rb->n;
  double q[NMAX], qd[NMAX], v[NMAX], tau[NMAX], qdd[NMAX], tex[NMAX];
  memcpy(q, q0, sizeof(double) * n);
  memcpy(qd, qd0, sizeof(double) * n);
  double S = 0.0;
  double tex0[NMAX];
  orc_ext_torque(rb, c, q0, tex0);
  for (int t = 0; t < T; t++) {
    double z[8];
    orc_normals(seed, iter, k, (uint32_t)t, z);
    for (int j = 0; j < n; j++) {
      double du = sigma[j] * z[j];
      if (noise_out) noise_out[t * n + j] = du;
      v[j] = plan[t * n + j] + du;
    }
    if (c->force_estimate) S += orc_force_estimate_cost(rb, c, q, v);
    for (int j = 0; j < n; j++) tex[j] = 0.0;
    if (c->contact) orc_contact(rb, c, plane, q, qd, tex);
    for (int j = 0; j < n; j++) tau[j] = v[j] + tex[j] + tex0[j];
    if (orc_forward_dynamics(rb, q, qd, tau, method, qdd) != 0) return NAN;
    for (int j = 0; j < n; j++) {
      qd[j] += qdd[j] * dt;
      q[j] += qd[j] * dt;
    }
    S += orc_stage_cost(rb, c, goal, plane, q, qd, v);
  }
  if (c->w_terminal != 0.0) {
    double R[NMAX][3][3], p[NMAX][3], Re[3][3], pe[3];
    orc_fk(rb, q, R, p, Re, pe);
    S += c->w_terminal * orc_motion_cost(c, goal, pe, Re);
  }
  return S;
}

/* Eq. 4a-4b and the warm-start shift.  S: K costs; noise: [k][t][j];
 * plan, ustar, plan_next: [t][j].  Non-finite S_k get weight 0.  If no S_k is
 * finite the plan is left as it is (ustar = plan_next = plan) and 1 is
 * returned.  stats (may be NULL): S_min, sum of weights, effective sample
 * size 1/sum(wbar^2), number of non-finite costs. */
int orc_mppi_update(int K, int T, int n, const double* S, const double* noise, const double* plan,
                    double lambda, double* ustar, double* plan_next, double* stats) {
  double Smin = INFINITY;
  int bad = 0;
  for (int k = 0; k < K; k++) {
    if (isfinite(S[k])) {
      if (S[k] < Smin) Smin = S[k];
    } else {
      bad++;
    }
  }
  if (!isfinite(Smin)) {
    for (int i = 0; i < T * n; i++) ustar[i] = plan_next[i] = plan[i];
    if (stats) { stats[0] = Smin; stats[1] = 0; stats[2] = 0; stats[3] = bad; }
    return 1;
  }
  double* w = (double*)malloc(sizeof(double) * (size_t)K);
  double Z = 0.0;
  for (int k = 0; k < K; k++) {
    w[k] = isfinite(S[k]) ? exp(-(S[k] - Smin) / lambda) : 0.0;
    Z += w[k];
  }
  for (int i = 0; i < T * n; i++) {
    double N = 0.0;
    for (int k = 0; k < K; k++) N += w[k] * noise[(size_t)k * T * n + i];
    ustar[i] = plan[i] + N / Z;
  }
  for (int t = 0; t < T; t++) {
    int src = (t + 1 < T) ? t + 1 : T - 1;
    for (int j = 0; j < n; j++) plan_next[t * n + j] = ustar[src * n + j];
  }
  if (stats) {
    double w2 = 0.0;
    for (int k = 0; k < K; k++) w2 += (w[k] / Z) * (w[k] / Z);
    stats[0] = Smin; stats[1] = Z; stats[2] = 1.0 / w2; stats[3] = bad;
  }
  free(w);
  return 0;
}

/* One full MPPI update: K rollouts, then Eq. 4 and the shift.  S_out (K) and
 * noise_out (K*T*n) may be NULL.  nthreads > 1 runs the rollouts with OpenMP
 * when the library was built with it.  Returns the update's status. */
int orc_mppi_step(const orc_robot* rb, const orc_cost* c, double dt, int T, int K, double lambda,
                  const double* sigma, uint64_t seed, uint64_t iter, const double* q0,
                  const double* qd0, const double goal[7], const double plane[4],
                  const double* plan, int method, int nthreads, double* S_out, double* noise_out,
                  double* ustar, double* plan_next, double* stats) {
  int n = rb->n;
  double* S = (double*)malloc(sizeof(double) * (size_t)K);
  double* noise = noise_out ? noise_out : (double*)malloc(sizeof(double) * (size_t)K * T * n);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int k = 0; k < K; k++)
    S[k] = orc_rollout(rb, c, dt, T, sigma, seed, iter, (uint32_t)k, q0, qd0, goal, plane, plan,
                       method, noise + (size_t)k * T * n);
  (void)nthreads;
  int rc = orc_mppi_update(K, T, n, S, noise, plan, lambda, ustar, plan_next, stats);
  if (S_out) memcpy(S_out, S, sizeof(double) * (size_t)K);
  free(S);
  if (!noise_out) free(noise);
  return rc;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Sharded update (the exchange step if the K samples were split over G     */
/* devices): each shard g reduces its own samples to (m_g, Z_g, N_g) with     */
/* m_g = min S, Z_g = sum exp(-(S - m_g)/lambda), N_g = sum exp(...) dtau     */
/* (T*n entries); the merge rescales by exp(-(m_g - m)/lambda), m = min m_g,  */
/* which is exactly Eq. 4 over all samples.                                   */

/* part: 2 + T*n doubles (m, Z, N[T*n]).  noise: [k][t][j] for this shard. */
void orc_mppi_partial(int K, int T, int n, const double* S, const double* noise, double lambda,
                      double* part) {
  double m = INFINITY;
  for (int k = 0; k < K; k++)
    if (isfinite(S[k]) && S[k] < m) m = S[k];
  part[0] = m;
  part[1] = 0.0;
  for (int i = 0; i < T * n; i++) part[2 + i] = 0.0;
  if (!isfinite(m)) return;
  for (int k = 0; k < K; k++) {
    if (!isfinite(S[k])) continue;
    double w = exp(-(S[k] - m) / lambda);
    part[1] += w;
    for (int i = 0; i < T * n; i++) part[2 + i] += w * noise[(size_t)k * T * n + i];
  }
}

/* Merges G partials (G x (2 + T*n)) into u* and the shifted plan; returns 1
 * (plan kept) when no shard had a finite cost. */
int orc_mppi_merge(int G, int T, int n, const double* parts, const double* plan, double lambda,
                   double* ustar, double* plan_next) {
  const int stride = 2 + T * n;
  double m = INFINITY;
  for (int g = 0; g < G; g++)
    if (parts[g * stride] < m) m = parts[g * stride];
  if (!isfinite(m)) {
    for (int i = 0; i < T * n; i++) ustar[i] = plan_next[i] = plan[i];
    return 1;
  }
  double Z = 0.0;
  for (int g = 0; g < G; g++)
    if (isfinite(parts[g * stride])) Z += parts[g * stride + 1] * exp(-(parts[g * stride] - m) / lambda);
  for (int i = 0; i < T * n; i++) {
    double N = 0.0;
    for (int g = 0; g < G; g++)
      if (isfinite(parts[g * stride]))
        N += parts[g * stride + 2 + i] * exp(-(parts[g * stride] - m) / lambda);
    ustar[i] = plan[i] + N / Z;
  }
  for (int t = 0; t < T; t++) {
    int src = (t + 1 < T) ? t + 1 : T - 1;
    for (int j = 0; j < n; j++) plan_next[t * n + j] = ustar[src * n + j];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Learned proposal: an MLP (input -> L hidden GELU layers -> linear output) */
/* and its gradients, in double precision, written from the definitions:     */
/*   z_l = W_l h_{l-1} + b_l,  h_l = gelu(z_l) (hidden),  y = W_L h_{L-1} + b_L */
/*   gelu(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2,                        */
/*   loss = mean over batch and outputs of (y - y*)^2.                        */
/* W_l is row-major [out][in].  With bf16 != 0 the tensors that the GPU keeps */
/* in BF16 (weights, layer inputs, the loss gradient and the backpropagated   */
/* deltas) are rounded to BF16 (round to nearest even) at the same points, so */
/* that only accumulation order separates the two sides.                      */

static double bf16_round(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {  /* finite: round to nearest even */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
  }
  u &= 0xffff0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_grad(double x) {
  return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * PI);
}

/* dims[0..L]: widths (input, hidden..., output); params: W_1, b_1, ..., W_L,
 * b_L flat.  X: [n][dims[0]]; Y: [n][dims[L]].  acts (may be NULL): the
 * pre-activations z_l of every layer, [n][dims[l]] each, concatenated. */
void orc_mlp_forward(int L, const int* dims, const double* params, int n, const double* X,
                     int bf16, double* Y, double* acts) {
  int maxw = 0;
  for (int l = 0; l <= L; l++) if (dims[l] > maxw) maxw = dims[l];
  double* h = (double*)malloc(sizeof(double) * maxw);
  double* z = (double*)malloc(sizeof(double) * maxw);
  for (int s = 0; s < n; s++) {
    for (int i = 0; i < dims[0]; i++) h[i] = bf16 ? bf16_round(X[(size_t)s * dims[0] + i]) : X[(size_t)s * dims[0] + i];
    const double* p = params;
    size_t aoff = 0;
    for (int l = 1; l <= L; l++) {
      const int in = dims[l - 1], out = dims[l];
      const double* W = p;
      const double* b = p + (size_t)in * out;
      for (int o = 0; o < out; o++) {
        double acc = 0.0;
        for (int i = 0; i < in; i++) acc += (bf16 ? bf16_round(W[(size_t)o * in + i]) : W[(size_t)o * in + i]) * h[i];
        z[o] = acc + b[o];
      }
      if (acts) for (int o = 0; o < out; o++) acts[aoff + (size_t)s * out + o] = z[o];
      aoff += (size_t)n * out;
      if (l < L) {
        for (int o = 0; o < out; o++) h[o] = bf16 ? bf16_round(gelu(z[o])) : gelu(z[o]);
      } else {
        for (int o = 0; o < out; o++) Y[(size_t)s * out + o] = z[o];
      }
      p += (size_t)in * out + out;
    }
  }
  free(h);
  free(z);
}

/* Loss and its gradient with respect to every parameter (same flat layout
 * as params).  Returns the loss. */
double orc_mlp_loss_grad(int L, const int* dims, const double* params, int n, const double* X,
                         const double* Yt, int bf16, double* grad) {
  size_t nact = 0, nparam = 0;
  for (int l = 1; l <= L; l++) {
    nact += (size_t)n * dims[l];
    nparam += (size_t)dims[l - 1] * dims[l] + dims[l];
  }
  double* acts = (double*)malloc(sizeof(double) * nact);
  double* Y = (double*)malloc(sizeof(double) * (size_t)n * dims[L]);
  orc_mlp_forward(L, dims, params, n, X, bf16, Y, acts);
  for (size_t i = 0; i < nparam; i++) grad[i] = 0.0;
  const int nout = dims[L];
  const double scale = 2.0 / ((double)n * nout);
  double loss = 0.0;
  for (size_t i = 0; i < (size_t)n * nout; i++) {
    const double e = Y[i] - Yt[i];
    loss += e * e;
  }
  loss /= (double)n * nout;
  /* offsets of every layer's parameters and pre-activations */
  size_t poff[16], aoff[16];
  {
    size_t p = 0, a = 0;
    for (int l = 1; l <= L; l++) {
      poff[l] = p;
      aoff[l] = a;
      p += (size_t)dims[l - 1] * dims[l] + dims[l];
      a += (size_t)n * dims[l];
    }
  }
  int maxw = 0;
  for (int l = 0; l <= L; l++) if (dims[l] > maxw) maxw = dims[l];
  double* d = (double*)malloc(sizeof(double) * maxw);   /* dloss/dz_l */
  double* dn = (double*)malloc(sizeof(double) * maxw);
  double* hin = (double*)malloc(sizeof(double) * maxw);
  for (int s = 0; s < n; s++) {
    for (int o = 0; o < nout; o++) {
      const double g = scale * (Y[(size_t)s * nout + o] - Yt[(size_t)s * nout + o]);
      d[o] = bf16 ? bf16_round(g) : g;
    }
    for (int l = L; l >= 1; l--) {
      const int in = dims[l - 1], out = dims[l];
      /* input of layer l */
      for (int i = 0; i < in; i++) {
        double v;
        if (l == 1) v = X[(size_t)s * in + i];
        else v = gelu(acts[aoff[l - 1] + (size_t)s * in + i]);
        hin[i] = bf16 ? bf16_round(v) : v;
      }
      const double* W = params + poff[l];
      double* gW = grad + poff[l];
      double* gb = grad + poff[l] + (size_t)in * out;
      for (int o = 0; o < out; o++) {
        gb[o] += d[o];
        for (int i = 0; i < in; i++) gW[(size_t)o * in + i] += d[o] * hin[i];
      }
      if (l > 1) {
        for (int i = 0; i < in; i++) {
          double acc = 0.0;
          for (int o = 0; o < out; o++) acc += (bf16 ? bf16_round(W[(size_t)o * in + i]) : W[(size_t)o * in + i]) * d[o];
          const double g = acc * gelu_grad(acts[aoff[l - 1] + (size_t)s * in + i]);
          dn[i] = bf16 ? bf16_round(g) : g;
        }
        for (int i = 0; i < in; i++) d[i] = dn[i];
      }
    }
  }
  free(acts);
  free(Y);
  free(d);
  free(dn);
  free(hin);
  return loss;
}

/* ------------------------------------------------------------------------ */
/* Two-proposal update (learned proposal with plain MPPI as the fallback):    */
/* samples k < k_split are drawn around the nominal plan u (the warm start),  */
/* samples k >= k_split around a second plan p (the learned proposal); with   */
/* the weights of Eq. 4a the update is the weighted mean of the sampled       */
/* controls, u*_t = sum_k wbar_k (u^(k)_t + dtau_{k,t}), which is Eq. 4b when */
/* k_split = K.  Non-finite costs get weight 0; if none is finite the plan is */
/* kept and 1 is returned.                                                    */
int orc_mppi_update_mix(int K, int T, int n, const double* S, const double* noise,
                        const double* plan, const double* prop, int k_split, double lambda,
                        double* ustar, double* plan_next) {
  double Smin = INFINITY;
  for (int k = 0; k < K; k++)
    if (isfinite(S[k]) && S[k] < Smin) Smin = S[k];
  if (!isfinite(Smin)) {
    for (int i = 0; i < T * n; i++) ustar[i] = plan_next[i] = plan[i];
    return 1;
  }
  double Z = 0.0;
  for (int k = 0; k < K; k++)
    if (isfinite(S[k])) Z += exp(-(S[k] - Smin) / lambda);
  for (int i = 0; i < T * n; i++) {
    double acc = 0.0;
    for (int k = 0; k < K; k++) {
      if (!isfinite(S[k])) continue;
      const double w = exp(-(S[k] - Smin) / lambda) / Z;
      const double base = (k < k_split) ? plan[i] : prop[i];
      acc += w * (base + noise[(size_t)k * T * n + i]);
    }
    ustar[i] = acc;
  }
  for (int t = 0; t < T; t++) {
    int src = (t + 1 < T) ? t + 1 : T - 1;
    for (int j = 0; j < n; j++) plan_next[t * n + j] = ustar[src * n + j];
  }
  return 0;
}
