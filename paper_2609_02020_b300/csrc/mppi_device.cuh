// Device-side building blocks of one torque-sampling MPPI rollout (sm_103a).
//
// One thread owns one sample k and walks it through the horizon with every
// quantity in registers: the 7 links are unrolled at compile time, so all
// per-link arrays below are register arrays, never local memory.
//
// Formulation (world frame, Plucker coordinates about the world origin):
//   joint i's motion axis  S_i = (z_i, p_i x z_i)   [angular; linear at O]
//   link velocity          V_i = V_{i-1} + S_i qd_i
//   bias acceleration      A_i = A_{i-1} + V_{i-1} x S_i qd_i,  A_0 = (0, -g)
//   link force             F_i = I_i A_i + V_i x* (I_i V_i)
//   bias torque            h_i = S_i . sum_{l>=i} F_l + b_i qd_i
//   inertia (CRBA)         M_ji = S_j . (I^c_i S_i), I^c_i = sum_{l>=i} I_l,
//                          plus diag(a) (Eq. 8's armature)
// so M(q) and h(q, qd) of Eq. 5 are rebuilt at every step as the paper
// requires (Sec. III-A), and Eq. 6 is solved with an LDL^T factorisation.
// A spatial inertia about O is (m, h = m c, I_O = Ibar + m(|c|^2 1 - c c^T)),
// Ibar = R I^G R^T (the rotated link inertia of Eq. 8).
#pragma once
#include <cstdint>

namespace mppi_dev {

constexpr int NJ = 7;
// link pairs (i, j >= i + 2) of the collision cost, by i then j
constexpr int NJ_SELF_PAIRS = (NJ - 1) * (NJ - 2) / 2;

// Link constants in the kernel's link frames (z = joint axis); the host
// rotates the caller's description into these frames once, at create time.
struct LinkK {
  float F[9];   // parent kernel frame -> this joint's frame before Rz(q), row-major
  float r[3];   // joint origin in the parent kernel frame
  float c[3];   // CoM in this link's kernel frame
  float I[6];   // inertia about the CoM, kernel frame: xx yy zz xy xz yz
  float m, arm, damp;
};

struct RobotK {
  LinkK L[NJ];
  float ee[3];    // end-effector point in the last kernel frame
  float Qee[9];   // last kernel frame -> end-effector (caller's link) frame
  float qmin[NJ], qmax[NJ], qdmax[NJ], taumax[NJ];
  float g[3];
};

struct CostK {
  float wpos[3], wori[3];
  float wforce, fdes, wreg;
  float wqlim, wqdlim, wtau, wpost;
  float qpost[NJ];
  float wterm;
  int contact;
  float kc, dc;
  int fest;                            // C_force on the wrench estimate (Eq. 13)
  float wf6[6], fdes6[6], wreg6[6];    // its diagonal weights, (force; moment)
  int coll;                            // C_collision (Eq. 15): 0 off, 1 indicator, 2 hinge
  float wcoll, dth_self, dth_obs;
  float lrad[NJ];                      // link capsule radii
  float seg_a[NJ], seg_ia[NJ];         // squared link segment lengths and reciprocals
  float seg_h[NJ];                     // half link segment lengths
  float self_b2[NJ_SELF_PAIRS];        // culling bounds of the self pairs (pair_skip_b2)
};

// Obstacle capsules read by the rollouts at every launch (device memory, so
// that they can change between updates without touching kernel parameters).
constexpr int OBS_MAX = 8;
struct ObsK {
  int n;
  int pad[3];
  float o[OBS_MAX][7];  // a xyz, b xyz, radius
};

struct ProbK {
  RobotK rb;
  CostK cost;
  float dt, lambda;
  float sigma[NJ];
  int T, K;
  uint32_t key0, key1;
  const float* fext;  // device F_ext (6) of the constant external wrench, or null
};

// Per-step inputs in device memory: q, qd, goal (p, quat wxyz), plane (n, d).
constexpr int IN_FLOATS = 25;
// The kernels' shared-memory copy of the inputs: the IN_FLOATS inputs, then
// (with the constant external wrench) tau_ext = J(q_0)^T F_ext.
constexpr int IN_STAGED = 32;
constexpr int IN_TEXT = IN_FLOATS;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller normals

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// The uniform u = ((x >> 8) + 1/2) 2^-24 as uh + delta: uh the FP32 value,
// rounded where u >= 1/2 (there the sum needs 25 significant bits), and
// delta the exact rest (0 or +-2^-25), so that both sides of any comparison
// start from the same uniforms.  Every operation here and in box_muller is
// an explicitly rounded intrinsic, so that no kernel's FMA contraction can
// change a normal: all kernels draw bit-identical noise.
__device__ __forceinline__ float uniform24(uint32_t x, float& delta) {
  constexpr float SCALE = 5.9604644775390625e-8f;  // 2^-24
  const float t = static_cast<float>(x >> 8);       // exact
  const float sum = __fadd_rn(t, 0.5f);             // rounded to even when t >= 2^23
  delta = __fmul_rn(__fadd_rn(__fsub_rn(t, sum), 0.5f), SCALE);  // exact
  return __fmul_rn(sum, SCALE);
}

// Box-Muller: z0 = r cos 2 pi u2, z1 = r sin 2 pi u2, r = sqrt(-2 ln u1).
// The rests of the uniforms enter to first order (their squares are below
// 1e-14): ln u1 = ln uh1 + delta1 / uh1 (keeps small radii near u1 = 1
// right: an uh1 rounded to 1 would give r = 0), and the angle's rest
// 2 pi delta2 rotates (cos, sin).
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
  float da, db;
  const float ua = uniform24(a, da), ub = uniform24(b, db);
  const float ln_u = __fadd_rn(logf(ua), __fmul_rn(da, __frcp_rn(ua)));
  const float r = sqrtf(__fmul_rn(-2.0f, ln_u));
  float s, c;
  sincospif(__fmul_rn(2.0f, ub), &s, &c);
  const float e = __fmul_rn(6.28318530717958648f, db);
  z0 = __fmul_rn(r, fmaf(-e, s, c));
  z1 = __fmul_rn(r, fmaf(e, c, s));
}

// Normals 4 call .. 4 call + 3 of (sample k, step t, update iter): one
// Philox4x32-10 call, two Box-Muller pairs.
__device__ __forceinline__ void normals4(uint32_t k0, uint32_t k1, uint64_t iter, uint32_t k,
                                         uint32_t t, uint32_t call, float z[4]) {
  uint32_t c[4] = {k, 2u * t + call, static_cast<uint32_t>(iter),
                   static_cast<uint32_t>(iter >> 32)};
  philox4x32_10(c, k0, k1);
  box_muller(c[0], c[1], z[0], z[1]);
  box_muller(c[2], c[3], z[2], z[3]);
}

// The 8 normals of (sample k, step t, update iter); joints use z[0..6].
__device__ __forceinline__ void normals8(uint32_t k0, uint32_t k1, uint64_t iter, uint32_t k,
                                         uint32_t t, float z[8]) {
  normals4(k0, k1, iter, k, t, 0u, z);
  normals4(k0, k1, iter, k, t, 1u, z + 4);
}

// ---------------------------------------------------------------------------
// small vector helpers

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
  return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}
// y = R x, R row-major 3x3
__device__ __forceinline__ void mv3(const float R[9], const float x[3], float y[3]) {
  y[0] = fmaf(R[0], x[0], fmaf(R[1], x[1], R[2] * x[2]));
  y[1] = fmaf(R[3], x[0], fmaf(R[4], x[1], R[5] * x[2]));
  y[2] = fmaf(R[6], x[0], fmaf(R[7], x[1], R[8] * x[2]));
}
// C = A B (3x3 row-major)
__device__ __forceinline__ void mm3(const float A[9], const float B[9], float Cm[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Cm[3 * i + j] = fmaf(A[3 * i], B[j], fmaf(A[3 * i + 1], B[3 + j], A[3 * i + 2] * B[6 + j]));
}

// Spatial inertia about O applied to a motion vector (w, v):
// H = I_O w + h x v,  L = m v - h x w.   In = (m, h0..2, Ixx Iyy Izz Ixy Ixz Iyz)
__device__ __forceinline__ void inertia_apply(const float In[10], const float w[3],
                                              const float v[3], float H[3], float L[3]) {
  const float m = In[0];
  const float h[3] = {In[1], In[2], In[3]};
  float hv[3], hw[3];
  cross3(h, v, hv);
  cross3(h, w, hw);
  H[0] = fmaf(In[4], w[0], fmaf(In[7], w[1], fmaf(In[8], w[2], hv[0])));
  H[1] = fmaf(In[7], w[0], fmaf(In[5], w[1], fmaf(In[9], w[2], hv[1])));
  H[2] = fmaf(In[8], w[0], fmaf(In[9], w[1], fmaf(In[6], w[2], hv[2])));
  L[0] = fmaf(m, v[0], -hw[0]);
  L[1] = fmaf(m, v[1], -hw[1]);
  L[2] = fmaf(m, v[2], -hw[2]);
}

// Per-link results of the forward sweep kept for the backward sweep.
struct LinkState {
  float z[3];   // joint axis (world)
  float w[3];   // p_i x z_i (linear part of S_i)
  float F[6];   // RNEA link force (moment about O; force)
  float In[10]; // spatial inertia about O
};

struct EEState {
  float p[3];   // end-effector position
  float R[9];   // end-effector orientation (row-major)
  float v[3];   // end-effector linear velocity
};

// Recursion state carried from link to link by the forward sweep.
struct ChainState {
  float R[9];          // world rotation of the current link frame
  float p[3];          // world position of the current joint
  float Vw[3], Vv[3];  // spatial velocity (angular; linear at O)
  float Aw[3], Av[3];  // spatial bias acceleration
};

__device__ __forceinline__ void chain_init(const RobotK& rb, ChainState& c) {
#pragma unroll
  for (int a = 0; a < 9; ++a) c.R[a] = (a % 4 == 0) ? 1.f : 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    c.p[a] = 0.f;
    c.Vw[a] = c.Vv[a] = c.Aw[a] = 0.f;
    c.Av[a] = -rb.g[a];
  }
}

// sin and cos of a joint angle, branch-free: Cody-Waite reduction by pi/2
// in three parts (Cody and Waite, Software Manual for the Elementary
// Functions, 1980), each part taken off with one fused multiply-add, then the
// Taylor series of sin and cos on |r| <= pi/4 up to r^9 and r^10 (truncation
// below 2e-9) and the quadrant's swap and signs.  Absolute error below
// 7e-8 for |x| < 1e4 (checked against FP64 sin and cos), and the reduction
// stays exact to that level while k = rint(2x/pi) < 2^20.
__device__ __forceinline__ void joint_sincos(float x, float& s, float& c) {
  const float k = rintf(x * 0.636619746685028076f);
  float r = fmaf(-k, 1.57079637050628662f, x);
  r = fmaf(-k, -4.37113882867379e-8f, r);
  r = fmaf(-k, -1.71512451000588e-15f, r);
  const float r2 = r * r;
  float ps = fmaf(r2, 2.75573188446e-6f, -1.98412701138e-4f);
  ps = fmaf(ps, r2, 8.33333376795e-3f);
  ps = fmaf(ps, r2, -1.66666671634e-1f);
  const float sr = fmaf(ps * r2, r, r);
  float pc = fmaf(r2, -2.75573199815e-7f, 2.48015876423e-5f);
  pc = fmaf(pc, r2, -1.38888892252e-3f);
  pc = fmaf(pc, r2, 4.16666679084e-2f);
  pc = fmaf(pc, r2, -0.5f);
  const float cr = fmaf(pc, r2, 1.0f);
  const int ki = static_cast<int>(k);
  const float sa = (ki & 1) ? cr : sr, ca = (ki & 1) ? sr : cr;
  s = (ki & 2) ? -sa : sa;
  c = ((ki + 1) & 2) ? -ca : ca;
}

// Frame of link i in the forward sweep: world rotation and origin of link
// i's frame, joint axis z and w = p x z.
__device__ __forceinline__ void forward_link_frame(const LinkK& L, float qi, ChainState& c,
                                                   float z[3], float w[3]) {
  float d[3];
  mv3(c.R, L.r, d);
  c.p[0] += d[0]; c.p[1] += d[1]; c.p[2] += d[2];
  float RF[9];
  mm3(c.R, L.F, RF);
  float s, co;
  joint_sincos(qi, s, co);
  // R = RF * Rz(q): columns 0 and 1 rotate, column 2 is the joint axis
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float c0 = RF[3 * r], c1 = RF[3 * r + 1];
    c.R[3 * r] = fmaf(co, c0, s * c1);
    c.R[3 * r + 1] = fmaf(co, c1, -s * c0);
    c.R[3 * r + 2] = RF[3 * r + 2];
  }
  z[0] = c.R[2]; z[1] = c.R[5]; z[2] = c.R[8];
  cross3(c.p, z, w);
}

// Spatial velocity and bias acceleration after a joint with motion axis
// (z, w) and speed qdi.
__device__ __forceinline__ void forward_link_motion(const float z[3], const float w[3], float qdi,
                                                    float Vw[3], float Vv[3], float Aw[3],
                                                    float Av[3]) {
  const float jw[3] = {z[0] * qdi, z[1] * qdi, z[2] * qdi};
  const float jv[3] = {w[0] * qdi, w[1] * qdi, w[2] * qdi};
  float t0[3], t1[3], t2[3];
  cross3(Vw, jw, t0);  // (V x S qd) angular
  cross3(Vw, jv, t1);
  cross3(Vv, jw, t2);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Aw[a] += t0[a];
    Av[a] += t1[a] + t2[a];
    Vw[a] += jw[a];
    Vv[a] += jv[a];
  }
}

// Chain part of one link of the forward sweep: the frame, then the velocity
// and bias acceleration after link i.
__device__ __forceinline__ void forward_link_chain(const LinkK& L, float qi, float qdi,
                                                   ChainState& c, float z[3], float w[3]) {
  forward_link_frame(L, qi, c, z, w);
  forward_link_motion(z, w, qdi, c.Vw, c.Vv, c.Aw, c.Av);
}

// Force part of one link of the forward sweep, from the link frame (R, p)
// and the link's spatial velocity V = (Vw, Vv) and bias acceleration
// A = (Aw, Av): the link spatial inertia about O and the RNEA link force
// F = I A + V x* (I V).
__device__ __forceinline__ void forward_link_force(const LinkK& L, const float R[9],
                                                   const float p[3], const float Vw[3],
                                                   const float Vv[3], const float Aw[3],
                                                   const float Av[3], float In[10], float F[6]) {
  float cw[3];
  mv3(R, L.c, cw);
  cw[0] += p[0]; cw[1] += p[1]; cw[2] += p[2];
  // Ibar = R I R^T via T = R I (I symmetric)
  float Tm[9];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    Tm[3 * r + 0] = fmaf(R[3 * r], L.I[0], fmaf(R[3 * r + 1], L.I[3], R[3 * r + 2] * L.I[4]));
    Tm[3 * r + 1] = fmaf(R[3 * r], L.I[3], fmaf(R[3 * r + 1], L.I[1], R[3 * r + 2] * L.I[5]));
    Tm[3 * r + 2] = fmaf(R[3 * r], L.I[4], fmaf(R[3 * r + 1], L.I[5], R[3 * r + 2] * L.I[2]));
  }
  const float m = L.m;
  const float cc = dot3(cw, cw);
  In[0] = m;
  In[1] = m * cw[0]; In[2] = m * cw[1]; In[3] = m * cw[2];
  In[4] = fmaf(Tm[0], R[0], fmaf(Tm[1], R[1], Tm[2] * R[2])) + m * (cc - cw[0] * cw[0]);
  In[5] = fmaf(Tm[3], R[3], fmaf(Tm[4], R[4], Tm[5] * R[5])) + m * (cc - cw[1] * cw[1]);
  In[6] = fmaf(Tm[6], R[6], fmaf(Tm[7], R[7], Tm[8] * R[8])) + m * (cc - cw[2] * cw[2]);
  In[7] = fmaf(Tm[0], R[3], fmaf(Tm[1], R[4], Tm[2] * R[5])) - m * cw[0] * cw[1];
  In[8] = fmaf(Tm[0], R[6], fmaf(Tm[1], R[7], Tm[2] * R[8])) - m * cw[0] * cw[2];
  In[9] = fmaf(Tm[3], R[6], fmaf(Tm[4], R[7], Tm[5] * R[8])) - m * cw[1] * cw[2];
  // F = I A + V x* (I V)
  float HA[3], LA[3], HV[3], LV[3];
  inertia_apply(In, Aw, Av, HA, LA);
  inertia_apply(In, Vw, Vv, HV, LV);
  float a0[3], a1[3], a2[3];
  cross3(Vw, HV, a0);
  cross3(Vv, LV, a1);
  cross3(Vw, LV, a2);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    F[a] = HA[a] + a0[a] + a1[a];
    F[3 + a] = LA[a] + a2[a];
  }
}

// One link of the forward sweep: joint transform, link spatial inertia about
// O, velocity, bias acceleration and the RNEA link force.
__device__ __forceinline__ void forward_link(const LinkK& L, float qi, float qdi, ChainState& c,
                                             LinkState& S) {
  forward_link_chain(L, qi, qdi, c, S.z, S.w);
  forward_link_force(L, c.R, c.p, c.Vw, c.Vv, c.Aw, c.Av, S.In, S.F);
}

// End-effector pose and linear velocity from the last link's chain state.
__device__ __forceinline__ void chain_ee(const RobotK& rb, const ChainState& c, EEState& ee) {
  float de[3];
  mv3(c.R, rb.ee, de);
  ee.p[0] = c.p[0] + de[0]; ee.p[1] = c.p[1] + de[1]; ee.p[2] = c.p[2] + de[2];
  mm3(c.R, rb.Qee, ee.R);
  float wp[3];
  cross3(c.Vw, ee.p, wp);
  ee.v[0] = c.Vv[0] + wp[0]; ee.v[1] = c.Vv[1] + wp[1]; ee.v[2] = c.Vv[2] + wp[2];
}

// End-effector position and linear velocity only (as chain_ee computes them).
__device__ __forceinline__ void chain_ee_pv(const RobotK& rb, const ChainState& c, EEState& ee) {
  float de[3];
  mv3(c.R, rb.ee, de);
  ee.p[0] = c.p[0] + de[0]; ee.p[1] = c.p[1] + de[1]; ee.p[2] = c.p[2] + de[2];
  float wp[3];
  cross3(c.Vw, ee.p, wp);
  ee.v[0] = c.Vv[0] + wp[0]; ee.v[1] = c.Vv[1] + wp[1]; ee.v[2] = c.Vv[2] + wp[2];
}

// Forward sweep at state (q, qd): kinematics (Fig. 1), RNEA forward
// recursion with qdd = 0, end-effector pose and velocity.
__device__ __forceinline__ void forward_sweep(const RobotK& rb, const float q[NJ],
                                              const float qd[NJ], LinkState ls[NJ], EEState& ee) {
  ChainState c;
  chain_init(rb, c);
#pragma unroll
  for (int i = 0; i < NJ; ++i) forward_link(rb.L[i], q[i], qd[i], c, ls[i]);
  chain_ee(rb, c, ee);
}

// One link of the backward sweep: accumulate the suffix force Fs and the
// composite inertia Ic; return the bias torque h_i and the composite
// momentum (H, Lm) of S_i, from which M_ji = S_j . (H, Lm) for j <= i.
__device__ __forceinline__ float backward_link(const LinkK& L, float qdi, const LinkState& S,
                                               float Fs[6], float Ic[10], float H[3],
                                               float Lm[3]) {
#pragma unroll
  for (int a = 0; a < 6; ++a) Fs[a] += S.F[a];
#pragma unroll
  for (int a = 0; a < 10; ++a) Ic[a] += S.In[a];
  const float h = fmaf(L.damp, qdi,
                       dot3(S.z, Fs) + fmaf(S.w[0], Fs[3], fmaf(S.w[1], Fs[4], S.w[2] * Fs[5])));
  inertia_apply(Ic, S.z, S.w, H, Lm);
  return h;
}

// Backward sweep: bias torque h (incl. damping) and the joint-space inertia
// M (lower triangle, packed row-major: M[i(i+1)/2 + j], j <= i) incl. armature.
__device__ __forceinline__ void backward_sweep(const RobotK& rb, const float qd[NJ],
                                               const LinkState ls[NJ], float h[NJ],
                                               float M[NJ * (NJ + 1) / 2]) {
  float Fs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float Ic[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = NJ - 1; i >= 0; --i) {
    float H[3], Lm[3];
    h[i] = backward_link(rb.L[i], qd[i], ls[i], Fs, Ic, H, Lm);
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const LinkState& Sj = ls[j];
      M[i * (i + 1) / 2 + j] = dot3(Sj.z, H) + dot3(Sj.w, Lm);
    }
    M[i * (i + 1) / 2 + i] += rb.L[i].arm;
  }
}

// LDL^T factorisation of an N x N symmetric positive definite matrix in
// packed lower-triangle storage (M[i(i+1)/2 + j], j <= i): overwrites the
// strict lower triangle with L (unit diagonal implied) and returns 1/D.
// Every loop has a constant trip count (bounds are guards) so that the
// factorisation unrolls completely and M stays in registers.  With
// FAST_RCP the pivots' reciprocals take the hardware approximation
// (__fdividef, about 2 ulp; the pivots are far from its 2^126 limit), which
// shortens the dependent chain of the factorisation.
template <int N, bool FAST_RCP = false>
__device__ __forceinline__ void ldlt_factor(float M[N * (N + 1) / 2], float invD[N]) {
  float D[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    // column j: D_j = M_jj - sum_k L_jk^2 D_k ; L_ij = (M_ij - sum_k L_ik L_jk D_k) / D_j
    float LD[N];  // L_jk D_k
    float d = M[j * (j + 1) / 2 + j];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (k < j) {
        const float Ljk = M[j * (j + 1) / 2 + k];
        LD[k] = Ljk * D[k];
        d = fmaf(-Ljk, LD[k], d);
      }
    }
    D[j] = d;
    invD[j] = FAST_RCP ? __fdividef(1.0f, d) : 1.0f / d;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (i > j) {
        float s = M[i * (i + 1) / 2 + j];
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k < j) s = fmaf(-M[i * (i + 1) / 2 + k], LD[k], s);
        M[i * (i + 1) / 2 + j] = s * invD[j];
      }
    }
  }
}

// y = L^-1 b for the unit lower factor L of ldlt_factor.
template <int N>
__device__ __forceinline__ void unit_lower_solve(const float L[N * (N + 1) / 2], const float b[N],
                                                 float y[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s = b[i];
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (k < i) s = fmaf(-L[i * (i + 1) / 2 + k], y[k], s);
    y[i] = s;
  }
}

// x = L^-T D^-1 y (the second half of an LDL^T solve).
template <int N>
__device__ __forceinline__ void ldlt_back(const float L[N * (N + 1) / 2], const float invD[N],
                                          const float y[N], float x[N]) {
#pragma unroll
  for (int ii = 0; ii < N; ++ii) {
    const int i = N - 1 - ii;
    float s = y[i] * invD[i];
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (k > i) s = fmaf(-L[k * (k + 1) / 2 + i], x[k], s);
    x[i] = s;
  }
}

// Solve M x = b with M symmetric positive definite (packed lower triangle),
// by LDL^T.  Overwrites M with the factors.
__device__ __forceinline__ void ldlt_solve(float M[NJ * (NJ + 1) / 2], const float b[NJ],
                                           float x[NJ]) {
  float invD[NJ], y[NJ];
  ldlt_factor<NJ>(M, invD);
  unit_lower_solve<NJ>(M, b, y);
  ldlt_back<NJ>(M, invD, y, x);
}

// ---------------------------------------------------------------------------
// Semi-implicit Euler step of Eq. 7 on a compensated state.  Each of q and qd
// is carried as an unevaluated sum hi + lo of two floats: hi is the nearest
// float of the state and the one the dynamics and costs see; lo is the
// rounding error of the last addition, recovered by Dekker's Fast2Sum and
// folded into the next step's increment.  Plain FP32 would round q to half
// an ulp (about 1e-7 rad) at every step, and over a horizon that rounding,
// fed back through the dynamics, is the largest error of an FP32 rollout
// against an exact one.  Fast2Sum is exact when |hi| >= |increment|; where
// it is not (a state near zero), the part it misses is below half an ulp of
// the increment (under 3e-8 rad/s for qd, 2e-9 rad for q).  Every operation
// is explicitly rounded, so that no FMA contraction breaks the recovery.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// qd' = qd + qdd dt, q' = q + qd' dt (Eq. 7) on (hi, lo) pairs.
__device__ __forceinline__ void euler_step(float qdd, float dt, float& q, float& q_lo, float& qd,
                                           float& qd_lo) {
  fast_two_sum(qd, __fmaf_rn(qdd, dt, qd_lo), qd, qd_lo);
  fast_two_sum(q, __fmaf_rn(qd, dt, __fmaf_rn(qd_lo, dt, q_lo)), q, q_lo);
}

// ---------------------------------------------------------------------------
// costs (Eq. 9-12, 14)

__device__ __forceinline__ float hinge2(float x) { return x > 0.f ? x * x : 0.f; }

// goal rotation matrix from the (normalised) quaternion wxyz
__device__ __forceinline__ void quat_to_R(const float qt[4], float R[9]) {
  const float n = rsqrtf(qt[0] * qt[0] + qt[1] * qt[1] + qt[2] * qt[2] + qt[3] * qt[3]);
  const float w = qt[0] * n, x = qt[1] * n, y = qt[2] * n, z = qt[3] * n;
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// C_motion (Eq. 11): weighted squared position error plus weighted squared
// rotation vector of R_des^T R_ee.
__device__ __forceinline__ float motion_cost(const CostK& c, const float pdes[3],
                                             const float Rd[9], const EEState& ee) {
  // E = Rd^T Re: E_ab = sum_r Rd[r][a] Re[r][b]
  auto E = [&](int a, int b) {
    return fmaf(Rd[a], ee.R[b], fmaf(Rd[3 + a], ee.R[3 + b], Rd[6 + a] * ee.R[6 + b]));
  };
  const float vx = E(2, 1) - E(1, 2), vy = E(0, 2) - E(2, 0), vz = E(1, 0) - E(0, 1);
  const float tr = E(0, 0) + E(1, 1) + E(2, 2);
  const float s2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
  const float s = 0.5f * sqrtf(s2);
  const float cth = 0.5f * (tr - 1.f);
  const float th = atan2f(s, cth);
  float r0, r1, r2;
  if (s > 1e-4f) {
    const float k = th / (2.f * s);
    r0 = k * vx; r1 = k * vy; r2 = k * vz;
  } else if (cth > 0.f) {
    r0 = 0.5f * vx; r1 = 0.5f * vy; r2 = 0.5f * vz;
  } else {
    // theta near pi: axis from the symmetric part B = (E + E^T)/2 - cos(th) 1
    const float B00 = E(0, 0) - cth, B11 = E(1, 1) - cth, B22 = E(2, 2) - cth;
    const float B01 = 0.5f * (E(0, 1) + E(1, 0)), B02 = 0.5f * (E(0, 2) + E(2, 0)),
                B12 = 0.5f * (E(1, 2) + E(2, 1));
    float a0, a1, a2;
    if (B00 >= B11 && B00 >= B22) { a0 = B00; a1 = B01; a2 = B02; }
    else if (B11 >= B22) { a0 = B01; a1 = B11; a2 = B12; }
    else { a0 = B02; a1 = B12; a2 = B22; }
    const float inv = rsqrtf(fmaf(a0, a0, fmaf(a1, a1, a2 * a2)));
    a0 *= inv; a1 *= inv; a2 *= inv;
    if (fmaf(a0, vx, fmaf(a1, vy, a2 * vz)) < 0.f) { a0 = -a0; a1 = -a1; a2 = -a2; }
    r0 = th * a0; r1 = th * a1; r2 = th * a2;
  }
  const float ex = pdes[0] - ee.p[0], ey = pdes[1] - ee.p[1], ez = pdes[2] - ee.p[2];
  float cst = c.wpos[0] * ex * ex + c.wpos[1] * ey * ey + c.wpos[2] * ez * ez;
  cst += c.wori[0] * r0 * r0 + c.wori[1] * r1 * r1 + c.wori[2] * r2 * r2;
  return cst;
}

// Squared distance between the segments p1 + s d1 and p2 + t d2, s, t in
// [0, 1], for Eq. 15 by Lumelsky's method (Inf. Process. Lett. 21, 1985):
// the closest point of the infinite lines, s clamped to [0, 1]; t follows
// from s and, when it leaves [0, 1], is clamped and s recomputed against
// that end point.  a = |d1|^2, e = |d2|^2 and their reciprocals ia, ie are
// given (0 for a point segment, which takes the one-sided projection), so
// that one division remains per pair.
__device__ __forceinline__ float segment_dist2(const float p1[3], const float d1[3], float a,
                                               float ia, const float p2[3], const float d2[3],
                                               float e, float ie) {
  const float r[3] = {p1[0] - p2[0], p1[1] - p2[1], p1[2] - p2[2]};
  const float f = dot3(d2, r), c = dot3(d1, r), b = dot3(d1, d2);
  float s, t;
  if (ia == 0.f) {
    s = 0.f;
    t = __saturatef(f * ie);
  } else if (ie == 0.f) {
    t = 0.f;
    s = __saturatef(-c * ia);
  } else {
    const float den = fmaf(a, e, -b * b);
    s = den > 0.f ? __saturatef(__fdividef(fmaf(b, f, -c * e), den)) : 0.f;
    t = fmaf(b, s, f) * ie;
    if (t < 0.f) {
      t = 0.f;
      s = __saturatef(-c * ia);
    } else if (t > 1.f) {
      t = 1.f;
      s = __saturatef((b - c) * ia);
    }
  }
  float g[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) g[k] = fmaf(s, d1[k], r[k]) - t * d2[k];
  return dot3(g, g);
}

// Culling of a collision pair, exact: the distance of two segments is at
// least |m_1 - m_2| - h_1 - h_2 (midpoints m, half lengths h), and the pair's
// term of Eq. 15 is zero unless the distance is below D = th + r_1 + r_2.
// A pair may therefore be skipped when |m_1 - m_2|^2 >= b2 =
// ((D + h_1 + h_2)(1 + 1e-4) + 1e-5)^2 (lengths in m): the margins exceed
// the FP32 rounding of both distances (segment_dist2 evaluates the distance
// of two points on the segments, never below the segments' distance by more
// than a few 1e-7 m), so a skipped pair is one whose term the full
// evaluation also finds zero.  With D <= 0 no term is ever charged (b2 = -1:
// always skipped).
__host__ __device__ inline float pair_skip_b2(float th, float r1, float r2, float h1, float h2) {
  const float D = th + r1 + r2;
  if (!(D > 0.f)) return -1.f;
  const float b = (D + h1 + h2) * 1.0001f + 1e-5f;
  return b * b;
}

// tau_ext = J(q0)^T F_ext for the external wrench F = (force f; moment m
// about the end-effector point), world frame (Eq. 5, constant over the
// horizon): with the joint axes S_j = (z_j, w_j = p_j x z_j) and the
// wrench's moment about the origin n_O = m + p_ee x f, tau_j = z_j . n_O +
// w_j . f.  One thread forms it for its block; not on the per-step path.
static __device__ __noinline__ void ext_torque(const RobotK& rb, const float* q0, const float* F,
                                               float* tau) {
  ChainState c;
  chain_init(rb, c);
  float z[NJ][3], w[NJ][3];
#pragma unroll 1
  for (int i = 0; i < NJ; ++i) forward_link_frame(rb.L[i], q0[i], c, z[i], w[i]);
  float de[3], p[3];
  mv3(c.R, rb.ee, de);
  p[0] = c.p[0] + de[0]; p[1] = c.p[1] + de[1]; p[2] = c.p[2] + de[2];
  const float f[3] = {F[0], F[1], F[2]};
  float nO[3];
  cross3(p, f, nO);
  nO[0] += F[3]; nO[1] += F[4]; nO[2] += F[5];
#pragma unroll 1
  for (int j = 0; j < NJ; ++j) tau[j] = dot3(z[j], nO) + dot3(w[j], f);
}

// Plane contact normal force at the end-effector (0 without contact).
__device__ __forceinline__ float contact_force(const CostK& c, const float plane[4],
                                               const EEState& ee) {
  const float delta = plane[3] - dot3(plane, ee.p);
  if (!(delta > 0.f)) return 0.f;
  const float vn = dot3(plane, ee.v);
  return fmaxf(0.f, fmaf(c.kc, delta, -c.dc * vn));
}

}  // namespace mppi_dev
