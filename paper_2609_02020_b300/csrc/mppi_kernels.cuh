// Kernels of one MPPI update (sm_103a):
//   rollout_kernel, rollout_kernel_rolled, rollout_kernel_ws
//                   - Eq. 1-3 with Eq. 5-7 and the running cost of Eq. 9-14
//                     (register-unrolled, one thread per sample; link loops
//                     rolled through shared memory; three warps per 32
//                     samples);
//   merge_kernel    - Eq. 4a-4b and the warm-start shift of a step: one block
//                     per plan entry (t, j) merging the rollout blocks'
//                     log-sum-exp partials (block_partial);
//   update_kernel   - Eq. 4a-4b and the shift from caller-supplied costs and
//                     noise, one block per plan entry reducing over all K.
#pragma once
#include <cfloat>
#include <cstdint>

#include "mppi_device.cuh"

namespace mppi_dev {

constexpr int T_MAX = 256;
constexpr int ROLLOUT_BLOCK = 32;
constexpr int UPDATE_BLOCK = 256;

// A rollout block's results are written: the update kernel, launched as a
// programmatic dependent, may start to launch (it still waits for this
// grid's completion before it reads them).
__device__ __forceinline__ void allow_dependent_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Wait for the completion of the grid this one was launched as a
// programmatic dependent of, and for its memory operations (no-op for a
// grid launched without that attribute).
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// atomicAdd with acquire-release semantics at GPU scope
__device__ __forceinline__ unsigned atomic_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
               : "=r"(old)
               : "l"(p), "r"(v)
               : "memory");
  return old;
}

template <typename V>
__device__ __forceinline__ V warp_sum(V x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ float warp_min(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// Log-sum-exp partials of one rollout block (the sharded form of Eq. 4: a
// block's share of the update, merged over blocks by merge_kernel).  Record
// of PART_HEAD + T*7 floats (stride part_stride(T)):
//   [0] m_b = min of the block's finite costs (+inf if none)
//   [1] Z_b = sum_k w_k, w_k = exp(-(S_k - m_b) / lambda), 0 for non-finite S_k
//   [2] sum_k w_k^2                      [3] sum of w_k over k >= k_split
//   [4] number of non-finite costs       [PART_HEAD + e] N_b[e] = sum_k w_k dtau_{k,e}
constexpr int PART_HEAD = 8;
__host__ __device__ constexpr int part_stride(int T) { return (PART_HEAD + T * NJ + 3) / 4 * 4; }

// Every thread of a block of NT threads calls it after the block's n costs
// (samples k0 .. k0 + n - 1, n <= 32) are in s_S[0..n); the block's noise
// dtau[T*7][K] was written earlier in the same kernel and is read back
// through L2 (ld.global.cg), 32 samples x 4 B per plan entry.
template <int NT>
__device__ __forceinline__ void block_partial(const float* s_S, float* s_w, int k0, int n, int K,
                                              int T, float lambda, int k_split, const float* noise,
                                              float* part) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    const float sk = l < n ? s_S[l] : 0.f;
    const bool fin = l < n && isfinite(sk);
    const float m = warp_min(fin ? sk : INFINITY);
    const float w = fin ? expf((m - sk) * (1.0f / lambda)) : 0.f;
    s_w[l] = w;
    const float z = warp_sum(w), z2 = warp_sum(w * w);
    const float zs = warp_sum(k0 + l >= k_split ? w : 0.f);
    const unsigned bad = __popc(__ballot_sync(0xffffffffu, l < n && !fin));
    if (l == 0) {
      part[0] = m;
      part[1] = z;
      part[2] = z2;
      part[3] = zs;
      part[4] = static_cast<float>(bad);
    }
  }
  __syncthreads();
  const int E = T * NJ;
  const bool vec = n == 32 && (K & 3) == 0;
  for (int e = threadIdx.x; e < E; e += NT) {
    const float* row = noise + static_cast<size_t>(e) * K + k0;
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    if (vec) {
      float4 v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = __ldcg(reinterpret_cast<const float4*>(row) + i);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        a[0] = fmaf(s_w[4 * i], v[i].x, a[0]);
        a[1] = fmaf(s_w[4 * i + 1], v[i].y, a[1]);
        a[2] = fmaf(s_w[4 * i + 2], v[i].z, a[2]);
        a[3] = fmaf(s_w[4 * i + 3], v[i].w, a[3]);
      }
    } else {
      for (int l = 0; l < n; ++l) a[l & 3] = fmaf(s_w[l], __ldcg(row + l), a[l & 3]);
    }
    part[PART_HEAD + e] = (a[0] + a[1]) + (a[2] + a[3]);
  }
}

// Offsets in the per-handle output record (floats): tau0, status, stats.
constexpr int OUT_TAU0 = 0;
constexpr int OUT_STATUS = 7;   // written as an int: 0 ok, 1 no finite cost
constexpr int OUT_STATS = 8;    // S_min, Z, n_eff, n_nonfinite
constexpr int OUT_SEQ = 12;     // host steps: the step's sequence word, written last
constexpr int OUT_PLAN = 16;    // shifted plan [T][7]

// Copies the inputs into the block's staged record (IN_STAGED floats) and,
// with the constant external wrench, forms tau_ext = J(q_0)^T F_ext after
// them (thread 0); the caller synchronises the block before use.
__device__ __forceinline__ void stage_inputs(const ProbK& P, const float* in, float* s_in) {
  if (threadIdx.x < IN_FLOATS) s_in[threadIdx.x] = in[threadIdx.x];
  if (P.fext && threadIdx.x == 0) ext_torque(P.rb, in, P.fext, s_in + IN_TEXT);
}

// One rollout (sample k of T steps) of the problem P: Eq. 1-3 with Eq. 5-7
// and the running cost of Eq. 9-14.  in: IN_FLOATS inputs and plan: [T][7]
// nominal torques (both usually staged in shared memory); returns S_k and,
// when STORE_NOISE, writes dtau to noise[(t*7 + j) * K + k].
template <bool STORE_NOISE>
__device__ __forceinline__ float rollout_sample(const ProbK& P, const float* in, const float* plan,
                                                uint64_t iter, int k, float* __restrict__ noise) {
  const int T = P.T, K = P.K;
  float q[NJ], qd[NJ], q_lo[NJ], qd_lo[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    q[j] = in[j];
    qd[j] = in[NJ + j];
    q_lo[j] = qd_lo[j] = 0.f;
  }
  const float pdes[3] = {in[14], in[15], in[16]};
  float Rd[9];
  {
    const float qt[4] = {in[17], in[18], in[19], in[20]};
    quat_to_R(qt, Rd);
  }
  const float plane[4] = {in[21], in[22], in[23], in[24]};
  const CostK& C = P.cost;
  const bool contact = C.contact != 0;

  LinkState ls[NJ];
  EEState ee;
  forward_sweep(P.rb, q, qd, ls, ee);
  float f = contact ? contact_force(C, plane, ee) : 0.f;
  double Sacc = 0.0;

  for (int t = 0; t < T; ++t) {
    // Eq. 2: v = u + dtau
    float z[8];
    normals8(P.key0, P.key1, iter, static_cast<uint32_t>(k), static_cast<uint32_t>(t), z);
    float v[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float du = P.sigma[j] * z[j];
      if (STORE_NOISE) noise[static_cast<size_t>(t * NJ + j) * K + k] = du;
      v[j] = plan[t * NJ + j] + du;
    }
    // Eq. 5-6: qdd = M^-1 (v + J^T F_ext - h)
    float h[NJ], M[NJ * (NJ + 1) / 2];
    backward_sweep(P.rb, qd, ls, h, M);
    float rhs[NJ];
    if (contact && f > 0.f) {
      const float Fc[3] = {f * plane[0], f * plane[1], f * plane[2]};
      float pxF[3];
      cross3(ee.p, Fc, pxF);
#pragma unroll
      for (int j = 0; j < NJ; ++j) rhs[j] = v[j] + dot3(ls[j].z, pxF) + dot3(ls[j].w, Fc) - h[j];
    } else {
#pragma unroll
      for (int j = 0; j < NJ; ++j) rhs[j] = v[j] - h[j];
    }
    if (P.fext) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) rhs[j] += in[IN_TEXT + j];
    }
    float qdd[NJ];
    ldlt_solve(M, rhs, qdd);
    // Eq. 7: semi-implicit Euler (compensated)
    const float dt = P.dt;
#pragma unroll
    for (int j = 0; j < NJ; ++j) euler_step(qdd[j], dt, q[j], q_lo[j], qd[j], qd_lo[j]);
    // kinematics and RNEA forward sweep at x_{t+1} (reused by step t+1)
    forward_sweep(P.rb, q, qd, ls, ee);
    // running cost l(x_{t+1}, v_t), Eq. 9-14
    float cst = motion_cost(C, pdes, Rd, ee);
    if (contact) {
      f = contact_force(C, plane, ee);
      const float e = C.fdes - f;
      cst += C.wforce * e * e + C.wreg * f * f;
    }
    float cj = 0.f;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      cj += C.wqlim * (hinge2(q[j] - P.rb.qmax[j]) + hinge2(P.rb.qmin[j] - q[j]));
      cj += C.wqdlim * hinge2(fabsf(qd[j]) - P.rb.qdmax[j]);
      const float e = q[j] - C.qpost[j];
      cj += C.wpost * e * e;
      cj += C.wtau * hinge2(fabsf(v[j]) - P.rb.taumax[j]);
    }
    Sacc += static_cast<double>(cst) + static_cast<double>(cj);
  }
  if (C.wterm != 0.f) Sacc += static_cast<double>(C.wterm * motion_cost(C, pdes, Rd, ee));
  return static_cast<float>(Sacc);
}

// One rollout per thread.  plan: [T][7] nominal torques; in: IN_FLOATS
// inputs; iter: update counter (device); S: [K] costs; noise: [T*7][K].
// Samples k < k_split roll out around plan; samples k >= k_split around the
// second proposal prop (ksplit_p null: every sample around plan).  part
// (with STORE_NOISE): each block's log-sum-exp partials (block_partial).
template <bool STORE_NOISE>
__global__ void __launch_bounds__(ROLLOUT_BLOCK)
rollout_kernel(const __grid_constant__ ProbK P, const float* __restrict__ in,
               const unsigned long long* __restrict__ iter_p, const float* __restrict__ plan,
               float* __restrict__ S, float* __restrict__ noise,
               const float* __restrict__ prop = nullptr, const int* __restrict__ ksplit_p = nullptr,
               float* __restrict__ part = nullptr) {
  __shared__ float s_plan[T_MAX * NJ];
  __shared__ float s_prop[T_MAX * NJ];
  __shared__ float s_in[IN_STAGED];
  const int T = P.T, K = P.K;
  const int k_split = ksplit_p ? *ksplit_p : K;
  for (int i = threadIdx.x; i < T * NJ; i += blockDim.x) s_plan[i] = plan[i];
  if (k_split < K)
    for (int i = threadIdx.x; i < T * NJ; i += blockDim.x) s_prop[i] = prop[i];
  stage_inputs(P, in, s_in);
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  float sk = 0.f;
  if (k < K) {
    sk = rollout_sample<STORE_NOISE>(P, s_in, k < k_split ? s_plan : s_prop, *iter_p, k, noise);
    S[k] = sk;
  }
  if (STORE_NOISE && part) {
    __shared__ float s_S[ROLLOUT_BLOCK], s_w[ROLLOUT_BLOCK];
    s_S[threadIdx.x] = sk;
    const int k0 = blockIdx.x * ROLLOUT_BLOCK;
    block_partial<ROLLOUT_BLOCK>(s_S, s_w, k0, min(ROLLOUT_BLOCK, K - k0), K, T, P.lambda, k_split,
                                 noise, part + static_cast<size_t>(blockIdx.x) * part_stride(T));
  }
  allow_dependent_launch();
}

// ---------------------------------------------------------------------------
// Rolled variant: the link loops are not unrolled, so one step's code is
// about a third of the unrolled variant's and stays in the instruction
// caches.  Per-link results cross from the forward to the backward sweep
// through shared memory, each thread owning the column `tid` of arrays laid
// out [row][B] (conflict-free).  Same arithmetic, same order, as
// rollout_sample.

constexpr int LINK_FIELDS = 22;  // z 3, w 3, F 6, In 10
constexpr int ROLLED_FLOATS_PER_THREAD = NJ * LINK_FIELDS + NJ * (NJ + 1) / 2 + 3 * NJ;

template <int B>
__device__ __forceinline__ void store_link(float* sl, int i, int tid, const LinkState& S) {
  float* b = sl + i * LINK_FIELDS * B + tid;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    b[a * B] = S.z[a];
    b[(3 + a) * B] = S.w[a];
  }
#pragma unroll
  for (int a = 0; a < 6; ++a) b[(6 + a) * B] = S.F[a];
#pragma unroll
  for (int a = 0; a < 10; ++a) b[(12 + a) * B] = S.In[a];
}

template <int B>
__device__ __forceinline__ void load_link(const float* sl, int i, int tid, LinkState& S) {
  const float* b = sl + i * LINK_FIELDS * B + tid;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    S.z[a] = b[a * B];
    S.w[a] = b[(3 + a) * B];
  }
#pragma unroll
  for (int a = 0; a < 6; ++a) S.F[a] = b[(6 + a) * B];
#pragma unroll
  for (int a = 0; a < 10; ++a) S.In[a] = b[(12 + a) * B];
}

template <int B>
__device__ __forceinline__ void load_axis(const float* sl, int j, int tid, float z[3], float w[3]) {
  const float* b = sl + j * LINK_FIELDS * B + tid;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    z[a] = b[a * B];
    w[a] = b[(3 + a) * B];
  }
}

// With STORE_P, also the link capsule end points into sP [NJ + 1][3][B]:
// joint origins p_0 .. p_6 and the end-effector point.
template <int B, bool STORE_P = false>
__device__ __forceinline__ void forward_sweep_rolled(const RobotK& rb, const float* sq,
                                                     const float* sqd, float* sl, int tid,
                                                     EEState& ee, float* sP = nullptr) {
  ChainState c;
  chain_init(rb, c);
#pragma unroll 1
  for (int i = 0; i < NJ; ++i) {
    LinkState S;
    forward_link(rb.L[i], sq[i * B + tid], sqd[i * B + tid], c, S);
    store_link<B>(sl, i, tid, S);
    if (STORE_P) {
#pragma unroll
      for (int a = 0; a < 3; ++a) sP[(3 * i + a) * B + tid] = c.p[a];
    }
  }
  chain_ee(rb, c, ee);
  if (STORE_P) {
#pragma unroll
    for (int a = 0; a < 3; ++a) sP[(3 * NJ + a) * B + tid] = ee.p[a];
  }
}

// Extra per-thread shared floats of the wrench-estimate cost: J^T rows
// [6][NJ] (overwritten by L^-1 J^T) and the gravity torque g [NJ].
constexpr int FEST_FLOATS_PER_THREAD = 6 * NJ + NJ;

// Wrench estimate of Eq. 13 at configuration q_t:
// F = Lambda J M^-1 tau with Lambda = (J M^-1 J^T)^-1, tau = v - g(q_t).
// With M = L D L^T (ldlt_factor) and Y = L^-1 J^T, J M^-1 J^T = Y^T D^-1 Y
// and J M^-1 tau = Y^T D^-1 (L^-1 tau); the 6 x 6 system is factorised by
// LDL^T as well.  J is the geometric Jacobian of the end-effector point p
// (rows: linear velocity of p, angular velocity), built from the joint axes
// (z_j, w_j = p_j x z_j) of the forward sweep: the linear row of joint j is
// w_j + z_j x p.  F = (force; moment about p), world frame.  Returns false
// when a pivot of the 6 x 6 factorisation is not positive (a kinematic
// singularity).  sl: link axes at q_t; sg: g(q_t); sY: [6][NJ][B] scratch.
template <int B>
__device__ __forceinline__ bool force_estimate(const float* sl, int tid,
                                               const float L[NJ * (NJ + 1) / 2],
                                               const float invD[NJ], const float v[NJ],
                                               const float* sg, const float p[3], float* sY,
                                               float F[6]) {
#pragma unroll 1
  for (int j = 0; j < NJ; ++j) {
    float z[3], w[3], zp[3];
    load_axis<B>(sl, j, tid, z, w);
    cross3(z, p, zp);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      sY[(a * NJ + j) * B + tid] = w[a] + zp[a];
      sY[((3 + a) * NJ + j) * B + tid] = z[a];
    }
  }
  float tau[NJ], lt[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) tau[j] = v[j] - sg[j * B + tid];
  unit_lower_solve<NJ>(L, tau, lt);
#pragma unroll
  for (int j = 0; j < NJ; ++j) lt[j] *= invD[j];  // D^-1 L^-1 tau
  float b[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    float jr[NJ], y[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) jr[j] = sY[(r * NJ + j) * B + tid];
    unit_lower_solve<NJ>(L, jr, y);
    float br = 0.f;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      sY[(r * NJ + j) * B + tid] = y[j];
      br = fmaf(y[j], lt[j], br);
    }
    b[r] = br;
  }
  float A[21];
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    float u[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) u[j] = sY[(r * NJ + j) * B + tid] * invD[j];
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < NJ; ++j) acc = fmaf(u[j], sY[(c * NJ + j) * B + tid], acc);
      A[r * (r + 1) / 2 + c] = acc;
    }
  }
  float invDA[6], yb[6];
  ldlt_factor<6>(A, invDA);
  unit_lower_solve<6>(A, b, yb);
  ldlt_back<6>(A, invDA, yb, F);
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 6; ++a) ok = ok && invDA[a] > 0.f && invDA[a] < INFINITY;
  return ok;
}

// C_force of Eq. 12 on the wrench estimate (diagonal six-axis weights);
// NaN at a kinematic singularity, so that the sample gets weight zero.
template <int B>
__device__ __forceinline__ float force_estimate_cost(const CostK& C, const float* sl, int tid,
                                                     const float L[NJ * (NJ + 1) / 2],
                                                     const float invD[NJ], const float v[NJ],
                                                     const float* sg, const float p[3],
                                                     float* sY) {
  float F[6];
  const bool ok = force_estimate<B>(sl, tid, L, invD, v, sg, p, sY, F);
  float cf = 0.f;
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const float e = C.fdes6[a] - F[a];
    cf = fmaf(C.wf6[a], e * e, fmaf(C.wreg6[a], F[a] * F[a], cf));
  }
  return ok ? cf : NAN;
}

// Backward sweep of the rolled kernels: bias torque h -> sh, the packed
// lower triangle of M (with armature) -> sM and, with FEST, the gravity
// torque g -> sg, from the link states in sl.
template <int B, bool FEST>
__device__ __forceinline__ void backward_sweep_rolled(const RobotK& rb, const float* sl,
                                                      const float* sqd, float* sh, float* sM,
                                                      float* sg, int tid) {
  float Fs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float Ic[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
  for (int ii = 0; ii < NJ; ++ii) {
    const int i = NJ - 1 - ii;
    LinkState S;
    load_link<B>(sl, i, tid, S);
    float H[3], Lm[3];
    sh[i * B + tid] = backward_link(rb.L[i], sqd[i * B + tid], S, Fs, Ic, H, Lm);
    if (FEST) {
      // gravity torque from the subtree's mass and first moment (Ic[0],
      // Ic[1..3]): g_i = -S_i . ((m c) x g, m g)
      float mcg[3];
      cross3(Ic + 1, rb.g, mcg);
      sg[i * B + tid] = -(dot3(S.z, mcg) + Ic[0] * dot3(S.w, rb.g));
    }
    const int row = i * (i + 1) / 2;
#pragma unroll 1
    for (int j = 0; j < i; ++j) {
      float zj[3], wj[3];
      load_axis<B>(sl, j, tid, zj, wj);
      sM[(row + j) * B + tid] = dot3(zj, H) + dot3(wj, Lm);
    }
    sM[(row + i) * B + tid] = dot3(S.z, H) + dot3(S.w, Lm) + rb.L[i].arm;
  }
}

// Optional cost terms of the rolled kernel, as template feature bits.
constexpr int FEAT_FEST = 1;  // C_force on the wrench estimate (Eq. 13)
constexpr int FEAT_COLL = 2;  // C_collision (Eq. 15)
constexpr int COLL_FLOATS_PER_THREAD = 3 * (NJ + 1);  // link capsule end points
// Block copy of the obstacles: per obstacle a xyz, b - a xyz, |b - a|^2, its
// reciprocal (0 for a sphere), the radius, the midpoint xyz and the half
// length; then the NJ link radii (padded to 8); then per obstacle the NJ
// link-obstacle culling bounds (pair_skip_b2).
constexpr int OBS_FIELDS = 13;
constexpr int OBS_SMEM_FLOATS = OBS_MAX * OBS_FIELDS + 8 + OBS_MAX * NJ;

__host__ __device__ constexpr int rolled_floats_per_thread(int feat) {
  return ROLLED_FLOATS_PER_THREAD + ((feat & FEAT_FEST) ? FEST_FLOATS_PER_THREAD : 0) +
         ((feat & FEAT_COLL) ? COLL_FLOATS_PER_THREAD : 0);
}

template <int B>
__device__ __forceinline__ void load_point(const float* sP, int i, int tid, float x[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) x[a] = sP[(3 * i + a) * B + tid];
}

// Fills the block copy of the obstacles (threads 0 .. n_obs - 1 one
// obstacle each, threads 0 .. NJ - 1 the link radii); returns n_obs.  The
// caller synchronises the block before use.
__device__ __forceinline__ int load_obstacles(const ObsK* obs, const CostK& C, float* s_obs) {
  const int n_obs = min(max(obs->n, 0), OBS_MAX);
  if (threadIdx.x < n_obs) {
    const float* o = obs->o[threadIdx.x];
    float* so = s_obs + OBS_FIELDS * threadIdx.x;
    float e = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      so[a] = o[a];
      so[3 + a] = o[3 + a] - o[a];
      e = fmaf(so[3 + a], so[3 + a], e);
      so[9 + a] = 0.5f * (o[a] + o[3 + a]);
    }
    so[6] = e;
    so[7] = e > 1e-12f ? 1.f / e : 0.f;
    so[8] = o[6];
    so[12] = 0.5f * sqrtf(e);
    float* b2 = s_obs + OBS_FIELDS * OBS_MAX + 8 + NJ * threadIdx.x;
#pragma unroll
    for (int i = 0; i < NJ; ++i) b2[i] = pair_skip_b2(C.dth_obs, C.lrad[i], o[6], C.seg_h[i], so[12]);
  }
  if (threadIdx.x < NJ) s_obs[OBS_FIELDS * OBS_MAX + threadIdx.x] = C.lrad[threadIdx.x];
  return n_obs;
}

__device__ __forceinline__ float dist2_3(const float a[3], const float b[3]) {
  const float d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
  return fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
}

// One pair's term of Eq. 15 from the squared segment distance g2: the
// indicator [d < th] compares g2 with (th + r1 + r2)^2 (d = sqrt(g2) - r1 -
// r2), the hinge takes (th - d)^2.
__device__ __forceinline__ float collision_term(int mode, float g2, float rsum, float th) {
  if (mode == 1) {
    const float R = th + rsum;
    return (R > 0.f && g2 < R * R) ? 1.f : 0.f;
  }
  const float d = sqrtf(g2) - rsum;
  return d < th ? (th - d) * (th - d) : 0.f;
}

// C_collision of Eq. 15 at the link points in sP: self pairs (i, j >= i + 2)
// by i then j, then every link against every obstacle (s_obs, n_obs of
// them) by link then obstacle; indicator (mode 1) or squared hinge (mode 2)
// against the pair's threshold, times w_collision.  The inner loops have
// constant trip counts (bounds are guards) so that independent pairs
// interleave.
template <int B>
__device__ __forceinline__ float collision_cost(const CostK& C, const float* sP, int tid,
                                                const float* s_obs, int n_obs) {
  const float* lrad = s_obs + OBS_FIELDS * OBS_MAX;
  const float* ob2 = lrad + 8;
  float acc = 0.f;
#pragma unroll 1
  for (int i = 0; i < NJ - 2; ++i) {
    float pi[3], di[3], mi[3];
    load_point<B>(sP, i, tid, pi);
    load_point<B>(sP, i + 1, tid, di);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mi[a] = 0.5f * (pi[a] + di[a]);
      di[a] -= pi[a];
    }
    const float ai = C.seg_a[i], iai = C.seg_ia[i], ri = lrad[i];
    const int n0 = i * (NJ - 2) - i * (i - 1) / 2;  // index of pair (i, i + 2)
#pragma unroll
    for (int jj = 0; jj < NJ - 2; ++jj) {
      const int j = i + 2 + jj;
      if (j < NJ) {
        float pj[3], dj[3], mj[3];
        load_point<B>(sP, j, tid, pj);
        load_point<B>(sP, j + 1, tid, dj);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          mj[a] = 0.5f * (pj[a] + dj[a]);
          dj[a] -= pj[a];
        }
        if (dist2_3(mi, mj) < C.self_b2[n0 + jj]) {
          const float g2 = segment_dist2(pi, di, ai, iai, pj, dj, C.seg_a[j], C.seg_ia[j]);
          acc += collision_term(C.coll, g2, ri + lrad[j], C.dth_self);
        }
      }
    }
  }
#pragma unroll 1
  for (int i = 0; i < NJ; ++i) {
    float pi[3], di[3], mi[3];
    load_point<B>(sP, i, tid, pi);
    load_point<B>(sP, i + 1, tid, di);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mi[a] = 0.5f * (pi[a] + di[a]);
      di[a] -= pi[a];
    }
    const float ai = C.seg_a[i], iai = C.seg_ia[i], ri = lrad[i];
#pragma unroll
    for (int o = 0; o < OBS_MAX; ++o) {
      if (o < n_obs) {
        const float* ob = s_obs + OBS_FIELDS * o;
        if (dist2_3(mi, ob + 9) < ob2[NJ * o + i]) {
          const float g2 = segment_dist2(pi, di, ai, iai, ob, ob + 3, ob[6], ob[7]);
          acc += collision_term(C.coll, g2, ri + ob[8], C.dth_obs);
        }
      }
    }
  }
  return C.wcoll * acc;
}

// sm: this block's work area of rolled_floats_per_thread(FEAT) * B floats;
// s_obs: the block's copy of the n_obs obstacles (FEAT_COLL).
template <bool STORE_NOISE, int B, int FEAT = 0>
__device__ __forceinline__ float rollout_sample_rolled(const ProbK& P, const float* in,
                                                       const float* plan, uint64_t iter, int k,
                                                       float* __restrict__ noise, float* sm,
                                                       int tid, const float* s_obs = nullptr,
                                                       int n_obs = 0) {
  constexpr bool FEST = (FEAT & FEAT_FEST) != 0;
  constexpr bool COLL = (FEAT & FEAT_COLL) != 0;
  float* sl = sm;                                   // [7][22][B]
  float* sM = sl + NJ * LINK_FIELDS * B;            // [28][B]
  float* sq = sM + (NJ * (NJ + 1) / 2) * B;         // [7][B]
  float* sqd = sq + NJ * B;                         // [7][B]
  float* sh = sqd + NJ * B;                         // [7][B]
  float* sY = sh + NJ * B;                          // [6][7][B] (FEST)
  float* sg = sY + 6 * NJ * B;                      // [7][B]    (FEST)
  float* sP = sh + NJ * B + (FEST ? FEST_FLOATS_PER_THREAD * B : 0);  // [8][3][B] (COLL)
  const int T = P.T, K = P.K;
  float q[NJ], qd[NJ], q_lo[NJ], qd_lo[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    q[j] = in[j];
    qd[j] = in[NJ + j];
    q_lo[j] = qd_lo[j] = 0.f;
    sq[j * B + tid] = q[j];
    sqd[j * B + tid] = qd[j];
  }
  const float pdes[3] = {in[14], in[15], in[16]};
  float Rd[9];
  {
    const float qt[4] = {in[17], in[18], in[19], in[20]};
    quat_to_R(qt, Rd);
  }
  const float plane[4] = {in[21], in[22], in[23], in[24]};
  const CostK& C = P.cost;
  const bool contact = C.contact != 0;

  EEState ee;
  forward_sweep_rolled<B, COLL>(P.rb, sq, sqd, sl, tid, ee, sP);
  float f = contact ? contact_force(C, plane, ee) : 0.f;
  double Sacc = 0.0;

  for (int t = 0; t < T; ++t) {
    float z[8];
    normals8(P.key0, P.key1, iter, static_cast<uint32_t>(k), static_cast<uint32_t>(t), z);
    float v[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float du = P.sigma[j] * z[j];
      if (STORE_NOISE) noise[static_cast<size_t>(t * NJ + j) * K + k] = du;
      v[j] = plan[t * NJ + j] + du;
    }
    // backward sweep: h and M (and g) into shared memory
    backward_sweep_rolled<B, FEST>(P.rb, sl, sqd, sh, sM, sg, tid);
    float M[NJ * (NJ + 1) / 2];
#pragma unroll
    for (int a = 0; a < NJ * (NJ + 1) / 2; ++a) M[a] = sM[a * B + tid];
    float rhs[NJ];
    if (contact && f > 0.f) {
      const float Fc[3] = {f * plane[0], f * plane[1], f * plane[2]};
      float pxF[3];
      cross3(ee.p, Fc, pxF);
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        float zj[3], wj[3];
        load_axis<B>(sl, j, tid, zj, wj);
        rhs[j] = v[j] + dot3(zj, pxF) + dot3(wj, Fc) - sh[j * B + tid];
      }
    } else {
#pragma unroll
      for (int j = 0; j < NJ; ++j) rhs[j] = v[j] - sh[j * B + tid];
    }
    if (P.fext) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) rhs[j] += in[IN_TEXT + j];
    }
    float qdd[NJ];
    float cfest = 0.f;
    if (FEST) {
      // the wrench estimate at (q_t, v_t) reuses the factors of M(q_t)
      float invD[NJ], y[NJ];
      ldlt_factor<NJ>(M, invD);
      cfest = force_estimate_cost<B>(C, sl, tid, M, invD, v, sg, ee.p, sY);
      unit_lower_solve<NJ>(M, rhs, y);
      ldlt_back<NJ>(M, invD, y, qdd);
    } else {
      ldlt_solve(M, rhs, qdd);
    }
    const float dt = P.dt;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      euler_step(qdd[j], dt, q[j], q_lo[j], qd[j], qd_lo[j]);
      sq[j * B + tid] = q[j];
      sqd[j * B + tid] = qd[j];
    }
    forward_sweep_rolled<B, COLL>(P.rb, sq, sqd, sl, tid, ee, sP);
    float cst = motion_cost(C, pdes, Rd, ee);
    if (contact) {
      f = contact_force(C, plane, ee);
      if (!FEST) {
        const float e = C.fdes - f;
        cst += C.wforce * e * e + C.wreg * f * f;
      }
    }
    if (FEST) cst += cfest;
    if (COLL) cst += collision_cost<B>(C, sP, tid, s_obs, n_obs);
    float cj = 0.f;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      cj += C.wqlim * (hinge2(q[j] - P.rb.qmax[j]) + hinge2(P.rb.qmin[j] - q[j]));
      cj += C.wqdlim * hinge2(fabsf(qd[j]) - P.rb.qdmax[j]);
      const float e = q[j] - C.qpost[j];
      cj += C.wpost * e * e;
      cj += C.wtau * hinge2(fabsf(v[j]) - P.rb.taumax[j]);
    }
    Sacc += static_cast<double>(cst) + static_cast<double>(cj);
  }
  if (C.wterm != 0.f) Sacc += static_cast<double>(C.wterm * motion_cost(C, pdes, Rd, ee));
  return static_cast<float>(Sacc);
}

// Dynamic shared memory of rollout_kernel_rolled for horizon T, block B and
// feature bits feat.
__host__ __device__ constexpr size_t rolled_smem_bytes(int T, int B, int feat = 0) {
  return sizeof(float) * (2 * static_cast<size_t>((T * NJ + 3) / 4 * 4) + 32 +
                          ((feat & FEAT_COLL) ? OBS_SMEM_FLOATS : 0) +
                          static_cast<size_t>(rolled_floats_per_thread(feat)) * B);
}

template <bool STORE_NOISE, int B, int FEAT = 0>
__global__ void __launch_bounds__(B)
rollout_kernel_rolled(const __grid_constant__ ProbK P, const float* __restrict__ in,
                      const unsigned long long* __restrict__ iter_p, const float* __restrict__ plan,
                      float* __restrict__ S, float* __restrict__ noise,
                      const float* __restrict__ prop = nullptr,
                      const int* __restrict__ ksplit_p = nullptr,
                      const ObsK* __restrict__ obs = nullptr, float* __restrict__ part = nullptr) {
  constexpr bool COLL = (FEAT & FEAT_COLL) != 0;
  extern __shared__ float dsm[];
  const int T = P.T, K = P.K;
  const int k_split = ksplit_p ? *ksplit_p : K;
  const int pstride = (T * NJ + 3) / 4 * 4;
  float* s_plan = dsm;
  float* s_prop = dsm + pstride;
  float* s_in = s_prop + pstride;
  float* s_obs = s_in + IN_STAGED;
  float* s_work = s_obs + (COLL ? OBS_SMEM_FLOATS : 0);
  for (int i = threadIdx.x; i < T * NJ; i += B) s_plan[i] = plan[i];
  if (k_split < K)
    for (int i = threadIdx.x; i < T * NJ; i += B) s_prop[i] = prop[i];
  stage_inputs(P, in, s_in);
  const int n_obs = COLL ? load_obstacles(obs, P.cost, s_obs) : 0;
  __syncthreads();
  const int k = blockIdx.x * B + threadIdx.x;
  float sk = 0.f;
  if (k < K) {
    sk = rollout_sample_rolled<STORE_NOISE, B, FEAT>(P, s_in, k < k_split ? s_plan : s_prop,
                                                     *iter_p, k, noise, s_work, threadIdx.x,
                                                     s_obs, n_obs);
    S[k] = sk;
  }
  if (STORE_NOISE && part) {
    __shared__ float s_S[B], s_w[B];
    s_S[threadIdx.x] = sk;
    const int k0 = blockIdx.x * B;
    block_partial<B>(s_S, s_w, k0, min(B, K - k0), K, T, P.lambda, k_split, noise,
                     part + static_cast<size_t>(blockIdx.x) * part_stride(T));
  }
  allow_dependent_launch();
}

// ---------------------------------------------------------------------------
// Warp-specialised rollout: three warps share 32 samples (lane l of every
// warp works on the block's sample l) so that one sample's step no longer
// runs on a single dependency chain.  For each state x_s (s = 0..T):
//   link phase: warp 0 walks the kinematic chain (link frames, joint axes,
//     velocities and bias accelerations) and hands each link over; warp 1
//     forms the link inertias and RNEA forces of links 0, 2, 4, warp 2 of
//     links 1, 3, 5, and warp 2 then forms the end-effector point and
//     contact force for the dynamics; warp 0 forms the last link's inertia
//     and force itself, from the chain state it holds (warp 1 with the
//     collision cost).
//   For s < T, after the forces: h and the rows of M are split over the
//     three warps (each forms the composite inertias it needs); warp 0
//     factorises M, waits for the step's inputs, solves for qdd and takes the
//     Euler step to x_{s+1}; warp 1 copies x_s and the last link's chain
//     state and then charges all of l(x_s, v_{s-1}); warp 2 draws v_{s+1}
//     one step ahead (v_0 at s = 0).
//   At s = T warp 1 charges l(x_T, v_{T-1}) and phi(x_T).
// With the collision cost (Eq. 15) warps 3 and 4 charge it from the link
// points; with the wrench-estimate cost (Eq. 12-13) warp 3 forms the
// end-effector Jacobian and the gravity torque at x_s after the forces and,
// past the step barrier (by then warp 0 has left the factors of M(x_s) in
// the rows' slots and warp 2 has drawn v_s), the estimate and its cost, off
// the critical path.
// Hand-offs go through shared memory under named barriers with fixed
// arrival counts.  Per state every barrier sees the same arrivals, and each
// slot is rewritten only after its readers have passed a barrier that the
// writer waits on first, so no wait depends on data.  Same arithmetic as
// rollout_sample, in the same order per quantity.

constexpr int WS_B = 32;              // samples per block
constexpr int WS_THREADS = 3 * WS_B;  // three warps
// One record of 52 floats per (link, sample): 16-byte aligned, and a stride
// of 52 words puts the eight lanes of each 128-bit access phase on distinct
// banks.  float4 0-5, the link state: (z0 z1 z2 w0)(w1 w2 . .)(F0..F3)
// (F4 F5 I0 I1)(I2..I5)(I6..I9), warp 0 writing the first two, the force
// warps the last four; float4 6-11, the hand-off of the link's frame and
// motion: (R0..R3)(R4..R7)(R8 p0 p1 p2)(Vw Vv0)(Vv1 Vv2 Aw0 Aw1)(Aw2 Av).
constexpr int WS_REC = 52;
constexpr int WS_HANDOFF = 6;  // float4 offset of the hand-off part
constexpr int V_SLOTS = 3;            // ring of inputs v_s, slot s % 3
// named barriers (0 is __syncthreads): one per link, link forces complete,
// rows of M complete, inputs of the step complete, and (collision or
// wrench-estimate cost) the extra warps' partial costs handed to warp 1
constexpr int BAR_LINK0 = 1, BAR_FORCES = 8, BAR_MROWS = 9, BAR_STEP = 10, BAR_DONE = 11;
constexpr int WS_FLOATS_PER_SAMPLE = NJ * WS_REC + NJ * (NJ + 1) / 2 + NJ /* h */ +
                                     2 * NJ /* q, qd */ + V_SLOTS * NJ /* v ring */;
// The last float4 of each record is free: link 0's holds the end-effector
// point and contact force for the dynamics, links 1 and 2's the collision
// warps' partial costs.
constexpr int WS_PAD = 48;

__device__ __forceinline__ void bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Threads at link i's barrier while s < T: warp 0 and the force warp of
// link i; for the last link warp 2, which forms the end-effector state, and
// its force warp (warp 1) only with the collision cost: without it warp 0
// forms the last link's force itself (with it, the register budget of four
// 160-thread blocks per SM leaves no room for that).  At s = T only the last
// link's barrier runs, for warp 1 and, with the collision cost, warps 3 and
// 4 (they read the last state's link points after it).
__host__ __device__ constexpr int ws_link_count(int i, bool last_state, bool coll) {
  return last_state ? (coll ? 4 : 2) * WS_B : (coll && i == NJ - 1 ? 3 : 2) * WS_B;
}
// Warps of the kernel, and threads at the barriers every warp meets: three,
// two more for the collision cost, one more for the wrench-estimate cost
// (the two optional costs together run in the rolled kernel).
__host__ __device__ constexpr int ws_warps(bool coll, bool fest) {
  return 3 + (coll ? 2 : 0) + (fest ? 1 : 0);
}
__host__ __device__ constexpr int ws_threads(bool coll, bool fest) {
  return ws_warps(coll, fest) * WS_B;
}

// Dynamic shared memory of rollout_kernel_ws (independent of T: the plans
// are read from global memory, where they stay in L1).  56.2 KB: four
// blocks fit on an SM.
__host__ __device__ constexpr size_t ws_smem_bytes(bool coll = false) {
  return sizeof(float) * (32 + (coll ? OBS_SMEM_FLOATS : 0) +
                          static_cast<size_t>(WS_FLOATS_PER_SAMPLE) * WS_B);
}

struct WsSmem {
  float *sl, *sc, *sM, *sh, *sq, *sqd, *sv;
};

__device__ __forceinline__ WsSmem ws_carve(float* base) {
  constexpr int B = WS_B;
  WsSmem m;
  m.sl = base;                              // [7][B] records (link state part)
  m.sc = base + 4 * WS_HANDOFF;             // the same records' hand-off part
  m.sM = m.sl + NJ * B * WS_REC;            // [28][B]
  m.sh = m.sM + (NJ * (NJ + 1) / 2) * B;    // [7][B]
  m.sq = m.sh + NJ * B;                     // [7][B]
  m.sqd = m.sq + NJ * B;                    // [7][B]
  m.sv = m.sqd + NJ * B;                    // [3][7][B]: v_s in slot s % 3
  return m;
}

__device__ __forceinline__ float4* ws_rec(float* base, int i, int tid) {
  return reinterpret_cast<float4*>(base + (i * WS_B + tid) * WS_REC);
}
__device__ __forceinline__ const float4* ws_rec(const float* base, int i, int tid) {
  return reinterpret_cast<const float4*>(base + (i * WS_B + tid) * WS_REC);
}

// end-effector point (3) and contact force of sample tid in the free tail
// of record 0, and the collision warps' partial costs of sample tid in those
// of records 1 and 2
__device__ __forceinline__ float* ws_ee(const WsSmem& m, int tid) {
  return m.sl + tid * WS_REC + WS_PAD;
}
__device__ __forceinline__ double* ws_s2(const WsSmem& m, int tid, int slot) {
  return reinterpret_cast<double*>(m.sl + ((1 + slot) * WS_B + tid) * WS_REC + WS_PAD);
}

__device__ __forceinline__ void ws_store_axis(float* sl, int i, int tid, const float z[3],
                                              const float w[3]) {
  float4* r = ws_rec(sl, i, tid);
  r[0] = make_float4(z[0], z[1], z[2], w[0]);
  r[1] = make_float4(w[1], w[2], 0.f, 0.f);
}
__device__ __forceinline__ void ws_load_axis(const float* sl, int i, int tid, float z[3],
                                             float w[3]) {
  const float4* r = ws_rec(sl, i, tid);
  const float4 a = r[0], b = r[1];
  z[0] = a.x; z[1] = a.y; z[2] = a.z;
  w[0] = a.w; w[1] = b.x; w[2] = b.y;
}
__device__ __forceinline__ void ws_store_force(float* sl, int i, int tid, const float F[6],
                                               const float In[10]) {
  float4* r = ws_rec(sl, i, tid);
  r[2] = make_float4(F[0], F[1], F[2], F[3]);
  r[3] = make_float4(F[4], F[5], In[0], In[1]);
  r[4] = make_float4(In[2], In[3], In[4], In[5]);
  r[5] = make_float4(In[6], In[7], In[8], In[9]);
}
__device__ __forceinline__ void ws_load_force(const float* sl, int i, int tid, float F[6],
                                              float In[10]) {
  const float4* r = ws_rec(sl, i, tid);
  const float4 a = r[2], b = r[3], c = r[4], d = r[5];
  F[0] = a.x; F[1] = a.y; F[2] = a.z; F[3] = a.w; F[4] = b.x; F[5] = b.y;
  In[0] = b.z; In[1] = b.w;
  In[2] = c.x; In[3] = c.y; In[4] = c.z; In[5] = c.w;
  In[6] = d.x; In[7] = d.y; In[8] = d.z; In[9] = d.w;
}
__device__ __forceinline__ void ws_load_inertia(const float* sl, int i, int tid, float In[10]) {
  const float4* r = ws_rec(sl, i, tid);
  const float4 b = r[3], c = r[4], d = r[5];
  In[0] = b.z; In[1] = b.w;
  In[2] = c.x; In[3] = c.y; In[4] = c.z; In[5] = c.w;
  In[6] = d.x; In[7] = d.y; In[8] = d.z; In[9] = d.w;
}
__device__ __forceinline__ void ws_store_chain(float* sc, int i, int tid, const ChainState& c) {
  float4* r = ws_rec(sc, i, tid);
  r[0] = make_float4(c.R[0], c.R[1], c.R[2], c.R[3]);
  r[1] = make_float4(c.R[4], c.R[5], c.R[6], c.R[7]);
  r[2] = make_float4(c.R[8], c.p[0], c.p[1], c.p[2]);
  r[3] = make_float4(c.Vw[0], c.Vw[1], c.Vw[2], c.Vv[0]);
  r[4] = make_float4(c.Vv[1], c.Vv[2], c.Aw[0], c.Aw[1]);
  r[5] = make_float4(c.Aw[2], c.Av[0], c.Av[1], c.Av[2]);
}
__device__ __forceinline__ void ws_load_chain(const float* sc, int i, int tid, ChainState& c) {
  const float4* r = ws_rec(sc, i, tid);
  const float4 a = r[0], b = r[1], d = r[2], e = r[3], f = r[4], g = r[5];
  c.R[0] = a.x; c.R[1] = a.y; c.R[2] = a.z; c.R[3] = a.w;
  c.R[4] = b.x; c.R[5] = b.y; c.R[6] = b.z; c.R[7] = b.w;
  c.R[8] = d.x; c.p[0] = d.y; c.p[1] = d.z; c.p[2] = d.w;
  c.Vw[0] = e.x; c.Vw[1] = e.y; c.Vw[2] = e.z; c.Vv[0] = e.w;
  c.Vv[1] = f.x; c.Vv[2] = f.y; c.Aw[0] = f.z; c.Aw[1] = f.w;
  c.Aw[2] = g.x; c.Av[0] = g.y; c.Av[1] = g.z; c.Av[2] = g.w;
}

// Row i of M from the composite momentum (H, Lm) of S_i:
// M_ij = S_j . (H, Lm) for j < i, M_ii = S_i . (H, Lm) + armature.
__device__ __forceinline__ void ws_row(const RobotK& rb, const WsSmem& m, int i, const float z[3],
                                       const float w[3], const float H[3], const float Lm[3],
                                       int tid) {
  constexpr int B = WS_B;
  const int row = i * (i + 1) / 2;
#pragma unroll 1
  for (int j = 0; j < i; ++j) {
    float zj[3], wj[3];
    ws_load_axis(m.sl, j, tid, zj, wj);
    m.sM[(row + j) * B + tid] = dot3(zj, H) + dot3(wj, Lm);
  }
  m.sM[(row + i) * B + tid] = dot3(z, H) + dot3(w, Lm) + rb.L[i].arm;
}

// warp 0's share of the backward sweep: h over all links (backward_link's
// suffix force sum and projection) and row NJ - 1 of M, whose composite
// inertia is the last link's own.
__device__ __forceinline__ void ws_backward_h(const RobotK& rb, const WsSmem& m, int tid) {
  constexpr int B = WS_B;
  float Fs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
  for (int i = NJ - 1; i >= 0; --i) {
    float z[3], w[3];
    ws_load_axis(m.sl, i, tid, z, w);
    {
      const float4* r = ws_rec(m.sl, i, tid);
      const float4 a = r[2], b = r[3];
      Fs[0] += a.x; Fs[1] += a.y; Fs[2] += a.z; Fs[3] += a.w; Fs[4] += b.x; Fs[5] += b.y;
    }
    m.sh[i * B + tid] = fmaf(rb.L[i].damp, m.sqd[i * B + tid],
                             dot3(z, Fs) + fmaf(w[0], Fs[3], fmaf(w[1], Fs[4], w[2] * Fs[5])));
    if (i == NJ - 1) {
      float In[10], Ic[10], H[3], Lm[3];
      ws_load_inertia(m.sl, i, tid, In);
#pragma unroll
      for (int a = 0; a < 10; ++a) Ic[a] = 0.f + In[a];
      inertia_apply(Ic, z, w, H, Lm);
      ws_row(rb, m, i, z, w, H, Lm, tid);
    }
  }
}

// the force warps' share: the composite inertias Ic_i = sum_{j >= i} In_j
// (added in backward_link's order) down to the lowest listed row, and the
// listed rows of M.
__device__ __forceinline__ void ws_backward_rows(const RobotK& rb, const WsSmem& m, unsigned rows,
                                                 int tid) {
  float Ic[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int lowest = __ffs(rows) - 1;
#pragma unroll 1
  for (int i = NJ - 1; i >= lowest; --i) {
    float In[10];
    ws_load_inertia(m.sl, i, tid, In);
#pragma unroll
    for (int a = 0; a < 10; ++a) Ic[a] += In[a];
    if (rows & (1u << i)) {
      float z[3], w[3], H[3], Lm[3];
      ws_load_axis(m.sl, i, tid, z, w);
      inertia_apply(Ic, z, w, H, Lm);
      ws_row(rb, m, i, z, w, H, Lm, tid);
    }
  }
}

// Rows of M of the force warps (each costs about 30 + 6 i, plus the
// composite inertias down to the lowest row); warp 0 forms h and row 6.
constexpr unsigned WS_ROWS1 = (1u << 5) | (1u << 2) | (1u << 1);
constexpr unsigned WS_ROWS2 = (1u << 4) | (1u << 3) | (1u << 0);

// warp 0
template <bool COLL, bool FEST>
__device__ __forceinline__ void ws_dynamics(const ProbK& P, const float* in, const WsSmem& m,
                                            int tid) {
  constexpr int NA = ws_threads(COLL, FEST);
  constexpr int B = WS_B;
  const int T = P.T;
  const CostK& C = P.cost;
  const bool contact = C.contact != 0;
  const float plane[4] = {in[21], in[22], in[23], in[24]};
  float q[NJ], qd[NJ], q_lo[NJ], qd_lo[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    q[j] = in[j];
    qd[j] = in[NJ + j];
    q_lo[j] = qd_lo[j] = 0.f;
    m.sq[j * B + tid] = q[j];
    m.sqd[j * B + tid] = qd[j];
  }
  for (int s = 0; s <= T; ++s) {
    const bool last = s == T;
    // link phase: the chain at x_s, handed over link by link
    ChainState c;
    chain_init(P.rb, c);
#pragma unroll 1
    for (int i = 0; i < NJ; ++i) {
      float z[3], w[3];
      forward_link_chain(P.rb.L[i], m.sq[i * B + tid], m.sqd[i * B + tid], c, z, w);
      ws_store_axis(m.sl, i, tid, z, w);
      ws_store_chain(m.sc, i, tid, c);
      if (!last || i == NJ - 1) bar_arrive(BAR_LINK0 + i, ws_link_count(i, last, COLL));
    }
    if (last) break;
    // the last link's force here, from the chain state in registers: no
    // hand-off on the way to the backward sweep
    if (!COLL) {
      float In[10], F[6];
      forward_link_force(P.rb.L[NJ - 1], c.R, c.p, c.Vw, c.Vv, c.Aw, c.Av, In, F);
      ws_store_force(m.sl, NJ - 1, tid, F, In);
    }
    bar_sync(BAR_FORCES, NA);
    ws_backward_h(P.rb, m, tid);
    bar_sync(BAR_MROWS, 3 * B);
    float M[NJ * (NJ + 1) / 2], invD[NJ];
#pragma unroll
    for (int a = 0; a < NJ * (NJ + 1) / 2; ++a) M[a] = m.sM[a * B + tid];
    ldlt_factor<NJ, true>(M, invD);
    if (FEST) {
      // the factors of M(x_s) for warp 3's wrench estimate, in the rows'
      // slots (free until the next state's rows): L below the diagonal,
      // 1/D on it; warp 3 reads them past the step barrier
#pragma unroll
      for (int i = 0; i < NJ; ++i) {
#pragma unroll
        for (int j = 0; j < i; ++j) m.sM[(i * (i + 1) / 2 + j) * B + tid] = M[i * (i + 1) / 2 + j];
        m.sM[(i * (i + 1) / 2 + i) * B + tid] = invD[i];
      }
    }
    bar_sync(BAR_STEP, NA);
    const float* v = m.sv + (s % V_SLOTS) * NJ * B + tid;
    const float* ees = ws_ee(m, tid);
    const float f = ees[3];
    float rhs[NJ];
    if (contact && f > 0.f) {
      const float pe[3] = {ees[0], ees[1], ees[2]};
      const float Fc[3] = {f * plane[0], f * plane[1], f * plane[2]};
      float pxF[3];
      cross3(pe, Fc, pxF);
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        float zj[3], wj[3];
        ws_load_axis(m.sl, j, tid, zj, wj);
        rhs[j] = v[j * B] + dot3(zj, pxF) + dot3(wj, Fc) - m.sh[j * B + tid];
      }
    } else {
#pragma unroll
      for (int j = 0; j < NJ; ++j) rhs[j] = v[j * B] - m.sh[j * B + tid];
    }
    if (P.fext) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) rhs[j] += in[IN_TEXT + j];
    }
    float y[NJ], qdd[NJ];
    unit_lower_solve<NJ>(M, rhs, y);
    ldlt_back<NJ>(M, invD, y, qdd);
    const float dt = P.dt;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      euler_step(qdd[j], dt, q[j], q_lo[j], qd[j], qd_lo[j]);
      m.sq[j * B + tid] = q[j];
      m.sqd[j * B + tid] = qd[j];
    }
  }
}

// warps 1 and 2, link phase: inertias and forces of links first, first + 2,
// ... (the last link's only with the collision cost)
template <bool COLL>
__device__ __forceinline__ void ws_forces(const ProbK& P, const WsSmem& m, int first, int tid) {
#pragma unroll 1
  for (int i = first; i < (COLL ? NJ : NJ - 1); i += 2) {
    bar_sync(BAR_LINK0 + i, ws_link_count(i, false, COLL));
    ChainState c;
    ws_load_chain(m.sc, i, tid, c);
    float In[10], F[6];
    forward_link_force(P.rb.L[i], c.R, c.p, c.Vw, c.Vv, c.Aw, c.Av, In, F);
    ws_store_force(m.sl, i, tid, F, In);
  }
}

// warp 1: forces of links 0, 2, 4 (and 6 with the collision cost) and the
// running cost; returns S_k
template <bool COLL, bool FEST>
__device__ __forceinline__ float ws_costs(const ProbK& P, const float* in, const WsSmem& m,
                                          int tid) {
  static_assert(!(COLL && FEST), "the two optional costs together run in the rolled kernel");
  constexpr int NA = ws_threads(COLL, FEST);
  constexpr int B = WS_B;
  const int T = P.T;
  const CostK& C = P.cost;
  const bool contact = C.contact != 0;
  const float pdes[3] = {in[14], in[15], in[16]};
  float Rd[9];
  {
    const float qt[4] = {in[17], in[18], in[19], in[20]};
    quat_to_R(qt, Rd);
  }
  const float plane[4] = {in[21], in[22], in[23], in[24]};
  double Sacc = 0.0;
  for (int s = 0; s <= T; ++s) {
    ChainState c;
    if (s < T) {
      ws_forces<COLL>(P, m, 0, tid);
      bar_sync(BAR_FORCES, NA);
      ws_backward_rows(P.rb, m, WS_ROWS1, tid);
      bar_arrive(BAR_MROWS, 3 * B);
      // x_s's last link, read before warp 0 may overwrite it
      if (s > 0) ws_load_chain(m.sc, NJ - 1, tid, c);
    } else {
      bar_sync(BAR_LINK0 + NJ - 1, ws_link_count(NJ - 1, true, COLL));
      ws_load_chain(m.sc, NJ - 1, tid, c);
    }
    // x_s and v_{s-1}, copied before warp 0 may overwrite them
    float q[NJ], qd[NJ], v[NJ];
    const float* vp = m.sv + ((s + V_SLOTS - 1) % V_SLOTS) * NJ * B + tid;  // v_{s-1}
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      q[j] = m.sq[j * B + tid];
      qd[j] = m.sqd[j * B + tid];
      v[j] = vp[j * B];
    }
    if (s < T) bar_arrive(BAR_STEP, NA);
    if (s == 0) continue;
    // running cost l(x_s, v_{s-1}), Eq. 9-14
    EEState ee;
    chain_ee(P.rb, c, ee);
    const float mc = motion_cost(C, pdes, Rd, ee);
    float cst = mc;
    if (contact && !FEST) {
      const float f = contact_force(C, plane, ee);
      const float ef = C.fdes - f;
      cst += C.wforce * ef * ef + C.wreg * f * f;
    }
    float cj = 0.f;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      cj += C.wqlim * (hinge2(q[j] - P.rb.qmax[j]) + hinge2(P.rb.qmin[j] - q[j]));
      cj += C.wqdlim * hinge2(fabsf(qd[j]) - P.rb.qdmax[j]);
      const float ep = q[j] - C.qpost[j];
      cj += C.wpost * ep * ep;
      cj += C.wtau * hinge2(fabsf(v[j]) - P.rb.taumax[j]);
    }
    Sacc += static_cast<double>(cst) + static_cast<double>(cj);
    // phi(x_T) = w_terminal C_motion(x_T): the same motion cost, not formed twice
    if (s == T && C.wterm != 0.f) Sacc += static_cast<double>(C.wterm * mc);
  }
  double S = Sacc;
  if (COLL) {
    bar_sync(BAR_DONE, 3 * B);
    S += *ws_s2(m, tid, 0) + *ws_s2(m, tid, 1);
  }
  if (FEST) {
    bar_sync(BAR_DONE, 2 * B);
    S += *ws_s2(m, tid, 0);
  }
  return static_cast<float>(S);
}

// warp 2: the inputs v_s = u_s + dtau_s (Eq. 2) into slot s % 3
template <bool STORE_NOISE>
__device__ __forceinline__ void ws_draw(const ProbK& P, const float* plan, uint64_t iter, int k,
                                        bool live, float* __restrict__ noise, const WsSmem& m,
                                        int s, int tid) {
  constexpr int B = WS_B;
  const int K = P.K;
  float* v = m.sv + (s % V_SLOTS) * NJ * B + tid;
  // the two Philox calls in a loop that is not unrolled (z through local
  // memory): this warp's code shares the instruction caches with the other
  // warps', and with both calls unrolled the rollout took 4-7 % longer
  float z[8];
#pragma unroll 1
  for (int call = 0; call < 2; ++call)
    normals4(P.key0, P.key1, iter, static_cast<uint32_t>(k), static_cast<uint32_t>(s),
             static_cast<uint32_t>(call), z + 4 * call);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const float du = P.sigma[j] * z[j];
    if (STORE_NOISE && live) noise[static_cast<size_t>(s * NJ + j) * K + k] = du;
    v[j * B] = __ldg(plan + s * NJ + j) + du;
  }
}

// warp 2: forces of the odd links, the end-effector point and contact force
// for the dynamics, and the inputs one step ahead
template <bool STORE_NOISE, bool COLL, bool FEST>
__device__ __forceinline__ void ws_noise(const ProbK& P, const float* in, const float* plan,
                                         uint64_t iter, int k, bool live,
                                         float* __restrict__ noise, const WsSmem& m, int tid,
                                         const float* prop = nullptr,
                                         const int* ksplit_p = nullptr, bool defer = false) {
  constexpr int NA = ws_threads(COLL, FEST);
  constexpr int B = WS_B;
  const int T = P.T;
  const CostK& C = P.cost;
  const bool contact = C.contact != 0;
  const float plane[4] = {in[21], in[22], in[23], in[24]};
  for (int s = 0; s < T; ++s) {
    ws_forces<COLL>(P, m, 1, tid);
    {
      bar_sync(BAR_LINK0 + NJ - 1, ws_link_count(NJ - 1, false, COLL));
      ChainState c;
      ws_load_chain(m.sc, NJ - 1, tid, c);
      EEState ee;
      chain_ee_pv(P.rb, c, ee);
      const float f = contact ? contact_force(C, plane, ee) : 0.f;
      float* ees = ws_ee(m, tid);
#pragma unroll
      for (int a = 0; a < 3; ++a) ees[a] = ee.p[a];
      ees[3] = f;
    }
    bar_sync(BAR_FORCES, NA);
    ws_backward_rows(P.rb, m, WS_ROWS2, tid);
    bar_arrive(BAR_MROWS, 3 * B);
    if (s == 0) {
      if (defer) {
        // the proposal kernel this grid overlaps: its plan and split are
        // needed from the first draw on
        grid_dependency_wait();
        if (k >= (ksplit_p ? *ksplit_p : P.K)) plan = prop;
      }
      ws_draw<STORE_NOISE>(P, plan, iter, k, live, noise, m, 0, tid);
    }
    bar_arrive(BAR_STEP, NA);
    if (s + 1 < T) ws_draw<STORE_NOISE>(P, plan, iter, k, live, noise, m, s + 1, tid);
  }
}

// Warps 3 and 4 (collision cost, Eq. 15): the link points of x_s are copied
// from the hand-off records (and the end-effector point from warp 2's slot)
// between the forces and the step barriers, then the pairs of this warp's
// part are charged: part 0 the 15 link-link pairs and link 0 against the
// obstacles, part 1 links 1-6 against the obstacles (18 pairs each with three
// obstacles; both warps must be done before the next state's forces barrier,
// so the longer part bounds the step).  Link i spans pts[i] .. pts[i + 1];
// same terms as collision_cost.
template <int PART>
__device__ __forceinline__ float ws_collision_pairs(const CostK& C, const float pts[NJ + 1][3],
                                                    const float* s_obs, int n_obs) {
  const float* lrad = s_obs + OBS_FIELDS * OBS_MAX;
  const float* ob2 = lrad + 8;
  float acc = 0.f;
  float d[NJ][3], mid[NJ][3];
#pragma unroll
  for (int i = 0; i < NJ; ++i)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d[i][a] = pts[i + 1][a] - pts[i][a];
      mid[i][a] = 0.5f * (pts[i][a] + pts[i + 1][a]);
    }
  if (PART == 0) {
    int n = 0;
#pragma unroll
    for (int i = 0; i < NJ - 2; ++i)
#pragma unroll
      for (int j = i + 2; j < NJ; ++j, ++n) {
        if (dist2_3(mid[i], mid[j]) < C.self_b2[n]) {
          const float g2 = segment_dist2(pts[i], d[i], C.seg_a[i], C.seg_ia[i], pts[j], d[j],
                                         C.seg_a[j], C.seg_ia[j]);
          acc += collision_term(C.coll, g2, lrad[i] + lrad[j], C.dth_self);
        }
      }
  }
  constexpr int i0 = PART == 0 ? 0 : 1, i1 = PART == 0 ? 1 : NJ;
#pragma unroll
  for (int i = i0; i < i1; ++i) {
#pragma unroll 1
    for (int o = 0; o < n_obs; ++o) {
      const float* ob = s_obs + OBS_FIELDS * o;
      if (dist2_3(mid[i], ob + 9) < ob2[NJ * o + i]) {
        const float g2 = segment_dist2(pts[i], d[i], C.seg_a[i], C.seg_ia[i], ob, ob + 3, ob[6],
                                       ob[7]);
        acc += collision_term(C.coll, g2, lrad[i] + ob[8], C.dth_obs);
      }
    }
  }
  return acc;
}

template <int PART>
__device__ __forceinline__ void ws_collision(const ProbK& P, const WsSmem& m, const float* s_obs,
                                             int n_obs, int tid) {
  constexpr int NA = ws_threads(true, false);
  const int T = P.T;
  const CostK& C = P.cost;
  double Sc = 0.0;
  for (int s = 0; s <= T; ++s) {
    float pts[NJ + 1][3];
    if (s < T) {
      bar_sync(BAR_FORCES, NA);
#pragma unroll
      for (int i = 0; i < NJ; ++i) {
        const float4 r = ws_rec(m.sc, i, tid)[2];  // (R8 p0 p1 p2)
        pts[i][0] = r.y; pts[i][1] = r.z; pts[i][2] = r.w;
      }
      const float* ees = ws_ee(m, tid);
#pragma unroll
      for (int a = 0; a < 3; ++a) pts[NJ][a] = ees[a];
      bar_arrive(BAR_STEP, NA);
    } else {
      bar_sync(BAR_LINK0 + NJ - 1, ws_link_count(NJ - 1, true, true));
#pragma unroll
      for (int i = 0; i < NJ; ++i) {
        const float4 r = ws_rec(m.sc, i, tid)[2];
        pts[i][0] = r.y; pts[i][1] = r.z; pts[i][2] = r.w;
      }
      ChainState c;
      ws_load_chain(m.sc, NJ - 1, tid, c);
      EEState ee;
      chain_ee(P.rb, c, ee);
#pragma unroll
      for (int a = 0; a < 3; ++a) pts[NJ][a] = ee.p[a];
    }
    if (s == 0) continue;
    Sc += static_cast<double>(C.wcoll * ws_collision_pairs<PART>(C, pts, s_obs, n_obs));
  }
  *ws_s2(m, tid, PART) = Sc;
  bar_arrive(BAR_DONE, 3 * WS_B);
}

// Warp 3 with the wrench-estimate cost (Eq. 12-13): for each x_s, s < T,
// the rows of the end-effector Jacobian (linear: w_j + z_j x p; angular:
// z_j) and g(q_s), from the subtree masses and first moments, are formed
// from the hand-off records between the forces and the step barriers (warp
// 0 rewrites the records only past the step barrier); past it, tau = v_s -
// g, the factors of M(q_s) that warp 0 left in the rows' slots before the
// barrier, and the estimate F = Jbar^T tau of force_estimate (Y = L^-1 J^T,
// A = Y^T D^-1 Y, F = A^-1 Y^T D^-1 L^-1 tau) and its cost, NaN at a
// kinematic singularity.  The rows' slots are rewritten only after the next
// forces barrier, which this warp reaches once it is done.  Same terms, in
// the same order per quantity, as force_estimate and force_estimate_cost,
// with Y in registers.
__device__ __forceinline__ void ws_estimate(const ProbK& P, const WsSmem& m, int tid) {
  constexpr int NA = ws_threads(false, true);
  constexpr int B = WS_B;
  const int T = P.T;
  const CostK& C = P.cost;
  double Sf = 0.0;
  for (int s = 0; s < T; ++s) {
    float Y[6][NJ], g[NJ];
    bar_sync(BAR_FORCES, NA);
    {
      const float* ees = ws_ee(m, tid);
      const float p[3] = {ees[0], ees[1], ees[2]};
      float Ic[4] = {0.f, 0.f, 0.f, 0.f};  // subtree mass and first moment
#pragma unroll
      for (int ii = 0; ii < NJ; ++ii) {
        const int i = NJ - 1 - ii;
        float z[3], w[3], zp[3];
        ws_load_axis(m.sl, i, tid, z, w);
        const float4* r = ws_rec(m.sl, i, tid);
        const float4 b = r[3], c = r[4];  // (F4 F5 I0 I1)(I2 I3 I4 I5)
        Ic[0] += b.z; Ic[1] += b.w; Ic[2] += c.x; Ic[3] += c.y;
        float mcg[3];
        cross3(Ic + 1, P.rb.g, mcg);
        g[i] = -(dot3(z, mcg) + Ic[0] * dot3(w, P.rb.g));
        cross3(z, p, zp);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          Y[a][i] = w[a] + zp[a];
          Y[3 + a][i] = z[a];
        }
      }
    }
    bar_sync(BAR_STEP, NA);
    float tau[NJ];
    const float* v = m.sv + (s % V_SLOTS) * NJ * B + tid;
#pragma unroll
    for (int j = 0; j < NJ; ++j) tau[j] = v[j * B] - g[j];
    float L[NJ * (NJ + 1) / 2], invD[NJ];
#pragma unroll
    for (int i = 0; i < NJ; ++i) {
#pragma unroll
      for (int j = 0; j < i; ++j) L[i * (i + 1) / 2 + j] = m.sM[(i * (i + 1) / 2 + j) * B + tid];
      invD[i] = m.sM[(i * (i + 1) / 2 + i) * B + tid];
      L[i * (i + 1) / 2 + i] = 1.f;
    }
    float lt[NJ];
    unit_lower_solve<NJ>(L, tau, lt);
#pragma unroll
    for (int j = 0; j < NJ; ++j) lt[j] *= invD[j];  // D^-1 L^-1 tau
    float b6[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      float y[NJ];
      unit_lower_solve<NJ>(L, Y[r], y);
      float br = 0.f;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        Y[r][j] = y[j];
        br = fmaf(y[j], lt[j], br);
      }
      b6[r] = br;
    }
    float A[21];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      float u[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) u[j] = Y[r][j] * invD[j];
#pragma unroll
      for (int c = 0; c <= r; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc = fmaf(u[j], Y[c][j], acc);
        A[r * (r + 1) / 2 + c] = acc;
      }
    }
    float invDA[6], yb[6], F[6];
    ldlt_factor<6>(A, invDA);
    unit_lower_solve<6>(A, b6, yb);
    ldlt_back<6>(A, invDA, yb, F);
    bool ok = true;
    float cf = 0.f;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      ok = ok && invDA[a] > 0.f && invDA[a] < INFINITY;
      const float e = C.fdes6[a] - F[a];
      cf = fmaf(C.wf6[a], e * e, fmaf(C.wreg6[a], F[a] * F[a], cf));
    }
    Sf += static_cast<double>(ok ? cf : NAN);
  }
  *ws_s2(m, tid, 0) = Sf;
  bar_arrive(BAR_DONE, 2 * WS_B);
}

template <bool STORE_NOISE, bool COLL, bool FEST>
__device__ __forceinline__ void rollout_ws_block(const ProbK& P, const float* __restrict__ in,
                                                 const unsigned long long* __restrict__ iter_p,
                                                 const float* __restrict__ plan,
                                                 float* __restrict__ S, float* __restrict__ noise,
                                                 const float* __restrict__ prop,
                                                 const int* __restrict__ ksplit_p,
                                                 const ObsK* __restrict__ obs,
                                                 float* __restrict__ part, int kwait = -1) {
  extern __shared__ float4 dsm4[];
  float* dsm = reinterpret_cast<float*>(dsm4);
  const int K = P.K;
  // kwait >= 0: this grid is the programmatic dependent of a proposal kernel
  // that may still be writing prop and *ksplit_p (kwait there unless its
  // wait gave up).  A block whose samples all lie below kwait rolls out
  // around plan either way and does not wait.  In the others (defer) warp 2
  // waits for that grid's completion just before its first draw, the state
  // phases of step 0 having run meanwhile, and every thread reads the split
  // after the rollout.  The last block always defers, so that this grid
  // completes after the proposal kernel and the merge, which waits for this
  // grid, finds its writes done.
  int k_split = K;
  bool defer = false;
  if (kwait < 0)
    k_split = ksplit_p ? *ksplit_p : K;
  else if ((blockIdx.x + 1) * WS_B <= kwait && blockIdx.x + 1 < gridDim.x)
    k_split = kwait;
  else
    defer = true;
  float* s_in = dsm;
  float* s_obs = s_in + IN_STAGED;  // COLL: the block copy of the obstacles (load_obstacles)
  stage_inputs(P, in, s_in);
  const int n_obs = COLL ? load_obstacles(obs, P.cost, s_obs) : 0;
  __syncthreads();
  const WsSmem m = ws_carve(s_in + IN_STAGED + (COLL ? OBS_SMEM_FLOATS : 0));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // lanes past K run sample K - 1 so that every warp meets every barrier;
  // they write nothing
  const int k_raw = blockIdx.x * WS_B + lane;
  const bool live = k_raw < K;
  const int k = live ? k_raw : K - 1;
  __shared__ float s_S[WS_B], s_w[WS_B];
  if (warp == 0) {
    ws_dynamics<COLL, FEST>(P, s_in, m, lane);
  } else if (warp == 1) {
    const float Sk = ws_costs<COLL, FEST>(P, s_in, m, lane);
    if (live) S[k] = Sk;
    s_S[lane] = Sk;
  } else if (warp == 2) {
    ws_noise<STORE_NOISE, COLL, FEST>(P, s_in, defer || k < k_split ? plan : prop, *iter_p, k,
                                      live, noise, m, lane, prop, ksplit_p, defer);
  } else if (COLL) {
    if (warp == 3) ws_collision<0>(P, m, s_obs, n_obs, lane);
    else ws_collision<1>(P, m, s_obs, n_obs, lane);
  } else if (FEST) {
    ws_estimate(P, m, lane);
  }
  if (defer) {
    grid_dependency_wait();
    k_split = ksplit_p ? *ksplit_p : K;
  }
  if (STORE_NOISE && part) {
    const int k0 = blockIdx.x * WS_B;
    block_partial<ws_threads(COLL, FEST)>(s_S, s_w, k0, min(WS_B, K - k0), K, P.T, P.lambda, k_split,
                                    noise, part + static_cast<size_t>(blockIdx.x) * part_stride(P.T));
  }
  allow_dependent_launch();
}

// The warp-specialised rollout (three warps per 32 samples, two more with the
// collision cost).
template <bool STORE_NOISE, bool COLL = false>
__global__ void __launch_bounds__(ws_threads(COLL, false))
rollout_kernel_ws(const __grid_constant__ ProbK P, const float* __restrict__ in,
                  const unsigned long long* __restrict__ iter_p, const float* __restrict__ plan,
                  float* __restrict__ S, float* __restrict__ noise,
                  const float* __restrict__ prop = nullptr,
                  const int* __restrict__ ksplit_p = nullptr,
                  const ObsK* __restrict__ obs = nullptr, float* __restrict__ part = nullptr,
                  int kwait = -1) {
  rollout_ws_block<STORE_NOISE, COLL, false>(P, in, iter_p, plan, S, noise, prop, ksplit_p, obs,
                                             part, kwait);
}

// The same for fewer samples: under an occupancy bound of four blocks per SM
// ptxas gives the kernel 122 registers instead of 95 (the same arithmetic,
// bit for bit), which is faster while few blocks share an SM and slower at
// four (see WS_SMALL_K_MAX).
template <bool STORE_NOISE>
__global__ void __launch_bounds__(ws_threads(false, false), 4)
rollout_kernel_ws_small(const __grid_constant__ ProbK P, const float* __restrict__ in,
                        const unsigned long long* __restrict__ iter_p,
                        const float* __restrict__ plan, float* __restrict__ S,
                        float* __restrict__ noise, const float* __restrict__ prop,
                        const int* __restrict__ ksplit_p, float* __restrict__ part,
                        int kwait = -1) {
  rollout_ws_block<STORE_NOISE, false, false>(P, in, iter_p, plan, S, noise, prop, ksplit_p,
                                              nullptr, part, kwait);
}

// The same with the wrench-estimate warp: four 128-thread blocks per SM (the
// shared-memory limit) need at most 128 registers per thread.
template <bool STORE_NOISE>
__global__ void __launch_bounds__(ws_threads(false, true), 4)
rollout_kernel_ws_fest(const __grid_constant__ ProbK P, const float* __restrict__ in,
                       const unsigned long long* __restrict__ iter_p,
                       const float* __restrict__ plan, float* __restrict__ S,
                       float* __restrict__ noise, const float* __restrict__ prop,
                       const int* __restrict__ ksplit_p, float* __restrict__ part) {
  rollout_ws_block<STORE_NOISE, false, true>(P, in, iter_p, plan, S, noise, prop, ksplit_p,
                                             nullptr, part);
}

// Wrench estimates F = Jbar^T (v - g(q)) (Eq. 13) for n pairs (q_i, v_i),
// [n][7] each, into F [n][6] (NaN rows at kinematic singularities), with the
// rollouts' own kinematics, dynamics and estimate.  Block B, dynamic shared
// memory fest_smem_bytes(B).
__host__ __device__ constexpr size_t fest_smem_bytes(int B) {
  return sizeof(float) * static_cast<size_t>(ROLLED_FLOATS_PER_THREAD + FEST_FLOATS_PER_THREAD) * B;
}

template <int B>
__global__ void __launch_bounds__(B)
force_estimate_kernel(const __grid_constant__ ProbK P, const float* __restrict__ q_in,
                      const float* __restrict__ v_in, int n, float* __restrict__ F_out) {
  extern __shared__ float dsm[];
  const int tid = threadIdx.x;
  const int i = blockIdx.x * B + tid;
  if (i >= n) return;  // no block-wide barrier below
  float* sl = dsm;
  float* sM = sl + NJ * LINK_FIELDS * B;
  float* sq = sM + (NJ * (NJ + 1) / 2) * B;
  float* sqd = sq + NJ * B;
  float* sh = sqd + NJ * B;
  float* sY = sh + NJ * B;
  float* sg = sY + 6 * NJ * B;
  float v[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    sq[j * B + tid] = q_in[static_cast<size_t>(i) * NJ + j];
    sqd[j * B + tid] = 0.f;
    v[j] = v_in[static_cast<size_t>(i) * NJ + j];
  }
  EEState ee;
  forward_sweep_rolled<B>(P.rb, sq, sqd, sl, tid, ee);
  backward_sweep_rolled<B, true>(P.rb, sl, sqd, sh, sM, sg, tid);
  float M[NJ * (NJ + 1) / 2], invD[NJ], F[6];
#pragma unroll
  for (int a = 0; a < NJ * (NJ + 1) / 2; ++a) M[a] = sM[a * B + tid];
  ldlt_factor<NJ>(M, invD);
  const bool ok = force_estimate<B>(sl, tid, M, invD, v, sg, ee.p, sY, F);
#pragma unroll
  for (int a = 0; a < 6; ++a) F_out[static_cast<size_t>(i) * 6 + a] = ok ? F[a] : NAN;
}

// ---------------------------------------------------------------------------
// block reductions

template <int BLOCK>
__device__ __forceinline__ float block_min(float x, float* sm) {
  x = warp_min(x);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = x;
  __syncthreads();
  if (w == 0) {
    x = lane < BLOCK / 32 ? sm[lane] : INFINITY;
    x = warp_min(x);
    if (lane == 0) sm[0] = x;
  }
  __syncthreads();
  const float r = sm[0];
  __syncthreads();
  return r;
}

template <int BLOCK, typename V>
__device__ __forceinline__ void block_sum3(V& a, V& b, V& c, V* sm) {
  a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sm[3 * w] = a; sm[3 * w + 1] = b; sm[3 * w + 2] = c; }
  __syncthreads();
  if (w == 0) {
    a = lane < BLOCK / 32 ? sm[3 * lane] : V(0);
    b = lane < BLOCK / 32 ? sm[3 * lane + 1] : V(0);
    c = lane < BLOCK / 32 ? sm[3 * lane + 2] : V(0);
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
  }
}


// Eq. 4a-4b for plan entry e = blockIdx.x = t*7 + j, and the shift.
// Costs that are not finite get weight 0; if none is finite the plan is kept
// (u* = u, next plan = u) and status 1 is reported.  out (may be null):
// tau0, status, stats and a copy of the shifted plan (OUT_* offsets).
// Each block walks K for the minimum cost and the count of non-finite costs,
// then for the weights and the weighted noise row; when S and the row are
// 16-byte aligned it reads float4 and keeps four independent accumulators so
// that the L2 loads overlap.
constexpr int UPDATE_THREADS = 512;
// float4 pairs (S, noise) in flight per thread in the weight walk: 8 for the
// single-problem update (126 blocks, one per SM: latency rules), 2 where
// blocks share SMs (serving: more resident blocks beat deeper batches)
constexpr int UPDATE_BATCH = 8;
constexpr int UPDATE_BATCH_SHARED = 2;

// The weight exp(-(S_k - S_min) / lambda) is formed in FP32 for both
// accumulator types: its rounding (a few 1e-7 relative) moves u* by about
// 1e-7 |dtau|, far below what the FP32 sums over K lose, and an FP64
// exponential per (entry, sample) would cost more than the whole update on
// this GPU's FP64 rate.  Acc = double then makes only the sums FP64.
template <typename Acc>
__device__ __forceinline__ void weight_acc(float s, float n, float m, float inv_l, Acc& z, Acc& z2,
                                           Acc& nacc, Acc& zb, bool second) {
  const Acc w = static_cast<Acc>(isfinite(s) ? expf((m - s) * inv_l) : 0.f);
  z += w;
  z2 += w * w;
  nacc += w * static_cast<Acc>(n);
  if (second) zb += w;
}

// Result of Eq. 4 for one plan entry, valid in thread 0 of the block.
template <typename Acc>
struct EntryResult {
  float u, us;  // nominal and updated value
  bool ok;      // some cost was finite
  float m;      // S_min
  Acc z, z2;    // sum of weights and of squared weights
  int bad;      // non-finite costs seen by this thread (block-reduced for e == 0)
};

// Block-wide Eq. 4a-4b for one entry: plan value u, costs S[K], noise row
// nrow[K].  Samples k >= k_split were drawn around the second proposal p:
// u* = sum_k wbar_k (u^(k) + dtau_k) = u + (Zb (p - u) + N) / Z, which is
// exactly u + N / Z when no sample used p (Zb = 0).  Every thread of the
// block must call it.  BATCH: float4 pairs in flight per thread (see
// UPDATE_BATCH).
template <typename Acc, int BATCH = UPDATE_BATCH>
__device__ __forceinline__ EntryResult<Acc> update_entry(int K, float lambda,
                                                          const float* __restrict__ S,
                                                          const float* __restrict__ nrow,
                                                          float u, bool count_bad, float p = 0.f,
                                                          int k_split = 0x7fffffff) {
  __shared__ float sm_f[32];
  __shared__ Acc sm_a[3 * 32];
  const bool vec = (K % 4 == 0) && ((reinterpret_cast<uintptr_t>(S) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(nrow) & 15) == 0);
  const int K4 = vec ? K / 4 : 0;
  float m = INFINITY;
  int bad = 0;
  {
    const float4* S4 = reinterpret_cast<const float4*>(S);
#pragma unroll 4
    for (int i = threadIdx.x; i < K4; i += UPDATE_THREADS) {
      const float4 v = S4[i];
      const float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (isfinite(a[c])) m = fminf(m, a[c]);
        else ++bad;
      }
    }
    for (int k = 4 * K4 + threadIdx.x; k < K; k += UPDATE_THREADS) {
      const float v = S[k];
      if (isfinite(v)) m = fminf(m, v);
      else ++bad;
    }
  }
  m = block_min<UPDATE_THREADS>(m, sm_f);
  const bool ok = isfinite(m);
  Acc z = Acc(0), z2 = Acc(0), nacc = Acc(0), zb = Acc(0);
  if (ok) {
    const float inv_l = 1.0f / lambda;
    const float4* S4 = reinterpret_cast<const float4*>(S);
    const float4* N4 = reinterpret_cast<const float4*>(nrow);
    Acc za[4] = {Acc(0), Acc(0), Acc(0), Acc(0)}, z2a[4] = {Acc(0), Acc(0), Acc(0), Acc(0)},
        na[4] = {Acc(0), Acc(0), Acc(0), Acc(0)}, zba[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
    // batches of BATCH float4 pairs per thread: all loads of a batch are
    // issued before the first weight, so one L2 round trip covers them
    // (K = 16384 with BATCH = 8: the whole walk in one batch)
    for (int base = threadIdx.x; base < K4; base += BATCH * UPDATE_THREADS) {
      float4 sb[BATCH], nb[BATCH];
#pragma unroll
      for (int j = 0; j < BATCH; ++j) {
        const int i = base + j * UPDATE_THREADS;
        if (i < K4) {
          sb[j] = S4[i];
          nb[j] = N4[i];
        }
      }
#pragma unroll
      for (int j = 0; j < BATCH; ++j) {
        const int i = base + j * UPDATE_THREADS;
        if (i >= K4) break;
        const float4 sv = sb[j];
        const float4 nv = nb[j];
        const int k = 4 * i;
        if constexpr (sizeof(Acc) == sizeof(double)) {
          // FP64 sums of four-sample FP32 partials: one FP64 add per quantity
          // and float4 instead of one FP64 multiply-add per sample (the FP32
          // partial of four terms loses no more than the FP32 weights do)
          float pz = 0.f, pz2 = 0.f, pn = 0.f, pb = 0.f;
          weight_acc(sv.x, nv.x, m, inv_l, pz, pz2, pn, pb, k >= k_split);
          weight_acc(sv.y, nv.y, m, inv_l, pz, pz2, pn, pb, k + 1 >= k_split);
          weight_acc(sv.z, nv.z, m, inv_l, pz, pz2, pn, pb, k + 2 >= k_split);
          weight_acc(sv.w, nv.w, m, inv_l, pz, pz2, pn, pb, k + 3 >= k_split);
          za[0] += pz;
          z2a[0] += pz2;
          na[0] += pn;
          zba[0] += pb;
        } else {
          weight_acc(sv.x, nv.x, m, inv_l, za[0], z2a[0], na[0], zba[0], k >= k_split);
          weight_acc(sv.y, nv.y, m, inv_l, za[1], z2a[1], na[1], zba[1], k + 1 >= k_split);
          weight_acc(sv.z, nv.z, m, inv_l, za[2], z2a[2], na[2], zba[2], k + 2 >= k_split);
          weight_acc(sv.w, nv.w, m, inv_l, za[3], z2a[3], na[3], zba[3], k + 3 >= k_split);
        }
      }
    }
    for (int k = 4 * K4 + threadIdx.x; k < K; k += UPDATE_THREADS)
      weight_acc(S[k], nrow[k], m, inv_l, za[0], z2a[0], na[0], zba[0], k >= k_split);
    z = (za[0] + za[1]) + (za[2] + za[3]);
    z2 = (z2a[0] + z2a[1]) + (z2a[2] + z2a[3]);
    nacc = (na[0] + na[1]) + (na[2] + na[3]);
    zb = (zba[0] + zba[1]) + (zba[2] + zba[3]);
  }
  block_sum3<UPDATE_THREADS>(z, z2, nacc, sm_a);
  Acc zbs = zb, d1 = Acc(0), d2 = Acc(0);
  if (k_split < K) {
    __syncthreads();
    block_sum3<UPDATE_THREADS>(zbs, d1, d2, sm_a);
  }
  Acc nbad = Acc(0);
  if (count_bad) {
    nbad = static_cast<Acc>(bad);
    d1 = d2 = Acc(0);
    __syncthreads();
    block_sum3<UPDATE_THREADS>(nbad, d1, d2, sm_a);
  }
  __syncthreads();  // shared scratch may be reused by the caller's next entry
  EntryResult<Acc> r;
  r.u = u;
  r.ok = ok;
  r.m = m;
  r.z = z;
  r.z2 = z2;
  r.bad = static_cast<int>(nbad);
  if (!ok) {
    r.us = u;
  } else if (k_split < K) {
    r.us = static_cast<float>(static_cast<Acc>(u) +
                              (zbs * (static_cast<Acc>(p) - static_cast<Acc>(u)) + nacc) / z);
  } else {
    r.us = static_cast<float>(static_cast<Acc>(u) + nacc / z);
  }
  return r;
}

// Plan outputs of one entry e = t*7 + j of Eq. 4 (thread 0 of its block):
// u* and the shifted plan (u*_{t+1} moves to t; the last entry repeats),
// also into the output record and the caller's buffers when given; when no
// cost was finite the plan is kept as it is, unshifted.
__device__ __forceinline__ void write_entry(int e, int T, bool ok, float us, float* ustar,
                                            float* plan_next, float* out, float* tau_dst,
                                            float* plan_dst) {
  const int t = e / NJ;
  if (ok) {
    if (t >= 1) plan_next[e - NJ] = us;
    if (t == T - 1) plan_next[e] = us;
    if (out) {
      if (t >= 1) out[OUT_PLAN + e - NJ] = us;
      if (t == T - 1) out[OUT_PLAN + e] = us;
    }
    if (plan_dst) {
      if (t >= 1) plan_dst[e - NJ] = us;
      if (t == T - 1) plan_dst[e] = us;
    }
  } else {
    plan_next[e] = us;
    if (out) out[OUT_PLAN + e] = us;
    if (plan_dst) plan_dst[e] = us;
  }
  ustar[e] = us;
  if (out && e < NJ) out[OUT_TAU0 + e] = us;
  if (tau_dst && e < NJ) tau_dst[e] = us;
}

// The record's status and Eq. 4a statistics (block of entry 0): status,
// S_min, Z, n_eff = Z^2 / sum w^2, number of non-finite costs.
__device__ __forceinline__ void write_stats(float* out, bool ok, float m, double z, double z2,
                                            double bad) {
  reinterpret_cast<int*>(out)[OUT_STATUS] = ok ? 0 : 1;
  out[OUT_STATS + 0] = m;
  out[OUT_STATS + 1] = static_cast<float>(z);
  out[OUT_STATS + 2] = ok ? static_cast<float>(z * z / z2) : 0.f;
  out[OUT_STATS + 3] = static_cast<float>(bad);
}

// Eq. 4 from caller-supplied costs S [K] and noise [T*7][K] (one block per
// plan entry), with the shift; out, iter_p, tau_dst, plan_dst may be null.
template <typename Acc>
__global__ void __launch_bounds__(UPDATE_THREADS)
update_kernel(int K, int T, float lambda, const float* __restrict__ S,
              const float* __restrict__ noise, const float* __restrict__ plan,
              float* __restrict__ ustar, float* __restrict__ plan_next, float* __restrict__ out,
              unsigned long long* __restrict__ iter_p, const float* __restrict__ prop = nullptr,
              const int* ksplit_p = nullptr, float* __restrict__ tau_dst = nullptr,
              float* __restrict__ plan_dst = nullptr) {
  const int e = blockIdx.x;
  const float* nrow = noise + static_cast<size_t>(e) * K;
  const float pe = prop ? prop[e] : 0.f;
  const int k_split = ksplit_p ? *ksplit_p : K;
  const EntryResult<Acc> r =
      update_entry<Acc>(K, lambda, S, nrow, plan[e], e == 0, k_split < K ? pe : 0.f, k_split);
  if (threadIdx.x != 0) return;
  write_entry(e, T, r.ok, r.us, ustar, plan_next, out, tau_dst, plan_dst);
  if (e == 0) {
    if (out) write_stats(out, r.ok, r.m, static_cast<double>(r.z), static_cast<double>(r.z2), r.bad);
    if (iter_p && r.ok) *iter_p += 1ull;
  }
}

// Log-sum-exp accumulator over rollout blocks: sums relative to the running
// minimum m (weights exp(-(S - m) / lambda)); a new minimum rescales what is
// held.  m = +inf holds nothing.
template <typename Acc>
struct Lse {
  float m;
  Acc z, n, zs, z2;
};

template <typename Acc>
__device__ __forceinline__ Lse<Acc> lse_merge(const Lse<Acc>& a, const Lse<Acc>& b, float inv_l) {
  if (!isfinite(b.m)) return a;
  if (!isfinite(a.m)) return b;
  Lse<Acc> r;
  r.m = fminf(a.m, b.m);
  const Acc ca = static_cast<Acc>(expf((r.m - a.m) * inv_l));
  const Acc cb = static_cast<Acc>(expf((r.m - b.m) * inv_l));
  r.z = ca * a.z + cb * b.z;
  r.n = ca * a.n + cb * b.n;
  r.zs = ca * a.zs + cb * b.zs;
  r.z2 = ca * ca * a.z2 + cb * cb * b.z2;
  return r;
}

template <typename Acc>
__device__ __forceinline__ Lse<Acc> lse_shfl(const Lse<Acc>& a, int o) {
  Lse<Acc> r;
  r.m = __shfl_xor_sync(0xffffffffu, a.m, o);
  r.z = __shfl_xor_sync(0xffffffffu, a.z, o);
  r.n = __shfl_xor_sync(0xffffffffu, a.n, o);
  r.zs = __shfl_xor_sync(0xffffffffu, a.zs, o);
  r.z2 = __shfl_xor_sync(0xffffffffu, a.z2, o);
  return r;
}

// Eq. 4a-4b of a step from the rollout blocks' partials (block_partial;
// nb records of pstride floats), one block per plan entry e:
//   m = min_b m_b,  c_b = exp(-(m_b - m) / lambda)  (0 for a block with no
//   finite cost),  Z = sum_b c_b Z_b,  N_e = sum_b c_b N_b[e],
//   u*_e = u_e + N_e / Z, or with a second proposal p for samples
//   k >= k_split: u*_e = u_e + (Zs (p_e - u_e) + N_e) / Z, Zs = sum_b c_b Zs_b
// (the merge rule of the sharded update), then the shift.  One pass over the
// partials: each thread folds its blocks into a running log-sum-exp
// accumulator, and the threads' accumulators merge by the same rule.
// Launched as a programmatic dependent of the rollouts.  When this update
// has a second proposal (k_split < K), the last block (done counter) resets
// the counter and, through ctl_reset (= ksplit_p's {k_split, K}), consumes
// the proposal (k_split := K).  With seq_in (host steps, whose output record
// is mapped host memory) every block fences its record entries to system
// scope before the count and the last block then writes *seq_in to the
// record's OUT_SEQ word, after which the host may read the whole record.
// Acc: the type of the sums over blocks.
constexpr int MERGE_THREADS = 256;

template <typename Acc>
__global__ void __launch_bounds__(MERGE_THREADS)
merge_kernel(int K, int T, float lambda, int nb, int pstride, const float* part,
             const float* __restrict__ plan, float* __restrict__ ustar,
             float* __restrict__ plan_next, float* __restrict__ out,
             unsigned long long* __restrict__ iter_p, const float* __restrict__ prop,
             const int* ksplit_p, float* __restrict__ tau_dst, float* __restrict__ plan_dst,
             unsigned* done, int* ctl_reset, const unsigned* seq_in) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __shared__ Lse<Acc> sm[MERGE_THREADS / 32];
  __shared__ float sm_bad[MERGE_THREADS / 32];
  const int e = blockIdx.x;
  const float u = plan[e];
  const float pe = prop ? prop[e] : 0.f;
  const int k_split = ksplit_p ? *ksplit_p : K;
  const float inv_l = 1.0f / lambda;
  Lse<Acc> acc{INFINITY, Acc(0), Acc(0), Acc(0), Acc(0)};
  float bad = 0.f;
  for (int b0 = threadIdx.x; b0 < nb; b0 += 4 * MERGE_THREADS) {
    // up to four partials per thread in flight before the first is used
    float4 hd[4];
    float nv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = b0 + j * MERGE_THREADS;
      if (b < nb) {
        const float* pb = part + static_cast<size_t>(b) * pstride;
        hd[j] = __ldcg(reinterpret_cast<const float4*>(pb));  // m_b, Z_b, sum w^2, Zs_b
        nv[j] = __ldcg(pb + PART_HEAD + e);
        if (e == 0) bad += __ldcg(pb + 4);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (b0 + j * MERGE_THREADS < nb) {
        const Lse<Acc> p{hd[j].x, static_cast<Acc>(hd[j].y), static_cast<Acc>(nv[j]),
                         static_cast<Acc>(hd[j].w), static_cast<Acc>(hd[j].z)};
        acc = lse_merge(acc, p, inv_l);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc = lse_merge(acc, lse_shfl(acc, o), inv_l);
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sm[w] = acc;
    sm_bad[w] = bad;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int i = 1; i < MERGE_THREADS / 32; ++i) {
    acc = lse_merge(acc, sm[i], inv_l);
    bad += sm_bad[i];
  }
  const bool ok = isfinite(acc.m);
  float us = u;
  if (ok) {
    us = k_split < K
             ? static_cast<float>(static_cast<Acc>(u) +
                                  (acc.zs * (static_cast<Acc>(pe) - static_cast<Acc>(u)) + acc.n) /
                                      acc.z)
             : static_cast<float>(static_cast<Acc>(u) + acc.n / acc.z);
  }
  write_entry(e, T, ok, us, ustar, plan_next, out, tau_dst, plan_dst);
  if (e == 0) {
    if (out) write_stats(out, ok, acc.m, static_cast<double>(acc.z), static_cast<double>(acc.z2),
                         static_cast<double>(bad));
    if (iter_p && ok) *iter_p += 1ull;
  }
  // the last block to finish resets the counter; with a second proposal in
  // this update it consumes it (every block read k_split above, and the
  // acquire-release count orders those reads before the reset), and in a
  // host step it writes the completion word after every block's entries
  const bool second = ctl_reset && k_split < K;
  if (second || seq_in) {
    if (seq_in) __threadfence_system();
    if (atomic_add_acq_rel(done, 1u) == gridDim.x - 1) {
      *done = 0u;
      if (second) ctl_reset[0] = ctl_reset[1];
      if (seq_in) {
        __threadfence_system();
        reinterpret_cast<volatile unsigned*>(out)[OUT_SEQ] = *seq_in;
      }
    }
  }
}

// The model itself as a plant: state i of n advanced by `substeps` steps of
// dt / substeps under the constant torque tau[i] (zero-order hold), with
// the same dynamics, contact and Euler step as the rollouts.  in: [n][25]
// records (q, qd, goal, plane); out: [n][14] (q, qd).
static __global__ void simulate_kernel(const __grid_constant__ ProbK P, int n, const float* __restrict__ in,
                                const float* __restrict__ tau, int substeps, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* r = in + static_cast<size_t>(i) * IN_FLOATS;
  float q[NJ], qd[NJ], u[NJ], q_lo[NJ], qd_lo[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    q[j] = r[j];
    qd[j] = r[NJ + j];
    q_lo[j] = qd_lo[j] = 0.f;
    u[j] = tau[static_cast<size_t>(i) * NJ + j];
  }
  const float plane[4] = {r[21], r[22], r[23], r[24]};
  const bool contact = P.cost.contact != 0;
  const float h = P.dt / static_cast<float>(substeps);
  for (int s = 0; s < substeps; ++s) {
    LinkState ls[NJ];
    EEState ee;
    forward_sweep(P.rb, q, qd, ls, ee);
    float hb[NJ], M[NJ * (NJ + 1) / 2];
    backward_sweep(P.rb, qd, ls, hb, M);
    float rhs[NJ];
    const float f = contact ? contact_force(P.cost, plane, ee) : 0.f;
    const float Fc[3] = {f * plane[0], f * plane[1], f * plane[2]};
    float pxF[3];
    cross3(ee.p, Fc, pxF);
#pragma unroll
    for (int j = 0; j < NJ; ++j) rhs[j] = u[j] + dot3(ls[j].z, pxF) + dot3(ls[j].w, Fc) - hb[j];
    float qdd[NJ];
    ldlt_solve(M, rhs, qdd);
#pragma unroll
    for (int j = 0; j < NJ; ++j) euler_step(qdd[j], h, q[j], q_lo[j], qd[j], qd_lo[j]);
  }
  float* o = out + static_cast<size_t>(i) * 2 * NJ;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    o[j] = q[j];
    o[NJ + j] = qd[j];
  }
}

// Raw Philox words of (iter, t) for samples k0 + i, i < count: out[8 i + 4 call + w].
static __global__ void noise_words_kernel(uint32_t key0, uint32_t key1, uint64_t iter, uint32_t k0,
                                   int count, uint32_t t, uint32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
#pragma unroll
  for (uint32_t call = 0; call < 2; ++call) {
    uint32_t c[4] = {k0 + static_cast<uint32_t>(i), 2u * t + call, static_cast<uint32_t>(iter),
                     static_cast<uint32_t>(iter >> 32)};
    philox4x32_10(c, key0, key1);
#pragma unroll
    for (int w = 0; w < 4; ++w) out[8 * i + 4 * call + w] = c[w];
  }
}

// Bias torque at rest, h(q, 0) = g(q) (gravity compensation), one thread.
static __global__ void gravity_kernel(const __grid_constant__ ProbK P, const float* __restrict__ q_in,
                                      float* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float q[NJ], qd[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    q[j] = q_in[j];
    qd[j] = 0.f;
  }
  LinkState ls[NJ];
  EEState ee;
  forward_sweep(P.rb, q, qd, ls, ee);
  float h[NJ], M[NJ * (NJ + 1) / 2];
  backward_sweep(P.rb, qd, ls, h, M);
  for (int j = 0; j < NJ; ++j) out[j] = h[j];
}

// End-effector pose at q (one thread): p (3) and R (9, row-major).
static __global__ void ee_pose_kernel(const __grid_constant__ ProbK P, const float* __restrict__ q_in,
                               float* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float q[NJ], qd[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    q[j] = q_in[j];
    qd[j] = 0.f;
  }
  LinkState ls[NJ];
  EEState ee;
  forward_sweep(P.rb, q, qd, ls, ee);
  for (int a = 0; a < 3; ++a) out[a] = ee.p[a];
  for (int a = 0; a < 9; ++a) out[3 + a] = ee.R[a];
}

}  // namespace mppi_dev
