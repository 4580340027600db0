// Host side of the C ABI declared in include/mppi.h: parameter checking, the
// one-time conversion of the arm into the kernels' link frames, device buffer
// ownership, kernel launches and CUDA-graph replay of one update.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>

#include "mppi.h"
#include "mppi_kernels.cuh"

using namespace mppi_dev;

#define MPPI_VERSION_STR "paper_2609_02020_b300 mppi 1.0 (sm_103a)"

// Rollout kernel used when mppi_config.variant is 0.  While there are too
// few samples to give each SM scheduler more than a couple of warps, one
// sample's dependency chain sets the time, and the warp-specialised kernel
// (three warps per 32 samples) shortens it most - as long as all of its
// blocks are resident at once (one wave; four 56 KB blocks per SM).  Beyond
// that, throughput bounds and the register-unrolled kernel's lower
// instruction count wins.  Measured on B300 at T = 18 (rollout only, us):
//   K        512    4096   16384   24576   32768   65536
//   ws        67      75      93     174     184     344
//   rolled   114     104     103     139     139     268
//   register 114     128     127     125     122     214
// The rolled kernel carries every optional cost term; the warp-specialised
// kernel the collision cost or the wrench-estimate cost alone.  With one of
// those (coll, fest) the alternative is the rolled kernel.
#ifndef WS_SMALL_K_MAX
// Up to this K the plain warp-specialised rollout runs as
// rollout_kernel_ws_small.  Rollout at T = 18 on B300 (us), the default
// instantiation against the small one: K = 512-2048: 62.5-64.0 against
// 60.2-61.5; 4096: 64.5 against 62.6; 8192: 68.2 against 67.5; 12288: 84.4
// for both; 16384: 86.6 against 87.7 (on another box both within 1 % at
// every K).
#define WS_SMALL_K_MAX 8192
#endif

static int default_variant(int K, bool coll, bool fest) {
  const int other = (coll || fest) ? 2 : 1;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = coll ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                   &per_sm, rollout_kernel_ws<true, true>, ws_threads(true, false),
                   ws_smem_bytes(true))
        : fest ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     &per_sm, rollout_kernel_ws_fest<true>, ws_threads(false, true),
                     ws_smem_bytes(false))
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     &per_sm, rollout_kernel_ws<true, false>, ws_threads(false, false),
                     ws_smem_bytes(false));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return other;
  }
  const long long ws_blocks = (static_cast<long long>(K) + WS_B - 1) / WS_B;
  return ws_blocks <= static_cast<long long>(sms) * per_sm ? 3 : other;
}

static_assert(MPPI_OBS_MAX == OBS_MAX, "obstacle capacity of the ABI and the kernels");

struct mppi_s {
  ProbK P;
  int reduce_fp64 = 0;
  int use_graph = 1;
  int variant = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // device buffers
  float* d_plan[2] = {nullptr, nullptr};  // ping-pong nominal plans [T][7]
  float* d_ustar = nullptr;               // u* before the shift [T][7]
  float* d_S = nullptr;                   // costs [K]
  float* d_noise = nullptr;               // noise [T*7][K]
  float* d_in = nullptr;                  // staged inputs (IN_FLOATS)
  float* d_out = nullptr;                 // tau0 / status / stats / plan
  float* d_scratch_plan = nullptr;        // [2][T][7] for timing runs
  float* d_misc = nullptr;                // 32 floats for small helper kernels
  uint32_t* d_words = nullptr;            // 8 x 1024 words for mppi_noise_words
  float* d_prop = nullptr;                // second proposal plan [T][7]
  int* d_ctl = nullptr;                   // {k_split of the next update, K}
  ObsK* d_obs = nullptr;                  // obstacle capsules of Eq. 15
  float* d_fext = nullptr;                // F_ext of the constant external wrench (6)
  float* d_part = nullptr;                // the rollout blocks' Eq. 4 partials [nb][part_stride(T)]
  unsigned* d_done = nullptr;             // merge blocks finished (reset by the last one)
  int feat = 0;                           // FEAT_* cost terms of the rollouts
  unsigned long long* d_iter = nullptr;
  // pinned host staging
  float* h_in = nullptr;
  float* h_out = nullptr;                 // pinned, mapped: host steps write it directly
  float* h_out_dev = nullptr;             // h_out as the device sees it
  bool out_on_host = false;               // the last update's record is in h_out, not d_out
  unsigned host_seq = 0;                  // sequence word of the last host step
  int cur = 0;  // index of the current nominal plan
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::string err;
  int out_floats = 0;
};

static thread_local std::string g_create_err;

static int fail(mppi_s* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

#define CUDA_TRY(h, call)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail((h), e_ == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

// ---------------------------------------------------------------------------
// arm conversion (double precision, once per handle)

namespace {

struct M3 {
  double a[3][3];
};

M3 m3_identity() {
  M3 r{};
  r.a[0][0] = r.a[1][1] = r.a[2][2] = 1.0;
  return r;
}
M3 m3_mul(const M3& A, const M3& B) {
  M3 C{};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) C.a[i][j] += A.a[i][k] * B.a[k][j];
  return C;
}
M3 m3_t(const M3& A) {
  M3 B{};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B.a[i][j] = A.a[j][i];
  return B;
}
void m3_v(const M3& A, const double x[3], double y[3]) {
  for (int i = 0; i < 3; ++i) y[i] = A.a[i][0] * x[0] + A.a[i][1] * x[1] + A.a[i][2] * x[2];
}
// fixed joint rotation from roll, pitch, yaw: Rz(yaw) Ry(pitch) Rx(roll)
M3 from_rpy(const double rpy[3]) {
  const double sr = std::sin(rpy[0]), cr = std::cos(rpy[0]);
  const double sp = std::sin(rpy[1]), cp = std::cos(rpy[1]);
  const double sy = std::sin(rpy[2]), cy = std::cos(rpy[2]);
  M3 R{};
  R.a[0][0] = cy * cp; R.a[0][1] = cy * sp * sr - sy * cr; R.a[0][2] = cy * sp * cr + sy * sr;
  R.a[1][0] = sy * cp; R.a[1][1] = sy * sp * sr + cy * cr; R.a[1][2] = sy * sp * cr - cy * sr;
  R.a[2][0] = -sp;     R.a[2][1] = cp * sr;                R.a[2][2] = cp * cr;
  return R;
}
// a rotation P with P e_z = a (a unit)
M3 z_to_axis(const double a[3]) {
  const double c = a[2];
  if (c > 1.0 - 1e-12) return m3_identity();
  if (c < -1.0 + 1e-12) {
    M3 R{};
    R.a[0][0] = 1.0; R.a[1][1] = -1.0; R.a[2][2] = -1.0;
    return R;
  }
  // axis k = e_z x a / |e_z x a|, angle acos(c)
  double k[3] = {-a[1], a[0], 0.0};
  const double s = std::sqrt(k[0] * k[0] + k[1] * k[1]);
  k[0] /= s; k[1] /= s;
  const double C = 1.0 - c;
  M3 R{};
  const double K[3][3] = {{0, -k[2], k[1]}, {k[2], 0, -k[0]}, {-k[1], k[0], 0}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R.a[i][j] = (i == j ? c : 0.0) + s * K[i][j] + C * k[i] * k[j];
  return R;
}

bool finite_all(const double* x, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

// Host image of the obstacle buffer from n capsules (a xyz, b xyz, radius).
template <typename R>
void fill_obs(int n, const R* obs, ObsK* out) {
  std::memset(out, 0, sizeof(*out));
  out->n = n;
  for (int o = 0; o < n; ++o)
    for (int a = 0; a < 7; ++a) out->o[o][a] = static_cast<float>(obs[7 * o + a]);
}

int convert(const mppi_robot* rb, const mppi_cost* c, const mppi_config* cfg, ProbK* P,
            std::string* why) {
  if (rb->n != MPPI_NJ) { *why = "robot.n must be 7"; return -1; }
  if (!(cfg->dt > 0.0) || !std::isfinite(cfg->dt)) { *why = "dt must be > 0"; return -1; }
  if (cfg->T < 1 || cfg->T > MPPI_T_MAX) { *why = "T must be in 1..256"; return -1; }
  if (cfg->K < 1 || cfg->K > MPPI_K_MAX) { *why = "K must be in 1..2^22"; return -1; }
  if (!(cfg->lambda > 0.0) || !std::isfinite(cfg->lambda)) { *why = "lambda must be > 0"; return -1; }
  for (int j = 0; j < 7; ++j)
    if (!(cfg->sigma[j] >= 0.0) || !std::isfinite(cfg->sigma[j])) { *why = "sigma must be >= 0"; return -1; }
  const double* flat = &rb->joint_xyz[0][0];
  const int nflat = static_cast<int>((reinterpret_cast<const char*>(&rb->gravity[3]) -
                                      reinterpret_cast<const char*>(flat)) / sizeof(double));
  if (!finite_all(flat, nflat)) { *why = "robot parameters must be finite"; return -1; }
  for (int j = 0; j < 7; ++j) {
    if (!(rb->mass[j] > 0.0)) { *why = "masses must be > 0"; return -1; }
    if (rb->armature[j] < 0.0 || rb->damping[j] < 0.0) { *why = "armature and damping must be >= 0"; return -1; }
    const double* a = rb->axis[j];
    const double na = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if (std::fabs(na - 1.0) > 1e-6) { *why = "joint axes must be unit vectors"; return -1; }
    if (!(rb->q_min[j] <= rb->q_max[j])) { *why = "q_min must be <= q_max"; return -1; }
  }
  const double* cflat = &c->w_pos[0];
  if (!finite_all(cflat, 3 + 3 + 3 + 4 + 7 + 1)) { *why = "cost weights must be finite"; return -1; }
  if (c->contact && (!std::isfinite(c->k_contact) || !std::isfinite(c->d_contact) ||
                     c->k_contact < 0.0 || c->d_contact < 0.0)) {
    *why = "contact stiffness and damping must be finite and >= 0";
    return -1;
  }
  if (c->force_estimate && (!finite_all(c->w_force6, 6) || !finite_all(c->f_des6, 6) ||
                            !finite_all(c->w_reg6, 6))) {
    *why = "wrench-estimate weights must be finite";
    return -1;
  }
  if (c->collision < 0 || c->collision > 2) { *why = "collision must be 0, 1 or 2"; return -1; }
  if (c->ext_wrench && !finite_all(c->f_ext, 6)) { *why = "f_ext must be finite"; return -1; }
  if (c->collision) {
    if (!std::isfinite(c->w_collision) || !std::isfinite(c->d_th_self) ||
        !std::isfinite(c->d_th_obs) || !finite_all(c->link_radius, 7)) {
      *why = "collision weights, thresholds and radii must be finite";
      return -1;
    }
    for (int j = 0; j < 7; ++j)
      if (c->link_radius[j] < 0.0) { *why = "link radii must be >= 0"; return -1; }
    if (c->n_obstacles < 0 || c->n_obstacles > MPPI_OBS_MAX) {
      *why = "n_obstacles must be in 0..8";
      return -1;
    }
    if (!finite_all(&c->obstacles[0][0], 7 * c->n_obstacles)) {
      *why = "obstacles must be finite";
      return -1;
    }
    for (int o = 0; o < c->n_obstacles; ++o)
      if (c->obstacles[o][6] < 0.0) { *why = "obstacle radii must be >= 0"; return -1; }
  }

  std::memset(P, 0, sizeof(*P));
  M3 Pprev = m3_identity();
  for (int i = 0; i < 7; ++i) {
    const double* a = rb->axis[i];
    const double an = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double au[3] = {a[0] / an, a[1] / an, a[2] / an};
    const M3 Pi = z_to_axis(au);
    const M3 E = from_rpy(rb->joint_rpy[i]);
    const M3 F = m3_mul(m3_mul(m3_t(Pprev), E), Pi);
    LinkK& L = P->rb.L[i];
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) L.F[3 * r + s] = static_cast<float>(F.a[r][s]);
    double rk[3], ck[3];
    m3_v(m3_t(Pprev), rb->joint_xyz[i], rk);
    m3_v(m3_t(Pi), rb->com[i], ck);
    for (int r = 0; r < 3; ++r) {
      L.r[r] = static_cast<float>(rk[r]);
      L.c[r] = static_cast<float>(ck[r]);
    }
    const double* t = rb->inertia[i];
    M3 Ig{};
    Ig.a[0][0] = t[0]; Ig.a[1][1] = t[1]; Ig.a[2][2] = t[2];
    Ig.a[0][1] = Ig.a[1][0] = t[3];
    Ig.a[0][2] = Ig.a[2][0] = t[4];
    Ig.a[1][2] = Ig.a[2][1] = t[5];
    const M3 Ik = m3_mul(m3_mul(m3_t(Pi), Ig), Pi);
    L.I[0] = static_cast<float>(Ik.a[0][0]);
    L.I[1] = static_cast<float>(Ik.a[1][1]);
    L.I[2] = static_cast<float>(Ik.a[2][2]);
    L.I[3] = static_cast<float>(Ik.a[0][1]);
    L.I[4] = static_cast<float>(Ik.a[0][2]);
    L.I[5] = static_cast<float>(Ik.a[1][2]);
    L.m = static_cast<float>(rb->mass[i]);
    L.arm = static_cast<float>(rb->armature[i]);
    L.damp = static_cast<float>(rb->damping[i]);
    Pprev = Pi;
  }
  double ek[3];
  m3_v(m3_t(Pprev), rb->ee_xyz, ek);
  const M3 Q = m3_t(Pprev);
  for (int r = 0; r < 3; ++r) {
    P->rb.ee[r] = static_cast<float>(ek[r]);
    P->rb.g[r] = static_cast<float>(rb->gravity[r]);
    for (int s = 0; s < 3; ++s) P->rb.Qee[3 * r + s] = static_cast<float>(Q.a[r][s]);
  }
  for (int j = 0; j < 7; ++j) {
    P->rb.qmin[j] = static_cast<float>(rb->q_min[j]);
    P->rb.qmax[j] = static_cast<float>(rb->q_max[j]);
    P->rb.qdmax[j] = static_cast<float>(rb->qd_max[j]);
    P->rb.taumax[j] = static_cast<float>(rb->tau_max[j]);
  }
  CostK& k = P->cost;
  for (int a = 0; a < 3; ++a) {
    k.wpos[a] = static_cast<float>(c->w_pos[a]);
    k.wori[a] = static_cast<float>(c->w_ori[a]);
  }
  k.wforce = static_cast<float>(c->w_force);
  k.fdes = static_cast<float>(c->f_des);
  k.wreg = static_cast<float>(c->w_reg);
  k.wqlim = static_cast<float>(c->w_qlim);
  k.wqdlim = static_cast<float>(c->w_qdlim);
  k.wtau = static_cast<float>(c->w_tau);
  k.wpost = static_cast<float>(c->w_posture);
  for (int j = 0; j < 7; ++j) k.qpost[j] = static_cast<float>(c->q_posture[j]);
  k.wterm = static_cast<float>(c->w_terminal);
  k.contact = c->contact ? 1 : 0;
  k.kc = static_cast<float>(c->k_contact);
  k.dc = static_cast<float>(c->d_contact);
  k.coll = c->collision;
  k.wcoll = static_cast<float>(c->w_collision);
  k.dth_self = static_cast<float>(c->d_th_self);
  k.dth_obs = static_cast<float>(c->d_th_obs);
  for (int j = 0; j < 7; ++j) {
    k.lrad[j] = static_cast<float>(c->link_radius[j]);
    // link j's segment runs from joint j's origin to joint j+1's (the
    // end-effector point for the last link): a rigid length
    const double* v = j + 1 < 7 ? rb->joint_xyz[j + 1] : rb->ee_xyz;
    const double a = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    k.seg_a[j] = static_cast<float>(a);
    k.seg_ia[j] = a > 1e-12 ? static_cast<float>(1.0 / a) : 0.f;
    k.seg_h[j] = static_cast<float>(0.5 * std::sqrt(a));
  }
  for (int i = 0, n = 0; i < 7 - 2; ++i)
    for (int j = i + 2; j < 7; ++j, ++n)
      k.self_b2[n] = pair_skip_b2(k.dth_self, k.lrad[i], k.lrad[j], k.seg_h[i], k.seg_h[j]);
  k.fest = c->force_estimate ? 1 : 0;
  for (int a = 0; a < 6; ++a) {
    k.wf6[a] = static_cast<float>(c->w_force6[a]);
    k.fdes6[a] = static_cast<float>(c->f_des6[a]);
    k.wreg6[a] = static_cast<float>(c->w_reg6[a]);
  }
  P->fext = nullptr;  // set by mppi_create once the handle's buffer exists
  P->dt = static_cast<float>(cfg->dt);
  P->lambda = static_cast<float>(cfg->lambda);
  for (int j = 0; j < 7; ++j) P->sigma[j] = static_cast<float>(cfg->sigma[j]);
  P->T = cfg->T;
  P->K = cfg->K;
  P->key0 = static_cast<uint32_t>(cfg->seed);
  P->key1 = static_cast<uint32_t>(cfg->seed >> 32);
  return 0;
}

// ---------------------------------------------------------------------------
// launches

template <int FEAT>
cudaError_t launch_rolled(mppi_s* h, int grid, const float* in, const float* plan, float* S,
                          float* noise, float* part) {
  const size_t smem = rolled_smem_bytes(h->P.T, ROLLOUT_BLOCK, FEAT);
  if (noise)
    rollout_kernel_rolled<true, ROLLOUT_BLOCK, FEAT><<<grid, ROLLOUT_BLOCK, smem, h->stream>>>(
        h->P, in, h->d_iter, plan, S, noise, h->d_prop, h->d_ctl, h->d_obs, part);
  else
    rollout_kernel_rolled<false, ROLLOUT_BLOCK, FEAT><<<grid, ROLLOUT_BLOCK, smem, h->stream>>>(
        h->P, in, h->d_iter, plan, S, nullptr, h->d_prop, h->d_ctl, h->d_obs, nullptr);
  return cudaGetLastError();
}

// Opt the rolled kernels of feature set FEAT in to more than 48 KB of
// dynamic shared memory when horizon T needs it.
template <int FEAT>
cudaError_t prepare_rolled(int T) {
  const size_t smem = rolled_smem_bytes(T, ROLLOUT_BLOCK, FEAT);
  if (smem <= 48 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(rollout_kernel_rolled<true, ROLLOUT_BLOCK, FEAT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(rollout_kernel_rolled<false, ROLLOUT_BLOCK, FEAT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(smem));
}

cudaError_t prepare_rollout(mppi_s* h) {
  if (h->feat == FEAT_COLL && h->variant == 3) {
    const int smem = static_cast<int>(ws_smem_bytes(true));
    cudaError_t e = cudaFuncSetAttribute(rollout_kernel_ws<true, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(rollout_kernel_ws<false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  }
  if (h->feat == FEAT_FEST && h->variant == 3) {
    const int smem = static_cast<int>(ws_smem_bytes(false));
    cudaError_t e = cudaFuncSetAttribute(rollout_kernel_ws_fest<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(rollout_kernel_ws_fest<false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  }
  switch (h->feat) {
    case FEAT_FEST: return prepare_rolled<FEAT_FEST>(h->P.T);
    case FEAT_COLL: return prepare_rolled<FEAT_COLL>(h->P.T);
    case FEAT_FEST | FEAT_COLL: return prepare_rolled<FEAT_FEST | FEAT_COLL>(h->P.T);
    default: break;
  }
  if (h->variant == 2) return prepare_rolled<0>(h->P.T);
  if (h->variant == 3) {
    const size_t smem = ws_smem_bytes();
    for (auto f : {rollout_kernel_ws_small<true>, rollout_kernel_ws_small<false>}) {
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaFuncSetAttribute(rollout_kernel_ws<true, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(rollout_kernel_ws<false, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  }
  return cudaSuccess;
}

// Launch configuration of a programmatic dependent launch on the handle's
// stream: the grid may start while the previous kernel still runs and waits
// (griddepcontrol.wait) before it reads what that kernel writes.
struct PdlLaunch {
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t lc;
  PdlLaunch(dim3 grid, dim3 block, size_t smem, cudaStream_t st) : at{}, lc{} {
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    lc.attrs = at;
    lc.numAttrs = 1;
  }
};

// part non-null (with noise): every rollout block also leaves its Eq. 4
// partials there for merge_kernel.  kwait >= 0: a proposal kernel that
// installs a second proposal with k_split = kwait immediately precedes on
// the stream; the plain warp-specialised kernel then overlaps it (blocks
// below kwait do not wait for it), the other kernels wait for it as usual.
cudaError_t launch_rollout(mppi_s* h, const float* in, const float* plan, float* S, float* noise,
                           float* part = nullptr, int kwait = -1) {
  if (!noise) part = nullptr;
  const int grid = (h->P.K + ROLLOUT_BLOCK - 1) / ROLLOUT_BLOCK;
  if (h->feat == FEAT_COLL && h->variant == 3) {
    // the collision cost on two more warps of the warp-specialised kernel
    const int wgrid = (h->P.K + WS_B - 1) / WS_B;
    const size_t smem = ws_smem_bytes(true);
    if (noise)
      rollout_kernel_ws<true, true><<<wgrid, ws_threads(true, false), smem, h->stream>>>(
          h->P, in, h->d_iter, plan, S, noise, h->d_prop, h->d_ctl, h->d_obs, part);
    else
      rollout_kernel_ws<false, true><<<wgrid, ws_threads(true, false), smem, h->stream>>>(
          h->P, in, h->d_iter, plan, S, nullptr, h->d_prop, h->d_ctl, h->d_obs, nullptr);
    return cudaGetLastError();
  }
  if (h->feat == FEAT_FEST && h->variant == 3) {
    // the wrench-estimate cost on a fourth warp of the warp-specialised kernel
    const int wgrid = (h->P.K + WS_B - 1) / WS_B;
    const size_t smem = ws_smem_bytes(false);
    if (noise)
      rollout_kernel_ws_fest<true><<<wgrid, ws_threads(false, true), smem, h->stream>>>(
          h->P, in, h->d_iter, plan, S, noise, h->d_prop, h->d_ctl, part);
    else
      rollout_kernel_ws_fest<false><<<wgrid, ws_threads(false, true), smem, h->stream>>>(
          h->P, in, h->d_iter, plan, S, nullptr, h->d_prop, h->d_ctl, nullptr);
    return cudaGetLastError();
  }
  // the optional cost terms run in the rolled kernel only
  switch (h->feat) {
    case FEAT_FEST: return launch_rolled<FEAT_FEST>(h, grid, in, plan, S, noise, part);
    case FEAT_COLL: return launch_rolled<FEAT_COLL>(h, grid, in, plan, S, noise, part);
    case FEAT_FEST | FEAT_COLL:
      return launch_rolled<FEAT_FEST | FEAT_COLL>(h, grid, in, plan, S, noise, part);
    default: break;
  }
  if (h->variant == 2) return launch_rolled<0>(h, grid, in, plan, S, noise, part);
  if (h->variant == 3) {
    const int wgrid = (h->P.K + WS_B - 1) / WS_B;
    const size_t smem = ws_smem_bytes();
    if (kwait >= 0) {
      PdlLaunch L(dim3(wgrid), dim3(WS_THREADS), smem, h->stream);
      const unsigned long long* iter = h->d_iter;
      const float* prop = h->d_prop;
      const int* ctl = h->d_ctl;
      float* pt = noise ? part : nullptr;
      if (h->P.K <= WS_SMALL_K_MAX)
        return noise ? cudaLaunchKernelEx(&L.lc, rollout_kernel_ws_small<true>, h->P, in, iter,
                                          plan, S, noise, prop, ctl, pt, kwait)
                     : cudaLaunchKernelEx(&L.lc, rollout_kernel_ws_small<false>, h->P, in, iter,
                                          plan, S, noise, prop, ctl, pt, kwait);
      const ObsK* no_obs = nullptr;
      return noise ? cudaLaunchKernelEx(&L.lc, rollout_kernel_ws<true, false>, h->P, in, iter,
                                        plan, S, noise, prop, ctl, no_obs, pt, kwait)
                   : cudaLaunchKernelEx(&L.lc, rollout_kernel_ws<false, false>, h->P, in, iter,
                                        plan, S, noise, prop, ctl, no_obs, pt, kwait);
    }
    if (h->P.K <= WS_SMALL_K_MAX) {
      if (noise)
        rollout_kernel_ws_small<true><<<wgrid, WS_THREADS, smem, h->stream>>>(
            h->P, in, h->d_iter, plan, S, noise, h->d_prop, h->d_ctl, part);
      else
        rollout_kernel_ws_small<false><<<wgrid, WS_THREADS, smem, h->stream>>>(
            h->P, in, h->d_iter, plan, S, nullptr, h->d_prop, h->d_ctl, nullptr);
      return cudaGetLastError();
    }
    if (noise)
      rollout_kernel_ws<true, false><<<wgrid, WS_THREADS, smem, h->stream>>>(
          h->P, in, h->d_iter, plan, S, noise, h->d_prop, h->d_ctl, nullptr, part);
    else
      rollout_kernel_ws<false, false><<<wgrid, WS_THREADS, smem, h->stream>>>(
          h->P, in, h->d_iter, plan, S, nullptr, h->d_prop, h->d_ctl, nullptr, nullptr);
    return cudaGetLastError();
  }
  if (noise)
    rollout_kernel<true><<<grid, ROLLOUT_BLOCK, 0, h->stream>>>(h->P, in, h->d_iter, plan, S, noise,
                                                               h->d_prop, h->d_ctl, part);
  else
    rollout_kernel<false><<<grid, ROLLOUT_BLOCK, 0, h->stream>>>(h->P, in, h->d_iter, plan, S,
                                                                nullptr, h->d_prop, h->d_ctl);
  return cudaGetLastError();
}

// Eq. 4 from caller-supplied costs and noise (mppi_update_device).
cudaError_t launch_update(mppi_s* h, const float* S, const float* noise, const float* plan,
                          float* ustar, float* plan_next) {
  const int K = h->P.K, T = h->P.T;
  const float lambda = h->P.lambda;
  const dim3 grid(T * NJ), block(UPDATE_THREADS);
  if (h->reduce_fp64)
    update_kernel<double><<<grid, block, 0, h->stream>>>(K, T, lambda, S, noise, plan, ustar,
                                                         plan_next, nullptr, nullptr);
  else
    update_kernel<float><<<grid, block, 0, h->stream>>>(K, T, lambda, S, noise, plan, ustar,
                                                        plan_next, nullptr, nullptr);
  return cudaGetLastError();
}

// Eq. 4 of a step from the rollout blocks' partials in d_part, with the
// shift into plan_next (and into tau_dst / plan_dst when given), the output
// record at `out` and iter += 1; the last block consumes a second proposal.
cudaError_t launch_merge(mppi_s* h, const float* plan, float* ustar, float* plan_next, float* out,
                         unsigned long long* iter, float* tau_dst = nullptr,
                         float* plan_dst = nullptr, const unsigned* seq_in = nullptr) {
  // programmatic dependent launch: the merge blocks may start as the rollout
  // kernel's retire and wait (griddepcontrol.wait) for its results, which
  // hides the launch gap between the two kernels
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(h->P.T * NJ);
  lc.blockDim = dim3(MERGE_THREADS);
  lc.dynamicSmemBytes = 0;
  lc.stream = h->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  const int K = h->P.K, T = h->P.T;
  const int nb = (K + ROLLOUT_BLOCK - 1) / ROLLOUT_BLOCK;
  const int ps = part_stride(T);
  const float lambda = h->P.lambda;
  const float* part = h->d_part;
  if (h->reduce_fp64)
    return cudaLaunchKernelEx(&lc, merge_kernel<double>, K, T, lambda, nb, ps, part, plan, ustar,
                              plan_next, out, iter, static_cast<const float*>(h->d_prop),
                              static_cast<const int*>(h->d_ctl), tau_dst, plan_dst, h->d_done,
                              h->d_ctl, seq_in);
  return cudaLaunchKernelEx(&lc, merge_kernel<float>, K, T, lambda, nb, ps, part, plan, ustar,
                            plan_next, out, iter, static_cast<const float*>(h->d_prop),
                            static_cast<const int*>(h->d_ctl), tau_dst, plan_dst, h->d_done,
                            h->d_ctl, seq_in);
}

// the whole update on device buffers: rollouts from the inputs at `in`
// (each block leaving its Eq. 4 partials), then the merge into the other
// plan (and into tau_dst / plan_dst when given) with the output record at
// `out` (default d_out); the merge's last block consumes a second proposal
// set for this update (k_split := K)
cudaError_t enqueue_update(mppi_s* h, int cur, const float* in = nullptr, float* tau_dst = nullptr,
                           float* plan_dst = nullptr, float* out = nullptr,
                           const unsigned* seq_in = nullptr, int kwait = -1) {
  cudaError_t e = launch_rollout(h, in ? in : h->d_in, h->d_plan[cur], h->d_S, h->d_noise,
                                 h->d_part, kwait);
  if (e != cudaSuccess) return e;
  return launch_merge(h, h->d_plan[cur], h->d_ustar, h->d_plan[cur ^ 1], out ? out : h->d_out,
                      h->d_iter, tau_dst, plan_dst, seq_in);
}

__global__ void set_int_kernel(int* dst, int v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}


// host-buffer step: H2D inputs, update, D2H outputs (captured once per parity)
cudaError_t enqueue_host_step(mppi_s* h, int cur) {
  // the inputs and, after them, the step's sequence word (104 B)
  cudaError_t e = cudaMemcpyAsync(h->d_in, h->h_in, sizeof(float) * (IN_FLOATS + 1),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return e;
  // the merge kernel writes the output record straight into pinned host
  // memory (tau0, status, stats, shifted plan: 568 B at T = 18), so no
  // device-to-host copy follows it, and the sequence word last
  return enqueue_update(h, cur, nullptr, nullptr, nullptr, h->h_out_dev,
                        reinterpret_cast<const unsigned*>(h->d_in + IN_FLOATS));
}

void destroy_graphs(mppi_s* h) {
  for (auto& g : h->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

int check_inputs(mppi_s* h, const float* q, const float* qd, const float* goal, const float* plane) {
  for (int j = 0; j < 7; ++j)
    if (!std::isfinite(q[j]) || !std::isfinite(qd[j]))
      return fail(h, MPPI_ERR_INVALID_ARG, "q and qd must be finite");
  for (int a = 0; a < 7; ++a)
    if (!std::isfinite(goal[a])) return fail(h, MPPI_ERR_INVALID_ARG, "goal must be finite");
  const double qn = double(goal[3]) * goal[3] + double(goal[4]) * goal[4] +
                    double(goal[5]) * goal[5] + double(goal[6]) * goal[6];
  if (!(qn > 1e-12)) return fail(h, MPPI_ERR_INVALID_ARG, "goal quaternion must be nonzero");
  if (h->P.cost.contact) {
    for (int a = 0; a < 4; ++a)
      if (!std::isfinite(plane[a])) return fail(h, MPPI_ERR_INVALID_ARG, "plane must be finite");
    const double nn = double(plane[0]) * plane[0] + double(plane[1]) * plane[1] +
                      double(plane[2]) * plane[2];
    if (std::fabs(nn - 1.0) > 1e-3) return fail(h, MPPI_ERR_INVALID_ARG, "plane normal must be unit");
  }
  return MPPI_OK;
}

int read_status(mppi_s* h) {
  int st;
  std::memcpy(&st, &h->h_out[OUT_STATUS], sizeof st);
  return st == 0 ? MPPI_OK : fail(h, MPPI_ERR_NONFINITE, "no sample had a finite cost; plan kept");
}

}  // namespace

// Message for mppi_last_error(NULL) from the other translation units.
void mppi_set_thread_error(const std::string& msg) { g_create_err = msg; }

// Handle internals for the other translation units of the library.
float* mppi_internal_plan(mppi_t h) { return h->d_plan[h->cur]; }
int mppi_internal_T(mppi_t h) { return h->P.T; }
cudaStream_t mppi_internal_stream(mppi_t h) { return h->stream; }
float* mppi_internal_prop(mppi_t h) { return h->d_prop; }
int mppi_internal_K(mppi_t h) { return h->P.K; }
int* mppi_internal_ctl(mppi_t h) { return h->d_ctl; }
cudaError_t mppi_internal_set_split(mppi_t h, int k_split) {
  set_int_kernel<<<1, 32, 0, h->stream>>>(h->d_ctl, k_split);
  return cudaGetLastError();
}

// Parameter conversion shared with the other translation units of the library.
int mppi_convert_params(const mppi_robot* rb, const mppi_cost* c, const mppi_config* cfg,
                        ProbK* P, std::string* why) {
  return convert(rb, c, cfg, P, why);
}

// ---------------------------------------------------------------------------
// FP32 FMA throughput probe (the roofline's peak for the rollout kernels)

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 8;  // 2048 threads: a full SM
constexpr int PEAK_CHAINS = 8;         // independent FMA chains per thread
constexpr int PEAK_ITERS = 8192;       // a multiple of the unroll below

// Every thread advances PEAK_CHAINS independent chains a <- a m + c; the
// store is taken only if the sum equals `never` (it cannot: the chains stay
// positive), which keeps the arithmetic live without memory traffic.
__global__ void __launch_bounds__(PEAK_THREADS)
fp32_peak_kernel(float* __restrict__ out, int iters, float never) {
  float a[PEAK_CHAINS];
#pragma unroll
  for (int j = 0; j < PEAK_CHAINS; ++j) a[j] = 1.0f + 1e-3f * static_cast<float>(threadIdx.x + j);
  const float m = 0.9999999f, c = 1e-7f;
#pragma unroll 16
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) a[j] = fmaf(a[j], m, c);
  }
  float sum = 0.f;
#pragma unroll
  for (int j = 0; j < PEAK_CHAINS; ++j) sum += a[j];
  if (sum == never) out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

int mppi_measure_fp32_peak(double* tflops) {
  if (!tflops) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null argument");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess)
    return fail(nullptr, MPPI_ERR_CUDA, std::string("fp32 peak: ") + cudaGetErrorString(e));
  const int grid = sms * PEAK_BLOCKS_PER_SM;
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  float ms[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  e = cudaMalloc(&out, sizeof(float) * size_t(grid) * PEAK_THREADS);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  if (e == cudaSuccess) {
    fp32_peak_kernel<<<grid, PEAK_THREADS, 0, st>>>(out, PEAK_ITERS, -1.0f);  // warm-up
    e = cudaGetLastError();
  }
  for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) {
      fp32_peak_kernel<<<grid, PEAK_THREADS, 0, st>>>(out, PEAK_ITERS, -1.0f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[r], ev[0], ev[1]);
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  if (e != cudaSuccess)
    return fail(nullptr, MPPI_ERR_CUDA, std::string("fp32 peak: ") + cudaGetErrorString(e));
  for (int i = 1; i < 5; ++i)  // insertion sort for the median
    for (int j = i; j > 0 && ms[j] < ms[j - 1]; --j) std::swap(ms[j], ms[j - 1]);
  const double flop = 2.0 * PEAK_CHAINS * double(PEAK_ITERS) * double(grid) * PEAK_THREADS;
  *tflops = flop / (double(ms[2]) * 1e-3) / 1e12;
  return MPPI_OK;
}

const char* mppi_version(void) { return MPPI_VERSION_STR; }

const char* mppi_last_error(mppi_t h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int mppi_create(const mppi_robot* robot, const mppi_cost* cost, const mppi_config* cfg,
                void* stream, mppi_t* out) {
  if (!robot || !cost || !cfg || !out) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  mppi_s* h = new (std::nothrow) mppi_s();
  if (!h) return fail(nullptr, MPPI_ERR_OOM, "host allocation failed");
  std::string why;
  if (convert(robot, cost, cfg, &h->P, &why) != 0) {
    delete h;
    return fail(nullptr, MPPI_ERR_INVALID_ARG, why);
  }
  h->reduce_fp64 = cfg->reduce_fp64 ? 1 : 0;
  h->use_graph = cfg->use_graph ? 1 : 0;
  if (cfg->variant < 0 || cfg->variant > 3) {
    delete h;
    return fail(nullptr, MPPI_ERR_INVALID_ARG, "variant must be 0, 1, 2 or 3");
  }
  h->feat = (h->P.cost.fest ? FEAT_FEST : 0) | (h->P.cost.coll ? FEAT_COLL : 0);
  if ((h->feat && cfg->variant == 1) || (h->feat == (FEAT_FEST | FEAT_COLL) && cfg->variant == 3)) {
    delete h;
    return fail(nullptr, MPPI_ERR_INVALID_ARG,
                "the optional costs need the rolled rollout kernel (variant 0 or 2) or, one at a "
                "time, the warp-specialised one (variant 3)");
  }
  if (h->feat != (FEAT_FEST | FEAT_COLL) && cfg->variant == 0) {
    // the occupancy query needs the ws kernel's shared-memory opt-in first
    h->variant = 3;
    if (prepare_rollout(h) != cudaSuccess) cudaGetLastError();
    h->variant = default_variant(cfg->K, h->feat == FEAT_COLL, h->feat == FEAT_FEST);
  } else {
    h->variant = cfg->variant == 0 ? 2 : cfg->variant;
  }
  const int T = cfg->T, K = cfg->K;
  auto bail = [&](cudaError_t e, const char* what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    mppi_destroy(h);
    return fail(nullptr, e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA, msg);
  };
  cudaError_t e;
  if (stream) {
    h->stream = static_cast<cudaStream_t>(stream);
  } else {
    if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(e, "cudaStreamCreate");
    h->own_stream = true;
  }
  const size_t plan_b = sizeof(float) * T * NJ;
  if ((e = cudaMalloc(&h->d_plan[0], plan_b)) != cudaSuccess) return bail(e, "cudaMalloc plan");
  if ((e = cudaMalloc(&h->d_plan[1], plan_b)) != cudaSuccess) return bail(e, "cudaMalloc plan");
  if ((e = cudaMalloc(&h->d_ustar, plan_b)) != cudaSuccess) return bail(e, "cudaMalloc ustar");
  if ((e = cudaMalloc(&h->d_scratch_plan, 2 * plan_b)) != cudaSuccess) return bail(e, "cudaMalloc scratch");
  if ((e = cudaMalloc(&h->d_S, sizeof(float) * K)) != cudaSuccess) return bail(e, "cudaMalloc S");
  if ((e = cudaMalloc(&h->d_noise, sizeof(float) * size_t(T) * NJ * K)) != cudaSuccess)
    return bail(e, "cudaMalloc noise");
  if ((e = cudaMalloc(&h->d_in, sizeof(float) * 32)) != cudaSuccess) return bail(e, "cudaMalloc in");
  if ((e = cudaMalloc(&h->d_misc, sizeof(float) * 32)) != cudaSuccess) return bail(e, "cudaMalloc misc");
  if ((e = cudaMalloc(&h->d_words, sizeof(uint32_t) * 8 * 1024)) != cudaSuccess)
    return bail(e, "cudaMalloc words");
  if ((e = cudaMalloc(&h->d_prop, plan_b)) != cudaSuccess) return bail(e, "cudaMalloc prop");
  if ((e = cudaMalloc(&h->d_ctl, 2 * sizeof(int))) != cudaSuccess) return bail(e, "cudaMalloc ctl");
  if ((e = cudaMalloc(&h->d_obs, sizeof(ObsK))) != cudaSuccess) return bail(e, "cudaMalloc obs");
  if (cost->ext_wrench) {
    if ((e = cudaMalloc(&h->d_fext, sizeof(float) * 8)) != cudaSuccess) return bail(e, "cudaMalloc fext");
    float F[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int a = 0; a < 6; ++a) F[a] = static_cast<float>(cost->f_ext[a]);
    if ((e = cudaMemcpy(h->d_fext, F, sizeof F, cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(e, "fext");
    h->P.fext = h->d_fext;
  }
  {
    const size_t nb = (static_cast<size_t>(K) + ROLLOUT_BLOCK - 1) / ROLLOUT_BLOCK;
    if ((e = cudaMalloc(&h->d_part, sizeof(float) * nb * part_stride(T))) != cudaSuccess)
      return bail(e, "cudaMalloc part");
  }
  if ((e = cudaMalloc(&h->d_done, sizeof(unsigned))) != cudaSuccess) return bail(e, "cudaMalloc done");
  if ((e = cudaMemset(h->d_done, 0, sizeof(unsigned))) != cudaSuccess) return bail(e, "done");
  {
    ObsK ob;
    fill_obs(cost->n_obstacles, &cost->obstacles[0][0], &ob);
    if ((e = cudaMemcpy(h->d_obs, &ob, sizeof ob, cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(e, "obs");
  }
  if ((e = prepare_rollout(h)) != cudaSuccess) return bail(e, "rollout shared memory");
  {
    const int ctl[2] = {K, K};
    if ((e = cudaMemcpy(h->d_ctl, ctl, sizeof ctl, cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(e, "ctl");
    if ((e = cudaMemset(h->d_prop, 0, plan_b)) != cudaSuccess) return bail(e, "memset prop");
  }
  h->out_floats = OUT_PLAN + T * NJ;
  if ((e = cudaMalloc(&h->d_out, sizeof(float) * h->out_floats)) != cudaSuccess)
    return bail(e, "cudaMalloc out");
  if ((e = cudaMalloc(&h->d_iter, sizeof(unsigned long long))) != cudaSuccess)
    return bail(e, "cudaMalloc iter");
  if ((e = cudaMallocHost(&h->h_in, sizeof(float) * 32)) != cudaSuccess) return bail(e, "cudaMallocHost");
  if ((e = cudaHostAlloc(&h->h_out, sizeof(float) * h->out_floats, cudaHostAllocMapped)) !=
      cudaSuccess)
    return bail(e, "cudaHostAlloc");
  if ((e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->h_out_dev), h->h_out, 0)) !=
      cudaSuccess)
    return bail(e, "cudaHostGetDevicePointer");
  std::memset(h->h_in, 0, sizeof(float) * 32);
  std::memset(h->h_out, 0, sizeof(float) * h->out_floats);
  if ((e = cudaMemsetAsync(h->d_plan[0], 0, plan_b, h->stream)) != cudaSuccess) return bail(e, "memset");
  if ((e = cudaMemsetAsync(h->d_plan[1], 0, plan_b, h->stream)) != cudaSuccess) return bail(e, "memset");
  if ((e = cudaMemsetAsync(h->d_ustar, 0, plan_b, h->stream)) != cudaSuccess) return bail(e, "memset");
  if ((e = cudaMemsetAsync(h->d_in, 0, sizeof(float) * 32, h->stream)) != cudaSuccess) return bail(e, "memset");
  if ((e = cudaMemsetAsync(h->d_out, 0, sizeof(float) * h->out_floats, h->stream)) != cudaSuccess)
    return bail(e, "memset");
  if ((e = cudaMemsetAsync(h->d_iter, 0, sizeof(unsigned long long), h->stream)) != cudaSuccess)
    return bail(e, "memset");
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(e, "sync");
  *out = h;
  return MPPI_OK;
}

int mppi_destroy(mppi_t h) {
  if (!h) return MPPI_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  destroy_graphs(h);
  cudaFree(h->d_plan[0]);
  cudaFree(h->d_plan[1]);
  cudaFree(h->d_ustar);
  cudaFree(h->d_scratch_plan);
  cudaFree(h->d_S);
  cudaFree(h->d_noise);
  cudaFree(h->d_in);
  cudaFree(h->d_misc);
  cudaFree(h->d_words);
  cudaFree(h->d_prop);
  cudaFree(h->d_ctl);
  cudaFree(h->d_obs);
  cudaFree(h->d_fext);
  cudaFree(h->d_part);
  cudaFree(h->d_done);
  cudaFree(h->d_out);
  cudaFree(h->d_iter);
  if (h->h_in) cudaFreeHost(h->h_in);
  if (h->h_out) cudaFreeHost(h->h_out);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return MPPI_OK;
}

int mppi_step(mppi_t h, const float q[7], const float qd[7], const float goal[7],
              const float plane[4], float tau0_out[7], float* plan_out) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!q || !qd || !goal || !tau0_out || (h->P.cost.contact && !plane))
    return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  static const float no_plane[4] = {0.f, 0.f, 1.f, -1e9f};
  if (!plane) plane = no_plane;
  int rc = check_inputs(h, q, qd, goal, plane);
  if (rc != MPPI_OK) return rc;
  std::memcpy(h->h_in, q, 7 * sizeof(float));
  std::memcpy(h->h_in + 7, qd, 7 * sizeof(float));
  std::memcpy(h->h_in + 14, goal, 7 * sizeof(float));
  std::memcpy(h->h_in + 21, plane, 4 * sizeof(float));
  const unsigned seq = ++h->host_seq;
  std::memcpy(h->h_in + IN_FLOATS, &seq, sizeof seq);
  const int cur = h->cur;
  if (h->use_graph) {
    if (!h->graph[cur]) {
      cudaGraph_t g;
      CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enqueue_host_step(h, cur);
      cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
      if (e != cudaSuccess) return fail(h, MPPI_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
      if (e2 != cudaSuccess) return fail(h, MPPI_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e2));
      e = cudaGraphInstantiate(&h->graph[cur], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        h->graph[cur] = nullptr;
        return fail(h, MPPI_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      }
    }
    CUDA_TRY(h, cudaGraphLaunch(h->graph[cur], h->stream));
  } else {
    CUDA_TRY(h, enqueue_host_step(h, cur));
  }
  // the record is complete once its sequence word reads this step's: poll
  // it (about 2.5 us sooner than a stream synchronisation); a stream that
  // finished or failed without it ends the poll, and the synchronisation
  // then reports the error
  {
    const volatile unsigned* word = reinterpret_cast<const volatile unsigned*>(h->h_out + OUT_SEQ);
    for (unsigned n = 1; *word != seq; ++n)
      if ((n & 4095u) == 0 && cudaStreamQuery(h->stream) != cudaErrorNotReady) break;
    std::atomic_thread_fence(std::memory_order_acquire);
    if (*word != seq) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  h->cur = cur ^ 1;  // the update wrote the next plan into the other buffer
  h->out_on_host = true;
  rc = read_status(h);
  std::memcpy(tau0_out, h->h_out + OUT_TAU0, 7 * sizeof(float));
  if (plan_out) std::memcpy(plan_out, h->h_out + OUT_PLAN, sizeof(float) * h->P.T * NJ);
  return rc;
}

int mppi_step_device(mppi_t h, const float* d_in, float* d_tau0, float* d_plan) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!d_in) return fail(h, MPPI_ERR_INVALID_ARG, "null d_in");
  // the kernels read the caller's inputs and write tau0 and the shifted plan
  // straight into the caller's buffers: two kernels and one 4-byte copy
  const int cur = h->cur;
  CUDA_TRY(h, enqueue_update(h, cur, d_in, d_tau0, d_plan));
  h->cur = cur ^ 1;
  h->out_on_host = false;
  return MPPI_OK;
}

// mppi_step_device queued directly behind a proposal kernel that installs
// a second proposal with k_split = n_plain (the learned proposal's fused
// call): the rollouts may overlap that kernel.
int mppi_internal_step_after_proposal(mppi_t h, const float* d_in, float* d_tau0, float* d_plan,
                                      int n_plain) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!d_in) return fail(h, MPPI_ERR_INVALID_ARG, "null d_in");
  if (n_plain < 0 || n_plain > h->P.K) return fail(h, MPPI_ERR_INVALID_ARG, "n_plain must be in 0..K");
  const int cur = h->cur;
  CUDA_TRY(h, enqueue_update(h, cur, d_in, d_tau0, d_plan, nullptr, nullptr, n_plain));
  h->cur = cur ^ 1;
  h->out_on_host = false;
  return MPPI_OK;
}

int mppi_sync(mppi_t h) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!h->out_on_host)
    CUDA_TRY(h, cudaMemcpyAsync(h->h_out + OUT_STATUS, h->d_out + OUT_STATUS, 5 * sizeof(float),
                                cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return read_status(h);
}

int mppi_get_costs(mppi_t h, float* S_out) {
  if (!h || !S_out) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, cudaMemcpyAsync(S_out, h->d_S, sizeof(float) * h->P.K, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MPPI_OK;
}

int mppi_get_noise(mppi_t h, float* noise_out) {
  if (!h || !noise_out) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, cudaMemcpyAsync(noise_out, h->d_noise, sizeof(float) * size_t(h->P.T) * NJ * h->P.K,
                              cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MPPI_OK;
}

int mppi_get_updated_plan(mppi_t h, float* u_out) {
  if (!h || !u_out) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, cudaMemcpyAsync(u_out, h->d_ustar, sizeof(float) * h->P.T * NJ, cudaMemcpyDeviceToHost,
                              h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MPPI_OK;
}

int mppi_get_stats(mppi_t h, double stats[4]) {
  if (!h || !stats) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  float tmp[4];
  if (h->out_on_host) {
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    std::memcpy(tmp, h->h_out + OUT_STATS, sizeof tmp);
  } else {
    CUDA_TRY(h, cudaMemcpyAsync(tmp, h->d_out + OUT_STATS, sizeof tmp, cudaMemcpyDeviceToHost,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  for (int i = 0; i < 4; ++i) stats[i] = tmp[i];
  return MPPI_OK;
}

int mppi_set_plan(mppi_t h, const float* u) {
  if (!h || !u) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  for (int i = 0; i < h->P.T * NJ; ++i)
    if (!std::isfinite(u[i])) return fail(h, MPPI_ERR_INVALID_ARG, "plan must be finite");
  CUDA_TRY(h, cudaMemcpyAsync(h->d_plan[h->cur], u, sizeof(float) * h->P.T * NJ,
                              cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MPPI_OK;
}

int mppi_get_plan(mppi_t h, float* u) {
  if (!h || !u) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, cudaMemcpyAsync(u, h->d_plan[h->cur], sizeof(float) * h->P.T * NJ,
                              cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MPPI_OK;
}

int mppi_set_iter(mppi_t h, uint64_t iter) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  unsigned long long v = iter;
  CUDA_TRY(h, cudaMemcpyAsync(h->d_iter, &v, sizeof v, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MPPI_OK;
}

int mppi_get_iter(mppi_t h, uint64_t* iter) {
  if (!h || !iter) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  unsigned long long v = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&v, h->d_iter, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  *iter = v;
  return MPPI_OK;
}

int mppi_rollout_device(mppi_t h, const float* d_in, float* d_S, float* d_noise) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!d_in || !d_S) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, launch_rollout(h, d_in, h->d_plan[h->cur], d_S, d_noise));
  return MPPI_OK;
}

int mppi_update_device(mppi_t h, const float* d_S, const float* d_noise, const float* d_plan,
                       float* d_ustar, float* d_plan_next) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!d_S || !d_noise || !d_plan || !d_ustar || !d_plan_next)
    return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, launch_update(h, d_S, d_noise, d_plan, d_ustar, d_plan_next));
  return MPPI_OK;
}

int mppi_ee_pose(mppi_t h, const float q[7], float pose_out[7]) {
  if (!h || !q || !pose_out) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, cudaMemcpyAsync(h->d_misc, q, 7 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  ee_pose_kernel<<<1, 32, 0, h->stream>>>(h->P, h->d_misc, h->d_misc + 16);
  cudaError_t e = cudaGetLastError();
  float r[12];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r, h->d_misc + 16, sizeof r, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, MPPI_ERR_CUDA, std::string("ee_pose: ") + cudaGetErrorString(e));
  // rotation matrix -> unit quaternion (w >= 0), Shepperd's method
  const double R[3][3] = {{r[3], r[4], r[5]}, {r[6], r[7], r[8]}, {r[9], r[10], r[11]}};
  const double tr = R[0][0] + R[1][1] + R[2][2];
  double w, x, y, z;
  if (tr > 0) {
    const double s = std::sqrt(tr + 1.0) * 2;
    w = 0.25 * s; x = (R[2][1] - R[1][2]) / s; y = (R[0][2] - R[2][0]) / s; z = (R[1][0] - R[0][1]) / s;
  } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
    const double s = std::sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]) * 2;
    w = (R[2][1] - R[1][2]) / s; x = 0.25 * s; y = (R[0][1] + R[1][0]) / s; z = (R[0][2] + R[2][0]) / s;
  } else if (R[1][1] > R[2][2]) {
    const double s = std::sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]) * 2;
    w = (R[0][2] - R[2][0]) / s; x = (R[0][1] + R[1][0]) / s; y = 0.25 * s; z = (R[1][2] + R[2][1]) / s;
  } else {
    const double s = std::sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]) * 2;
    w = (R[1][0] - R[0][1]) / s; x = (R[0][2] + R[2][0]) / s; y = (R[1][2] + R[2][1]) / s; z = 0.25 * s;
  }
  const double n = std::sqrt(w * w + x * x + y * y + z * z);
  const double sg = w < 0 ? -1.0 : 1.0;
  pose_out[0] = r[0]; pose_out[1] = r[1]; pose_out[2] = r[2];
  pose_out[3] = static_cast<float>(sg * w / n);
  pose_out[4] = static_cast<float>(sg * x / n);
  pose_out[5] = static_cast<float>(sg * y / n);
  pose_out[6] = static_cast<float>(sg * z / n);
  return MPPI_OK;
}

int mppi_simulate_device(mppi_t h, int n, const float* d_in, const float* d_tau, int substeps,
                         float* d_out) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!d_in || !d_tau || !d_out) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  if (n < 1 || substeps < 1 || substeps > 1000)
    return fail(h, MPPI_ERR_INVALID_ARG, "n must be >= 1 and substeps in 1..1000");
  simulate_kernel<<<(n + 63) / 64, 64, 0, h->stream>>>(h->P, n, d_in, d_tau, substeps, d_out);
  CUDA_TRY(h, cudaGetLastError());
  return MPPI_OK;
}

int mppi_set_plan_device(mppi_t h, const float* d_u) {
  if (!h || !d_u) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, cudaMemcpyAsync(h->d_plan[h->cur], d_u, sizeof(float) * h->P.T * NJ,
                              cudaMemcpyDeviceToDevice, h->stream));
  return MPPI_OK;
}

int mppi_get_plan_device(mppi_t h, float* d_u) {
  if (!h || !d_u) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, cudaMemcpyAsync(d_u, h->d_plan[h->cur], sizeof(float) * h->P.T * NJ,
                              cudaMemcpyDeviceToDevice, h->stream));
  return MPPI_OK;
}

int mppi_get_updated_plan_device(mppi_t h, float* d_u) {
  if (!h || !d_u) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, cudaMemcpyAsync(d_u, h->d_ustar, sizeof(float) * h->P.T * NJ,
                              cudaMemcpyDeviceToDevice, h->stream));
  return MPPI_OK;
}

// out[e] = ustar[e] - nominal[e]
__global__ void correction_kernel(const float* __restrict__ ustar, const float* __restrict__ nominal,
                                  int n, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = ustar[i] - nominal[i];
}

int mppi_get_correction_device(mppi_t h, float* d_out) {
  if (!h || !d_out) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  // the last update read its nominal plan from the buffer it did not write
  const int n = h->P.T * NJ;
  correction_kernel<<<(n + 127) / 128, 128, 0, h->stream>>>(h->d_ustar, h->d_plan[h->cur ^ 1], n,
                                                            d_out);
  CUDA_TRY(h, cudaGetLastError());
  return MPPI_OK;
}

int mppi_set_proposal_device(mppi_t h, const float* d_prop, int n_plain) {
  if (!h || !d_prop) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  if (n_plain < 0 || n_plain > h->P.K) return fail(h, MPPI_ERR_INVALID_ARG, "n_plain must be in 0..K");
  CUDA_TRY(h, cudaMemcpyAsync(h->d_prop, d_prop, sizeof(float) * h->P.T * NJ,
                              cudaMemcpyDeviceToDevice, h->stream));
  CUDA_TRY(h, mppi_internal_set_split(h, n_plain));
  return MPPI_OK;
}

int mppi_noise_words(mppi_t h, uint64_t iter, uint32_t k0, int count, uint32_t t, uint32_t* out) {
  if (!h || !out) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  if (count < 1 || count > 1024) return fail(h, MPPI_ERR_INVALID_ARG, "count must be in 1..1024");
  noise_words_kernel<<<(count + 127) / 128, 128, 0, h->stream>>>(h->P.key0, h->P.key1, iter, k0,
                                                                 count, t, h->d_words);
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, cudaMemcpyAsync(out, h->d_words, sizeof(uint32_t) * 8 * count, cudaMemcpyDeviceToHost,
                              h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MPPI_OK;
}

int mppi_gravity_torque(mppi_t h, const float q[7], float tau_out[7]) {
  if (!h || !q || !tau_out) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, cudaMemcpyAsync(h->d_misc, q, 7 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  gravity_kernel<<<1, 32, 0, h->stream>>>(h->P, h->d_misc, h->d_misc + 16);
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, cudaMemcpyAsync(tau_out, h->d_misc + 16, 7 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MPPI_OK;
}

int mppi_set_obstacles(mppi_t h, int n, const float* obs) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (n < 0 || n > MPPI_OBS_MAX || (n > 0 && !obs))
    return fail(h, MPPI_ERR_INVALID_ARG, "n must be in 0..8 with obstacles given");
  for (int i = 0; i < 7 * n; ++i)
    if (!std::isfinite(obs[i])) return fail(h, MPPI_ERR_INVALID_ARG, "obstacles must be finite");
  for (int o = 0; o < n; ++o)
    if (obs[7 * o + 6] < 0.f) return fail(h, MPPI_ERR_INVALID_ARG, "obstacle radii must be >= 0");
  ObsK ob;
  fill_obs(n, obs, &ob);
  // pageable source: the call returns once the image has been staged
  CUDA_TRY(h, cudaMemcpyAsync(h->d_obs, &ob, sizeof ob, cudaMemcpyHostToDevice, h->stream));
  return MPPI_OK;
}

int mppi_set_obstacles_device(mppi_t h, int n, const float* d_obs) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (n < 0 || n > MPPI_OBS_MAX || (n > 0 && !d_obs))
    return fail(h, MPPI_ERR_INVALID_ARG, "n must be in 0..8 with obstacles given");
  if (n > 0)
    CUDA_TRY(h, cudaMemcpyAsync(&h->d_obs->o[0][0], d_obs, sizeof(float) * 7 * n,
                                cudaMemcpyDeviceToDevice, h->stream));
  set_int_kernel<<<1, 32, 0, h->stream>>>(&h->d_obs->n, n);
  CUDA_TRY(h, cudaGetLastError());
  return MPPI_OK;
}

int mppi_set_external_wrench(mppi_t h, const float F[6]) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!h->d_fext) return fail(h, MPPI_ERR_INVALID_ARG, "the handle has no external wrench");
  if (!F) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  float img[6];
  for (int a = 0; a < 6; ++a) {
    if (!std::isfinite(F[a])) return fail(h, MPPI_ERR_INVALID_ARG, "F_ext must be finite");
    img[a] = F[a];
  }
  // pageable source: the call returns once the image has been staged
  CUDA_TRY(h, cudaMemcpyAsync(h->d_fext, img, sizeof img, cudaMemcpyHostToDevice, h->stream));
  return MPPI_OK;
}

int mppi_set_external_wrench_device(mppi_t h, const float* d_F) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!h->d_fext) return fail(h, MPPI_ERR_INVALID_ARG, "the handle has no external wrench");
  if (!d_F) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(h, cudaMemcpyAsync(h->d_fext, d_F, sizeof(float) * 6, cudaMemcpyDeviceToDevice,
                              h->stream));
  return MPPI_OK;
}

int mppi_get_variant(mppi_t h, int* variant) {
  if (!h || !variant) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  *variant = h->variant;
  return MPPI_OK;
}

int mppi_force_estimate_device(mppi_t h, const float* d_q, const float* d_v, int n, float* d_F) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!d_q || !d_v || !d_F) return fail(h, MPPI_ERR_INVALID_ARG, "null argument");
  if (n < 1 || n > MPPI_K_MAX) return fail(h, MPPI_ERR_INVALID_ARG, "n must be in 1..2^22");
  const int grid = (n + ROLLOUT_BLOCK - 1) / ROLLOUT_BLOCK;
  force_estimate_kernel<ROLLOUT_BLOCK><<<grid, ROLLOUT_BLOCK, fest_smem_bytes(ROLLOUT_BLOCK),
                                         h->stream>>>(h->P, d_q, d_v, n, d_F);
  CUDA_TRY(h, cudaGetLastError());
  return MPPI_OK;
}

int mppi_time_kernels(mppi_t h, const float* d_in, int iters, float* ms_rollout, float* ms_update) {
  if (!h) return fail(nullptr, MPPI_ERR_INVALID_ARG, "null handle");
  if (!d_in || iters < 1 || !ms_rollout || !ms_update) return fail(h, MPPI_ERR_INVALID_ARG, "bad argument");
  cudaEvent_t ev[3];
  for (auto& x : ev) CUDA_TRY(h, cudaEventCreate(&x));
  float tr = 0.f, tu = 0.f;
  const size_t plan_f = size_t(h->P.T) * NJ;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < iters && e == cudaSuccess; ++i) {
    e = cudaEventRecord(ev[0], h->stream);
    if (e == cudaSuccess)
      e = launch_rollout(h, d_in, h->d_plan[h->cur], h->d_S, h->d_noise, h->d_part);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], h->stream);
    if (e == cudaSuccess)
      e = launch_merge(h, h->d_plan[h->cur], h->d_scratch_plan, h->d_scratch_plan + plan_f,
                       nullptr, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
    float a = 0.f, b = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[1], ev[2]);
    tr += a;
    tu += b;
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess)
    return fail(h, MPPI_ERR_CUDA, std::string("time_kernels: ") + cudaGetErrorString(e));
  *ms_rollout = tr / iters;
  *ms_update = tu / iters;
  return MPPI_OK;
}

}  // extern "C"
