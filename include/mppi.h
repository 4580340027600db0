/*
 * mppi.h - C ABI of the B300 (sm_103a) torque-sampling MPPI library.
 *
 * One update of Model Predictive Path Integral control for a 7-joint
 * torque-controlled serial arm, as set out in "Real-Time Dynamics-Based
 * Torque-Sampling MPPI for Compliant and Force Aware Manipulation":
 *   - K noisy torque sequences v_{k,t} = u_t + dtau_{k,t}, dtau ~ N(0, Sigma)
 *     (Eq. 2, Sec. III-A);
 *   - each rolled out over T steps through the rigid-body dynamics
 *     M qdd + h = tau + tau_ext (Eq. 5), qdd = M^-1 (v + tau_ext - h) (Eq. 6),
 *     and the Euler update qd += qdd dt, q += qd dt (Eq. 7), with M and h
 *     rebuilt at every step (Sec. III-A);
 *   - trajectory cost S_k = phi(x_T) + sum_t l(x_{t+1}, v_t) (Eq. 3) with
 *     l = C_motion + C_force + C_joint (Eq. 9-12, 14);
 *   - weights w_k = exp(-(S_k - S_min)/lambda) and the update
 *     u*_t = u_t + sum_k w_k dtau_{k,t} / sum_k w_k (Eq. 4a-4b);
 *   - u*_0 is applied and the plan shifted by one step to warm-start the next
 *     update (Sec. II, last paragraph).
 *
 * Everything per update runs in CUDA kernels on the GPU: the library owns the
 * device buffers it allocates in mppi_create and frees them in mppi_destroy.
 * All entry points return MPPI_OK (0) or a negative MPPI_ERR_* code; the
 * message of the last failure on a handle is available from mppi_last_error
 * (and from mppi_last_error(NULL) for failures of mppi_create and
 * mppi_step_static).  On any error
 * the nominal plan is left as it was.  A handle may be used by one host thread
 * at a time; distinct handles are independent.
 *
 * Conventions shared by every entry point:
 *   - joint vectors are 7 floats in joint order; plans are row-major [T][7]
 *     (N m);
 *   - goal = (p_des x, y, z [m], unit quaternion w, x, y, z of R_des);
 *   - plane = (n_x, n_y, n_z, d): unit normal n, free space is n . p >= d;
 *     ignored when the cost's contact flag is 0;
 *   - noise: Philox4x32-10 (Salmon et al., SC'11) with key (seed_lo, seed_hi)
 *     and counter (k, 2t + c, iter_lo, iter_hi), c in {0, 1}; each output
 *     word x gives u = ((x >> 8) + 0.5) / 2^24, pairs (u1, u2) give the
 *     Box-Muller normals sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2); call c=0
 *     supplies joints 0-3 and c=1 joints 4-6; dtau_{k,t,j} = sigma_j z_j.
 *     A step is therefore reproducible from (seed, iter, plan, inputs).
 *   - iter starts at 0 and increases by one after every successful update.
 */
#ifndef MPPI_H
#define MPPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MPPI_API __attribute__((visibility("default")))
#else
#define MPPI_API
#endif

#define MPPI_NJ 7 /* joints of the arm; the library supports exactly 7 */

/* status codes */
#define MPPI_OK 0
#define MPPI_ERR_INVALID_ARG (-1) /* a pointer, size or parameter is invalid   */
#define MPPI_ERR_OOM (-2)         /* a device or pinned-host allocation failed */
#define MPPI_ERR_CUDA (-3)        /* a CUDA runtime call failed                */
#define MPPI_ERR_TIMEOUT (-4)     /* a bounded device wait ran out             */
#define MPPI_ERR_NONFINITE (-5)   /* no sample had a finite cost; plan kept    */

/* Arm description (Fig. 1: joint transforms, CoM offsets, masses, inertias
 * held by every rollout).  Frames follow the usual URDF chain: link i's frame
 * is its parent's frame translated by joint_xyz[i], rotated by
 * Rz(yaw) Ry(pitch) Rx(roll) of joint_rpy[i], then rotated by q_i about the
 * unit vector axis[i].  The caller owns the record; mppi_create copies it. */
typedef struct mppi_robot {
  int n;                      /* must be MPPI_NJ                               */
  double joint_xyz[7][3];     /* joint i origin in the parent link frame [m]   */
  double joint_rpy[7][3];     /* fixed rotation parent -> joint frame [rad]    */
  double axis[7][3];          /* unit joint axis in the joint frame            */
  double com[7][3];           /* CoM of link i in link i's frame [m]           */
  double mass[7];             /* [kg], > 0                                     */
  double inertia[7][6];       /* I^G about the CoM, link frame: xx yy zz xy xz yz */
  double armature[7];         /* diag(a) of Eq. 8 [kg m^2], >= 0               */
  double damping[7];          /* viscous joint damping [N m s/rad], >= 0       */
  double ee_xyz[3];           /* end-effector point in link 7's frame [m]      */
  double q_min[7], q_max[7];  /* joint position limits [rad]                   */
  double qd_max[7];           /* joint speed limits [rad/s]                    */
  double tau_max[7];          /* torque limits [N m]                           */
  double gravity[3];          /* world gravity [m/s^2]                         */
} mppi_robot;

/* Running cost l(x_{t+1}, v_t) = C_motion + C_force + C_joint [+ C_collision]
 * (Eq. 9-12, 14-15):
 *   C_motion = sum_a w_pos[a] (p_des - p_ee)_a^2 + sum_a w_ori[a] r_a^2,
 *              r = log(R_des^T R_ee) as a rotation vector (Eq. 11);
 *   C_force  = w_force (f_des - f)^2 + w_reg f^2 on the contact normal force
 *              f (Eq. 12), only when contact != 0;
 *   C_joint  = w_qlim sum_j [max(0, q_j - q_max_j)^2 + max(0, q_min_j - q_j)^2]
 *            + w_qdlim sum_j max(0, |qd_j| - qd_max_j)^2
 *            + w_posture sum_j (q_j - q_posture_j)^2
 *            + w_tau sum_j max(0, |v_j| - tau_max_j)^2;
 *   phi(x_T) = w_terminal C_motion(x_T).
 * Contact (contact != 0): penetration delta = d - n . p_ee; when delta > 0,
 * f = max(0, k_contact delta - d_contact n . v_ee), else 0; the wrench
 * (f n, 0) enters the dynamics as tau_ext = J^T F_ext (Eq. 5).
 * Wrench estimate (force_estimate != 0; Eq. 12-13): C_force becomes
 *   sum_a w_force6[a] (f_des6[a] - F_a)^2 + w_reg6[a] F_a^2,
 *   F = Jbar^T (v_t - g(q_t)),  Jbar = M^-1 J^T (J M^-1 J^T)^-1,
 * the end-effector wrench (force xyz; moment about the end-effector point
 * xyz, world frame) that the input v_t, net of the gravity torque g, exerts
 * at the configuration q_t where it acts (M with armature, J the geometric
 * Jacobian of the end-effector point); charged at step t in place of the
 * contact normal-force term.  A sample that meets a kinematic singularity
 * (J M^-1 J^T not positive definite) gets a non-finite cost and weight 0.
 * Collision (collision != 0; Eq. 15): link i is the capsule around the
 * segment from joint i's origin to joint i+1's (link 7 ends at the
 * end-effector point) with radius link_radius[i]; obstacles are capsules
 * (segment a-b, radius; a = b gives a sphere).  The pairs are links i, j
 * with j >= i + 2 (15 pairs) and every link with every obstacle.  For each
 * pair the clearance d is the segment distance (Lumelsky's method) minus
 * both radii, and the pair adds w_collision * [d < d_th] (collision = 1, the
 * indicator of Eq. 15) or w_collision * max(0, d_th - d)^2 (collision = 2, a
 * smooth reading), with d_th = d_th_self or d_th_obs; charged on x_{t+1}.
 * The obstacles are read by every update from a device buffer of the handle,
 * set at creation from n_obstacles / obstacles and replaced by
 * mppi_set_obstacles[_device] between updates (also under CUDA graphs).
 * Either optional cost alone runs on more warps of the warp-specialised
 * kernel (the collision cost on two, the wrench estimate on one) while its
 * blocks for K samples fit on the device at once, else in the rolled kernel
 * (variant 0 chooses; 2 and 3 force one; 1 is rejected).  Both together run
 * in the rolled kernel (variant 0 or 2; 1 and 3 are rejected).
 * mppi_step_static and the server take neither cost.
 * Constant external wrench (ext_wrench != 0; Eq. 5-6 as the paper states
 * them): tau_ext = J(q_0)^T F_ext, with F_ext (force xyz [N]; moment about
 * the end-effector point xyz [N m], world frame) the external wrench and J
 * the end-effector Jacobian at the update's initial state q_0, is "constant
 * over the prediction horizon": the same tau_ext enters M qdd + h = v +
 * tau_ext at every step of every rollout, beside the plane contact's torque
 * when contact is on.  F_ext starts at f_ext below and is replaced between
 * updates by mppi_set_external_wrench[_device] (also under CUDA graphs).
 * mppi_step_static and the server do not take it. */
typedef struct mppi_cost {
  double w_pos[3], w_ori[3];
  double w_force, f_des, w_reg;
  double w_qlim, w_qdlim, w_tau, w_posture;
  double q_posture[7];
  double w_terminal;
  int contact;
  double k_contact, d_contact;
  int force_estimate;          /* 1: C_force on the wrench estimate below      */
  double w_force6[6], f_des6[6], w_reg6[6];  /* its weights, (force; moment) */
  int collision;               /* C_collision: 0 off, 1 indicator, 2 hinge     */
  double w_collision;          /* its weight                                   */
  double d_th_self, d_th_obs;  /* clearance thresholds [m]: link-link, -object */
  double link_radius[7];       /* link capsule radii [m], >= 0                 */
  int n_obstacles;             /* initial obstacles, 0..MPPI_OBS_MAX           */
  double obstacles[8][7];      /* capsules: a xyz, b xyz, radius [m]           */
  int ext_wrench;              /* 1: constant tau_ext = J(q_0)^T F_ext         */
  double f_ext[6];             /* initial F_ext: force xyz; moment xyz         */
} mppi_cost;

#define MPPI_OBS_MAX 8

/* Problem sizes and sampler parameters (Eq. 2-4). */
typedef struct mppi_config {
  double dt;        /* integration step [s], > 0                            */
  int T;            /* horizon steps, 1..MPPI_T_MAX                          */
  int K;            /* samples, 1..MPPI_K_MAX                                */
  double lambda;    /* temperature, > 0                                      */
  double sigma[7];  /* noise standard deviation per joint [N m], >= 0        */
  uint64_t seed;    /* Philox key                                            */
  int reduce_fp64;  /* 0: FP32 weight reduction; 1: FP64 sums over K (the
                     * weights themselves are FP32 in both modes)              */
  int use_graph;    /* 1: mppi_step replays a captured CUDA graph            */
  int variant;      /* rollout kernel: 0 default, 1 links unrolled in registers,
                       2 link loops rolled through shared memory, 3 three
                       warps per 32 samples (kinematic chain / link forces and
                       costs / link forces and noise; one more warp for the
                       wrench estimate, two more for the collision cost)    */
} mppi_config;

#define MPPI_T_MAX 256
#define MPPI_K_MAX (1 << 22)

typedef struct mppi_s* mppi_t;

/* Create a controller.  Validates every parameter (MPPI_ERR_INVALID_ARG),
 * allocates the device buffers (noise [T*7][K], costs [K], plans, staging;
 * MPPI_ERR_OOM on failure) on the current CUDA device.  `stream` is a
 * cudaStream_t on which all work of this handle is queued; NULL makes the
 * library create its own non-blocking stream.  The initial plan is zero and
 * iter is 0.  On success *out receives the handle. */
MPPI_API int mppi_create(const mppi_robot* robot, const mppi_cost* cost, const mppi_config* cfg,
                void* stream, mppi_t* out);

/* Release every resource of the handle (NULL is accepted). */
MPPI_API int mppi_destroy(mppi_t h);

/* One MPPI update from host memory: copies (q, qd, goal, plane) to the
 * device, runs the rollouts and the update, and returns tau0 = u*_0 (7
 * floats) and, when plan_out is not NULL, the shifted plan [T][7] that the
 * next update samples around.  The merge kernel writes its output record
 * straight into the handle's pinned host buffer (no separate device-to-host
 * copy), a sequence word last.  Blocks until the result is in host memory:
 * the calling thread polls that word (it does not sleep), and a stream that
 * ends or fails without it is synchronised and its error returned; the
 * stream may still be retiring the update's last instructions when the call
 * returns (later calls on the handle are ordered after it).
 * Returns MPPI_ERR_NONFINITE (plan unchanged, iter unchanged) when no sample
 * has a finite cost. */
MPPI_API int mppi_step(mppi_t h, const float q[7], const float qd[7], const float goal[7],
              const float plane[4], float tau0_out[7], float* plan_out);

/* One MPPI update from device memory, queued on the handle's stream without
 * waiting.  d_in: 25 device floats (q[7], qd[7], goal[7], plane[4]), read by
 * the rollouts in place (keep it unchanged until the update has run).
 * d_tau0 (7 floats) and d_plan ([T][7]) receive u*_0 and the shifted plan
 * when not NULL.  The status of the last update is read by mppi_sync. */
MPPI_API int mppi_step_device(mppi_t h, const float* d_in, float* d_tau0, float* d_plan);

/* Wait for the handle's queued work; returns the status of the last update
 * (MPPI_OK or MPPI_ERR_NONFINITE) or MPPI_ERR_CUDA. */
MPPI_API int mppi_sync(mppi_t h);

/* Per-sample costs S_k of the last update (K floats, host memory). */
MPPI_API int mppi_get_costs(mppi_t h, float* S_out);

/* Noise dtau of the last update as stored by the rollouts: host array of
 * T*7*K floats laid out [t*7 + j][k]. */
MPPI_API int mppi_get_noise(mppi_t h, float* noise_out);

/* u* of the last update before the shift ([T][7], host memory). */
MPPI_API int mppi_get_updated_plan(mppi_t h, float* u_out);

/* Statistics of the last update: S_min, sum of weights Z, effective sample
 * size 1/sum(wbar^2), number of non-finite costs. */
MPPI_API int mppi_get_stats(mppi_t h, double stats[4]);

/* Nominal plan the next update samples around ([T][7], host memory). */
MPPI_API int mppi_set_plan(mppi_t h, const float* u);
MPPI_API int mppi_get_plan(mppi_t h, float* u);

/* Update counter used in the Philox counter (for checkpoint / resume). */
MPPI_API int mppi_set_iter(mppi_t h, uint64_t iter);
MPPI_API int mppi_get_iter(mppi_t h, uint64_t* iter);

/* Rollouts only (Eq. 1-3, 5-7) for the plan held by the handle and the
 * inputs at d_in (as in mppi_step_device): writes S [K] to d_S and, when not
 * NULL, the noise [T*7][K] to d_noise.  Does not change the plan or iter. */
MPPI_API int mppi_rollout_device(mppi_t h, const float* d_in, float* d_S, float* d_noise);

/* Update only (Eq. 4a-4b and the shift) from caller-supplied device arrays:
 * costs d_S [K], noise d_noise [T*7][K], nominal plan d_plan [T][7]; writes
 * u* to d_ustar and the shifted plan to d_plan_next ([T][7] each).  Uses the
 * handle's K, T, lambda and reduction precision; does not touch its plan. */
MPPI_API int mppi_update_device(mppi_t h, const float* d_S, const float* d_noise, const float* d_plan,
                       float* d_ustar, float* d_plan_next);

/* The handle's model used as a plant: n independent states advanced by one
 * control period dt under a torque held constant (zero-order hold, as the
 * paper's robot side does between updates, Sec. IV-A), in `substeps` Euler
 * steps of Eq. 5-7 with the handle's contact model.  d_in: [n][25] device
 * records (q, qd, goal, plane); d_tau: [n][7]; d_out: [n][14] (q, qd after
 * dt).  Queued on the handle's stream.  substeps in 1..1000. */
MPPI_API int mppi_simulate_device(mppi_t h, int n, const float* d_in, const float* d_tau,
                                  int substeps, float* d_out);

/* Device-to-device plan access on the handle's stream (no host wait):
 * current nominal plan in/out and u* of the last update ([T][7] each). */
MPPI_API int mppi_set_plan_device(mppi_t h, const float* d_u);
MPPI_API int mppi_get_plan_device(mppi_t h, float* d_u);
MPPI_API int mppi_get_updated_plan_device(mppi_t h, float* d_u);

/* Second proposal for the NEXT update only (learned proposal with plain MPPI
 * as its fallback): samples k < n_plain are drawn around the nominal plan
 * (the warm start) and samples k >= n_plain around d_prop ([T][7], device,
 * copied).  The update is then the importance-weighted mean of the sampled
 * controls, u*_t = sum_k wbar_k (u^(k)_t + dtau_{k,t}) with the weights of
 * Eq. 4a, so whichever proposal produces the cheaper rollouts dominates.
 * n_plain in 0..K; after the update every sample is around the nominal plan
 * again.  Queued on the handle's stream. */
MPPI_API int mppi_set_proposal_device(mppi_t h, const float* d_prop, int n_plain);

/* Gravity-compensation torque g(q) = h(q, 0) of Eq. 5 (host arrays),
 * computed on the device by the rollouts' own RNEA. */
MPPI_API int mppi_gravity_torque(mppi_t h, const float q[7], float tau_out[7]);

/* Replaces the obstacle capsules that the following updates read (Eq. 15):
 * n in 0..MPPI_OBS_MAX rows of (a xyz, b xyz, radius), finite, radius >= 0.
 * Host array; copied in the handle's stream order (the caller may reuse the
 * array when the call returns). */
MPPI_API int mppi_set_obstacles(mppi_t h, int n, const float* obs);
/* The same from a device array d_obs [n][7] (not validated: non-finite
 * obstacles make every cost non-finite and the update keeps its plan);
 * queued on the handle's stream. */
MPPI_API int mppi_set_obstacles_device(mppi_t h, int n, const float* d_obs);

/* Replaces the external wrench F_ext of a handle created with ext_wrench
 * (force xyz; moment about the end-effector point xyz, world frame; see
 * mppi_cost): F, a host array of 6 finite floats, is copied in the handle's
 * stream order and the next update projects it at its own initial state.
 * MPPI_ERR_INVALID_ARG when the handle has no external wrench or F is not
 * finite. */
MPPI_API int mppi_set_external_wrench(mppi_t h, const float F[6]);
/* The same from a device array d_F of 6 floats (not validated: a
 * non-finite wrench makes every cost non-finite and the update keeps its
 * plan); queued on the handle's stream. */
MPPI_API int mppi_set_external_wrench_device(mppi_t h, const float* d_F);

/* End-effector wrench estimates of Eq. 13, F = Jbar^T (v - g(q)), for n
 * pairs (q_i, v_i) of device arrays d_q, d_v [n][7] into d_F [n][6]
 * (force xyz; moment about the end-effector point xyz, world frame), by the
 * rollouts' own kinematics, dynamics and estimate (see mppi_cost).  Rows at
 * a kinematic singularity (J M^-1 J^T not positive definite) are NaN.
 * n in 1..MPPI_K_MAX; queued on the handle's stream without waiting; the
 * arrays are caller-owned and must stay valid until the stream reaches it. */
MPPI_API int mppi_force_estimate_device(mppi_t h, const float* d_q, const float* d_v, int n,
                                        float* d_F);

/* The correction the last update made to its nominal plan, u* - u [T][7]
 * (Eq. 4b's weighted noise sum, plus the second proposal's share when one
 * was set), into the caller's device array d_out; queued on the handle's
 * stream.  Before any update it is u* - u of the initial buffers (zero).
 * For building training pairs of a learned proposal; the paper has no
 * counterpart. */
MPPI_API int mppi_get_correction_device(mppi_t h, float* d_out);

/* The rollout kernel the handle runs (1, 2 or 3 as in mppi_config.variant;
 * variant 0 resolves at creation: the warp-specialised kernel while its
 * blocks for K samples fit on the device at once, else the register kernel,
 * or the rolled kernel when an optional cost is on; with both optional costs
 * the rolled kernel; see mppi_cost). */
MPPI_API int mppi_get_variant(mppi_t h, int* variant);

/* End-effector pose (p xyz, quaternion wxyz) at joint angles q, computed on
 * the device by the rollouts' own kinematics (host arrays). */
MPPI_API int mppi_ee_pose(mppi_t h, const float q[7], float pose_out[7]);

/* FP32 FMA throughput of the current device in TFLOP/s (2 FLOP per FFMA),
 * measured by a kernel of independent FMA chains over every SM, timed with
 * CUDA events on a stream of its own (median of five launches after one
 * warm-up, about a millisecond each).  Measurement support for the roofline
 * of the rollout kernels, whose bound is FP32 arithmetic; the paper has no
 * counterpart.  Allocates and frees a small device buffer; returns
 * MPPI_ERR_CUDA on a CUDA failure (message in mppi_last_error(NULL)). */
MPPI_API int mppi_measure_fp32_peak(double* tflops);

/* Device time of the two kernels of one update, averaged over `iters`
 * updates from the inputs at d_in (CUDA events on the handle's stream).  The
 * plan and iter are restored afterwards. */
MPPI_API int mppi_time_kernels(mppi_t h, const float* d_in, int iters, float* ms_rollout,
                      float* ms_update);

/* The raw Philox4x32-10 words behind the noise (Eq. 2) of update `iter`,
 * step t, samples k0 .. k0+count-1, computed by the rollouts' own device
 * generator with the handle's seed: out (host) receives count x 8 words,
 * [k][call*4 + word].  count must be in 1..1024.  For bit-exact checks of
 * the integer stream. */
MPPI_API int mppi_noise_words(mppi_t h, uint64_t iter, uint32_t k0, int count, uint32_t t,
                              uint32_t* out);

/* Allocation-free update.  The paper has no counterpart: this entry point is
 * for callers that cannot allocate device memory while they run, such as a
 * hard-real-time control thread (cudaMalloc may block on the device and has
 * no latency bound) or a plug-in whose host application owns all device
 * memory through its own pool.  It runs one update (the rollouts, the
 * weighted update of the plan and the shift, as mppi_step_device does),
 * without a handle and without any allocation:
 *   robot, cost, cfg: as for mppi_create (host records, copied per call);
 *     cfg->K must be <= MPPI_STATIC_K_MAX, else MPPI_ERR_INVALID_ARG;
 *     cfg->reduce_fp64 selects FP32 or FP64 sums over K as for a handle;
 *     the rollouts always run the register kernel, so cfg->variant must be
 *     0 or 1 (else MPPI_ERR_INVALID_ARG); neither optional cost term;
 *   iter: the update counter used in the Philox counter;
 *   d_in: 25 device floats (q, qd, goal, plane); d_plan: nominal plan [T][7];
 *   d_ustar, d_plan_next: device outputs [T][7] (u* and the shifted plan;
 *     when no sample has a finite cost both receive d_plan unchanged);
 *   stream: cudaStream_t to queue on (NULL: the legacy default stream).
 * The work is queued and the call returns without waiting.  The per-sample
 * costs live in one file-scope device array of MPPI_STATIC_K_MAX floats
 * (about 256 KB), which every GPU that loads the library holds until the
 * process exits; the noise is regenerated instead of stored.  Every call
 * shares that array and overwrites it, so calls whose work overlaps on the
 * GPU (different streams, or different host threads, on the same device)
 * race and must be serialised by the caller.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The
 * address is kept for the process, so the entry point must not be used
 * across a cudaDeviceReset of that device.  Errors
 * are reported by the return code, with the message in
 * mppi_last_error(NULL). */
#define MPPI_STATIC_K_MAX 65536
MPPI_API int mppi_step_static(const mppi_robot* robot, const mppi_cost* cost,
                              const mppi_config* cfg, uint64_t iter, const float* d_in,
                              const float* d_plan, float* d_ustar, float* d_plan_next,
                              void* stream);

/* Message of the last failure on h, or of the last mppi_create or
 * mppi_step_static failure of the calling thread when h is NULL.  Never NULL. */
MPPI_API const char* mppi_last_error(mppi_t h);

/* Library version string. */
MPPI_API const char* mppi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MPPI_H */
