// Allocation-free MPPI update: the entry point mppi_step_static of mppi.h.
//
// Some callers cannot allocate device memory when they run an update: a
// hard-real-time control thread may not call cudaMalloc, which can block on
// the device and has no latency bound, and a plug-in inside a host
// application whose device memory is owned by that application's own pool
// has no allocator of its own to call.  This entry point serves them: the
// caller passes the inputs and the output buffers, and the only other device
// memory used is the file-scope array below, which exists once per device
// for as long as the library is loaded.
//
// Differences from the handle-based path: the per-sample costs live in the
// static array instead of a cudaMalloc'd buffer, and the noise is not stored
// at all; the update kernel regenerates every dtau from the same Philox
// counter (bit-identical values), so the scratch is K floats, not 7*T*K.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "mppi.h"
#include "mppi_kernels.cuh"

using namespace mppi_dev;

int mppi_convert_params(const mppi_robot* rb, const mppi_cost* c, const mppi_config* cfg,
                        ProbK* P, std::string* why);
void mppi_set_thread_error(const std::string& msg);

namespace {

constexpr int kMaxDevices = 64;

// Scratch of mppi_step_static: the update counter read by the rollouts and
// the per-sample costs S[K].  Every call overwrites both before reading them.
struct StaticScratch {
  unsigned long long iter;
  unsigned long long pad[31];  // keeps S on a 256-byte boundary
  float S[MPPI_STATIC_K_MAX];
};
static __device__ __align__(256) StaticScratch g_static_scratch;

// Device address of g_static_scratch, looked up once per device.  In host
// code the symbol itself names a host-side stand-in, not device memory.
StaticScratch* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int fail(int code, const std::string& msg) {
  mppi_set_thread_error(msg);
  return code;
}

// The dtau_{k,t,j} the rollouts drew: same counter, same operations as
// normals8, so the value is bit-identical to the stored noise.
__device__ __forceinline__ float regen_noise(uint32_t key0, uint32_t key1, uint64_t iter,
                                             uint32_t k, uint32_t t, int j, float sigma) {
  const uint32_t call = static_cast<uint32_t>(j) >> 2;
  const int w = j & 3;
  uint32_t c[4] = {k, 2u * t + call, static_cast<uint32_t>(iter),
                   static_cast<uint32_t>(iter >> 32)};
  philox4x32_10(c, key0, key1);
  float z0, z1;
  if (w < 2) box_muller(c[0], c[1], z0, z1);
  else box_muller(c[2], c[3], z0, z1);
  return sigma * ((w & 1) ? z1 : z0);
}

__global__ void static_set_iter_kernel(StaticScratch* sc, unsigned long long iter) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc->iter = iter;
}

// The weighted update of the plan and the shift for plan entry e =
// blockIdx.x, with the noise regenerated instead of read back: the weights
// exp(-(S_k - S_min) / lambda) in FP32, their sums in Acc (float, or double
// when cfg->reduce_fp64 asks for it, as for a handle).
template <typename Acc>
__global__ void __launch_bounds__(UPDATE_BLOCK)
update_regen_kernel(const __grid_constant__ ProbK P, const StaticScratch* __restrict__ sc,
                    const float* __restrict__ plan, float* __restrict__ ustar,
                    float* __restrict__ plan_next) {
  __shared__ float sm_f[32];
  __shared__ Acc sm_a[3 * 32];
  const int K = P.K, T = P.T;
  const int e = blockIdx.x;
  const int t = e / NJ, j = e % NJ;
  const uint64_t iter = sc->iter;
  const float* S = sc->S;
  float m = INFINITY;
  for (int k = threadIdx.x; k < K; k += UPDATE_BLOCK) {
    const float s = S[k];
    if (isfinite(s)) m = fminf(m, s);
  }
  m = block_min<UPDATE_BLOCK>(m, sm_f);
  const bool ok = isfinite(m);
  Acc z = Acc(0), z2 = Acc(0), nacc = Acc(0);
  if (ok) {
    const float inv_l = 1.0f / P.lambda;
    for (int k = threadIdx.x; k < K; k += UPDATE_BLOCK) {
      const float s = S[k];
      const Acc w = static_cast<Acc>(isfinite(s) ? expf((m - s) * inv_l) : 0.f);
      z += w;
      z2 += w * w;
      nacc += w * static_cast<Acc>(regen_noise(P.key0, P.key1, iter, static_cast<uint32_t>(k),
                                               static_cast<uint32_t>(t), j, P.sigma[j]));
    }
  }
  block_sum3<UPDATE_BLOCK>(z, z2, nacc, sm_a);
  if (threadIdx.x != 0) return;
  const float u = plan[e];
  if (ok) {
    const float us = static_cast<float>(static_cast<Acc>(u) + nacc / z);
    ustar[e] = us;
    if (t >= 1) plan_next[e - NJ] = us;
    if (t == T - 1) plan_next[e] = us;
  } else {
    ustar[e] = u;
    plan_next[e] = u;
  }
}

// Looks up (once per device) the device address of the static scratch.  The
// address belongs to the device's primary context as it was at the lookup;
// a cudaDeviceReset ends that context, so the entry point is not for use
// across a device reset.
int scratch_for_current_device(StaticScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MPPI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(MPPI_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(MPPI_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<StaticScratch*>(p);
  }
  *out = g_scratch_addr[dev];
  return MPPI_OK;
}

}  // namespace

extern "C" {

int mppi_step_static(const mppi_robot* robot, const mppi_cost* cost, const mppi_config* cfg,
                     uint64_t iter, const float* d_in, const float* d_plan, float* d_ustar,
                     float* d_plan_next, void* stream) {
  if (!robot || !cost || !cfg || !d_in || !d_plan || !d_ustar || !d_plan_next)
    return fail(MPPI_ERR_INVALID_ARG, "null argument");
  if (cfg->K > MPPI_STATIC_K_MAX)
    return fail(MPPI_ERR_INVALID_ARG, "K exceeds MPPI_STATIC_K_MAX (65536) for mppi_step_static");
  if (cfg->variant != 0 && cfg->variant != 1)
    return fail(MPPI_ERR_INVALID_ARG,
                "mppi_step_static runs the register rollout kernel: variant must be 0 or 1");
  ProbK P;
  std::string why;
  if (mppi_convert_params(robot, cost, cfg, &P, &why) != 0) return fail(MPPI_ERR_INVALID_ARG, why);
  if (P.cost.fest || P.cost.coll || cost->ext_wrench)
    return fail(MPPI_ERR_INVALID_ARG,
                "mppi_step_static takes neither the wrench-estimate nor the collision cost nor "
                "the constant external wrench");
  StaticScratch* sc = nullptr;
  int rc = scratch_for_current_device(&sc);
  if (rc != MPPI_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  static_set_iter_kernel<<<1, 32, 0, st>>>(sc, static_cast<unsigned long long>(iter));
  const int grid = (P.K + ROLLOUT_BLOCK - 1) / ROLLOUT_BLOCK;
  rollout_kernel<false><<<grid, ROLLOUT_BLOCK, 0, st>>>(P, d_in, &sc->iter, d_plan, sc->S, nullptr);
  if (cfg->reduce_fp64)
    update_regen_kernel<double><<<P.T * NJ, UPDATE_BLOCK, 0, st>>>(P, sc, d_plan, d_ustar, d_plan_next);
  else
    update_regen_kernel<float><<<P.T * NJ, UPDATE_BLOCK, 0, st>>>(P, sc, d_plan, d_ustar, d_plan_next);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MPPI_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return MPPI_OK;
}

}  // extern "C"
