// Batched serving of many independent MPPI problems: include/mppi_serve.h.
//
// Device side: two persistent kernels per tick.  serve_rollout_kernel pulls
// tiles (problem, first sample) from an atomic counter and runs the same
// per-sample rollout as the single-problem kernels, with the tile's problem
// parameters, plan and inputs staged in shared memory; serve_update_kernel
// pulls plan entries (problem, t*7 + j) and runs the same block-wide Eq. 4
// reduction as update_kernel.  Neither kernel waits on another block.
//
// Host side: a pool allocator for request scratch, a FIFO of requests, and a
// scheduler that batches admissible requests into ticks on up to four lanes
// (stream + descriptor + captured graph each) so ticks overlap on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <random>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "mppi.h"
#include "mppi_kernels.cuh"
#include "mppi_serve.h"

using namespace mppi_dev;

int mppi_convert_params(const mppi_robot* rb, const mppi_cost* c, const mppi_config* cfg,
                        ProbK* P, std::string* why);
void mppi_set_thread_error(const std::string& msg);

namespace {

// ---------------------------------------------------------------------------
// tick descriptor (host and device share the layout)

constexpr int MAX_BATCH = 1024;
constexpr int MAX_PROBLEMS = 4096;
constexpr int MAX_LANES = 4;
constexpr int RES_FLOATS = 8;  // tau0[7], status

struct TickItem {
  int prob, K, T, tile_begin;
  int upd_begin, pad0, pad1, pad2;
  unsigned long long iter;
  const float* plan;
  float* plan_next;
  float* ustar;
  float* S;
  float* noise;
  float in[IN_FLOATS];
  float pad3[7];
};

struct TickHeader {
  int n_items, n_tiles, n_upd, pad;
};

constexpr size_t kItemsOffset = 16;
constexpr size_t desc_bytes(int n) { return kItemsOffset + sizeof(TickItem) * static_cast<size_t>(n); }

__device__ __forceinline__ const TickItem* desc_items(const char* d) {
  return reinterpret_cast<const TickItem*>(d + kItemsOffset);
}

constexpr int PROBK_FLOATS = static_cast<int>((sizeof(ProbK) + 15) / 16 * 4);

// Variant 3 (warp-specialised): 32 samples per tile on 96 threads, the
// problem's parameters plus the warp-specialised kernel's records; the plan
// is read from global memory.
__host__ __device__ constexpr size_t serve_smem_bytes(int variant, int B) {
  return variant == 3
             ? sizeof(float) * static_cast<size_t>(PROBK_FLOATS) + ws_smem_bytes()
             : sizeof(float) * (static_cast<size_t>(PROBK_FLOATS) + T_MAX * NJ + 32 +
                                (variant == 2 ? static_cast<size_t>(ROLLED_FLOATS_PER_THREAD) * B
                                              : 0));
}
__host__ __device__ constexpr int serve_threads(int variant, int B) {
  return variant == 3 ? WS_THREADS : B;
}

// Largest i with key(items[i]) <= x (items sorted by key, items[0] key 0).
template <typename F>
__device__ __forceinline__ int find_item(const TickItem* items, int n, int x, F key) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (key(items[mid]) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int VARIANT, int B>
__global__ void __launch_bounds__(B)
serve_rollout_kernel(const char* __restrict__ desc, const ProbK* __restrict__ probs,
                     int* __restrict__ counters) {
  extern __shared__ __align__(16) float dsm[];
  ProbK* sP = reinterpret_cast<ProbK*>(dsm);
  float* s_plan = dsm + PROBK_FLOATS;
  float* s_in = s_plan + T_MAX * NJ;
  float* s_work = s_in + 32;
  __shared__ int s_tile, s_item;
  const TickHeader* H = reinterpret_cast<const TickHeader*>(desc);
  const TickItem* items = desc_items(desc);
  const int n_tiles = H->n_tiles, n_items = H->n_items;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      const int tile = atomicAdd(&counters[0], 1);
      s_tile = tile;
      if (tile < n_tiles)
        s_item = find_item(items, n_items, tile, [](const TickItem& I) { return I.tile_begin; });
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= n_tiles) break;
    const int it = s_item;
    const TickItem& I = items[it];
    if (it != cur) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&probs[I.prob]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(sP);
      for (int w = threadIdx.x; w < static_cast<int>(sizeof(ProbK) / 4); w += B) dst[w] = src[w];
      for (int i = threadIdx.x; i < I.T * NJ; i += B) s_plan[i] = I.plan[i];
      if (threadIdx.x < IN_FLOATS) s_in[threadIdx.x] = I.in[threadIdx.x];
      cur = it;
      __syncthreads();
    }
    const int k = (tile - I.tile_begin) * B + threadIdx.x;
    if (k < I.K) {
      float s;
      if (VARIANT == 2)
        s = rollout_sample_rolled<true, B>(*sP, s_in, s_plan, I.iter, k, I.noise, s_work,
                                           threadIdx.x);
      else
        s = rollout_sample<true>(*sP, s_in, s_plan, I.iter, k, I.noise);
      I.S[k] = s;
    }
    __syncthreads();
  }
}

// Warp-specialised tiles: the three roles of rollout_kernel_ws on the
// tile's 32 samples, the problem's parameters in shared memory; every warp
// meets every barrier of a tile, and the block synchronises between tiles.
__global__ void __launch_bounds__(WS_THREADS)
serve_rollout_kernel_ws(const char* __restrict__ desc, const ProbK* __restrict__ probs,
                        int* __restrict__ counters) {
  extern __shared__ float4 dsm4[];
  float* dsm = reinterpret_cast<float*>(dsm4);
  ProbK* sP = reinterpret_cast<ProbK*>(dsm);
  float* s_in = dsm + PROBK_FLOATS;
  const WsSmem m = ws_carve(s_in + 32);
  __shared__ int s_tile, s_item;
  const TickHeader* H = reinterpret_cast<const TickHeader*>(desc);
  const TickItem* items = desc_items(desc);
  const int n_tiles = H->n_tiles, n_items = H->n_items;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      const int tile = atomicAdd(&counters[0], 1);
      s_tile = tile;
      if (tile < n_tiles)
        s_item = find_item(items, n_items, tile, [](const TickItem& I) { return I.tile_begin; });
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= n_tiles) break;
    const int it = s_item;
    const TickItem& I = items[it];
    if (it != cur) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&probs[I.prob]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(sP);
      for (int w = threadIdx.x; w < static_cast<int>(sizeof(ProbK) / 4); w += WS_THREADS)
        dst[w] = src[w];
      if (threadIdx.x < IN_FLOATS) s_in[threadIdx.x] = I.in[threadIdx.x];
      cur = it;
      __syncthreads();
    }
    const int k_raw = (tile - I.tile_begin) * WS_B + lane;
    const bool live = k_raw < I.K;
    const int k = live ? k_raw : I.K - 1;
    if (warp == 0) {
      ws_dynamics<false, false>(*sP, s_in, m, lane);
    } else if (warp == 1) {
      const float Sk = ws_costs<false, false>(*sP, s_in, m, lane);
      if (live) I.S[k] = Sk;
    } else {
      ws_noise<true, false, false>(*sP, s_in, I.plan, I.iter, k, live, I.noise, m, lane);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(UPDATE_THREADS)
serve_update_kernel(const char* __restrict__ desc, const ProbK* __restrict__ probs,
                    int* __restrict__ counters, float* __restrict__ res) {
  __shared__ int s_u, s_item;
  const TickHeader* H = reinterpret_cast<const TickHeader*>(desc);
  const TickItem* items = desc_items(desc);
  const int n_upd = H->n_upd, n_items = H->n_items;
  for (;;) {
    if (threadIdx.x == 0) {
      const int u = atomicAdd(&counters[1], 1);
      s_u = u;
      if (u < n_upd)
        s_item = find_item(items, n_items, u, [](const TickItem& I) { return I.upd_begin; });
    }
    __syncthreads();
    const int u = s_u;
    if (u >= n_upd) break;
    const int it = s_item;
    const TickItem& I = items[it];
    const int e = u - I.upd_begin;
    const EntryResult<float> r =
        update_entry<float, UPDATE_BATCH_SHARED>(I.K, probs[I.prob].lambda, I.S,
                                                 I.noise + static_cast<size_t>(e) * I.K,
                                                 I.plan[e], false);
    if (threadIdx.x == 0) {
      const int t = e / NJ;
      if (r.ok) {
        if (t >= 1) I.plan_next[e - NJ] = r.us;
        if (t == I.T - 1) I.plan_next[e] = r.us;
      } else {
        I.plan_next[e] = r.us;
      }
      I.ustar[e] = r.us;
      if (e < NJ) res[it * RES_FLOATS + e] = r.us;
      if (e == 0) reinterpret_cast<int*>(res)[it * RES_FLOATS + 7] = r.ok ? 0 : 1;
    }
  }
}

using RolloutFn = void (*)(const char*, const ProbK*, int*);

RolloutFn rollout_fn(int variant, int B) {
  if (variant == 3) return serve_rollout_kernel_ws;
  if (variant == 2) {
    if (B == 32) return serve_rollout_kernel<2, 32>;
    if (B == 64) return serve_rollout_kernel<2, 64>;
    return serve_rollout_kernel<2, 128>;
  }
  if (B == 32) return serve_rollout_kernel<1, 32>;
  if (B == 64) return serve_rollout_kernel<1, 64>;
  return serve_rollout_kernel<1, 128>;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t scratch_bytes(int K, int T) {
  const size_t s = (sizeof(float) * K + 255) / 256 * 256;
  const size_t n = (sizeof(float) * static_cast<size_t>(NJ) * T * K + 255) / 256 * 256;
  return s + n;
}

}  // namespace

// ---------------------------------------------------------------------------
// pool

struct mppi_pool_s {
  size_t size = 0, used = 0, peak = 0;
  std::map<size_t, size_t> free_;  // offset -> bytes
  std::unordered_map<size_t, size_t> live_;
};

static constexpr size_t kGran = 256;

static int pool_alloc(mppi_pool_s* p, size_t bytes, size_t* off) {
  bytes = (std::max<size_t>(bytes, 1) + kGran - 1) / kGran * kGran;
  for (auto it = p->free_.begin(); it != p->free_.end(); ++it) {
    if (it->second < bytes) continue;
    const size_t o = it->first, rest = it->second - bytes;
    p->free_.erase(it);
    if (rest) p->free_[o + bytes] = rest;
    p->live_[o] = bytes;
    p->used += bytes;
    p->peak = std::max(p->peak, p->used);
    *off = o;
    return MPPI_OK;
  }
  return MPPI_ERR_OOM;
}

static int pool_free(mppi_pool_s* p, size_t off) {
  auto it = p->live_.find(off);
  if (it == p->live_.end()) return MPPI_ERR_INVALID_ARG;
  const size_t sz = it->second;
  p->used -= sz;
  p->live_.erase(it);
  size_t start = off, len = sz;
  auto nx = p->free_.find(off + sz);  // free neighbour after
  if (nx != p->free_.end()) {
    len += nx->second;
    p->free_.erase(nx);
  }
  auto ge = p->free_.lower_bound(off);  // free neighbour before
  if (ge != p->free_.begin()) {
    auto pv = std::prev(ge);
    if (pv->first + pv->second == off) {
      start = pv->first;
      len += pv->second;
      p->free_.erase(pv);
    }
  }
  p->free_[start] = len;
  return MPPI_OK;
}

static size_t pool_largest(const mppi_pool_s* p) {
  size_t m = 0;
  for (const auto& kv : p->free_) m = std::max(m, kv.second);
  return m;
}

// ---------------------------------------------------------------------------
// server

namespace {

struct Problem {
  ProbK P;
  int K = 0, T = 0;
  float* d_plan[2] = {nullptr, nullptr};
  float* d_ustar = nullptr;
  int cur = 0;
  uint64_t iter = 0;
  bool inflight = false;
  int queued = 0;
  float in[IN_FLOATS];
  bool has_in = false;
};

struct Req {
  uint64_t ticket;
  int id;
  float in[IN_FLOATS];
  double t_submit;
};

struct Fin {
  int status;
  float tau0[NJ];
  double t_submit, t_done;
};

struct Adm {
  uint64_t ticket;
  int id;
  size_t off;
  double t_submit;
};

struct Lane {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t graph = nullptr;     // tick with the tuned rollout kernel
  cudaGraphExec_t graph_ws = nullptr;  // tick with the warp-specialised kernel
  char* h_desc = nullptr;
  char* d_desc = nullptr;
  float* h_res = nullptr;
  float* d_res = nullptr;
  int* d_cnt = nullptr;
  bool busy = false;
  std::vector<Adm> adm;
};

}  // namespace

struct mppi_server_s {
  mppi_server_config cfg{};
  int sm_count = 0;
  char* d_pool = nullptr;
  mppi_pool_s pool;
  ProbK* d_probs = nullptr;
  std::vector<Problem> probs;
  Lane lanes[MAX_LANES];
  int n_lanes = 1;
  int variant = 1, block = 32;
  int rollout_grid = 0, update_grid = 0;
  int ws_grid = 0;  // resident warp-specialised blocks: the tiles of one wave
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req> pending;
  std::unordered_map<uint64_t, Fin> fin;
  std::unordered_set<uint64_t> outstanding;
  uint64_t next_ticket = 1;
  std::thread thr;
  std::atomic<bool> running{false};
  std::atomic<bool> stop_flag{false};
  int sticky_err = MPPI_OK;
  // statistics
  double completed = 0, ticks = 0, items_total = 0, rsteps = 0;
  size_t max_queue = 0;
};

namespace {

int sfail(mppi_server_s* s, int code, const std::string& msg) {
  mppi_set_thread_error(msg);
  (void)s;
  return code;
}

#define SCUDA(s, call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return sfail((s), e_ == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA,     \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

int configure_kernels(mppi_server_s* s) {
  for (int v = 1; v <= 2; ++v)
    for (int B : {32, 64, 128}) {
      RolloutFn f = rollout_fn(v, B);
      SCUDA(s, cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(serve_smem_bytes(v, B))));
    }
  SCUDA(s, cudaFuncSetAttribute(rollout_fn(3, WS_B), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(serve_smem_bytes(3, WS_B))));
  return MPPI_OK;
}

// Shapes the autotuner tries: (variant, samples per tile).
constexpr int kShapes[][2] = {{1, 32}, {1, 64}, {1, 128}, {2, 32}, {2, 64}, {2, 128}, {3, WS_B}};

int set_launch_shape(mppi_server_s* s, int variant, int B) {
  if (variant == 3) B = WS_B;
  int nb = 0;
  SCUDA(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rollout_fn(variant, B),
                                                          serve_threads(variant, B),
                                                          serve_smem_bytes(variant, B)));
  if (nb < 1) return sfail(s, MPPI_ERR_CUDA, "rollout kernel does not fit on an SM");
  int nu = 0;
  SCUDA(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nu, serve_update_kernel, UPDATE_THREADS, 0));
  s->variant = variant;
  s->block = B;
  s->rollout_grid = nb * s->sm_count;
  s->update_grid = std::max(1, nu) * s->sm_count;
  for (int l = 0; l < s->n_lanes; ++l)
    if (s->lanes[l].graph) {
      cudaGraphExecDestroy(s->lanes[l].graph);
      s->lanes[l].graph = nullptr;
    }
  return MPPI_OK;
}

cudaError_t enqueue_kernels(mppi_server_s* s, Lane& L, bool ws) {
  cudaError_t e = cudaMemsetAsync(L.d_cnt, 0, 2 * sizeof(int), L.st);
  if (e != cudaSuccess) return e;
  if (ws)
    serve_rollout_kernel_ws<<<s->ws_grid, WS_THREADS, serve_smem_bytes(3, WS_B), L.st>>>(
        L.d_desc, s->d_probs, L.d_cnt);
  else
    rollout_fn(s->variant, s->block)<<<s->rollout_grid, serve_threads(s->variant, s->block),
                                        serve_smem_bytes(s->variant, s->block), L.st>>>(
        L.d_desc, s->d_probs, L.d_cnt);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  serve_update_kernel<<<s->update_grid, UPDATE_THREADS, 0, L.st>>>(L.d_desc, s->d_probs, L.d_cnt,
                                                                    L.d_res);
  return cudaGetLastError();
}

int ensure_graph(mppi_server_s* s, Lane& L, bool ws) {
  cudaGraphExec_t& G = ws ? L.graph_ws : L.graph;
  if (G) return MPPI_OK;
  cudaGraph_t g;
  SCUDA(s, cudaStreamBeginCapture(L.st, cudaStreamCaptureModeThreadLocal));
  const cudaError_t e = enqueue_kernels(s, L, ws);
  const cudaError_t e2 = cudaStreamEndCapture(L.st, &g);
  if (e != cudaSuccess) return sfail(s, MPPI_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  if (e2 != cudaSuccess) return sfail(s, MPPI_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e2));
  const cudaError_t e3 = cudaGraphInstantiate(&G, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) {
    G = nullptr;
    return sfail(s, MPPI_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e3));
  }
  return MPPI_OK;
}

// Fills the lane's host descriptor from admitted (problem, inputs) pairs and
// the scratch offsets; returns the number of rollout tiles.
void fill_desc(mppi_server_s* s, Lane& L, const std::vector<const float*>& inputs,
               int tile_samples) {
  TickHeader* H = reinterpret_cast<TickHeader*>(L.h_desc);
  TickItem* items = reinterpret_cast<TickItem*>(L.h_desc + kItemsOffset);
  int tiles = 0, upd = 0;
  for (size_t i = 0; i < L.adm.size(); ++i) {
    const Adm& a = L.adm[i];
    Problem& p = s->probs[a.id];
    TickItem& I = items[i];
    std::memset(&I, 0, sizeof I);
    I.prob = a.id;
    I.K = p.K;
    I.T = p.T;
    I.tile_begin = tiles;
    I.upd_begin = upd;
    I.iter = p.iter;
    I.plan = p.d_plan[p.cur];
    I.plan_next = p.d_plan[p.cur ^ 1];
    I.ustar = p.d_ustar;
    I.S = reinterpret_cast<float*>(s->d_pool + a.off);
    I.noise = reinterpret_cast<float*>(s->d_pool + a.off + (sizeof(float) * p.K + 255) / 256 * 256);
    std::memcpy(I.in, inputs[i], sizeof(I.in));
    tiles += (p.K + tile_samples - 1) / tile_samples;
    upd += p.T * NJ;
  }
  H->n_items = static_cast<int>(L.adm.size());
  H->n_tiles = tiles;
  H->n_upd = upd;
  H->pad = 0;
}

// Retires a finished lane (lock held).
void retire(mppi_server_s* s, Lane& L) {
  const double t = now_s();
  for (size_t i = 0; i < L.adm.size(); ++i) {
    const Adm& a = L.adm[i];
    Problem& p = s->probs[a.id];
    Fin f;
    int st;
    std::memcpy(&st, &L.h_res[i * RES_FLOATS + 7], sizeof st);
    f.status = st == 0 ? MPPI_OK : MPPI_ERR_NONFINITE;
    std::memcpy(f.tau0, &L.h_res[i * RES_FLOATS], sizeof f.tau0);
    f.t_submit = a.t_submit;
    f.t_done = t;
    s->fin[a.ticket] = f;
    p.cur ^= 1;  // a non-finite update wrote the unchanged plan to the other buffer
    if (st == 0) p.iter += 1;
    p.inflight = false;
    p.queued -= 1;
    pool_free(&s->pool, a.off);
    s->completed += 1;
    s->rsteps += static_cast<double>(p.K) * p.T;
  }
  L.adm.clear();
  L.busy = false;
}

// One scheduling round (lock held): retire finished lanes, then launch at
// most one tick.  *launched = requests in the new tick.
int round_locked(mppi_server_s* s, int* launched, bool* progress) {
  *launched = 0;
  for (int l = 0; l < s->n_lanes; ++l) {
    Lane& L = s->lanes[l];
    if (!L.busy) continue;
    const cudaError_t q = cudaEventQuery(L.ev);
    if (q == cudaSuccess) {
      retire(s, L);
      *progress = true;
    } else if (q != cudaErrorNotReady) {
      s->sticky_err = MPPI_ERR_CUDA;
      return sfail(s, MPPI_ERR_CUDA, std::string("tick failed: ") + cudaGetErrorString(q));
    }
  }
  if (s->pending.empty()) return MPPI_OK;
  Lane* L = nullptr;
  for (int l = 0; l < s->n_lanes; ++l)
    if (!s->lanes[l].busy) {
      L = &s->lanes[l];
      break;
    }
  if (!L) return MPPI_OK;
  // admission: arrival order; one request per problem per tick; a problem
  // with a tick in flight waits; the first request whose scratch does not
  // fit in the pool stops admission (no overtaking by smaller requests)
  std::vector<const float*> inputs;
  std::vector<size_t> taken;
  std::unordered_set<int> chosen;
  for (size_t i = 0; i < s->pending.size() && static_cast<int>(L->adm.size()) < s->cfg.max_batch; ++i) {
    const Req& r = s->pending[i];
    Problem& p = s->probs[r.id];
    if (p.inflight || chosen.count(r.id)) continue;
    size_t off = 0;
    if (pool_alloc(&s->pool, scratch_bytes(p.K, p.T), &off) != MPPI_OK) break;
    L->adm.push_back(Adm{r.ticket, r.id, off, r.t_submit});
    inputs.push_back(r.in);
    chosen.insert(r.id);
    taken.push_back(i);
  }
  if (L->adm.empty()) return MPPI_OK;
  // a tick whose 32-sample tiles all fit in one wave of the warp-specialised
  // kernel is latency-bound and runs on it; bigger ticks are throughput-bound
  // and run on the tuned kernel (variant 0 only)
  long long ws_tiles = 0;
  for (const Adm& a : L->adm) ws_tiles += (s->probs[a.id].K + WS_B - 1) / WS_B;
  const bool ws = s->cfg.variant == 0 ? ws_tiles <= s->ws_grid : s->variant == 3;
  int rc = ensure_graph(s, *L, ws);
  if (rc != MPPI_OK) {
    for (const Adm& a : L->adm) pool_free(&s->pool, a.off);
    L->adm.clear();
    return rc;
  }
  fill_desc(s, *L, inputs, ws ? WS_B : s->block);
  const cudaGraphExec_t G = ws ? L->graph_ws : L->graph;
  for (const Adm& a : L->adm) s->probs[a.id].inflight = true;
  const size_t n = L->adm.size();
  cudaError_t e = cudaMemcpyAsync(L->d_desc, L->h_desc, desc_bytes(static_cast<int>(n)),
                                  cudaMemcpyHostToDevice, L->st);
  if (e == cudaSuccess) e = cudaGraphLaunch(G, L->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L->h_res, L->d_res, sizeof(float) * RES_FLOATS * n, cudaMemcpyDeviceToHost, L->st);
  if (e == cudaSuccess) e = cudaEventRecord(L->ev, L->st);
  if (e != cudaSuccess) {
    s->sticky_err = MPPI_ERR_CUDA;
    return sfail(s, MPPI_ERR_CUDA, std::string("tick launch: ") + cudaGetErrorString(e));
  }
  L->busy = true;
  for (size_t j = taken.size(); j-- > 0;) s->pending.erase(s->pending.begin() + taken[j]);
  s->ticks += 1;
  s->items_total += static_cast<double>(n);
  *launched = static_cast<int>(n);
  *progress = true;
  return MPPI_OK;
}

bool idle_locked(const mppi_server_s* s) {
  if (!s->pending.empty()) return false;
  for (int l = 0; l < s->n_lanes; ++l)
    if (s->lanes[l].busy) return false;
  return true;
}

// After the last tick or request the scheduler keeps polling (yielding its
// core) for this long before it sleeps on the condition variable: a request
// that arrives meanwhile is admitted within microseconds instead of after a
// thread wake-up (tens of microseconds).
constexpr double kSpinSeconds = 2e-3;

void scheduler_main(mppi_server_s* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  double t_active = now_s();
  while (!s->stop_flag.load()) {
    int launched = 0;
    bool progress = false;
    if (round_locked(s, &launched, &progress) != MPPI_OK) {
      s->cv.notify_all();
      break;
    }
    if (progress) {
      s->cv.notify_all();
      t_active = now_s();
      continue;
    }
    bool any_busy = false;
    for (int l = 0; l < s->n_lanes; ++l) any_busy |= s->lanes[l].busy;
    if (any_busy || now_s() - t_active < kSpinSeconds) {
      // a tick is on the GPU, or one may come soon: poll at a fine grain
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    } else {
      s->cv.wait_for(lk, std::chrono::microseconds(200));
    }
  }
  s->running.store(false);
  s->cv.notify_all();
}

const float kDefaultInput[IN_FLOATS] = {0, 0, 0, 0, 0, 0, 0,  0, 0, 0, 0, 0, 0, 0,
                                        0.3f, 0.f, 0.5f, 1.f, 0.f, 0.f, 0.f,
                                        0.f, 0.f, 1.f, -1e9f};

}  // namespace

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

int mppi_pool_create(size_t bytes, mppi_pool_t* out) {
  if (!out || bytes < kGran) return MPPI_ERR_INVALID_ARG;
  mppi_pool_s* p = new (std::nothrow) mppi_pool_s();
  if (!p) return MPPI_ERR_OOM;
  p->size = bytes / kGran * kGran;
  p->free_[0] = p->size;
  *out = p;
  return MPPI_OK;
}

int mppi_pool_destroy(mppi_pool_t pool) {
  delete pool;
  return MPPI_OK;
}

int mppi_pool_alloc(mppi_pool_t pool, size_t bytes, size_t* offset) {
  if (!pool || !offset) return MPPI_ERR_INVALID_ARG;
  return pool_alloc(pool, bytes, offset);
}

int mppi_pool_free(mppi_pool_t pool, size_t offset) {
  if (!pool) return MPPI_ERR_INVALID_ARG;
  return pool_free(pool, offset);
}

int mppi_pool_stats(mppi_pool_t pool, size_t out[4]) {
  if (!pool || !out) return MPPI_ERR_INVALID_ARG;
  out[0] = pool->size;
  out[1] = pool->used;
  out[2] = pool->peak;
  out[3] = pool_largest(pool);
  return MPPI_OK;
}

int mppi_server_create(const mppi_server_config* cfg, mppi_server_t* out) {
  if (!cfg || !out) return sfail(nullptr, MPPI_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (cfg->max_problems < 1 || cfg->max_problems > MAX_PROBLEMS)
    return sfail(nullptr, MPPI_ERR_INVALID_ARG, "max_problems must be in 1..4096");
  if (cfg->max_batch < 1 || cfg->max_batch > MAX_BATCH)
    return sfail(nullptr, MPPI_ERR_INVALID_ARG, "max_batch must be in 1..1024");
  if (cfg->lanes < 1 || cfg->lanes > MAX_LANES)
    return sfail(nullptr, MPPI_ERR_INVALID_ARG, "lanes must be in 1..4");
  if (cfg->variant < 0 || cfg->variant > 3)
    return sfail(nullptr, MPPI_ERR_INVALID_ARG, "variant must be 0, 1, 2 or 3");
  if (cfg->rollout_block != 0 && cfg->rollout_block != 32 && cfg->rollout_block != 64 &&
      cfg->rollout_block != 128)
    return sfail(nullptr, MPPI_ERR_INVALID_ARG, "rollout_block must be 0, 32, 64 or 128");
  if (cfg->pool_bytes < (1u << 20)) return sfail(nullptr, MPPI_ERR_INVALID_ARG, "pool_bytes must be >= 1 MiB");
  mppi_server_s* s = new (std::nothrow) mppi_server_s();
  if (!s) return sfail(nullptr, MPPI_ERR_OOM, "host allocation failed");
  s->cfg = *cfg;
  s->n_lanes = cfg->lanes;
  auto bail = [&](int rc) {
    mppi_server_destroy(s);
    return rc;
  };
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return bail(sfail(nullptr, MPPI_ERR_CUDA, cudaGetErrorString(e)));
  s->pool.size = cfg->pool_bytes / kGran * kGran;
  s->pool.free_[0] = s->pool.size;
  if ((e = cudaMalloc(&s->d_pool, s->pool.size)) != cudaSuccess)
    return bail(sfail(nullptr, MPPI_ERR_OOM, std::string("pool: ") + cudaGetErrorString(e)));
  if ((e = cudaMalloc(&s->d_probs, sizeof(ProbK) * cfg->max_problems)) != cudaSuccess)
    return bail(sfail(nullptr, MPPI_ERR_OOM, cudaGetErrorString(e)));
  for (int l = 0; l < s->n_lanes; ++l) {
    Lane& L = s->lanes[l];
    if ((e = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMallocHost(&L.h_desc, desc_bytes(cfg->max_batch))) != cudaSuccess ||
        (e = cudaMalloc(&L.d_desc, desc_bytes(cfg->max_batch))) != cudaSuccess ||
        (e = cudaMallocHost(&L.h_res, sizeof(float) * RES_FLOATS * cfg->max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&L.d_res, sizeof(float) * RES_FLOATS * cfg->max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&L.d_cnt, 2 * sizeof(int))) != cudaSuccess)
      return bail(sfail(nullptr, e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA,
                        std::string("lane set-up: ") + cudaGetErrorString(e)));
  }
  s->probs.reserve(cfg->max_problems);
  int rc = configure_kernels(s);
  if (rc != MPPI_OK) return bail(rc);
  {
    int nws = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nws, serve_rollout_kernel_ws, WS_THREADS, serve_smem_bytes(3, WS_B));
    if (e != cudaSuccess || nws < 1) return bail(sfail(nullptr, MPPI_ERR_CUDA, "ws occupancy"));
    s->ws_grid = nws * s->sm_count;
  }
  rc = set_launch_shape(s, cfg->variant ? cfg->variant : 1, cfg->rollout_block ? cfg->rollout_block : 32);
  if (rc != MPPI_OK) return bail(rc);
  *out = s;
  return MPPI_OK;
}

int mppi_server_destroy(mppi_server_t s) {
  if (!s) return MPPI_OK;
  mppi_server_stop(s);
  for (int l = 0; l < s->n_lanes; ++l) {
    Lane& L = s->lanes[l];
    if (L.st) cudaStreamSynchronize(L.st);
    if (L.graph) cudaGraphExecDestroy(L.graph);
    if (L.graph_ws) cudaGraphExecDestroy(L.graph_ws);
    if (L.ev) cudaEventDestroy(L.ev);
    if (L.h_desc) cudaFreeHost(L.h_desc);
    if (L.h_res) cudaFreeHost(L.h_res);
    cudaFree(L.d_desc);
    cudaFree(L.d_res);
    cudaFree(L.d_cnt);
    if (L.st) cudaStreamDestroy(L.st);
  }
  for (Problem& p : s->probs) {
    cudaFree(p.d_plan[0]);
    cudaFree(p.d_plan[1]);
    cudaFree(p.d_ustar);
  }
  cudaFree(s->d_probs);
  cudaFree(s->d_pool);
  delete s;
  return MPPI_OK;
}

int mppi_server_add_problem(mppi_server_t s, const mppi_robot* robot, const mppi_cost* cost,
                            const mppi_config* cfg, int* id) {
  if (!s || !robot || !cost || !cfg || !id) return sfail(s, MPPI_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (static_cast<int>(s->probs.size()) >= s->cfg.max_problems)
    return sfail(s, MPPI_ERR_OOM, "problem table full");
  Problem p;
  std::string why;
  if (mppi_convert_params(robot, cost, cfg, &p.P, &why) != 0) return sfail(s, MPPI_ERR_INVALID_ARG, why);
  if (p.P.cost.fest || p.P.cost.coll || cost->ext_wrench)
    return sfail(s, MPPI_ERR_INVALID_ARG,
                 "the server takes neither the wrench-estimate nor the collision cost nor the "
                 "constant external wrench");
  p.K = cfg->K;
  p.T = cfg->T;
  if (scratch_bytes(p.K, p.T) > s->pool.size)
    return sfail(s, MPPI_ERR_OOM, "the problem's scratch exceeds the pool");
  const size_t pb = sizeof(float) * p.T * NJ;
  cudaError_t e;
  if ((e = cudaMalloc(&p.d_plan[0], pb)) != cudaSuccess || (e = cudaMalloc(&p.d_plan[1], pb)) != cudaSuccess ||
      (e = cudaMalloc(&p.d_ustar, pb)) != cudaSuccess) {
    cudaFree(p.d_plan[0]);
    cudaFree(p.d_plan[1]);
    cudaFree(p.d_ustar);
    return sfail(s, MPPI_ERR_OOM, std::string("plans: ") + cudaGetErrorString(e));
  }
  const int nid = static_cast<int>(s->probs.size());
  SCUDA(s, cudaMemset(p.d_plan[0], 0, pb));
  SCUDA(s, cudaMemset(p.d_plan[1], 0, pb));
  SCUDA(s, cudaMemset(p.d_ustar, 0, pb));
  SCUDA(s, cudaMemcpy(&s->d_probs[nid], &p.P, sizeof(ProbK), cudaMemcpyHostToDevice));
  std::memcpy(p.in, kDefaultInput, sizeof p.in);
  s->probs.push_back(p);
  *id = nid;
  return MPPI_OK;
}

static int check_id(mppi_server_s* s, int id) {
  if (id < 0 || id >= static_cast<int>(s->probs.size())) return sfail(s, MPPI_ERR_INVALID_ARG, "unknown problem id");
  return MPPI_OK;
}

int mppi_server_set_plan(mppi_server_t s, int id, const float* u) {
  if (!s || !u) return sfail(s, MPPI_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int rc = check_id(s, id);
  if (rc != MPPI_OK) return rc;
  Problem& p = s->probs[id];
  if (p.queued > 0) return sfail(s, MPPI_ERR_INVALID_ARG, "the problem has queued or running updates");
  SCUDA(s, cudaMemcpy(p.d_plan[p.cur], u, sizeof(float) * p.T * NJ, cudaMemcpyHostToDevice));
  return MPPI_OK;
}

int mppi_server_get_plan(mppi_server_t s, int id, float* u) {
  if (!s || !u) return sfail(s, MPPI_ERR_INVALID_ARG, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  int rc = check_id(s, id);
  if (rc != MPPI_OK) return rc;
  while (s->probs[id].inflight) {
    if (s->running.load()) {
      s->cv.wait_for(lk, std::chrono::milliseconds(1));
    } else {
      int launched;
      bool progress = false;
      rc = round_locked(s, &launched, &progress);
      if (rc != MPPI_OK) return rc;
      if (!progress) {
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
      }
    }
  }
  Problem& p = s->probs[id];
  SCUDA(s, cudaMemcpy(u, p.d_plan[p.cur], sizeof(float) * p.T * NJ, cudaMemcpyDeviceToHost));
  return MPPI_OK;
}

int mppi_server_get_iter(mppi_server_t s, int id, uint64_t* iter) {
  if (!s || !iter) return sfail(s, MPPI_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int rc = check_id(s, id);
  if (rc != MPPI_OK) return rc;
  *iter = s->probs[id].iter;
  return MPPI_OK;
}

int mppi_server_set_input(mppi_server_t s, int id, const float in[25]) {
  if (!s || !in) return sfail(s, MPPI_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int rc = check_id(s, id);
  if (rc != MPPI_OK) return rc;
  std::memcpy(s->probs[id].in, in, sizeof(float) * IN_FLOATS);
  s->probs[id].has_in = true;
  return MPPI_OK;
}

static int submit_locked(mppi_server_s* s, int id, const float* in, double t_submit, uint64_t* ticket) {
  int rc = check_id(s, id);
  if (rc != MPPI_OK) return rc;
  for (int a = 0; a < IN_FLOATS; ++a)
    if (!std::isfinite(in[a])) return sfail(s, MPPI_ERR_INVALID_ARG, "inputs must be finite");
  Req r;
  r.ticket = s->next_ticket++;
  r.id = id;
  std::memcpy(r.in, in, sizeof r.in);
  r.t_submit = t_submit;
  s->pending.push_back(r);
  s->outstanding.insert(r.ticket);
  s->probs[id].queued += 1;
  s->max_queue = std::max(s->max_queue, s->pending.size());
  *ticket = r.ticket;
  return MPPI_OK;
}

int mppi_server_submit(mppi_server_t s, int id, const float in[25], uint64_t* ticket) {
  if (!s || !in || !ticket) return sfail(s, MPPI_ERR_INVALID_ARG, "null argument");
  int rc;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->sticky_err != MPPI_OK) return sfail(s, s->sticky_err, "server stopped after a CUDA error");
    rc = submit_locked(s, id, in, now_s(), ticket);
  }
  s->cv.notify_all();
  return rc;
}

static int take_locked(mppi_server_s* s, uint64_t ticket, float* tau0, int* done) {
  auto it = s->fin.find(ticket);
  if (it == s->fin.end()) {
    if (!s->outstanding.count(ticket)) return sfail(s, MPPI_ERR_INVALID_ARG, "unknown ticket");
    *done = 0;
    return MPPI_OK;
  }
  if (tau0) std::memcpy(tau0, it->second.tau0, sizeof(float) * NJ);
  const int st = it->second.status;
  s->fin.erase(it);
  s->outstanding.erase(ticket);
  *done = 1;
  return st;
}

int mppi_server_poll(mppi_server_t s, uint64_t ticket, float tau0[7], int* done) {
  if (!s || !done) return sfail(s, MPPI_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  return take_locked(s, ticket, tau0, done);
}

int mppi_server_wait(mppi_server_t s, uint64_t ticket, float tau0[7]) {
  if (!s) return sfail(s, MPPI_ERR_INVALID_ARG, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    int done = 0;
    const int rc = take_locked(s, ticket, tau0, &done);
    if (done || rc != MPPI_OK) return rc;
    if (s->sticky_err != MPPI_OK) return sfail(s, s->sticky_err, "server stopped after a CUDA error");
    if (s->running.load()) {
      s->cv.wait_for(lk, std::chrono::milliseconds(1));
    } else {
      int launched;
      bool progress = false;
      const int r2 = round_locked(s, &launched, &progress);
      if (r2 != MPPI_OK) return r2;
      if (!progress) {
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
      }
    }
  }
}

int mppi_server_start(mppi_server_t s) {
  if (!s) return sfail(s, MPPI_ERR_INVALID_ARG, "null server");
  if (s->running.load()) return MPPI_OK;
  if (s->thr.joinable()) s->thr.join();
  {
    // capture every lane's tick graphs now rather than on a first request
    std::lock_guard<std::mutex> lk(s->mu);
    for (int l = 0; l < s->n_lanes; ++l) {
      Lane& L = s->lanes[l];
      if (L.busy) continue;
      int rc = ensure_graph(s, L, false);
      if (rc == MPPI_OK && (s->cfg.variant == 0 || s->variant == 3)) rc = ensure_graph(s, L, true);
      if (rc != MPPI_OK) return rc;
    }
  }
  s->stop_flag.store(false);
  s->running.store(true);
  s->thr = std::thread(scheduler_main, s);
  return MPPI_OK;
}

int mppi_server_stop(mppi_server_t s) {
  if (!s) return sfail(s, MPPI_ERR_INVALID_ARG, "null server");
  s->stop_flag.store(true);
  s->cv.notify_all();
  if (s->thr.joinable()) s->thr.join();
  s->running.store(false);
  return MPPI_OK;
}

int mppi_server_tick(mppi_server_t s, int* launched) {
  if (!s || !launched) return sfail(s, MPPI_ERR_INVALID_ARG, "null argument");
  if (s->running.load()) return sfail(s, MPPI_ERR_INVALID_ARG, "the scheduler thread is running");
  std::lock_guard<std::mutex> lk(s->mu);
  bool progress = false;
  return round_locked(s, launched, &progress);
}

int mppi_server_drain(mppi_server_t s) {
  if (!s) return sfail(s, MPPI_ERR_INVALID_ARG, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  while (!idle_locked(s)) {
    if (s->sticky_err != MPPI_OK) return sfail(s, s->sticky_err, "server stopped after a CUDA error");
    if (s->running.load()) {
      s->cv.wait_for(lk, std::chrono::milliseconds(1));
    } else {
      int launched;
      bool progress = false;
      const int rc = round_locked(s, &launched, &progress);
      if (rc != MPPI_OK) return rc;
      if (!progress) {
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
      }
    }
  }
  return MPPI_OK;
}

int mppi_server_autotune(mppi_server_t s, float* best_ms) {
  if (!s) return sfail(s, MPPI_ERR_INVALID_ARG, "null server");
  if (s->running.load()) return sfail(s, MPPI_ERR_INVALID_ARG, "stop the scheduler thread first");
  std::lock_guard<std::mutex> lk(s->mu);
  if (!idle_locked(s)) return sfail(s, MPPI_ERR_INVALID_ARG, "the server has work queued or running");
  if (s->probs.empty()) return sfail(s, MPPI_ERR_INVALID_ARG, "no problem registered");
  Lane& L = s->lanes[0];
  std::vector<const float*> inputs;
  for (int i = 0; i < static_cast<int>(s->probs.size()) && static_cast<int>(L.adm.size()) < s->cfg.max_batch; ++i) {
    size_t off = 0;
    if (pool_alloc(&s->pool, scratch_bytes(s->probs[i].K, s->probs[i].T), &off) != MPPI_OK) break;
    L.adm.push_back(Adm{0, i, off, 0.0});
    inputs.push_back(s->probs[i].in);
  }
  auto release = [&]() {
    for (const Adm& a : L.adm) pool_free(&s->pool, a.off);
    L.adm.clear();
  };
  const int keep_v = s->variant, keep_b = s->block;
  float best = 1e30f;
  int best_v = keep_v, best_b = keep_b;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = MPPI_OK;
  for (const auto& shape : kShapes) {
    if (rc != MPPI_OK) break;
    const int v = shape[0], B = shape[1];
    if (s->cfg.variant && v != s->cfg.variant) continue;
    {
      if (s->cfg.rollout_block && v != 3 && B != s->cfg.rollout_block) continue;
      rc = set_launch_shape(s, v, B);
      if (rc != MPPI_OK) break;
      fill_desc(s, L, inputs, v == 3 ? WS_B : B);
      const size_t n = L.adm.size();
      cudaError_t e = cudaMemcpyAsync(L.d_desc, L.h_desc, desc_bytes(static_cast<int>(n)),
                                      cudaMemcpyHostToDevice, L.st);
      float ms = 1e30f;
      for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaMemsetAsync(L.d_cnt, 0, 2 * sizeof(int), L.st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, L.st);
        if (e == cudaSuccess) {
          rollout_fn(v, B)<<<s->rollout_grid, serve_threads(v, B), serve_smem_bytes(v, B), L.st>>>(
              L.d_desc, s->d_probs, L.d_cnt);
          e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, L.st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0) ms = std::min(ms, t);  // the first run warms up
      }
      if (e != cudaSuccess) {
        rc = sfail(s, MPPI_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
        break;
      }
      if (ms < best) {
        best = ms;
        best_v = v;
        best_b = B;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
  const int rc2 = set_launch_shape(s, best_v, best_b);
  if (rc != MPPI_OK) return rc;
  if (rc2 != MPPI_OK) return rc2;
  if (best_ms) *best_ms = best;
  return MPPI_OK;
}

int mppi_server_stats(mppi_server_t s, double out[8]) {
  if (!s || !out) return sfail(s, MPPI_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out[0] = s->completed;
  out[1] = s->ticks;
  out[2] = s->ticks > 0 ? s->items_total / s->ticks : 0.0;
  out[3] = static_cast<double>(s->pool.peak);
  out[4] = static_cast<double>(s->pool.size);
  out[5] = s->variant;
  out[6] = s->block;
  out[7] = s->rsteps;
  return MPPI_OK;
}

int mppi_server_load_test(mppi_server_t s, double rate_hz, double seconds, uint64_t seed,
                          double out[8]) {
  if (!s || !out || !(rate_hz > 0) || !(seconds > 0)) return sfail(s, MPPI_ERR_INVALID_ARG, "bad argument");
  if (!s->running.load()) return sfail(s, MPPI_ERR_INVALID_ARG, "start the scheduler thread first");
  int nprob;
  double ticks0, items0, rsteps0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    nprob = static_cast<int>(s->probs.size());
    ticks0 = s->ticks;
    items0 = s->items_total;
    rsteps0 = s->rsteps;
    s->max_queue = 0;
  }
  if (nprob == 0) return sfail(s, MPPI_ERR_INVALID_ARG, "no problem registered");
  std::mt19937_64 rng(seed);
  std::exponential_distribution<double> gap(rate_hz);
  std::uniform_int_distribution<int> pick(0, nprob - 1);
  std::vector<uint64_t> tickets;
  std::vector<double> t_arr;
  const double t0 = now_s();
  double t = t0;
  for (;;) {
    t += gap(rng);
    if (t - t0 > seconds) break;
    while (now_s() < t) {
      if (t - now_s() > 2e-4) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    const int id = pick(rng);
    uint64_t tk = 0;
    int rc;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->sticky_err != MPPI_OK) return sfail(s, s->sticky_err, "server stopped after a CUDA error");
      rc = submit_locked(s, id, s->probs[id].in, t, &tk);
    }
    s->cv.notify_all();
    if (rc != MPPI_OK) return rc;
    tickets.push_back(tk);
    t_arr.push_back(t);
  }
  std::vector<double> lat;
  lat.reserve(tickets.size());
  double t_last = t0;
  for (size_t i = 0; i < tickets.size(); ++i) {
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
      auto it = s->fin.find(tickets[i]);
      if (it != s->fin.end()) {
        lat.push_back(it->second.t_done - it->second.t_submit);
        t_last = std::max(t_last, it->second.t_done);
        s->fin.erase(it);
        s->outstanding.erase(tickets[i]);
        break;
      }
      if (s->sticky_err != MPPI_OK) return sfail(s, s->sticky_err, "server stopped after a CUDA error");
      s->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
  }
  std::vector<double> sorted = lat;
  std::sort(sorted.begin(), sorted.end());
  auto pct = [&](double q) {
    if (sorted.empty()) return 0.0;
    const size_t i = std::min(sorted.size() - 1, static_cast<size_t>(q * (sorted.size() - 1) + 0.5));
    return sorted[i];
  };
  double mean = 0;
  for (double x : lat) mean += x;
  mean = lat.empty() ? 0 : mean / lat.size();
  const double span = std::max(1e-9, t_last - t0);
  std::lock_guard<std::mutex> lk(s->mu);
  out[0] = static_cast<double>(lat.size());
  out[1] = pct(0.50) * 1e3;
  out[2] = pct(0.99) * 1e3;
  out[3] = mean * 1e3;
  out[4] = lat.size() / span;
  out[5] = (s->rsteps - rsteps0) / span;
  out[6] = (s->ticks - ticks0) > 0 ? (s->items_total - items0) / (s->ticks - ticks0) : 0.0;
  out[7] = static_cast<double>(s->max_queue);
  return MPPI_OK;
}

}  // extern "C"
