// Learned proposal network (include/mppi_mlp.h): BF16 training and inference
// kernels on the tcgen05 tensor cores with FP32 accumulation.
//
// Every product of the forward and backward passes is one "TN" GEMM of
// mppi_tc.cuh, C = A B^T with both operands K-major: the forward pass
// multiplies the activations [n][in] by the weights [out][in]; the backward
// pass forms dW = dZ^T H from transposed copies [out][n] and [in][n] that
// the producing epilogues write beside the row-major ones, and dH = dZ W
// from a transposed BF16 copy of the weights [in][out].  BF16 buffers have
// leading dimensions padded to 8 elements (16-byte TMA strides); TMA's zero
// fill covers every ragged edge, and the padding itself is zeroed once.
// The single-row proposal of one MPPI handle runs as one cluster of 8 CTAs
// (propose_kernel): no grid barriers, activations exchanged through
// distributed shared memory.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "mppi.h"
#include "mppi_mlp.h"
#include "mppi_tc.cuh"

void mppi_set_thread_error(const std::string& msg);
float* mppi_internal_plan(mppi_t h);
int mppi_internal_T(mppi_t h);
cudaStream_t mppi_internal_stream(mppi_t h);
float* mppi_internal_prop(mppi_t h);
int mppi_internal_K(mppi_t h);
int* mppi_internal_ctl(mppi_t h);
extern "C" int mppi_internal_step_after_proposal(mppi_t h, const float* d_in, float* d_tau0,
                                                 float* d_plan, int n_plain);

namespace {

using bf16 = __nv_bfloat16;
using mppi_tc::TcArgs;
using mppi_tc::gelu_f;

constexpr int MAX_LAYERS = 8;

__host__ __device__ constexpr long long pad8(long long n) { return (n + 7) / 8 * 8; }

// db[n] = sum_m D[m][n] from the transposed deltas DT [N][ldt] (BF16, FP32 sum)
__global__ void colsum_kernel(const bf16* __restrict__ DT, long long ldt, int M, int N,
                              float* __restrict__ db) {
  const int n = blockIdx.x;
  float s = 0.f;
  for (int m = threadIdx.x; m < M; m += blockDim.x) s += __bfloat162float(DT[n * ldt + m]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += part[w];
    db[n] = t;
  }
}

// xb[i][f] = xbT[f][i] = bf16((x[i][f] - mean[f]) / std[f])
__global__ void normalize_in_kernel(const float* __restrict__ x, int n, int d,
                                    const float* __restrict__ mean, const float* __restrict__ sd,
                                    bf16* __restrict__ xb, long long ldx, bf16* __restrict__ xbT,
                                    long long ldt) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<long long>(n) * d) return;
  const int r = static_cast<int>(i / d), f = static_cast<int>(i % d);
  const bf16 v = __float2bfloat16((x[i] - mean[f]) / sd[f]);
  xb[r * ldx + f] = v;
  xbT[f * ldt + r] = v;
}

// dY = dYT^T = bf16(scale (y - (t - mean)/std)); loss += sum of squares / (n d)
__global__ void loss_grad_kernel(const float* __restrict__ y, const float* __restrict__ t, int n,
                                 int d, const float* __restrict__ mean,
                                 const float* __restrict__ sd, bf16* __restrict__ dy,
                                 long long ldy, bf16* __restrict__ dyT, long long ldt,
                                 float* __restrict__ loss) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  float e2 = 0.f;
  if (i < static_cast<long long>(n) * d) {
    const int r = static_cast<int>(i / d), f = static_cast<int>(i % d);
    const float e = y[i] - (t[i] - mean[f]) / sd[f];
    const bf16 g = __float2bfloat16(2.0f * e / (static_cast<float>(n) * d));
    dy[r * ldy + f] = g;
    dyT[f * ldt + r] = g;
    e2 = e * e;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
  if ((threadIdx.x & 31) == 0 && e2 != 0.f) atomicAdd(loss, e2 / (static_cast<float>(n) * d));
}

// Per-column mean and deviation (unbiased) of X [n][d] in FP64, two passes;
// deviations below floor are raised to it.  One block per column.
__global__ void colstats_kernel(const float* __restrict__ X, int n, int d, float floor,
                                float* __restrict__ mean, float* __restrict__ sd) {
  const int f = blockIdx.x;
  __shared__ double part[8];
  __shared__ double s_mean;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += X[static_cast<long long>(i) * d + f];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += part[w];
    s_mean = t / n;
  }
  __syncthreads();
  const double mu = s_mean;
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double e = X[static_cast<long long>(i) * d + f] - mu;
    v += e * e;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += part[w];
    const double sdv = n > 1 ? sqrt(t / (n - 1)) : 0.0;
    mean[f] = static_cast<float>(mu);
    sd[f] = fmaxf(static_cast<float>(sdv), floor);
  }
}

// y = yn * std + mean (in place allowed)
__global__ void denormalize_kernel(const float* __restrict__ yn, int n, int d,
                                   const float* __restrict__ mean, const float* __restrict__ sd,
                                   float* __restrict__ y) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<long long>(n) * d) return;
  const int f = static_cast<int>(i % d);
  y[i] = yn[i] * sd[f] + mean[f];
}

// Adam on the flat FP32 parameters.
struct AdamArgs {
  float* p;
  const float* g;
  float* m;
  float* v;
  long long n;
  float lr, b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
};
__global__ void adam_kernel(const AdamArgs a) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= a.n) return;
  const float g = a.g[i];
  const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
  const float v = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
  a.m[i] = m;
  a.v[i] = v;
  a.p[i] -= a.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
}

// BF16 copies of one weight matrix W [out][in] (FP32, row-major): wb [out][ldw]
// and its transpose wbT [in][ldwt].
__global__ void to_bf16_kernel(const float* __restrict__ W, int out, int in, bf16* __restrict__ wb,
                               long long ldw, bf16* __restrict__ wbT, long long ldwt) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<long long>(out) * in) return;
  const int o = static_cast<int>(i / in), k = static_cast<int>(i % in);
  const bf16 v = __float2bfloat16(W[i]);
  wb[o * ldw + k] = v;
  wbT[k * ldwt + o] = v;
}

// Single-row inference for one handle (the learned proposal): one cluster
// of PC_CTAS CTAs.  The input record (q, qd, goal) and the nominal plan are
// standardised and rounded to BF16 in every CTA; for each layer, CTA r forms
// output columns 32 r .. 32 r + 31 (warp w: four of them, lane l: inputs
// 8 l .. 8 l + 7, a shuffle sum over the lanes), rounds hidden outputs to
// BF16 after the GELU as the batched path does, and stores them into every
// CTA's activation buffer through distributed shared memory with st.async
// (lane r of the column's warp stores into CTA r), each store counting its
// 4 bytes on the receiving CTA's mbarrier of that
// buffer; a CTA starts layer l + 1 once its barrier has counted all of
// layer l's outputs (no cluster-wide barrier between layers).  A buffer is
// written again two layers later, which no CTA reaches before every CTA has
// read it (each CTA's next outputs follow its reads).  All weight fragments (16 B per lane,
// column and layer) are loaded before the first layer, so the network's
// 400 KB of BF16 weights cost one L2 round trip, spread over 8 SMs.  The
// output is the correction to the nominal plan: dst = plan + net(x).
constexpr int PC_CTAS = 8;
constexpr int PC_THREADS = 256;
constexpr int PC_LMAX = 4;   // layers with weights
constexpr int MAXW = 256;    // layer widths
constexpr int PC_COLS = 4;   // output columns per warp

struct ProposeArgs {
  const float* in;      // 25-float input record
  const float* plan;    // nominal plan [7T]
  const bf16* wb;       // BF16 weights, layer l at wb_off[l] with leading dimension ldw[l]
  const float* p;       // FP32 parameters (biases at boff[l])
  long long wb_off[MAX_LAYERS + 1], ldw[MAX_LAYERS + 1], boff[MAX_LAYERS + 1];
  int dims[MAX_LAYERS + 1];
  int L;
  const float *mean_in, *sd_in, *mean_out, *sd_out;
  float* dst;           // [n_out]
  int* k_split;         // the handle's k_split of its next update
  int n_plain;
  int* err;             // set when a wait for a layer's inputs gave up
};

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One activation store into CTA r's buffer, counted on CTA r's mbarrier.
__device__ __forceinline__ void st_async_remote(const float* local_dst, const uint64_t* local_bar,
                                                uint32_t r, float v) {
  uint32_t dst, bar;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(dst) : "r"(mppi_tc::smem_u32(local_dst)), "r"(r));
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(bar) : "r"(mppi_tc::smem_u32(local_bar)), "r"(r));
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];"
               ::"r"(dst), "r"(__float_as_uint(v)), "r"(bar) : "memory");
}

// Bounded wait for phase `parity` of a local barrier that other CTAs'
// st.async complete (acquire at cluster scope).
__device__ __forceinline__ bool wait_cluster_tx(const uint64_t* bar, uint32_t parity) {
  const uint32_t b = mppi_tc::smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(b), "r"(parity) : "memory");
    if (ok) return true;
    if (clock64() - t0 > mppi_tc::WAIT_CYCLES) return false;
  }
}

__global__ void __cluster_dims__(PC_CTAS, 1, 1) __launch_bounds__(PC_THREADS)
propose_kernel(const ProposeArgs a) {
  __shared__ float act[2][MAXW];
  __shared__ __align__(8) uint64_t bar[2];  // one per activation buffer
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // an update queued behind this kernel as its programmatic dependent may
  // start now: its blocks that need the proposal wait for this grid
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  uint32_t rank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  // every weight fragment of this lane, all layers, before any arithmetic
  uint4 wf[PC_LMAX][PC_COLS];
#pragma unroll
  for (int l = 0; l < PC_LMAX; ++l)
#pragma unroll
    for (int c = 0; c < PC_COLS; ++c) {
      wf[l][c] = make_uint4(0u, 0u, 0u, 0u);
      if (l < a.L) {
        const int col = static_cast<int>(rank) * (PC_COLS * PC_THREADS / 32) + warp * PC_COLS + c;
        if (col < a.dims[l + 1] && 8 * lane < a.dims[l])
          wf[l][c] = __ldg(reinterpret_cast<const uint4*>(a.wb + a.wb_off[l + 1] +
                                                          col * a.ldw[l + 1]) + lane);
      }
    }
  // the biases of this warp's columns and the output layer's constants,
  // also before the first layer (lane 0 uses them)
  float bias[PC_LMAX][PC_COLS], oplan[PC_COLS], omean[PC_COLS], osd[PC_COLS];
#pragma unroll
  for (int c = 0; c < PC_COLS; ++c) {
    const int col = static_cast<int>(rank) * (PC_COLS * PC_THREADS / 32) + warp * PC_COLS + c;
#pragma unroll
    for (int l = 0; l < PC_LMAX; ++l)
      bias[l][c] = (l < a.L && col < a.dims[l + 1]) ? __ldg(a.p + a.boff[l + 1] + col) : 0.f;
    const bool oc = col < a.dims[a.L];
    oplan[c] = oc ? a.plan[col] : 0.f;
    omean[c] = oc ? __ldg(a.mean_out + col) : 0.f;
    osd[c] = oc ? __ldg(a.sd_out + col) : 0.f;
  }
  const int n0 = a.dims[0];
  for (int i = tid; i < MAXW; i += PC_THREADS) {
    float x = 0.f;
    if (i < n0) x = __bfloat162float(__float2bfloat16(
                    ((i < 21 ? a.in[i] : a.plan[i - 21]) - a.mean_in[i]) / a.sd_in[i]));
    act[0][i] = x;
    act[1][i] = 0.f;
  }
  if (rank == 0 && tid == 0) *a.k_split = a.n_plain;  // samples k >= n_plain use the proposal
  if (tid == 0) {
    mppi_tc::mbar_init(mppi_tc::smem_u32(&bar[0]), 1);
    mppi_tc::mbar_init(mppi_tc::smem_u32(&bar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  cluster_sync_all();  // every CTA of the cluster runs and has its barriers set
  bool ok = true;
#pragma unroll
  for (int l = 0; l < PC_LMAX; ++l) {
    if (l >= a.L) break;
    const int out = a.dims[l + 1];
    const bool last = l + 1 == a.L;
    const int cur = l & 1;
    // every store of this CTA is issued before the last layer: arrive now,
    // wait before leaving (no CTA leaves while another may store into it)
    if (last) asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    // layer l's inputs: for l >= 1 the (l - 1) / 2-th use of buffer l % 2
    if (l > 0) ok = ok && wait_cluster_tx(&bar[cur], static_cast<uint32_t>((l - 1) >> 1) & 1u);
    // the next layer's buffer: its previous use was waited for a layer ago
    if (!last && tid == 0) mppi_tc::mbar_expect_tx(mppi_tc::smem_u32(&bar[cur ^ 1]), 4u * out);
    if (!ok) continue;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = act[cur][8 * lane + j];
#pragma unroll
    for (int c = 0; c < PC_COLS; ++c) {
      const int col = static_cast<int>(rank) * (PC_COLS * PC_THREADS / 32) + warp * PC_COLS + c;
      const __nv_bfloat162* w2 = reinterpret_cast<const __nv_bfloat162*>(&wf[l][c]);
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(w2[j]);
        s = fmaf(x[2 * j], f.x, fmaf(x[2 * j + 1], f.y, s));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      // every lane holds the sum: lane r < PC_CTAS stores it into CTA r
      if (col < out) {
        const float z = s + bias[l][c];
        if (last) {
          if (lane == 0) a.dst[col] = oplan[c] + (z * osd[c] + omean[c]);
        } else if (lane < PC_CTAS) {
          const float h = __bfloat162float(__float2bfloat16(gelu_f(z)));
          st_async_remote(&act[cur ^ 1][col], &bar[cur ^ 1], static_cast<uint32_t>(lane), h);
        }
      }
    }
  }
  if (!ok && tid == 0) {
    *a.err = 1;
    *a.k_split = 0x7fffffff;  // the next update samples around the plain warm start only
  }
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

int fail(int code, const std::string& msg) {
  mppi_set_thread_error(msg);
  return code;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode != nullptr;
}

// Tensor map of a K-major BF16 operand: rows x K elements, leading dimension
// ld elements (a multiple of 8), boxes of box_rows x 64 with 128-byte swizzle.
bool kmajor_map(CUtensorMap* map, const bf16* ptr, int rows, int K, long long ld, int box_rows) {
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(bf16)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(mppi_tc::BK), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(ptr), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct mppi_mlp_s {
  mppi_mlp_config cfg{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int L = 0;                   // layers with weights (hidden + output)
  int dims[MAX_LAYERS + 1];
  size_t woff[MAX_LAYERS + 1], boff[MAX_LAYERS + 1], nparam = 0;
  // parameters, gradients, Adam moments (FP32)
  float *p = nullptr, *g = nullptr, *am = nullptr, *av = nullptr;
  // BF16 weights: layer l at wb + wb_off[l], [out][ldw[l]], and its
  // transpose at wbT + wbt_off[l], [in][ldwt[l]]
  bf16 *wb = nullptr, *wbT = nullptr;
  size_t wb_off[MAX_LAYERS + 1], wbt_off[MAX_LAYERS + 1], wb_total = 0, wbt_total = 0;
  long long ldw[MAX_LAYERS + 1], ldwt[MAX_LAYERS + 1];
  long long step = 0;
  // standardisation
  float *mean_in = nullptr, *sd_in = nullptr, *mean_out = nullptr, *sd_out = nullptr;
  // activations for max_batch rows (BF16 row-major [B][ld] and transposed [width][ldb])
  long long ldb = 0, ldx = 0, ldh = 0, ldd = 0;
  bf16 *xb = nullptr, *xbT = nullptr;
  float* z[MAX_LAYERS + 1] = {};      // pre-activations [B][dims[l]]
  bf16* hb[MAX_LAYERS + 1] = {};      // BF16 gelu(z) of hidden layers [B][ldh]
  bf16* hbT[MAX_LAYERS + 1] = {};     // and transposed [dims[l]][ldb]
  bf16 *d0 = nullptr, *d1 = nullptr, *d0T = nullptr, *d1T = nullptr;  // deltas (ping-pong)
  float* loss = nullptr;
  int* err = nullptr;                 // set by a GEMM whose waits gave up
};

namespace {

int blocks(long long n, int t = 256) { return static_cast<int>((n + t - 1) / t); }

// C = A B^T on the tensor cores: A [M][K] (leading dimension lda), B [N][K]
// (ldb), both BF16 K-major; the epilogue in g.
cudaError_t gemm_tc(mppi_mlp_s* m, const bf16* A, long long lda, const bf16* B, long long ldb,
                    TcArgs g) {
  CUtensorMap ta, tb;
  if (!kmajor_map(&ta, A, g.M, g.K, lda, mppi_tc::BM) ||
      !kmajor_map(&tb, B, g.N, g.K, ldb, mppi_tc::BN))
    return cudaErrorInvalidValue;
  g.err = m->err;
  const dim3 grid((g.N + mppi_tc::BN - 1) / mppi_tc::BN, (g.M + mppi_tc::BM - 1) / mppi_tc::BM);
  mppi_tc::gemm_tc_kernel<<<grid, mppi_tc::THREADS, mppi_tc::SMEM_BYTES, m->st>>>(ta, tb, g);
  return cudaGetLastError();
}

TcArgs args0() {
  TcArgs g;
  std::memset(&g, 0, sizeof g);
  return g;
}

// forward of n standardised BF16 rows in m->xb; output (standardised) in z[L]
cudaError_t forward_rows(mppi_mlp_s* m, int n) {
  const bf16* h = m->xb;
  long long ldh_in = m->ldx;
  for (int l = 1; l <= m->L; ++l) {
    const int in = m->dims[l - 1], out = m->dims[l];
    TcArgs g = args0();
    g.M = n; g.N = out; g.K = in;
    g.bias = m->p + m->boff[l];
    g.Cf = m->z[l]; g.ldc = out;
    if (l < m->L) {
      g.epi = mppi_tc::EPI_GELU;
      g.Ch = m->hb[l]; g.ldh = m->ldh;
      g.ChT = m->hbT[l]; g.ldht = m->ldb;
    } else {
      g.epi = mppi_tc::EPI_F32;
    }
    cudaError_t e = gemm_tc(m, h, ldh_in, m->wb + m->wb_off[l], m->ldw[l], g);
    if (e != cudaSuccess) return e;
    h = m->hb[l];
    ldh_in = m->ldh;
  }
  return cudaSuccess;
}

cudaError_t normalize_rows(mppi_mlp_s* m, const float* x, int n) {
  const int nin = m->dims[0];
  normalize_in_kernel<<<blocks(static_cast<long long>(n) * nin), 256, 0, m->st>>>(
      x, n, nin, m->mean_in, m->sd_in, m->xb, m->ldx, m->xbT, m->ldb);
  return cudaGetLastError();
}

// loss and gradient into m->g for n rows (x raw, t raw targets)
cudaError_t loss_grad_rows(mppi_mlp_s* m, const float* x, const float* t, int n) {
  const int nout = m->dims[m->L];
  cudaError_t e = normalize_rows(m, x, n);
  if (e == cudaSuccess) e = forward_rows(m, n);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->loss, 0, sizeof(float), m->st);
  if (e != cudaSuccess) return e;
  loss_grad_kernel<<<blocks(static_cast<long long>(n) * nout), 256, 0, m->st>>>(
      m->z[m->L], t, n, nout, m->mean_out, m->sd_out, m->d0, m->ldd, m->d0T, m->ldb, m->loss);
  bf16 *dcur = m->d0, *dnext = m->d1, *dcurT = m->d0T, *dnextT = m->d1T;
  for (int l = m->L; l >= 1; --l) {
    const int in = m->dims[l - 1], out = m->dims[l];
    const bf16* hinT = l == 1 ? m->xbT : m->hbT[l - 1];
    // dW_l [out][in] = dZ^T H: A = dZ^T [out][n], B = H^T [in][n], K = n
    TcArgs g = args0();
    g.M = out; g.N = in; g.K = n;
    g.epi = mppi_tc::EPI_F32;
    g.Cf = m->g + m->woff[l]; g.ldc = in;
    if ((e = gemm_tc(m, dcurT, m->ldb, hinT, m->ldb, g)) != cudaSuccess) return e;
    colsum_kernel<<<out, 256, 0, m->st>>>(dcurT, m->ldb, n, out, m->g + m->boff[l]);
    if (l > 1) {
      // dZ_{l-1} [n][in] = (dZ W_l) * gelu'(z_{l-1}): A = dZ [n][out], B = W_l^T [in][out]
      TcArgs h = args0();
      h.M = n; h.N = in; h.K = out;
      h.epi = mppi_tc::EPI_GELU_GRAD;
      h.Ch = dnext; h.ldh = m->ldd;
      h.ChT = dnextT; h.ldht = m->ldb;
      h.Zin = m->z[l - 1]; h.ldz = in;
      if ((e = gemm_tc(m, dcur, m->ldd, m->wbT + m->wbt_off[l], m->ldwt[l], h)) != cudaSuccess)
        return e;
      std::swap(dcur, dnext);
      std::swap(dcurT, dnextT);
    }
  }
  return cudaGetLastError();
}

cudaError_t refresh_bf16(mppi_mlp_s* m) {
  for (int l = 1; l <= m->L; ++l) {
    const long long n = static_cast<long long>(m->dims[l]) * m->dims[l - 1];
    to_bf16_kernel<<<blocks(n), 256, 0, m->st>>>(m->p + m->woff[l], m->dims[l], m->dims[l - 1],
                                                 m->wb + m->wb_off[l], m->ldw[l],
                                                 m->wbT + m->wbt_off[l], m->ldwt[l]);
  }
  return cudaGetLastError();
}

// MPPI_ERR_TIMEOUT when a GEMM's bounded wait gave up (read after a sync)
// One bounded wait on an mbarrier that nothing completes, with the GEMMs'
// wait helper and error flag (the flag set when the wait gives up).
__global__ void wait_check_kernel(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mppi_tc::mbar_init(mppi_tc::smem_u32(&bar), 1);
  __syncthreads();
  if (!mppi_tc::mbar_wait(mppi_tc::smem_u32(&bar), 0, limit) && threadIdx.x == 0) *err = 1;
}

int check_err(mppi_mlp_s* m) {
  int h = 0;
  if (cudaMemcpy(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(MPPI_ERR_CUDA, "reading the GEMM status");
  if (h) {
    cudaMemset(m->err, 0, sizeof(int));
    return fail(MPPI_ERR_TIMEOUT, "a tensor-core GEMM gave up waiting for its operands");
  }
  return MPPI_OK;
}

int enqueue_propose(mppi_mlp_t m, mppi_t h, const float* d_in, int n_plain);

}  // namespace

extern "C" {

int mppi_mlp_create(const mppi_mlp_config* cfg, void* stream, mppi_mlp_t* out) {
  if (!cfg || !out) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (cfg->n_layers < 1 || cfg->n_layers > 6) return fail(MPPI_ERR_INVALID_ARG, "n_layers must be in 1..6");
  if (cfg->n_in < 1 || cfg->n_in > 1024 || cfg->n_hidden < 1 || cfg->n_hidden > 1024 ||
      cfg->n_out < 1 || cfg->n_out > 1024)
    return fail(MPPI_ERR_INVALID_ARG, "layer widths must be in 1..1024");
  if (cfg->max_batch < 1 || cfg->max_batch > 65536) return fail(MPPI_ERR_INVALID_ARG, "max_batch must be in 1..65536");
  if (!encoder()) return fail(MPPI_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  mppi_mlp_s* m = new (std::nothrow) mppi_mlp_s();
  if (!m) return fail(MPPI_ERR_OOM, "host allocation failed");
  m->cfg = *cfg;
  m->L = cfg->n_layers + 1;
  m->dims[0] = cfg->n_in;
  for (int l = 1; l < m->L; ++l) m->dims[l] = cfg->n_hidden;
  m->dims[m->L] = cfg->n_out;
  size_t off = 0, woff = 0, wtoff = 0;
  int maxw = 0;
  for (int l = 1; l <= m->L; ++l) {
    m->woff[l] = off;
    off += static_cast<size_t>(m->dims[l]) * m->dims[l - 1];
    m->boff[l] = off;
    off += m->dims[l];
    m->ldw[l] = pad8(m->dims[l - 1]);
    m->ldwt[l] = pad8(m->dims[l]);
    m->wb_off[l] = woff;
    woff += static_cast<size_t>(m->dims[l]) * m->ldw[l];
    m->wbt_off[l] = wtoff;
    wtoff += static_cast<size_t>(m->dims[l - 1]) * m->ldwt[l];
    maxw = std::max(maxw, m->dims[l]);
  }
  m->nparam = off;
  m->wb_total = woff;
  m->wbt_total = wtoff;
  const size_t B = cfg->max_batch;
  m->ldb = pad8(cfg->max_batch);
  m->ldx = pad8(cfg->n_in);
  m->ldh = pad8(cfg->n_hidden);
  m->ldd = pad8(maxw);
  auto bail = [&](cudaError_t e) {
    mppi_mlp_destroy(m);
    return fail(e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA, cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(mppi_tc::gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                mppi_tc::SMEM_BYTES)) != cudaSuccess)
    return bail(e);
  if (stream) {
    m->st = static_cast<cudaStream_t>(stream);
  } else {
    if ((e = cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
    m->own_stream = true;
  }
  auto zalloc = [&](void** ptr, size_t bytes) {
    cudaError_t r = cudaMalloc(ptr, bytes);
    return r == cudaSuccess ? cudaMemset(*ptr, 0, bytes) : r;  // padding stays zero
  };
  if ((e = cudaMalloc(&m->p, sizeof(float) * off)) != cudaSuccess ||
      (e = cudaMalloc(&m->g, sizeof(float) * off)) != cudaSuccess ||
      (e = cudaMalloc(&m->am, sizeof(float) * off)) != cudaSuccess ||
      (e = cudaMalloc(&m->av, sizeof(float) * off)) != cudaSuccess ||
      (e = zalloc(reinterpret_cast<void**>(&m->wb), sizeof(bf16) * woff)) != cudaSuccess ||
      (e = zalloc(reinterpret_cast<void**>(&m->wbT), sizeof(bf16) * wtoff)) != cudaSuccess ||
      (e = cudaMalloc(&m->mean_in, sizeof(float) * cfg->n_in)) != cudaSuccess ||
      (e = cudaMalloc(&m->sd_in, sizeof(float) * cfg->n_in)) != cudaSuccess ||
      (e = cudaMalloc(&m->mean_out, sizeof(float) * cfg->n_out)) != cudaSuccess ||
      (e = cudaMalloc(&m->sd_out, sizeof(float) * cfg->n_out)) != cudaSuccess ||
      (e = zalloc(reinterpret_cast<void**>(&m->xb), sizeof(bf16) * B * m->ldx)) != cudaSuccess ||
      (e = zalloc(reinterpret_cast<void**>(&m->xbT), sizeof(bf16) * cfg->n_in * m->ldb)) != cudaSuccess ||
      (e = zalloc(reinterpret_cast<void**>(&m->d0), sizeof(bf16) * B * m->ldd)) != cudaSuccess ||
      (e = zalloc(reinterpret_cast<void**>(&m->d1), sizeof(bf16) * B * m->ldd)) != cudaSuccess ||
      (e = zalloc(reinterpret_cast<void**>(&m->d0T), sizeof(bf16) * maxw * m->ldb)) != cudaSuccess ||
      (e = zalloc(reinterpret_cast<void**>(&m->d1T), sizeof(bf16) * maxw * m->ldb)) != cudaSuccess ||
      (e = cudaMalloc(&m->loss, sizeof(float))) != cudaSuccess ||
      (e = zalloc(reinterpret_cast<void**>(&m->err), sizeof(int))) != cudaSuccess)
    return bail(e);
  for (int l = 1; l <= m->L; ++l) {
    if ((e = cudaMalloc(&m->z[l], sizeof(float) * B * m->dims[l])) != cudaSuccess) return bail(e);
    if (l < m->L) {
      if ((e = zalloc(reinterpret_cast<void**>(&m->hb[l]), sizeof(bf16) * B * m->ldh)) != cudaSuccess ||
          (e = zalloc(reinterpret_cast<void**>(&m->hbT[l]), sizeof(bf16) * m->dims[l] * m->ldb)) != cudaSuccess)
        return bail(e);
    }
  }
  // Kaiming-uniform weights (bound sqrt(6 / fan_in) for GELU layers, sqrt(3 / fan_in) at the output)
  std::vector<float> hp(off, 0.f);
  std::mt19937_64 rng(cfg->seed);
  for (int l = 1; l <= m->L; ++l) {
    const float bound = std::sqrt((l < m->L ? 6.0f : 3.0f) / m->dims[l - 1]);
    std::uniform_real_distribution<float> U(-bound, bound);
    for (size_t i = 0; i < static_cast<size_t>(m->dims[l]) * m->dims[l - 1]; ++i) hp[m->woff[l] + i] = U(rng);
  }
  std::vector<float> zeros(std::max(cfg->n_in, cfg->n_out), 0.f), ones(std::max(cfg->n_in, cfg->n_out), 1.f);
  if ((e = cudaMemcpy(m->mean_in, zeros.data(), sizeof(float) * cfg->n_in, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(m->sd_in, ones.data(), sizeof(float) * cfg->n_in, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(m->mean_out, zeros.data(), sizeof(float) * cfg->n_out, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(m->sd_out, ones.data(), sizeof(float) * cfg->n_out, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e);
  *out = m;
  const int rc = mppi_mlp_set_params(m, hp.data());
  if (rc != MPPI_OK) {
    mppi_mlp_destroy(m);
    *out = nullptr;
  }
  return rc;
}

int mppi_mlp_destroy(mppi_mlp_t m) {
  if (!m) return MPPI_OK;
  if (m->st) cudaStreamSynchronize(m->st);
  cudaFree(m->p); cudaFree(m->g); cudaFree(m->am); cudaFree(m->av);
  cudaFree(m->wb); cudaFree(m->wbT);
  cudaFree(m->mean_in); cudaFree(m->sd_in); cudaFree(m->mean_out); cudaFree(m->sd_out);
  cudaFree(m->xb); cudaFree(m->xbT); cudaFree(m->d0); cudaFree(m->d1); cudaFree(m->d0T);
  cudaFree(m->d1T); cudaFree(m->loss); cudaFree(m->err);
  for (int l = 0; l <= MAX_LAYERS; ++l) {
    cudaFree(m->z[l]);
    cudaFree(m->hb[l]);
    cudaFree(m->hbT[l]);
  }
  if (m->own_stream && m->st) cudaStreamDestroy(m->st);
  delete m;
  return MPPI_OK;
}

int mppi_mlp_check_wait(mppi_mlp_t m, long long cycles) {
  if (!m || cycles < 1 || cycles > mppi_tc::WAIT_CYCLES)
    return fail(MPPI_ERR_INVALID_ARG, "bad argument");
  wait_check_kernel<<<1, 32, 0, m->st>>>(m->err, cycles);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
  return check_err(m);
}

int mppi_mlp_num_params(mppi_mlp_t m, size_t* n) {
  if (!m || !n) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  *n = m->nparam;
  return MPPI_OK;
}

int mppi_mlp_get_params(mppi_mlp_t m, float* host) {
  if (!m || !host) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  cudaError_t e = cudaMemcpyAsync(host, m->p, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  return e == cudaSuccess ? MPPI_OK : fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
}

int mppi_mlp_set_params(mppi_mlp_t m, const float* host) {
  if (!m || !host) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  for (size_t i = 0; i < m->nparam; ++i)
    if (!std::isfinite(host[i])) return fail(MPPI_ERR_INVALID_ARG, "parameters must be finite");
  cudaError_t e = cudaMemcpyAsync(m->p, host, sizeof(float) * m->nparam, cudaMemcpyHostToDevice, m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->am, 0, sizeof(float) * m->nparam, m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->av, 0, sizeof(float) * m->nparam, m->st);
  if (e == cudaSuccess) e = refresh_bf16(m);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  m->step = 0;
  return e == cudaSuccess ? MPPI_OK : fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
}

int mppi_mlp_set_normalization(mppi_mlp_t m, const float* mean_in, const float* std_in,
                               const float* mean_out, const float* std_out) {
  if (!m || !mean_in || !std_in || !mean_out || !std_out) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  for (int i = 0; i < m->cfg.n_in; ++i)
    if (!(std_in[i] > 0.f) || !std::isfinite(mean_in[i])) return fail(MPPI_ERR_INVALID_ARG, "bad input standardisation");
  for (int i = 0; i < m->cfg.n_out; ++i)
    if (!(std_out[i] > 0.f) || !std::isfinite(mean_out[i])) return fail(MPPI_ERR_INVALID_ARG, "bad output standardisation");
  cudaError_t e = cudaMemcpyAsync(m->mean_in, mean_in, sizeof(float) * m->cfg.n_in, cudaMemcpyHostToDevice, m->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->sd_in, std_in, sizeof(float) * m->cfg.n_in, cudaMemcpyHostToDevice, m->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->mean_out, mean_out, sizeof(float) * m->cfg.n_out, cudaMemcpyHostToDevice, m->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->sd_out, std_out, sizeof(float) * m->cfg.n_out, cudaMemcpyHostToDevice, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  return e == cudaSuccess ? MPPI_OK : fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
}

int mppi_mlp_fit_normalization(mppi_mlp_t m, const float* d_x, const float* d_y, int n,
                               float floor) {
  if (!m || !d_x || !d_y) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  if (n < 2) return fail(MPPI_ERR_INVALID_ARG, "n must be at least 2");
  if (!(floor > 0.f)) return fail(MPPI_ERR_INVALID_ARG, "floor must be > 0");
  colstats_kernel<<<m->cfg.n_in, 256, 0, m->st>>>(d_x, n, m->cfg.n_in, floor, m->mean_in, m->sd_in);
  colstats_kernel<<<m->cfg.n_out, 256, 0, m->st>>>(d_y, n, m->cfg.n_out, floor, m->mean_out,
                                                   m->sd_out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  return e == cudaSuccess ? MPPI_OK : fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
}

int mppi_mlp_forward(mppi_mlp_t m, const float* d_x, int n, float* d_y) {
  if (!m || !d_x || !d_y) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  if (n < 1 || n > m->cfg.max_batch) return fail(MPPI_ERR_INVALID_ARG, "n must be in 1..max_batch");
  const int nout = m->dims[m->L];
  cudaError_t e = normalize_rows(m, d_x, n);
  if (e == cudaSuccess) e = forward_rows(m, n);
  if (e == cudaSuccess) {
    denormalize_kernel<<<blocks(static_cast<long long>(n) * nout), 256, 0, m->st>>>(m->z[m->L], n, nout, m->mean_out, m->sd_out, d_y);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? MPPI_OK : fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
}

int mppi_mlp_loss_grad(mppi_mlp_t m, const float* d_x, const float* d_y, int n, float* loss,
                       float* grad_host) {
  if (!m || !d_x || !d_y || !loss) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  if (n < 1 || n > m->cfg.max_batch) return fail(MPPI_ERR_INVALID_ARG, "n must be in 1..max_batch");
  cudaError_t e = loss_grad_rows(m, d_x, d_y, n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st);
  if (e == cudaSuccess && grad_host)
    e = cudaMemcpyAsync(grad_host, m->g, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
  return check_err(m);
}

int mppi_mlp_train_step(mppi_mlp_t m, const float* d_x, const float* d_y, int n, float lr,
                        float* loss) {
  if (!m || !d_x || !d_y) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  if (n < 1 || n > m->cfg.max_batch) return fail(MPPI_ERR_INVALID_ARG, "n must be in 1..max_batch");
  if (!(lr > 0.f)) return fail(MPPI_ERR_INVALID_ARG, "lr must be > 0");
  cudaError_t e = loss_grad_rows(m, d_x, d_y, n);
  if (e == cudaSuccess) {
    m->step += 1;
    AdamArgs a;
    a.p = m->p; a.g = m->g; a.m = m->am; a.v = m->av; a.n = static_cast<long long>(m->nparam);
    a.lr = lr; a.b1 = m->cfg.beta1; a.b2 = m->cfg.beta2; a.eps = m->cfg.eps;
    a.c1 = 1.f - std::pow(m->cfg.beta1, static_cast<float>(m->step));
    a.c2 = 1.f - std::pow(m->cfg.beta2, static_cast<float>(m->step));
    adam_kernel<<<blocks(a.n), 256, 0, m->st>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = refresh_bf16(m);
  if (e == cudaSuccess && loss) {
    e = cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    if (e == cudaSuccess) return check_err(m);
  }
  return e == cudaSuccess ? MPPI_OK : fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
}

int mppi_mlp_propose(mppi_mlp_t m, mppi_t h, const float* d_in, int n_plain) {
  return enqueue_propose(m, h, d_in, n_plain);
}

int mppi_mlp_propose_step_device(mppi_mlp_t m, mppi_t h, const float* d_in, int n_plain,
                                 float* d_tau0, float* d_plan) {
  int rc = enqueue_propose(m, h, d_in, n_plain);
  if (rc != MPPI_OK) return rc;
  rc = mppi_internal_step_after_proposal(h, d_in, d_tau0, d_plan, n_plain);
  if (rc != MPPI_OK) mppi_set_thread_error(mppi_last_error(h));
  return rc;
}

}  // extern "C"

namespace {

int enqueue_propose(mppi_mlp_t m, mppi_t h, const float* d_in, int n_plain) {
  if (!m || !h || !d_in) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  const int T = mppi_internal_T(h);
  if (n_plain < 0 || n_plain > mppi_internal_K(h)) return fail(MPPI_ERR_INVALID_ARG, "n_plain must be in 0..K");
  if (m->L > PC_LMAX) return fail(MPPI_ERR_INVALID_ARG, "propose supports at most 3 hidden layers");
  for (int l = 0; l <= m->L; ++l)
    if (m->dims[l] > MAXW) return fail(MPPI_ERR_INVALID_ARG, "propose supports layer widths <= 256");
  if (m->cfg.n_in != 21 + 7 * T || m->cfg.n_out != 7 * T)
    return fail(MPPI_ERR_INVALID_ARG, "network widths do not match 21 + 7T inputs and 7T outputs");
  // queued on the handle's stream so that the proposal lands before its next update
  cudaStream_t hs = mppi_internal_stream(h);
  ProposeArgs a;
  std::memset(&a, 0, sizeof a);
  a.in = d_in;
  a.plan = mppi_internal_plan(h);
  a.wb = m->wb;
  a.p = m->p;
  a.L = m->L;
  for (int l = 0; l <= m->L; ++l) {
    a.dims[l] = m->dims[l];
    a.wb_off[l] = static_cast<long long>(m->wb_off[l]);
    a.ldw[l] = m->ldw[l];
    a.boff[l] = static_cast<long long>(m->boff[l]);
  }
  a.mean_in = m->mean_in;
  a.sd_in = m->sd_in;
  a.mean_out = m->mean_out;
  a.sd_out = m->sd_out;
  a.dst = mppi_internal_prop(h);
  a.k_split = mppi_internal_ctl(h);
  a.n_plain = n_plain;
  a.err = m->err;
  if (!a.dst || !a.k_split) return fail(MPPI_ERR_INVALID_ARG, "proposal buffers missing");
  propose_kernel<<<PC_CTAS, PC_THREADS, 0, hs>>>(a);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MPPI_OK : fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace
