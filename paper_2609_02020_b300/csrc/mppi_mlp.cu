// Learned proposal network (include/mppi_mlp.h): BF16 tensor-core training
// and inference kernels with FP32 accumulation.
//
// One GEMM kernel serves every product of the forward and backward passes:
// C[m][n] = sum_k A(m,k) B(k,n) with A and B in BF16 given by two strides
// each (so transposed operands need no copy), 64x64 output tiles per block,
// 32-deep K slices staged in shared memory as [row][k] for A and [n][k] for
// B, and warp-level mma.sync.m16n8k16 (row.col, BF16 in, FP32 accumulate).
// The epilogue fuses the bias, the GELU and the GELU derivative.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "mppi.h"
#include "mppi_mlp.h"

void mppi_set_thread_error(const std::string& msg);
float* mppi_internal_plan(mppi_t h);
int mppi_internal_T(mppi_t h);
cudaStream_t mppi_internal_stream(mppi_t h);
float* mppi_internal_prop(mppi_t h);
int mppi_internal_K(mppi_t h);
cudaError_t mppi_internal_set_split(mppi_t h, int k_split);

namespace {

using bf16 = __nv_bfloat16;
namespace cg = cooperative_groups;

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;
constexpr int MAX_LAYERS = 8;

enum Epi : int {
  EPI_F32 = 0,        // Cf = acc + bias
  EPI_GELU = 1,       // Cf = z = acc + bias;  Ch = bf16(gelu(z))
  EPI_GELU_GRAD = 2,  // Ch = bf16(acc * gelu'(Zin))
  EPI_F32_ACC = 3,    // Cf += acc
};

struct GemmArgs {
  int M, N, K;
  const bf16* A;
  long long sam, sak;
  const bf16* B;
  long long sbk, sbn;
  const float* bias;
  int epi;
  float* Cf;
  long long ldc;
  bf16* Ch;
  long long ldh;
  const float* Zin;
  long long ldz;
};

__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  // no side effects beyond its outputs: not volatile, so loads may be scheduled around it
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g) {
  __shared__ __align__(16) bf16 As[GBM][GBK + GPAD];
  __shared__ __align__(16) bf16 Bs[GBN][GBK + GPAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const bf16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < g.K; k0 += GBK) {
    // stage A(m0.., k0..) as [row][k]; walk the operand's contiguous index fastest
    for (int i = tid; i < GBM * GBK; i += 128) {
      int r, kk;
      if (g.sak == 1) { r = i / GBK; kk = i % GBK; }
      else { r = i % GBM; kk = i / GBM; }
      const int m = m0 + r, k = k0 + kk;
      As[r][kk] = (m < g.M && k < g.K) ? g.A[m * g.sam + k * g.sak] : zero;
    }
    for (int i = tid; i < GBN * GBK; i += 128) {
      int c, kk;
      if (g.sbk == 1) { c = i / GBK; kk = i % GBK; }
      else { c = i % GBN; kk = i / GBN; }
      const int n = n0 + c, k = k0 + kk;
      Bs[c][kk] = (n < g.N && k < g.K) ? g.B[k * g.sbk + n * g.sbn] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm + mt * 16 + gid, c = ks + tig * 2;
        af[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r][c]);
        af[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][c]);
        af[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r][c + 8]);
        af[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][c + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int n = wn + nt * 8 + gid, c = ks + tig * 2;
        bfr[nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][c]);
        bfr[nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][c + 8]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt]);
    }
    __syncthreads();
  }
  // epilogue: c0, c1 at (row gid, cols 2 tig, 2 tig + 1); c2, c3 at row gid + 8
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int m = m0 + wm + mt * 16 + gid + (h >= 2 ? 8 : 0);
        const int n = n0 + wn + nt * 8 + tig * 2 + (h & 1);
        if (m >= g.M || n >= g.N) continue;
        const float v = acc[mt][nt][h];
        switch (g.epi) {
          case EPI_F32:
            g.Cf[m * g.ldc + n] = v + (g.bias ? g.bias[n] : 0.f);
            break;
          case EPI_GELU: {
            const float z = v + (g.bias ? g.bias[n] : 0.f);
            g.Cf[m * g.ldc + n] = z;
            g.Ch[m * g.ldh + n] = __float2bfloat16(gelu_f(z));
            break;
          }
          case EPI_GELU_GRAD:
            g.Ch[m * g.ldh + n] = __float2bfloat16(v * gelu_grad_f(g.Zin[m * g.ldz + n]));
            break;
          default:
            g.Cf[m * g.ldc + n] += v;
            break;
        }
      }
}

// db[n] = sum_m D[m][n] (BF16 deltas, FP32 sum)
__global__ void colsum_kernel(const bf16* __restrict__ D, int M, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += __bfloat162float(D[static_cast<long long>(m) * N + n]);
  db[n] = s;
}

// xb = bf16((x - mean) / std)
__global__ void normalize_in_kernel(const float* __restrict__ x, int n, int d,
                                    const float* __restrict__ mean, const float* __restrict__ sd,
                                    bf16* __restrict__ xb) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<long long>(n) * d) return;
  const int f = static_cast<int>(i % d);
  xb[i] = __float2bfloat16((x[i] - mean[f]) / sd[f]);
}

// dY = bf16(scale (y - (t - mean)/std)); loss += sum of squares / (n d)
__global__ void loss_grad_kernel(const float* __restrict__ y, const float* __restrict__ t, int n,
                                 int d, const float* __restrict__ mean,
                                 const float* __restrict__ sd, bf16* __restrict__ dy,
                                 float* __restrict__ loss) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  float e2 = 0.f;
  if (i < static_cast<long long>(n) * d) {
    const int f = static_cast<int>(i % d);
    const float e = y[i] - (t[i] - mean[f]) / sd[f];
    dy[i] = __float2bfloat16(2.0f * e / (static_cast<float>(n) * d));
    e2 = e * e;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
  if ((threadIdx.x & 31) == 0 && e2 != 0.f) atomicAdd(loss, e2 / (static_cast<float>(n) * d));
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

// Adam on the flat FP32 parameters; refreshes the BF16 weight copies.
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

__global__ void to_bf16_kernel(const float* __restrict__ src, long long n, bf16* __restrict__ dst) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16(src[i]);
}

// Fused inference for one row (the learned proposal of one handle): input
// assembly (q, qd, goal of the input record, then the nominal plan), the
// input standardisation, every layer on the tensor cores (the row padded to
// an m16 tile; each warp owns n8 column tiles) with the same BF16 rounding
// points as the batched path, and the output de-standardisation; the output
// is the correction to the nominal plan, so dst = plan + net(x).  The layer's
// n8 tiles are spread over the warps of PC_BLOCKS blocks so that the weights
// stream through several SMs, each warp loading all of its weight fragments
// up front; a cooperative launch's grid barrier separates the layers, whose
// activations pass through a small global buffer.  Layer widths <= MAXW.
constexpr int PC_THREADS = 128;
constexpr int PC_BLOCKS = 8;    // 32 warps: one n8 tile of every layer each
constexpr int PC_LMAX = 4;      // layers with weights
constexpr int PC_KMAX = 16;     // k16 steps per layer (widths <= 256)
constexpr int MAXW = 256;

struct ProposeArgs {
  const float* in;      // 25-float input record
  const float* plan;    // nominal plan [7T]
  const bf16* wb;       // BF16 weights, layer l at wb_off[l]
  const float* p;       // FP32 parameters (biases at boff[l])
  long long wb_off[MAX_LAYERS + 1], boff[MAX_LAYERS + 1];
  int dims[MAX_LAYERS + 1];
  int L;
  const float *mean_in, *sd_in, *mean_out, *sd_out;
  bf16* act;            // [2][MAXW] activations between layers
  float* dst;           // [n_out]
};

// B fragments (W[n][k] pairs along k) of one n8 tile for k16 step j.
__device__ __forceinline__ void load_wfrag(const bf16* W, int in, int out, int n, int j, int tig,
                                           uint32_t b[2]) {
  const bf16 zero = __float2bfloat16(0.f);
  const int c = 16 * j + tig * 2;
  const bf16* Wn = W + static_cast<long long>(n) * in;
  if ((in % 2) == 0 && n < out && c + 9 < in) {  // rows start 4-byte aligned
    b[0] = *reinterpret_cast<const uint32_t*>(Wn + c);
    b[1] = *reinterpret_cast<const uint32_t*>(Wn + c + 8);
  } else {
    __nv_bfloat162 b0, b1;
    b0.x = (n < out && c < in) ? Wn[c] : zero;
    b0.y = (n < out && c + 1 < in) ? Wn[c + 1] : zero;
    b1.x = (n < out && c + 8 < in) ? Wn[c + 8] : zero;
    b1.y = (n < out && c + 9 < in) ? Wn[c + 9] : zero;
    b[0] = *reinterpret_cast<uint32_t*>(&b0);
    b[1] = *reinterpret_cast<uint32_t*>(&b1);
  }
}

__global__ void __launch_bounds__(PC_THREADS) propose_kernel(const ProposeArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ __align__(16) bf16 xin[MAXW];
  const int tid = threadIdx.x, lane = tid & 31;
  const int gw = blockIdx.x * (PC_THREADS / 32) + (tid >> 5);  // this warp's n8 tile
  const int gid = lane >> 2, tig = lane & 3;
  const bf16 zero = __float2bfloat16(0.f);
  const int n = gw * 8 + gid;
  // every weight fragment this warp needs, all layers, loaded before any
  // arithmetic: one memory latency for the whole network
  uint32_t wf[PC_LMAX][PC_KMAX][2];
#pragma unroll
  for (int l = 0; l < PC_LMAX; ++l)
#pragma unroll
    for (int j = 0; j < PC_KMAX; ++j) {
      if (l < a.L && 16 * j < a.dims[l]) {
        load_wfrag(a.wb + a.wb_off[l + 1], a.dims[l], a.dims[l + 1], n, j, tig, wf[l][j]);
      } else {
        wf[l][j][0] = 0u;
        wf[l][j][1] = 0u;
      }
    }
  bf16* cur = a.act;
  bf16* nxt = a.act + MAXW;
  const int n0 = a.dims[0];
  for (int i = blockIdx.x * PC_THREADS + tid; i < MAXW; i += gridDim.x * PC_THREADS) {
    float x = 0.f;
    if (i < n0) x = ((i < 21 ? a.in[i] : a.plan[i - 21]) - a.mean_in[i]) / a.sd_in[i];
    cur[i] = i < n0 ? __float2bfloat16(x) : zero;
    nxt[i] = zero;
  }
  grid.sync();
#pragma unroll
  for (int l = 0; l < PC_LMAX; ++l) {
    if (l >= a.L) break;
    const int in = a.dims[l], out = a.dims[l + 1];
    for (int i = tid; i < MAXW; i += PC_THREADS) xin[i] = cur[i];
    __syncthreads();
    if (gw * 8 < out) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < PC_KMAX; ++j) {
        if (16 * j >= in) break;
        const int c = 16 * j + tig * 2;
        uint32_t af[4];  // A: only row 0 (gid == 0) is non-zero
        af[0] = gid == 0 ? *reinterpret_cast<const uint32_t*>(&xin[c]) : 0u;
        af[1] = 0u;
        af[2] = gid == 0 ? *reinterpret_cast<const uint32_t*>(&xin[c + 8]) : 0u;
        af[3] = 0u;
        mma_bf16(acc, af, wf[l][j]);
      }
      if (gid == 0) {  // c0, c1: row 0, columns 2 tig, 2 tig + 1
        const float* bias = a.p + a.boff[l + 1];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = gw * 8 + tig * 2 + h;
          if (col >= out) continue;
          const float z = acc[h] + bias[col];
          if (l + 1 < a.L) nxt[col] = __float2bfloat16(gelu_f(z));
          else a.dst[col] = a.plan[col] + (z * a.sd_out[col] + a.mean_out[col]);
        }
      }
    }
    if (l + 1 < a.L) {
      grid.sync();
      bf16* t = cur;
      cur = nxt;
      nxt = t;
    }
  }
}

int fail(int code, const std::string& msg) {
  mppi_set_thread_error(msg);
  return code;
}

}  // namespace

struct mppi_mlp_s {
  mppi_mlp_config cfg{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int L = 0;                   // layers with weights (hidden + output)
  int dims[MAX_LAYERS + 1];
  size_t woff[MAX_LAYERS + 1], boff[MAX_LAYERS + 1], nparam = 0;
  // parameters, gradients, Adam moments (FP32), BF16 weight copies
  float *p = nullptr, *g = nullptr, *am = nullptr, *av = nullptr;
  bf16* wb = nullptr;
  size_t wb_off[MAX_LAYERS + 1];
  long long step = 0;
  // standardisation
  float *mean_in = nullptr, *sd_in = nullptr, *mean_out = nullptr, *sd_out = nullptr;
  // activations for max_batch rows
  bf16* xb = nullptr;                 // [B][n_in]
  float* z[MAX_LAYERS + 1] = {};      // pre-activations [B][dims[l]]
  bf16* hb[MAX_LAYERS + 1] = {};      // BF16 gelu(z) of hidden layers
  bf16 *d0 = nullptr, *d1 = nullptr;  // deltas (ping-pong) [B][max width]
  float* loss = nullptr;
  bf16* pact = nullptr;               // [2][MAXW] activations of mppi_mlp_propose
};

namespace {

cudaError_t gemm(cudaStream_t st, const GemmArgs& g) {
  dim3 grid((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM);
  gemm_bf16_kernel<<<grid, 128, 0, st>>>(g);
  return cudaGetLastError();
}

GemmArgs args0() {
  GemmArgs g;
  std::memset(&g, 0, sizeof g);
  return g;
}

int blocks(long long n, int t = 256) { return static_cast<int>((n + t - 1) / t); }

// forward of n standardised BF16 rows in m->xb; output (standardised) in z[L]
cudaError_t forward_rows(mppi_mlp_s* m, int n) {
  const bf16* h = m->xb;
  for (int l = 1; l <= m->L; ++l) {
    const int in = m->dims[l - 1], out = m->dims[l];
    GemmArgs g = args0();
    g.M = n; g.N = out; g.K = in;
    g.A = h; g.sam = in; g.sak = 1;
    g.B = m->wb + m->wb_off[l]; g.sbk = 1; g.sbn = in;  // B(k, n) = W[n][k]
    g.bias = m->p + m->boff[l];
    g.Cf = m->z[l]; g.ldc = out;
    if (l < m->L) {
      g.epi = EPI_GELU;
      g.Ch = m->hb[l]; g.ldh = out;
    } else {
      g.epi = EPI_F32;
    }
    cudaError_t e = gemm(m->st, g);
    if (e != cudaSuccess) return e;
    h = m->hb[l];
  }
  return cudaSuccess;
}

// loss and gradient into m->g for n rows (x raw, t raw targets)
cudaError_t loss_grad_rows(mppi_mlp_s* m, const float* x, const float* t, int n) {
  const int nin = m->dims[0], nout = m->dims[m->L];
  normalize_in_kernel<<<blocks(static_cast<long long>(n) * nin), 256, 0, m->st>>>(x, n, nin, m->mean_in, m->sd_in, m->xb);
  cudaError_t e = forward_rows(m, n);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(m->loss, 0, sizeof(float), m->st)) != cudaSuccess) return e;
  loss_grad_kernel<<<blocks(static_cast<long long>(n) * nout), 256, 0, m->st>>>(
      m->z[m->L], t, n, nout, m->mean_out, m->sd_out, m->d0, m->loss);
  bf16* dcur = m->d0;
  bf16* dnext = m->d1;
  for (int l = m->L; l >= 1; --l) {
    const int in = m->dims[l - 1], out = m->dims[l];
    const bf16* hin = l == 1 ? m->xb : m->hb[l - 1];
    // dW_l = dcur^T hin : A(m=o, k=row) = dcur[row][o], B(k=row, n=i) = hin[row][i]
    GemmArgs g = args0();
    g.M = out; g.N = in; g.K = n;
    g.A = dcur; g.sam = 1; g.sak = out;
    g.B = hin; g.sbk = in; g.sbn = 1;
    g.epi = EPI_F32;
    g.Cf = m->g + m->woff[l]; g.ldc = in;
    if ((e = gemm(m->st, g)) != cudaSuccess) return e;
    colsum_kernel<<<blocks(out), 256, 0, m->st>>>(dcur, n, out, m->g + m->boff[l]);
    if (l > 1) {
      // dz_{l-1} = (dcur W_l) * gelu'(z_{l-1}) : A = dcur [row][o], B(k=o, n=i) = W[o][i]
      GemmArgs h = args0();
      h.M = n; h.N = in; h.K = out;
      h.A = dcur; h.sam = out; h.sak = 1;
      h.B = m->wb + m->wb_off[l]; h.sbk = in; h.sbn = 1;
      h.epi = EPI_GELU_GRAD;
      h.Ch = dnext; h.ldh = in;
      h.Zin = m->z[l - 1]; h.ldz = in;
      if ((e = gemm(m->st, h)) != cudaSuccess) return e;
      std::swap(dcur, dnext);
    }
  }
  return cudaGetLastError();
}

cudaError_t refresh_bf16(mppi_mlp_s* m) {
  for (int l = 1; l <= m->L; ++l) {
    const long long n = static_cast<long long>(m->dims[l]) * m->dims[l - 1];
    to_bf16_kernel<<<blocks(n), 256, 0, m->st>>>(m->p + m->woff[l], n, m->wb + m->wb_off[l]);
  }
  return cudaGetLastError();
}

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
  mppi_mlp_s* m = new (std::nothrow) mppi_mlp_s();
  if (!m) return fail(MPPI_ERR_OOM, "host allocation failed");
  m->cfg = *cfg;
  m->L = cfg->n_layers + 1;
  m->dims[0] = cfg->n_in;
  for (int l = 1; l < m->L; ++l) m->dims[l] = cfg->n_hidden;
  m->dims[m->L] = cfg->n_out;
  size_t off = 0, woff = 0;
  int maxw = 0;
  for (int l = 1; l <= m->L; ++l) {
    m->woff[l] = off;
    off += static_cast<size_t>(m->dims[l]) * m->dims[l - 1];
    m->boff[l] = off;
    off += m->dims[l];
    m->wb_off[l] = woff;
    woff += static_cast<size_t>(m->dims[l]) * m->dims[l - 1];
    maxw = std::max(maxw, m->dims[l]);
  }
  m->nparam = off;
  const size_t B = cfg->max_batch;
  auto bail = [&](cudaError_t e) {
    mppi_mlp_destroy(m);
    return fail(e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA, cudaGetErrorString(e));
  };
  cudaError_t e;
  if (stream) {
    m->st = static_cast<cudaStream_t>(stream);
  } else {
    if ((e = cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
    m->own_stream = true;
  }
  if ((e = cudaMalloc(&m->p, sizeof(float) * off)) != cudaSuccess ||
      (e = cudaMalloc(&m->g, sizeof(float) * off)) != cudaSuccess ||
      (e = cudaMalloc(&m->am, sizeof(float) * off)) != cudaSuccess ||
      (e = cudaMalloc(&m->av, sizeof(float) * off)) != cudaSuccess ||
      (e = cudaMalloc(&m->wb, sizeof(bf16) * woff)) != cudaSuccess ||
      (e = cudaMalloc(&m->mean_in, sizeof(float) * cfg->n_in)) != cudaSuccess ||
      (e = cudaMalloc(&m->sd_in, sizeof(float) * cfg->n_in)) != cudaSuccess ||
      (e = cudaMalloc(&m->mean_out, sizeof(float) * cfg->n_out)) != cudaSuccess ||
      (e = cudaMalloc(&m->sd_out, sizeof(float) * cfg->n_out)) != cudaSuccess ||
      (e = cudaMalloc(&m->xb, sizeof(bf16) * B * cfg->n_in)) != cudaSuccess ||
      (e = cudaMalloc(&m->d0, sizeof(bf16) * B * maxw)) != cudaSuccess ||
      (e = cudaMalloc(&m->d1, sizeof(bf16) * B * maxw)) != cudaSuccess ||
      (e = cudaMalloc(&m->loss, sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&m->pact, sizeof(bf16) * 2 * MAXW)) != cudaSuccess)
    return bail(e);
  for (int l = 1; l <= m->L; ++l) {
    if ((e = cudaMalloc(&m->z[l], sizeof(float) * B * m->dims[l])) != cudaSuccess) return bail(e);
    if (l < m->L && (e = cudaMalloc(&m->hb[l], sizeof(bf16) * B * m->dims[l])) != cudaSuccess) return bail(e);
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
  cudaFree(m->p); cudaFree(m->g); cudaFree(m->am); cudaFree(m->av); cudaFree(m->wb);
  cudaFree(m->mean_in); cudaFree(m->sd_in); cudaFree(m->mean_out); cudaFree(m->sd_out);
  cudaFree(m->xb); cudaFree(m->d0); cudaFree(m->d1); cudaFree(m->loss); cudaFree(m->pact);
  for (int l = 0; l <= MAX_LAYERS; ++l) {
    cudaFree(m->z[l]);
    cudaFree(m->hb[l]);
  }
  if (m->own_stream && m->st) cudaStreamDestroy(m->st);
  delete m;
  return MPPI_OK;
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

int mppi_mlp_forward(mppi_mlp_t m, const float* d_x, int n, float* d_y) {
  if (!m || !d_x || !d_y) return fail(MPPI_ERR_INVALID_ARG, "null argument");
  if (n < 1 || n > m->cfg.max_batch) return fail(MPPI_ERR_INVALID_ARG, "n must be in 1..max_batch");
  const int nin = m->dims[0], nout = m->dims[m->L];
  normalize_in_kernel<<<blocks(static_cast<long long>(n) * nin), 256, 0, m->st>>>(d_x, n, nin, m->mean_in, m->sd_in, m->xb);
  cudaError_t e = forward_rows(m, n);
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
  return e == cudaSuccess ? MPPI_OK : fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
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
  }
  return e == cudaSuccess ? MPPI_OK : fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
}

int mppi_mlp_propose(mppi_mlp_t m, mppi_t h, const float* d_in, int n_plain) {
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
    a.boff[l] = static_cast<long long>(m->boff[l]);
  }
  a.mean_in = m->mean_in;
  a.sd_in = m->sd_in;
  a.mean_out = m->mean_out;
  a.sd_out = m->sd_out;
  a.act = m->pact;
  a.dst = mppi_internal_prop(h);
  if (!a.dst || !a.act) return fail(MPPI_ERR_INVALID_ARG, "proposal buffers missing");
  void* kargs[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(propose_kernel),
                                              dim3(PC_BLOCKS), dim3(PC_THREADS), kargs, 0, hs);
  if (e == cudaSuccess) e = mppi_internal_set_split(h, n_plain);
  return e == cudaSuccess ? MPPI_OK : fail(MPPI_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
