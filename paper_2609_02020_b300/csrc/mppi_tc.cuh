// BF16 GEMM on the fifth-generation tensor cores of sm_103a (tcgen05) for the
// learned proposal's network: C = A B^T with A [M][K] and B [N][K] both
// K-major (row-major with K contiguous), FP32 accumulation in tensor memory
// (TMEM), fused epilogues.
//
// One CTA of eight warps computes a 128 x 64 tile of C:
//   - thread 0 stages 128 x 64 (A) and 64 x 64 (B) BF16 tiles of a K slice
//     into shared memory with TMA (cp.async.bulk.tensor, 128-byte swizzle,
//     zero fill beyond the tensors' edges) through a ring of STAGES slots,
//     each slot's arrival tracked by an mbarrier with a transaction count;
//   - the same thread issues tcgen05.mma (M = 128, N = 64, K = 16 per
//     instruction) from shared-memory matrix descriptors into a 128-lane x
//     64-column FP32 accumulator in TMEM, and tcgen05.commit returns each
//     slot to the ring once the MMAs that read it are done;
//   - after the last slice, all eight warps read the accumulator back with
//     tcgen05.ld (warp w reaches TMEM lanes 32(w % 4)..32(w % 4)+31, i.e.
//     rows of the tile; warps w and w + 4 take the two halves of the
//     columns) and apply the epilogue.
// Every mbarrier wait gives up after WAIT_CYCLES and sets an error flag; the
// kernel then skips its stores, still waits (bounded) for its MMAs and
// frees its TMEM.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace mppi_tc {

using bf16 = __nv_bfloat16;

constexpr int BM = 128, BN = 64, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;        // 16 KB, a multiple of the 1 KB swizzle atom
constexpr int B_BYTES = BN * BK * 2;        // 8 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + 128;
constexpr uint32_t TMEM_COLS = 64;          // FP32 accumulator: 128 lanes x BN columns
constexpr long long WAIT_CYCLES = 2000000000ll;  // about a second
// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A
// and B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3
// at bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                           (static_cast<uint32_t>(BN >> 3) << 17) |
                           (static_cast<uint32_t>(BM >> 4) << 24);

enum Epi : int {
  EPI_F32 = 0,        // Cf = acc + bias
  EPI_GELU = 1,       // Cf = z = acc + bias;  Ch = ChT^T = bf16(gelu(z))
  EPI_GELU_GRAD = 2,  // Ch = ChT^T = bf16(acc * gelu'(Zin))
  EPI_F32_ACC = 3,    // Cf += acc
};

struct TcArgs {
  int M, N, K;
  int epi;
  const float* bias;
  float* Cf;
  long long ldc;
  bf16* Ch;
  long long ldh;
  bf16* ChT;          // transposed BF16 copy [N][M] (may be null)
  long long ldht;
  const float* Zin;
  long long ldz;
  int* err;           // set to 1 when a wait gave up
};

__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}
// Bounded wait for the completion of phase `phase` of the barrier.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase,
                                          long long limit = WAIT_CYCLES) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase))
    if (clock64() - t0 > limit) return false;
  return true;
}

// 2-D TMA load of the box at (x = K element, y = row) into shared memory.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle
// (rows of 128 bytes, 8-row swizzle atoms of 1 KB): start address >> 4
// (bits 0-13), leading-dimension offset 16 B (bits 16-29, unused by this
// layout), stride between 8-row groups 1024 B (bits 32-45), descriptor
// version 1 (bits 46-47), swizzle mode 2 = 128 B (bits 61-63).  A K step of
// 16 BF16 (32 B) inside the 128-byte row advances the start address by 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(1) << 16) |
         (static_cast<uint64_t>(1024 >> 4) << 32) | (static_cast<uint64_t>(1) << 46) |
         (static_cast<uint64_t>(2) << 61);
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t taddr, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}

// The mbarrier receives one arrival once every tcgen05 operation this thread
// issued before has completed.
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (lane i of the
// warp gets TMEM lane base + i).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int THREADS = 256;

__global__ void __launch_bounds__(THREADS, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
               const TcArgs g) {
  extern __shared__ uint8_t dsm_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(base);
  const uint32_t bars = sbase + STAGES * STAGE_BYTES;  // full[S], empty[S], done
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
  const uint32_t done = bars + 8u * (2 * STAGES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + STAGES * STAGE_BYTES + 8 * (2 * STAGES + 1));
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nk = (g.K + BK - 1) / BK;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tmem_slot;

  if (tid == 0) {
    bool ok = true;
    const int pre = nk < STAGES ? nk : STAGES;
    for (int s = 0; s < pre; ++s) {
      mbar_expect_tx(full(s), STAGE_BYTES);
      tma_load_2d(sbase + s * STAGE_BYTES, &tA, full(s), s * BK, m0);
      tma_load_2d(sbase + s * STAGE_BYTES + A_BYTES, &tB, full(s), s * BK, n0);
    }
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = static_cast<uint32_t>(kb / STAGES) & 1u;
      if (!mbar_wait(full(s), ph)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint64_t ad = sw128_desc(sbase + s * STAGE_BYTES);
      const uint64_t bd = sw128_desc(sbase + s * STAGE_BYTES + A_BYTES);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)
        tc_mma(taddr, ad + 2 * k, bd + 2 * k, (kb > 0 || k > 0) ? 1u : 0u);
      tc_commit(empty(s));
      if (kb + STAGES < nk) {
        if (!mbar_wait(empty(s), ph)) {
          ok = false;
          break;
        }
        mbar_expect_tx(full(s), STAGE_BYTES);
        tma_load_2d(sbase + s * STAGE_BYTES, &tA, full(s), (kb + STAGES) * BK, m0);
        tma_load_2d(sbase + s * STAGE_BYTES + A_BYTES, &tB, full(s), (kb + STAGES) * BK, n0);
      }
    }
    if (!ok) {
      s_abort = 1;
      atomicExch(g.err, 1);
    }
    tc_commit(done);  // arrives once every MMA issued above has completed
  }
  // block-uniform outcome, so that the warp-collective TMEM loads below run
  // in every warp or in none
  const bool got = __syncthreads_and(mbar_wait(done, 0) ? 1 : 0) != 0;
  tc_fence_after();
  if (got && !s_abort) {
    const int quad = warp & 3;  // the TMEM lanes this warp may read
    const int m = m0 + 32 * quad + lane;
    const uint32_t trow = taddr + (static_cast<uint32_t>(32 * quad) << 16);
    const int cbeg = (warp >> 2) * (BN / 2);
    const float* __restrict__ bias = g.bias;
    const float* __restrict__ zin = g.Zin;
    float* __restrict__ cf = g.Cf;
    bf16* __restrict__ ch = g.Ch;
    bf16* __restrict__ cht = g.ChT;
#pragma unroll 1
    for (int c0 = cbeg; c0 < cbeg + BN / 2; c0 += 16) {
      float v[16];
      tc_ld16(trow + c0, v);
      const int nb = n0 + c0;
      // every operand of the chunk is loaded before the first use, so that
      // the loads overlap (one memory latency per chunk)
      float aux[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = nb + j;
        aux[j] = 0.f;
        if (n < g.N) {
          if (g.epi == EPI_GELU_GRAD) {
            if (m < g.M) aux[j] = __ldg(zin + m * g.ldz + n);
          } else if (bias) {
            aux[j] = __ldg(bias + n);
          }
        }
      }
      if (m >= g.M) continue;
      const bool full = nb + 16 <= g.N;
      // vector stores only where the whole row chunk is 16-byte aligned
      const bool cf_vec = full && (g.ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(cf) & 15) == 0;
      const bool ch_vec = full && (g.ldh & 7) == 0 && (reinterpret_cast<uintptr_t>(ch) & 15) == 0;
      if (g.epi == EPI_F32 || g.epi == EPI_F32_ACC) {
        float o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) o[j] = v[j] + aux[j];
        float* row = cf + m * g.ldc + nb;
        if (g.epi == EPI_F32_ACC) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (nb + j < g.N) row[j] += o[j];
        } else if (cf_vec) {
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(row + j) = make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (nb + j < g.N) row[j] = o[j];
        }
        continue;
      }
      bf16 hv[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (g.epi == EPI_GELU) {
          const float z = v[j] + aux[j];
          v[j] = z;
          hv[j] = __float2bfloat16(gelu_f(z));
        } else {  // EPI_GELU_GRAD
          hv[j] = __float2bfloat16(v[j] * gelu_grad_f(aux[j]));
        }
      }
      if (g.epi == EPI_GELU) {
        float* row = cf + m * g.ldc + nb;
        if (cf_vec) {
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(row + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (nb + j < g.N) row[j] = v[j];
        }
      }
      bf16* hrow = ch + m * g.ldh + nb;
      if (ch_vec) {
        *reinterpret_cast<uint4*>(hrow) = *reinterpret_cast<const uint4*>(hv);
        *reinterpret_cast<uint4*>(hrow + 8) = *reinterpret_cast<const uint4*>(hv + 8);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (nb + j < g.N) hrow[j] = hv[j];
      }
      if (cht) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (nb + j < g.N) cht[(nb + j) * g.ldht + m] = hv[j];
      }
    }
  } else if (tid == 0 && !got) {
    atomicExch(g.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(TMEM_COLS)
                 : "memory");
}

}  // namespace mppi_tc
