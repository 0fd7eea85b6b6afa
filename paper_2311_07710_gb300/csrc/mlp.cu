// Learned warm start: a tensor-core (tcgen05) BF16 GEMM and the forward,
// backward and Adam kernels of the warm-start network (sm_103a).
//
// The paper has no learned component; Algorithm 1 takes its starting point
// (x^{0,0}, y^{0,0}) as an input and this network produces one for a member of
// a parameterised QP family from its data (c, b).  Network: per-feature
// normalisation u = (v - mean) * scale of v = [c; b], h_0 = u P' with a fixed
// random projection P (d x F), depth hidden layers h_j = relu(h_{j-1} W_j' + b_j)
// of width w, output o = h W_out' + b_out, prediction [x0; y0] = omean + ostd * o.
// Training minimises the mean squared error to the normalised solver outputs
// [x*; y*] with Adam.  Weights and activations are stored in bfloat16, every
// product accumulates in float32 in tensor memory, master weights, gradients
// and Adam moments are float32.
//
// GEMM: D[M x N] = A[M x K] * B[N x K]^T with A and B row-major bfloat16 (both
// K-major), persistent: one CUDA block per SM walks 128 x 256 tiles (128 x 128
// when N < 256) and k splits.  Thread 0 of warp 0 streams 64-wide K slices of
// A and B into a 4-stage shared-memory ring with TMA (128-byte swizzle),
// thread 0 of warp 1 issues tcgen05.mma (M=128, N=256, K=16, kind::f16 with
// bf16 A and B) on each stage into one of two float32 accumulators in tensor
// memory and releases the stage with tcgen05.commit, and warps 2..5 drain the
// other accumulator with tcgen05.ld into the fused epilogue (warp w reads TMEM
// lanes 32 (w mod 4) .. +32), so a tile's epilogue overlaps the next tile's
// main loop.  Split-K: a unit takes a range of k slices and writes raw float32
// partials that a second kernel sums in a fixed order.  Every mbarrier wait is
// bounded; a wait that gives up sets the error flag, the roles leave their
// loops, the copies still in flight land (bounded), the tensor memory is freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pdqp.h"
#include "pdqp_ws.h"

typedef __nv_bfloat16 bf16;

namespace mlp {

// Tile: BM = 128 rows of A, BN = 128 or 256 rows of B (the N width of the MMA
// and of the tensor-memory accumulator), BK = 64 (one 128-byte swizzle row).
constexpr int BM = 128, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;                    // 16 KiB
template <int BN> struct Tile {
  static constexpr int B_BYTES = BN * BK * 2;           // 16 or 32 KiB
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */;
};
constexpr uint64_t WAIT_NS = 200000000ULL;            // a wait gives up after 0.2 s without progress

struct Epi {
  float* out_f;                  // float32 output [M x ldo] or null
  bf16* out_b;                   // bf16 output [M x ldo] or null
  const float* bias;             // [N] or null
  const bf16* mask;              // [M x ldm]: keep where mask > 0, else 0 (ReLU derivative), or null
  int ldo, ldm;
  int relu;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the completion of the phase with the given parity: gives up
// (false) after WAIT_NS without progress (progress = a counter another thread
// of the block advances, or null) or as soon as the error flag is set.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* err,
                                          const volatile int* progress = nullptr) {
  const uint32_t a = smem_u32(bar);
  uint64_t start = 0;
  int seen = progress ? *progress : 0;
  for (uint32_t i = 0;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 255) == 255) {
      const uint64_t now = global_ns();
      if (start == 0) start = now;
      if (progress && *progress != seen) {
        seen = *progress;
        start = now;
      }
      if (now - start > WAIT_NS || *err) return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::
          "r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzle: rows of 64 bf16 (128 B), 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = (uint64_t)(smem_u32(p) & 0x3FFFF) >> 4;
  uint64_t d = 0;
  d |= addr;                         // bits 0-13: start address / 16
  d |= (uint64_t)1 << 16;            // bits 16-29: leading byte offset / 16 (ignored with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;  // bits 32-45: stride byte offset / 16
  d |= (uint64_t)1 << 46;            // bits 46-48: descriptor version 1
  d |= (uint64_t)2 << 61;            // bits 61-63: 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: bf16 A and B, both K-major, float32 D.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
  return (1u << 4)                      // D format: f32
         | (1u << 7)                    // A format: bf16
         | (1u << 10)                   // B format: bf16
         | ((uint32_t)(n >> 3) << 17)   // N / 8
         | ((uint32_t)(m >> 4) << 24);  // M / 16
}

__device__ __forceinline__ float epi_value(float r, int row, int col, const Epi& e) {
  if (e.bias) r += e.bias[col];
  if (e.relu) r = fmaxf(r, 0.f);
  if (e.mask && !(__bfloat162float(e.mask[(size_t)row * e.ldm + col]) > 0.f)) r = 0.f;
  return r;
}

// Epilogue of 32 accumulator columns of one row: the raw float32 split-K
// partial of split z (ld = N), or the fused epilogue into the outputs.
__device__ __forceinline__ void store_chunk(const uint32_t (&v)[32], int row, int cb, int z, int M, int N,
                                            const Epi& epi, float* __restrict__ partial) {
  if (partial) {   // raw float32 partial of this k range, ld = N
    float* dst = partial + ((size_t)z * M + row) * N + cb;
    if (cb + 32 <= N && (N & 3) == 0) {
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *(float4*)(dst + i) = make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]),
                                          __uint_as_float(v[i + 2]), __uint_as_float(v[i + 3]));
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (cb + i < N) dst[i] = __uint_as_float(v[i]);
    }
    return;
  }
  float r[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) r[i] = __uint_as_float(v[i]);
  if (cb + 32 <= N) {
#pragma unroll
    for (int i = 0; i < 32; ++i) r[i] = epi_value(r[i], row, cb + i, epi);
    const size_t o = (size_t)row * epi.ldo + cb;
    if (epi.out_f) {
      if ((epi.ldo & 3) == 0) {
#pragma unroll
        for (int i = 0; i < 32; i += 4) *(float4*)(epi.out_f + o + i) = make_float4(r[i], r[i + 1], r[i + 2], r[i + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) epi.out_f[o + i] = r[i];
      }
    }
    if (epi.out_b) {
      if ((epi.ldo & 7) == 0) {
#pragma unroll
        for (int i = 0; i < 32; i += 8) {
          uint4 q;
          __nv_bfloat162 h0 = __floats2bfloat162_rn(r[i], r[i + 1]), h1 = __floats2bfloat162_rn(r[i + 2], r[i + 3]),
                         h2 = __floats2bfloat162_rn(r[i + 4], r[i + 5]), h3 = __floats2bfloat162_rn(r[i + 6], r[i + 7]);
          q.x = *(uint32_t*)&h0;
          q.y = *(uint32_t*)&h1;
          q.z = *(uint32_t*)&h2;
          q.w = *(uint32_t*)&h3;
          *(uint4*)(epi.out_b + o + i) = q;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) epi.out_b[o + i] = __float2bfloat16_rn(r[i]);
      }
    }
  } else {   // the ragged last columns: a test per column keeps the indexing static
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      if (cb + i < N) {
        const float x = epi_value(r[i], row, cb + i, epi);
        const size_t o = (size_t)row * epi.ldo + cb + i;
        if (epi.out_f) epi.out_f[o] = x;
        if (epi.out_b) epi.out_b[o] = __float2bfloat16_rn(x);
      }
    }
  }
}

// 32 float32 accumulator columns of this warp's TMEM lanes, from column address taddr
__device__ __forceinline__ void tmem_ld32(uint32_t (&v)[32], uint32_t taddr) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// D = A B' (bf16 A, B K-major, float32 accumulation in tensor memory), persistent:
// one CTA per SM takes work units u = blockIdx.x,
// blockIdx.x + gridDim.x, ... (a unit is one BM x BN tile of one k split;
// the tiles in bands of tile rows, see `unit`).
// Warp roles: warp 0 lane 0 issues the TMA loads of every unit through the
// STAGES ring, warp 1 lane 0 the MMAs, warps 2..5 drain the accumulators
// (warp w reads TMEM lanes 32 (w mod 4) .. +32).  Two accumulators of BN
// columns: the epilogue of one unit overlaps the main loop of the next.
// Every wait is bounded (WAIT_NS without progress, or the error flag), after
// which the roles leave their loops, the copies in flight land, and the TMEM
// is freed.
template <int BN>
__global__ void __launch_bounds__(192, 1)
    k_gemm_tn_p(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                int K, int ktps, int splits, Epi epi, float* __restrict__ partial, int* err) {
  constexpr int STAGE_BYTES = Tile<BN>::STAGE_BYTES;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;       // [2]: the MMAs of a unit are done
  uint64_t* acc_empty = acc_full + 2;        // [2]: the epilogue has read the accumulator
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);
  __shared__ volatile int s_fail;
  __shared__ int s_issued;                   // stage loads issued, for the cleanup
  __shared__ volatile int s_progress;        // stages consumed by the MMA issuer
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tn = (N + BN - 1) / BN, tm = (M + BM - 1) / BM;
  const int KT = (K + BK - 1) / BK;
  const int units = tm * tn * splits;

  if (threadIdx.x == 0) {
    s_fail = 0;
    s_issued = 0;
    s_progress = 0;
    for (int q = 0; q < STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], 4);           // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {   // two accumulators: 128 lanes x 2 BN float32 columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;

  // tiles in bands of GROUP tile rows, column-major inside a band: the CTAs
  // running together cover about GROUP rows of A and gridDim / GROUP columns of
  // B tiles, a working set that stays in L2
  constexpr int GROUP = 8;
  auto unit = [&](int u, int& m0, int& n0, int& kt0, int& nk, int& z) {
    z = u / (tm * tn);
    const int t = u - z * (tm * tn);
    const int band = t / (GROUP * tn), first = band * GROUP;
    const int rows = min(tm - first, GROUP);
    const int q = t - band * GROUP * tn;
    m0 = (first + q % rows) * BM;
    n0 = (q / rows) * BN;
    kt0 = z * ktps;
    nk = min(KT, kt0 + ktps) - kt0;
  };

  if (warp == 0 && lane == 0) {   // TMA producer
    int i = 0;
    for (int u = blockIdx.x; u < units && !s_fail; u += gridDim.x) {
      int m0, n0, kt0, nk, z;
      unit(u, m0, n0, kt0, nk, z);
      for (int k = 0; k < nk; ++k, ++i) {
        const int q = i % STAGES;
        if (i >= STAGES && !mbar_wait(&empty[q], ((i / STAGES) - 1) & 1, err, &s_progress)) {
          s_fail = 1;
          break;
        }
        unsigned char* a = sm + q * STAGE_BYTES;
        mbar_expect_tx(&full[q], STAGE_BYTES);
        tma_load_2d(a, &mapA, &full[q], (kt0 + k) * BK, m0);
        tma_load_2d(a + A_BYTES, &mapB, &full[q], (kt0 + k) * BK, n0);
        s_issued = i + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {   // MMA issuer
    const uint32_t idesc = instr_desc(BM, BN);
    int i = 0, lt = 0;
    for (int u = blockIdx.x; u < units && !s_fail; u += gridDim.x, ++lt) {
      int m0, n0, kt0, nk, z;
      unit(u, m0, n0, kt0, nk, z);
      const int buf = lt & 1;
      // the epilogue has drained this accumulator (its first use passes at once)
      if (!mbar_wait(&acc_empty[buf], ((lt >> 1) & 1) ^ 1, err)) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const uint32_t acc_tm = tmem + (uint32_t)(buf * BN);
      for (int k = 0; k < nk; ++k, ++i) {
        const int q = i % STAGES;
        if (!mbar_wait(&full[q], (i / STAGES) & 1, err)) {
          s_fail = 1;
          break;
        }
        s_progress = i + 1;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const unsigned char* a = sm + q * STAGE_BYTES;
        const uint64_t da = smem_desc(a), db = smem_desc(a + A_BYTES);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t step = (uint64_t)((kk * 16 * 2) >> 4);   // 32 bytes further along K
          const uint32_t acc = (k > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_tm),
              "l"(da + step), "l"(db + step), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(&empty[q])));
      }
      if (s_fail) break;
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(&acc_full[buf])));
    }
  } else if (warp >= 2) {   // epilogue
    const int sp = warp & 3;
    int lt = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x, ++lt) {
      int m0, n0, kt0, nk, z;
      unit(u, m0, n0, kt0, nk, z);
      const int buf = lt & 1;
      if (s_fail || !mbar_wait(&acc_full[buf], (lt >> 1) & 1, err, &s_progress)) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const int row = m0 + sp * 32 + lane;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(v, tmem + ((uint32_t)(sp * 32) << 16) + (uint32_t)(buf * BN + c0));
        if (row < M) store_chunk(v, row, n0 + c0, z, M, N, epi, splits > 1 ? partial : nullptr);
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&acc_empty[buf])) : "memory");
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (s_fail && threadIdx.x == 0) {   // record the failure; let the copies in flight land
    atomicExch(err, 1);
    const int issued = s_issued;
    for (int i = max(0, issued - STAGES); i < issued; ++i) {
      int never = 0;
      mbar_wait(&full[i % STAGES], (i / STAGES) & 1, &never);
    }
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * BN));
}

// The bounded wait of the tensor-core kernels on an mbarrier that nothing
// completes: it gives up after WAIT_NS and raises the error flag, as a GEMM
// whose copies or MMAs never landed would (the host then reads
// PDQP_DEVICE_TIMEOUT and the context stays usable).
__global__ void k_wait_probe(int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, err)) atomicExch(err, 1);
}

// Sum of the split-K partials in a fixed order, then the epilogue.
__global__ void k_splitk_epi(const float* __restrict__ part, int splits, int M, int N, Epi epi) {
  const long long MN = (long long)M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < MN; i += (long long)gridDim.x * blockDim.x) {
    float r = 0.f;
    for (int z = 0; z < splits; ++z) r += part[z * MN + i];
    const int row = (int)(i / N), col = (int)(i % N);
    r = epi_value(r, row, col, epi);
    const size_t o = (size_t)row * epi.ldo + col;
    if (epi.out_f) epi.out_f[o] = r;
    if (epi.out_b) epi.out_b[o] = __float2bfloat16_rn(r);
  }
}

// --------------------------------------------------------------------------
// network kernels
// --------------------------------------------------------------------------
__device__ __forceinline__ long long visit(long long a, long long s, long long count, long long i) {
  return (a * i + s) % count;
}

// u = bf16((fl32(v) - mean) * scale) for rows [row0, row0+rows) of v = [C | B]
__global__ void k_prep_input(const double* __restrict__ C, const double* __restrict__ B, int n, int m, long long row0,
                             int rows, const float* __restrict__ mean, const float* __restrict__ scale,
                             bf16* __restrict__ U, int ldu) {
  const int F = n + m;
  const long long total = (long long)rows * F;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / F), f = (int)(i % F);
    const long long smp = row0 + r;
    const double v = f < n ? C[smp * n + f] : B[smp * m + (f - n)];
    U[(size_t)r * ldu + f] = __float2bfloat16_rn(__fmul_rn(__fsub_rn((float)v, mean[f]), scale[f]));
  }
}

// t = (fl32(v) - omean) * oinv, float32, for rows [0, count) of [X | Y]
__global__ void k_prep_target(const double* __restrict__ X, const double* __restrict__ Y, int n, int m,
                              long long count, const float* __restrict__ omean, const float* __restrict__ oinv,
                              float* __restrict__ T, int ldt) {
  const int F = n + m;
  const long long total = count * F;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / F;
    const int f = (int)(i % F);
    const double v = f < n ? X[r * n + f] : Y[r * m + (f - n)];
    T[r * ldt + f] = __fmul_rn(__fsub_rn((float)v, omean[f]), oinv[f]);
  }
}

// per-feature mean and population std over `count` rows (two passes, float64);
// std below 1e-8 counts as 1
__global__ void k_fit_stats(const double* __restrict__ V, long long count, int nf, float* __restrict__ mean,
                            float* __restrict__ scale, float* __restrict__ stdv) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  double s = 0.0;
  for (long long r = 0; r < count; ++r) s += V[r * nf + f];
  const double mu = s / (double)count;
  double q = 0.0;
  for (long long r = 0; r < count; ++r) {
    const double d = V[r * nf + f] - mu;
    q += d * d;
  }
  double sd = sqrt(q / (double)count);
  if (sd < 1e-8) sd = 1.0;
  mean[f] = (float)mu;
  scale[f] = (float)(1.0 / sd);
  if (stdv) stdv[f] = (float)sd;
}

__global__ void k_gather_rows(const bf16* __restrict__ src, int ld, long long a, long long s, long long count,
                              long long row0, int rows, int d, bf16* __restrict__ dst, int ldd) {
  const int vec = d / 8;   // d is a multiple of 8
  const long long total = (long long)rows * vec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / vec), k = (int)(i % vec) * 8;
    const long long smp = visit(a, s, count, row0 + r);
    *(uint4*)(dst + (size_t)r * ldd + k) = *(const uint4*)(src + (size_t)smp * ld + k);
  }
}

// Gradient tiles (32 rows x 32 features per block of 32 x 8 threads).
// MODE 0 (output layer): g = (o - t) * scale with t the target row of sample
// visit(row0 + r); also the squared-error partial of the block.
// MODE 1 (hidden layer): g = in.
// Writes g as bf16 row-major [rows x ldg] and transposed [F x ldgt], and the
// float32 column sums of the tile to colpart[blockIdx.y][f].
template <int MODE>
__global__ void __launch_bounds__(256) k_grad_tiles(const float* __restrict__ in, int ldi, const float* __restrict__ T,
                                                    int ldt, long long a, long long sft, long long count,
                                                    long long row0, int rows, int F, float scale, bf16* __restrict__ gb,
                                                    int ldg, bf16* __restrict__ gt, int ldgt,
                                                    float* __restrict__ colpart, int ldc, double* __restrict__ lossp) {
  __shared__ float tile[32][33];
  __shared__ double red[8];
  const int f0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int f = f0 + tx;
  double ls = 0.0;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i;
    float g = 0.f;
    if (r < rows && f < F) {
      const float o = in[(size_t)r * ldi + f];
      if (MODE == 0) {
        const long long smp = visit(a, sft, count, row0 + r);
        const float d = __fsub_rn(o, T[(size_t)smp * ldt + f]);
        ls += (double)d * (double)d;
        g = __fmul_rn(d, scale);
      } else {
        g = o;
      }
      gb[(size_t)r * ldg + f] = __float2bfloat16_rn(g);
    }
    tile[i][tx] = g;
  }
  __syncthreads();
  if (ty == 0 && f < F) {
    float s = 0.f;
    for (int i = 0; i < 32; ++i) s += tile[i][tx];
    colpart[(size_t)blockIdx.y * ldc + f] = s;
  }
  for (int i = ty; i < 32; i += 8) {
    const int ff = f0 + i, rr = r0 + tx;
    if (ff < F && rr < rows) gt[(size_t)ff * ldgt + rr] = __float2bfloat16_rn(tile[tx][i]);
  }
  if (MODE == 0) {
    for (int o = 16; o > 0; o >>= 1) ls += __shfl_down_sync(0xffffffffu, ls, o);
    if (tx == 0) red[ty] = ls;
    __syncthreads();
    if (tx == 0 && ty == 0) {
      double t = 0.0;
      for (int i = 0; i < 8; ++i) t += red[i];
      lossp[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  }
}

__global__ void k_colsum(const float* __restrict__ part, int ntiles, int F, int ld, float* __restrict__ out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  float s = 0.f;
  for (int t = 0; t < ntiles; ++t) s += part[(size_t)t * ld + f];
  out[f] = s;
}

// acc += inv * sum(parts) (one block of 256 threads, fixed order)
__global__ void k_loss_acc(const double* __restrict__ parts, int n, double inv, double* __restrict__ acc) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += parts[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *acc += inv * red[0];
}

__global__ void k_transpose_bf16(const bf16* __restrict__ in, int ldi, int rows, int cols, bf16* __restrict__ out,
                                 int ldo) {
  __shared__ bf16 t[32][34];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[(size_t)r * ldi + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(size_t)c * ldo + r] = t[threadIdx.x][i];
  }
}

struct AdamArgs {
  float lr, b1, b2, eps, c1, c2;   // c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
  int update;                      // 0: only refresh the bf16 copies
};

__device__ __forceinline__ float adam_one(float w, float g, float& m, float& v, const AdamArgs& a) {
  m = a.b1 * m + (1.f - a.b1) * g;
  v = a.b2 * v + (1.f - a.b2) * g * g;
  return w - a.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
}

// Adam on a rows x cols weight (all float32 arrays row-major, ld = cols), then
// the bf16 copy [rows x ldb] and the transposed bf16 copy [cols x ldt].
__global__ void __launch_bounds__(256) k_adam_mat(float* __restrict__ W, float* __restrict__ mW,
                                                  float* __restrict__ vW, const float* __restrict__ g, int rows,
                                                  int cols, AdamArgs a, bf16* __restrict__ Wb, int ldb,
                                                  bf16* __restrict__ Wt, int ldt) {
  __shared__ bf16 t[32][34];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) {
      const size_t k = (size_t)r * cols + c;
      float w = W[k];
      if (a.update) {
        float m = mW[k], v = vW[k];
        w = adam_one(w, g[k], m, v, a);
        W[k] = w;
        mW[k] = m;
        vW[k] = v;
      }
      const bf16 h = __float2bfloat16_rn(w);
      Wb[(size_t)r * ldb + c] = h;
      t[i][threadIdx.x] = h;
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) Wt[(size_t)c * ldt + r] = t[threadIdx.x][i];
  }
}

__global__ void k_adam_vec(float* __restrict__ b, float* __restrict__ mb, float* __restrict__ vb,
                           const float* __restrict__ g, int n, AdamArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !a.update) return;
  float m = mb[i], v = vb[i];
  b[i] = adam_one(b[i], g[i], m, v, a);
  mb[i] = m;
  vb[i] = v;
}

__global__ void k_f32_to_bf16_2d(const float* __restrict__ in, int rows, int cols, bf16* __restrict__ out, int ldo) {
  const long long total = (long long)rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / cols), c = (int)(i % cols);
    out[(size_t)r * ldo + c] = __float2bfloat16_rn(in[i]);
  }
}

// [x0 | y0] = omean + ostd * o in float64, rows [row0, row0+rows)
__global__ void k_write_pred(const float* __restrict__ O, int ldo, int rows, int n, int m,
                             const float* __restrict__ omean, const float* __restrict__ ostd, long long row0,
                             double* __restrict__ X0, double* __restrict__ Y0) {
  const int F = n + m;
  const long long total = (long long)rows * F;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / F), f = (int)(i % F);
    const double v = __dadd_rn((double)omean[f], __dmul_rn((double)ostd[f], (double)O[(size_t)r * ldo + f]));
    const long long smp = row0 + r;
    if (f < n) {
      if (X0) X0[smp * n + f] = v;
    } else if (Y0) {
      Y0[smp * m + (f - n)] = v;
    }
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// Tensor map of a row-major rows x cols bf16 matrix with leading dimension ld
// (elements): boxes of box_rows rows x 64 columns, 128-byte swizzle, zero fill
// outside the matrix.
static bool make_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if (((uintptr_t)base & 15) || (((size_t)ld * 2) & 15) || cols > ld) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int num_sms() {   // of the current device, read once (a thread-safe static)
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

// the B tile width: 256 when N fills it, else 128
inline int tile_n(int N) { return N >= 256 ? 256 : 128; }

// number of K splits: enough blocks to cover the SMs, at least 4 k-tiles each
int plan_splits(int M, int N, int K, int requested) {
  const int BN = tile_n(N);
  const int KT = (K + BK - 1) / BK;
  int splits = requested;
  if (splits <= 0) {
    const long long tiles = (long long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    splits = 1;
    if (tiles < num_sms()) splits = (int)std::min<long long>(KT / 4, (num_sms() + tiles - 1) / tiles);
  }
  splits = std::max(1, std::min(splits, KT));
  const int ktps = (KT + splits - 1) / splits;
  return (KT + ktps - 1) / ktps;
}

size_t splitk_floats(int M, int N, int K, int splits) {
  const int s = plan_splits(M, N, K, splits);
  return s > 1 ? (size_t)s * M * N : 0;
}

// D = A B^T (+ epilogue).  A: M x K (lda), B: N x K (ldb), bf16 row-major.
// `work` holds at least splitk_floats(M, N, K, splits) floats, else no split.
cudaError_t gemm_tn(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, const Epi& epi, int splits,
                    float* work, size_t work_floats, int* err, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  const int BN = tile_n(N);
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, lda, BM) || !make_map(&mb, B, N, K, ldb, BN)) return cudaErrorInvalidValue;
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_gemm_tn_p<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tile<128>::SMEM_BYTES);
    cudaFuncSetAttribute(k_gemm_tn_p<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tile<256>::SMEM_BYTES);
  });
  const int KT = (K + BK - 1) / BK;
  int sp = plan_splits(M, N, K, splits);
  if (sp > 1 && (!work || work_floats < (size_t)sp * M * N)) sp = 1;
  const int ktps = (KT + sp - 1) / sp;
  const long long units = (long long)((N + BN - 1) / BN) * ((M + BM - 1) / BM) * sp;
  const int grid = (int)std::min<long long>(units, num_sms());
  if (BN == 256)
    k_gemm_tn_p<256><<<grid, 192, Tile<256>::SMEM_BYTES, s>>>(ma, mb, M, N, K, ktps, sp, epi, work, err);
  else
    k_gemm_tn_p<128><<<grid, 192, Tile<128>::SMEM_BYTES, s>>>(ma, mb, M, N, K, ktps, sp, epi, work, err);
  if (sp > 1) {
    const long long MN = (long long)M * N;
    const int blocks = (int)std::min<long long>((MN + 255) / 256, 8LL * num_sms());
    k_splitk_epi<<<blocks, 256, 0, s>>>(work, sp, M, N, epi);
  }
  return cudaGetLastError();
}

inline int grid_for(long long total, int threads = 256) {
  return (int)std::max<long long>(1, std::min<long long>((total + threads - 1) / threads, 16LL * num_sms()));
}
inline int r8(long long v) { return (int)((v + 7) / 8 * 8); }

}  // namespace mlp

// ==========================================================================
// the network handle
// ==========================================================================
using namespace mlp;

struct WsLayer {
  int out = 0, in = 0;
  float *W = nullptr, *b = nullptr, *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr, *gW = nullptr,
        *gb = nullptr;
  bf16 *Wb = nullptr, *Wt = nullptr;   // [out x in] and [in x ldt]
  int ldt = 0;
};

struct pdqp_ws_s {
  int n = 0, m = 0, F = 0, Fp = 0, d = 0, width = 0, depth = 0, maxb = 0;
  int ldc = 0;                         // leading dimension of colpart: max(Fp, width)
  std::vector<WsLayer> L;              // depth hidden layers, then the output layer
  bf16* P = nullptr;                   // [d x Fp], fixed projection
  float *in_mean = nullptr, *in_scale = nullptr, *out_mean = nullptr, *out_std = nullptr, *out_inv = nullptr;
  bool have_norm = false, have_proj = false;
  long long step = 0;                  // Adam steps taken
  std::vector<bf16*> H, Ht;            // activations [maxb x ld] and transposes [ld x maxb]
  bf16* U = nullptr;                   // normalised inputs [maxb x Fp]
  float* O = nullptr;                  // outputs [maxb x Fp]
  float* G = nullptr;                  // hidden gradients [maxb x width]
  bf16 *dOb = nullptr, *dOt = nullptr, *dZb = nullptr, *dZt = nullptr;
  float* colpart = nullptr;            // [(maxb/32 + 1) x ldc]
  double* lossp = nullptr;             // [(maxb/32 + 1) x (Fp/32 + 1)]
  double* lossacc = nullptr;
  float* work = nullptr;               // split-K partials
  size_t work_floats = 0;
  int* err = nullptr;
  // training set
  long long tcount = 0;
  bf16* H0all = nullptr;               // [count x d]
  float* Tall = nullptr;               // [count x Fp]
  std::vector<void*> allocs;
  std::string last_error;
};

namespace {

struct WsFail {
  pdqp_status st;
  std::string msg;
};

thread_local std::string g_ws_error;

#define WCK(x)                                                                                          \
  do {                                                                                                  \
    cudaError_t e_ = (x);                                                                               \
    if (e_ != cudaSuccess)                                                                              \
      throw WsFail{e_ == cudaErrorMemoryAllocation ? PDQP_ERR_OOM : PDQP_ERR_CUDA,                      \
                   std::string(#x) + ": " + cudaGetErrorString(e_)};                                    \
  } while (0)

template <class T>
T* walloc(pdqp_ws_s* w, size_t count) {
  void* p = nullptr;
  WCK(cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)));
  w->allocs.push_back(p);
  return (T*)p;
}

void wfree(pdqp_ws_s* w, void* p) {
  if (!p) return;
  cudaFree(p);
  auto it = std::find(w->allocs.begin(), w->allocs.end(), p);
  if (it != w->allocs.end()) w->allocs.erase(it);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void check_space(const void* p, int mem, const char* what) {
  if (mem != PDQP_MEM_HOST && mem != PDQP_MEM_DEVICE) throw WsFail{PDQP_ERR_INVALID, "mem_space"};
  if (!p) return;
  if ((mem == PDQP_MEM_DEVICE) != is_device_ptr(p))
    throw WsFail{PDQP_ERR_INVALID, std::string(what) + " does not live in the given mem_space"};
}

// A device view of `count` elements: the pointer itself, or a temporary copy.
template <class T>
struct DevView {
  T* p = nullptr;
  bool owned = false;
  DevView(const T* src, size_t count, int mem, cudaStream_t s) {
    if (!src || mem == PDQP_MEM_DEVICE || count == 0) {
      p = const_cast<T*>(src);
      return;
    }
    WCK(cudaMalloc(&p, count * sizeof(T)));
    owned = true;
    const cudaError_t e = cudaMemcpyAsync(p, src, count * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      cudaFree(p);
      p = nullptr;
      owned = false;
      WCK(e);
    }
  }
  ~DevView() {
    if (owned) cudaFree(p);   // cudaFree waits for the work queued on the copy
  }
  DevView(const DevView&) = delete;
  DevView& operator=(const DevView&) = delete;
};

void gemm(pdqp_ws_s* w, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, const Epi& e,
          cudaStream_t s) {
  const size_t need = splitk_floats(M, N, K, 0);
  if (need > w->work_floats) {
    WCK(cudaStreamSynchronize(s));
    wfree(w, w->work);
    w->work = nullptr;
    w->work_floats = 0;
    w->work = walloc<float>(w, need);
    w->work_floats = need;
  }
  WCK(gemm_tn(A, lda, B, ldb, M, N, K, e, 0, w->work, w->work_floats, w->err, s));
}

Epi epi_of(float* of, bf16* ob, int ldo, const float* bias, int relu, const bf16* mask = nullptr, int ldm = 0) {
  Epi e;
  e.out_f = of;
  e.out_b = ob;
  e.ldo = ldo;
  e.bias = bias;
  e.relu = relu;
  e.mask = mask;
  e.ldm = ldm;
  return e;
}

// forward from H[0] (rows x d) to O; hidden activations in H[1..depth]
void forward(pdqp_ws_s* w, int rows, cudaStream_t s) {
  for (int j = 0; j < w->depth; ++j) {
    const WsLayer& l = w->L[j];
    gemm(w, w->H[j], l.in, l.Wb, l.in, rows, l.out, l.in, epi_of(nullptr, w->H[j + 1], l.out, l.b, 1), s);
  }
  const WsLayer& o = w->L[w->depth];
  gemm(w, w->H[w->depth], o.in, o.Wb, o.in, rows, w->F, o.in, epi_of(w->O, nullptr, w->Fp, o.b, 0), s);
}

// Backward of the mean squared error against targets T (the target of row r
// is row visit(a, sft, count, row0 + r) of T); leaves the gradients in gW/gb
// and adds loss / (rows F) to *lossacc.
void backward(pdqp_ws_s* w, int rows, const float* T, long long a, long long sft, long long count, long long row0,
              cudaStream_t s) {
  const int F = w->F, Fp = w->Fp, mb = w->maxb;
  const int rt = (rows + 31) / 32;
  {
    dim3 grid((F + 31) / 32, rt), blk(32, 8);
    const float scale = (float)(2.0 / ((double)rows * F));
    k_grad_tiles<0><<<grid, blk, 0, s>>>(w->O, Fp, T, Fp, a, sft, count, row0, rows, F, scale, w->dOb, Fp, w->dOt,
                                         mb, w->colpart, w->ldc, w->lossp);
    k_loss_acc<<<1, 256, 0, s>>>(w->lossp, (int)(grid.x * grid.y), 1.0 / ((double)rows * F), w->lossacc);
  }
  WsLayer& o = w->L[w->depth];
  k_colsum<<<(F + 255) / 256, 256, 0, s>>>(w->colpart, rt, F, w->ldc, o.gb);
  {
    const int c = o.in;
    dim3 grid((c + 31) / 32, rt), blk(32, 8);
    k_transpose_bf16<<<grid, blk, 0, s>>>(w->H[w->depth], c, rows, c, w->Ht[w->depth], mb);
  }
  // gW_out = dO' H_depth  (F x width), K = rows
  gemm(w, w->dOt, mb, w->Ht[w->depth], mb, F, o.in, rows, epi_of(o.gW, nullptr, o.in, nullptr, 0), s);
  // dZ of the last hidden layer = (dO W_out) * (H_depth > 0)
  gemm(w, w->dOb, Fp, o.Wt, o.ldt, rows, o.in, F, epi_of(w->G, nullptr, o.in, nullptr, 0, w->H[w->depth], o.in), s);
  for (int j = w->depth - 1; j >= 0; --j) {
    WsLayer& l = w->L[j];
    {
      dim3 grid((l.out + 31) / 32, rt), blk(32, 8);
      k_grad_tiles<1><<<grid, blk, 0, s>>>(w->G, l.out, nullptr, 0, 1, 0, 1LL << 62, 0, rows, l.out, 1.f, w->dZb,
                                           l.out, w->dZt, mb, w->colpart, w->ldc, nullptr);
    }
    k_colsum<<<(l.out + 255) / 256, 256, 0, s>>>(w->colpart, rt, l.out, w->ldc, l.gb);
    {
      dim3 grid((l.in + 31) / 32, rt), blk(32, 8);
      k_transpose_bf16<<<grid, blk, 0, s>>>(w->H[j], l.in, rows, l.in, w->Ht[j], mb);
    }
    gemm(w, w->dZt, mb, w->Ht[j], mb, l.out, l.in, rows, epi_of(l.gW, nullptr, l.in, nullptr, 0), s);
    if (j > 0)
      gemm(w, w->dZb, l.out, l.Wt, l.ldt, rows, l.in, l.out, epi_of(w->G, nullptr, l.in, nullptr, 0, w->H[j], l.in),
           s);
  }
}

void adam(pdqp_ws_s* w, float lr, float b1, float b2, float eps, cudaStream_t s) {
  w->step += 1;
  AdamArgs a;
  a.lr = lr;
  a.b1 = b1;
  a.b2 = b2;
  a.eps = eps;
  a.c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)w->step)));
  a.c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)w->step)));
  a.update = 1;
  for (WsLayer& l : w->L) {
    dim3 grid((l.in + 31) / 32, (l.out + 31) / 32), blk(32, 8);
    k_adam_mat<<<grid, blk, 0, s>>>(l.W, l.mW, l.vW, l.gW, l.out, l.in, a, l.Wb, l.in, l.Wt, l.ldt);
    k_adam_vec<<<(l.out + 255) / 256, 256, 0, s>>>(l.b, l.mb, l.vb, l.gb, l.out, a);
  }
}

void refresh_copies(WsLayer& l, cudaStream_t s) {
  AdamArgs a{};
  a.update = 0;
  dim3 grid((l.in + 31) / 32, (l.out + 31) / 32), blk(32, 8);
  k_adam_mat<<<grid, blk, 0, s>>>(l.W, l.mW, l.vW, l.gW, l.out, l.in, a, l.Wb, l.in, l.Wt, l.ldt);
}

// normalised inputs of rows [row0, row0+rows) -> U -> H0 = U P'
void project(pdqp_ws_s* w, const double* C, const double* B, long long row0, int rows, bf16* H0, cudaStream_t s) {
  k_prep_input<<<grid_for((long long)rows * w->F), 256, 0, s>>>(C, B, w->n, w->m, row0, rows, w->in_mean,
                                                                w->in_scale, w->U, w->Fp);
  gemm(w, w->U, w->Fp, w->P, w->Fp, rows, w->d, w->F, epi_of(nullptr, H0, w->d, nullptr, 0), s);
}

void finish(pdqp_ws_s* w, cudaStream_t s) {
  int herr = 0;
  WCK(cudaGetLastError());
  WCK(cudaMemcpyAsync(&herr, w->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  WCK(cudaStreamSynchronize(s));
  if (herr) {
    cudaMemsetAsync(w->err, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    throw WsFail{PDQP_DEVICE_TIMEOUT, "a tensor-core GEMM wait gave up (device timeout)"};
  }
}

template <class Fn>
pdqp_status guard(pdqp_ws_s* w, Fn fn) {
  try {
    fn();
    return PDQP_OK;
  } catch (const WsFail& f) {
    (w ? w->last_error : g_ws_error) = f.msg;
    return f.st;
  } catch (const std::bad_alloc&) {
    (w ? w->last_error : g_ws_error) = "host allocation failed";
    return PDQP_ERR_OOM;
  }
}

void need_ready(const pdqp_ws_s* w) {
  if (!w->have_norm) throw WsFail{PDQP_ERR_INVALID, "normalisation not set: call pdqp_ws_fit or pdqp_ws_set_normalization"};
  if (!w->have_proj) throw WsFail{PDQP_ERR_INVALID, "projection not set: call pdqp_ws_set_params with layer -1"};
}

void need_data(const pdqp_ws_s* w, const void* C, const void* B, const void* X, const void* Y, int mem, bool targets) {
  if (!C || (w->m > 0 && !B) || (targets && (!X || (w->m > 0 && !Y))))
    throw WsFail{PDQP_ERR_INVALID, "null C, B, X or Y"};
  for (const void* p : {C, B, X, Y}) check_space(p, mem, "data array");
}

// visit order of an epoch: i -> (a i + sft) mod count, (a, sft) from SplitMix64
// (Steele, Lea & Flood 2014) of the seed and the epoch
void visit_order(uint64_t seed, int epoch, long long count, long long* a_out, long long* s_out) {
  auto mix = [](uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  auto gcd = [](long long p, long long q) {
    while (q) {
      const long long t = p % q;
      p = q;
      q = t;
    }
    return p;
  };
  const uint64_t z = mix(seed * 0x9E3779B97F4A7C15ULL + (uint64_t)epoch * 0xD1B54A32D192ED03ULL);
  long long a = (long long)(z % (uint64_t)count) | 1;
  while (gcd(a, count) != 1) a += 2;
  a %= count;
  if (a == 0) a = 1;
  *a_out = a;
  *s_out = (long long)((z >> 32) % (uint64_t)count);
}

}  // namespace

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

pdqp_status pdqp_ws_create(pdqp_ws_handle* out, int64_t n, int64_t m, int32_t d, int32_t width, int32_t depth,
                           int32_t max_batch, void* stream) {
  if (!out) return PDQP_ERR_INVALID;
  *out = nullptr;
  return guard(nullptr, [&] {
    if (n < 1 || m < 0 || n + m > (1LL << 26)) throw WsFail{PDQP_ERR_INVALID, "sizes: need n >= 1, m >= 0, n + m <= 2^26"};
    if (d < 8 || width < 8 || d % 8 || width % 8 || d > 16384 || width > 16384)
      throw WsFail{PDQP_ERR_INVALID, "d and width: multiples of 8 in [8, 16384]"};
    if (depth < 1 || depth > 16) throw WsFail{PDQP_ERR_INVALID, "depth in [1, 16]"};
    if (max_batch < 8 || max_batch % 8 || max_batch > 8192)
      throw WsFail{PDQP_ERR_INVALID, "max_batch: multiple of 8 in [8, 8192]"};
    cudaStream_t s = (cudaStream_t)stream;
    pdqp_ws_s* w = new pdqp_ws_s();
    try {
      w->n = (int)n;
      w->m = (int)m;
      w->F = (int)(n + m);
      w->Fp = r8(w->F);
      w->d = d;
      w->width = width;
      w->depth = depth;
      w->maxb = max_batch;
      const int Fp = w->Fp, mb = max_batch;
      w->L.resize(depth + 1);
      for (int j = 0; j <= depth; ++j) {
        WsLayer& l = w->L[j];
        l.in = j == 0 ? d : width;
        l.out = j == depth ? w->F : width;
        l.ldt = r8(l.out);
        const size_t ne = (size_t)l.out * l.in;
        l.W = walloc<float>(w, ne);
        l.mW = walloc<float>(w, ne);
        l.vW = walloc<float>(w, ne);
        l.gW = walloc<float>(w, ne);
        l.b = walloc<float>(w, l.out);
        l.mb = walloc<float>(w, l.out);
        l.vb = walloc<float>(w, l.out);
        l.gb = walloc<float>(w, l.out);
        l.Wb = walloc<bf16>(w, ne);
        l.Wt = walloc<bf16>(w, (size_t)l.in * l.ldt);
        for (void* p : {(void*)l.W, (void*)l.mW, (void*)l.vW, (void*)l.gW})
          WCK(cudaMemsetAsync(p, 0, ne * sizeof(float), s));
        for (void* p : {(void*)l.b, (void*)l.mb, (void*)l.vb, (void*)l.gb})
          WCK(cudaMemsetAsync(p, 0, l.out * sizeof(float), s));
        WCK(cudaMemsetAsync(l.Wb, 0, ne * sizeof(bf16), s));
        WCK(cudaMemsetAsync(l.Wt, 0, (size_t)l.in * l.ldt * sizeof(bf16), s));
      }
      w->P = walloc<bf16>(w, (size_t)d * Fp);
      WCK(cudaMemsetAsync(w->P, 0, (size_t)d * Fp * sizeof(bf16), s));
      for (float** p : {&w->in_mean, &w->in_scale, &w->out_mean, &w->out_std, &w->out_inv}) {
        *p = walloc<float>(w, Fp);
        WCK(cudaMemsetAsync(*p, 0, (size_t)Fp * sizeof(float), s));
      }
      w->H.resize(depth + 1);
      w->Ht.resize(depth + 1);
      for (int j = 0; j <= depth; ++j) {
        const int c = j == 0 ? d : width;
        w->H[j] = walloc<bf16>(w, (size_t)mb * c);
        w->Ht[j] = walloc<bf16>(w, (size_t)c * mb);
      }
      w->U = walloc<bf16>(w, (size_t)mb * Fp);
      WCK(cudaMemsetAsync(w->U, 0, (size_t)mb * Fp * sizeof(bf16), s));
      w->O = walloc<float>(w, (size_t)mb * Fp);
      w->G = walloc<float>(w, (size_t)mb * width);
      w->dOb = walloc<bf16>(w, (size_t)mb * Fp);
      w->dOt = walloc<bf16>(w, (size_t)Fp * mb);
      w->dZb = walloc<bf16>(w, (size_t)mb * width);
      w->dZt = walloc<bf16>(w, (size_t)width * mb);
      w->ldc = std::max(Fp, width);
      w->colpart = walloc<float>(w, (size_t)(mb / 32 + 1) * w->ldc);
      w->lossp = walloc<double>(w, (size_t)(mb / 32 + 1) * (Fp / 32 + 1));
      w->lossacc = walloc<double>(w, 1);
      w->err = walloc<int>(w, 1);
      WCK(cudaMemsetAsync(w->err, 0, sizeof(int), s));
      WCK(cudaMemsetAsync(w->lossacc, 0, sizeof(double), s));
      WCK(cudaStreamSynchronize(s));
    } catch (...) {
      pdqp_ws_destroy(w);
      throw;
    }
    *out = w;
  });
}

void pdqp_ws_destroy(pdqp_ws_handle w) {
  if (!w) return;
  cudaDeviceSynchronize();
  for (void* p : w->allocs) cudaFree(p);
  delete w;
}

const char* pdqp_ws_last_error(pdqp_ws_handle w) { return w ? w->last_error.c_str() : g_ws_error.c_str(); }

pdqp_status pdqp_ws_set_params(pdqp_ws_handle w, int32_t layer, const float* W, const float* b, int32_t mem,
                               void* stream) {
  if (!w) return PDQP_ERR_INVALID;
  return guard(w, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (layer < -1 || layer > w->depth) throw WsFail{PDQP_ERR_INVALID, "layer out of range"};
    if (!W) throw WsFail{PDQP_ERR_INVALID, "null W"};
    check_space(W, mem, "W");
    check_space(b, mem, "b");
    if (layer == -1) {
      DevView<float> v(W, (size_t)w->d * w->F, mem, s);
      k_f32_to_bf16_2d<<<grid_for((long long)w->d * w->F), 256, 0, s>>>(v.p, w->d, w->F, w->P, w->Fp);
      WCK(cudaGetLastError());
      WCK(cudaStreamSynchronize(s));
      w->have_proj = true;
      return;
    }
    const cudaMemcpyKind kind = mem == PDQP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    WsLayer& l = w->L[layer];
    WCK(cudaMemcpyAsync(l.W, W, (size_t)l.out * l.in * sizeof(float), kind, s));
    if (b) WCK(cudaMemcpyAsync(l.b, b, (size_t)l.out * sizeof(float), kind, s));
    else WCK(cudaMemsetAsync(l.b, 0, (size_t)l.out * sizeof(float), s));
    refresh_copies(l, s);
    WCK(cudaGetLastError());
    WCK(cudaStreamSynchronize(s));
  });
}

pdqp_status pdqp_ws_get_params(pdqp_ws_handle w, int32_t layer, int32_t what, float* W, float* b, int32_t mem,
                               void* stream) {
  if (!w) return PDQP_ERR_INVALID;
  return guard(w, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (layer < 0 || layer > w->depth) throw WsFail{PDQP_ERR_INVALID, "layer out of range"};
    if (what < 0 || what > 3)
      throw WsFail{PDQP_ERR_INVALID, "what: 0 parameters, 1 gradients, 2 first moments, 3 second moments"};
    check_space(W, mem, "W");
    check_space(b, mem, "b");
    const WsLayer& l = w->L[layer];
    const float* srcW[4] = {l.W, l.gW, l.mW, l.vW};
    const float* srcb[4] = {l.b, l.gb, l.mb, l.vb};
    const cudaMemcpyKind kind = mem == PDQP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (W) WCK(cudaMemcpyAsync(W, srcW[what], (size_t)l.out * l.in * sizeof(float), kind, s));
    if (b) WCK(cudaMemcpyAsync(b, srcb[what], (size_t)l.out * sizeof(float), kind, s));
    WCK(cudaStreamSynchronize(s));
  });
}

pdqp_status pdqp_ws_set_normalization(pdqp_ws_handle w, const float* in_mean, const float* in_scale,
                                      const float* out_mean, const float* out_std, const float* out_inv, int32_t mem,
                                      void* stream) {
  if (!w) return PDQP_ERR_INVALID;
  return guard(w, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    const float* src[5] = {in_mean, in_scale, out_mean, out_std, out_inv};
    float* dst[5] = {w->in_mean, w->in_scale, w->out_mean, w->out_std, w->out_inv};
    for (int i = 0; i < 5; ++i) {
      if (!src[i]) throw WsFail{PDQP_ERR_INVALID, "null normalisation vector"};
      check_space(src[i], mem, "normalisation vector");
    }
    const cudaMemcpyKind kind = mem == PDQP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int i = 0; i < 5; ++i) WCK(cudaMemcpyAsync(dst[i], src[i], (size_t)w->F * sizeof(float), kind, s));
    WCK(cudaStreamSynchronize(s));
    w->have_norm = true;
  });
}

pdqp_status pdqp_ws_get_normalization(pdqp_ws_handle w, float* in_mean, float* in_scale, float* out_mean,
                                      float* out_std, float* out_inv, int32_t mem, void* stream) {
  if (!w) return PDQP_ERR_INVALID;
  return guard(w, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    float* dst[5] = {in_mean, in_scale, out_mean, out_std, out_inv};
    const float* src[5] = {w->in_mean, w->in_scale, w->out_mean, w->out_std, w->out_inv};
    const cudaMemcpyKind kind = mem == PDQP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int i = 0; i < 5; ++i) {
      check_space(dst[i], mem, "normalisation vector");
      if (dst[i]) WCK(cudaMemcpyAsync(dst[i], src[i], (size_t)w->F * sizeof(float), kind, s));
    }
    WCK(cudaStreamSynchronize(s));
  });
}

pdqp_status pdqp_ws_fit(pdqp_ws_handle w, const double* C, const double* B, const double* X, const double* Y,
                        int64_t count, int32_t mem, void* stream) {
  if (!w) return PDQP_ERR_INVALID;
  return guard(w, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (count < 1) throw WsFail{PDQP_ERR_INVALID, "count >= 1"};
    need_data(w, C, B, X, Y, mem, true);
    const int n = w->n, m = w->m;
    {
      DevView<double> c(C, (size_t)count * n, mem, s), x(X, (size_t)count * n, mem, s);
      k_fit_stats<<<(n + 127) / 128, 128, 0, s>>>(c.p, count, n, w->in_mean, w->in_scale, nullptr);
      k_fit_stats<<<(n + 127) / 128, 128, 0, s>>>(x.p, count, n, w->out_mean, w->out_inv, w->out_std);
      WCK(cudaGetLastError());
      WCK(cudaStreamSynchronize(s));
    }
    if (m > 0) {
      DevView<double> b(B, (size_t)count * m, mem, s), y(Y, (size_t)count * m, mem, s);
      k_fit_stats<<<(m + 127) / 128, 128, 0, s>>>(b.p, count, m, w->in_mean + n, w->in_scale + n, nullptr);
      k_fit_stats<<<(m + 127) / 128, 128, 0, s>>>(y.p, count, m, w->out_mean + n, w->out_inv + n, w->out_std + n);
      WCK(cudaGetLastError());
      WCK(cudaStreamSynchronize(s));
    }
    w->have_norm = true;
  });
}

pdqp_status pdqp_ws_grad(pdqp_ws_handle w, const double* C, const double* B, const double* X, const double* Y,
                         int64_t count, double* loss, int32_t mem, void* stream) {
  if (!w) return PDQP_ERR_INVALID;
  return guard(w, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    need_ready(w);
    if (count < 1 || count > w->maxb) throw WsFail{PDQP_ERR_INVALID, "count in [1, max_batch]"};
    need_data(w, C, B, X, Y, mem, true);
    const int n = w->n, m = w->m;
    DevView<double> c(C, (size_t)count * n, mem, s), b(B, (size_t)count * m, mem, s),
        x(X, (size_t)count * n, mem, s), y(Y, (size_t)count * m, mem, s);
    float* T = walloc<float>(w, (size_t)count * w->Fp);
    try {
      k_prep_target<<<grid_for(count * w->F), 256, 0, s>>>(x.p, y.p, n, m, count, w->out_mean, w->out_inv, T, w->Fp);
      project(w, c.p, b.p, 0, (int)count, w->H[0], s);
      forward(w, (int)count, s);
      WCK(cudaMemsetAsync(w->lossacc, 0, sizeof(double), s));
      backward(w, (int)count, T, 1, 0, 1LL << 62, 0, s);
      finish(w, s);
      double h = 0.0;
      WCK(cudaMemcpy(&h, w->lossacc, sizeof(double), cudaMemcpyDeviceToHost));
      if (loss) *loss = h;
    } catch (...) {
      cudaStreamSynchronize(s);
      wfree(w, T);
      throw;
    }
    wfree(w, T);
  });
}

pdqp_status pdqp_ws_train(pdqp_ws_handle w, const pdqp_ws_train_options* opt, const double* C, const double* B,
                          const double* X, const double* Y, int64_t count, double* losses, int32_t mem,
                          void* stream) {
  if (!w || !opt) return PDQP_ERR_INVALID;
  return guard(w, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    need_ready(w);
    const int batch = opt->batch;
    if (batch < 8 || batch > w->maxb || batch % 8) throw WsFail{PDQP_ERR_INVALID, "batch: multiple of 8 in [8, max_batch]"};
    if (count < batch) throw WsFail{PDQP_ERR_INVALID, "count >= batch"};
    if (opt->epochs < 0 || !(opt->lr > 0.f) || !(opt->beta1 >= 0.f && opt->beta1 < 1.f) ||
        !(opt->beta2 >= 0.f && opt->beta2 < 1.f) || !(opt->eps >= 0.f))
      throw WsFail{PDQP_ERR_INVALID, "options: epochs >= 0, lr > 0, 0 <= beta < 1, eps >= 0"};
    need_data(w, C, B, X, Y, mem, true);
    const int n = w->n, m = w->m, F = w->F, Fp = w->Fp, d = w->d;
    // the training set: H0 = projected normalised inputs (bf16), T = normalised targets (float32)
    if (w->tcount != count) {
      wfree(w, w->H0all);
      wfree(w, w->Tall);
      w->H0all = nullptr;
      w->Tall = nullptr;
      w->tcount = 0;
      w->H0all = walloc<bf16>(w, (size_t)count * d);
      w->Tall = walloc<float>(w, (size_t)count * Fp);
      w->tcount = count;
    }
    {
      DevView<double> c(C, (size_t)count * n, mem, s), b(B, (size_t)count * m, mem, s);
      for (long long r0 = 0; r0 < count; r0 += w->maxb) {
        const int rows = (int)std::min<long long>(w->maxb, count - r0);
        project(w, c.p, b.p, r0, rows, w->H0all + (size_t)r0 * d, s);
      }
      finish(w, s);
    }
    {
      DevView<double> x(X, (size_t)count * n, mem, s), y(Y, (size_t)count * m, mem, s);
      k_prep_target<<<grid_for(count * F), 256, 0, s>>>(x.p, y.p, n, m, count, w->out_mean, w->out_inv, w->Tall, Fp);
      finish(w, s);
    }
    const long long steps = count / batch;
    for (int e = 0; e < opt->epochs; ++e) {
      long long a = 1, sft = 0;
      visit_order(opt->seed, e, count, &a, &sft);
      WCK(cudaMemsetAsync(w->lossacc, 0, sizeof(double), s));
      for (long long st = 0; st < steps; ++st) {
        const long long row0 = st * batch;
        k_gather_rows<<<grid_for((long long)batch * d / 8), 256, 0, s>>>(w->H0all, d, a, sft, count, row0, batch, d,
                                                                         w->H[0], d);
        forward(w, batch, s);
        backward(w, batch, w->Tall, a, sft, count, row0, s);
        adam(w, opt->lr, opt->beta1, opt->beta2, opt->eps, s);
      }
      finish(w, s);
      if (losses) {
        double h = 0.0;
        WCK(cudaMemcpy(&h, w->lossacc, sizeof(double), cudaMemcpyDeviceToHost));
        losses[e] = h / (double)steps;
      }
    }
  });
}

pdqp_status pdqp_ws_infer(pdqp_ws_handle w, const double* C, const double* B, int64_t count, double* X0,
                          double* Y0, int32_t mem, void* stream) {
  if (!w) return PDQP_ERR_INVALID;
  return guard(w, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    need_ready(w);
    if (count < 1) throw WsFail{PDQP_ERR_INVALID, "count >= 1"};
    if (!X0 && !Y0) throw WsFail{PDQP_ERR_INVALID, "both outputs null"};
    need_data(w, C, B, X0, Y0, mem, false);
    const int n = w->n, m = w->m;
    DevView<double> c(C, (size_t)count * n, mem, s), b(B, (size_t)count * m, mem, s);
    double *x0 = X0, *y0 = m > 0 ? Y0 : nullptr;
    double *tx = nullptr, *ty = nullptr;
    if (mem == PDQP_MEM_HOST) {
      if (x0) tx = x0 = walloc<double>(w, (size_t)count * n);
      if (y0) ty = y0 = walloc<double>(w, (size_t)count * m);
    }
    try {
      for (long long r0 = 0; r0 < count; r0 += w->maxb) {
        const int rows = (int)std::min<long long>(w->maxb, count - r0);
        project(w, c.p, b.p, r0, rows, w->H[0], s);
        forward(w, rows, s);
        k_write_pred<<<grid_for((long long)rows * w->F), 256, 0, s>>>(w->O, w->Fp, rows, n, m, w->out_mean,
                                                                      w->out_std, r0, x0, y0);
      }
      finish(w, s);
      if (tx) WCK(cudaMemcpy(X0, tx, (size_t)count * n * sizeof(double), cudaMemcpyDeviceToHost));
      if (ty) WCK(cudaMemcpy(Y0, ty, (size_t)count * m * sizeof(double), cudaMemcpyDeviceToHost));
    } catch (...) {
      cudaStreamSynchronize(s);
      wfree(w, tx);
      wfree(w, ty);
      throw;
    }
    wfree(w, tx);
    wfree(w, ty);
  });
}

// Raw GEMM.  The error flag of its bounded waits lives in device memory of the
// library (no allocation per call); pdqp_gemm_bf16_check reads and clears it.
static __device__ int g_gemm_err;

static int* gemm_err_ptr() {
  static int* p = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* q = nullptr;
    if (cudaGetSymbolAddress(&q, g_gemm_err) == cudaSuccess) p = (int*)q;
  });
  return p;
}

pdqp_status pdqp_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B, int32_t ldb,
                           const float* bias, int32_t relu, const void* mask, int32_t ldm, float* D_f32, void* D_bf16,
                           int32_t ldd, int32_t splits, float* workspace, int64_t workspace_bytes, void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || (!D_f32 && !D_bf16) || lda < K || ldb < K || ldd < N || splits < 0)
    return PDQP_ERR_INVALID;
  if ((lda % 8) || (ldb % 8) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return PDQP_ERR_INVALID;
  if (mask && ldm < N) return PDQP_ERR_INVALID;
  for (const void* p : {A, B, (const void*)bias, mask, (const void*)D_f32, (const void*)D_bf16, (const void*)workspace})
    if (p && !is_device_ptr(p)) return PDQP_ERR_INVALID;
  const int sp = plan_splits(M, N, K, splits);
  if (splits > 0 && sp > 1 && (!workspace || (size_t)workspace_bytes < (size_t)sp * M * N * sizeof(float)))
    return PDQP_ERR_INVALID;
  int* err = gemm_err_ptr();
  if (!err) return PDQP_ERR_CUDA;
  Epi e;
  e.out_f = D_f32;
  e.out_b = (bf16*)D_bf16;
  e.bias = bias;
  e.mask = (const bf16*)mask;
  e.ldo = ldd;
  e.ldm = ldm;
  e.relu = relu;
  const size_t wf = workspace ? (size_t)workspace_bytes / sizeof(float) : 0;
  if (gemm_tn((const bf16*)A, lda, (const bf16*)B, ldb, M, N, K, e, splits, workspace, wf, err,
              (cudaStream_t)stream) != cudaSuccess)
    return PDQP_ERR_CUDA;
  return PDQP_OK;
}

pdqp_status pdqp_gemm_bf16_check(void* stream) {
  int* err = gemm_err_ptr();
  if (!err) return PDQP_ERR_CUDA;
  int h = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PDQP_ERR_CUDA;
  if (h) {
    cudaMemsetAsync(err, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return PDQP_DEVICE_TIMEOUT;
  }
  return PDQP_OK;
}

pdqp_status pdqp_gemm_bf16_wait_probe(void* stream) {
  int* err = gemm_err_ptr();
  if (!err) return PDQP_ERR_CUDA;
  k_wait_probe<<<1, 32, 0, (cudaStream_t)stream>>>(err);
  if (cudaGetLastError() != cudaSuccess) return PDQP_ERR_CUDA;
  return pdqp_gemm_bf16_check(stream);
}

int32_t pdqp_gemm_bf16_splits(int32_t M, int32_t N, int32_t K, int32_t splits) {
  if (M < 1 || N < 1 || K < 1 || splits < 0) return 0;
  return plan_splits(M, N, K, splits);
}

}  // extern "C"
