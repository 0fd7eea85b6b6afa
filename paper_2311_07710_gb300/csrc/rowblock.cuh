// Row-block helpers shared by the iteration kernels (iteration.cu) and the
// other kernels (kernels.cu): counted launches, block sums, the staging of a
// row block's products in shared memory, the occupancy targets and the
// low-rank row term.
#pragma once

#include "solver.h"

namespace pdqp {

// Launch a kernel and count it.
template <typename... KArgs, typename... Args>
static inline void launch(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                          Args... args) {
  if (grid <= 0) return;
  kern<<<grid, block, smem, s>>>(args...);
  count_launch();
}
template <typename... KArgs, typename... Args>
static inline void launch(void (*kern)(KArgs...), dim3 grid, int block, size_t smem, cudaStream_t s, Args... args) {
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
  kern<<<grid, block, smem, s>>>(args...);
  count_launch();
}

static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Deterministic sum over the block (valid in every thread).
template <typename T>
__device__ __forceinline__ T block_sum(T v) {
  __shared__ T sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  T t = lane < (int)(blockDim.x >> 5) ? sh[lane] : T(0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// ==========================================================================
// Row-block staging: the products val[e] * vec[col[e]] of one block's
// nonzeros go to shared memory prod[0..ne); srp[t] = rp[r0+t] - e0.
// ==========================================================================
// How the staging gathers the vector: through the read-only path (GATHER_LDG),
// through L2 (GATHER_CG: vectors that other CTAs of the same launch write), or
// with plain loads of a generic pointer (GATHER_PLAIN: a copy in shared memory).
enum { GATHER_LDG = 0, GATHER_CG = 1, GATHER_PLAIN = 2 };

template <int GM, typename X>
__device__ __forceinline__ X gather_load(const X* p) {
  if constexpr (GM == GATHER_LDG) return __ldg(p);
  else if constexpr (GM == GATHER_CG) return __ldcg(p);
  else return *p;
}

// Four consecutive entries of an index or value array by one 16-byte load
// (p 16-byte aligned).
__device__ __forceinline__ void load4(const int* __restrict__ p, int (&v)[4]) {
  const int4 q = __ldg(reinterpret_cast<const int4*>(p));
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const float* __restrict__ p, float (&v)[4]) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* __restrict__ p, double (&v)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// The block's index and value streams are read as aligned quads (16-byte
// loads: a quarter of the load requests of element loads, the requests the
// gathers compete with); quad q holds entries a0 + 4q .. a0 + 4q + 3 with
// a0 = e0 rounded down to a multiple of 4 (the arrays carry 8 entries of
// padding, so the last quad stays inside them), and only the block's own
// entries are gathered and staged.  The staged products and their order are
// those of element-wise staging.
// cmin: entries whose column is below it are staged as 0 without their gather
// (a caller that needs only the sums over the columns >= cmin).
// SC: the gathered entries of the columns below csplit are multiplied by sc
// first (a vector kept unnormalised, normalised where it is read).
template <int NT, int GM = GATHER_LDG, typename V, typename X, bool SC = false>
__device__ __forceinline__ void stage_products(const BCsr<V>& M, const X* __restrict__ vec, int e0, int ne,
                                               int r0, int nr, V* prod, int* srp, int cmin = 0, V sc = V(1),
                                               int csplit = 0) {
  // float data: one quad (four gathers) per phase, so that 256 threads fit 32
  // registers and 8 blocks an SM; float64 data (4 blocks per SM either way)
  // keeps two quads' gathers in flight at once
  constexpr int QPT = BNNZ / NT / 4 + 1;           // quads per thread, one more for the misalignment
  constexpr int QPP = sizeof(V) == 4 ? 1 : 2;      // quads per phase
  const int tid = threadIdx.x;
  const int a0 = e0 & ~3, o = e0 - a0;
  const int nq = (o + ne + 3) >> 2;
  // matrices of small instances (M.pf): the block's index and value quads
  // towards L2 at once (a bulk prefetch, a hint with no completion to wait
  // for), so that the later phases' loads find them there instead of waiting
  // for DRAM behind the earlier phases' gathers; both ranges start on a quad
  // (16 bytes) and span whole quads
  if (M.pf && tid == 0 && nq > 0) {
    const unsigned long long gc = (unsigned long long)__cvta_generic_to_global(M.col + a0);
    const unsigned long long gv = (unsigned long long)__cvta_generic_to_global(M.val + a0);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gc), "r"(nq * 16) : "memory");
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gv), "r"(nq * 4 * (int)sizeof(V)) : "memory");
  }
  for (int t = tid; t <= nr; t += NT) srp[t] = M.rp[r0 + t] - e0;
#pragma unroll
  for (int h = 0; h < QPT; h += QPP) {
    int ci[QPP][4];
    V vv[QPP][4];
#pragma unroll
    for (int k = 0; k < QPP; ++k) {
      const int q = tid + (h + k) * NT;
      if (h + k < QPT && q < nq) {
        load4(M.col + a0 + 4 * q, ci[k]);
        load4(M.val + a0 + 4 * q, vv[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < QPP; ++k) {
      const int q = tid + (h + k) * NT;
      if (h + k < QPT && q < nq) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int e = 4 * q + i - o;   // the entry's place in the block
          if constexpr (SC) {
            if (e >= 0 && e < ne) {
              const int c = ci[k][i];
              V p = V(0);
              if (c >= cmin) {
                const V x = (V)gather_load<GM>(vec + c);
                p = vv[k][i] * (c < csplit ? r_mul(x, sc) : x);
              }
              prod[e] = p;
            }
          } else {
            if (e >= 0 && e < ne) prod[e] = ci[k][i] >= cmin ? vv[k][i] * (V)gather_load<GM>(vec + ci[k][i]) : V(0);
          }
        }
      }
    }
  }
}

// The index and value quads of row block b towards L2 (a bulk prefetch, a
// hint; blocks of one long row are skipped): one thread.  The range starts on a
// quad and spans whole quads, inside the arrays' 8 entries of padding.
template <typename V>
__device__ __forceinline__ void prefetch_rowblock(const BCsr<V>& M, int b) {
  const int e0 = M.rp[M.blk[b]], e1 = M.rp[M.blk[b + 1]];
  if (e1 <= e0 || e1 - e0 > BNNZ) return;
  const int a0 = e0 & ~3, nq = (e1 - a0 + 3) >> 2;
  const unsigned long long gc = (unsigned long long)__cvta_generic_to_global(M.col + a0);
  const unsigned long long gv = (unsigned long long)__cvta_generic_to_global(M.val + a0);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gc), "r"(nq * 16) : "memory");
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gv), "r"(nq * 4 * (int)sizeof(V)) : "memory");
}

// Matrices of small instances (M.pf): thread 0 of the CUDA block at position q
// of a launch also prefetches the row block that the CUDA block one wave later
// (q + PF_AHEAD: 8 resident blocks on each of 152 SMs) will stage, so that its
// first phase, too, finds its quads in L2.
constexpr int PF_AHEAD = 1216;
template <typename V>
__device__ __forceinline__ void prefetch_ahead(const BCsr<V>& M, const int* act, int q, int grid) {
  const int q2 = q + PF_AHEAD;
  if (!M.pf || threadIdx.x != 0 || q2 >= grid) return;
  const int b2 = act ? act[q2] : q2;
  if (b2 >= 0) prefetch_rowblock(M, b2);
}

// Occupancy target of the row-block kernels (blocks per SM).  They wait on
// dependent gathers, so more resident warps hide more latency: with the
// two-phase staging above, 256 threads of float data fit 32 registers without
// spills (8 blocks, the whole SM: k_primal 97 -> 76 us, k_dual 67 -> 51 us at
// n=1e6 against 4 blocks at 64 registers); the float64 kernels are bound by
// the float64 pipes and gain nothing from 5 or 6 blocks, so they keep 64
// registers (4); NT = 512 runs 4 blocks at 32 registers.
template <typename V, int NT, bool LR = false> struct MinBlocks { static constexpr int value = 4; };
template <> struct MinBlocks<float, 256, false> { static constexpr int value = 8; };


// the row term F~_j . w (16-byte loads of the row when r allows)
template <typename FV, typename V, typename W>
__device__ __forceinline__ V lr_row(const FV* __restrict__ F, const W* __restrict__ w, int r, int j) {
  V s = V(0);
  const FV* f = F + (size_t)j * r;
  constexpr int VW = 16 / sizeof(FV);
  if (r % VW == 0) {
    for (int kk = 0; kk < r; kk += VW) {
      if constexpr (VW == 4) {
        const float4 q = *reinterpret_cast<const float4*>(f + kk);
        s += (V)q.x * (V)w[kk] + (V)q.y * (V)w[kk + 1] + (V)q.z * (V)w[kk + 2] + (V)q.w * (V)w[kk + 3];
      } else {
        const double2 q = *reinterpret_cast<const double2*>(f + kk);
        s += (V)q.x * (V)w[kk] + (V)q.y * (V)w[kk + 1];
      }
    }
  } else {
    for (int kk = 0; kk < r; ++kk) s += (V)f[kk] * (V)w[kk];
  }
  return s;
}

// member-major [count][L] (member stride `stride`) <-> interleaved [L][ld],
// through 32 x 32 shared-memory tiles
template <typename V>
__global__ void __launch_bounds__(256) k_to_il(const V* __restrict__ src, long long stride, int L, int count,
                                               V* __restrict__ dst, int ld) {
  __shared__ V t[32][33];
  const int j0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int mem = m0 + k, jj = j0 + threadIdx.x;
    if (mem < count && jj < L) t[k][threadIdx.x] = src[(size_t)mem * stride + jj];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int jj = j0 + k, mem = m0 + threadIdx.x;
    if (jj < L && mem < count) dst[(size_t)jj * ld + mem] = t[threadIdx.x][k];
  }
}
template <typename V>
__global__ void __launch_bounds__(256) k_from_il(const V* __restrict__ src, int ld, int L, int count,
                                                 V* __restrict__ dst, long long stride) {
  __shared__ V t[32][33];
  const int j0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int jj = j0 + k, mem = m0 + threadIdx.x;
    if (jj < L && mem < count) t[k][threadIdx.x] = src[(size_t)jj * ld + mem];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int mem = m0 + k, jj = j0 + threadIdx.x;
    if (mem < count && jj < L) dst[(size_t)mem * stride + jj] = t[threadIdx.x][k];
  }
}

// the transposes take a 2-D block of 32 x 8 threads
template <typename V>
static void to_il(const V* src, long long stride, int L, int count, V* dst, int ld, cudaStream_t s) {
  if (L <= 0 || !src) return;
  k_to_il<V><<<dim3(cdiv(L, 32), cdiv(count, 32)), dim3(32, 8), 0, s>>>(src, stride, L, count, dst, ld);
  count_launch();
}
template <typename V>
static void from_il(const V* src, int ld, int L, int count, V* dst, long long stride, cudaStream_t s) {
  if (L <= 0) return;
  k_from_il<V><<<dim3(cdiv(L, 32), cdiv(count, 32)), dim3(32, 8), 0, s>>>(src, ld, L, count, dst, stride);
  count_launch();
}

template <typename V> static const V* lr_factor(Work& w);
template <> inline const double* lr_factor<double>(Work& w) { return w.Fd; }
template <> inline const float* lr_factor<float>(Work& w) { return w.Fs; }
template <typename V> static const V* lr_weights(Work& w);
template <> inline const double* lr_weights<double>(Work& w) { return w.wlr; }
template <> inline const float* lr_weights<float>(Work& w) { return w.wlr_f; }

// F~' v into w.wlr / w.wlr_f for one vector (kernels.cu)
void lowrank_ft1(Work& w, const float* F, const float* v, cudaStream_t s);
void lowrank_ft1(Work& w, const double* F, const double* v, cudaStream_t s);

}  // namespace pdqp
