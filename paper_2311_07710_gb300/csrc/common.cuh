// Shared device-side definitions of the rAPDHG kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define PDQP_MAX_CHECK 4096   // longest check period (length of the step table)
#define PDQP_RED_BLOCKS 304   // partial-sum blocks of the reductions (2 x 152 SMs)

enum { ST_RUNNING = 0, ST_OPTIMAL = 1, ST_ITER_LIMIT = 2, ST_NUMERICAL = 3 };

// Step scalars of one inner iteration, written by the decision kernel for the
// next chunk of `check_period` iterations (Algorithm 1 with Theorem 1's beta,
// theta and the Section 6 step size).
struct StepEntry {
  double tau_p;          // primal step (eta/omega, or Theorem 1's eta_k)
  double sigma_d;        // dual step (eta*omega, or Theorem 1's tau_k)
  double inv_beta;       // 1/beta_k: weight of the new iterate in the averages
  double inv_beta_next;  // 1/beta_{k+1}: forms x_md of the next iteration
  double theta_next;     // theta_{k+1}: forms the extrapolated point of the next iteration
  float tau_p_f, sigma_d_f, inv_beta_f, inv_beta_next_f, theta_next_f;
};

// Scalar solver state, resident in device memory so that the iteration runs
// without host round trips.
struct DevState {
  double omega;          // primal weight
  double eta_last;       // eta of the last tabulated iteration
  double anchor_kkt;     // relKKT(z^{n,0})
  double prev_cand_kkt;  // candidate relKKT of the previous check in this epoch
  double normA, normQ;
  long long k_epoch;     // inner iteration counter k of the current epoch
  long long k_total;     // total iterations
  long long restarts;
  int status;            // ST_*
  int has_prev;          // prev_cand_kkt is valid
  int restart;           // the last check restarted
  int cand_avg;          // the candidate of the last check is the average
  int out_avg;           // the returned iterate is the average
  int pad0;
  double parts[2][6];    // r_primal, r_dual, r_gap, rel_kkt, primal_obj, dual_obj (cur, avg)
  double out_parts[6];
  double bnorm_inf, cnorm_inf;   // ||b||_inf, ||c||_inf of the original data
  // power iteration
  double pi_lam[2], pi_lam_prev[2], pi_inv_norm[2];
  double pi_hi_prev[2];  // bracket [pi_lam_prev, pi_hi_prev] of the previous Ritz value
  int pi_done[2];
  int pi_iters;
  int pad1;
};

// Layout of one instance inside a block-diagonal batch.
struct Inst {
  int n, m, m_eq;        // sizes
  int xoff, yoff;        // first variable / row of the instance
  int bP0, bP1;          // row blocks of P
  int bA0, bA1;          // row blocks of A
  int cP0, cA0;          // first chunk of KKT_CHUNK row blocks (P, A)
};

constexpr int KKT_CHUNK = 32;   // row blocks per chunk of the relKKT partial sums
inline __host__ __device__ int kkt_chunks(int b0, int b1) { return (b1 - b0 + KKT_CHUNK - 1) / KKT_CHUNK; }

// Batch-wide counters read by the host between chunks.
struct BatchState {
  int running;           // instances still iterating
  int lz_running;        // instances whose norm estimates are still running
  int act_A, act_P;      // batches: row blocks of A / P of the running instances (lists in Work)
  double run_n, run_m, run_nnzA, run_nnzP;   // sizes summed over the running instances
};

// Constant parameters of one solve.
struct SolveParams {
  int step_rule, restart_rule, accelerate, fixed_K, check_period, mixed;
  long long max_iter;
  double eps, beta_suff, beta_nec, beta_art, pw_theta, eps_zero, norm_tol;
  int norm_iters;
  int spmv_threads;     // threads per row block of the iteration kernels (256 or 512)
};

// Device view of one CSR matrix.
template <typename V>
struct Csr {
  const int* __restrict__ rp;
  const int* __restrict__ col;
  const V* __restrict__ val;
};

// Sum over an aligned group of L lanes (L a power of two <= 32); every lane
// of the warp executes it.
template <int L, typename T>
__device__ __forceinline__ T group_sum(T s) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, L);
  return s;
}

// NaN-propagating max.
// Max of two non-negative doubles (NaN-propagating for NaNs with a clear sign
// bit, as fabs leaves them): for such values the order of the bit patterns as
// signed 64-bit integers is the order of the doubles, +inf < NaN, so the max
// runs on the integer pipes instead of the (slow) float64 ones.
__device__ __forceinline__ double nmax(double a, double b) {
  return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}

// float -> double built from the IEEE bit fields with integer instructions
// (the conversion instruction issues on GB300's slow float64 pipe): exponent
// rebiased by 1023 - 127, fraction moved up 29 bits; a subnormal normalised at
// its leading one; zeros, infinities and NaNs keep their class.  The same
// value as the conversion for every float (NaN payloads aside).
__device__ __forceinline__ double f2d(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  unsigned long long b = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 255u) {
    b |= (0x7FFULL << 52) | ((unsigned long long)m << 29);
  } else if (e != 0u) {
    b |= ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (m != 0u) {
    const int p = 31 - __clz(m);                  // leading one of the subnormal fraction
    b |= ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xFFFFFFFFFFFFFULL);
  }
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double f2d(double x) { return x; }

// Block reduction of NF per-thread fields through shared-memory scratch `sh`
// (NF * NT doubles; it may alias data the block no longer reads).  Field f is
// a max (bit f of MAXMASK) or a sum, fixed at compile time, so that a max
// field costs no float64 instruction (GB300's float64 pipes retire about two
// lanes per clock per SM).  Stage 1: warp w folds fields w, w + NT/32, ...:
// each lane combines the NT/32 values of its column in a fixed order.  Stage
// 2: four lanes per field, eight of its 32 column values each in a fixed
// order, then two shuffle levels.  The result is valid in thread 0.
template <int NF, int NT, unsigned MAXMASK>
__device__ __forceinline__ void block_reduce_smem(double (&v)[NF], double* sh) {
  static_assert(NT % 32 == 0 && 4 * NF <= NT, "block_reduce_smem: NT must be a multiple of 32, >= 4 NF");
  constexpr int NW = NT / 32;
  constexpr int NW2 = (4 * NF + 31) / 32;          // warps of stage 2
  __syncthreads();
#pragma unroll
  for (int f = 0; f < NF; ++f) sh[f * NT + threadIdx.x] = v[f];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if (f % NW == w) {                             // warp-uniform; the operation is known here
      constexpr unsigned one = 1u;
      const bool mx = (MAXMASK >> f) & one;
      double t = sh[f * NT + lane];
#pragma unroll
      for (int k = 1; k < NW; ++k) {
        const double x = sh[f * NT + lane + 32 * k];
        t = mx ? nmax(t, x) : t + x;
      }
      sh[f * NT + lane] = t;                       // the column's total (this warp owns field f)
    }
  }
  __syncthreads();
  if (w < NW2) {                                   // whole warps: every lane reaches the shuffles
    const int g = threadIdx.x >> 2, q = threadIdx.x & 3;
    const bool on = g < NF;
    const bool mx = on && ((MAXMASK >> g) & 1u);
    double t = on ? sh[g * NT + 8 * q] : 0.0;
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      const double x = on ? sh[g * NT + 8 * q + k] : 0.0;
      t = mx ? nmax(t, x) : t + x;
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      const double x = __shfl_xor_sync(0xffffffffu, t, o);
      t = mx ? nmax(t, x) : t + x;
    }
    __syncwarp();
    if (on && q == 0) sh[g * NT] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int f = 0; f < NF; ++f) v[f] = sh[f * NT];
  }
}

// Block reduction of NF fields (sum or NaN-propagating max per field); the
// result is valid in thread 0.  blockDim.x must be a multiple of 32, <= 1024.
template <int NF>
__device__ __forceinline__ void block_reduce(double (&v)[NF], const bool (&is_max)[NF]) {
  __shared__ double sh[32][NF];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double t = __shfl_xor_sync(0xffffffffu, v[f], o);
      v[f] = is_max[f] ? nmax(v[f], t) : v[f] + t;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int f = 0; f < NF; ++f) sh[w][f] = v[f];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      double t = lane < nw ? sh[lane][f] : (is_max[f] ? 0.0 : 0.0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double s = __shfl_xor_sync(0xffffffffu, t, o);
        t = is_max[f] ? nmax(t, s) : t + s;
      }
      v[f] = t;
    }
  }
  __syncthreads();
}

// Explicitly rounded arithmetic: kernels that must produce the same bits for
// the same row (the row updates of every iteration-kernel variant, the relKKT
// row terms of the row-block and the member-interleaved checks) compute with
// these, so that every operation's rounding is fixed in the source (no fused
// multiply-add left to the compiler's choice at each inlined call site).
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

