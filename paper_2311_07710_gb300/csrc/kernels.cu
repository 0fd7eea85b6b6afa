// Device kernels of the rAPDHG solver (sm_103a) other than the iteration
// kernels (iteration.cu): scaling, spectral norms, the relative KKT error of
// Section 5 in float64 for the current and the averaged iterate (k_kkt_m /
// k_kkt_n, every `check_period` iterations), the Section 6 restart rule and
// step table (k_decide), restarts (k_restart_apply), mixed-precision rebasing,
// the low-rank term and the allocation-free KKT entry point.
//
// All SpMV-shaped kernels work on row blocks (see BCsr): the block's nonzeros
// are contiguous, so its 256 threads issue their index and value loads
// together (coalesced, 8 per thread; in two phases of 4 for float data), then
// the independent gathers, stage the products in shared memory, and finish
// one row per thread -- a row's update reads and writes consecutive entries
// of the row-indexed vectors.
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "rowblock.cuh"

namespace pdqp {

std::atomic<long long> g_launches{0};
thread_local bool t_capturing = false;
thread_local long long t_captured = 0;

static int pick_lanes(long long nnz, long long rows) {
  const double avg = rows > 0 ? (double)nnz / (double)rows : 0.0;
  int L = 2;
  while (L < 32 && L < avg) L <<= 1;
  return L;
}

#define DISPATCH_L(L, ...)                                  \
  switch (L) {                                              \
    case 2: { constexpr int LL = 2; __VA_ARGS__; } break;   \
    case 4: { constexpr int LL = 4; __VA_ARGS__; } break;   \
    case 8: { constexpr int LL = 8; __VA_ARGS__; } break;   \
    case 16: { constexpr int LL = 16; __VA_ARGS__; } break; \
    default: { constexpr int LL = 32; __VA_ARGS__; } break; \
  }

// --------------------------------------------------------------------------
// Per-row relative KKT kernels on separate Q, A, A' CSR arrays (used by
// pdqp_kkt_noalloc, which takes caller-owned arrays).
// Relative KKT error (Section 5 "Progress metric", equality/bound form) in
// float64, for NIT iterates at once, measured on the original problem:
// (Ax)_i = (A~ x~)_i / D1_i, (Qx)_j = (Q~ x~)_j / D2_j, (A'y)_j = (A~' y~)_j / D2_j.
// Partial sums go to part[block][field]; k_kkt_finish_noalloc finishes them.
// --------------------------------------------------------------------------
struct KktArgs {
  Csr<double> A, Q, At;                 // scaled (or original with D = null)
  const double* x[2];                   // float64 iterates (scaled space)
  const double* y[2];
  const float* dx[2];                   // mixed mode: iterate = base + delta
  const float* dy[2];
  const double* xhi;
  const double* yhi;
  const double* ax;                     // anchors (scaled); null: delta from base (mixed)
  const double* ay;
  const double* D1;                     // null = 1
  const double* D2;
  const double *b, *c, *l, *u;          // original data
  double* prodAx[2];                    // optional: store A~x~ etc. (mixed-mode correction)
  double* prodQx[2];
  double* prodATy[2];
  double* part;
  int n, m, m_eq;
};

template <bool MIXED>
__device__ __forceinline__ double it_x(const KktArgs& a, int it, int k) {
  if (MIXED) return a.xhi[k] + (double)a.dx[it][k];
  return a.x[it][k];
}
template <bool MIXED>
__device__ __forceinline__ double it_y(const KktArgs& a, int it, int k) {
  if (MIXED) return a.yhi[k] + (double)a.dy[it][k];
  return a.y[it][k];
}

template <int L, int NIT, bool MIXED>
__global__ void __launch_bounds__(256) k_kkt_m(KktArgs a) {
  // fields: it*4 + {0 max|viol|, 1 max|Ax|, 2 b'y, 3 |dy|^2}, 8: max|b|
  double f[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int rpb = 256 / L, lane = threadIdx.x % L;
  for (int base = blockIdx.x * rpb; base < a.m; base += gridDim.x * rpb) {
    const int row = base + threadIdx.x / L;
    const bool valid = row < a.m;
    double s[NIT];
#pragma unroll
    for (int it = 0; it < NIT; ++it) s[it] = 0.0;
    if (valid) {
      for (int k = a.A.rp[row] + lane; k < a.A.rp[row + 1]; k += L) {
        const double v = a.A.val[k];
        const int cidx = a.A.col[k];
#pragma unroll
        for (int it = 0; it < NIT; ++it) s[it] = fma(v, it_x<MIXED>(a, it, cidx), s[it]);
      }
    }
#pragma unroll
    for (int it = 0; it < NIT; ++it) s[it] = group_sum<L>(s[it]);
    if (valid && lane == 0) {
      const double d1 = a.D1 ? a.D1[row] : 1.0;
      const double bi = a.b[row];
#pragma unroll
      for (int it = 0; it < NIT; ++it) {
        if (a.prodAx[it]) a.prodAx[it][row] = s[it];
        const double Ax = s[it] / d1;
        const double viol = row < a.m_eq ? fabs(Ax - bi) : fmax(bi - Ax, 0.0);
        f[it * 4 + 0] = nmax(f[it * 4 + 0], viol);
        f[it * 4 + 1] = nmax(f[it * 4 + 1], fabs(Ax));
        const double yt = it_y<MIXED>(a, it, row);
        f[it * 4 + 2] += bi * (d1 * yt);
        const double dy = MIXED ? (double)a.dy[it][row] : (a.ay ? yt - a.ay[row] : 0.0);
        f[it * 4 + 3] += dy * dy;
      }
      f[8] = nmax(f[8], fabs(bi));
    }
  }
  const bool is_max[9] = {true, true, false, false, true, true, false, false, true};
  block_reduce<9>(f, is_max);
  if (threadIdx.x == 0)
    for (int k = 0; k < 9; ++k) a.part[blockIdx.x * 32 + k] = f[k];
}

template <int L, int NIT, bool MIXED>
__global__ void __launch_bounds__(256) k_kkt_n(KktArgs a) {
  // fields (offset 9): it*7 + {0 max|res|, 1 max|Qx|, 2 max|A'y|, 3 x'Qx, 4 c'x,
  // 5 sum(l lam+ - u lam-), 6 |dx|^2}, 14: max|c|
  double f[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) f[k] = 0.0;
  const int rpb = 256 / L, lane = threadIdx.x % L;
  for (int base = blockIdx.x * rpb; base < a.n; base += gridDim.x * rpb) {
    const int row = base + threadIdx.x / L;
    const bool valid = row < a.n;
    double sq[NIT], sa[NIT];
#pragma unroll
    for (int it = 0; it < NIT; ++it) { sq[it] = 0.0; sa[it] = 0.0; }
    if (valid) {
      for (int k = a.Q.rp[row] + lane; k < a.Q.rp[row + 1]; k += L) {
        const double v = a.Q.val[k];
        const int cidx = a.Q.col[k];
#pragma unroll
        for (int it = 0; it < NIT; ++it) sq[it] = fma(v, it_x<MIXED>(a, it, cidx), sq[it]);
      }
      if (a.m > 0)
        for (int k = a.At.rp[row] + lane; k < a.At.rp[row + 1]; k += L) {
          const double v = a.At.val[k];
          const int cidx = a.At.col[k];
#pragma unroll
          for (int it = 0; it < NIT; ++it) sa[it] = fma(v, it_y<MIXED>(a, it, cidx), sa[it]);
        }
    }
#pragma unroll
    for (int it = 0; it < NIT; ++it) { sq[it] = group_sum<L>(sq[it]); sa[it] = group_sum<L>(sa[it]); }
    if (valid && lane == 0) {
      const double d2 = a.D2 ? a.D2[row] : 1.0;
      const double cj = a.c[row], lj = a.l[row], uj = a.u[row];
      const bool lf = isfinite(lj), uf = isfinite(uj);
#pragma unroll
      for (int it = 0; it < NIT; ++it) {
        if (a.prodQx[it]) { a.prodQx[it][row] = sq[it]; a.prodATy[it][row] = sa[it]; }
        const double Qx = sq[it] / d2, ATy = sa[it] / d2;
        const double xt = it_x<MIXED>(a, it, row);
        const double xj = d2 * xt;
        const double g = Qx + cj - ATy;
        const double lam = (lf && uf) ? g : (lf ? fmax(g, 0.0) : (uf ? fmin(g, 0.0) : 0.0));
        double* fi = f + it * 7;
        fi[0] = nmax(fi[0], fabs(g - lam));
        fi[1] = nmax(fi[1], fabs(Qx));
        fi[2] = nmax(fi[2], fabs(ATy));
        fi[3] += xj * Qx;
        fi[4] += cj * xj;
        fi[5] += (lam > 0.0 ? lj * lam : 0.0) - (lam < 0.0 ? uj * (-lam) : 0.0);
        const double dx = MIXED ? (double)a.dx[it][row] : (a.ax ? xt - a.ax[row] : 0.0);
        fi[6] += dx * dx;
      }
      f[14] = nmax(f[14], fabs(cj));
    }
  }
  const bool is_max[15] = {true, true, true, false, false, false, false,
                           true, true, true, false, false, false, false, true};
  block_reduce<15>(f, is_max);
  if (threadIdx.x == 0)
    for (int k = 0; k < 15; ++k) a.part[blockIdx.x * 32 + 9 + k] = f[k];
}

// relKKT parts from the reduced fields of iterate `it`
__device__ void kkt_from_fields(const double* F, int it, double* out) {
  const double maxviol = F[it * 4 + 0], maxAx = F[it * 4 + 1], by = F[it * 4 + 2];
  const double maxb = F[8];
  const double* G = F + 9 + it * 7;
  const double maxres = G[0], maxQx = G[1], maxATy = G[2], xQx = G[3], cx = G[4], bterm = G[5];
  const double maxc = F[23];
  const double rp = maxviol / (1.0 + fmax(maxAx, maxb));
  const double rd = maxres / (1.0 + fmax(fmax(maxQx, maxATy), maxc));
  const double pobj = 0.5 * xQx + cx;
  const double dobj = -0.5 * xQx + by + bterm;
  const double rg = fabs(pobj - dobj) / (1.0 + fmax(fabs(pobj), fabs(dobj)));
  double rel = nmax(nmax(rp, rd), rg);
  if (pobj != pobj || dobj != dobj) rel = pobj - dobj;   // NaN
  out[0] = rp; out[1] = rd; out[2] = rg; out[3] = rel; out[4] = pobj; out[5] = dobj;
}

// reduce the partials of k_kkt_m / k_kkt_n (fields 0..23) in thread 0
__device__ void reduce_kkt_partials(const double* __restrict__ part, int nblk, double* F) {
  double f[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) f[k] = 0.0;
  const bool is_max[24] = {true, true, false, false, true, true, false, false, true,
                           true, true, true, false, false, false, false,
                           true, true, true, false, false, false, false, true};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 24; ++k) f[k] = is_max[k] ? nmax(f[k], part[b * 32 + k]) : f[k] + part[b * 32 + k];
  block_reduce<24>(f, is_max);
  if (threadIdx.x == 0)
    for (int k = 0; k < 24; ++k) F[k] = f[k];
}

// ==========================================================================
// Low-rank term of Q: Q_total = Q + F F' with F (n x r, row-major) applied as
// F (F' v) and never formed.  w = F~' v is a two-stage reduction (row tiles
// then one reduce); the row term F~_j . w is added where Q v appears.
// ==========================================================================

// F~ = D2 F (float64 and float32 copies)
__global__ void k_lr_scale(const float* __restrict__ F, const double* __restrict__ D2, int n, int r,
                           double* __restrict__ Fd, float* __restrict__ Ff) {
  const long long N = (long long)n * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    const double v = D2[e / r] * (double)F[e];
    Fd[e] = v;
    if (Ff) Ff[e] = (float)v;
  }
}

// Partial F~' v for NV vectors v: CUDA block b takes a contiguous range of
// rows; thread (g, k) sums column k over the rows of its range with index =
// g mod G, in the factor's precision (float32 for the
// float32 iteration, float64 for the float64 iteration and the checks);
// part[block][vec][k].
template <typename FV, typename X, int NV>
__global__ void k_lr_ft(const FV* __restrict__ F, int n, int r, const X* __restrict__ v0, const X* __restrict__ v1,
                        double* __restrict__ part) {
  const int G = blockDim.x / r;
  const int g = threadIdx.x / r, kk = threadIdx.x % r;
  FV acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = FV(0);
  if (g < G) {
    // a contiguous range of rows per block; eight rows in flight per thread
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int j0 = blockIdx.x * per, j1 = min(n, j0 + per);
    int j = j0 + g;
    for (; j + 7 * G < j1; j += 8 * G) {
      FV f[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) f[u] = F[(size_t)(j + u * G) * r + kk];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        acc[0] += f[u] * (FV)v0[j + u * G];
        if (NV > 1) acc[NV - 1] += f[u] * (FV)v1[j + u * G];
      }
    }
    for (; j < j1; j += G) {
      const FV f = F[(size_t)j * r + kk];
      acc[0] += f * (FV)v0[j];
      if (NV > 1) acc[NV - 1] += f * (FV)v1[j];
    }
  }
  __shared__ FV sh[2][256];
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  if (threadIdx.x < r) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      FV s = FV(0);
      for (int gg = 0; gg < G; ++gg) s += sh[q][gg * r + threadIdx.x];
      part[((size_t)blockIdx.x * NV + q) * r + threadIdx.x] = (double)s;
    }
  }
}

// w[vec][k] = sum of the block partials: one CUDA block (256 threads) per
// (vec, k), a fixed-order tree; a float32 copy for the float32 iteration
__global__ void __launch_bounds__(256) k_lr_reduce(const double* __restrict__ part, int nparts, int r, int nv,
                                                   double* __restrict__ w, float* __restrict__ wf) {
  const int q = blockIdx.x / r, kk = blockIdx.x % r;
  __shared__ double sh[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += 256) s += part[((size_t)b * nv + q) * r + kk];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w[q * r + kk] = sh[0];
    if (wf) wf[q * r + kk] = (float)sh[0];
  }
}

// --------------------------------------------------------------------------
// Relative KKT error (Section 5 "Progress metric", equality/bound form) in
// float64 for NIT iterates, on the original problem:
// (Ax)_i = (A~x~)_i / D1_i, (Qx)_j = (Q~x~)_j / D2_j, (A'y)_j = (A~'y~)_j / D2_j.
// Block partial sums go to part_m[field][block] / part_n[field][block].
// --------------------------------------------------------------------------
struct KktB {
  BCsr<double> A, P;                    // scaled (or original with D = null)
  const double* x[2];                   // iterates (scaled space), x: [n], y: [m]
  const double* y[2];
  const double2* xx;                    // optional: (x[0], x[1]) and (y[0], y[1]) as pairs, so
  const double2* yy;                    //   that one 16-byte gather fetches both (null: x[], y[])
  const double* ax;                     // anchors for the restart distances (null: none)
  const double* ay;
  const double *D1, *D2, *iD1, *iD2;    // null = 1
  const double *b, *c, *l, *u;          // original data
  double* prodAx[2];                    // optional: A~x~, Q~x~, A~'y~ per iterate
  double* prodQx[2];
  double* prodATy[2];
  double* part_m;                       // [9][ngrp_m] one partial per relKKT group
  double* part_n;                       // [15][ngrp_n]
  int ngrp_m, ngrp_n;
  int n, m;
  const unsigned char* ineq;            // per row of A: inequality
  const Inst* inst;
  const int *grp_inst_A, *grp_first_A;  // relKKT groups (KKT_GROUP row blocks of one instance)
  const int *grp_inst_P, *grp_first_P;
  const DevState* st;                   // null: no status test
  const double* F;                      // low-rank factor F~ (null: none)
  const double* wlr;                    // [2][r]: F~' x per iterate
  int r;
};

// The row blocks [b0, b1) of relKKT group g and its instance: groups are
// KKT_GROUP consecutive row blocks from the instance's first (of P: side 1,
// of A: side 0), so a batch and a standalone solve form the same groups.
struct KktGroup { int inst, b0, b1; };
__device__ __forceinline__ KktGroup kkt_group(const KktB& a, int side, int g) {
  KktGroup r;
  r.inst = side ? a.grp_inst_P[g] : a.grp_inst_A[g];
  const Inst in = a.inst[r.inst];
  const int first = side ? a.grp_first_P[r.inst] : a.grp_first_A[r.inst];
  const int bb = side ? in.bP0 : in.bA0, be = side ? in.bP1 : in.bA1;
  r.b0 = bb + (g - first) * KKT_GROUP;
  r.b1 = min(r.b0 + KKT_GROUP, be);
  return r;
}

// Sign and class tests on the bits (integer instructions: GB300's float64
// pipe is the bound of these kernels): v > 0, v < 0, v finite.
__device__ __forceinline__ bool gt0_bits(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool lt0_bits(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool finite_bits(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7FF) != 0x7FF;
}

// Dynamic shared memory of the row-block relKKT kernels: the block's values,
// the gathered vector entries of each iterate, the row pointers (and the
// Q / A' split); the value and entry area is reused for the field reduction.
template <int NIT>
constexpr size_t kkt_smem_bytes() {
  return (size_t)(NIT + 1) * BNNZ * sizeof(double) + (size_t)(2 * BROWS + 1) * sizeof(int);
}

// Stage one row block: sval[e] = val[e0+e], sx[it][e] = the iterate's entry at
// col[e0+e] (gather(it, c)); srp[t] = rp[r0+t] - e0.
template <int NIT, typename G>
__device__ __forceinline__ void kkt_stage(const BCsr<double>& M, int e0, int ne, int r0, int nr, double* sval,
                                          double* sx, int* srp, G gather) {
  const int tid = threadIdx.x;
  int ci[BEPT];
#pragma unroll
  for (int k = 0; k < BEPT; ++k) {
    const int e = tid + k * BNT;
    if (e < ne) { ci[k] = M.col[e0 + e]; sval[e] = M.val[e0 + e]; }
  }
  for (int t = tid; t <= nr; t += BNT) srp[t] = M.rp[r0 + t] - e0;
#pragma unroll
  for (int k = 0; k < BEPT; ++k) {
    const int e = tid + k * BNT;
    if (e < ne)
#pragma unroll
      for (int it = 0; it < NIT; ++it) sx[it * BNNZ + e] = gather(it, ci[k]);
  }
}

// kkt_stage for two iterates from a pair array: one 16-byte gather
// (gather2(c), a double2) fills both iterates' entries of a nonzero.
template <typename G2>
__device__ __forceinline__ void kkt_stage_pairs(const BCsr<double>& M, int e0, int ne, int r0, int nr, double* sval,
                                                double* sx, int* srp, G2 gather2) {
  const int tid = threadIdx.x;
  int ci[BEPT];
#pragma unroll
  for (int k = 0; k < BEPT; ++k) {
    const int e = tid + k * BNT;
    if (e < ne) { ci[k] = M.col[e0 + e]; sval[e] = M.val[e0 + e]; }
  }
  for (int t = tid; t <= nr; t += BNT) srp[t] = M.rp[r0 + t] - e0;
#pragma unroll
  for (int k = 0; k < BEPT; ++k) {
    const int e = tid + k * BNT;
    if (e < ne) {
      const double2 v = gather2(ci[k]);
      sx[e] = v.x;
      sx[BNNZ + e] = v.y;
    }
  }
}

// m side of one row and iterate IT: fields IT*4 + {0 max|viol|, 1 max|Ax|,
// 2 b'y, 3 |dy|^2}, 8: max|b|
// (every operation explicitly rounded: the row-block and the member-interleaved
// checks inline this and must agree bit for bit)
template <int IT>
__device__ __forceinline__ void kkt_m_row(const KktB& a, double (&f)[9], int r, double s) {
  const double bi = a.b[r];
  if (a.prodAx[IT]) a.prodAx[IT][r] = s;
  const double Ax = a.iD1 ? r_mul(s, a.iD1[r]) : s;
  const double v = r_sub(Ax, bi);                 // bi - Ax = -v exactly
  const double viol = a.ineq[r] ? (lt0_bits(v) ? -v : 0.0) : fabs(v);
  f[IT * 4 + 0] = nmax(f[IT * 4 + 0], viol);
  f[IT * 4 + 1] = nmax(f[IT * 4 + 1], fabs(Ax));
  const double yt = a.y[IT][r];
  f[IT * 4 + 2] = r_fma(bi, a.D1 ? r_mul(a.D1[r], yt) : yt, f[IT * 4 + 2]);
  const double dy = a.ay ? r_sub(yt, a.ay[r]) : 0.0;
  f[IT * 4 + 3] = r_fma(dy, dy, f[IT * 4 + 3]);
  if (IT == 0) f[8] = nmax(f[8], fabs(bi));
}

// n side of one row and iterate IT: fields IT*7 + {0 max|res|, 1 max|Qx|,
// 2 max|A'y|, 3 x'Qx, 4 c'x, 5 sum(l lam+ - u lam-), 6 |dx|^2}, 14: max|c|
template <int IT, bool LR>
__device__ __forceinline__ void kkt_n_row(const KktB& a, double (&f)[15], int r, double sq, double sa) {
  const double cj = a.c[r], lj = a.l[r], uj = a.u[r];
  double sqt = sq;
  if constexpr (LR) sqt = r_add(sqt, lr_row<double, double, double>(a.F, a.wlr + IT * a.r, a.r, r));
  if (a.prodQx[IT]) { a.prodQx[IT][r] = sqt; a.prodATy[IT][r] = -sa; }
  const double Qx = a.iD2 ? r_mul(sqt, a.iD2[r]) : sqt, ATy = a.iD2 ? r_mul(-sa, a.iD2[r]) : -sa;
  const double xt = a.x[IT][r];
  const double xj = a.D2 ? r_mul(a.D2[r], xt) : xt;
  const double g = r_sub(r_add(Qx, cj), ATy);
  // lam = proj of g onto Lambda_j: R (both bounds finite), R+ (only l), R- (only u), {0}
  const bool lf = finite_bits(lj), uf = finite_bits(uj);
  const double lam = (lf && uf) ? g : (lf ? (gt0_bits(g) ? g : 0.0) : (uf ? (lt0_bits(g) ? g : 0.0) : 0.0));
  f[IT * 7 + 0] = nmax(f[IT * 7 + 0], fabs(r_sub(g, lam)));
  f[IT * 7 + 1] = nmax(f[IT * 7 + 1], fabs(Qx));
  f[IT * 7 + 2] = nmax(f[IT * 7 + 2], fabs(ATy));
  f[IT * 7 + 3] = r_fma(xj, Qx, f[IT * 7 + 3]);
  f[IT * 7 + 4] = r_fma(cj, xj, f[IT * 7 + 4]);
  // l lam+ - u lam-: lam > 0 only with l finite, lam < 0 only with u finite
  const double bound = gt0_bits(lam) ? lj : (lt0_bits(lam) ? uj : 0.0);
  f[IT * 7 + 5] = r_fma(bound, lam, f[IT * 7 + 5]);
  const double dx = a.ax ? r_sub(xt, a.ax[r]) : 0.0;
  f[IT * 7 + 6] = r_fma(dx, dx, f[IT * 7 + 6]);
  if (IT == 0) f[14] = nmax(f[14], fabs(cj));
}

// The row phase splits into (iterate, row) work items, so that a block of 256
// threads stays busy when it holds fewer than 256 rows; a branch on the
// iterate keeps every field index known at compile time (the fields stay in
// registers).  Row sums by FMA over the staged values and entries.
template <int NIT>
__global__ void __launch_bounds__(BNT) k_kkt_m(KktB a) {
  extern __shared__ __align__(16) double kkt_sm[];
  double* sval = kkt_sm;
  double* sx = kkt_sm + BNNZ;
  int* srp = reinterpret_cast<int*>(kkt_sm + (NIT + 1) * BNNZ);
  double f[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int tid = threadIdx.x;
  const KktGroup G = kkt_group(a, 0, blockIdx.x);
  if (a.st && a.st[G.inst].status != ST_RUNNING) return;
  for (int bk = G.b0; bk < G.b1; ++bk) {   // the group's row blocks, one after another
    if (bk > G.b0) __syncthreads();          // the staging buffers are read up to here
    const int r0 = a.A.blk[bk], r1 = a.A.blk[bk + 1];
    const int nr = r1 - r0;
    const int e0 = a.A.rp[r0];
    const int ne = a.A.rp[r1] - e0;
    if (ne <= BNNZ) {
      if (NIT == 2 && a.xx)
        kkt_stage_pairs(a.A, e0, ne, r0, nr, sval, sx, srp, [&](int c) { return __ldg(a.xx + c); });
      else
        kkt_stage<NIT>(a.A, e0, ne, r0, nr, sval, sx, srp, [&](int it, int c) { return __ldg(a.x[it] + c); });
      __syncthreads();
      for (int q = tid; q < nr * NIT; q += BNT) {
        const int it = q >= nr ? 1 : 0, t = q - it * nr;
        const double* xv = sx + it * BNNZ;
        double s = 0.0;
        for (int e = srp[t]; e < srp[t + 1]; ++e) s = fma(sval[e], xv[e], s);
        if (it == 0) kkt_m_row<0>(a, f, r0 + t, s);
        else kkt_m_row<NIT - 1>(a, f, r0 + t, s);
      }
    } else {
      double s[NIT];
#pragma unroll
      for (int it = 0; it < NIT; ++it) s[it] = 0.0;
      for (int e = e0 + tid; e < e0 + ne; e += BNT) {
        const double v = a.A.val[e];
        const int c = a.A.col[e];
#pragma unroll
        for (int it = 0; it < NIT; ++it) s[it] = fma(v, __ldg(a.x[it] + c), s[it]);
      }
#pragma unroll
      for (int it = 0; it < NIT; ++it) s[it] = block_sum(s[it]);
      if (tid == 0) {
        kkt_m_row<0>(a, f, r0, s[0]);
        if (NIT > 1) kkt_m_row<NIT - 1>(a, f, r0, s[NIT - 1]);
      }
    }
  }
  block_reduce_smem<9, BNT, 0x133u>(f, kkt_sm);
  if (tid == 0)
    for (int k = 0; k < 9; ++k) a.part_m[(size_t)k * a.ngrp_m + blockIdx.x] = f[k];
}

// 80 registers (3 blocks per SM): capped at 64 for 4 blocks it spills and is
// slower (n=1e6 checks 4.67 -> 5.15 ms per solve)
template <int NIT, bool LR>
__global__ void __launch_bounds__(BNT) k_kkt_n(KktB a) {
  extern __shared__ __align__(16) double kkt_sm[];
  double* sval = kkt_sm;
  double* sx = kkt_sm + BNNZ;
  int* srp = reinterpret_cast<int*>(kkt_sm + (NIT + 1) * BNNZ);
  int* ssp = srp + BROWS + 1;
  double f[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) f[k] = 0.0;
  const int tid = threadIdx.x;
  const KktGroup G = kkt_group(a, 1, blockIdx.x);
  if (a.st && a.st[G.inst].status != ST_RUNNING) return;
  const int n = a.n;
  for (int bk = G.b0; bk < G.b1; ++bk) {   // the group's row blocks, one after another
    if (bk > G.b0) __syncthreads();          // the staging buffers are read up to here
    const int r0 = a.P.blk[bk], r1 = a.P.blk[bk + 1];
    const int nr = r1 - r0;
    const int e0 = a.P.rp[r0];
    const int ne = a.P.rp[r1] - e0;
    if (ne <= BNNZ) {
      if (NIT == 2 && a.xx)
        kkt_stage_pairs(a.P, e0, ne, r0, nr, sval, sx, srp,
                        [&](int c) { return c < n ? __ldg(a.xx + c) : __ldg(a.yy + (c - n)); });
      else
        kkt_stage<NIT>(a.P, e0, ne, r0, nr, sval, sx, srp, [&](int it, int c) {
          return c < n ? __ldg(a.x[it] + c) : __ldg(a.y[it] + (c - n));
        });
      for (int t = tid; t < nr; t += BNT) ssp[t] = a.P.split[r0 + t] - e0;
      __syncthreads();
      for (int q = tid; q < nr * NIT; q += BNT) {
        const int it = q >= nr ? 1 : 0, t = q - it * nr;
        const double* xv = sx + it * BNNZ;
        double sq = 0.0, sa = 0.0;
        for (int e = srp[t]; e < ssp[t]; ++e) sq = fma(sval[e], xv[e], sq);
        for (int e = ssp[t]; e < srp[t + 1]; ++e) sa = fma(sval[e], xv[e], sa);
        if (it == 0) kkt_n_row<0, LR>(a, f, r0 + t, sq, sa);
        else kkt_n_row<NIT - 1, LR>(a, f, r0 + t, sq, sa);
      }
    } else {
      const int sp = a.P.split[r0];
      double sq[NIT], sa[NIT];
#pragma unroll
      for (int it = 0; it < NIT; ++it) { sq[it] = 0.0; sa[it] = 0.0; }
      for (int e = e0 + tid; e < e0 + ne; e += BNT) {
        const double v = a.P.val[e];
        const int c = a.P.col[e];
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
          if (e < sp) sq[it] = fma(v, __ldg(a.x[it] + c), sq[it]);
          else sa[it] = fma(v, __ldg(a.y[it] + (c - n)), sa[it]);
        }
      }
#pragma unroll
      for (int it = 0; it < NIT; ++it) { sq[it] = block_sum(sq[it]); sa[it] = block_sum(sa[it]); }
      if (tid == 0) {
        kkt_n_row<0, LR>(a, f, r0, sq[0], sa[0]);
        if (NIT > 1) kkt_n_row<NIT - 1, LR>(a, f, r0, sq[NIT - 1], sa[NIT - 1]);
      }
    }
  }
  block_reduce_smem<15, BNT, 0x4387u>(f, kkt_sm);
  if (tid == 0)
    for (int k = 0; k < 15; ++k) a.part_n[(size_t)k * a.ngrp_n + blockIdx.x] = f[k];
}

// launch both relKKT kernels with their dynamic shared memory
template <int NIT>
static void launch_kkt(const Work& w, const KktB& a, cudaStream_t s) {
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_kkt_m<NIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kkt_smem_bytes<NIT>());
    cudaFuncSetAttribute(k_kkt_n<NIT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kkt_smem_bytes<NIT>());
    cudaFuncSetAttribute(k_kkt_n<NIT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kkt_smem_bytes<NIT>());
  });
  if (w.m > 0) launch(k_kkt_m<NIT>, w.ngrp_A, BNT, kkt_smem_bytes<NIT>(), s, a);
  if (a.F) launch(k_kkt_n<NIT, true>, w.ngrp_P, BNT, kkt_smem_bytes<NIT>(), s, a);
  else launch(k_kkt_n<NIT, false>, w.ngrp_P, BNT, kkt_smem_bytes<NIT>(), s, a);
}

// --------------------------------------------------------------------------
// The check of a family handle (members sharing the matrix) on
// member-interleaved vectors: k_kkt_sums_il forms every member's row sums of
// A x, Q x and A'y for the current and the average iterate with one warp per
// row for 64 members (coalesced 16-byte loads of the gathered entries), each
// sum sequential over the row's entries by FMA as the row-block kernels sum
// their staged values; the sums go back to the member-major layout and
// k_kkt_m_sums / k_kkt_n_sums take them through the row terms and the block
// reduction of k_kkt_m / k_kkt_n, item for item: the partials are bitwise
// those of the row-block check.
// --------------------------------------------------------------------------
struct KktIL {
  const int *rpA, *colA, *rpP, *colP, *splitP;   // one member's A and P (local columns)
  const double *valA, *valP;                     // scaled values
  const double* x[2];                            // interleaved iterates [n x ld], [m x ld]
  const double* y[2];
  double* sA[2];                                 // interleaved row sums: A x [m x ld]
  double* sQ[2];                                 // Q x [n x ld]
  double* sT[2];                                 // A'y [n x ld] (P's -A' part summed)
  int n, m, ld, count;
  const DevState* st;
};

constexpr int KIL_MEM = 64;   // members per warp (two float64 per lane)

__global__ void __launch_bounds__(256, 4) k_kkt_sums_il(KktIL a, int side) {
  __shared__ int run_any;
  const int lane = threadIdx.x & 31, r = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int m0 = blockIdx.y * KIL_MEM + 2 * lane;
  const bool run0 = m0 < a.count && a.st[m0].status == ST_RUNNING;
  const bool run1 = m0 + 1 < a.count && a.st[m0 + 1].status == ST_RUNNING;
  if (threadIdx.x == 0) run_any = 0;
  __syncthreads();
  if (run0 || run1) run_any = 1;
  __syncthreads();
  if (!run_any) return;
  const int rows = side == 0 ? a.m : a.n;
  if (r >= rows) return;    // uniform over the warp: every lane stays for the shuffles
  const size_t ld = (size_t)a.ld;
  const int lane_ = threadIdx.x & 31;
  double s[2][2][2] = {};   // [part: Q or A x / A'y][iterate][member]
  // the row's entries 32 at a time by one coalesced load, handed to every
  // lane by shuffle; each sum sequential over the entries by FMA
  auto accum = [&](const int* __restrict__ col, const double* __restrict__ val, int e0, int e1, int part,
                   const double* const* z, int coff) {
    for (int base = e0; base < e1; base += 32) {
      int cl = 0;
      double vl = 0.0;
      if (base + lane_ < e1) { cl = __ldg(col + base + lane_); vl = __ldg(val + base + lane_); }
      const int cnt = min(32, e1 - base);
      for (int k = 0; k < cnt; ++k) {
        const double v = __shfl_sync(0xffffffffu, vl, k);
        const size_t c = (size_t)(__shfl_sync(0xffffffffu, cl, k) - coff) * ld + m0;
        const double2 z0 = __ldg(reinterpret_cast<const double2*>(z[0] + c));
        const double2 z1 = __ldg(reinterpret_cast<const double2*>(z[1] + c));
        s[part][0][0] = r_fma(v, z0.x, s[part][0][0]);
        s[part][0][1] = r_fma(v, z0.y, s[part][0][1]);
        s[part][1][0] = r_fma(v, z1.x, s[part][1][0]);
        s[part][1][1] = r_fma(v, z1.y, s[part][1][1]);
      }
    }
  };
  const size_t idx = (size_t)r * ld + m0;
  if (side == 0) {
    accum(a.colA, a.valA, a.rpA[r], a.rpA[r + 1], 0, a.x, 0);
    for (int it = 0; it < 2; ++it)
      *reinterpret_cast<double2*>(a.sA[it] + idx) = make_double2(s[0][it][0], s[0][it][1]);
  } else {
    const int sp = a.splitP[r];
    accum(a.colP, a.valP, a.rpP[r], sp, 0, a.x, 0);
    accum(a.colP, a.valP, sp, a.rpP[r + 1], 1, a.y, a.n);
    for (int it = 0; it < 2; ++it) {
      *reinterpret_cast<double2*>(a.sQ[it] + idx) = make_double2(s[0][it][0], s[0][it][1]);
      *reinterpret_cast<double2*>(a.sT[it] + idx) = make_double2(s[1][it][0], s[1][it][1]);
    }
  }
}

// k_kkt_m / k_kkt_n on given row sums (member-major; rows of at most one row block)
__global__ void __launch_bounds__(BNT) k_kkt_m_sums(KktB a, const double* __restrict__ s0,
                                                     const double* __restrict__ s1) {
  __shared__ double sh[9 * BNT];
  double f[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int tid = threadIdx.x;
  const KktGroup G = kkt_group(a, 0, blockIdx.x);
  if (a.st && a.st[G.inst].status != ST_RUNNING) return;
  for (int bk = G.b0; bk < G.b1; ++bk) {
    const int r0 = a.A.blk[bk], nr = a.A.blk[bk + 1] - r0;
    for (int q = tid; q < nr * 2; q += BNT) {
      const int it = q >= nr ? 1 : 0, t = q - it * nr;
      if (it == 0) kkt_m_row<0>(a, f, r0 + t, s0[r0 + t]);
      else kkt_m_row<1>(a, f, r0 + t, s1[r0 + t]);
    }
  }
  block_reduce_smem<9, BNT, 0x133u>(f, sh);
  if (tid == 0)
    for (int k = 0; k < 9; ++k) a.part_m[(size_t)k * a.ngrp_m + blockIdx.x] = f[k];
}

__global__ void __launch_bounds__(BNT) k_kkt_n_sums(KktB a, const double* __restrict__ q0,
                                                     const double* __restrict__ q1, const double* __restrict__ t0,
                                                     const double* __restrict__ t1) {
  __shared__ double sh[15 * BNT];
  double f[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) f[k] = 0.0;
  const int tid = threadIdx.x;
  const KktGroup G = kkt_group(a, 1, blockIdx.x);
  if (a.st && a.st[G.inst].status != ST_RUNNING) return;
  for (int bk = G.b0; bk < G.b1; ++bk) {
    const int r0 = a.P.blk[bk], nr = a.P.blk[bk + 1] - r0;
    for (int q = tid; q < nr * 2; q += BNT) {
      const int it = q >= nr ? 1 : 0, t = q - it * nr;
      if (it == 0) kkt_n_row<0, false>(a, f, r0 + t, q0[r0 + t], t0[r0 + t]);
      else kkt_n_row<1, false>(a, f, r0 + t, q1[r0 + t], t1[r0 + t]);
    }
  }
  block_reduce_smem<15, BNT, 0x4387u>(f, sh);
  if (tid == 0)
    for (int k = 0; k < 15; ++k) a.part_n[(size_t)k * a.ngrp_n + blockIdx.x] = f[k];
}

// the check's relKKT partials of a family handle through the interleaved sums
static void launch_kkt_il(Work& w, const KktB& a, cudaStream_t s) {
  const int n = w.fam_n, m = w.fam_m, cnt = w.fam_count, ld = w.fam_ld;
  double* const* I = w.ilk;
  to_il<double>(a.x[0], n, n, cnt, I[ILK_X0], ld, s);
  to_il<double>(a.x[1], n, n, cnt, I[ILK_X1], ld, s);
  to_il<double>(a.y[0], m, m, cnt, I[ILK_Y0], ld, s);
  to_il<double>(a.y[1], m, m, cnt, I[ILK_Y1], ld, s);
  KktIL k{};
  k.rpA = w.A.rp; k.colA = w.A.col; k.valA = w.A.sval;
  k.rpP = w.P.rp; k.colP = w.famP_col; k.valP = w.P.sval; k.splitP = w.P.split;
  k.x[0] = I[ILK_X0]; k.x[1] = I[ILK_X1]; k.y[0] = I[ILK_Y0]; k.y[1] = I[ILK_Y1];
  k.sA[0] = I[ILK_SA0]; k.sA[1] = I[ILK_SA1];
  k.sQ[0] = I[ILK_SQ0]; k.sQ[1] = I[ILK_SQ1]; k.sT[0] = I[ILK_ST0]; k.sT[1] = I[ILK_ST1];
  k.n = n; k.m = m; k.ld = ld; k.count = cnt; k.st = w.st;
  if (m > 0) launch(k_kkt_sums_il, dim3(cdiv(m, 8), ld / KIL_MEM), 256, 0, s, k, 0);
  launch(k_kkt_sums_il, dim3(cdiv(n, 8), ld / KIL_MEM), 256, 0, s, k, 1);
  double* const* S = w.kks;
  from_il<double>(I[ILK_SA0], ld, m, cnt, S[0], m, s);
  from_il<double>(I[ILK_SA1], ld, m, cnt, S[1], m, s);
  from_il<double>(I[ILK_SQ0], ld, n, cnt, S[2], n, s);
  from_il<double>(I[ILK_SQ1], ld, n, cnt, S[3], n, s);
  from_il<double>(I[ILK_ST0], ld, n, cnt, S[4], n, s);
  from_il<double>(I[ILK_ST1], ld, n, cnt, S[5], n, s);
  if (w.m > 0) launch(k_kkt_m_sums, w.ngrp_A, BNT, 0, s, a, (const double*)S[0], (const double*)S[1]);
  launch(k_kkt_n_sums, w.ngrp_P, BNT, 0, s, a, (const double*)S[2], (const double*)S[3], (const double*)S[4],
         (const double*)S[5]);
}

// reduce the field-major partials of k_kkt_m / k_kkt_n (blocks [bm0, bm1) of
// [nbm] and [bn0, bn1) of [nbn]) into F[0..23] (thread 0)
__device__ void reduce_kkt_blocks(const double* __restrict__ pm, int nbm, int bm0, int bm1,
                                  const double* __restrict__ pn, int nbn, int bn0, int bn1, double* F) {
  double f[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) f[k] = 0.0;
  const bool is_max[24] = {true, true, false, false, true, true, false, false, true,
                           true, true, true, false, false, false, false,
                           true, true, true, false, false, false, false, true};
  for (int b = bm0 + threadIdx.x; b < bm1; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double v = pm[(size_t)k * nbm + b];
      f[k] = is_max[k] ? nmax(f[k], v) : f[k] + v;
    }
  for (int b = bn0 + threadIdx.x; b < bn1; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      const double v = pn[(size_t)k * nbn + b];
      f[9 + k] = is_max[9 + k] ? nmax(f[9 + k], v) : f[9 + k] + v;
    }
  block_reduce<24>(f, is_max);
  if (threadIdx.x == 0)
    for (int k = 0; k < 24; ++k) F[k] = f[k];
}

// --------------------------------------------------------------------------
// Preconditioning (Section 5 "Preprocessing"): norms of the rows of D K D,
// K = [[Q, A'], [A, 0]] -- the rows of P (index j) and of A (index n+i); the
// columns of P already index d = (D2, D1).
// --------------------------------------------------------------------------
// One pass of the scaling (KIND 0: Ruiz, the inf-norm; 1: l2; 2: Pock-Chambolle,
// the l1 norm) over the rows of M: the norm nu_r of row r of D K D =
// d_r * norm_j(|m_rj| d_j) (the column factor per nonzero, the row factor once
// per row) and the row's new factor d_r / sqrt(nu_r) (nu_r = 0: unchanged),
// written to dnew, the other of two buffers (every row of K has one writer and
// the pass reads only d).
template <int KIND>
__global__ void __launch_bounds__(BNT) k_scale_pass(BCsr<double> M, const double* __restrict__ d, int doff,
                                                    int dcol_off, double* __restrict__ dnew) {
  __shared__ double pv[BNNZ];
  __shared__ int srp[BROWS + 1];
  const int tid = threadIdx.x;
  const int r0 = M.blk[blockIdx.x], r1 = M.blk[blockIdx.x + 1];
  const int nr = r1 - r0;
  const int e0 = M.rp[r0];
  const int ne = M.rp[r1] - e0;
  auto take = [&](double acc, double v) {   // v >= 0
    return KIND == 0 ? nmax(acc, v) : (KIND == 1 ? fma(v, v, acc) : acc + v);
  };
  auto update = [&](int r, double acc) {
    const double dr = d[doff + r];
    const double nu = KIND == 1 ? sqrt(acc) * dr : acc * dr;
    dnew[doff + r] = dr / sqrt(nu > 0.0 ? nu : 1.0);
  };
  if (ne <= BNNZ) {
    // m_rj d_j staged from 16-byte loads; |m_rj d_j| = |m_rj| d_j (d > 0;
    // rounding to nearest is symmetric in the sign)
    stage_products<BNT>(M, d + dcol_off, e0, ne, r0, nr, pv, srp);
    __syncthreads();
    for (int t = tid; t < nr; t += BNT) {
      double acc = 0.0;
      if constexpr (KIND == 0) {
        // the largest |m_rj d_j|: non-negative doubles order as their bit
        // patterns (integer instructions, not the float64 pipe)
        unsigned long long best = 0;
        for (int e = srp[t]; e < srp[t + 1]; ++e) {
          const unsigned long long b = (unsigned long long)__double_as_longlong(pv[e]) & 0x7FFFFFFFFFFFFFFFULL;
          best = b > best ? b : best;
        }
        acc = __longlong_as_double((long long)best);
      } else {
        for (int e = srp[t]; e < srp[t + 1]; ++e) acc = take(acc, fabs(pv[e]));
      }
      update(r0 + t, acc);
    }
  } else {
    double acc = 0.0;
    for (int e = e0 + tid; e < e0 + ne; e += BNT) acc = take(acc, fabs(M.val[e]) * d[dcol_off + M.col[e]]);
    if (KIND == 0) {
      __shared__ double sh[BNT];
      sh[tid] = acc;
      __syncthreads();
      for (int o = BNT / 2; o > 0; o >>= 1) {
        if (tid < o) sh[tid] = nmax(sh[tid], sh[tid + o]);
        __syncthreads();
      }
      acc = sh[0];
    } else {
      acc = block_sum(acc);
    }
    if (tid == 0) update(r0, acc);
  }
}

__global__ void k_fill(double* __restrict__ p, double v, long long N) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) p[i] = v;
}

__global__ void k_inverse(const double* __restrict__ d, double* __restrict__ id, int N) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) id[i] = 1.0 / d[i];
}

// Scaled values of a row-blocked matrix: (d_row * v) * d_col, or for the A'
// part of P (entries e >= split) (d_col * v) * d_row, which keeps every entry
// bitwise equal to the corresponding entry (D1 A D2)_ij.
__global__ void __launch_bounds__(BNT) k_scale_vals(BCsr<double> M, const double* __restrict__ d, int doff,
                                                    int dcol_off, double* __restrict__ out,
                                                    float* __restrict__ out_f) {
  __shared__ int srp[BROWS + 1];
  const int tid = threadIdx.x;
  const int r0 = M.blk[blockIdx.x], r1 = M.blk[blockIdx.x + 1];
  const int nr = r1 - r0;
  const int e0 = M.rp[r0];
  const int ne = M.rp[r1] - e0;
  for (int t = tid; t <= nr; t += BNT) srp[t] = M.rp[r0 + t] - e0;
  __syncthreads();
  for (int e = tid; e < ne; e += BNT) {
    // row of element e: the last t with srp[t] <= e
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (srp[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const int r = r0 + lo;
    const double dr = d[doff + r], dcv = d[dcol_off + M.col[e0 + e]], v = M.val[e0 + e];
    const bool tr = M.split && (e0 + e) >= M.split[r];
    const double sv = tr ? (dcv * v) * dr : (dr * v) * dcv;
    out[e0 + e] = sv;
    if (out_f) out_f[e0 + e] = (float)sv;
  }
}

// c~ = D2 c, l~ = l / D2, u~ = u / D2 (n);  b~ = D1 b (m)
__global__ void k_scale_vectors(int n, int m, const double* __restrict__ D1, const double* __restrict__ D2,
                                const double* __restrict__ c, const double* __restrict__ b,
                                const double* __restrict__ l, const double* __restrict__ u,
                                double* __restrict__ cs, double* __restrict__ bs, double* __restrict__ ls,
                                double* __restrict__ us, float* __restrict__ fcs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double d = D2[i];
    cs[i] = d * c[i];
    ls[i] = l[i] / d;
    us[i] = u[i] / d;
  }
  if (i < m) bs[i] = D1[i] * b[i];
}

// --------------------------------------------------------------------------
// Spectral norms ||A~||_2 = sqrt(lambda_max(A~'A~)) and ||Q~||_2 by the Lanczos
// method: the largest Ritz value of the tridiagonal T_k built by the plain
// three-term recurrence from the normalised all-ones vector, for both
// operators at once.  Per step: w = Op v (two SpMV kernels), alpha = v'w,
// r = w - alpha v - beta_prev v_prev, beta = |r|, theta = lambda_max(T_k),
// v_next = r / beta.  Stop when theta changes by <= tol relative, when
// beta <= 1e-12 theta (invariant subspace) or after the step limit.
// --------------------------------------------------------------------------
constexpr int LZ_MAX = 512;

struct LzArgs {
  int n, m, count;
  double* al;                      // [count][2][LZ_MAX] alphas (A'A, Q)
  double* be;                      // [count][2][LZ_MAX] betas
  DevState* st;                    // [count]
  const Inst* inst;                // [count]
  const int* blk_inst_P;           // instance of each P row block
  const int* blk_inst_A;
  const int* row_inst_n;
  int nblkP;
  // 1: the new Lanczos vector is stored as r and normalised where it is read
  // (its readers multiply by pi_inv_norm, k_lz_orth writes v = r / beta back);
  // 0: k_lz_norm normalises it in place (a low-rank term reads it as well)
  int lazy;
  double* cpart;                   // [2][nchunk] chunk sums of the row-block partials
  unsigned* ticket;                // [nchunk] zero between launches
  int nchunk;
  // batches late in the estimates: the row blocks of the instances still
  // estimating (null: every row block); nactP entries of actP
  const int *actA, *actP;
  int nactP;
};

// After row block b of instance i wrote its two partials (part[b],
// part[nblkP + b]; one thread): the last of its chunk's blocks to finish -- a
// ticket taken after a fence -- sums the chunk's partials in block order into
// the chunk sums and resets the ticket.  Chunks are KKT_CHUNK consecutive row
// blocks from the instance's first, so a batch, a family member and a
// standalone solve sum alike, and the per-instance reductions (one CUDA block
// each) read tens of chunk sums instead of thousands of partials.  No waits:
// every block of a chunk runs the kernel to this point or none does (the
// early exits test the instance's state only).
__device__ __forceinline__ void lz_chunk_close(const LzArgs& a, const double* part, int b, int i) {
  const Inst in = a.inst[i];
  const int c = (b - in.bP0) / KKT_CHUNK;
  const int c0 = in.bP0 + c * KKT_CHUNK, c1 = min(c0 + KKT_CHUNK, in.bP1);
  const int g = in.cP0 + c;
  __threadfence();
  if (atomicAdd(a.ticket + g, 1u) != (unsigned)(c1 - c0 - 1)) return;
  __threadfence();
  double s0 = 0.0, s1 = 0.0;
  for (int k = c0; k < c1; ++k) {
    s0 += __ldcg(part + k);
    s1 += __ldcg(part + (size_t)a.nblkP + k);
  }
  a.cpart[g] = s0;
  a.cpart[(size_t)a.nchunk + g] = s1;
  a.ticket[g] = 0u;
}

// the factor that normalises operator o's stored vector (1 when it is stored
// normalised), in the vectors' precision
template <typename V>
__device__ __forceinline__ V lz_scale(const LzArgs& a, const DevState& st, int o) {
  return a.lazy ? (V)st.pi_inv_norm[o] : V(1);
}

__device__ __forceinline__ double* lz_al(const LzArgs& a, int i, int o) { return a.al + ((size_t)i * 2 + o) * LZ_MAX; }
__device__ __forceinline__ double* lz_be(const LzArgs& a, int i, int o) { return a.be + ((size_t)i * 2 + o) * LZ_MAX; }

template <typename V, int NT>
__global__ void __launch_bounds__(NT, MinBlocks<V, NT>::value) k_lz_m(BCsr<V> A, LzArgs la, const V* __restrict__ vA,
                                                                   V* __restrict__ wm) {
  const int bk = la.actA ? la.actA[blockIdx.x] : (int)blockIdx.x;
  const DevState& st = la.st[la.blk_inst_A[bk]];
  if (st.pi_done[0]) return;
  __shared__ V prod[BNNZ];
  __shared__ int srp[BROWS + 1];
  const int tid = threadIdx.x;
  const V gA = lz_scale<V>(la, st, 0);
  const int r0 = A.blk[bk], r1 = A.blk[bk + 1];
  const int nr = r1 - r0;
  const int e0 = A.rp[r0];
  const int ne = A.rp[r1] - e0;
  if (ne <= BNNZ) {
    stage_products<NT, GATHER_LDG, V, V, true>(A, vA, e0, ne, r0, nr, prod, srp, 0, gA, la.n);
    __syncthreads();
    for (int t = tid; t < nr; t += NT) {
      V s = V(0);
      for (int e = srp[t]; e < srp[t + 1]; ++e) s += prod[e];
      wm[r0 + t] = s;
    }
  } else {
    V s = V(0);
    for (int e = e0 + tid; e < e0 + ne; e += NT) s += A.val[e] * r_mul(__ldg(vA + A.col[e]), gA);
    s = block_sum(s);
    if (tid == 0) wm[r0] = s;
  }
}

// rows of P with input [v_Q ; w_m]: wA = A~'w_m, wQ = Q~ v_Q; partial v'w per row block
template <typename V, int NT, bool LR = false>
__global__ void __launch_bounds__(NT, MinBlocks<V, NT, LR>::value) k_lz_n(BCsr<V> P, LzArgs la, const V* __restrict__ zin,
                                                                   const V* __restrict__ vA, V* __restrict__ wA,
                                                                   V* __restrict__ wQ, double* __restrict__ part,
                                                                   const V* __restrict__ F,
                                                                   const V* __restrict__ wlr, int rk) {
  __shared__ __align__(16) V prod[BNNZ];
  __shared__ int srp[BROWS + 1];
  __shared__ int ssp[BROWS];
  const int bk = la.actP ? la.actP[blockIdx.x] : (int)blockIdx.x;
  const DevState& st = la.st[la.blk_inst_P[bk]];
  const bool doA = !st.pi_done[0];
  const bool doQ = !st.pi_done[1];
  if (!doA && !doQ) return;                    // its instance's alpha reduction skips it
  double f[2] = {0.0, 0.0};
  const int tid = threadIdx.x;
  const V gA = lz_scale<V>(la, st, 0), gQ = lz_scale<V>(la, st, 1);   // v_A, v_Q normalisation
  const int r0 = P.blk[bk], r1 = P.blk[bk + 1];
  const int nr = r1 - r0;
  const int e0 = P.rp[r0];
  const int ne = P.rp[r1] - e0;
  auto row = [&](int r, V sQ, V sA) {
    if (doA) { const V u = -sA; wA[r] = u; f[0] = fma(f2d(r_mul(vA[r], gA)), f2d(u), f[0]); }
    if (doQ) {
      if (LR) sQ += lr_row<V, V, V>(F, wlr, rk, r);
      wQ[r] = sQ;
      f[1] = fma(f2d(r_mul(zin[r], gQ)), f2d(sQ), f[1]);
    }
  };
  if (ne <= BNNZ) {
    // once the instance's ||Q|| has converged only the A' part is gathered;
    // the v_Q entries (columns < n) are normalised as they are gathered
    stage_products<NT, GATHER_LDG, V, V, true>(P, zin, e0, ne, r0, nr, prod, srp, doQ ? 0 : la.n, gQ, la.n);
    for (int t = tid; t < nr; t += NT) ssp[t] = P.split[r0 + t] - e0;
    __syncthreads();
    for (int t = tid; t < nr; t += NT) {
      V q = V(0), w = V(0);
      for (int e = srp[t]; e < ssp[t]; ++e) q += prod[e];
      for (int e = ssp[t]; e < srp[t + 1]; ++e) w += prod[e];
      row(r0 + t, q, w);
    }
  } else {
    const int sp = P.split[r0];
    V q = V(0), w = V(0);
    for (int e = e0 + tid; e < e0 + ne; e += NT) {
      const V x = __ldg(zin + P.col[e]);
      const V v = P.val[e] * (e < sp ? r_mul(x, gQ) : x);
      if (e < sp) q += v; else w += v;
    }
    q = block_sum(q);
    w = block_sum(w);
    if (tid == 0) row(r0, q, w);
  }
  static_assert(sizeof(V) * BNNZ >= 2 * NT * sizeof(double), "staging buffer too small for the reduction");
  block_reduce_smem<2, NT, 0u>(f, reinterpret_cast<double*>(prod));
  if (tid == 0) {
    part[bk] = f[0];
    part[(size_t)la.nblkP + bk] = f[1];
    lz_chunk_close(la, part, bk, la.blk_inst_P[bk]);
  }
}

// Per-thread sums of the two fields (part[b], part[stride + b]) over [b0, b1)
// (stride blockDim): four independent accumulators, combined in a fixed order.
__device__ __forceinline__ void lz_block_sums(const double* __restrict__ part, int nblkP, int b0, int b1,
                                              double (&f)[2]) {
  double acc[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
  const int st = blockDim.x;
  int b = b0 + threadIdx.x;
  for (; b + 3 * st < b1; b += 4 * st) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc[0][u] += part[b + u * st];
      acc[1][u] += part[(size_t)nblkP + b + u * st];
    }
  }
  for (int u = 0; b < b1; b += st, ++u) {
    acc[0][u] += part[b];
    acc[1][u] += part[(size_t)nblkP + b];
  }
  f[0] = (acc[0][0] + acc[0][1]) + (acc[0][2] + acc[0][3]);
  f[1] = (acc[1][0] + acc[1][1]) + (acc[1][2] + acc[1][3]);
}

// one CUDA block per instance: alpha_k = sum of its chunk sums
template <int NT>
__global__ void __launch_bounds__(NT) k_lz_alpha(LzArgs a) {
  const int i = blockIdx.x;
  DevState& st = a.st[i];
  if (st.pi_done[0] && st.pi_done[1]) return;
  const Inst in = a.inst[i];
  double f[2] = {0.0, 0.0};
  lz_block_sums(a.cpart, a.nchunk, in.cP0, in.cP0 + kkt_chunks(in.bP0, in.bP1), f);
  const bool is_max[2] = {false, false};
  block_reduce<2>(f, is_max);
  if (threadIdx.x == 0) {
    const int k = st.pi_iters;
    for (int o = 0; o < 2; ++o)
      if (!st.pi_done[o]) lz_al(a, i, o)[k] = f[o];
  }
}

// r = w - alpha v - beta_prev v_prev over v_prev, one warp per P row block (8
// per CTA: the per-block prologue of the instance's scalars runs in parallel);
// partial |r|^2 per row block.  With lazy normalisation v is the stored vector
// times 1/beta of the last step, written back here as the normalised vector
// that the next step's three-term update reads as v_prev.  The update runs in
// the vectors' precision (two FMAs), only |r|^2 in float64.
template <typename V>
__global__ void __launch_bounds__(256) k_lz_orth(LzArgs a, BCsr<V> P, const V* __restrict__ wA,
                                                 const V* __restrict__ wQ, V* __restrict__ vA,
                                                 V* __restrict__ vA_prev, V* __restrict__ vQ,
                                                 V* __restrict__ vQ_prev, double* __restrict__ part) {
  const int q = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (q >= (a.actP ? a.nactP : a.nblkP)) return;   // warp-uniform
  const int b = a.actP ? a.actP[q] : q;
  const int i = a.blk_inst_P[b];
  const DevState& st = a.st[i];
  const bool doA = !st.pi_done[0], doQ = !st.pi_done[1];
  if (!doA && !doQ) return;
  const int k = st.pi_iters;
  const V alA = (V)(doA ? lz_al(a, i, 0)[k] : 0.0), alQ = (V)(doQ ? lz_al(a, i, 1)[k] : 0.0);
  const V bpA = (V)((doA && k > 0) ? lz_be(a, i, 0)[k - 1] : 0.0);
  const V bpQ = (V)((doQ && k > 0) ? lz_be(a, i, 1)[k - 1] : 0.0);
  const V gA = lz_scale<V>(a, st, 0), gQ = lz_scale<V>(a, st, 1);
  double f[2] = {0.0, 0.0};
  const int r0 = P.blk[b], r1 = P.blk[b + 1];
  // four rows per lane at a time: their loads in flight together; the rows
  // enter |r|^2 in increasing order
  constexpr int U = 4;
  for (int r = r0 + lane; r < r1; r += 32 * U) {
    V w[2][U], v[2][U], vp[2][U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int rr = r + 32 * u;
      if (rr < r1) {
        if (doA) { w[0][u] = __ldg(wA + rr); v[0][u] = vA[rr]; vp[0][u] = vA_prev[rr]; }
        if (doQ) { w[1][u] = __ldg(wQ + rr); v[1][u] = vQ[rr]; vp[1][u] = vQ_prev[rr]; }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int rr = r + 32 * u;
      if (rr < r1) {
        if (doA) {
          const V x = r_mul(v[0][u], gA);
          if (a.lazy) vA[rr] = x;
          const V t = fma(-bpA, vp[0][u], fma(-alA, x, w[0][u]));
          vA_prev[rr] = t;
          f[0] = fma(f2d(t), f2d(t), f[0]);
        }
        if (doQ) {
          const V x = r_mul(v[1][u], gQ);
          if (a.lazy) vQ[rr] = x;
          const V t = fma(-bpQ, vp[1][u], fma(-alQ, x, w[1][u]));
          vQ_prev[rr] = t;
          f[1] = fma(f2d(t), f2d(t), f[1]);
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f[0] += __shfl_xor_sync(0xffffffffu, f[0], o);
    f[1] += __shfl_xor_sync(0xffffffffu, f[1], o);
  }
  if (lane == 0) {
    part[b] = f[0];
    part[(size_t)a.nblkP + b] = f[1];
    lz_chunk_close(a, part, b, i);
  }
}

// Number of eigenvalues of the k x k tridiagonal (al, be2 = squared betas)
// below x: the sign changes of the Sturm sequence p_0 = 1,
// p_i = (al_i - x) p_{i-1} - be_{i-1}^2 p_{i-2} (p_i = det(T_i - x I)); a zero p_i
// takes the sign opposite to p_{i-1}.  Division free, three float64 operations
// per step: signs, zeros and the range check (rescale both terms by 2^-/+500
// when |p_i| leaves [2^-500, 2^500]) work on the bits.
__device__ __forceinline__ int sturm_count(const double* __restrict__ al, const double* __restrict__ be2, int k,
                                           double x) {
  double pm = 1.0, pc = al[0] - x;
  long long bc = __double_as_longlong(pc);
  if ((bc << 1) == 0) { pc = -1e-300; bc = __double_as_longlong(pc); }
  int c = (int)((unsigned long long)bc >> 63);
  for (int i = 1; i < k; ++i) {
    double pn = fma(al[i] - x, pc, -be2[i - 1] * pm);
    long long bn = __double_as_longlong(pn);
    if ((bn << 1) == 0) {
      pn = bc < 0 ? 1e-300 : -1e-300;
      bn = __double_as_longlong(pn);
    }
    c += (int)((unsigned long long)(bn ^ bc) >> 63);
    pm = pc;
    pc = pn;
    bc = bn;
    const int ex = (int)((bn >> 52) & 0x7FF);
    if (ex > 1023 + 500 || ex < 1023 - 500) {
      const double f = ex > 1023 ? 0x1p-500 : 0x1p500;
      pc *= f;
      pm *= f;
      bc = __double_as_longlong(pc);
    }
  }
  return c;
}

// The same count in float32 on the tridiagonal divided by its Gershgorin scale
// (|al_i| <= 1, be2_i <= 1, |x| <= 1, so a step grows the terms at most 3x):
// rescale by 2^-/+60 when |p_i| leaves [2^-60, 2^60].  Only a guess: the float64
// count checks every bracket built from it.
__device__ __forceinline__ int sturm_count_f32(const float* __restrict__ al, const float* __restrict__ be2, int k,
                                               float x) {
  float pm = 1.f, pc = al[0] - x;
  int bc = __float_as_int(pc);
  if ((bc << 1) == 0) { pc = -0x1p-100f; bc = __float_as_int(pc); }
  int c = (int)((unsigned)bc >> 31);
  for (int i = 1; i < k; ++i) {
    float pn = fmaf(al[i] - x, pc, -be2[i - 1] * pm);
    int bn = __float_as_int(pn);
    if ((bn << 1) == 0) {
      pn = bc < 0 ? 0x1p-100f : -0x1p-100f;
      bn = __float_as_int(pn);
    }
    c += (int)((unsigned)(bn ^ bc) >> 31);
    pm = pc;
    pc = pn;
    bc = bn;
    const int ex = (bn >> 23) & 0xFF;
    if (ex > 127 + 60 || ex < 127 - 60) {
      const float f = ex > 127 ? 0x1p-60f : 0x1p60f;
      pc *= f;
      pm *= f;
      bc = __float_as_int(pc);
    }
  }
  return c;
}

// Gershgorin bracket [lo, hi) of the spectrum of the k x k tridiagonal, one
// warp: lanes take every 32nd row, then a shuffle tree
__device__ __forceinline__ void gershgorin_warp(const double* __restrict__ al, const double* __restrict__ be, int k,
                                                double& lo, double& hi) {
  const int lane = threadIdx.x & 31;
  lo = 1e300;
  hi = -1e300;
  for (int i = lane; i < k; i += 32) {
    const double r = (i > 0 ? be[i - 1] : 0.0) + (i < k - 1 ? be[i] : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  hi += 1e-300 + fabs(hi) * 1e-15;
}

// 32-point multisection of a bracket [lo, hi) of lambda_max in one warp, down
// to 4e-15 relative; returns its midpoint
// the multisection's rounds: at most LZ_ROUNDS per bracket, and none once it
// is 4e-15 relative
constexpr int LZ_ROUNDS = 16;
__device__ __forceinline__ bool lz_bracket_open(double lo, double hi, int rounds) {
  return rounds < LZ_ROUNDS && hi - lo > 4e-15 * fabs(hi);
}

// one round of the 32-point multisection of [lo, hi) (in every lane of the warp)
__device__ __forceinline__ void refine_round_warp(const double* __restrict__ al, const double* __restrict__ be2,
                                                  int k, double& lo, double& hi) {
  const int lane = threadIdx.x & 31;
  const double step = (hi - lo) * (1.0 / 33.0);
  const double x = lo + step * (double)(lane + 1);
  const unsigned ge = __ballot_sync(0xffffffffu, sturm_count(al, be2, k, x) < k);   // lambda_max >= x
  if (ge == 0u) {
    hi = lo + step;
  } else {
    const int t = 31 - __clz(ge);
    const double nlo = lo + step * (double)(t + 1);
    hi = t == 31 ? hi : lo + step * (double)(t + 2);
    lo = nlo;
  }
}

__device__ double refine_max_eig_warp(const double* __restrict__ al, const double* __restrict__ be2, int k,
                                      double lo, double hi, int rounds = 0) {
  for (; lz_bracket_open(lo, hi, rounds); ++rounds) refine_round_warp(al, be2, k, lo, hi);
  return 0.5 * (lo + hi);
}

// A bracket [lo, hi) of lambda_max of the k x k tridiagonal, about 1e-6 of its
// Gershgorin scale wide, that float64 Sturm counts at both ends confirm: four
// float32 multisection rounds (alf, be2f: the tridiagonal divided by the
// scale, written here), a margin of 2^-16 of the scale on both sides, then one
// float64 round whose outer lanes sit on the ends.  Falls back to the
// Gershgorin bracket when the check fails.  One warp.
__device__ void bracket_max_eig_warp(const double* __restrict__ al, const double* __restrict__ be,
                                     const double* __restrict__ be2, float* __restrict__ alf,
                                     float* __restrict__ be2f, int k, double& lo, double& hi) {
  const int lane = threadIdx.x & 31;
  double glo, ghi;
  gershgorin_warp(al, be, k, glo, ghi);
  lo = glo;
  hi = ghi;
  const double G = fmax(fabs(glo), fabs(ghi));
  if (!(G > 1e-280 && G < 1e280) || ghi - glo <= 1e-5 * G) return;
  const double iG = 1.0 / G;
  for (int i = lane; i < k; i += 32) {
    alf[i] = (float)(al[i] * iG);
    if (i < k - 1) be2f[i] = (float)(be2[i] * iG * iG);
  }
  __syncwarp();
  float flo = (float)(glo * iG), fhi = (float)(ghi * iG);
  for (int round = 0; round < 4; ++round) {
    const float step = (fhi - flo) * (1.f / 33.f);
    const float x = flo + step * (float)(lane + 1);
    const unsigned ge = __ballot_sync(0xffffffffu, sturm_count_f32(alf, be2f, k, x) < k);
    if (ge == 0u) {
      fhi = flo + step;
    } else {
      const int t = 31 - __clz(ge);
      const float nlo = flo + step * (float)(t + 1);
      fhi = t == 31 ? fhi : flo + step * (float)(t + 2);
      flo = nlo;
    }
  }
  const double clo = fmax(glo, ((double)flo - 0x1p-16) * G);
  const double chi = fmin(ghi, ((double)fhi + 0x1p-16) * G);
  const double step = (chi - clo) * (1.0 / 31.0);
  const double x = lane == 31 ? chi : clo + step * (double)lane;
  const unsigned ge = __ballot_sync(0xffffffffu, sturm_count(al, be2, k, x) < k);
  if ((ge & 1u) && !(ge >> 31)) {              // lambda_max in [clo, chi)
    const int t = 31 - __clz(ge);
    lo = clo + step * (double)t;
    hi = t == 30 ? chi : clo + step * (double)(t + 1);
  }
}

// one CUDA block of NT >= 128 threads per instance (all of them sum the
// instance's chunk sums of |r|^2): beta, theta = lambda_max(T_k) and the stop test for both
// operators (warps 0, 1: A'A; warps 2, 3: Q).  The stop
// test |theta_k - theta_{k-1}| <= tol theta_k (or beta_k <= 1e-12 theta_k, or the
// step limit) needs the precise Ritz values only where the brackets of
// theta_k and theta_{k-1} cannot decide it: then the first warp of the pair
// refines theta_k and the second theta_{k-1} from their brackets, and the
// outcome is the one the precise values give at every step.
// kcap: the tridiagonals' capacity in the dynamic shared memory, at least the
// step's k = pi_iters + 1 of every instance still running (2 kcap (3 doubles +
// 2 floats) bytes).
template <int NT>
__global__ void __launch_bounds__(NT) k_lz_beta(LzArgs a, double tol, int max_steps, int kcap) {
  const int i = blockIdx.x;
  DevState& st = a.st[i];
  if (st.pi_done[0] && st.pi_done[1]) return;     // uniform: nothing left to do
  const Inst in = a.inst[i];
  double f[2] = {0.0, 0.0};
  lz_block_sums(a.cpart, a.nchunk, in.cP0, in.cP0 + kkt_chunks(in.bP0, in.bP1), f);
  const bool is_max[2] = {false, false};
  block_reduce<2>(f, is_max);
  __shared__ double beta[2], s_lo[2], s_hi[2], s_theta[2][2];
  __shared__ int done_in[2], s_precise[2];
  // [2][kcap] each: alphas, |betas|, squared betas (float64), then the scaled
  // float32 copies of the alphas and squared betas
  extern __shared__ __align__(16) double lz_sm[];
  double* const s_al_ = lz_sm;
  double* const s_be_ = lz_sm + 2 * kcap;
  double* const s_be2_ = lz_sm + 4 * kcap;
  float* const s_alf_ = reinterpret_cast<float*>(lz_sm + 6 * kcap);
  float* const s_be2f_ = s_alf_ + 2 * kcap;
  auto s_al = [&](int o) { return s_al_ + o * kcap; };
  auto s_be = [&](int o) { return s_be_ + o * kcap; };
  auto s_be2 = [&](int o) { return s_be2_ + o * kcap; };
  auto s_alf = [&](int o) { return s_alf_ + o * kcap; };
  auto s_be2f = [&](int o) { return s_be2f_ + o * kcap; };
  const int k = st.pi_iters + 1;                  // alphas 0..k-1, betas 0..k-2 form T_k
  if (threadIdx.x == 0) {
    beta[0] = sqrt(f[0]); beta[1] = sqrt(f[1]);
    done_in[0] = st.pi_done[0]; done_in[1] = st.pi_done[1];
  }
  for (int o = 0; o < 2; ++o)
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
      s_al(o)[t] = lz_al(a, i, o)[t];
      if (t < k - 1) {
        const double bb = lz_be(a, i, o)[t];
        s_be(o)[t] = fabs(bb);
        s_be2(o)[t] = bb * bb;
      }
    }
  __syncthreads();
  const bool ritz = threadIdx.x < 128;            // warps 0..3 work on the Ritz values
  const int o = (threadIdx.x >> 6) & 1, second = (threadIdx.x >> 5) & 1, lane = threadIdx.x & 31;
  const double plo = st.pi_lam_prev[o], phi = st.pi_hi_prev[o];   // bracket of theta_{k-1}
  if (ritz && !done_in[o] && !second) {           // warp-uniform
    double lo, hi;
    bracket_max_eig_warp(s_al(o), s_be(o), s_be2(o), s_alf(o), s_be2f(o), k, lo, hi);
    const double mag = fmax(fabs(lo), fabs(hi));
    const double gap = fmax(fmax(lo - phi, plo - hi), 0.0);   // least |theta_k - theta_{k-1}|
    const bool go_on = k < max_steps && beta[o] > 1e-12 * mag && gap > tol * mag;
    if (lane == 0) {
      s_lo[o] = lo;
      s_hi[o] = hi;
      s_precise[o] = !go_on;
    }
  }
  // Where the brackets leave the stop test open: refine theta_k's bracket and
  // theta_{k-1}'s (when it is not exact), one round each at a time, until the
  // brackets decide the test for certain (every value in them gives the same
  // outcome) or both are at full precision (then their midpoints decide, as
  // the precise values do).  Most steps near convergence go on, and learn it
  // in a round or two; a stop needs theta_k in full and refines it the rest
  // of the way, through the same rounds as a single refinement would take.
  __shared__ double s_plo[2], s_phi[2];
  __shared__ int s_rk[2], s_rp[2], s_dec[2];       // rounds done; decision: 0 open, 1 go on, 2 stop
  __syncthreads();                                 // s_lo, s_hi, s_precise written above
  if (threadIdx.x < 2) {
    const int q = threadIdx.x;
    s_plo[q] = st.pi_lam_prev[q];
    s_phi[q] = st.pi_hi_prev[q];
    s_rk[q] = 0;
    s_rp[q] = 0;
    s_dec[q] = (!done_in[q] && s_precise[q]) ? 0 : 1;
  }
  __syncthreads();
  for (int pass = 0; pass <= 2 * LZ_ROUNDS + 1; ++pass) {    // every thread takes the same passes
    if (ritz && !second && lane == 0 && s_dec[o] == 0) {
      const double lk = s_lo[o], hk = s_hi[o], lp = s_plo[o], hp = s_phi[o], b = beta[o];
      const bool open_k = lz_bracket_open(lk, hk, s_rk[o]);
      const bool open_p = lp != hp && lz_bracket_open(lp, hp, s_rp[o]);
      int dec = 0;
      if (k >= max_steps) {
        dec = 2;
      } else if (!open_k && !open_p) {                        // full precision: the midpoints decide
        const double th = 0.5 * (lk + hk), tp = lp == hp ? lp : 0.5 * (lp + hp);
        dec = (fabs(th - tp) <= tol * fabs(th) || b <= 1e-12 * fabs(th)) ? 2 : 1;
      } else {   // certain outcomes: the tests hold for every value in the brackets
        const double dmax = fmax(hk - lp, hp - lk), dmin = fmax(fmax(lk - hp, lp - hk), 0.0);
        const double amax = fmax(fabs(lk), fabs(hk));                      // largest |theta_k|
        const double amin = (lk <= 0.0 && hk >= 0.0) ? 0.0 : fmin(fabs(lk), fabs(hk));   // least
        if (dmax <= tol * amin || b <= 1e-12 * amin) dec = 2;
        else if (dmin > tol * amax && b > 1e-12 * amax) dec = 1;
      }
      s_dec[o] = dec;
    }
    __syncthreads();
    if (s_dec[0] != 0 && s_dec[1] != 0) break;               // uniform: shared values after the barrier
    if (ritz && s_dec[o] == 0) {                              // warp-uniform
      if (!second && lz_bracket_open(s_lo[o], s_hi[o], s_rk[o])) {
        double lo = s_lo[o], hi = s_hi[o];
        refine_round_warp(s_al(o), s_be2(o), k, lo, hi);
        __syncwarp();
        if (lane == 0) { s_lo[o] = lo; s_hi[o] = hi; ++s_rk[o]; }
      } else if (second && s_plo[o] != s_phi[o] && lz_bracket_open(s_plo[o], s_phi[o], s_rp[o])) {
        double lo = s_plo[o], hi = s_phi[o];
        refine_round_warp(s_al(o), s_be2(o), k - 1, lo, hi);
        __syncwarp();
        if (lane == 0) { s_plo[o] = lo; s_phi[o] = hi; ++s_rp[o]; }
      }
    }
    __syncthreads();
  }
  // a stop needs theta_k in full (the rest of its refinement)
  if (ritz && !second && !done_in[o] && s_precise[o] && s_dec[o] == 2) {
    const double th = refine_max_eig_warp(s_al(o), s_be2(o), k, s_lo[o], s_hi[o], s_rk[o]);
    if (lane == 0) s_theta[o][0] = th;
  }
  __syncthreads();
  if (ritz && !done_in[o] && !second && lane == 0) {
    const double b = beta[o];
    if (!s_precise[o] || s_dec[o] == 1) {        // goes on: keep the (refined) bracket
      st.pi_lam[o] = 0.5 * (s_lo[o] + s_hi[o]);
      st.pi_lam_prev[o] = s_lo[o];
      st.pi_hi_prev[o] = s_hi[o];
      lz_be(a, i, o)[k - 1] = b;
      st.pi_inv_norm[o] = 1.0 / b;
    } else {                                      // stops with theta_k in full
      st.pi_lam[o] = s_theta[o][0];
      st.pi_done[o] = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) st.pi_iters = k;
}

// v_next = r / beta (in the buffer that held v_prev)
template <typename V>
__global__ void k_lz_norm(LzArgs a, V* __restrict__ vA_next, V* __restrict__ vQ_next) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += gridDim.x * blockDim.x) {
    const DevState& st = a.st[a.row_inst_n[r]];
    // pi_inv_norm changes only when the operator continues; the product in the
    // vectors' precision
    if (!st.pi_done[0]) vA_next[r] = vA_next[r] * (V)st.pi_inv_norm[0];
    if (!st.pi_done[1]) vQ_next[r] = vQ_next[r] * (V)st.pi_inv_norm[1];
  }
}

// Start vector entry of row j (its index within its instance) of an instance
// of n variables: +-1/sqrt(n), negative where the top bit of the SplitMix64
// finaliser (Steele, Lea & Flood 2014) of j is set.  Not the all-ones vector,
// an eigenvector of Laplacian-like operators (of L + cI for its smallest
// eigenvalue; of A'A in its null space when A's rows sum to zero).
__device__ __forceinline__ double lz_start(int j, int n) {
  unsigned long long z = (unsigned long long)j + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  const double v = 1.0 / sqrt((double)n);
  return (z >> 63) ? -v : v;
}

// start vectors per instance; Lanczos state
template <typename V>
__global__ void k_lz_init(LzArgs a, V* __restrict__ vA0, V* __restrict__ vA1, V* __restrict__ vQ0,
                          V* __restrict__ vQ1) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += gridDim.x * blockDim.x) {
    const Inst& in = a.inst[a.row_inst_n[r]];
    const V v = (V)lz_start(r - in.xoff, in.n);
    vA0[r] = v; vQ0[r] = v; vA1[r] = V(0); vQ1[r] = V(0);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.count; i += gridDim.x * blockDim.x) {
    DevState& st = a.st[i];
    st.pi_done[0] = a.inst[i].m > 0 ? 0 : 1;
    st.pi_done[1] = 0;
    st.pi_lam[0] = 0.0; st.pi_lam[1] = 0.0;
    st.pi_lam_prev[0] = 0.0; st.pi_lam_prev[1] = 0.0;
    st.pi_hi_prev[0] = 0.0; st.pi_hi_prev[1] = 0.0;
    st.pi_inv_norm[0] = 1.0; st.pi_inv_norm[1] = 1.0;
    st.pi_iters = 0;
  }
}

template <typename V>
__global__ void k_fill_v(V* __restrict__ p, V v, long long N) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) p[i] = v;
}

__global__ void k_set_norms(DevState* sts, int count, double nA, double nQ) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    DevState* st = sts + i;
    st->normA = nA > 0.0 ? nA : sqrt(fmax(st->pi_lam[0], 0.0));
    st->normQ = nQ > 0.0 ? nQ : fmax(st->pi_lam[1], 0.0);
  }
}

// |c~|^2 over each row block of P, |b~|^2 over each row block of A
__global__ void k_omega_part(const int* __restrict__ blkP, int nblkP, const int* __restrict__ blkA,
                             const double* __restrict__ cs, const double* __restrict__ bs,
                             double* __restrict__ partP, double* __restrict__ partA) {
  const bool isP = blockIdx.x < nblkP;
  const int b = isP ? blockIdx.x : blockIdx.x - nblkP;
  const int* blk = isP ? blkP : blkA;
  const double* v = isP ? cs : bs;
  double f = 0.0;
  for (int r = blk[b] + threadIdx.x; r < blk[b + 1]; r += blockDim.x) f += v[r] * v[r];
  f = block_sum(f);
  if (threadIdx.x == 0) (isP ? partP : partA)[b] = f;
}

// ||c~||, ||b~|| of each instance -> InitializePrimalWeight (one CUDA block per instance)
__global__ void k_init_omega(DevState* sts, const Inst* __restrict__ insts, const double* __restrict__ partP,
                             const double* __restrict__ partA, double eps_zero) {
  const int i = blockIdx.x;
  const Inst in = insts[i];
  double f[2] = {0.0, 0.0};
  for (int b = in.bP0 + threadIdx.x; b < in.bP1; b += blockDim.x) f[0] += partP[b];
  for (int b = in.bA0 + threadIdx.x; b < in.bA1; b += blockDim.x) f[1] += partA[b];
  const bool is_max[2] = {false, false};
  block_reduce<2>(f, is_max);
  if (threadIdx.x == 0) {
    DevState* st = sts + i;
    const double nc = sqrt(f[0]), nb = sqrt(f[1]);
    st->omega = (nc > eps_zero && nb > eps_zero) ? nc / nb : 1.0;
    st->eta_last = 0.0;
    st->status = ST_RUNNING;
  }
}

// --------------------------------------------------------------------------
// Start point: x = proj_X(x0 / D2), y = proj_Y(y0 / D1), zeros by default
// (Section 5 "Algorithms"); averages, x_md, x_tilde and anchors = start.
// --------------------------------------------------------------------------
__global__ void k_init_iterates(int n, int m, const unsigned char* __restrict__ ineq, const double* __restrict__ x0,
                                const double* __restrict__ y0, const double* __restrict__ D1,
                                const double* __restrict__ D2, const double* __restrict__ ls,
                                const double* __restrict__ us, double* x, double* xbar, double* xmd0,
                                double* xt, double* ax, double* y, double* ybar, double* ay) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double v = x0 ? x0[i] / D2[i] : 0.0;
    v = fmin(fmax(v, ls[i]), us[i]);
    x[i] = v; xbar[i] = v; xmd0[i] = v; xt[i] = v; ax[i] = v;
  }
  if (i < m) {
    double v = y0 ? y0[i] / D1[i] : 0.0;
    if (ineq[i]) v = fmax(v, 0.0);
    y[i] = v; ybar[i] = v; ay[i] = v;
  }
}


// Section 6 bound 0.99 (k+2) / (q + sqrt(|A|^2 (k+2)^2 + q^2)), q = |Q|/omega
// (its k = 0 value is the k = 0 step 1.98 / (q + sqrt(4|A|^2 + q^2))).
__device__ __forceinline__ double pdqp_bound(long long k, double q, double nA) {
  if (k == 0) return 1.98 / (q + sqrt(4.0 * (nA * nA) + q * q));
  const double kk = (double)(k + 2);
  return 0.99 * kk / (q + sqrt((nA * nA) * (kk * kk) + q * q));
}

// Step scalars of inner iteration k.  Within an epoch omega is fixed and the
// recurrence eta_k = min((1 + 1/k) eta_{k-1}, bound_k) started at eta_0 =
// bound_0 always picks bound_k, because bound_k / bound_{k-1} <= (k+2)/(k+1) <
// (k+1)/k; so each entry evaluates min((1 + 1/k) bound_{k-1}, bound_k) on its
// own, which reproduces the recurrence value for value.
__device__ StepEntry make_step(long long k, const DevState& S, const SolveParams& p) {
  double beta = 1.0, beta1 = 1.0, theta1 = 1.0;
  if (p.accelerate) {
    beta = (double)(k + 2) / 2.0;
    beta1 = (double)(k + 3) / 2.0;
    theta1 = (double)(k + 1) / ((double)(k + 1) + 1.0);
  }
  double tau, sig;
  if (p.step_rule == 1) {   // Theorem 1
    tau = (double)(k + 1) / (2.0 * (S.normQ + p.fixed_K * S.normA));
    sig = (double)(k + 1) / (2.0 * p.fixed_K * S.normA);
  } else {
    const double q = S.normQ / S.omega;
    double eta;
    if (!p.accelerate || k == 0) eta = pdqp_bound(0, q, S.normA);
    else eta = fmin((1.0 + 1.0 / (double)k) * pdqp_bound(k - 1, q, S.normA), pdqp_bound(k, q, S.normA));
    tau = eta / S.omega;
    sig = eta * S.omega;
  }
  StepEntry e;
  e.tau_p = tau; e.sigma_d = sig; e.inv_beta = 1.0 / beta; e.inv_beta_next = 1.0 / beta1;
  e.theta_next = theta1;
  e.tau_p_f = (float)tau; e.sigma_d_f = (float)sig; e.inv_beta_f = (float)e.inv_beta;
  e.inv_beta_next_f = (float)e.inv_beta_next; e.theta_next_f = (float)theta1;
  return e;
}

// Tabulate the next `check_period` entries (k = k_epoch + j), all threads.
__device__ void fill_steps_block(const DevState& S, const SolveParams& p, StepEntry* tab) {
  for (int j = threadIdx.x; j < p.check_period; j += blockDim.x) tab[j] = make_step(S.k_epoch + j, S, p);
}

__device__ void decide_thread0(DevState* __restrict__ st, const double* F, const SolveParams& p, int mode,
                               long long chunk_len, int inf_status);

// Chunk sums of the relKKT group partials: CUDA block (i, c) reduces chunk c
// of instance i -- its KKT_CHUNK / KKT_GROUP consecutive groups from the
// instance's first (KKT_CHUNK row blocks) -- for every field in a fixed order,
// so that a batch and a standalone solve sum identically and the decision
// kernel reads tens of values, not thousands.  gfm, gfn: first group of each
// instance (A, P).
constexpr int KKT_GPC = KKT_CHUNK / KKT_GROUP;   // groups per chunk (8: lanes 0..7)
__global__ void __launch_bounds__(32) k_kkt_chunks(const Inst* __restrict__ insts, const int* __restrict__ gfm,
                                                   const double* __restrict__ pm, int ngm,
                                                   const int* __restrict__ gfn, const double* __restrict__ pn,
                                                   int ngn, double* __restrict__ cm, int ncm,
                                                   double* __restrict__ cn, int ncn) {
  const int i = blockIdx.x;
  const Inst in = insts[i];
  const int lane = threadIdx.x, c = blockIdx.y;
  if (in.bP0 + c * KKT_CHUNK < in.bP1) {
    const bool is_max[15] = {true, true, true, false, false, false, false,
                             true, true, true, false, false, false, false, true};
    const int g = gfn[i] + c * KKT_GPC + lane;
    const bool on = lane < KKT_GPC && g < gfn[i + 1];
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      double v = on ? pn[(size_t)k * ngn + g] : 0.0;
#pragma unroll
      for (int o = KKT_GPC / 2; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max[k] ? nmax(v, t) : v + t;
      }
      if (lane == 0) cn[(size_t)k * ncn + in.cP0 + c] = v;
    }
  }
  if (in.m > 0 && in.bA0 + c * KKT_CHUNK < in.bA1) {
    const bool is_max[9] = {true, true, false, false, true, true, false, false, true};
    const int g = gfm[i] + c * KKT_GPC + lane;
    const bool on = lane < KKT_GPC && g < gfm[i + 1];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double v = on ? pm[(size_t)k * ngm + g] : 0.0;
#pragma unroll
      for (int o = KKT_GPC / 2; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max[k] ? nmax(v, t) : v + t;
      }
      if (lane == 0) cm[(size_t)k * ncm + in.cA0 + c] = v;
    }
  }
}


// mode 0: evaluate z^{0,0} (anchor, maybe already optimal); mode 1: a check
// after `chunk_len` more iterations (Section 6 restart rule, termination
// eq. (terminate), iteration limit).
// one CUDA block of 64 threads per instance (one step-table entry per thread)
__global__ void __launch_bounds__(64) k_decide(DevState* __restrict__ sts, const Inst* __restrict__ insts,
                                                const double* __restrict__ pm, int nbm,
                                                const double* __restrict__ pn, int nbn,
                                                StepEntry* __restrict__ tabs, int C, SolveParams p, int mode,
                                                long long chunk_len, const InfState* __restrict__ inf) {
  const int i = blockIdx.x;
  DevState* st = sts + i;
  if (mode == 1 && st->status != ST_RUNNING) return;     // uniform
  const Inst in = insts[i];
  __shared__ double F[24];
  // pm / pn hold the chunk sums of k_kkt_chunks
  reduce_kkt_blocks(pm, nbm, in.cA0, in.m > 0 ? in.cA0 + kkt_chunks(in.bA0, in.bA1) : in.cA0, pn, nbn, in.cP0,
                    in.cP0 + kkt_chunks(in.bP0, in.bP1), F);
  if (threadIdx.x == 0) decide_thread0(st, F, p, mode, chunk_len, inf ? inf[i].status : 0);
  __syncthreads();
  if (st->status == ST_RUNNING) fill_steps_block(*st, p, tabs + (size_t)i * C);
}

// number of instances still iterating / still estimating norms
__global__ void k_count_running(const DevState* __restrict__ sts, const Inst* __restrict__ inst,
                                const int* __restrict__ rpA, const int* __restrict__ rpP, int count,
                                BatchState* bst) {
  int run = 0, lz = 0;
  double f[4] = {0.0, 0.0, 0.0, 0.0};   // rows of P and A, nonzeros of A and P of the running instances
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const bool r = sts[i].status == ST_RUNNING;
    run += r;
    lz += !(sts[i].pi_done[0] && sts[i].pi_done[1]);
    if (r) {
      const Inst in = inst[i];
      f[0] += in.n;
      f[1] += in.m;
      if (in.m > 0) f[2] += rpA[in.yoff + in.m] - rpA[in.yoff];
      f[3] += rpP[in.xoff + in.n] - rpP[in.xoff];
    }
  }
  run = block_sum(run);
  lz = block_sum(lz);
  const bool is_max[4] = {false, false, false, false};
  block_reduce<4>(f, is_max);
  if (threadIdx.x == 0) {
    bst->running = run; bst->lz_running = lz;
    bst->run_n = f[0]; bst->run_m = f[1]; bst->run_nnzA = f[2]; bst->run_nnzP = f[3];
  }
}

__device__ void decide_thread0(DevState* __restrict__ st, const double* F, const SolveParams& p, int mode,
                               long long chunk_len, int inf_status) {
  DevState& S = *st;
  double P[2][6];
  kkt_from_fields(F, 0, P[0]);
  kkt_from_fields(F, 1, P[1]);
  for (int it = 0; it < 2; ++it)
    for (int k = 0; k < 6; ++k) S.parts[it][k] = P[it][k];
  S.restart = 0;
  if (mode == 0) {
    S.anchor_kkt = P[0][3];
    S.has_prev = 0;
    S.k_epoch = 0; S.k_total = 0; S.restarts = 0;
    S.out_avg = 0;
    for (int k = 0; k < 6; ++k) S.out_parts[k] = P[0][k];
    const double r = P[0][3];
    S.status = (r != r) ? ST_NUMERICAL : (r <= p.eps ? ST_OPTIMAL : ST_RUNNING);
    return;
  }
  S.k_total += chunk_len;
  S.k_epoch += chunk_len;
  const double kc = P[0][3], ka = P[1][3];
  const int cand_avg = (kc < ka) ? 0 : 1;          // GetRestartCandidate, ties -> average
  const double cand = cand_avg ? ka : kc;
  S.out_avg = cand_avg;
  for (int k = 0; k < 6; ++k) S.out_parts[k] = P[cand_avg][k];
  if (kc != kc || ka != ka) { S.status = ST_NUMERICAL; return; }
  if (cand <= p.eps) { S.status = ST_OPTIMAL; return; }
  if (S.k_total >= p.max_iter) { S.status = ST_ITER_LIMIT; return; }
  if (inf_status) { S.status = inf_status; return; }   // a certificate of this check (optional)
  int restart = 0, to_avg = cand_avg;
  double new_anchor = cand;
  if (p.restart_rule == 0) {
    restart = (cand <= p.beta_suff * S.anchor_kkt) ||
              (cand <= p.beta_nec * S.anchor_kkt && S.has_prev && cand > S.prev_cand_kkt) ||
              ((double)S.k_epoch >= p.beta_art * (double)S.k_total);
  } else if (p.restart_rule == 1) {
    to_avg = 1; new_anchor = ka; restart = ka <= 0.5 * S.anchor_kkt;
  } else if (p.restart_rule == 2) {
    to_avg = 1; new_anchor = ka; restart = S.k_epoch >= p.fixed_K;
  }
  if (!restart) {
    S.prev_cand_kkt = (p.restart_rule == 0) ? cand : new_anchor;
    S.has_prev = 1;
  } else {
    const double dx2 = F[9 + to_avg * 7 + 6], dy2 = F[to_avg * 4 + 3];
    if (p.step_rule == 0) {   // PrimalWeightUpdate
      const double dx = sqrt(dx2), dy = sqrt(dy2);
      if (dx > p.eps_zero && dy > p.eps_zero)
        S.omega = exp(p.pw_theta * log(dy / dx) + (1.0 - p.pw_theta) * log(S.omega));
    }
    S.restarts += 1;
    S.anchor_kkt = new_anchor;
    S.has_prev = 0;
    S.k_epoch = 0;
    S.restart = 1;
    S.cand_avg = to_avg;
  }
}

// Restart of the outer loop from the candidate: x = x_bar = x_md = x_tilde = x_c,
// y = y_bar = y_c, anchors = z_c (Algorithm 1 "restart the outer loop").
// Row blocks of the instances still running (batches): indices in act, their
// number in *n (in any order: a block's rows do not depend on its place in
// the grid).
__global__ void k_compact_blocks(const int* __restrict__ blk_inst, int nblk, const DevState* __restrict__ st,
                                 int* __restrict__ act, int* __restrict__ n) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x)
    if (st[blk_inst[b]].status == ST_RUNNING) act[atomicAdd(n, 1)] = b;
}

__global__ void k_restart_apply(const DevState* __restrict__ sts, const int* __restrict__ inst_n,
                                const int* __restrict__ inst_m, int n, int m, double* x, double* xbar,
                                double* xmd0, double* xt, double* ax, double* y, double* ybar, double* ay) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(n, m); i += gridDim.x * blockDim.x) {
    if (i < n) {
      const DevState& s = sts[inst_n[i]];
      if (s.status == ST_RUNNING && s.restart) {
        const double v = s.cand_avg ? xbar[i] : x[i];
        x[i] = v; xbar[i] = v; xmd0[i] = v; xt[i] = v; ax[i] = v;
      }
    }
    if (i < m) {
      const DevState& s = sts[inst_m[i]];
      if (s.status == ST_RUNNING && s.restart) {
        const double v = s.cand_avg ? ybar[i] : y[i];
        y[i] = v; ybar[i] = v; ay[i] = v;
      }
    }
  }
}

// Original-space output of the returned iterate (or of the raw state).
__global__ void k_unscale_out(int n, int m, const double* __restrict__ D1, const double* __restrict__ D2,
                              const double* __restrict__ xs0, const double* __restrict__ xs1,
                              const double* __restrict__ ys0, const double* __restrict__ ys1,
                              const DevState* __restrict__ sts, const int* __restrict__ inst_n,
                              const int* __restrict__ inst_m, int pick, double* x_out, double* y_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (x_out && i < n) {
    const int sel = pick < 0 ? sts[inst_n[i]].out_avg : pick;
    x_out[i] = D2[i] * (sel ? xs1[i] : xs0[i]);
  }
  if (y_out && i < m) {
    const int sel = pick < 0 ? sts[inst_m[i]].out_avg : pick;
    y_out[i] = D1[i] * (sel ? ys1[i] : ys0[i]);
  }
}

// --------------------------------------------------------------------------
// Mixed precision (float32 iteration, float64 checks).  The iteration runs on
// the shifted problem in (dx, dy) = (x - x_hi, y - y_hi) around a float64 base
// z_hi: c' = c~ + Q~x_hi - A~'y_hi, b' = b~ - A~x_hi, l' = l~ - x_hi,
// u' = u~ - x_hi and dy_I >= -y_hi,I.  Each check materialises the float64
// iterates proj(z_hi + dz); each restart moves z_hi to the candidate and
// recomputes the shifted data from the float64 products of that check (the
// residual correction).
// --------------------------------------------------------------------------
struct MixedArgs {
  int n, m;
  const unsigned char* ineq;
  const DevState* sts;
  const int *inst_n, *inst_m;
  const double *cs, *bs, *ls, *us, *D1, *D2;
  double *xhi, *yhi;
  float *fx, *fxbar, *fxt, *fxmd0, *fy, *fybar;
  float *fc, *fl, *fu, *fb, *fylo;
  double *x64[2], *y64[2];               // materialised iterates (current, average)
  double2 *xx, *yy;                      // the same as pairs for the relKKT gathers (null: not written)
  const double *prodAx, *prodQx, *prodATy;   // [2][m], [2][n], [2][n]
};

__global__ void k_init_mixed(MixedArgs a, const double* __restrict__ x0, const double* __restrict__ y0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) {
    double v = x0 ? x0[i] / a.D2[i] : 0.0;
    a.xhi[i] = fmin(fmax(v, a.ls[i]), a.us[i]);
    a.fx[i] = 0.f; a.fxbar[i] = 0.f; a.fxt[i] = 0.f; a.fxmd0[i] = 0.f;
  }
  if (i < a.m) {
    double v = y0 ? y0[i] / a.D1[i] : 0.0;
    if (a.ineq[i]) v = fmax(v, 0.0);
    a.yhi[i] = v;
    a.fy[i] = 0.f; a.fybar[i] = 0.f;
  }
}

// (x, x_bar) and (y, y_bar) as pairs for the relKKT gathers (float64 mode)
__global__ void k_pair_iterates(int n, int m, const double* __restrict__ x, const double* __restrict__ xbar,
                                const double* __restrict__ y, const double* __restrict__ ybar,
                                double2* __restrict__ xx, double2* __restrict__ yy) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(n, m); i += gridDim.x * blockDim.x) {
    if (i < n) xx[i] = make_double2(x[i], xbar[i]);
    if (i < m) yy[i] = make_double2(y[i], ybar[i]);
  }
}

__global__ void k_materialize(MixedArgs a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(a.n, a.m); i += gridDim.x * blockDim.x) {
    if (i < a.n) {
      const double h = a.xhi[i], lo = a.ls[i], hi = a.us[i];
      const double v0 = fmin(fmax(h + (double)a.fx[i], lo), hi), v1 = fmin(fmax(h + (double)a.fxbar[i], lo), hi);
      a.x64[0][i] = v0;
      a.x64[1][i] = v1;
      if (a.xx) a.xx[i] = make_double2(v0, v1);
    }
    if (i < a.m) {
      const double h = a.yhi[i];
      double v0 = h + (double)a.fy[i], v1 = h + (double)a.fybar[i];
      if (a.ineq[i]) { v0 = fmax(v0, 0.0); v1 = fmax(v1, 0.0); }
      a.y64[0][i] = v0;
      a.y64[1][i] = v1;
      if (a.yy) a.yy[i] = make_double2(v0, v1);
    }
  }
}

// Move the base to the candidate (or, with force, re-derive the shifted data
// at the current base) and zero the float32 deltas.
__global__ void k_mixed_rebase(MixedArgs a, int force) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(a.n, a.m); i += gridDim.x * blockDim.x) {
    if (i < a.n) {
      const DevState& s = a.sts[a.inst_n[i]];
      if (force || (s.status == ST_RUNNING && s.restart)) {
        const int ca = force ? 0 : s.cand_avg;
        const double xh = a.x64[ca][i];
        a.xhi[i] = xh;
        a.fc[i] = (float)(a.cs[i] + a.prodQx[(size_t)ca * a.n + i] - a.prodATy[(size_t)ca * a.n + i]);
        a.fl[i] = (float)(a.ls[i] - xh);
        a.fu[i] = (float)(a.us[i] - xh);
        a.fx[i] = 0.f; a.fxbar[i] = 0.f; a.fxt[i] = 0.f; a.fxmd0[i] = 0.f;
      }
    }
    if (i < a.m) {
      const DevState& s = a.sts[a.inst_m[i]];
      if (force || (s.status == ST_RUNNING && s.restart)) {
        const int ca = force ? 0 : s.cand_avg;
        const double yh = a.y64[ca][i];
        a.yhi[i] = yh;
        a.fb[i] = (float)(a.bs[i] - a.prodAx[(size_t)ca * a.m + i]);
        a.fylo[i] = a.ineq[i] ? (float)(-yh) : -INFINITY;
        a.fy[i] = 0.f; a.fybar[i] = 0.f;
      }
    }
  }
}

// ==========================================================================
// Host-side launchers
// ==========================================================================
void scale_reset(Work& w, cudaStream_t s) {
  const long long N = (long long)w.n + w.m;
  launch(k_fill, cdiv(N, 256), 256, 0, s, w.dsc, 1.0, N);
}

// pass `pass` of a sequence reads the factors from dsc (even) or nu (odd) and
// writes them to the other buffer
template <int KIND>
static void scale_pass_t(Work& w, const double* d, double* dn, cudaStream_t s) {
  launch(k_scale_pass<KIND>, w.P.nblk, BNT, 0, s, w.P.borig(), d, 0, 0, dn);
  launch(k_scale_pass<KIND>, w.A.nblk, BNT, 0, s, w.A.borig(), d, w.n, 0, dn);
}

void scale_pass(Work& w, int kind, int pass, cudaStream_t s) {
  const double* d = (pass & 1) ? w.nu : w.dsc;
  double* dn = (pass & 1) ? w.dsc : w.nu;
  if (kind == 0) scale_pass_t<0>(w, d, dn, s);
  else if (kind == 1) scale_pass_t<1>(w, d, dn, s);
  else scale_pass_t<2>(w, d, dn, s);
}

// every member's copy of the template's nnz_t values (members strided over grid.y)
template <typename T>
__global__ void k_rep_scaled(const T* __restrict__ t, long long nnz_t, int count, T* __restrict__ out) {
  for (int q = blockIdx.y; q < count; q += gridDim.y) {
    T* o = out + (long long)q * nnz_t;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz_t;
         e += (long long)gridDim.x * blockDim.x)
      o[e] = t[e];
  }
}

template <typename T>
static void rep_scaled(const T* t, long long nnz_t, int count, T* out, int num_sms, cudaStream_t s) {
  if (nnz_t <= 0 || count <= 0 || !t || !out) return;
  const int gx = (int)std::min<long long>(cdiv(nnz_t, 256), std::max(1, 4 * num_sms / std::max(count, 1) + 1));
  launch(k_rep_scaled<T>, dim3(gx, std::min(count, 65535)), 256, 0, s, t, nnz_t, count, out);
}

void scale_apply(Work& w, bool mixed, cudaStream_t s, const Work* tmpl) {
  const int N = w.n + w.m;
  launch(k_inverse, cdiv(N, 256), 256, 0, s, (const double*)w.dsc, w.idsc, N);
  if (tmpl) {
    // a family handle: every member's scaled values are the template's (the
    // same factors and values, the same formula), copied instead of scaled
    rep_scaled<double>(tmpl->P.sval, tmpl->P.nnz, w.count, w.P.sval, w.num_sms, s);
    rep_scaled<double>(tmpl->A.sval, tmpl->A.nnz, w.count, w.A.sval, w.num_sms, s);
    if (mixed) {
      rep_scaled<float>(tmpl->P.sval_f, tmpl->P.nnz, w.count, w.P.sval_f, w.num_sms, s);
      rep_scaled<float>(tmpl->A.sval_f, tmpl->A.nnz, w.count, w.A.sval_f, w.num_sms, s);
    }
  } else {
    launch(k_scale_vals, w.P.nblk, BNT, 0, s, w.P.borig(), (const double*)w.dsc, 0, 0, w.P.sval,
           mixed ? w.P.sval_f : (float*)nullptr);
    launch(k_scale_vals, w.A.nblk, BNT, 0, s, w.A.borig(), (const double*)w.dsc, w.n, 0, w.A.sval,
           mixed ? w.A.sval_f : (float*)nullptr);
  }
  const int NN = w.n > w.m ? w.n : w.m;
  if (w.r > 0)
    launch(k_lr_scale, std::min(cdiv((long long)w.n * w.r, 256), 8 * w.num_sms), 256, 0, s, (const float*)w.F,
           (const double*)w.D2, w.n, w.r, w.Fd, mixed ? w.Fs : (float*)nullptr);
  launch(k_scale_vectors, cdiv(NN, 256), 256, 0, s, w.n, w.m, (const double*)w.D1, (const double*)w.D2,
         (const double*)w.c, (const double*)w.b, (const double*)w.l, (const double*)w.u, w.cs, w.bs, w.ls, w.us,
         (float*)nullptr);
}

// w = F' v (nv = 1) or F' [v0, v1] (nv = 2) into w.wlr
template <typename FV, typename X>
static void lowrank_ft(Work& w, const FV* F, const X* v0, const X* v1, cudaStream_t s) {
  const int grid = std::min(cdiv(w.n, LR_ROWS), 4 * w.num_sms);
  if (v1) launch(k_lr_ft<FV, X, 2>, grid, 256, 0, s, F, w.n, w.r, v0, v1, w.lr_part);
  else launch(k_lr_ft<FV, X, 1>, grid, 256, 0, s, F, w.n, w.r, v0, v1, w.lr_part);
  launch(k_lr_reduce, w.r * (v1 ? 2 : 1), 256, 0, s, (const double*)w.lr_part, grid, w.r, v1 ? 2 : 1, w.wlr,
         w.wlr_f);
}

void lowrank_ft1(Work& w, const float* F, const float* v, cudaStream_t s) {
  lowrank_ft<float, float>(w, F, v, (const float*)nullptr, s);
}
void lowrank_ft1(Work& w, const double* F, const double* v, cudaStream_t s) {
  lowrank_ft<double, double>(w, F, v, (const double*)nullptr, s);
}

static LzArgs lz_args(Work& w) {
  LzArgs la{};
  la.n = w.n; la.m = w.m; la.count = w.count;
  la.al = w.lz_al; la.be = w.lz_be; la.st = w.st; la.inst = w.inst;
  la.blk_inst_P = w.blk_inst_P; la.blk_inst_A = w.blk_inst_A; la.row_inst_n = w.row_inst_n;
  la.nblkP = w.P.nblk;
  la.lazy = w.r == 0 ? 1 : 0;
  la.cpart = w.cpart_n; la.ticket = w.lz_ticket; la.nchunk = w.nchunk_n;
  if (w.lz_compact) { la.actA = w.act_A; la.actP = w.act_P; la.nactP = w.bst_host->act_P; }
  return la;
}

template <typename V>
static void lanczos_init_t(Work& w, V* const* pu, V* const* pz, cudaStream_t s) {
  const int grid = std::min(cdiv(std::max(w.n, w.count), 256), 4 * w.num_sms);
  launch(k_lz_init<V>, grid, 256, 0, s, lz_args(w), pu[0], pu[1], pz[0], pz[1]);
}

void lanczos_init(Work& w, bool mixed, cudaStream_t s) {
  if (mixed) lanczos_init_t<float>(w, w.fpu, w.fpz, s);
  else lanczos_init_t<double>(w, w.pu, w.pz, s);
}

template <typename V, int NT>
static void lanczos_step_t(Work& w, int t, const SolveParams& p, BCsr<V> A, BCsr<V> P, V* const* pu, V* const* pz,
                           V* const* lw, cudaStream_t s) {
  const int cur = t & 1, prv = cur ^ 1;
  const LzArgs la = lz_args(w);
  // all row blocks, or late in a batch's estimates those of the instances still running
  const int gA = w.lz_compact ? w.bst_host->act_A : w.A.nblk, gP = w.lz_compact ? w.bst_host->act_P : w.P.nblk;
  if (w.m > 0) launch(k_lz_m<V, NT>, gA, NT, 0, s, A, la, (const V*)pu[cur], pz[cur] + w.n);
  const V* F = nullptr;
  if (w.r > 0) {
    F = lr_factor<V>(w);
    lowrank_ft<V, V>(w, F, (const V*)pz[cur], (const V*)nullptr, s);
  }
  if (F)
    launch(k_lz_n<V, NT, true>, gP, NT, 0, s, P, la, (const V*)pz[cur], (const V*)pu[cur], lw[0], lw[1],
           w.part_n, F, lr_weights<V>(w), w.r);
  else
    launch(k_lz_n<V, NT, false>, gP, NT, 0, s, P, la, (const V*)pz[cur], (const V*)pu[cur], lw[0], lw[1],
           w.part_n, F, lr_weights<V>(w), w.r);
  // the per-instance reductions read the chunk sums (a few hundred for the
  // largest instance), so 128 threads each suffice
  launch(k_lz_alpha<128>, w.count, 128, 0, s, la);
  launch(k_lz_orth<V>, cdiv(gP, 8), 256, 0, s, la, P, (const V*)lw[0], (const V*)lw[1], pu[cur], pu[prv],
         pz[cur], pz[prv], w.part_n);
  // the tridiagonals have t + 1 rows at step t: shared memory for that many
  // (the blocks per SM grow as the arrays shrink)
  const int kcap = (t + 1 + 3) & ~3;
  launch(k_lz_beta<128>, w.count, 128, (size_t)kcap * 2 * (3 * sizeof(double) + 2 * sizeof(float)), s, la,
         p.norm_tol, p.norm_iters < LZ_MAX ? p.norm_iters : LZ_MAX, kcap);
  if (!la.lazy) launch(k_lz_norm<V>, std::min(cdiv(w.n, 256), 4 * w.num_sms), 256, 0, s, la, pu[prv], pz[prv]);
}

// The norm estimates run at one width whatever the iteration kernels' variant
// (long rows are summed with the block's stride), so that variant never
// changes the step sizes.
void lanczos_step(Work& w, int t, const SolveParams& p, bool mixed, cudaStream_t s) {
  if (mixed) lanczos_step_t<float, 256>(w, t, p, w.A.bscaled_f(), w.P.bscaled_f(), w.fpu, w.fpz, w.flw, s);
  else lanczos_step_t<double, 256>(w, t, p, w.A.bscaled(), w.P.bscaled(), w.pu, w.pz, w.lw, s);
}

// the row blocks of the instances whose estimates are still running: of A
// where ||A|| is, of P where either is (the counts go to bst, read by the
// host at its next synchronisation)
__global__ void k_compact_lz(const int* __restrict__ blk_inst, int nblk, const DevState* __restrict__ st, int side,
                             int* __restrict__ act, int* __restrict__ n) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
    const DevState& S = st[blk_inst[b]];
    const bool run = side ? !(S.pi_done[0] && S.pi_done[1]) : !S.pi_done[0];
    if (run) act[atomicAdd(n, 1)] = b;
  }
}

void lanczos_compact(Work& w, cudaStream_t s) {
  cudaMemsetAsync(&w.bst->act_A, 0, 2 * sizeof(int), s);
  if (w.A.nblk > 0)
    launch(k_compact_lz, std::min(cdiv(w.A.nblk, 256), 4 * w.num_sms), 256, 0, s, (const int*)w.blk_inst_A, w.A.nblk,
           (const DevState*)w.st, 0, w.act_A, &w.bst->act_A);
  launch(k_compact_lz, std::min(cdiv(w.P.nblk, 256), 4 * w.num_sms), 256, 0, s, (const int*)w.blk_inst_P, w.P.nblk,
         (const DevState*)w.st, 1, w.act_P, &w.bst->act_P);
}

void count_running(Work& w, cudaStream_t s) {
  launch(k_count_running, 1, 256, 0, s, (const DevState*)w.st, (const Inst*)w.inst, (const int*)w.A.rp,
         (const int*)w.P.rp, w.count, w.bst);
}

void norms_finish(Work& w, double normA_opt, double normQ_opt, cudaStream_t s) {
  launch(k_set_norms, cdiv(w.count, 256), 256, 0, s, w.st, w.count, normA_opt, normQ_opt);
}

// dsc = [D2 of every member ; D1 of every member] from the template's [D2 ; D1]
__global__ void k_family_scaling(const double* __restrict__ t, int n_t, int m_t, long long N, long long total,
                                 double* __restrict__ dsc) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    dsc[i] = i < N ? t[i % n_t] : t[n_t + (i - N) % m_t];
}

__global__ void k_family_norms(const DevState* __restrict__ t, int count, DevState* __restrict__ sts) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    DevState* st = sts + i;
    st->normA = t->normA;
    st->normQ = t->normQ;
    st->pi_iters = t->pi_iters;
    for (int o = 0; o < 2; ++o) {
      st->pi_lam[o] = t->pi_lam[o];
      st->pi_done[o] = t->pi_done[o];
    }
  }
}

void family_scaling(Work& w, const Work& t, cudaStream_t s) {
  const long long N = (long long)w.n, total = N + w.m;
  launch(k_family_scaling, std::min(cdiv(total, 256), 8 * w.num_sms), 256, 0, s, (const double*)t.dsc, t.n, t.m, N,
         total, w.dsc);
}

void family_norms(Work& w, const Work& t, cudaStream_t s) {
  launch(k_family_norms, cdiv(w.count, 256), 256, 0, s, (const DevState*)t.st, w.count, w.st);
}

static MixedArgs mixed_args(Work& w) {
  MixedArgs a{};
  a.n = w.n; a.m = w.m;
  a.ineq = w.row_ineq; a.sts = w.st; a.inst_n = w.row_inst_n; a.inst_m = w.row_inst_m;
  a.cs = w.cs; a.bs = w.bs; a.ls = w.ls; a.us = w.us; a.D1 = w.D1; a.D2 = w.D2;
  a.xhi = w.xhi; a.yhi = w.yhi;
  a.fx = w.fx; a.fxbar = w.fxbar; a.fxt = w.fxt; a.fxmd0 = w.fZ[0]; a.fy = w.fy; a.fybar = w.fybar;
  a.fc = w.fc; a.fl = w.fl; a.fu = w.fu; a.fb = w.fb; a.fylo = w.fylo;
  a.x64[0] = w.x; a.x64[1] = w.xbar; a.y64[0] = w.yk; a.y64[1] = w.ybar;
  a.prodAx = w.prodAx; a.prodQx = w.prodQx; a.prodATy = w.prodATy;
  return a;
}

void init_iterates(Work& w, const double* x0, const double* y0, const SolveParams& p, cudaStream_t s) {
  launch(k_omega_part, w.P.nblk + w.A.nblk, 256, 0, s, (const int*)w.P.blk, w.P.nblk, (const int*)w.A.blk,
         (const double*)w.cs, (const double*)w.bs, w.part_n, w.part_m);
  launch(k_init_omega, w.count, 512, 0, s, w.st, (const Inst*)w.inst, (const double*)w.part_n,
         (const double*)w.part_m, p.eps_zero);
  const int N = w.n > w.m ? w.n : w.m;
  if (p.mixed) {
    w.fy = w.fZ[1] + w.n;
    w.y = w.yk;
    launch(k_init_mixed, cdiv(N, 256), 256, 0, s, mixed_args(w), x0, y0);
    return;
  }
  w.y = w.Z[1] + w.n;
  launch(k_init_iterates, cdiv(N, 256), 256, 0, s, w.n, w.m, (const unsigned char*)w.row_ineq, x0, y0,
         (const double*)w.D1,
         (const double*)w.D2, (const double*)w.ls, (const double*)w.us, w.x, w.xbar, w.Z[0], w.xt, w.ax, w.y,
         w.ybar, w.ay);
}

static KktB kkt_args(Work& w, bool scaled) {
  KktB a{};
  a.A = scaled ? w.A.bscaled() : w.A.borig();
  a.P = scaled ? w.P.bscaled() : w.P.borig();
  a.x[0] = w.x; a.x[1] = w.xbar; a.y[0] = w.y; a.y[1] = w.ybar;
  a.ax = w.ax; a.ay = w.ay;
  if (scaled) { a.D1 = w.D1; a.D2 = w.D2; a.iD1 = w.iD1; a.iD2 = w.iD2; }
  a.b = w.b; a.c = w.c; a.l = w.l; a.u = w.u;
  a.part_m = w.part_m; a.part_n = w.part_n;
  a.ngrp_m = w.ngrp_A; a.ngrp_n = w.ngrp_P;
  a.inst = w.inst;
  a.grp_inst_A = w.grp_inst_A; a.grp_first_A = w.grp_first_A;
  a.grp_inst_P = w.grp_inst_P; a.grp_first_P = w.grp_first_P;
  a.n = w.n; a.m = w.m;
  a.ineq = w.row_ineq;
  a.st = w.st;
  return a;
}

// ==========================================================================
// Infeasibility certificates (optional; not in the paper).  The rays are the
// current and the average iterate's displacement from the anchor the relKKT
// check measures restart distances from (the epoch's first iterate; in mixed
// precision the float64 base), projected onto the recession cones of X (0
// where both bounds are finite, [0, inf) where only l is, (-inf, 0] where
// only u is) and of Y (y_I >= 0).  Their tests are relKKT quantities of
// homogeneous problems, so the relKKT kernels evaluate them on the original
// problem: a primal ray d with b = 0 and the recession cone as the box gives
// the violation of A d, |Qd|_inf and c'd; a dual ray y with x = 0 and c = 0
// gives b'y + l'lam+ - u'lam- (lam = proj_Lambda(-A'y)), the Farkas value
// b'y - sup_{x in X} (A'y)'x where -A'y lies in Lambda, and |-A'y - lam|_inf,
// what leaves Lambda, as the dual residual.
// ==========================================================================
__global__ void k_rec_bounds(int n, const double* __restrict__ l, const double* __restrict__ u,
                             double* __restrict__ lrec, double* __restrict__ urec) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    lrec[i] = isfinite(l[i]) ? 0.0 : -INFINITY;
    urec[i] = isfinite(u[i]) ? 0.0 : INFINITY;
  }
}

// Rays of the instances still running (the rows of the others keep the
// certificate they ended with).
__global__ void k_rays(int n, int m, const DevState* __restrict__ st, const int* __restrict__ inst_n,
                       const int* __restrict__ inst_m, const unsigned char* __restrict__ ineq,
                       const double* __restrict__ l, const double* __restrict__ u, const double* __restrict__ x0,
                       const double* __restrict__ x1, const double* __restrict__ ax, const double* __restrict__ y0,
                       const double* __restrict__ y1, const double* __restrict__ ay, double* __restrict__ rx0,
                       double* __restrict__ rx1, double* __restrict__ ry0, double* __restrict__ ry1) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(n, m); i += gridDim.x * blockDim.x) {
    if (i < n && st[inst_n[i]].status == ST_RUNNING) {
      const bool lo = isfinite(l[i]), up = isfinite(u[i]);
      double d0 = x0[i] - ax[i], d1 = x1[i] - ax[i];
      if (lo && up) { d0 = 0.0; d1 = 0.0; }
      else if (lo) { d0 = fmax(d0, 0.0); d1 = fmax(d1, 0.0); }
      else if (up) { d0 = fmin(d0, 0.0); d1 = fmin(d1, 0.0); }
      rx0[i] = d0;
      rx1[i] = d1;
    }
    if (i < m && st[inst_m[i]].status == ST_RUNNING) {
      double r0 = y0[i] - ay[i], r1 = y1[i] - ay[i];
      if (ineq[i]) { r0 = fmax(r0, 0.0); r1 = fmax(r1, 0.0); }
      ry0[i] = r0;
      ry1[i] = r1;
    }
  }
}

// PASS 0 (primal rays): d passes if c'd < 0 and max(|viol(A d)|_inf,
// |Qd|_inf) <= eps |c'd|.  PASS 1 (dual rays): y passes if its Farkas value
// v > 0 and the residual <= eps v; then the instance's status: primal
// infeasible if a dual ray passed, else dual infeasible if a primal ray did
// (the current iterate's ray before the average's).
template <int PASS>
__global__ void __launch_bounds__(64) k_infeas(InfState* __restrict__ inf, const DevState* __restrict__ sts,
                                               const Inst* __restrict__ insts, const double* __restrict__ pm,
                                               int nbm, const double* __restrict__ pn, int nbn, double eps) {
  const int i = blockIdx.x;
  if (sts[i].status != ST_RUNNING) return;     // uniform
  const Inst in = insts[i];
  __shared__ double F[24];
  reduce_kkt_blocks(pm, nbm, in.cA0, in.m > 0 ? in.cA0 + kkt_chunks(in.bA0, in.bA1) : in.cA0, pn, nbn, in.cP0,
                    in.cP0 + kkt_chunks(in.bP0, in.bP1), F);
  if (threadIdx.x != 0) return;
  InfState& I = inf[i];
  if (PASS == 0) {
    I.dual_it = -1;
    I.dual_scale = 0.0;
    for (int it = 0; it < 2; ++it) {
      const double viol = F[it * 4 + 0], qd = F[9 + it * 7 + 1], cd = F[9 + it * 7 + 4];
      if (cd < 0.0 && fmax(viol, qd) <= eps * -cd) {
        I.dual_it = it;
        I.dual_scale = -cd;
        break;
      }
    }
  } else {
    I.status = 0;
    for (int it = 0; it < 2; ++it) {
      const double res = F[9 + it * 7 + 0], v = F[it * 4 + 2] + F[9 + it * 7 + 5];
      if (v > 0.0 && res <= eps * v) {
        I.status = ST_PRIMAL_INF;
        I.cert_it = it;
        I.scale = v;
        break;
      }
    }
    if (!I.status && I.dual_it >= 0) {
      I.status = ST_DUAL_INF;
      I.cert_it = I.dual_it;
      I.scale = I.dual_scale;
    }
  }
}

// The normalised certificate of every instance that ended infeasible, in
// original coordinates, over its rows of x_out / y_out (the other vector 0).
__global__ void k_write_cert(int n, int m, const double* __restrict__ D1, const double* __restrict__ D2,
                             const DevState* __restrict__ st, const InfState* __restrict__ inf,
                             const int* __restrict__ inst_n, const int* __restrict__ inst_m,
                             const double* __restrict__ rx0, const double* __restrict__ rx1,
                             const double* __restrict__ ry0, const double* __restrict__ ry1,
                             double* __restrict__ x_out, double* __restrict__ y_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(n, m); i += gridDim.x * blockDim.x) {
    if (i < n && x_out) {
      const int k = inst_n[i], s = st[k].status;
      if (s == ST_PRIMAL_INF) x_out[i] = 0.0;
      else if (s == ST_DUAL_INF) x_out[i] = D2[i] * (inf[k].cert_it ? rx1 : rx0)[i] / inf[k].scale;
    }
    if (i < m && y_out) {
      const int k = inst_m[i], s = st[k].status;
      if (s == ST_DUAL_INF) y_out[i] = 0.0;
      else if (s == ST_PRIMAL_INF) y_out[i] = D1[i] * (inf[k].cert_it ? ry1 : ry0)[i] / inf[k].scale;
    }
  }
}

// Both passes over the rays of the iterates the check's relKKT pass `main`
// read (and its anchors).
static void infeas_check(Work& w, const KktB& main, cudaStream_t s) {
  const int NN = w.n > w.m ? w.n : w.m;
  const int grid_v = cdiv(NN, 256) < 4 * w.num_sms ? cdiv(NN, 256) : 4 * w.num_sms;
  launch(k_rays, grid_v, 256, 0, s, w.n, w.m, (const DevState*)w.st, (const int*)w.row_inst_n,
         (const int*)w.row_inst_m, (const unsigned char*)w.row_ineq, (const double*)w.l, (const double*)w.u,
         main.x[0], main.x[1], main.ax, main.y[0], main.y[1], main.ay, w.inf_x[0], w.inf_x[1], w.inf_y[0],
         w.inf_y[1]);
  const dim3 cgrid(w.count, std::max(w.maxchunk_n, w.maxchunk_m));
  for (int pass = 0; pass < 2; ++pass) {
    KktB a = kkt_args(w, true);
    a.part_m = w.inf_part_m;
    a.part_n = w.inf_part_n;
    a.ax = w.inf_zn;
    a.ay = w.inf_zm;
    if (pass == 0) {   // primal rays: b = 0, the box's recession cone as the box
      a.x[0] = w.inf_x[0]; a.x[1] = w.inf_x[1];
      a.y[0] = w.inf_zm; a.y[1] = w.inf_zm;
      a.b = w.inf_zm; a.l = w.inf_lrec; a.u = w.inf_urec;
      if (w.r > 0) {
        lowrank_ft<double, double>(w, w.Fd, a.x[0], a.x[1], s);
        a.F = w.Fd; a.wlr = w.wlr; a.r = w.r;
      }
    } else {           // dual rays: x = 0, c = 0
      a.x[0] = w.inf_zn; a.x[1] = w.inf_zn;
      a.y[0] = w.inf_y[0]; a.y[1] = w.inf_y[1];
      a.c = w.inf_zn;
    }
    launch_kkt<2>(w, a, s);
    launch(k_kkt_chunks, cgrid, 32, 0, s, (const Inst*)w.inst, (const int*)w.grp_first_A,
           (const double*)w.inf_part_m, w.ngrp_A, (const int*)w.grp_first_P, (const double*)w.inf_part_n,
           w.ngrp_P, w.inf_cpart_m, std::max(w.nchunk_m, 1), w.inf_cpart_n, std::max(w.nchunk_n, 1));
    if (pass == 0)
      launch(k_infeas<0>, w.count, 64, 0, s, w.inf, (const DevState*)w.st, (const Inst*)w.inst,
             (const double*)w.inf_cpart_m, std::max(w.nchunk_m, 1), (const double*)w.inf_cpart_n,
             std::max(w.nchunk_n, 1), w.eps_inf);
    else
      launch(k_infeas<1>, w.count, 64, 0, s, w.inf, (const DevState*)w.st, (const Inst*)w.inst,
             (const double*)w.inf_cpart_m, std::max(w.nchunk_m, 1), (const double*)w.inf_cpart_n,
             std::max(w.nchunk_n, 1), w.eps_inf);
  }
}

void infeas_prepare(Work& w, cudaStream_t s) {
  launch(k_rec_bounds, cdiv(w.n, 256), 256, 0, s, w.n, (const double*)w.l, (const double*)w.u, w.inf_lrec,
         w.inf_urec);
}

void write_certificates(Work& w, double* x_out, double* y_out, cudaStream_t s) {
  if (!w.detect || !w.inf || (!x_out && !y_out)) return;
  const int N = w.n > w.m ? w.n : w.m;
  launch(k_write_cert, cdiv(N, 256), 256, 0, s, w.n, w.m, (const double*)w.D1, (const double*)w.D2,
         (const DevState*)w.st, (const InfState*)w.inf, (const int*)w.row_inst_n, (const int*)w.row_inst_m,
         (const double*)w.inf_x[0], (const double*)w.inf_x[1], (const double*)w.inf_y[0],
         (const double*)w.inf_y[1], x_out, y_out);
}

void check(Work& w, const SolveParams& p, int mode, long long chunk_len, bool mixed, cudaStream_t s) {
  if (w.prof.on) w.prof.begin(2, s);
  const int NN = w.n > w.m ? w.n : w.m;
  const int grid_v = cdiv(NN, 256) < 4 * w.num_sms ? cdiv(NN, 256) : 4 * w.num_sms;
  const bool mp = w.mp && !mixed && !w.il_active;   // products maintained by the iteration
  const bool pairs = !w.il_active && w.kkt_xx && !mp;
  if (mixed) {
    MixedArgs ma = mixed_args(w);
    if (pairs) { ma.xx = w.kkt_xx; ma.yy = w.kkt_yy; }
    launch(k_materialize, grid_v, 256, 0, s, ma);
  } else if (pairs) {
    launch(k_pair_iterates, grid_v, 256, 0, s, w.n, w.m, (const double*)w.x, (const double*)w.xbar,
           (const double*)w.y, (const double*)w.ybar, w.kkt_xx, w.kkt_yy);
  }
  KktB a = kkt_args(w, true);
  if (pairs) { a.xx = w.kkt_xx; a.yy = w.kkt_yy; }
  if (mixed) {
    a.ax = w.xhi; a.ay = w.yhi;
    for (int it = 0; it < 2; ++it) {
      a.prodAx[it] = w.prodAx + (size_t)it * w.m;
      a.prodQx[it] = w.prodQx + (size_t)it * w.n;
      a.prodATy[it] = w.prodATy + (size_t)it * w.n;
    }
  }
  if (w.r > 0) {
    lowrank_ft<double, double>(w, w.Fd, a.x[0], a.x[1], s);
    a.F = w.Fd; a.wlr = w.wlr; a.r = w.r;
  }
  if (w.il_active) {
    launch_kkt_il(w, a, s);   // a family handle on interleaved vectors (no low-rank term)
  } else if (mp) {            // row sums from the maintained products and one gather of x each for A x, Q x
    mp_check_products(w, mode, chunk_len, s);
    if (w.m > 0) launch(k_kkt_m_sums, w.ngrp_A, BNT, 0, s, a, (const double*)w.mp_sA[0], (const double*)w.mp_sA[1]);
    launch(k_kkt_n_sums, w.ngrp_P, BNT, 0, s, a, (const double*)w.mp_sQ[0], (const double*)w.mp_sQ[1],
           (const double*)w.mp_aty, (const double*)w.mp_atyb);
  } else {
    launch_kkt<2>(w, a, s);
  }
  {
    const dim3 grid(w.count, std::max(w.maxchunk_n, w.maxchunk_m));
    launch(k_kkt_chunks, grid, 32, 0, s, (const Inst*)w.inst, (const int*)w.grp_first_A, (const double*)w.part_m,
           w.ngrp_A, (const int*)w.grp_first_P, (const double*)w.part_n, w.ngrp_P, w.cpart_m,
           std::max(w.nchunk_m, 1), w.cpart_n, std::max(w.nchunk_n, 1));
  }
  const bool certify = w.detect && w.inf && mode == 1;
  if (certify) infeas_check(w, a, s);
  launch(k_decide, w.count, 64, 0, s, w.st, (const Inst*)w.inst, (const double*)w.cpart_m,
         std::max(w.nchunk_m, 1), (const double*)w.cpart_n, std::max(w.nchunk_n, 1), w.tab, w.tab_stride, p, mode,
         chunk_len, certify ? (const InfState*)w.inf : (const InfState*)nullptr);
  if (mixed) {
    launch(k_mixed_rebase, grid_v, 256, 0, s, mixed_args(w), mode == 0 ? 1 : 0);
  } else if (mode == 1) {
    launch(k_restart_apply, grid_v, 256, 0, s, (const DevState*)w.st, (const int*)w.row_inst_n,
           (const int*)w.row_inst_m, w.n, w.m, w.x, w.xbar, w.Z[0], w.xt, w.ax, w.y, w.ybar, w.ay);
  }
  launch(k_count_running, 1, 256, 0, s, (const DevState*)w.st, (const Inst*)w.inst, (const int*)w.A.rp,
         (const int*)w.P.rp, w.count, w.bst);
  if (w.count > 1) {   // the running instances' row blocks, for compacted launches
    cudaMemsetAsync(&w.bst->act_A, 0, 2 * sizeof(int), s);
    // -1 past the count: the padding blocks of a replayed compacted grid skip
    if (w.A.nblk > 0) cudaMemsetAsync(w.act_A, 0xFF, (size_t)w.A.nblk * sizeof(int), s);
    cudaMemsetAsync(w.act_P, 0xFF, (size_t)w.P.nblk * sizeof(int), s);
    if (w.A.nblk > 0)
      launch(k_compact_blocks, std::min(cdiv(w.A.nblk, 256), 4 * w.num_sms), 256, 0, s, (const int*)w.blk_inst_A,
             w.A.nblk, (const DevState*)w.st, w.act_A, &w.bst->act_A);
    launch(k_compact_blocks, std::min(cdiv(w.P.nblk, 256), 4 * w.num_sms), 256, 0, s, (const int*)w.blk_inst_P,
           w.P.nblk, (const DevState*)w.st, w.act_P, &w.bst->act_P);
  }
  if (w.prof.on) w.prof.end(s);
}

void write_output(Work& w, double* x_out, double* y_out, cudaStream_t s) {
  const int N = w.n > w.m ? w.n : w.m;
  launch(k_unscale_out, cdiv(N, 256), 256, 0, s, w.n, w.m, (const double*)w.D1, (const double*)w.D2,
         (const double*)w.x, (const double*)w.xbar, (const double*)w.y, (const double*)w.ybar,
         (const DevState*)w.st, (const int*)w.row_inst_n, (const int*)w.row_inst_m, -1, x_out, y_out);
}

void write_state(Work& w, double* x, double* y, double* xbar, double* ybar, cudaStream_t s) {
  const int N = w.n > w.m ? w.n : w.m;
  launch(k_unscale_out, cdiv(N, 256), 256, 0, s, w.n, w.m, (const double*)w.D1, (const double*)w.D2,
         (const double*)w.x, (const double*)w.xbar, (const double*)w.y, (const double*)w.ybar,
         (const DevState*)w.st, (const int*)w.row_inst_n, (const int*)w.row_inst_m, 0, x, y);
  launch(k_unscale_out, cdiv(N, 256), 256, 0, s, w.n, w.m, (const double*)w.D1, (const double*)w.D2,
         (const double*)w.x, (const double*)w.xbar, (const double*)w.y, (const double*)w.ybar,
         (const DevState*)w.st, (const int*)w.row_inst_n, (const int*)w.row_inst_m, 1, xbar, ybar);
}

// relKKT of a user (x, y) on the original matrices (D = 1)
__global__ void __launch_bounds__(1024) k_kkt_finish_user(const double* __restrict__ pm, int nbm,
                                                          const double* __restrict__ pn, int nbn, DevState* st) {
  __shared__ double F[24];
  reduce_kkt_blocks(pm, nbm, 0, nbm, pn, nbn, 0, nbn, F);
  if (threadIdx.x == 0) kkt_from_fields(F, 0, st->out_parts);
}

void eval_kkt_user(Work& w, const double* x, const double* y, cudaStream_t s) {
  KktB a = kkt_args(w, false);
  a.x[0] = x; a.x[1] = x; a.y[0] = y; a.y[1] = y;
  a.ax = nullptr; a.ay = nullptr;
  a.st = nullptr;
  if (w.r > 0) {
    lowrank_ft<double, double>(w, w.Fo, x, (const double*)nullptr, s);
    a.F = w.Fo; a.wlr = w.wlr; a.r = w.r;
  }
  launch_kkt<1>(w, a, s);
  launch(k_kkt_finish_user, 1, 1024, 0, s, (const double*)w.part_m, w.m > 0 ? w.ngrp_A : 0,
         (const double*)w.part_n, w.ngrp_P, w.st);
}

}  // namespace pdqp

// ---------------------------------------------------------------- profiler
void Profiler::begin(int k, cudaStream_t s, double b) {
  const size_t need = 2 * (kind.size() + 1);
  while (ev.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
    ev.push_back(e);
  }
  cudaEventRecord(ev[2 * kind.size()], s);
  kind.push_back(k);
  kbytes.push_back(b);
}
void Profiler::end(cudaStream_t s) {
  if (kind.empty()) return;
  cudaEventRecord(ev[2 * kind.size() - 1], s);
}
void Profiler::harvest() {
  for (size_t i = 0; i < kind.size(); ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
      ms[kind[i]] += t;
      launches[kind[i]] += 1;
      bytes[kind[i]] += kbytes[i];
    } else {
      cudaGetLastError();   // a failed timing query must not surface as a later error
    }
  }
  kind.clear();
  kbytes.clear();
}
void Profiler::reset() {
  kind.clear();
  kbytes.clear();
  for (int i = 0; i < 4; ++i) { launches[i] = 0; ms[i] = 0.0; bytes[i] = 0.0; }
}
Profiler::~Profiler() {
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
}

// ==========================================================================
// Allocation-free relative-KKT evaluation: pdqp_kkt_noalloc.
//
// Some callers cannot call cudaMalloc once they are running: a real-time
// control loop (for example an MPC controller re-solving every few
// milliseconds) must not block on the allocator or synchronise the device,
// and a host process with a fixed device-memory budget may not allocate at
// all after start-up.  This entry point
// evaluates the relative KKT error of a caller-given (x, y) with caller-owned
// device arrays only; its per-block partial sums live in the file-scope array
// below, which every GPU that loads this library holds until the process exits.
// ==========================================================================
#include <mutex>

#include "pdqp.h"

#define PDQP_NOALLOC_MAX_ROWS 65536                          // max n and max m per call
#define PDQP_NOALLOC_MAX_BLOCKS (PDQP_NOALLOC_MAX_ROWS / 8)  // a block covers >= 8 rows
#define PDQP_NOALLOC_MAX_DEVICES 64
// a block of 256 threads covers 256 / L rows with L <= 32 lanes per row
// (pick_lanes), so at most MAX_ROWS / 8 blocks ever touch the scratch
static_assert(PDQP_NOALLOC_MAX_BLOCKS * (256 / 32) >= PDQP_NOALLOC_MAX_ROWS, "noalloc scratch too small");

// 8192 blocks x 32 partial sums x 8 bytes = 2 MiB per device.
static __device__ __align__(256) double g_noalloc_scratch[PDQP_NOALLOC_MAX_BLOCKS * 32];

static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[PDQP_NOALLOC_MAX_DEVICES] = {};

// The variant of the finishing step that writes the six parts to caller memory.
__global__ void k_kkt_finish_noalloc(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  __shared__ double F[24];
  pdqp::reduce_kkt_partials(part, nblk, F);
  if (threadIdx.x == 0) pdqp::kkt_from_fields(F, 0, out);
}

extern "C" pdqp_status pdqp_kkt_noalloc(int64_t n, int64_t m, int64_t m_eq, const int32_t* Q_rowptr,
                                        const int32_t* Q_col, const double* Q_val, int64_t nnz_Q,
                                        const int32_t* A_rowptr, const int32_t* A_col, const double* A_val,
                                        const int32_t* At_rowptr, const int32_t* At_col, const double* At_val,
                                        int64_t nnz_A, const double* c, const double* b, const double* l,
                                        const double* u, const double* x, const double* y, double* parts,
                                        void* stream) {
  if (n < 1 || n > PDQP_NOALLOC_MAX_ROWS || m < 0 || m > PDQP_NOALLOC_MAX_ROWS || m_eq < 0 || m_eq > m ||
      nnz_Q < 0 || nnz_A < 0 || nnz_Q > INT32_MAX || nnz_A > INT32_MAX)
    return PDQP_ERR_INVALID;   // sizes beyond 65536 rows do not fit the static scratch
  if (!Q_rowptr || (nnz_Q > 0 && (!Q_col || !Q_val)) || !c || !l || !u || !x || !parts)
    return PDQP_ERR_INVALID;
  if (m > 0 && (!A_rowptr || !At_rowptr || !b || !y || (nnz_A > 0 && (!A_col || !A_val || !At_col || !At_val))))
    return PDQP_ERR_INVALID;
  // every array the kernels touch must be device (or managed) memory: a host
  // pointer would make them fault.  The query allocates nothing.
  {
    const void* ptrs[] = {Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, At_rowptr, At_col, At_val,
                          c, b, l, u, x, y, parts};
    for (const void* p : ptrs) {
      if (!p) continue;
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return PDQP_ERR_INVALID;
      }
      if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return PDQP_ERR_INVALID;
    }
  }
  // an error left pending by earlier work on this thread is not ours: leave it
  // for the caller to read and launch nothing
  if (cudaPeekAtLastError() != cudaSuccess) return PDQP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= PDQP_NOALLOC_MAX_DEVICES) return PDQP_ERR_CUDA;
  double* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the array
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PDQP_ERR_CUDA;
      }
      g_noalloc_addr[dev] = (double*)p;
    }
    scratch = g_noalloc_addr[dev];
  }
  const int LA = pdqp::pick_lanes(nnz_A, m);
  const int LN = pdqp::pick_lanes(nnz_Q + nnz_A, n);
  const int gm = m > 0 ? pdqp::cdiv(m, 256 / LA) : 0;
  const int gn = pdqp::cdiv(n, 256 / LN);
  const int nblk = gm > gn ? gm : gn;
  if (nblk > PDQP_NOALLOC_MAX_BLOCKS) return PDQP_ERR_INVALID;   // unreachable by the sizes above
  // blocks that one of the two kernels does not launch contribute zeros
  if (cudaMemsetAsync(scratch, 0, (size_t)nblk * 32 * sizeof(double), s) != cudaSuccess) return PDQP_ERR_CUDA;
  pdqp::KktArgs a{};
  a.A = Csr<double>{A_rowptr, A_col, A_val};
  a.Q = Csr<double>{Q_rowptr, Q_col, Q_val};
  a.At = Csr<double>{At_rowptr, At_col, At_val};
  a.x[0] = x; a.x[1] = x; a.y[0] = y; a.y[1] = y;
  a.b = b; a.c = c; a.l = l; a.u = u;
  a.part = scratch;
  a.n = (int)n; a.m = (int)m; a.m_eq = (int)m_eq;
  if (gm > 0) { DISPATCH_L(LA, pdqp::launch(pdqp::k_kkt_m<LL, 1, false>, gm, 256, 0, s, a)); }
  DISPATCH_L(LN, pdqp::launch(pdqp::k_kkt_n<LL, 1, false>, gn, 256, 0, s, a));
  pdqp::launch(k_kkt_finish_noalloc, 1, 256, 0, s, (const double*)scratch, nblk, parts);
  return cudaGetLastError() == cudaSuccess ? PDQP_OK : PDQP_ERR_CUDA;
}
