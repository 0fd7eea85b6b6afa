// The inner iteration of Algorithm 1 (Section 2) as two fused row-block
// kernels per iteration:
//   k_dual   : rows of A   -- v = A x_tilde, y+ = proj_Y(y - sigma (v - b)),
//              y_bar+ = (1 - 1/beta) y_bar + y+/beta
//   k_primal : rows of P = [Q | -A'] gathering [x_md ; y+] -- g = Q x_md + c - A'y+,
//              x+ = proj_[l,u](x - tau g), x_bar+ = (1 - 1/beta) x_bar + x+/beta,
//              and the next iteration's x_md and x_tilde
// with their pipelined persistent variants, the segment sums of long rows,
// and the host loop that launches a chunk of iterations.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "rowblock.cuh"

namespace cg = cooperative_groups;

namespace pdqp {

// --------------------------------------------------------------------------
// One inner iteration of Algorithm 1: the dual half-step (rows of A)
// --------------------------------------------------------------------------
template <typename V>
struct DualB {
  BCsr<V> A;
  const V* __restrict__ xt;      // extrapolated primal point x_tilde
  const V* __restrict__ yold;    // y^k
  V* __restrict__ ynew;          // y^{k+1}
  V* __restrict__ ybar;
  const V* __restrict__ b;
  const V* __restrict__ ylo;     // lower bound of inequality duals (mixed-mode shift) or null (0)
  const StepEntry* __restrict__ tab;    // [instance][C]
  const int* __restrict__ blk_inst;     // instance of each row block
  const DevState* __restrict__ st;      // per instance
  const unsigned char* __restrict__ ineq;   // per row: inequality
  int C;
  const int2* __restrict__ blk_seg;     // long rows: {first segment, segments} per block (null: none)
  const V* __restrict__ lpart;          // segment sums of the long rows
  const int* __restrict__ act;          // row block of each CUDA block (null: the block index)
};

template <typename V> __device__ __forceinline__ V step_sigma(const StepEntry& e);
template <> __device__ __forceinline__ double step_sigma<double>(const StepEntry& e) { return e.sigma_d; }
template <> __device__ __forceinline__ float step_sigma<float>(const StepEntry& e) { return e.sigma_d_f; }
template <typename V> __device__ __forceinline__ V step_tau(const StepEntry& e);
template <> __device__ __forceinline__ double step_tau<double>(const StepEntry& e) { return e.tau_p; }
template <> __device__ __forceinline__ float step_tau<float>(const StepEntry& e) { return e.tau_p_f; }
template <typename V> __device__ __forceinline__ V step_ib(const StepEntry& e);
template <> __device__ __forceinline__ double step_ib<double>(const StepEntry& e) { return e.inv_beta; }
template <> __device__ __forceinline__ float step_ib<float>(const StepEntry& e) { return e.inv_beta_f; }
template <typename V> __device__ __forceinline__ V step_ibn(const StepEntry& e);
template <> __device__ __forceinline__ double step_ibn<double>(const StepEntry& e) { return e.inv_beta_next; }
template <> __device__ __forceinline__ float step_ibn<float>(const StepEntry& e) { return e.inv_beta_next_f; }
template <typename V> __device__ __forceinline__ V step_thn(const StepEntry& e);
template <> __device__ __forceinline__ double step_thn<double>(const StepEntry& e) { return e.theta_next; }
template <> __device__ __forceinline__ float step_thn<float>(const StepEntry& e) { return e.theta_next_f; }

// The dual update of one row from its sum s = (A x_tilde)_r: y+ and y_bar+
// (shared by the row-block and the member-interleaved kernels).
template <typename V>
__device__ __forceinline__ void dual_update(const StepEntry& e, V s, V yo, V bi, V yb, V lo, bool ineq, V& yn,
                                            V& ybn) {
  const V sigma = step_sigma<V>(e), ib = step_ib<V>(e);
  yn = r_fma(-sigma, r_sub(s, bi), yo);                       // y - sigma (A x_tilde - b)
  if (ineq) yn = fmax(yn, lo);
  ybn = r_fma(ib, yn, r_mul(r_sub(V(1), ib), yb));            // (1 - 1/beta) y_bar + y+/beta
}

template <typename V>
__device__ __forceinline__ void dual_row(const DualB<V>& a, const StepEntry& e, int r, V s, V yo, V bi, V yb,
                                         V lo) {
  V yn, ybn;
  dual_update<V>(e, s, yo, bi, yb, lo, a.ineq[r] != 0, yn, ybn);
  a.ybar[r] = ybn;
  a.ynew[r] = yn;
}

// The dual half-step of row block bk (one CUDA block): prod and srp are the
// block's staging buffers; GM is how x_tilde is gathered (see stage_products).
template <typename V, int NT, int GM>
__device__ __forceinline__ void dual_block(const DualB<V>& a, int bk, int j, V* prod, int* srp) {
  const int tid = threadIdx.x;
  const int inst = a.blk_inst[bk];
  if (a.st[inst].status != ST_RUNNING) return;    // uniform over the block
  const int r0 = a.A.blk[bk], r1 = a.A.blk[bk + 1];
  const int nr = r1 - r0;
  const int e0 = a.A.rp[r0];
  const int ne = a.A.rp[r1] - e0;
  // operands of this thread's first row, fetched before the SpMV
  V yo = V(0), bi = V(0), yb = V(0), lo = V(0);
  if (tid < nr) {
    const int r = r0 + tid;
    yo = a.yold[r]; bi = a.b[r]; yb = a.ybar[r];
    if (a.ylo) lo = a.ylo[r];
  }
  const StepEntry& es = a.tab[inst * a.C + j];
  if (ne <= BNNZ) {
    stage_products<NT, GM>(a.A, a.xt, e0, ne, r0, nr, prod, srp);
    __syncthreads();
    for (int t = tid; t < nr; t += NT) {
      V s = V(0);
      for (int e = srp[t]; e < srp[t + 1]; ++e) s += prod[e];
      const int r = r0 + t;
      if (t >= BNT) {
        yo = a.yold[r]; bi = a.b[r]; yb = a.ybar[r];
        lo = a.ylo ? a.ylo[r] : V(0);
      }
      dual_row(a, es, r, s, yo, bi, yb, lo);
    }
  } else if (a.blk_seg) {   // a long row: the sum of its segments (k_long_partials), in order
    if (tid == 0) {
      const int2 sg = a.blk_seg[bk];
      V s = V(0);
      for (int q = 0; q < sg.y; ++q) s += a.lpart[sg.x + q];
      dual_row(a, es, r0, s, yo, bi, yb, lo);
    }
  } else {   // a single row longer than a block
    V s = V(0);
    for (int e = e0 + tid; e < e0 + ne; e += NT)
      s += a.A.val[e] * gather_load<GM>(a.xt + a.A.col[e]);
    s = block_sum(s);
    if (tid == 0) dual_row(a, es, r0, s, yo, bi, yb, lo);
  }
}

template <typename V, int NT>
__global__ void __launch_bounds__(NT, MinBlocks<V, NT>::value) k_dual(DualB<V> a, int j) {
  __shared__ V prod[BNNZ];
  __shared__ int srp[BROWS + 1];
  const int bk = a.act ? a.act[blockIdx.x] : (int)blockIdx.x;   // compacted batches: running blocks only
  if (bk < 0) return;                                             // padding of a compacted grid
  dual_block<V, NT, GATHER_LDG>(a, bk, j, prod, srp);
}

// --------------------------------------------------------------------------
// One inner iteration of Algorithm 1: the primal half-step (rows of P)
// --------------------------------------------------------------------------
template <typename V>
struct PrimalB {
  BCsr<V> P;
  const V* __restrict__ zin;     // [x_md ; y^{k+1}] of this iteration
  V* __restrict__ zout;          // x_md of the next iteration -> zout[0:n]
  V* __restrict__ x;
  V* __restrict__ xbar;
  V* __restrict__ xt;            // x_tilde of the next iteration
  const V* __restrict__ c;
  const V* __restrict__ l;
  const V* __restrict__ u;
  const StepEntry* __restrict__ tab;    // [instance][C]
  const int* __restrict__ blk_inst;
  const DevState* __restrict__ st;
  int C;
  const V* __restrict__ F;              // low-rank factor F~ (null: none)
  const V* __restrict__ wlr;            // F~' x_md of this iteration
  int r;
  const int2* __restrict__ blk_seg;     // long rows: {first segment, segments} per block (null: none)
  const V* __restrict__ lpart;          // segment sums of the long rows
  const int* __restrict__ act;          // row block of each CUDA block (null: the block index)
};

// The primal update of one row from g = (Q x_md - A'y+)_r + c_r (+ the
// low-rank term): x+, x_bar+ and the next iteration's x_md and x_tilde
// (shared by the row-block and the member-interleaved kernels).
template <typename V>
__device__ __forceinline__ void primal_update(const StepEntry& e, V g, V xo, V xb0, V lr, V ur, V& xn, V& xb, V& zo,
                                              V& xtn) {
  const V tau = step_tau<V>(e), ib = step_ib<V>(e), ibn = step_ibn<V>(e), thn = step_thn<V>(e);
  xn = fmin(fmax(r_fma(-tau, g, xo), lr), ur);               // proj_X(x - tau g)
  xb = r_fma(ib, xn, r_mul(r_sub(V(1), ib), xb0));            // (1 - 1/beta) x_bar + x+/beta
  zo = r_fma(ibn, xn, r_mul(r_sub(V(1), ibn), xb));           // next x_md
  xtn = r_fma(thn, r_sub(xn, xo), xn);                        // next x_tilde
}

template <typename V, bool LR = false>
__device__ __forceinline__ void primal_row(const PrimalB<V>& a, const StepEntry& e, int r, V s, V xo, V xb0,
                                           V cr, V lr, V ur) {
  V g = r_add(s, cr);
  if constexpr (LR) g = r_add(g, lr_row<V, V, V>(a.F, a.wlr, a.r, r));
  V xn, xb, zo, xtn;
  primal_update<V>(e, g, xo, xb0, lr, ur, xn, xb, zo, xtn);
  a.xbar[r] = xb;
  a.zout[r] = zo;
  a.xt[r] = xtn;
  a.x[r] = xn;
}

// The primal half-step of row block bk (one CUDA block), as dual_block.
template <typename V, int NT, bool LR, int GM>
__device__ __forceinline__ void primal_block(const PrimalB<V>& a, int bk, int j, V* prod, int* srp) {
  const int tid = threadIdx.x;
  const int inst = a.blk_inst[bk];
  if (a.st[inst].status != ST_RUNNING) return;    // uniform over the block
  const int r0 = a.P.blk[bk], r1 = a.P.blk[bk + 1];
  const int nr = r1 - r0;
  const int e0 = a.P.rp[r0];
  const int ne = a.P.rp[r1] - e0;
  V xo = V(0), xb = V(0), cr = V(0), lr = V(0), ur = V(0);
  if (tid < nr) {
    const int r = r0 + tid;
    xo = a.x[r]; xb = a.xbar[r]; cr = a.c[r]; lr = a.l[r]; ur = a.u[r];
  }
  const StepEntry& es = a.tab[inst * a.C + j];
  if (ne <= BNNZ) {
    stage_products<NT, GM>(a.P, a.zin, e0, ne, r0, nr, prod, srp);
    __syncthreads();
    for (int t = tid; t < nr; t += NT) {
      V s = V(0);
      for (int e = srp[t]; e < srp[t + 1]; ++e) s += prod[e];
      const int r = r0 + t;
      if (t >= BNT) { xo = a.x[r]; xb = a.xbar[r]; cr = a.c[r]; lr = a.l[r]; ur = a.u[r]; }
      primal_row<V, LR>(a, es, r, s, xo, xb, cr, lr, ur);
    }
  } else if (a.blk_seg) {
    if (tid == 0) {
      const int2 sg = a.blk_seg[bk];
      V s = V(0);
      for (int q = 0; q < sg.y; ++q) s += a.lpart[sg.x + q];
      primal_row<V, LR>(a, es, r0, s, xo, xb, cr, lr, ur);
    }
  } else {
    V s = V(0);
    for (int e = e0 + tid; e < e0 + ne; e += NT)
      s += a.P.val[e] * gather_load<GM>(a.zin + a.P.col[e]);
    s = block_sum(s);
    if (tid == 0) primal_row<V, LR>(a, es, r0, s, xo, xb, cr, lr, ur);
  }
}

// LR: the problem has a low-rank term (its row term gets its own instantiation
// so that the plain kernel keeps its 32 registers)
template <typename V, int NT, bool LR = false>
__global__ void __launch_bounds__(NT, MinBlocks<V, NT, LR>::value) k_primal(PrimalB<V> a, int j) {
  __shared__ V prod[BNNZ];
  __shared__ int srp[BROWS + 1];
  const int bk = a.act ? a.act[blockIdx.x] : (int)blockIdx.x;
  if (bk < 0) return;
  // (the dual half-step measured no gain from it: 202.6 -> 203.9 ms of a control-QP
  // batch solve, against 225.4 -> 219.9 here)
  prefetch_ahead(a.P, a.act, (int)blockIdx.x, (int)gridDim.x);
  primal_block<V, NT, LR, GATHER_LDG>(a, bk, j, prod, srp);
}

// --------------------------------------------------------------------------
// A whole chunk of iterations in one launch, for small problems (whose
// per-iteration kernels are bound by launch and gather latency): one cluster
// of C = 16 CTAs (8 where 16 cannot be co-scheduled).  Every CTA keeps its own copy of x_tilde and of both
// [x_md ; y] buffers in shared memory and gathers from it; after each
// half-step it writes the rows it updated into every CTA's copy (distributed
// shared memory) and the cluster meets at a barrier (release / acquire).  CTA
// c takes row blocks c, c + C, ... of A and of P.  The row arithmetic
// is that of k_dual / k_primal, so the iterates are bitwise theirs, and every
// result still goes to global memory for the checks.  Every thread of every
// CTA takes the same 2 * len + 1 barriers: no path leaves the loop early
// (blocks of an instance that stopped are skipped).  No low-rank term, no
// long rows, and the copies must fit in shared memory (the host checks).
// --------------------------------------------------------------------------
constexpr int CHUNK_NT = 512;
constexpr int CHUNK_MAX_BLOCKS = 64;               // row blocks of A and of P, each
constexpr int CHUNK_SMEM_MAX = 200 * 1024;

// every thread of the cluster arrives (release) and waits (acquire); the
// unaligned form does not need the warp converged at the barrier
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}

template <typename V>
constexpr size_t chunk_head_bytes() {     // staging buffers, rounded to 16 bytes
  return ((size_t)BNNZ * sizeof(V) + (BROWS + 1) * sizeof(int) + 15) / 16 * 16;
}
template <typename V>
static size_t chunk_smem_bytes(int n, int m) {
  return chunk_head_bytes<V>() + (size_t)(3 * (size_t)n + 2 * (size_t)m) * sizeof(V);
}

// write v into slot p of every CTA's copy (p: this CTA's shared address)
template <typename V>
__device__ __forceinline__ void broadcast(cg::cluster_group& cl, int ctas, V* p, V v) {
  for (int q = 0; q < ctas; ++q) *cl.map_shared_rank(p, q) = v;
}

// Resident row blocks: where every CTA takes at most one row block of A and
// one of P, each CTA keeps its blocks in shared memory for the launch: the
// row offsets, column indices and values, and the rows' own operands (of A:
// b, y_bar, the inequality flag and the mixed-precision lower bound; of P: x,
// x_bar, c, l, u), which only this CTA updates.  A half-step's dependent chain
// then runs from the gathers out of the shared-memory vector copies to the
// writes into every CTA's copies, straight from registers, with no global
// round trip on it (the results still go to global memory for the checks).
// The products val[e] * v[col[e]], the row sums in order and the row updates
// are dual_block / primal_block's, so the iterates stay theirs.
constexpr int RES_ROWS = 5;   // operand rows per resident block
template <typename V>
struct ResBlock {
  int r0, nr, ne;
  V* val;            // [BNNZ]
  V* row[RES_ROWS];  // [BROWS] each
  int* col;          // [BNNZ]
  int* srp;          // [BROWS + 1]
};
template <typename V>
__host__ __device__ inline size_t chunk_res_offset(int n, int m) {   // behind the vector copies, 16-byte aligned
  return (chunk_head_bytes<V>() + (size_t)(3 * (size_t)n + 2 * (size_t)m) * sizeof(V) + 15) / 16 * 16;
}
template <typename V>
constexpr size_t chunk_res_block_bytes() {   // one resident block, a multiple of 16 bytes
  return ((size_t)(BNNZ + RES_ROWS * BROWS) * sizeof(V) + (size_t)BNNZ * sizeof(int) + (BROWS + 1) * sizeof(int) +
          15) / 16 * 16;
}
template <typename V>
constexpr size_t chunk_res_bytes() { return 2 * chunk_res_block_bytes<V>(); }
template <typename V>
__device__ __forceinline__ ResBlock<V> res_view(unsigned char* base) {
  ResBlock<V> rb;
  rb.val = reinterpret_cast<V*>(base);
  for (int k = 0; k < RES_ROWS; ++k) rb.row[k] = rb.val + BNNZ + k * BROWS;
  rb.col = reinterpret_cast<int*>(rb.val + BNNZ + RES_ROWS * BROWS);
  rb.srp = rb.col + BNNZ;
  rb.r0 = rb.nr = rb.ne = 0;
  return rb;
}
template <typename V>
__device__ __forceinline__ void res_load(const BCsr<V>& M, int b, ResBlock<V>& rb, const V* o0, const V* o1,
                                         const V* o2, const V* o3, const V* o4) {
  const int r0 = M.blk[b], r1 = M.blk[b + 1];
  const int e0 = M.rp[r0];
  rb.r0 = r0;
  rb.nr = r1 - r0;
  rb.ne = M.rp[r1] - e0;   // <= BNNZ: no long rows in the cluster chunk
  for (int t = threadIdx.x; t <= rb.nr; t += CHUNK_NT) rb.srp[t] = M.rp[r0 + t] - e0;
  for (int e = threadIdx.x; e < rb.ne; e += CHUNK_NT) {
    rb.col[e] = M.col[e0 + e];
    rb.val[e] = M.val[e0 + e];
  }
  const V* src[RES_ROWS] = {o0, o1, o2, o3, o4};
  for (int t = threadIdx.x; t < rb.nr; t += CHUNK_NT)
#pragma unroll
    for (int k = 0; k < RES_ROWS; ++k) rb.row[k][t] = src[k] ? src[k][r0 + t] : V(0);
}

static_assert(BROWS <= CHUNK_NT, "a resident block's rows take one thread each");

// dual_block on a resident block: rows[0] b, [1] y_bar, [2] 1 for an
// inequality row, [3] the lower bound; y^k from the shared-memory copy yk, y+
// into every CTA's copy at ycopy
template <typename V>
__device__ __forceinline__ void dual_block_res(const DualB<V>& a, int bk, int j, V* prod, ResBlock<V>& rb,
                                               cg::cluster_group& cl, int ctas, const V* yk, V* ycopy) {
  const int tid = threadIdx.x;
  const int inst = a.blk_inst[bk];
  if (a.st[inst].status != ST_RUNNING) return;    // uniform over the block
  const StepEntry& es = a.tab[inst * a.C + j];
  for (int e = tid; e < rb.ne; e += CHUNK_NT) prod[e] = rb.val[e] * a.xt[rb.col[e]];
  __syncthreads();
  if (tid < rb.nr) {
    V s = V(0);
    for (int e = rb.srp[tid]; e < rb.srp[tid + 1]; ++e) s += prod[e];
    const int r = rb.r0 + tid;
    V yn, ybn;
    dual_update<V>(es, s, yk[r], rb.row[0][tid], rb.row[1][tid], rb.row[3][tid], rb.row[2][tid] != V(0), yn, ybn);
    rb.row[1][tid] = ybn;
    a.ybar[r] = ybn;
    a.ynew[r] = yn;
    broadcast(cl, ctas, ycopy + r, yn);
  }
}

// primal_block on a resident block: rows[0] x, [1] x_bar, [2] c, [3] l, [4] u;
// the next x_md into every CTA's copy at zcopy, the next x_tilde at xcopy
template <typename V>
__device__ __forceinline__ void primal_block_res(const PrimalB<V>& a, int bk, int j, V* prod, ResBlock<V>& rb,
                                                 cg::cluster_group& cl, int ctas, V* zcopy, V* xcopy) {
  const int tid = threadIdx.x;
  const int inst = a.blk_inst[bk];
  if (a.st[inst].status != ST_RUNNING) return;
  const StepEntry& es = a.tab[inst * a.C + j];
  for (int e = tid; e < rb.ne; e += CHUNK_NT) prod[e] = rb.val[e] * a.zin[rb.col[e]];
  __syncthreads();
  if (tid < rb.nr) {
    V s = V(0);
    for (int e = rb.srp[tid]; e < rb.srp[tid + 1]; ++e) s += prod[e];
    const int r = rb.r0 + tid;
    const V g = r_add(s, rb.row[2][tid]);
    V xn, xb, zo, xtn;
    primal_update<V>(es, g, rb.row[0][tid], rb.row[1][tid], rb.row[3][tid], rb.row[4][tid], xn, xb, zo, xtn);
    rb.row[0][tid] = xn;
    rb.row[1][tid] = xb;
    a.xbar[r] = xb;
    a.zout[r] = zo;
    a.xt[r] = xtn;
    a.x[r] = xn;
    broadcast(cl, ctas, zcopy + r, zo);
    broadcast(cl, ctas, xcopy + r, xtn);
  }
}

template <typename V>
__global__ void __launch_bounds__(CHUNK_NT)
    k_chunk_cluster(DualB<V> da, PrimalB<V> pa, int nblkA, int nblkP, V* z0, V* z1, int n, int m, int j0,
                    int len, int resident) {
  extern __shared__ __align__(16) unsigned char chunk_sm[];
  V* prod = reinterpret_cast<V*>(chunk_sm);
  int* srp = reinterpret_cast<int*>(prod + BNNZ);
  V* xs = reinterpret_cast<V*>(chunk_sm + chunk_head_bytes<V>());   // x_tilde
  V* zs[2] = {xs + n, xs + n + (n + m)};                            // [x_md ; y], both buffers
  cg::cluster_group cl = cg::this_cluster();
  const int cta = (int)cl.block_rank(), ctas = (int)cl.num_blocks();   // the grid is one cluster
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += CHUNK_NT) xs[i] = __ldcg(pa.xt + i);
  for (int i = tid; i < n + m; i += CHUNK_NT) {
    zs[0][i] = __ldcg(z0 + i);
    zs[1][i] = __ldcg(z1 + i);
  }
  // resident blocks (the host passes resident = 1 only where nblkA, nblkP <=
  // ctas and their copies fit behind the vectors)
  unsigned char* rbase = chunk_sm + chunk_res_offset<V>(n, m);
  ResBlock<V> rA = res_view<V>(rbase), rP = res_view<V>(rbase + chunk_res_bytes<V>() / 2);
  if (resident) {
    // the inequality flags as values of V (1 or 0) in a scratch slot first
    if (cta < nblkA) {
      res_load(da.A, cta, rA, da.b, da.ybar, (const V*)nullptr, da.ylo, (const V*)nullptr);
      for (int t = tid; t < rA.nr; t += CHUNK_NT) rA.row[2][t] = da.ineq[rA.r0 + t] ? V(1) : V(0);
    }
    if (cta < nblkP) res_load(pa.P, cta, rP, pa.x, pa.xbar, pa.c, pa.l, pa.u);
  }
  cluster_barrier();                              // every copy is whole before anyone writes into it
  DualB<V> dl = da;
  dl.xt = xs;
  PrimalB<V> pl = pa;
  for (int j = j0; j < j0 + len; ++j) {
    V* zj = (j & 1) ? z1 : z0;
    V* zn = (j & 1) ? z0 : z1;
    V* zsj = zs[j & 1];
    V* zsn = zs[(j + 1) & 1];
    dl.yold = zn + n;
    dl.ynew = zj + n;
    for (int bk = cta; bk < nblkA; bk += ctas) {
      __syncthreads();                            // the previous block's rows are done with prod
      if (resident) {
        dual_block_res<V>(dl, bk, j, prod, rA, cl, ctas, zsn + n, zsj + n);
        continue;
      }
      dual_block<V, CHUNK_NT, GATHER_PLAIN>(dl, bk, j, prod, srp);
      if (da.st[da.blk_inst[bk]].status == ST_RUNNING) {
        const int r0 = da.A.blk[bk], nr = da.A.blk[bk + 1] - r0;
        for (int t = tid; t < nr; t += CHUNK_NT) broadcast(cl, ctas, zsj + n + r0 + t, dl.ynew[r0 + t]);
      }
    }
    cluster_barrier();
    pl.zin = zsj;
    pl.zout = zn;
    for (int bk = cta; bk < nblkP; bk += ctas) {
      __syncthreads();
      if (resident) {
        primal_block_res<V>(pl, bk, j, prod, rP, cl, ctas, zsn, xs);
        continue;
      }
      primal_block<V, CHUNK_NT, false, GATHER_PLAIN>(pl, bk, j, prod, srp);
      if (pa.st[pa.blk_inst[bk]].status == ST_RUNNING) {
        const int r0 = pa.P.blk[bk], nr = pa.P.blk[bk + 1] - r0;
        for (int t = tid; t < nr; t += CHUNK_NT) {
          broadcast(cl, ctas, zsn + r0 + t, zn[r0 + t]);
          broadcast(cl, ctas, xs + r0 + t, pl.xt[r0 + t]);
        }
      }
    }
    cluster_barrier();
  }
}

// Segment sums of the long rows: one CUDA block per segment of LSEG nonzeros
// of M v (skipping instances that stopped); the iteration kernels add a row's
// segments in order.
template <typename V>
__global__ void __launch_bounds__(256) k_long_partials(BCsr<V> M, const V* __restrict__ vec,
                                                       const int4* __restrict__ lseg, const int* __restrict__ blk_inst,
                                                       const DevState* __restrict__ st, V* __restrict__ out) {
  const int4 g = lseg[blockIdx.x];
  if (st[blk_inst[g.w]].status != ST_RUNNING) return;
  V s = V(0);
  for (int e = g.y + threadIdx.x; e < g.z; e += 256) s += M.val[e] * __ldg(vec + M.col[e]);
  s = block_sum(s);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}


// ==========================================================================
// Pipelined persistent variants of the two half-steps.  Each CUDA block loops
// over row blocks b = blockIdx.x, blockIdx.x + gridDim.x, ...; while it
// gathers and finishes block b, the index, value and row-pointer ranges of its
// next block stream into the other shared-memory stage with cp.async (16-byte
// copies of the 16-byte aligned superset of each range).  Block bounds come
// from one int4 {r0, r1, e0, e1} per block.  Global index/value/rowptr arrays
// carry 8 elements of padding so the aligned superset never leaves them.
// ==========================================================================
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

template <typename V>
struct PipeSmem {
  int col[2][BNNZ + 8];
  V val[2][BNNZ + 8];
  int rp[2][BROWS + 8];
  V prod[BNNZ];
};

// Queue the copies of block m = {r0, r1, e0, e1} into stage s (no copy for a long row).
template <int NT, typename V>
__device__ __forceinline__ void pipe_issue(PipeSmem<V>& sm, int s, const int4 m, const int* __restrict__ col,
                                           const V* __restrict__ val, const int* __restrict__ rp) {
  const int tid = threadIdx.x;
  if (m.w - m.z <= BNNZ) {
    const int a0 = m.z & ~3, a1 = (m.w + 3) & ~3;
    for (int c = tid; c < (a1 - a0) >> 2; c += NT) cp_async16(&sm.col[s][c << 2], col + a0 + (c << 2));
    constexpr int PER = 16 / sizeof(V);
    for (int c = tid; c < (a1 - a0) / PER; c += NT) cp_async16(&sm.val[s][c * PER], val + a0 + c * PER);
    const int q0 = m.x & ~3, q1 = (m.y + 1 + 3) & ~3;
    for (int c = tid; c < (q1 - q0) >> 2; c += NT) cp_async16(&sm.rp[s][c << 2], rp + q0 + (c << 2));
  }
  cp_async_commit();
}

template <typename V, int NT>
__global__ void __launch_bounds__(NT) k_dual_pipe(DualB<V> a, const int4* __restrict__ meta, int nblk, int j) {
  extern __shared__ __align__(16) unsigned char smraw[];
  PipeSmem<V>& sm = *reinterpret_cast<PipeSmem<V>*>(smraw);
  const int tid = threadIdx.x;
  int b = blockIdx.x;
  if (b >= nblk) return;
  int4 mc = meta[b];
  pipe_issue<NT>(sm, 0, mc, a.A.col, a.A.val, a.A.rp);
  for (int s = 0; b < nblk; b += gridDim.x, s ^= 1) {
    const int bn = b + gridDim.x;
    int4 mn = make_int4(0, 0, 0, 0);
    if (bn < nblk) mn = meta[bn];
    pipe_issue<NT>(sm, s ^ 1, mn, a.A.col, a.A.val, a.A.rp);
    const int r0 = mc.x, nr = mc.y - mc.x, e0 = mc.z, ne = mc.w - mc.z;
    const int inst = a.blk_inst[b];
    const bool live = a.st[inst].status == ST_RUNNING;
    const StepEntry& es = a.tab[inst * a.C + j];
    V yo = V(0), bi = V(0), yb = V(0), lo = V(0);
    if (live && tid < nr) {
      const int r = r0 + tid;
      yo = a.yold[r]; bi = a.b[r]; yb = a.ybar[r];
      if (a.ylo) lo = a.ylo[r];
    }
    cp_async_wait1();
    __syncthreads();
    if (!live) {
    } else if (ne <= BNNZ) {
      const int off = e0 - (e0 & ~3), roff = r0 - (r0 & ~3);
#pragma unroll
      for (int k = 0; k < BNNZ / NT; ++k) {
        const int e = tid + k * NT;
        if (e < ne) sm.prod[e] = sm.val[s][e + off] * __ldg(a.xt + sm.col[s][e + off]);
      }
      __syncthreads();
      for (int t = tid; t < nr; t += NT) {
        V acc = V(0);
        const int eb = sm.rp[s][t + roff] - e0, ee = sm.rp[s][t + 1 + roff] - e0;
        for (int e = eb; e < ee; ++e) acc += sm.prod[e];
        const int r = r0 + t;
        if (t >= NT) {
          yo = a.yold[r]; bi = a.b[r]; yb = a.ybar[r];
          lo = a.ylo ? a.ylo[r] : V(0);
        }
        dual_row(a, es, r, acc, yo, bi, yb, lo);
      }
    } else if (a.blk_seg) {   // a long row: the sum of its segments (k_long_partials), as k_dual
      if (tid == 0) {
        const int2 sg = a.blk_seg[b];
        V acc = V(0);
        for (int q = 0; q < sg.y; ++q) acc += a.lpart[sg.x + q];
        dual_row(a, es, r0, acc, yo, bi, yb, lo);
      }
    } else {
      V acc = V(0);
      for (int e = e0 + tid; e < e0 + ne; e += NT) acc += a.A.val[e] * __ldg(a.xt + a.A.col[e]);
      acc = block_sum(acc);
      if (tid == 0) dual_row(a, es, r0, acc, yo, bi, yb, lo);
    }
    __syncthreads();
    mc = mn;
  }
}

template <typename V, int NT>
__global__ void __launch_bounds__(NT) k_primal_pipe(PrimalB<V> a, const int4* __restrict__ meta, int nblk, int j) {
  extern __shared__ __align__(16) unsigned char smraw[];
  PipeSmem<V>& sm = *reinterpret_cast<PipeSmem<V>*>(smraw);
  const int tid = threadIdx.x;
  int b = blockIdx.x;
  if (b >= nblk) return;
  int4 mc = meta[b];
  pipe_issue<NT>(sm, 0, mc, a.P.col, a.P.val, a.P.rp);
  for (int s = 0; b < nblk; b += gridDim.x, s ^= 1) {
    const int bn = b + gridDim.x;
    int4 mn = make_int4(0, 0, 0, 0);
    if (bn < nblk) mn = meta[bn];
    pipe_issue<NT>(sm, s ^ 1, mn, a.P.col, a.P.val, a.P.rp);
    const int r0 = mc.x, nr = mc.y - mc.x, e0 = mc.z, ne = mc.w - mc.z;
    const int inst = a.blk_inst[b];
    const bool live = a.st[inst].status == ST_RUNNING;
    const StepEntry& es = a.tab[inst * a.C + j];
    V xo = V(0), xb = V(0), cr = V(0), lr = V(0), ur = V(0);
    if (live && tid < nr) {
      const int r = r0 + tid;
      xo = a.x[r]; xb = a.xbar[r]; cr = a.c[r]; lr = a.l[r]; ur = a.u[r];
    }
    cp_async_wait1();
    __syncthreads();
    if (!live) {
    } else if (ne <= BNNZ) {
      const int off = e0 - (e0 & ~3), roff = r0 - (r0 & ~3);
#pragma unroll
      for (int k = 0; k < BNNZ / NT; ++k) {
        const int e = tid + k * NT;
        if (e < ne) sm.prod[e] = sm.val[s][e + off] * __ldg(a.zin + sm.col[s][e + off]);
      }
      __syncthreads();
      for (int t = tid; t < nr; t += NT) {
        V acc = V(0);
        const int eb = sm.rp[s][t + roff] - e0, ee = sm.rp[s][t + 1 + roff] - e0;
        for (int e = eb; e < ee; ++e) acc += sm.prod[e];
        const int r = r0 + t;
        if (t >= NT) { xo = a.x[r]; xb = a.xbar[r]; cr = a.c[r]; lr = a.l[r]; ur = a.u[r]; }
        if (a.F) primal_row<V, true>(a, es, r, acc, xo, xb, cr, lr, ur);
        else primal_row<V, false>(a, es, r, acc, xo, xb, cr, lr, ur);
      }
    } else if (a.blk_seg) {   // a long row: the sum of its segments, as k_primal
      if (tid == 0) {
        const int2 sg = a.blk_seg[b];
        V acc = V(0);
        for (int q = 0; q < sg.y; ++q) acc += a.lpart[sg.x + q];
        if (a.F) primal_row<V, true>(a, es, r0, acc, xo, xb, cr, lr, ur);
        else primal_row<V, false>(a, es, r0, acc, xo, xb, cr, lr, ur);
      }
    } else {
      V acc = V(0);
      for (int e = e0 + tid; e < e0 + ne; e += NT) acc += a.P.val[e] * __ldg(a.zin + a.P.col[e]);
      acc = block_sum(acc);
      if (tid == 0) {
        if (a.F) primal_row<V, true>(a, es, r0, acc, xo, xb, cr, lr, ur);
        else primal_row<V, false>(a, es, r0, acc, xo, xb, cr, lr, ur);
      }
    }
    __syncthreads();
    mc = mn;
  }
}

// resident blocks per SM of a pipelined kernel (its shared-memory limit set
// once; a function-local static is initialised once, thread-safely)
template <typename K>
static int pipe_blocks(K kern, int nt, size_t smem) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
  return per_sm > 0 ? per_sm : 1;
}
template <typename V, int NT>
static int pipe_grid(void (*kern)(DualB<V>, const int4*, int, int)) {
  static const int blocks = pipe_blocks(kern, NT, sizeof(PipeSmem<V>));
  return blocks;
}
template <typename V, int NT>
static int pipe_grid_p(void (*kern)(PrimalB<V>, const int4*, int, int)) {
  static const int blocks = pipe_blocks(kern, NT, sizeof(PipeSmem<V>));
  return blocks;
}

// Algorithmic bytes of one dual (kind 0) or primal (kind 1) launch over the
// instances running at the last check: the matrix streams (index + value),
// the row pointers, each vector read or written once (the gathered vector
// counted once); sv = bytes per value.
static double launch_bytes(const Work& w, int kind, double sv) {
  const BatchState& b = *w.bst_host;
  if (kind == 0) return b.run_nnzA * (sv + 4.0) + 4.0 * (b.run_m + 1.0) + sv * (b.run_n + 5.0 * b.run_m);
  return b.run_nnzP * (sv + 4.0) + 4.0 * (b.run_n + 1.0) + sv * (10.0 * b.run_n + b.run_m);
}

template <typename V, int NT>
static void run_chunk_pipe(Work& w, int j0, int len, BCsr<V> A, BCsr<V> P, V* xt, V* const* Z, V* ybar, const V* b,
                           const V* ylo, V* x, V* xbar, const V* c, const V* l, const V* u, cudaStream_t s) {
  Profiler& Pr = w.prof;
  DualB<V> da{A, xt, nullptr, nullptr, ybar, b, ylo, w.tab, w.blk_inst_A, w.st, w.row_ineq, w.tab_stride};
  PrimalB<V> pa{P, nullptr, nullptr, x, xbar, xt, c, l, u, w.tab, w.blk_inst_P, w.st, w.tab_stride,
                w.r > 0 ? lr_factor<V>(w) : nullptr, lr_weights<V>(w), w.r};
  const int gd = std::min(w.A.nblk, w.num_sms * pipe_grid<V, NT>(k_dual_pipe<V, NT>));
  const int gp = std::min(w.P.nblk, w.num_sms * pipe_grid_p<V, NT>(k_primal_pipe<V, NT>));
  const size_t smem = sizeof(PipeSmem<V>);
  // long rows: segment sums first, the same as the row-block variants
  V* lpA = sizeof(V) == 4 ? (V*)w.A.lpart_f : (V*)w.A.lpart_d;
  V* lpP = sizeof(V) == 4 ? (V*)w.P.lpart_f : (V*)w.P.lpart_d;
  if (w.A.nlseg) { da.blk_seg = w.A.blk_seg; da.lpart = lpA; }
  if (w.P.nlseg) { pa.blk_seg = w.P.blk_seg; pa.lpart = lpP; }
  for (int j = j0; j < j0 + len; ++j) {
    if (w.r > 0) lowrank_ft1(w, pa.F, (const V*)Z[j & 1], s);
    if (w.m > 0) {
      da.yold = Z[(j + 1) & 1] + w.n;
      da.ynew = Z[j & 1] + w.n;
      if (Pr.on) Pr.begin(0, s, launch_bytes(w, 0, sizeof(V)));
      if (w.A.nlseg)
        launch(k_long_partials<V>, w.A.nlseg, 256, 0, s, A, (const V*)xt, (const int4*)w.A.lseg,
               (const int*)w.blk_inst_A, (const DevState*)w.st, lpA);
      launch(k_dual_pipe<V, NT>, gd, NT, smem, s, da, (const int4*)w.A.meta, w.A.nblk, j);
      if (Pr.on) Pr.end(s);
    }
    pa.zin = Z[j & 1];
    pa.zout = Z[(j + 1) & 1];
    if (Pr.on) Pr.begin(1, s, launch_bytes(w, 1, sizeof(V)));
    if (w.P.nlseg)
      launch(k_long_partials<V>, w.P.nlseg, 256, 0, s, P, (const V*)pa.zin, (const int4*)w.P.lseg,
             (const int*)w.blk_inst_P, (const DevState*)w.st, lpP);
    launch(k_primal_pipe<V, NT>, gp, NT, smem, s, pa, (const int4*)w.P.meta, w.P.nblk, j);
    if (Pr.on) Pr.end(s);
  }
}

template <typename V, int NT>
static void run_chunk(Work& w, int j0, int len, BCsr<V> A, BCsr<V> P, V* xt, V* const* Z, V* ybar, const V* b,
                      const V* ylo, V* x, V* xbar, const V* c, const V* l, const V* u, cudaStream_t s,
                      bool compact) {
  Profiler& Pr = w.prof;
  DualB<V> da{A, xt, nullptr, nullptr, ybar, b, ylo, w.tab, w.blk_inst_A, w.st, w.row_ineq, w.tab_stride};
  PrimalB<V> pa{P, nullptr, nullptr, x, xbar, xt, c, l, u, w.tab, w.blk_inst_P, w.st, w.tab_stride,
                w.r > 0 ? lr_factor<V>(w) : nullptr, lr_weights<V>(w), w.r};
  // long rows: segment sums first (float or float64 buffers by V)
  V* lpA = sizeof(V) == 4 ? (V*)w.A.lpart_f : (V*)w.A.lpart_d;
  V* lpP = sizeof(V) == 4 ? (V*)w.P.lpart_f : (V*)w.P.lpart_d;
  if (w.A.nlseg) { da.blk_seg = w.A.blk_seg; da.lpart = lpA; }
  if (w.P.nlseg) { pa.blk_seg = w.P.blk_seg; pa.lpart = lpP; }
  int gA = w.A.nblk, gP = w.P.nblk;
  if (compact) {   // only the running instances' row blocks (counts of the last check)
    da.act = w.act_A;
    pa.act = w.act_P;
    // a grid padded for a replayed graph (entries past the count are -1), or
    // the counts themselves
    gA = w.act_grid_A > 0 ? w.act_grid_A : w.bst_host->act_A;
    gP = w.act_grid_P > 0 ? w.act_grid_P : w.bst_host->act_P;
  }
  for (int j = j0; j < j0 + len; ++j) {
    if (w.r > 0) lowrank_ft1(w, pa.F, (const V*)Z[j & 1], s);
    if (w.m > 0) {
      da.yold = Z[(j + 1) & 1] + w.n;
      da.ynew = Z[j & 1] + w.n;
      if (Pr.on) Pr.begin(0, s, launch_bytes(w, 0, sizeof(V)));
      if (w.A.nlseg)
        launch(k_long_partials<V>, w.A.nlseg, 256, 0, s, A, (const V*)xt, (const int4*)w.A.lseg,
               (const int*)w.blk_inst_A, (const DevState*)w.st, lpA);
      launch(k_dual<V, NT>, gA, NT, 0, s, da, j);
      if (Pr.on) Pr.end(s);
    }
    pa.zin = Z[j & 1];
    pa.zout = Z[(j + 1) & 1];
    if (Pr.on) Pr.begin(1, s, launch_bytes(w, 1, sizeof(V)));
    if (w.P.nlseg)
      launch(k_long_partials<V>, w.P.nlseg, 256, 0, s, P, (const V*)pa.zin, (const int4*)w.P.lseg,
             (const int*)w.blk_inst_P, (const DevState*)w.st, lpP);
    if (w.r > 0) launch(k_primal<V, NT, true>, gP, NT, 0, s, pa, j);
    else launch(k_primal<V, NT, false>, gP, NT, 0, s, pa, j);
    if (Pr.on) Pr.end(s);
  }
}

// ==========================================================================
// Family handles: members that share the matrix, run on member-interleaved
// vectors v[j * ld + member] (ld = members rounded up to 32).  A warp takes
// one row for 32 members: each matrix entry is read once for them and meets
// their 32 values of the gathered vector in one coalesced load, where the
// member-major layout gathers 32 scattered sectors.  The row sum runs over
// the row's entries in CSR order with separately rounded products and sums,
// as the row-block kernels sum their staged products, and the row update is
// the same function: a member's iterates are bitwise those of its standalone
// solve.  The vectors are transposed into this layout at the start of a
// chunk and back at its end, so the checks, restarts and rebases run on the
// member-major layout as for any batch.
// ==========================================================================
constexpr int IL_NT = 256;
constexpr int IL_RPB = IL_NT / 32;     // rows per CUDA block (one warp each)


template <typename V>
struct FamIL {
  const int* __restrict__ rp;          // one member's CSR (A, or P with local columns)
  const int* __restrict__ col;
  const V* __restrict__ val;           // scaled values (the same for every member)
  int rows, ld, count, C;
  const StepEntry* __restrict__ tab;   // [member][C]
  const DevState* __restrict__ st;     // [member]
  const V* __restrict__ zin;           // gathered vector (x_tilde, or [x_md ; y+])
  // dual: yold, ynew, ybar, b, ylo (may be null), ineq;  primal: x, xbar, zout, xt, c, l, u
  const V* __restrict__ v0;
  V* __restrict__ w0;
  V* __restrict__ w1;
  V* __restrict__ w2;
  V* __restrict__ w3;
  const V* __restrict__ r0;
  const V* __restrict__ r1;
  const V* __restrict__ r2;
  const unsigned char* __restrict__ ineq;
};

// 16 bytes of consecutive members per lane: 4 float or 2 double
template <typename V> struct IlVec;
template <> struct IlVec<float> { using T = float4; static constexpr int W = 4; };
template <> struct IlVec<double> { using T = double2; static constexpr int W = 2; };
constexpr int IL_LD_ALIGN = 128;       // members per warp in float32 (the leading dimension's unit)

template <typename V>
__device__ __forceinline__ void il_load(const V* p, V (&v)[IlVec<V>::W]) {
  const typename IlVec<V>::T q = __ldg(reinterpret_cast<const typename IlVec<V>::T*>(p));
  if constexpr (IlVec<V>::W == 4) { v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w; }
  else { v[0] = q.x; v[1] = q.y; }
}
template <typename V>
__device__ __forceinline__ void il_load_rw(const V* p, V (&v)[IlVec<V>::W]) {   // a vector the kernel writes
  const typename IlVec<V>::T q = *reinterpret_cast<const typename IlVec<V>::T*>(p);
  if constexpr (IlVec<V>::W == 4) { v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w; }
  else { v[0] = q.x; v[1] = q.y; }
}
template <typename V>
__device__ __forceinline__ void il_store(V* p, const V (&v)[IlVec<V>::W]) {
  typename IlVec<V>::T q;
  if constexpr (IlVec<V>::W == 4) { q.x = v[0]; q.y = v[1]; q.z = v[2]; q.w = v[3]; }
  else { q.x = v[0]; q.y = v[1]; }
  *reinterpret_cast<typename IlVec<V>::T*>(p) = q;
}

// The row sums of this lane's W members: for each, sequential over the row's
// entries, each product and sum rounded on its own (no fused multiply-add),
// as prod[e] is staged and summed by the row-block kernels.  The warp reads
// the row's indices and values 32 at a time in one coalesced load and hands
// each entry to all lanes by shuffle, so that the L1 data pipe (the bound of
// this kernel) moves only the gathered members' values.  Every lane of the
// warp runs it (the shuffles need the whole warp).
template <typename V>
__device__ __forceinline__ void il_row_sum(const FamIL<V>& a, int r, int m0, V (&s)[IlVec<V>::W]) {
  constexpr int W = IlVec<V>::W;
  const int lane = threadIdx.x & 31;
  const int e0 = a.rp[r], e1 = a.rp[r + 1];
#pragma unroll
  for (int q = 0; q < W; ++q) s[q] = V(0);
  for (int base = e0; base < e1; base += 32) {
    int cl = 0;
    V vl = V(0);
    if (base + lane < e1) { cl = __ldg(a.col + base + lane); vl = __ldg(a.val + base + lane); }
    const int cnt = min(32, e1 - base);
    int k = 0;
    for (; k + 4 <= cnt; k += 4) {
      int c[4];
      V v[4], z[4][W];
#pragma unroll
      for (int i = 0; i < 4; ++i) { c[i] = __shfl_sync(0xffffffffu, cl, k + i); v[i] = __shfl_sync(0xffffffffu, vl, k + i); }
#pragma unroll
      for (int i = 0; i < 4; ++i) il_load(a.zin + (size_t)c[i] * a.ld + m0, z[i]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < W; ++q) s[q] = r_add(s[q], r_mul(v[i], z[i][q]));
    }
    for (; k < cnt; ++k) {
      const int c = __shfl_sync(0xffffffffu, cl, k);
      const V v = __shfl_sync(0xffffffffu, vl, k);
      V z[W];
      il_load(a.zin + (size_t)c * a.ld + m0, z);
#pragma unroll
      for (int q = 0; q < W; ++q) s[q] = r_add(s[q], r_mul(v, z[q]));
    }
  }
}

// Per-member step entries and running flags of the block's 32 W members;
// false when none of them runs (uniform over the block).
template <typename V>
__device__ __forceinline__ bool il_members(const FamIL<V>& a, int j, StepEntry* es, int* run) {
  constexpr int GM = 32 * IlVec<V>::W;
  int any = 0;
  for (int k = threadIdx.x; k < GM; k += blockDim.x) {
    const int mem = blockIdx.y * GM + k;
    const bool ok = mem < a.count && a.st[mem].status == ST_RUNNING;
    run[k] = ok;
    if (ok) es[k] = a.tab[(size_t)mem * a.C + j];
    any |= ok;
  }
  return __syncthreads_or(any) != 0;
}

template <typename V>
__global__ void __launch_bounds__(IL_NT, 4) k_dual_il(FamIL<V> a, int j) {
  constexpr int W = IlVec<V>::W, GM = 32 * W;
  __shared__ StepEntry es[GM];
  __shared__ int run[GM];
  if (!il_members(a, j, es, run)) return;
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * IL_RPB + (threadIdx.x >> 5);
  if (r >= a.rows) return;
  const int k0 = lane * W, m0 = blockIdx.y * GM + k0;
  const size_t idx = (size_t)r * a.ld + m0;
  V yo[W], bi[W], yb[W], lo[W], s[W], yn[W], ybn[W];
  il_load_rw(a.v0 + idx, yo);
  il_load(a.r0 + idx, bi);
  il_load_rw(a.w1 + idx, yb);
  if (a.r1) il_load(a.r1 + idx, lo);
  else
#pragma unroll
    for (int q = 0; q < W; ++q) lo[q] = V(0);
  il_row_sum(a, r, m0, s);
  const bool ineq = a.ineq[r] != 0;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    if (run[k0 + q]) dual_update<V>(es[k0 + q], s[q], yo[q], bi[q], yb[q], lo[q], ineq, yn[q], ybn[q]);
    else { ybn[q] = yb[q]; yn[q] = a.w0[idx + q]; }    // a member that stopped keeps its values
  }
  il_store(a.w1 + idx, ybn);   // y_bar
  il_store(a.w0 + idx, yn);    // y+
}

template <typename V>
__global__ void __launch_bounds__(IL_NT, 4) k_primal_il(FamIL<V> a, int j) {
  constexpr int W = IlVec<V>::W, GM = 32 * W;
  __shared__ StepEntry es[GM];
  __shared__ int run[GM];
  if (!il_members(a, j, es, run)) return;
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * IL_RPB + (threadIdx.x >> 5);
  if (r >= a.rows) return;
  const int k0 = lane * W, m0 = blockIdx.y * GM + k0;
  const size_t idx = (size_t)r * a.ld + m0;
  V xo[W], xb0[W], cr[W], lr[W], ur[W], s[W], xn[W], xb[W], zo[W], xtn[W];
  il_load_rw(a.w0 + idx, xo);
  il_load_rw(a.w1 + idx, xb0);
  il_load(a.r0 + idx, cr);
  il_load(a.r1 + idx, lr);
  il_load(a.r2 + idx, ur);
  il_row_sum(a, r, m0, s);
#pragma unroll
  for (int q = 0; q < W; ++q) {
    if (run[k0 + q]) {
      const V g = r_add(s[q], cr[q]);
      primal_update<V>(es[k0 + q], g, xo[q], xb0[q], lr[q], ur[q], xn[q], xb[q], zo[q], xtn[q]);
    } else {   // a member that stopped keeps its values
      xn[q] = xo[q]; xb[q] = xb0[q]; zo[q] = a.w2[idx + q]; xtn[q] = a.w3[idx + q];
    }
  }
  il_store(a.w1 + idx, xb);    // x_bar
  il_store(a.w2 + idx, zo);    // x_md of the next iteration
  il_store(a.w3 + idx, xtn);   // x_tilde of the next iteration
  il_store(a.w0 + idx, xn);    // x
}

// Algorithmic bytes of one family launch: the shared matrix once, the vectors
// of each running member once (kind 0 dual, 1 primal; sv = bytes per value).
static double il_launch_bytes(const Work& w, int kind, double sv) {
  const double members = w.fam_n > 0 ? w.bst_host->run_n / w.fam_n : 0.0;
  if (kind == 0)
    return w.fam_nnzA * (sv + 4.0) + 4.0 * (w.fam_m + 1.0) + sv * members * (w.fam_n + 5.0 * w.fam_m);
  return w.fam_nnzP * (sv + 4.0) + 4.0 * (w.fam_n + 1.0) + sv * members * (10.0 * w.fam_n + w.fam_m);
}

template <typename V>
static void run_chunk_il(Work& w, int j0, int len, const V* Aval, const V* Pval, V* xt, V* const* Z, V* ybar,
                         const V* b, const V* ylo, V* x, V* xbar, const V* c, const V* l, const V* u,
                         cudaStream_t s) {
  Profiler& Pr = w.prof;
  V* const* I = reinterpret_cast<V* const*>(sizeof(V) == 4 ? (void* const*)w.ilf : (void* const*)w.ild);
  const int n = w.fam_n, m = w.fam_m, cnt = w.fam_count, ld = w.fam_ld;
  const long long N = (long long)cnt * n;
  auto tin = [&](const V* src, long long stride, int L, V* dst) { to_il<V>(src, stride, L, cnt, dst, ld, s); };
  // member-major -> interleaved: everything the iterations read
  for (int p = 0; p < 2; ++p) {
    tin(Z[p], n, n, I[IL_Z0 + p]);
    tin(Z[p] + N, m, m, I[IL_Z0 + p] + (size_t)n * ld);
  }
  tin(x, n, n, I[IL_X]);
  tin(xbar, n, n, I[IL_XBAR]);
  tin(xt, n, n, I[IL_XT]);
  tin(ybar, m, m, I[IL_YBAR]);
  tin(c, n, n, I[IL_C]);
  tin(l, n, n, I[IL_L]);
  tin(u, n, n, I[IL_U]);
  tin(b, m, m, I[IL_B]);
  tin(ylo, m, m, I[IL_YLO]);
  const int groups = ld / (32 * IlVec<V>::W);
  FamIL<V> da{};
  da.rp = w.A.rp; da.col = w.A.col; da.val = Aval;
  da.rows = m; da.ld = ld; da.count = cnt; da.C = w.tab_stride; da.tab = w.tab; da.st = w.st;
  da.zin = I[IL_XT];
  da.w1 = I[IL_YBAR]; da.r0 = I[IL_B]; da.r1 = ylo ? I[IL_YLO] : nullptr; da.ineq = w.row_ineq;
  FamIL<V> pa{};
  pa.rp = w.P.rp; pa.col = w.famP_col; pa.val = Pval;
  pa.rows = n; pa.ld = ld; pa.count = cnt; pa.C = w.tab_stride; pa.tab = w.tab; pa.st = w.st;
  pa.w0 = I[IL_X]; pa.w1 = I[IL_XBAR]; pa.w3 = I[IL_XT]; pa.r0 = I[IL_C]; pa.r1 = I[IL_L]; pa.r2 = I[IL_U];
  for (int j = j0; j < j0 + len; ++j) {
    if (m > 0) {
      da.v0 = I[IL_Z0 + ((j + 1) & 1)] + (size_t)n * ld;   // y^k
      da.w0 = I[IL_Z0 + (j & 1)] + (size_t)n * ld;         // y^{k+1}
      if (Pr.on) Pr.begin(0, s, il_launch_bytes(w, 0, sizeof(V)));
      launch(k_dual_il<V>, dim3(cdiv(m, IL_RPB), groups), IL_NT, 0, s, da, j);
      if (Pr.on) Pr.end(s);
    }
    pa.zin = I[IL_Z0 + (j & 1)];
    pa.w2 = I[IL_Z0 + ((j + 1) & 1)];
    if (Pr.on) Pr.begin(1, s, il_launch_bytes(w, 1, sizeof(V)));
    launch(k_primal_il<V>, dim3(cdiv(n, IL_RPB), groups), IL_NT, 0, s, pa, j);
    if (Pr.on) Pr.end(s);
  }
  // interleaved -> member-major: everything the iterations wrote
  auto back = [&](const V* src, int L, V* dst, long long stride) { from_il<V>(src, ld, L, cnt, dst, stride, s); };
  for (int p = 0; p < 2; ++p) {
    back(I[IL_Z0 + p], n, Z[p], n);
    back(I[IL_Z0 + p] + (size_t)n * ld, m, Z[p] + N, m);
  }
  back(I[IL_X], n, x, n);
  back(I[IL_XBAR], n, xbar, n);
  back(I[IL_XT], n, xt, n);
  back(I[IL_YBAR], m, ybar, m);
}

bool chunk_cluster_ok(const Work& w, bool mixed) {
  const size_t smem = mixed ? chunk_smem_bytes<float>(w.n, w.m) : chunk_smem_bytes<double>(w.n, w.m);
  return w.r == 0 && w.A.nlseg == 0 && w.P.nlseg == 0 && w.A.nblk <= CHUNK_MAX_BLOCKS &&
         w.P.nblk <= CHUNK_MAX_BLOCKS && w.P.nblk > 0 && smem <= (size_t)CHUNK_SMEM_MAX;
}

// cluster size: 16 CTAs if a 16-CTA cluster of the largest footprint fits, else 8
static int g_chunk_ctas = 8;

template <typename V>
static int chunk_cluster_size() {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 16;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(CHUNK_NT);
  cfg.dynamicSmemBytes = CHUNK_SMEM_MAX;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_chunk_cluster<V>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 8;
  }
  return clusters >= 1 ? 16 : 8;
}

void prepare_chunk_cluster() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_chunk_cluster<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, CHUNK_SMEM_MAX);
    cudaFuncSetAttribute(k_chunk_cluster<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, CHUNK_SMEM_MAX);
    cudaFuncSetAttribute(k_chunk_cluster<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_chunk_cluster<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    g_chunk_ctas = std::min(chunk_cluster_size<float>(), chunk_cluster_size<double>());
  });
}

template <typename V>
static void run_chunk_cluster(Work& w, int j0, int len, BCsr<V> A, BCsr<V> P, V* xt, V* const* Z, V* ybar,
                              const V* b, const V* ylo, V* x, V* xbar, const V* c, const V* l, const V* u,
                              cudaStream_t s) {
  Profiler& Pr = w.prof;
  DualB<V> da{A, xt, nullptr, nullptr, ybar, b, ylo, w.tab, w.blk_inst_A, w.st, w.row_ineq, w.tab_stride};
  PrimalB<V> pa{P, nullptr, nullptr, x, xbar, xt, c, l, u, w.tab, w.blk_inst_P, w.st, w.tab_stride,
                nullptr, nullptr, 0};
  // kind 3: one launch holds both half-steps of `len` iterations
  if (Pr.on) Pr.begin(3, s, len * (launch_bytes(w, 0, sizeof(V)) + launch_bytes(w, 1, sizeof(V))));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = g_chunk_ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(g_chunk_ctas);               // one cluster
  cfg.blockDim = dim3(CHUNK_NT);
  const int nblkA = w.m > 0 ? w.A.nblk : 0;
  const size_t res_end = chunk_res_offset<V>(w.n, w.m) + chunk_res_bytes<V>();
  const int resident = nblkA <= g_chunk_ctas && w.P.nblk <= g_chunk_ctas && res_end <= (size_t)CHUNK_SMEM_MAX;
  cfg.dynamicSmemBytes = resident ? res_end : chunk_smem_bytes<V>(w.n, w.m);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_chunk_cluster<V>, da, pa, nblkA, w.P.nblk, Z[0], Z[1], w.n, w.m, j0, len, resident);
  count_launch();
  if (Pr.on) Pr.end(s);
}

void iterate_chunk(Work& w, int len, bool mixed, int nt, cudaStream_t s, int j0, bool compact) {
  if (nt == 3) {   // a family handle on member-interleaved vectors
    if (len <= 0) return;
    if (mixed) {
      run_chunk_il<float>(w, j0, len, w.A.sval_f, w.P.sval_f, w.fxt, w.fZ, w.fybar, w.fb, w.fylo, w.fx, w.fxbar, w.fc,
                          w.fl, w.fu, s);
      w.fy = w.fZ[(j0 + len - 1) & 1] + w.n;
    } else {
      run_chunk_il<double>(w, j0, len, w.A.sval, w.P.sval, w.xt, w.Z, w.ybar, w.bs, nullptr, w.x, w.xbar, w.cs, w.ls,
                           w.us, s);
      w.y = w.Z[(j0 + len - 1) & 1] + w.n;
    }
    return;
  }
  if (nt == 2) {   // the whole chunk in one cluster launch (small problems)
    if (mixed) {
      run_chunk_cluster<float>(w, j0, len, w.A.bscaled_f(), w.P.bscaled_f(), w.fxt, w.fZ, w.fybar, w.fb, w.fylo,
                               w.fx, w.fxbar, w.fc, w.fl, w.fu, s);
      w.fy = w.fZ[(j0 + len - 1) & 1] + w.n;
    } else {
      run_chunk_cluster<double>(w, j0, len, w.A.bscaled(), w.P.bscaled(), w.xt, w.Z, w.ybar, w.bs, nullptr, w.x,
                                w.xbar, w.cs, w.ls, w.us, s);
      w.y = w.Z[(j0 + len - 1) & 1] + w.n;
    }
    return;
  }
  if (nt == 1) {   // pipelined persistent kernels, 256 threads
    if (mixed) {
      run_chunk_pipe<float, 256>(w, j0, len, w.A.bscaled_f(), w.P.bscaled_f(), w.fxt, w.fZ, w.fybar, w.fb, w.fylo, w.fx,
                                 w.fxbar, w.fc, w.fl, w.fu, s);
      w.fy = w.fZ[(j0 + len - 1) & 1] + w.n;
    } else {
      run_chunk_pipe<double, 256>(w, j0, len, w.A.bscaled(), w.P.bscaled(), w.xt, w.Z, w.ybar, w.bs, nullptr, w.x,
                                  w.xbar, w.cs, w.ls, w.us, s);
      w.y = w.Z[(j0 + len - 1) & 1] + w.n;
    }
    return;
  }
  if (mixed) {
    if (nt != 512)
      run_chunk<float, 256>(w, j0, len, w.A.bscaled_f(), w.P.bscaled_f(), w.fxt, w.fZ, w.fybar, w.fb, w.fylo, w.fx,
                            w.fxbar, w.fc, w.fl, w.fu, s, compact);
    else
      run_chunk<float, 512>(w, j0, len, w.A.bscaled_f(), w.P.bscaled_f(), w.fxt, w.fZ, w.fybar, w.fb, w.fylo, w.fx,
                            w.fxbar, w.fc, w.fl, w.fu, s, compact);
    w.fy = w.fZ[(j0 + len - 1) & 1] + w.n;
  } else {
    if (nt != 512)
      run_chunk<double, 256>(w, j0, len, w.A.bscaled(), w.P.bscaled(), w.xt, w.Z, w.ybar, w.bs, nullptr, w.x, w.xbar,
                             w.cs, w.ls, w.us, s, compact);
    else
      run_chunk<double, 512>(w, j0, len, w.A.bscaled(), w.P.bscaled(), w.xt, w.Z, w.ybar, w.bs, nullptr, w.x, w.xbar,
                             w.cs, w.ls, w.us, s, compact);
    w.y = w.Z[(j0 + len - 1) & 1] + w.n;
  }
}

}  // namespace pdqp
