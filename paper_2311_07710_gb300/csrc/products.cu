// Maintained products (an option of float64 solves, not in the paper): the
// updates of Algorithm 1 (Section 2) are linear in the iterates, so the
// products the relKKT check needs can travel with the iterates instead of
// being formed again at every check.  With
//   x_tilde^k = x^k + theta_k (x^k - x^{k-1}),
//   x_md^k    = (1 - 1/beta_k) x_bar^k + x^k / beta_k,
//   x_bar^k   = (1 - 1/beta_{k-1}) x_bar^{k-1} + x^k / beta_{k-1}   (x_bar^0 = x^0)
// the dual half-step gathers x^k (not x_tilde^k) and forms
//   A x_tilde^k = A x^k + theta_k (A x^k - A x^{k-1}),
//   A x_bar^k   = (1 - 1/beta_{k-1}) A x_bar^{k-1} + A x^k / beta_{k-1},
// and the primal half-step gathers [x^k ; y^{k+1}] over P = [Q | -A'] with the
// two parts summed apart:
//   Q x_bar^k  = (1 - 1/beta_{k-1}) Q x_bar^{k-1} + Q x^k / beta_{k-1},
//   Q x_md^k   = (1 - 1/beta_k) Q x_bar^k + Q x^k / beta_k,
//   A'y_bar^{k+1} = (1 - 1/beta_k) A'y_bar^k + A'y^{k+1} / beta_k.
// The state carried is A x^k, A x_bar^k [m], Q x_bar^k, A'y^{k+1},
// A'y_bar^{k+1} [n].  A check after iteration k needs, for (x^{k+1}, y^{k+1})
// and the averages, A x and Q x of x^{k+1} (one gather of x each: A, and the
// Q part of P) and has the rest from the state; the next iteration starts
// from those two products instead of gathering them again (of the candidate
// it restarts from: the average's products are the maintained ones), so a
// chunk and its check gather what a chunk alone gathers.  In exact
// arithmetic the iterates are those of the direct products; the rounding
// differs (products and sums of products are formed in another order).
// Float64 only (in mixed precision the products would be float32 ones and
// the check must be float64); no low-rank term, no long rows, the row-block
// kernels at 256 threads.
#include "rowblock.cuh"

namespace pdqp {

constexpr int MP_NT = 256;

// theta_k and 1/beta_{k-1} of inner iteration k = k_epoch + j of an epoch:
// the previous entry's theta_next and inv_beta (entry j - 1 tabulates
// iteration k - 1); the first iteration of a chunk evaluates them by the
// expressions the step table uses (Theorem 1's beta_k = (k+2)/2,
// theta_{k+1} = (k+1)/(k+2); 1 without acceleration), so the values are the
// same bits either way, and only then divides (float64 divisions issue on
// GB300's slow float64 pipe).  k = 0 starts the epoch (x_tilde^0 = x_bar^0 = x^0).
struct PrevStep {
  bool first;
  double theta, ib_prev;
};
__device__ __forceinline__ PrevStep prev_step(const StepEntry* row, int j, long long k_epoch, int accelerate) {
  PrevStep q;
  if (j > 0) {
    const StepEntry& e = row[j - 1];
    q.first = false;
    q.theta = e.theta_next;
    q.ib_prev = e.inv_beta;
    return q;
  }
  const long long k = k_epoch;
  q.first = k == 0;
  q.theta = 1.0;
  q.ib_prev = 1.0;
  if (accelerate && k > 0) {
    q.theta = (double)k / ((double)k + 1.0);
    q.ib_prev = 1.0 / ((double)(k + 1) / 2.0);
  }
  return q;
}

struct MpIter {
  BCsr<double> A, P;
  const double* __restrict__ xg;      // dual: x^k, gathered
  const double* __restrict__ zin;     // primal: [x^k ; y^{k+1}]
  double* __restrict__ zout;          // primal: x^{k+1} -> zout[0:n] (what the next primal gathers)
  const double* __restrict__ yold;
  double* __restrict__ ynew;
  double* __restrict__ ybar;
  const double* __restrict__ b;
  double* __restrict__ x;
  double* __restrict__ xbar;
  const double *__restrict__ c, *__restrict__ l, *__restrict__ u;
  double* __restrict__ ax;            // A x^k of the last dual half-step [m]
  double* __restrict__ axb;           // A x_bar^k [m]
  double* __restrict__ qxb;           // Q x_bar^k of the last primal half-step [n]
  double* __restrict__ aty;           // P's -A' part of y^{k+1} [n]
  double* __restrict__ atyb;          // and of y_bar^{k+1}
  const double* sA[2];                // the last check's A x of its current / average iterate
  const double* sQ[2];                // and Q x
  const StepEntry* __restrict__ tab;
  const int *__restrict__ blk_inst_A, *__restrict__ blk_inst_P;
  const DevState* __restrict__ st;
  const unsigned char* __restrict__ ineq;
  const int *__restrict__ actA, *__restrict__ actP;   // compacted batches (null: every row block)
  int C, n, accelerate;
};

__device__ __forceinline__ void dual_row_mp(const MpIter& a, const StepEntry& e, const PrevStep& ps, int r, double s,
                                            double yo, double bi, double yb, double axp, double axbp) {
  const double axt = ps.first ? s : r_fma(ps.theta, r_sub(s, axp), s);                      // A x_tilde^k
  const double axb = ps.first ? s : r_fma(ps.ib_prev, s, r_mul(r_sub(1.0, ps.ib_prev), axbp));   // A x_bar^k
  const double sigma = e.sigma_d, ib = e.inv_beta;
  double yn = r_fma(-sigma, r_sub(axt, bi), yo);           // y - sigma (A x_tilde - b)
  if (a.ineq[r]) yn = fmax(yn, 0.0);
  const double ybn = r_fma(ib, yn, r_mul(r_sub(1.0, ib), yb));
  a.ax[r] = s;
  a.axb[r] = axb;
  a.ybar[r] = ybn;
  a.ynew[r] = yn;
}

// fresh: the first iteration after a check, whose A x^k that check formed
// (of the iterate the instance continues or restarts from)
__global__ void __launch_bounds__(MP_NT, MinBlocks<double, MP_NT>::value) k_dual_mp(MpIter a, int j, int fresh) {
  __shared__ double prod[BNNZ];
  __shared__ int srp[BROWS + 1];
  const int bk = a.actA ? a.actA[blockIdx.x] : (int)blockIdx.x;
  if (bk < 0) return;                               // padding of a compacted grid
  const int inst = a.blk_inst_A[bk];
  const DevState& S = a.st[inst];
  if (S.status != ST_RUNNING) return;               // uniform over the block
  const int tid = threadIdx.x;
  const int r0 = a.A.blk[bk], r1 = a.A.blk[bk + 1], nr = r1 - r0;
  const int e0 = a.A.rp[r0], ne = a.A.rp[r1] - e0;  // <= BNNZ: no long rows (the host checks)
  const StepEntry& es = a.tab[inst * a.C + j];
  const PrevStep ps = prev_step(a.tab + (size_t)inst * a.C, j, S.k_epoch, a.accelerate);
  double yo = 0.0, bi = 0.0, yb = 0.0, axp = 0.0, axbp = 0.0;
  auto operands = [&](int r) {
    yo = a.yold[r]; bi = a.b[r]; yb = a.ybar[r];
    if (!ps.first) { axp = a.ax[r]; axbp = a.axb[r]; }
  };
  if (tid < nr) operands(r0 + tid);
  if (fresh) {
    const double* fr = (S.restart && S.cand_avg) ? a.sA[1] : a.sA[0];
    for (int t = tid; t < nr; t += MP_NT) {
      if (t >= MP_NT) operands(r0 + t);
      dual_row_mp(a, es, ps, r0 + t, fr[r0 + t], yo, bi, yb, axp, axbp);
    }
    return;
  }
  stage_products<MP_NT, GATHER_LDG>(a.A, a.xg, e0, ne, r0, nr, prod, srp);
  __syncthreads();
  for (int t = tid; t < nr; t += MP_NT) {
    double s = 0.0;
    for (int e = srp[t]; e < srp[t + 1]; ++e) s += prod[e];
    if (t >= MP_NT) operands(r0 + t);
    dual_row_mp(a, es, ps, r0 + t, s, yo, bi, yb, axp, axbp);
  }
}

__device__ __forceinline__ void primal_row_mp(const MpIter& a, const StepEntry& e, const PrevStep& ps, int r,
                                              double q, double t, double xo, double xb0, double cr, double lr,
                                              double ur, double qbp, double tbp) {
  const double qb = ps.first ? q : r_fma(ps.ib_prev, q, r_mul(r_sub(1.0, ps.ib_prev), qbp));   // Q x_bar^k
  const double tau = e.tau_p, ib = e.inv_beta;
  const double qmd = r_fma(ib, q, r_mul(r_sub(1.0, ib), qb));                                // Q x_md^k
  const double g = r_add(r_add(qmd, t), cr);                 // Q x_md + c - A'y+
  const double xn = fmin(fmax(r_fma(-tau, g, xo), lr), ur);  // proj_X(x - tau g)
  const double xb = r_fma(ib, xn, r_mul(r_sub(1.0, ib), xb0));
  const double tb = ps.first ? t : r_fma(ib, t, r_mul(r_sub(1.0, ib), tbp));                 // -A'y_bar^{k+1}
  a.x[r] = xn;
  a.zout[r] = xn;
  a.xbar[r] = xb;
  a.qxb[r] = qb;
  a.aty[r] = t;
  a.atyb[r] = tb;
}

// fresh: Q x^k comes from the check before (only the A' part is gathered)
__global__ void __launch_bounds__(MP_NT, MinBlocks<double, MP_NT>::value) k_primal_mp(MpIter a, int j, int fresh) {
  __shared__ double prod[BNNZ];
  __shared__ int srp[BROWS + 1];
  __shared__ int ssp[BROWS];
  const int bk = a.actP ? a.actP[blockIdx.x] : (int)blockIdx.x;
  if (bk < 0) return;
  const int inst = a.blk_inst_P[bk];
  const DevState& S = a.st[inst];
  if (S.status != ST_RUNNING) return;
  const int tid = threadIdx.x;
  const int r0 = a.P.blk[bk], r1 = a.P.blk[bk + 1], nr = r1 - r0;
  const int e0 = a.P.rp[r0], ne = a.P.rp[r1] - e0;
  const StepEntry& es = a.tab[inst * a.C + j];
  const PrevStep ps = prev_step(a.tab + (size_t)inst * a.C, j, S.k_epoch, a.accelerate);
  double xo = 0.0, xb = 0.0, cr = 0.0, lr = 0.0, ur = 0.0, qbp = 0.0, tbp = 0.0;
  auto operands = [&](int r) {
    xo = a.x[r]; xb = a.xbar[r]; cr = a.c[r]; lr = a.l[r]; ur = a.u[r];
    if (!ps.first) { qbp = a.qxb[r]; tbp = a.atyb[r]; }
  };
  if (tid < nr) operands(r0 + tid);
  stage_products<MP_NT, GATHER_LDG>(a.P, a.zin, e0, ne, r0, nr, prod, srp, fresh ? a.n : 0);
  for (int t = tid; t < nr; t += MP_NT) ssp[t] = a.P.split[r0 + t] - e0;
  __syncthreads();
  const double* fr = (S.restart && S.cand_avg) ? a.sQ[1] : a.sQ[0];
  for (int t = tid; t < nr; t += MP_NT) {
    double q = 0.0, w = 0.0;
    if (fresh) q = fr[r0 + t];
    else
      for (int e = srp[t]; e < ssp[t]; ++e) q += prod[e];
    for (int e = ssp[t]; e < srp[t + 1]; ++e) w += prod[e];
    if (t >= MP_NT) operands(r0 + t);
    primal_row_mp(a, es, ps, r0 + t, q, w, xo, xb, cr, lr, ur, qbp, tbp);
  }
}

// ---------------------------------------------------------------- the check
struct MpCheck {
  BCsr<double> A, P;
  const double *__restrict__ x, *__restrict__ y;   // the iterate checked (scaled)
  const double* __restrict__ axb;                  // A x_bar^k, Q x_bar^k of the last iteration k
  const double* __restrict__ qxb;
  double *sA0, *sA1, *sQ0, *sQ1;                   // out: A x, A x_bar [m]; Q x, Q x_bar [n]
  double *aty, *atyb;                              // mode 0: out, P's -A' part of y (= of y_bar)
  const StepEntry* __restrict__ tab;
  const int *__restrict__ blk_inst_A, *__restrict__ blk_inst_P;
  const DevState* __restrict__ st;
  int C, n, mode, last;                            // last: the step-table entry of the chunk's last iteration
};

// The products val[e] * v(col[e]) of one row block as stage_products forms
// them (0 where v gives none), so that sums over them are bitwise the
// iteration kernels' sums.
template <typename G>
__device__ __forceinline__ void stage_mp(const BCsr<double>& M, int e0, int ne, int r0, int nr, double* prod,
                                         int* srp, G v) {
  const int tid = threadIdx.x;
  for (int t = tid; t <= nr; t += MP_NT) srp[t] = M.rp[r0 + t] - e0;
  int ci[BEPT];
  double vv[BEPT];
#pragma unroll
  for (int k = 0; k < BEPT; ++k) {
    const int e = tid + k * MP_NT;
    if (e < ne) { ci[k] = __ldg(M.col + e0 + e); vv[k] = __ldg(M.val + e0 + e); }
  }
#pragma unroll
  for (int k = 0; k < BEPT; ++k) {
    const int e = tid + k * MP_NT;
    if (e < ne) prod[e] = v(ci[k], vv[k]);
  }
}

__global__ void __launch_bounds__(MP_NT, 4) k_mp_check_m(MpCheck a) {
  __shared__ double prod[BNNZ];
  __shared__ int srp[BROWS + 1];
  const int bk = blockIdx.x;
  const int inst = a.blk_inst_A[bk];
  if (a.st[inst].status != ST_RUNNING) return;
  const int r0 = a.A.blk[bk], r1 = a.A.blk[bk + 1], nr = r1 - r0;
  const int e0 = a.A.rp[r0], ne = a.A.rp[r1] - e0;
  stage_products<MP_NT, GATHER_LDG>(a.A, a.x, e0, ne, r0, nr, prod, srp);
  __syncthreads();
  const double ib = a.mode ? a.tab[inst * a.C + a.last].inv_beta : 1.0;
  for (int t = threadIdx.x; t < nr; t += MP_NT) {
    double s = 0.0;
    for (int e = srp[t]; e < srp[t + 1]; ++e) s += prod[e];
    const int r = r0 + t;
    a.sA0[r] = s;
    a.sA1[r] = a.mode ? r_fma(ib, s, r_mul(r_sub(1.0, ib), a.axb[r])) : s;   // x_bar^{k+1} (= x at mode 0)
  }
}

__global__ void __launch_bounds__(MP_NT, 4) k_mp_check_n(MpCheck a) {
  __shared__ double prod[BNNZ];
  __shared__ int srp[BROWS + 1];
  __shared__ int ssp[BROWS];
  const int bk = blockIdx.x;
  const int inst = a.blk_inst_P[bk];
  if (a.st[inst].status != ST_RUNNING) return;
  const int r0 = a.P.blk[bk], r1 = a.P.blk[bk + 1], nr = r1 - r0;
  const int e0 = a.P.rp[r0], ne = a.P.rp[r1] - e0;
  const int n = a.n;
  if (a.mode)   // the Q part of x^{k+1}; the A' parts are maintained
    stage_mp(a.P, e0, ne, r0, nr, prod, srp, [&](int c, double v) { return c < n ? v * __ldg(a.x + c) : 0.0; });
  else          // the start point: both parts
    stage_mp(a.P, e0, ne, r0, nr, prod, srp,
             [&](int c, double v) { return v * (c < n ? __ldg(a.x + c) : __ldg(a.y + (c - n))); });
  for (int t = threadIdx.x; t < nr; t += MP_NT) ssp[t] = a.P.split[r0 + t] - e0;
  __syncthreads();
  const double ib = a.mode ? a.tab[inst * a.C + a.last].inv_beta : 1.0;
  for (int t = threadIdx.x; t < nr; t += MP_NT) {
    double q = 0.0;
    for (int e = srp[t]; e < ssp[t]; ++e) q += prod[e];
    const int r = r0 + t;
    a.sQ0[r] = q;
    a.sQ1[r] = a.mode ? r_fma(ib, q, r_mul(r_sub(1.0, ib), a.qxb[r])) : q;
    if (!a.mode) {
      double w = 0.0;
      for (int e = ssp[t]; e < srp[t + 1]; ++e) w += prod[e];
      a.aty[r] = w;
      a.atyb[r] = w;
    }
  }
}

void mp_check_products(Work& w, int mode, long long chunk_len, cudaStream_t s) {
  MpCheck a{};
  a.A = w.A.bscaled();
  a.P = w.P.bscaled();
  a.x = w.x;
  a.y = w.y;
  a.axb = w.mp_axb;
  a.qxb = w.mp_qxb;
  a.sA0 = w.mp_sA[0]; a.sA1 = w.mp_sA[1];
  a.sQ0 = w.mp_sQ[0]; a.sQ1 = w.mp_sQ[1];
  a.aty = w.mp_aty; a.atyb = w.mp_atyb;
  a.tab = w.tab;
  a.blk_inst_A = w.blk_inst_A;
  a.blk_inst_P = w.blk_inst_P;
  a.st = w.st;
  a.C = w.tab_stride;
  a.n = w.n;
  a.mode = mode == 1 && chunk_len > 0 ? 1 : 0;
  a.last = (int)chunk_len - 1;
  if (w.m > 0) launch(k_mp_check_m, w.A.nblk, MP_NT, 0, s, a);
  launch(k_mp_check_n, w.P.nblk, MP_NT, 0, s, a);
}

// ------------------------------------------------------------ the iterations
// algorithmic bytes of one launch (kind 0 dual, 1 primal) over the running
// instances: the row-block kernels' bytes plus the maintained vectors (dual:
// A x, A x_bar read and written; primal: Q x_bar and A'y_bar read, Q x_bar,
// A'y, A'y_bar written; x^{k+1} written twice, no x_md, x_tilde); a fresh
// launch reads the check's product instead of gathering it
static double mp_launch_bytes(const Work& w, int kind, bool fresh) {
  const BatchState& b = *w.bst_host;
  if (kind == 0) {
    if (fresh) return 8.0 * 10.0 * b.run_m;
    return b.run_nnzA * 12.0 + 4.0 * (b.run_m + 1.0) + 8.0 * (b.run_n + 9.0 * b.run_m);
  }
  const double nnz = fresh ? b.run_nnzA : b.run_nnzP;   // the A' part of P holds A's nonzeros
  return nnz * 12.0 + 4.0 * (b.run_n + 1.0) + 8.0 * (14.0 * b.run_n + b.run_m);
}

static void run_chunk_mp(Work& w, int j0, int len, cudaStream_t s, bool compact) {
  Profiler& Pr = w.prof;
  MpIter a{};
  a.A = w.A.bscaled();
  a.P = w.P.bscaled();
  a.xg = w.x;
  a.ybar = w.ybar;
  a.b = w.bs;
  a.x = w.x;
  a.xbar = w.xbar;
  a.c = w.cs; a.l = w.ls; a.u = w.us;
  a.ax = w.mp_ax; a.axb = w.mp_axb; a.qxb = w.mp_qxb; a.aty = w.mp_aty; a.atyb = w.mp_atyb;
  a.sA[0] = w.mp_sA[0]; a.sA[1] = w.mp_sA[1];
  a.sQ[0] = w.mp_sQ[0]; a.sQ[1] = w.mp_sQ[1];
  a.tab = w.tab;
  a.blk_inst_A = w.blk_inst_A;
  a.blk_inst_P = w.blk_inst_P;
  a.st = w.st;
  a.ineq = w.row_ineq;
  a.C = w.tab_stride;
  a.n = w.n;
  a.accelerate = w.mp_accelerate;
  int gA = w.A.nblk, gP = w.P.nblk;
  if (compact) {   // the running instances' row blocks (as the row-block variants)
    a.actA = w.act_A;
    a.actP = w.act_P;
    gA = w.act_grid_A > 0 ? w.act_grid_A : w.bst_host->act_A;
    gP = w.act_grid_P > 0 ? w.act_grid_P : w.bst_host->act_P;
  }
  for (int j = j0; j < j0 + len; ++j) {
    const int fresh = j == 0 ? 1 : 0;   // every chunk from step 0 follows a check
    if (w.m > 0) {
      a.yold = w.Z[(j + 1) & 1] + w.n;
      a.ynew = w.Z[j & 1] + w.n;
      if (Pr.on) Pr.begin(0, s, mp_launch_bytes(w, 0, fresh));
      launch(k_dual_mp, gA, MP_NT, 0, s, a, j, fresh);
      if (Pr.on) Pr.end(s);
    }
    a.zin = w.Z[j & 1];
    a.zout = w.Z[(j + 1) & 1];
    if (Pr.on) Pr.begin(1, s, mp_launch_bytes(w, 1, fresh));
    launch(k_primal_mp, gP, MP_NT, 0, s, a, j, fresh);
    if (Pr.on) Pr.end(s);
  }
  w.y = w.Z[(j0 + len - 1) & 1] + w.n;
}

void iterate(Work& w, int len, bool mixed, int nt, cudaStream_t s, int j0, bool compact) {
  if (!w.mp) {
    iterate_chunk(w, len, mixed, nt, s, j0, compact);
    return;
  }
  if (len > 0) run_chunk_mp(w, j0, len, s, compact);
}

}  // namespace pdqp
