// Host-side view of the device buffers of one problem and the kernel-launch
// entry points used by the C ABI driver.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "common.cuh"

// Slots of the member-interleaved vectors of a family handle.
enum { IL_Z0 = 0, IL_Z1, IL_X, IL_XBAR, IL_XT, IL_YBAR, IL_C, IL_L, IL_U, IL_B, IL_YLO, IL_SLOTS };
// ... and of the family check (float64): the iterates and the row sums.
enum { ILK_X0 = 0, ILK_X1, ILK_Y0, ILK_Y1, ILK_SA0, ILK_SA1, ILK_SQ0, ILK_SQ1, ILK_ST0, ILK_ST1, ILK_SLOTS };

// Row blocks: every CUDA block of the SpMV kernels takes whole rows
// [blk[b], blk[b+1]) holding at most BNNZ nonzeros and BROWS rows; a row longer
// than BNNZ forms a block of its own.
constexpr int BNT = 256;            // threads per block
constexpr int BEPT = 8;             // nonzeros staged per thread
constexpr int BNNZ = BNT * BEPT;    // nonzeros per row block
constexpr int BROWS = 512;          // rows per row block
constexpr int LSEG = 2048;          // nonzeros per segment of a long row
constexpr int LR_ROWS = 256;        // rows per tile of the low-rank F' v reduction

template <typename V>
struct BCsr {
  const int* __restrict__ rp;
  const int* __restrict__ col;
  const V* __restrict__ val;
  const int* __restrict__ blk;     // row-block starts [nblk+1]
  const int* __restrict__ split;   // P only: first index of the A' part of each row
  int pf = 0;                      // 1: prefetch each row block's index and value quads to L2 (stage_products)
};

struct DCsr {
  int rows = 0;
  long long nnz = 0;
  int nblk = 0;
  int* rp = nullptr;          // [rows+1]
  int* col = nullptr;         // [nnz]
  int* blk = nullptr;         // [nblk+1]
  int* split = nullptr;       // [rows] (P only)
  int* meta = nullptr;        // int4 {r0, r1, e0, e1} per row block
  double* val = nullptr;      // original values
  double* sval = nullptr;     // scaled values, float64
  float* sval_f = nullptr;    // scaled values, float32 (mixed precision)
  // rows longer than BNNZ (each a row block of its own) are also cut into
  // segments of LSEG nonzeros that separate CUDA blocks sum in parallel
  int nlseg = 0;
  int4* lseg = nullptr;       // [nlseg] {row, first nonzero, end nonzero, row block}
  int2* blk_seg = nullptr;    // [nblk] {first segment, segments} of a long-row block
  double* lpart_d = nullptr;  // [nlseg] segment sums, float64
  float* lpart_f = nullptr;   // [nlseg] segment sums, float32
  // 1 when every instance's gathered vector is small (a few L1s): the row
  // blocks' gathers hit nearby and their index and value streams set the pace,
  // so the staging prefetches those to L2 (a batch of control QPs: 8111 -> 8374
  // solves/s); random gathers into a large vector bind otherwise and the extra
  // requests cost (n=1e6: 13.20 -> 13.08 solves/s)
  int pf = 0;
  Csr<double> orig() const { return Csr<double>{rp, col, val}; }
  Csr<double> scaled() const { return Csr<double>{rp, col, sval}; }
  Csr<float> scaled_f() const { return Csr<float>{rp, col, sval_f}; }
  BCsr<double> borig() const { return BCsr<double>{rp, col, val, blk, split, pf}; }
  BCsr<double> bscaled() const { return BCsr<double>{rp, col, sval, blk, split, pf}; }
  BCsr<float> bscaled_f() const { return BCsr<float>{rp, col, sval_f, blk, split, pf}; }
};

// Optional CUDA-event timing of kernel launches (per kind, see pdqp_profile).
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;   // pool; pairs (begin, end)
  std::vector<int> kind;         // kind of each pair in flight
  std::vector<double> kbytes;    // algorithmic bytes of each pair in flight
  long long launches[4] = {0, 0, 0, 0};
  double ms[4] = {0, 0, 0, 0};
  double bytes[4] = {0, 0, 0, 0};
  void begin(int k, cudaStream_t s, double b = 0.0);
  void end(cudaStream_t s);
  void harvest();                // after the stream was synchronised
  void reset();
  ~Profiler();
};

// Statuses of an instance beyond the ST_* of the device state: an
// infeasibility certificate was found (optional detection, not in the paper).
enum { ST_PRIMAL_INF = 4, ST_DUAL_INF = 5 };

// Per-instance result of the certificate tests of the last check: status
// ST_PRIMAL_INF / ST_DUAL_INF / 0, the iterate whose ray passed (0 current,
// 1 average) and the ray's objective term (Farkas value or |c'd|) that
// normalises it; dual_it / dual_scale hold the unbounded-direction test
// between the two passes.
struct InfState {
  int status, cert_it, dual_it, pad;
  double scale, dual_scale;
};

// Row blocks per CUDA block of the relKKT kernels; a chunk of KKT_CHUNK row
// blocks is KKT_CHUNK / KKT_GROUP groups.
constexpr int KKT_GROUP = 4;
static_assert(KKT_CHUNK % KKT_GROUP == 0, "a relKKT chunk holds whole groups");

struct Work {
  int n = 0, m = 0, m_eq = 0;   // totals over the batch (m_eq: single-instance value)
  int count = 1;                // instances stacked block-diagonally
  int num_sms = 152;
  Inst* inst = nullptr;             // [count]
  std::vector<Inst> inst_host;
  int* blk_inst_P = nullptr;        // [P.nblk] instance of every row block
  int* blk_inst_A = nullptr;        // [A.nblk]
  int* row_inst_n = nullptr;        // [n] instance of every variable
  int* row_inst_m = nullptr;        // [m] instance of every row
  unsigned char* row_ineq = nullptr;   // [m] 1 for an inequality row
  BatchState* bst = nullptr;
  BatchState* bst_host = nullptr;   // pinned mirror
  int tab_stride = 0;               // entries per instance in tab (the check period)
  DCsr P, A;   // P = [Q | -A'] (n rows, columns n+i for the A' part), A (m rows)
  double *c = nullptr, *b = nullptr, *l = nullptr, *u = nullptr;        // original data
  double *cs = nullptr, *bs = nullptr, *ls = nullptr, *us = nullptr;    // scaled data
  double *D1 = nullptr, *D2 = nullptr;        // views into dsc: D2 = dsc[0:n], D1 = dsc[n:n+m]
  double *iD1 = nullptr, *iD2 = nullptr;      // views into idsc = 1 / dsc
  double *dsc = nullptr, *idsc = nullptr, *nu = nullptr;   // scaling vector, inverse, row norms [n+m]
  double *ones = nullptr;                     // [max(n,m)] of 1.0
  // float64 iterates (scaled space).  Z[p] = [x_md ; y] (n+m): the primal
  // kernel of inner iteration j gathers Z[j&1] and writes the next x_md to
  // Z[(j+1)&1]; the dual kernel reads y from Z[(j+1)&1] and writes y+ to Z[j&1].
  double *x = nullptr, *xbar = nullptr, *xt = nullptr, *Z[2] = {nullptr, nullptr};
  double *ybar = nullptr, *ax = nullptr, *ay = nullptr;
  double *y = nullptr;         // the current y: Z[(len-1)&1] + n after a chunk of len iterations
  double *yk = nullptr;        // mixed mode: float64 materialised current y [m]
  // float32 iterates of the mixed mode (deltas from the float64 base xhi, yhi)
  float *fx = nullptr, *fxbar = nullptr, *fxt = nullptr, *fZ[2] = {nullptr, nullptr};
  float *fy = nullptr, *fybar = nullptr;
  float *fc = nullptr, *fb = nullptr, *fl = nullptr, *fu = nullptr, *fylo = nullptr;  // shifted data
  double *xhi = nullptr, *yhi = nullptr;
  double *prodAx = nullptr, *prodQx = nullptr, *prodATy = nullptr;      // [2][m], [2][n], [2][n]
  // low-rank factor (Q_total = Q + F F'), row-major n x r
  int r = 0;
  float* F = nullptr;        // original, float32
  double* Fo = nullptr;      // original, float64
  float* Fs = nullptr;       // D2 F, float32
  double* Fd = nullptr;      // D2 F, float64
  double* wlr = nullptr;     // [2][r] F~' v of the current products
  float* wlr_f = nullptr;    // [2][r] the same in float32 (float32 iteration)
  double* lr_part = nullptr; // [tiles][2][r] partial sums
  // Lanczos vectors: pu[p] (n) for A~'A~, pz[p] = [v_Q ; A~v_A] (n+m) the P input
  double *pu[2] = {nullptr, nullptr}, *pz[2] = {nullptr, nullptr};
  float *fpu[2] = {nullptr, nullptr}, *fpz[2] = {nullptr, nullptr};
  double *lw[2] = {nullptr, nullptr};    // Lanczos products A~'A~v and Q~v [n]
  float *flw[2] = {nullptr, nullptr};
  double *lz_al = nullptr, *lz_be = nullptr;   // [count][2][512] Lanczos coefficients
  unsigned* lz_ticket = nullptr;   // [nchunk_n] Lanczos chunk tickets (0 between launches)
  // relKKT groups: KKT_GROUP consecutive row blocks of one instance per CUDA
  // block of the check kernels (one field reduction per group)
  int ngrp_P = 0, ngrp_A = 0;
  int *grp_inst_P = nullptr, *grp_inst_A = nullptr;     // [ngrp] instance of each group
  int *grp_first_P = nullptr, *grp_first_A = nullptr;   // [count + 1] first group of each instance
  double2 *kkt_xx = nullptr, *kkt_yy = nullptr;   // [n], [m]: (x, x_bar), (y, y_bar) pairs the relKKT kernels gather
  // reductions
  double *part = nullptr;    // [PDQP_RED_BLOCKS][32] (legacy layout, pdqp_kkt_noalloc kernels)
  double *part_m = nullptr;  // [9][A.nblk]  field-major partial sums of the row-block kernels
  double *part_n = nullptr;  // [15][P.nblk]
  double *cpart_m = nullptr; // [9][nchunk_m]  chunk sums of part_m (KKT_CHUNK blocks each)
  double *cpart_n = nullptr; // [15][nchunk_n]
  int nchunk_m = 0, nchunk_n = 0, maxchunk_m = 0, maxchunk_n = 0;
  int* act_A = nullptr;      // batches: [A.nblk] row blocks of the running instances (count in bst)
  int* act_P = nullptr;      // [P.nblk]; -1 past the count
  int lz_compact = 0;          // Lanczos steps over the lists of w.act_A / w.act_P (counts in bst_host)
  int act_grid_A = 0, act_grid_P = 0;   // > 0: the grids of compacted launches (padded, for a captured graph)
  StepEntry* tab = nullptr;  // [count][tab_stride]
  DevState* st = nullptr;    // [count]
  DevState* st_host = nullptr;   // pinned mirror [count]
  // user-vector staging (float64)
  double *stage_n = nullptr, *stage_m = nullptr;
  // infeasibility certificates (this solve's options; buffers on first use)
  int detect = 0;
  double eps_inf = 1e-8;
  // Family handles (members that share the matrix): one member's sizes and
  // its P columns in local numbering (the A' part at fam_n + k), and the
  // member-interleaved copies of the iteration vectors, v[j * fam_ld + member],
  // that the family iteration kernels run on within a chunk (slots IL_*).
  int fam_count = 0, fam_n = 0, fam_m = 0, fam_ld = 0;
  long long fam_nnzP = 0, fam_nnzA = 0;
  int* famP_col = nullptr;
  bool fam_il = false;                       // eligible: no long rows, no low-rank term
  double* ild[11] = {};                      // float64 (allocated on first use)
  float* ilf[11] = {};                       // float32
  double* ilk[10] = {};                      // the check's interleaved iterates and row sums (ILK_*)
  double* kks[6] = {};                       // the check's row sums, member-major: A x (2) [m], Q x (2), A'y (2) [n]
  bool il_active = false;                    // this solve runs the interleaved kernels
  InfState* inf = nullptr;                   // [count]
  double *inf_x[2] = {nullptr, nullptr};     // rays of the current / average iterate, scaled [n]
  double *inf_y[2] = {nullptr, nullptr};     // [m]
  double *inf_zn = nullptr, *inf_zm = nullptr;       // zeros [n], [m]
  double *inf_lrec = nullptr, *inf_urec = nullptr;   // the box's recession cone: 0 / -inf / +inf [n]
  double *inf_part_m = nullptr, *inf_part_n = nullptr, *inf_cpart_m = nullptr, *inf_cpart_n = nullptr;
  // maintained products (float64 solves with options.maintained_products):
  // A~x^k, A~x_bar^k [m] of the last dual half-step; Q~x_bar^k and P's -A~'
  // part of y^{k+1}, y_bar^{k+1} [n] of the last primal half-step; the
  // check's A~x, A~x_bar [m] and Q~x, Q~x_bar [n] of its two iterates
  int mp = 0;                                // this solve maintains them
  int mp_accelerate = 0;                     // its options.accelerate
  double *mp_ax = nullptr, *mp_axb = nullptr, *mp_qxb = nullptr, *mp_aty = nullptr, *mp_atyb = nullptr;
  double *mp_sA[2] = {nullptr, nullptr}, *mp_sQ[2] = {nullptr, nullptr};
  Profiler prof;
};

namespace pdqp {

// Kernels the library launched (a graph replay counts the kernels it holds).
// A thread capturing a graph counts its launches in t_captured instead.
extern std::atomic<long long> g_launches;
extern thread_local bool t_capturing;
extern thread_local long long t_captured;
inline void count_launch() {
  if (t_capturing) ++t_captured;
  else g_launches.fetch_add(1, std::memory_order_relaxed);
}

// setup
// scaling pass number `pass` (kind: 0 inf, 1 l2, 2 l1): reads the factors
// from w.dsc (even pass) or w.nu (odd), writes them to the other buffer
void scale_pass(Work& w, int kind, int pass, cudaStream_t s);
void scale_reset(Work& w, cudaStream_t s);
// tmpl: a family handle's template, already scaled with the same factors:
// its scaled values are copied to every member
void scale_apply(Work& w, bool mixed, cudaStream_t s, const Work* tmpl = nullptr);
void lanczos_init(Work& w, bool mixed, cudaStream_t s);
void lanczos_step(Work& w, int t, const SolveParams& p, bool mixed, cudaStream_t s);
void norms_finish(Work& w, double normA_opt, double normQ_opt, cudaStream_t s);
// A family handle's members share the matrix, so its scaling vector and norm
// estimates are those of its one-member template t: copy them to every member.
void family_scaling(Work& w, const Work& t, cudaStream_t s);
void family_norms(Work& w, const Work& t, cudaStream_t s);
void count_running(Work& w, cudaStream_t s);
// batches: list the row blocks of the instances whose norm estimates still
// run (w.act_A / w.act_P, counts in w.bst) for compacted Lanczos steps
void lanczos_compact(Work& w, cudaStream_t s);
void init_iterates(Work& w, const double* x0, const double* y0, const SolveParams& p, cudaStream_t s);

// iteration
// Iterations j0 .. j0+len-1 of a chunk (j indexes the chunk's step table).
// compact: launch only the row blocks of the running instances (batches; the
// counts of the last check must be in bst_host).
// nt: 256 or 512 threads per row block, 1 the pipelined persistent kernels, 2
// the whole chunk in one cluster launch (only where chunk_cluster_ok), 3 the
// member-interleaved family kernels (only where w.fam_il, buffers allocated).
void iterate_chunk(Work& w, int len, bool mixed, int nt, cudaStream_t s, int j0 = 0, bool compact = false);
// iterate_chunk, or with w.mp the maintained-products kernels (float64, 256
// threads per row block; nt is not used; the chunk starts at j0 = 0 right
// after a check, whose products of the iterate it starts from)
void iterate(Work& w, int len, bool mixed, int nt, cudaStream_t s, int j0 = 0, bool compact = false);
// with w.mp: the check's products A~x, A~x_bar, Q~x, Q~x_bar of (x, x_bar)
// after chunk_len iterations (mode 1), or of the start point (mode 0, which
// also forms the A~' products of y)
void mp_check_products(Work& w, int mode, long long chunk_len, cudaStream_t s);
// few row blocks, no long rows, no low-rank term, the vector copies fit in shared memory
bool chunk_cluster_ok(const Work& w, bool mixed);
void prepare_chunk_cluster();           // once, outside any stream capture
void check(Work& w, const SolveParams& p, int mode, long long chunk_len, bool mixed, cudaStream_t s);

// infeasibility certificates: fill the recession-cone bounds once the
// buffers exist; after write_output, the certificates of the instances that
// ended infeasible replace their iterates
void infeas_prepare(Work& w, cudaStream_t s);
void write_certificates(Work& w, double* x_out, double* y_out, cudaStream_t s);

// results
void write_output(Work& w, double* x_out, double* y_out, cudaStream_t s);
void write_state(Work& w, double* x, double* y, double* xbar, double* ybar, cudaStream_t s);
void eval_kkt_user(Work& w, const double* x, const double* y, cudaStream_t s);

}  // namespace pdqp
