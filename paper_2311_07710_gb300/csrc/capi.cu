// C ABI of the rAPDHG solver: input validation, device memory, the host loop
// over chunks of `check_period` iterations, and result marshalling.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <atomic>
#include <climits>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "pdqp.h"
#include "solver.h"

// One chunk (check_period iterations + the check) captured as a CUDA graph,
// keyed by the solve parameters.
struct ChunkGraph {
  bool valid = false;
  SolveParams key{};
  int key_detect = 0;          // the certificate tests are part of the captured check
  int key_mp = 0;              // maintained products (their own iteration and check kernels)
  double key_eps_inf = 0.0;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;       // kernel nodes in the graph (counted per replay)
  int gA = 0, gP = 0;          // compacted chunks: the grids over the running row blocks
};

struct pdqp_problem {
  Work w;
  std::string err;
  cudaStream_t alloc_stream = nullptr;   // stream of the call that allocates (create, solve, set_lowrank_Q)
  bool mixed_ready = false;
  int last_precision = PDQP_PREC_FP64;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};   // solve start, setup done, loop done
  cudaStream_t cap = nullptr;                         // private stream for graph capture
  ChunkGraph graph;
  std::vector<ChunkGraph> cgraphs;                    // compacted chunks, by padded grids (ChunkGraph::gA, gP)
  std::vector<pdqp_info> infos;                       // per instance, from the last solve
  std::vector<void*> allocs;
  int tuned_nt[2] = {0, 0};                           // autotuned variant per precision (0: not yet)
  cudaEvent_t tune_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // Where the last solve stopped (what pdqp_get_state exports): its parameters,
  // the step-table position (iterations run since the table was last filled;
  // 0 at a check) and the iterations of the solve loop.
  bool solved = false;
  SolveParams end_p{};
  int end_pos = 0;
  long long end_k_total = 0;
  bool end_mp = false;         // the last solve maintained its products (no resumable state)
  // A state loaded by pdqp_set_state: the next solve continues from it.
  bool resume = false;
  SolveParams resume_p{};
  int resume_pos = 0, resume_recheck = 0;
  long long resume_k_total = 0;
  // A family handle's one-member problem: the members share its matrix, so the
  // scaling and the norm estimates run on it once and are copied to all.
  pdqp_problem* tmpl = nullptr;
};

static thread_local std::string g_create_error;

namespace {

struct Fail {
  pdqp_status st;
  std::string msg;
};

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      throw Fail{e_ == cudaErrorMemoryAllocation ? PDQP_ERR_OOM : PDQP_ERR_CUDA,      \
                 std::string(#call) + ": " + cudaGetErrorString(e_)};                \
  } while (0)

// Device memory of the handles and of their build temporaries comes from a
// library-owned stream-ordered pool per device that keeps up to POOL_KEEP bytes
// of freed blocks (the rest goes back to the device at synchronisation points),
// so handles of similar sizes reuse memory instead of paying cudaMalloc /
// cudaFree, which synchronise the device.
// The pool keeps a quarter of the device's memory (at least POOL_KEEP): a
// family handle holds tens of GB (its members' copies of the shared matrix),
// and mapping that much afresh for every handle, then unmapping it at its
// destruction, took ~30 ms each way.
constexpr uint64_t POOL_KEEP = 8ULL << 30;
cudaMemPool_t lib_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  CK(cudaMemPoolCreate(&pool, &props));
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  uint64_t keep = std::max<uint64_t>(POOL_KEEP, (uint64_t)total_b / 4);
  CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  pools[dev] = pool;
  return pool;
}

void* pool_alloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  const cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, lib_pool(), s);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    throw Fail{PDQP_ERR_OOM, "device memory exhausted"};
  }
  CK(e);
  return p;
}

// frees of a handle being destroyed (its work is done: every call that runs
// work on it synchronises its stream before returning) go to a stream of the library
cudaStream_t free_stream() {
  static cudaStream_t fs = [] {
    cudaStream_t t = nullptr;
    cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
    return t;
  }();
  return fs;
}

template <typename T>
T* dalloc(pdqp_problem* h, size_t count) {
  if (count == 0) count = 1;
  void* p = pool_alloc(count * sizeof(T), h->alloc_stream);
  h->allocs.push_back(p);
  return (T*)p;
}

template <typename T>
void to_device(T* dst, const T* src, size_t count, cudaStream_t s) {
  if (count) CK(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
}

// Fetch `count` elements of a caller array (host or device) into a host vector.
template <typename T>
std::vector<T> fetch(const T* p, size_t count, int mem, cudaStream_t s) {
  std::vector<T> v(count);
  if (count == 0) return v;
  if (mem == PDQP_MEM_DEVICE) {
    CK(cudaMemcpyAsync(v.data(), p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  } else {
    std::memcpy(v.data(), p, count * sizeof(T));
  }
  return v;
}

void check_space(const void* p, int mem, const char* what) {
  if (!p) return;
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) { cudaGetLastError(); at.type = cudaMemoryTypeUnregistered; }
  const bool dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  if (mem == PDQP_MEM_DEVICE && !dev)
    throw Fail{PDQP_ERR_INVALID, std::string(what) + " is not device memory but mem_space = PDQP_MEM_DEVICE"};
  if (mem == PDQP_MEM_HOST && at.type == cudaMemoryTypeDevice)
    throw Fail{PDQP_ERR_INVALID, std::string(what) + " is device memory but mem_space = PDQP_MEM_HOST"};
}

void validate_csr(const char* name, int64_t rows, int64_t cols, const std::vector<int32_t>& rp,
                  const std::vector<int32_t>& col, const std::vector<double>& val) {
  if (rp.empty() || rp[0] != 0) throw Fail{PDQP_ERR_INVALID, std::string(name) + ": rowptr[0] != 0"};
  for (int64_t i = 0; i < rows; ++i) {
    if (rp[i + 1] < rp[i]) throw Fail{PDQP_ERR_INVALID, std::string(name) + ": rowptr decreases"};
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      if (col[k] < 0 || col[k] >= cols)
        throw Fail{PDQP_ERR_INVALID, std::string(name) + ": column index out of range"};
      if (k > rp[i] && col[k] <= col[k - 1])
        throw Fail{PDQP_ERR_INVALID, std::string(name) + ": column indices not strictly increasing in a row"};
      if (!std::isfinite(val[k])) throw Fail{PDQP_ERR_INVALID, std::string(name) + ": non-finite value"};
    }
  }
}

// Transpose a CSR matrix (rows x cols) by a stable counting sort on the column
// index, so that the rows of the transpose are sorted.
void transpose_csr(int64_t rows, int64_t cols, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                   const std::vector<double>& val, std::vector<int32_t>& trp, std::vector<int32_t>& tcol,
                   std::vector<double>& tval) {
  const int64_t nnz = rp[rows];
  trp.assign(cols + 1, 0);
  for (int64_t k = 0; k < nnz; ++k) trp[col[k] + 1]++;
  for (int64_t j = 0; j < cols; ++j) trp[j + 1] += trp[j];
  std::vector<int32_t> cur(trp.begin(), trp.end() - 1);
  tcol.resize(nnz);
  tval.resize(nnz);
  for (int64_t i = 0; i < rows; ++i)
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t p = cur[col[k]]++;
      tcol[p] = (int32_t)i;
      tval[p] = val[k];
    }
}

// Blocks of rows [r0, r1), their ends appended to blk: each block is the
// longest run of rows from its first that holds at most BROWS rows and BNNZ
// nonzeros (one binary search on the nondecreasing row pointers per block); a
// row of more than BNNZ nonzeros is a block of its own.  Only differences of
// row pointers enter, so a block's rows do not depend on where rp starts.
void append_row_blocks(int64_t r0, int64_t r1, const std::vector<int32_t>& rp, std::vector<int32_t>& blk) {
  int64_t s = r0;
  while (s < r1) {
    int64_t e = s + 1;
    if ((int64_t)rp[s + 1] - rp[s] <= BNNZ) {
      const int64_t hi = std::min<int64_t>(r1, s + BROWS);
      e = std::upper_bound(rp.begin() + s + 1, rp.begin() + hi + 1, (int64_t)rp[s] + BNNZ,
                           [](int64_t v, int32_t x) { return v < (int64_t)x; }) -
          rp.begin() - 1;
    }
    blk.push_back((int32_t)e);
    s = e;
  }
}

// Row blocks of rows [0, rows), starting with 0.
std::vector<int32_t> row_blocks(int64_t rows, const std::vector<int32_t>& rp) {
  std::vector<int32_t> blk{0};
  append_row_blocks(0, rows, rp, blk);
  return blk;
}

// Segments of the long rows (blocks holding a single row of more than BNNZ
// nonzeros): LSEG nonzeros each, summed by separate CUDA blocks.
void build_long_segments(pdqp_problem* h, DCsr& M, const std::vector<int32_t>& rp, const std::vector<int32_t>& blk,
                         cudaStream_t s) {
  std::vector<int4> seg;
  std::vector<int2> bseg(blk.size() > 1 ? blk.size() - 1 : 1, make_int2(0, 0));
  for (size_t b = 0; b + 1 < blk.size(); ++b) {
    const int r0 = blk[b], r1 = blk[b + 1];
    const long long e0 = rp[r0], e1 = rp[r1];
    if (r1 - r0 != 1 || e1 - e0 <= BNNZ) continue;
    bseg[b] = make_int2((int)seg.size(), (int)((e1 - e0 + LSEG - 1) / LSEG));
    for (long long e = e0; e < e1; e += LSEG)
      seg.push_back(make_int4(r0, (int)e, (int)std::min(e1, e + LSEG), (int)b));
  }
  M.nlseg = (int)seg.size();
  if (M.nlseg == 0) return;
  M.lseg = dalloc<int4>(h, seg.size());
  to_device(M.lseg, seg.data(), seg.size(), s);
  M.blk_seg = dalloc<int2>(h, bseg.size());
  to_device(M.blk_seg, bseg.data(), bseg.size(), s);
  M.lpart_d = dalloc<double>(h, seg.size());
  M.lpart_f = dalloc<float>(h, seg.size());
  CK(cudaStreamSynchronize(s));   // the host vectors die here
}

void upload_csr(pdqp_problem* h, DCsr& M, int rows, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                const std::vector<double>& val, const std::vector<int32_t>* split, const std::vector<int32_t>& blk,
                cudaStream_t s) {
  M.rows = rows;
  M.nnz = rp[rows];
  // 8 elements of padding: the pipelined kernels copy 16-byte aligned supersets
  M.rp = dalloc<int>(h, rows + 1 + 8);
  M.col = dalloc<int>(h, M.nnz + 8);
  M.val = dalloc<double>(h, M.nnz + 8);
  M.sval = dalloc<double>(h, M.nnz + 8);
  CK(cudaMemsetAsync(M.rp, 0, (rows + 1 + 8) * sizeof(int), s));
  CK(cudaMemsetAsync(M.col, 0, (M.nnz + 8) * sizeof(int), s));
  CK(cudaMemsetAsync(M.val, 0, (M.nnz + 8) * sizeof(double), s));
  CK(cudaMemsetAsync(M.sval, 0, (M.nnz + 8) * sizeof(double), s));
  to_device(M.rp, rp.data(), rows + 1, s);
  to_device(M.col, col.data(), M.nnz, s);
  to_device(M.val, val.data(), M.nnz, s);
  M.nblk = (int)blk.size() - 1;
  M.blk = dalloc<int>(h, blk.size());
  to_device(M.blk, blk.data(), blk.size(), s);
  std::vector<int32_t> meta(4 * (size_t)(M.nblk > 0 ? M.nblk : 1), 0);
  for (int b = 0; b < M.nblk; ++b) {
    meta[4 * b + 0] = blk[b];
    meta[4 * b + 1] = blk[b + 1];
    meta[4 * b + 2] = rp[blk[b]];
    meta[4 * b + 3] = rp[blk[b + 1]];
  }
  M.meta = dalloc<int>(h, meta.size());
  to_device(M.meta, meta.data(), meta.size(), s);
  if (split) {
    M.split = dalloc<int>(h, rows);
    to_device(M.split, split->data(), rows, s);
  }
  build_long_segments(h, M, rp, blk, s);
  CK(cudaStreamSynchronize(s));   // the host vectors die with the caller
}

// Buffers of the certificate tests (first solve that asks for them).
void alloc_infeas(pdqp_problem* h, cudaStream_t s) {
  Work& w = h->w;
  if (w.inf) return;
  const size_t n = (size_t)w.n, m = (size_t)w.m;
  w.inf = dalloc<InfState>(h, w.count);
  for (int k = 0; k < 2; ++k) {
    w.inf_x[k] = dalloc<double>(h, n);
    w.inf_y[k] = dalloc<double>(h, m);
    CK(cudaMemsetAsync(w.inf_x[k], 0, std::max<size_t>(n, 1) * sizeof(double), s));
    CK(cudaMemsetAsync(w.inf_y[k], 0, std::max<size_t>(m, 1) * sizeof(double), s));
  }
  w.inf_zn = dalloc<double>(h, n);
  w.inf_zm = dalloc<double>(h, m);
  w.inf_lrec = dalloc<double>(h, n);
  w.inf_urec = dalloc<double>(h, n);
  w.inf_part_m = dalloc<double>(h, (size_t)9 * std::max(w.A.nblk, 1));
  w.inf_part_n = dalloc<double>(h, (size_t)15 * std::max(w.P.nblk, 1));
  w.inf_cpart_m = dalloc<double>(h, (size_t)9 * std::max(w.nchunk_m, 1));
  w.inf_cpart_n = dalloc<double>(h, (size_t)15 * std::max(w.nchunk_n, 1));
  CK(cudaMemsetAsync(w.inf, 0, sizeof(InfState) * w.count, s));
  CK(cudaMemsetAsync(w.inf_zn, 0, std::max<size_t>(n, 1) * sizeof(double), s));
  CK(cudaMemsetAsync(w.inf_zm, 0, std::max<size_t>(m, 1) * sizeof(double), s));
  CK(cudaMemsetAsync(w.inf_part_m, 0, (size_t)9 * std::max(w.A.nblk, 1) * sizeof(double), s));
  CK(cudaMemsetAsync(w.inf_part_n, 0, (size_t)15 * std::max(w.P.nblk, 1) * sizeof(double), s));
  pdqp::infeas_prepare(w, s);
  CK(cudaGetLastError());
}

void alloc_mixed(pdqp_problem* h) {
  if (h->mixed_ready) return;
  Work& w = h->w;
  const int n = w.n, m = w.m;
  w.P.sval_f = dalloc<float>(h, w.P.nnz + 8);
  w.A.sval_f = dalloc<float>(h, w.A.nnz + 8);
  CK(cudaMemsetAsync(w.P.sval_f, 0, (w.P.nnz + 8) * sizeof(float), h->alloc_stream));
  CK(cudaMemsetAsync(w.A.sval_f, 0, (w.A.nnz + 8) * sizeof(float), h->alloc_stream));
  w.fx = dalloc<float>(h, n); w.fxbar = dalloc<float>(h, n); w.fxt = dalloc<float>(h, n);
  w.fZ[0] = dalloc<float>(h, (size_t)n + m); w.fZ[1] = dalloc<float>(h, (size_t)n + m);
  w.fybar = dalloc<float>(h, m); w.yk = dalloc<double>(h, m);
  w.fpu[0] = dalloc<float>(h, n); w.fpu[1] = dalloc<float>(h, n);
  w.fpz[0] = dalloc<float>(h, (size_t)n + m); w.fpz[1] = dalloc<float>(h, (size_t)n + m);
  w.flw[0] = dalloc<float>(h, n); w.flw[1] = dalloc<float>(h, n);
  w.fc = dalloc<float>(h, n); w.fl = dalloc<float>(h, n); w.fu = dalloc<float>(h, n);
  w.fb = dalloc<float>(h, m); w.fylo = dalloc<float>(h, m);
  w.xhi = dalloc<double>(h, n); w.yhi = dalloc<double>(h, m);
  w.prodAx = dalloc<double>(h, 2 * (size_t)m);
  w.prodQx = dalloc<double>(h, 2 * (size_t)n);
  w.prodATy = dalloc<double>(h, 2 * (size_t)n);
  h->mixed_ready = true;
}

// The member-interleaved vectors of a family handle for one precision (on
// the first solve that uses them).
void alloc_il(pdqp_problem* h, bool mixed) {
  Work& w = h->w;
  const size_t ld = (size_t)w.fam_ld, n = (size_t)w.fam_n, m = (size_t)w.fam_m;
  const size_t len[IL_SLOTS] = {n + m, n + m, n, n, n, m, n, n, n, m, m};
  for (int k = 0; k < IL_SLOTS; ++k) {
    if (mixed && !w.ilf[k]) w.ilf[k] = dalloc<float>(h, len[k] * ld);
    if (!mixed && !w.ild[k]) w.ild[k] = dalloc<double>(h, len[k] * ld);
  }
  const size_t klen[ILK_SLOTS] = {n, n, m, m, m, m, n, n, n, n};
  for (int k = 0; k < ILK_SLOTS; ++k)
    if (!w.ilk[k]) w.ilk[k] = dalloc<double>(h, klen[k] * ld);
  const size_t cnt = (size_t)w.fam_count;
  const size_t slen[6] = {m, m, n, n, n, n};
  for (int k = 0; k < 6; ++k)
    if (!w.kks[k]) w.kks[k] = dalloc<double>(h, slen[k] * cnt);
}

// the maintained products' vectors (first solve with options.maintained_products)
void alloc_mp(pdqp_problem* h) {
  Work& w = h->w;
  if (w.mp_ax) return;
  const size_t n = std::max(w.n, 1), m = std::max(w.m, 1);
  w.mp_ax = dalloc<double>(h, m);
  w.mp_axb = dalloc<double>(h, m);
  w.mp_qxb = dalloc<double>(h, n);
  w.mp_aty = dalloc<double>(h, n);
  w.mp_atyb = dalloc<double>(h, n);
  for (int k = 0; k < 2; ++k) {
    w.mp_sA[k] = dalloc<double>(h, m);
    w.mp_sQ[k] = dalloc<double>(h, n);
  }
}

SolveParams make_params(const pdqp_options& o) {
  SolveParams p{};
  p.step_rule = o.step_rule;
  p.restart_rule = o.restart_rule;
  p.accelerate = o.accelerate ? 1 : 0;
  p.fixed_K = o.fixed_K;
  p.check_period = o.check_period;
  p.mixed = o.precision == PDQP_PREC_MIXED;
  p.max_iter = o.max_iter;
  p.eps = o.eps;
  p.beta_suff = o.beta_suff;
  p.beta_nec = o.beta_nec;
  p.beta_art = o.beta_art;
  p.pw_theta = o.pw_theta;
  p.eps_zero = o.eps_zero;
  p.norm_tol = o.norm_tol;
  p.norm_iters = o.norm_iters;
  p.spmv_threads = o.spmv_threads;
  return p;
}

void validate_options(const pdqp_options& o) {
  auto bad = [](const char* m) { throw Fail{PDQP_ERR_INVALID, m}; };
  if (o.precision != PDQP_PREC_FP64 && o.precision != PDQP_PREC_MIXED) bad("options.precision");
  if (o.step_rule != PDQP_STEP_ADAPTIVE && o.step_rule != PDQP_STEP_THEORY) bad("options.step_rule");
  if (o.restart_rule < 0 || o.restart_rule > 3) bad("options.restart_rule");
  if (o.check_period < 2 || o.check_period > PDQP_MAX_CHECK || (o.check_period & 1))
    bad("options.check_period must be even and in [2, 4096]");
  if (o.max_iter < 1) bad("options.max_iter must be >= 1");
  if (!(o.eps >= 0.0)) bad("options.eps must be >= 0");
  if ((o.restart_rule == PDQP_RESTART_FIXED || o.step_rule == PDQP_STEP_THEORY) && o.fixed_K < 1)
    bad("options.fixed_K must be >= 1");
  if (o.norm_iters < 1 || o.norm_iters > 512) bad("options.norm_iters must be in [1, 512]");
  if (o.spmv_threads != 0 && o.spmv_threads != 1 && o.spmv_threads != 2 && o.spmv_threads != 3 &&
      o.spmv_threads != 256 && o.spmv_threads != 512)
    bad("options.spmv_threads must be 0, 1, 2, 3, 256 or 512");
  if (o.detect_infeasibility != 0 && o.detect_infeasibility != 1) bad("options.detect_infeasibility must be 0 or 1");
  if (o.detect_infeasibility && !(o.eps_infeasible > 0.0 && o.eps_infeasible < 1.0))
    bad("options.eps_infeasible must be in (0, 1)");
  if (o.maintained_products != 0 && o.maintained_products != 1) bad("options.maintained_products must be 0 or 1");
  if (o.maintained_products && o.precision != PDQP_PREC_FP64)
    bad("options.maintained_products needs precision PDQP_PREC_FP64 (the check's products must be float64)");
  if (o.maintained_products && o.spmv_threads != 0 && o.spmv_threads != 256)
    bad("options.maintained_products runs the 256-thread row-block kernels: spmv_threads must be 0 or 256");
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Read the batch counters (8 bytes) -- the only host round trip per chunk.
void sync_batch(pdqp_problem* h, cudaStream_t s) {
  CK(cudaMemcpyAsync(h->w.bst_host, h->w.bst, sizeof(BatchState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h->w.prof.on) h->w.prof.harvest();
}

// Read every instance's scalar state.
void sync_state(pdqp_problem* h, cudaStream_t s) {
  CK(cudaMemcpyAsync(h->w.st_host, h->w.st, sizeof(DevState) * h->w.count, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h->w.prof.on) h->w.prof.harvest();
}

void fill_info(pdqp_info* info, const DevState& S, pdqp_status status, bool lanczos) {
  std::memset(info, 0, sizeof(*info));
  info->status = status;
  info->iterations = S.k_total;
  info->restarts = S.restarts;
  info->r_primal = S.out_parts[0];
  info->r_dual = S.out_parts[1];
  info->r_gap = S.out_parts[2];
  info->rel_kkt = S.out_parts[3];
  info->primal_obj = S.out_parts[4];
  info->dual_obj = S.out_parts[5];
  info->norm_A = S.normA;
  info->norm_Q = S.normQ;
  info->omega = S.omega;
  info->norm_iters = lanczos ? S.pi_iters : 0;
}

// Launch one full chunk through the cached graph (capturing it first if needed).
// Batches whose running instances hold less than half of the row blocks
// launch only those blocks (direct launches sized by the last check's counts)
// instead of replaying the full-grid chunk graph.
bool compact_now(const Work& w, const SolveParams& p) {
  if (w.count <= 1 || p.spmv_threads == 1 || p.spmv_threads == 2 || p.spmv_threads == 3) return false;
  return 2LL * w.bst_host->act_P < (long long)w.P.nblk;
}

// Iterations j0 .. j0+len-1 with variant nt captured into a graph (for the
// tuner: each candidate is timed as the solve loop runs it, replayed).
cudaGraphExec_t capture_iterations(pdqp_problem* h, int len, bool mixed, int nt, int j0, long long* kernels) {
  Work& w = h->w;
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  pdqp::t_capturing = true;    // captured, not launched
  pdqp::t_captured = 0;
  pdqp::iterate(w, len, mixed, nt, h->cap, j0);
  pdqp::t_capturing = false;
  *kernels = pdqp::t_captured;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamEndCapture(h->cap, &graph));
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(e);
  return exec;
}

// Capture one chunk (check_period iterations and the check) into c: over all
// row blocks, or (compact) over the compacted lists of the running instances'
// row blocks at the grids gA, gP.
void capture_chunk(pdqp_problem* h, const SolveParams& p, bool mixed, bool compact, int gA, int gP,
                   ChunkGraph& c) {
  Work& w = h->w;
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  pdqp::t_capturing = true;    // captured, not launched
  pdqp::t_captured = 0;
  w.act_grid_A = compact ? std::max(gA, 1) : 0;
  w.act_grid_P = compact ? std::max(gP, 1) : 0;
  pdqp::iterate(w, p.check_period, mixed, p.spmv_threads, h->cap, 0, compact);
  w.act_grid_A = w.act_grid_P = 0;
  pdqp::check(w, p, 1, p.check_period, mixed, h->cap);
  pdqp::t_capturing = false;
  c.kernels = pdqp::t_captured;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamEndCapture(h->cap, &graph));
  const cudaError_t e = cudaGraphInstantiate(&c.exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(e);
  c.key = p;
  c.key_detect = w.detect;
  c.key_eps_inf = w.eps_inf;
  c.key_mp = w.mp;
  c.valid = true;
  c.gA = gA;
  c.gP = gP;
}

// a captured chunk is valid for the solve parameters and certificate options
// it was captured with
bool graph_matches(const ChunkGraph& c, const Work& w, const SolveParams& p) {
  return c.valid && std::memcmp(&c.key, &p, sizeof(SolveParams)) == 0 && c.key_detect == w.detect &&
         c.key_eps_inf == w.eps_inf && c.key_mp == w.mp;
}

void launch_chunk_graph(pdqp_problem* h, const SolveParams& p, bool mixed, cudaStream_t s) {
  ChunkGraph& g = h->graph;
  if (!graph_matches(g, h->w, p)) {
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    g.valid = false;
    capture_chunk(h, p, mixed, false, 0, 0, g);
  }
  CK(cudaGraphLaunch(g.exec, s));
  pdqp::g_launches += g.kernels;
}

// Drop every captured chunk graph (a buffer they point into was replaced).
void drop_graphs(pdqp_problem* h) {
  if (h->graph.exec) { cudaGraphExecDestroy(h->graph.exec); h->graph.exec = nullptr; }
  h->graph.valid = false;
  for (auto& c : h->cgraphs)
    if (c.exec) cudaGraphExecDestroy(c.exec);
  h->cgraphs.clear();
}

// A compacted chunk (a batch whose running instances hold less than half of
// the row blocks) through a graph captured at grids padded to powers of two:
// the block lists are device data that each check rewrites (-1 past the
// count), so one graph serves until the padded size changes -- a few graphs
// per solve, against two direct launches per iteration in the batch's tail.
static int pad_grid(int c, int cap) {
  if (c <= 0) return 0;
  int g = 1;
  while (g < c) g <<= 1;
  return std::min(g, cap);
}

void launch_compact_graph(pdqp_problem* h, const SolveParams& p, bool mixed, cudaStream_t s) {
  Work& w = h->w;
  const int gA = pad_grid(w.bst_host->act_A, w.A.nblk), gP = pad_grid(w.bst_host->act_P, w.P.nblk);
  ChunkGraph* g = nullptr;
  for (ChunkGraph& c : h->cgraphs)
    if (c.gA == gA && c.gP == gP && graph_matches(c, w, p)) g = &c;
  if (!g) {
    if (h->cgraphs.size() >= 32) {   // many option sets on one handle: start the cache over
      for (auto& c : h->cgraphs)
        if (c.exec) cudaGraphExecDestroy(c.exec);
      h->cgraphs.clear();
    }
    ChunkGraph c;
    capture_chunk(h, p, mixed, true, gA, gP, c);
    h->cgraphs.push_back(c);
    g = &h->cgraphs.back();
  }
  CK(cudaGraphLaunch(g->exec, s));
  pdqp::g_launches += g->kernels;
}

pdqp_status finish_status(int st) {
  switch (st) {
    case ST_OPTIMAL: return PDQP_OK;
    case ST_ITER_LIMIT: return PDQP_ITER_LIMIT;
    case ST_NUMERICAL: return PDQP_NUMERICAL;
    case ST_PRIMAL_INF: return PDQP_PRIMAL_INFEASIBLE;
    case ST_DUAL_INF: return PDQP_DUAL_INFEASIBLE;
    default: return PDQP_ERR_CUDA;
  }
}

// The autotuned iteration-kernel variant of each problem shape (sizes,
// nonzeros, row blocks, batch count, low-rank rank, precision), kept for the
// process: a new handle of a shape tuned before starts with its variant
// instead of timing the candidates again (every variant gives the same bits,
// so this changes only the time).
struct TuneKey {
  long long n, m, nnzP, nnzA;
  int nblkP, nblkA, nlsegP, nlsegA, count, r, mixed;
  bool operator<(const TuneKey& o) const {
    return std::tie(n, m, nnzP, nnzA, nblkP, nblkA, nlsegP, nlsegA, count, r, mixed) <
           std::tie(o.n, o.m, o.nnzP, o.nnzA, o.nblkP, o.nblkA, o.nlsegP, o.nlsegA, o.count, o.r, o.mixed);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

TuneKey tune_key(const Work& w, bool mixed) {
  return TuneKey{w.n, w.m, w.P.nnz, w.A.nnz, w.P.nblk, w.A.nblk, w.P.nlseg, w.A.nlseg, w.count, w.r, mixed ? 1 : 0};
}
int tuned_lookup(const Work& w, bool mixed) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(tune_key(w, mixed));
  return it == g_tuned.end() ? 0 : it->second;
}
void tuned_store(const Work& w, bool mixed, int nt) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[tune_key(w, mixed)] = nt;
}

pdqp_status solve_impl(pdqp_problem* h, const pdqp_options& o, const double* x0, const double* y0,
                       double* x_out, double* y_out, pdqp_info* info, int mem, cudaStream_t s) {
  const double t0 = now_s();
  Work& w = h->w;
  h->alloc_stream = s;   // buffers a solve adds (mixed precision, a longer step table)
  validate_options(o);
  if (mem != PDQP_MEM_HOST && mem != PDQP_MEM_DEVICE) throw Fail{PDQP_ERR_INVALID, "mem_space"};
  check_space(x0, mem, "x0");
  check_space(y0, mem, "y0");
  check_space(x_out, mem, "x_out");
  check_space(y_out, mem, "y_out");
  const bool mixed = o.precision == PDQP_PREC_MIXED;
  const bool cluster_ok = pdqp::chunk_cluster_ok(w, mixed);
  if (o.spmv_threads == 2 && !cluster_ok)
    throw Fail{PDQP_ERR_INVALID, "options.spmv_threads = 2 needs at most 64 row blocks of A and of P, no row "
                                 "longer than a row block, no low-rank term and 3n + 2m values within 200 KB"};
  if (cluster_ok) pdqp::prepare_chunk_cluster();
  // family handles run on member-interleaved vectors unless a row-block
  // variant is asked for (no low-rank term, no long rows)
  const bool il_ok = w.fam_il && w.r == 0;
  if (o.spmv_threads == 3 && !il_ok)
    throw Fail{PDQP_ERR_INVALID, "options.spmv_threads = 3 needs a family handle without long rows or low-rank term"};
  // maintained products: float64 row-block kernels over the whole handle
  const bool mp = o.maintained_products != 0;
  if (mp && w.r > 0) throw Fail{PDQP_ERR_INVALID, "options.maintained_products: the problem has a low-rank term"};
  if (mp && (w.A.nlseg > 0 || w.P.nlseg > 0))
    throw Fail{PDQP_ERR_INVALID, "options.maintained_products: a row of A or P holds more nonzeros than a row block"};
  if (mp && h->resume)
    throw Fail{PDQP_ERR_INVALID, "options.maintained_products: a solve resumed from pdqp_set_state is not supported"};
  const bool use_il = il_ok && !mp && (o.spmv_threads == 0 || o.spmv_threads == 3);
  if (mixed) alloc_mixed(h);
  if (use_il) alloc_il(h, mixed);
  w.il_active = use_il;
  if (!use_il && !w.kkt_xx) {   // the row-block checks gather both iterates of a column at once
    w.kkt_xx = dalloc<double2>(h, std::max(w.n, 1));
    w.kkt_yy = dalloc<double2>(h, std::max(w.m, 1));
  }
  w.detect = o.detect_infeasibility ? 1 : 0;
  w.eps_inf = o.eps_infeasible;
  if (w.detect) alloc_infeas(h, s);
  SolveParams p = make_params(o);
  if (use_il) p.spmv_threads = 3;
  w.mp = mp ? 1 : 0;
  w.mp_accelerate = p.accelerate;
  if (mp) {
    alloc_mp(h);
    p.spmv_threads = 256;
  }

  // a state loaded by pdqp_set_state: the solve continues from it, so the
  // parameters that shape the trajectory must be the saved solve's
  const bool resuming = h->resume;
  if (resuming) {
    const SolveParams& q = h->resume_p;
    if (x0 || y0) throw Fail{PDQP_ERR_INVALID, "a resumed solve starts from the loaded state: x0 and y0 must be NULL"};
    if (p.step_rule != q.step_rule || p.restart_rule != q.restart_rule || p.accelerate != q.accelerate ||
        p.fixed_K != q.fixed_K || p.check_period != q.check_period || p.mixed != q.mixed ||
        p.beta_suff != q.beta_suff || p.beta_nec != q.beta_nec || p.beta_art != q.beta_art ||
        p.pw_theta != q.pw_theta || p.eps_zero != q.eps_zero)
      throw Fail{PDQP_ERR_INVALID, "a resumed solve needs the saved solve's precision, check period, step, "
                                   "restart and primal-weight options"};
    if (o.max_iter <= h->resume_k_total)
      throw Fail{PDQP_ERR_INVALID, "options.max_iter must exceed the iterations of the loaded state"};
  }
  h->resume = false;
  h->solved = false;

  // start point in device memory
  const double* dx0 = x0;
  const double* dy0 = y0;
  if (mem == PDQP_MEM_HOST) {
    if (x0) { to_device(w.stage_n, x0, w.n, s); dx0 = w.stage_n; }
    if (y0) { to_device(w.stage_m, y0, w.m, s); dy0 = w.stage_m; }
  }

  h->last_precision = o.precision;
  if (w.tab_stride < o.check_period) {
    w.tab = dalloc<StepEntry>(h, (size_t)w.count * o.check_period);
    w.tab_stride = o.check_period;
    drop_graphs(h);
  }
  CK(cudaEventRecord(h->ev[0], s));
  // preprocessing (Section 5): 10 Ruiz passes, l2, Pock-Chambolle (a resumed
  // solve has its scaling vector from the loaded state)
  // A family handle runs both on its template (one member, the same row
  // blocks, sums and thread mapping as each member's part of the replicated
  // matrix, hence the same bits) unless a low-rank term, which the template
  // lacks, enters the norm of Q.
  pdqp_problem* const ft = h->tmpl;
  Work& sw = ft ? ft->w : w;
  if (ft) ft->alloc_stream = s;
  if (!resuming) {
    pdqp::scale_reset(sw, s);
    if (o.scaling) {
      int pass = 0;
      for (int i = 0; i < o.ruiz_iters; ++i) pdqp::scale_pass(sw, 0, pass++, s);
      if (o.l2_scaling) pdqp::scale_pass(sw, 1, pass++, s);
      if (o.pock_chambolle) pdqp::scale_pass(sw, 2, pass++, s);
      if ((pass & 1) && sw.n + sw.m > 0)   // the factors are in the second buffer
        CK(cudaMemcpyAsync(sw.dsc, sw.nu, ((size_t)sw.n + sw.m) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    if (ft) pdqp::family_scaling(w, sw, s);
  }
  // a fresh family solve scales the template and copies its values to the
  // members; a resumed one scales its own (its factors come from the state)
  const bool rep_vals = ft && !resuming;
  if (rep_vals) {
    if (mixed) alloc_mixed(ft);
    pdqp::scale_apply(sw, mixed, s);
  }
  pdqp::scale_apply(w, mixed, s, rep_vals ? &sw : nullptr);

  // spectral norms of the scaled matrices (a resumed solve keeps its own)
  const bool run_lanczos = !resuming && !(o.norm_A > 0.0 && o.norm_Q > 0.0);
  pdqp_problem* const lh = ft && w.r == 0 ? ft : h;
  Work& lw = lh->w;
  if (run_lanczos) {   // (on the template: a fresh solve, so it was scaled above)
    pdqp::lanczos_init(lw, mixed, s);
    lw.lz_compact = 0;
    for (int t = 0; t < o.norm_iters; ++t) {
      pdqp::lanczos_step(lw, t, p, mixed, s);
      if ((t & 7) == 7) {
        pdqp::count_running(lw, s);
        if (lw.count > 1) pdqp::lanczos_compact(lw, s);
        sync_batch(lh, s);
        if (lw.bst_host->lz_running == 0) break;
        // once the instances still estimating hold less than half of the row
        // blocks, the next steps launch over theirs only
        lw.lz_compact = lw.count > 1 && 2LL * lw.bst_host->act_P < (long long)lw.P.nblk ? 1 : 0;
      }
    }
    lw.lz_compact = 0;
  }
  if (!resuming) {
    pdqp::norms_finish(lw, o.norm_A, o.norm_Q, s);
    if (lh != h) pdqp::family_norms(w, lw, s);
  }
  CK(cudaEventRecord(h->ev[1], s));
  long long k_total = 0;
  int pos = 0;   // step-table position: iterations since the table was last filled
  if (!resuming) {
    pdqp::init_iterates(w, dx0, dy0, p, s);
    pdqp::check(w, p, 0, 0, mixed, s);
  } else {
    // the loaded state stopped mid-period (at the iteration limit): run the rest
    // of that period on its step table, then its check; or it stopped at a
    // check that the iteration limit ended before the restart decision: take
    // that check again (same iterates, same values) to make the decision
    k_total = h->resume_k_total;
    pos = h->resume_pos;
    if (pos > 0) {
      const int len = (int)std::min<long long>(o.check_period - pos, o.max_iter - k_total);
      pdqp::iterate(w, len, mixed, p.spmv_threads, s, pos);
      pdqp::check(w, p, 1, len, mixed, s);
      k_total += len;
      pos = (pos + len) % o.check_period;
    } else if (h->resume_recheck) {
      pdqp::check(w, p, 1, 0, mixed, s);
    } else {
      pdqp::count_running(w, s);
    }
  }
  CK(cudaGetLastError());
  sync_batch(h, s);

  bool timed_out = false;
  // autotuning of the iteration-kernel variant: the first full chunk runs
  // two rounds of TUNE iterations with each candidate (interleaved, so that no
  // candidate always runs first on a cold cache), keeps the fastest by its
  // better round and runs the rest of the chunk with it; the iterates do not
  // depend on the variant.  Problems of a few row blocks also try the
  // one-launch cluster chunk.  Each candidate's iterations are captured into a
  // graph and replayed, as the solve loop runs them (direct launches would
  // charge the per-iteration variants launch gaps that graphs do not have);
  // with the event profiler on, they are launched directly.
  static const int kCand[4] = {256, 512, 1, 2};
  const int ncand = cluster_ok ? 4 : 3;
  constexpr int TUNE = 4, ROUNDS = 2;
  const bool autotune = o.spmv_threads == 0 && !use_il && !mp;
  int& tuned = h->tuned_nt[mixed ? 1 : 0];
  if (autotune && !tuned) tuned = tuned_lookup(w, mixed);   // a handle of the same shape tuned before
  if (autotune && tuned) p.spmv_threads = tuned;
  while (w.bst_host->running > 0) {
    const long long len = std::min<long long>(o.check_period, o.max_iter - k_total);
    const bool tune_now = autotune && !tuned && len == o.check_period && len >= 2 * ncand * ROUNDS * TUNE;
    // per-kernel event timing needs direct launches (events recorded by graph
    // nodes cannot be timed), so profiling bypasses the graph
    if (tune_now) {
      for (auto& e : h->tune_ev)
        if (!e) CK(cudaEventCreate(&e));
      float best_ms[4] = {0.f, 0.f, 0.f, 0.f};
      int j = 0;
      const bool replay = !w.prof.on && !o.no_graphs;
      if (replay) pdqp::iterate(w, 0, mixed, 1, s, 0);   // one-time setup of the pipelined variant
      for (int r = 0; r < ROUNDS; ++r) {
        cudaGraphExec_t ex[4] = {nullptr, nullptr, nullptr, nullptr};
        long long kern[4] = {0, 0, 0, 0};
        if (replay)
          for (int c = 0; c < ncand; ++c) ex[c] = capture_iterations(h, TUNE, mixed, kCand[c], j + c * TUNE, &kern[c]);
        CK(cudaEventRecord(h->tune_ev[0], s));
        for (int c = 0; c < ncand; ++c) {
          if (replay) {
            CK(cudaGraphLaunch(ex[c], s));
            pdqp::g_launches += kern[c];
          } else {
            pdqp::iterate(w, TUNE, mixed, kCand[c], s, j);
          }
          j += TUNE;
          CK(cudaEventRecord(h->tune_ev[c + 1], s));
        }
        CK(cudaEventSynchronize(h->tune_ev[ncand]));
        for (int c = 0; c < ncand; ++c)
          if (ex[c]) cudaGraphExecDestroy(ex[c]);
        for (int c = 0; c < ncand; ++c) {
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, h->tune_ev[c], h->tune_ev[c + 1]));
          if (r == 0 || ms < best_ms[c]) best_ms[c] = ms;
        }
      }
      int bc = 0;
      for (int c = 1; c < ncand; ++c)
        if (best_ms[c] < best_ms[bc]) bc = c;
      tuned = kCand[bc];
      tuned_store(w, mixed, tuned);
      p.spmv_threads = tuned;
      pdqp::iterate(w, (int)len - j, mixed, p.spmv_threads, s, j);
      pdqp::check(w, p, 1, len, mixed, s);
    } else if (len == o.check_period && !o.no_graphs && !w.prof.on) {
      if (compact_now(w, p)) launch_compact_graph(h, p, mixed, s);
      else launch_chunk_graph(h, p, mixed, s);
    } else {
      pdqp::iterate(w, (int)len, mixed, p.spmv_threads, s, 0, compact_now(w, p));
      pdqp::check(w, p, 1, len, mixed, s);
    }
    CK(cudaGetLastError());
    k_total += len;
    pos = (int)(len % o.check_period);
    sync_batch(h, s);
    if (w.bst_host->running > 0 && now_s() - t0 > o.time_limit) { timed_out = true; break; }
  }
  CK(cudaEventRecord(h->ev[2], s));

  // the returned iterate
  if (x_out || y_out) {
    double* ox = x_out;
    double* oy = y_out;
    if (mem == PDQP_MEM_HOST) { ox = x_out ? w.stage_n : nullptr; oy = y_out ? w.stage_m : nullptr; }
    pdqp::write_output(w, ox, oy, s);
    pdqp::write_certificates(w, ox, oy, s);
    if (mem == PDQP_MEM_HOST) {
      if (x_out) CK(cudaMemcpyAsync(x_out, w.stage_n, w.n * sizeof(double), cudaMemcpyDeviceToHost, s));
      if (y_out && w.m) CK(cudaMemcpyAsync(y_out, w.stage_m, w.m * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
  }
  CK(cudaGetLastError());
  sync_state(h, s);
  // per-instance results; the call returns the worst status
  h->infos.assign(w.count, pdqp_info{});
  pdqp_status result = PDQP_OK;
  float t_setup = 0.f, t_iter = 0.f;
  CK(cudaEventElapsedTime(&t_setup, h->ev[0], h->ev[1]));
  CK(cudaEventElapsedTime(&t_iter, h->ev[1], h->ev[2]));
  const double secs = now_s() - t0;
  for (int i = 0; i < w.count; ++i) {
    const DevState& S = w.st_host[i];
    const pdqp_status si = (timed_out && S.status == ST_RUNNING) ? PDQP_TIME_LIMIT : finish_status(S.status);
    fill_info(&h->infos[i], S, si, run_lanczos);
    h->infos[i].setup_seconds = 1e-3 * t_setup;
    h->infos[i].iterate_seconds = 1e-3 * t_iter;
    h->infos[i].seconds = secs;
    h->infos[i].spmv_threads = p.spmv_threads == 0 ? 256 : p.spmv_threads;
    if (si > result) result = si;
  }
  if (info) {
    *info = h->infos[0];
    info->status = result;
    for (int i = 1; i < w.count; ++i) info->iterations = std::max(info->iterations, h->infos[i].iterations);
  }
  h->solved = true;
  h->end_mp = mp;
  h->end_p = p;
  h->end_pos = pos;
  h->end_k_total = k_total;
  return result;
}

// One instance as given by the caller (host or device pointers per mem_space).
// rebase: the pointers point into a packed (block-diagonal) batch, so the row
// pointers are shifted to start at 0 and col_base is taken off every column.
struct InstanceIn {
  int64_t n = 0, m = 0, m_eq = 0;
  const int32_t *Q_rowptr = nullptr, *Q_col = nullptr;
  const double* Q_val = nullptr;
  const int32_t *A_rowptr = nullptr, *A_col = nullptr;
  const double* A_val = nullptr;
  const double *c = nullptr, *b = nullptr, *l = nullptr, *u = nullptr;
  bool rebase = false;
  int64_t col_base = 0;
};

// Row pointers shifted to start at 0, columns shifted by -base; a value that
// leaves int32 becomes -1, which validation rejects.
void rebase_rowptr(std::vector<int32_t>& rp) {
  const int64_t b0 = rp.empty() ? 0 : rp[0];
  for (auto& v : rp) {
    const int64_t t = (int64_t)v - b0;
    v = (t < INT32_MIN || t > INT32_MAX) ? -1 : (int32_t)t;
  }
}

void rebase_cols(std::vector<int32_t>& col, int64_t base) {
  for (auto& v : col) {
    const int64_t t = (int64_t)v - base;
    v = (t < 0 || t > INT32_MAX) ? -1 : (int32_t)t;
  }
}

// Host-side stacking of `count` instances: P = [Q | -A'] and A with global
// columns, row blocks that never cross an instance, per-row / per-block
// instance tables and the data vectors.
struct Stack {
  int64_t N = 0, M = 0;
  int count = 0;
  std::vector<int32_t> prp{0}, pcol, psplit, arp{0}, acol, pblk{0}, ablk{0}, binst_p, binst_a, rinst_n, rinst_m;
  std::vector<double> pval, aval, hc, hb, hl, hu;
  std::vector<unsigned char> ineq;
  std::vector<Inst> insts;
};

// One instance's rows of P = [Q | -A'] and of A with global column indices,
// its row pointers and P's split from 0, its row blocks in local rows.
struct Piece {
  std::vector<int32_t> prp, pcol, psplit, arp, acol, pbl, abl;
  std::vector<double> pval, aval, c, l, u, b;
};

// Validate and assemble instance i (its first variable xoff, first row yoff,
// N variables in the whole stack); throws Fail.
Piece make_piece(const InstanceIn& in, int64_t xoff, int64_t yoff, int64_t N, int mem, cudaStream_t s) {
  const int64_t n = in.n, m = in.m;
  for (auto pr : {(const void*)in.Q_rowptr, (const void*)in.Q_col, (const void*)in.Q_val,
                  (const void*)in.A_rowptr, (const void*)in.A_col, (const void*)in.A_val, (const void*)in.c,
                  (const void*)in.b, (const void*)in.l, (const void*)in.u})
    check_space(pr, mem, "input array");
  std::vector<int32_t> qrp = fetch(in.Q_rowptr, n + 1, mem, s);
  if (in.rebase) rebase_rowptr(qrp);
  const int64_t nnzQ = qrp[n];
  if (nnzQ < 0 || (nnzQ > 0 && (!in.Q_col || !in.Q_val))) throw Fail{PDQP_ERR_INVALID, "Q: bad nnz or null arrays"};
  std::vector<int32_t> qcol = fetch(in.Q_col, nnzQ, mem, s);
  if (in.rebase) rebase_cols(qcol, in.col_base);
  std::vector<double> qval = fetch(in.Q_val, nnzQ, mem, s);
  Piece P;
  std::vector<int32_t> icol;
  std::vector<double> ival;
  P.arp.assign(m + 1, 0);
  if (m > 0) {
    P.arp = fetch(in.A_rowptr, m + 1, mem, s);
    if (in.rebase) rebase_rowptr(P.arp);
    const int64_t nnzA = P.arp[m];
    if (nnzA < 0 || (nnzA > 0 && (!in.A_col || !in.A_val))) throw Fail{PDQP_ERR_INVALID, "A: bad nnz or null arrays"};
    icol = fetch(in.A_col, nnzA, mem, s);
    if (in.rebase) rebase_cols(icol, in.col_base);
    ival = fetch(in.A_val, nnzA, mem, s);
  }
  P.c = fetch(in.c, n, mem, s);
  P.l = fetch(in.l, n, mem, s);
  P.u = fetch(in.u, n, mem, s);
  if (m > 0) P.b = fetch(in.b, m, mem, s);
  validate_csr("Q", n, n, qrp, qcol, qval);
  validate_csr("A", m, n, P.arp, icol, ival);
  for (int64_t j = 0; j < n; ++j) {
    if (!std::isfinite(P.c[j])) throw Fail{PDQP_ERR_INVALID, "c: non-finite entry"};
    if (std::isnan(P.l[j]) || std::isnan(P.u[j]) || P.l[j] > P.u[j] || P.l[j] == INFINITY || P.u[j] == -INFINITY)
      throw Fail{PDQP_ERR_INVALID, "bounds: need l <= u, l < +inf, u > -inf"};
  }
  for (int64_t r = 0; r < m; ++r)
    if (!std::isfinite(P.b[r])) throw Fail{PDQP_ERR_INVALID, "b: non-finite entry"};
  std::vector<int32_t> trp, tcol;
  std::vector<double> tval;
  if (m > 0) transpose_csr(m, n, P.arp, icol, ival, trp, tcol, tval);
  else trp.assign(n + 1, 0);
  // rows of P = [Q | -A'] with global columns: x part xoff + j, y part N + yoff + r
  const size_t nnzP = (size_t)nnzQ + tcol.size();
  if (nnzP > (size_t)INT32_MAX - 16) throw Fail{PDQP_ERR_INVALID, "nnz(Q) + nnz(A) exceeds 2^31"};
  P.pcol.resize(nnzP);
  P.pval.resize(nnzP);
  P.prp.resize(n + 1);
  P.psplit.resize(n);
  P.prp[0] = 0;
  size_t e = 0;
  for (int64_t j = 0; j < n; ++j) {
    for (int32_t k = qrp[j]; k < qrp[j + 1]; ++k, ++e) {
      P.pcol[e] = (int32_t)(xoff + qcol[k]);
      P.pval[e] = qval[k];
    }
    P.psplit[j] = (int32_t)e;
    for (int32_t k = trp[j]; k < trp[j + 1]; ++k, ++e) {
      P.pcol[e] = (int32_t)(N + yoff + tcol[k]);
      P.pval[e] = -tval[k];
    }
    P.prp[j + 1] = (int32_t)e;
  }
  P.acol.resize(icol.size());
  for (size_t k = 0; k < icol.size(); ++k) P.acol[k] = (int32_t)(xoff + icol[k]);
  P.aval = std::move(ival);
  P.pbl = row_blocks(n, P.prp);
  P.abl = m > 0 ? row_blocks(m, P.arp) : std::vector<int32_t>{0};
  return P;
}

// Run fn(i) for i in [0, count) on up to 16 host threads; the Fail of the
// lowest failing i is rethrown (as a sequential loop would throw it).
template <class Fn>
void parallel_instances(int count, Fn fn) {
  const int nt = std::max(1, std::min<int>({count, 16, (int)std::max(1u, std::thread::hardware_concurrency())}));
  std::atomic<int> next{0};
  std::mutex mu;
  int fail_i = INT_MAX;
  Fail fail{PDQP_OK, ""};
  bool other = false;
  auto body = [&] {
    for (int i; (i = next.fetch_add(1)) < count;) {
      try {
        fn(i);
      } catch (const Fail& f) {
        std::lock_guard<std::mutex> lock(mu);
        if (i < fail_i) { fail_i = i; fail = f; }
      } catch (...) {
        std::lock_guard<std::mutex> lock(mu);
        other = true;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(body);
  body();
  for (auto& t : pool) t.join();
  if (fail_i != INT_MAX) throw fail;
  if (other) throw std::bad_alloc();
}

// Validate every instance and stack them block-diagonally: the instances are
// assembled in parallel, then copied into place after a prefix over sizes.
Stack stack_instances(int count, const InstanceIn* ins, int mem, cudaStream_t s) {
  if (count < 1) throw Fail{PDQP_ERR_INVALID, "count must be >= 1"};
  if (mem != PDQP_MEM_HOST && mem != PDQP_MEM_DEVICE) throw Fail{PDQP_ERR_INVALID, "mem_space"};
  Stack S;
  S.count = count;
  int64_t N = 0, M = 0;
  std::vector<int64_t> xoff(count), yoff(count);
  for (int i = 0; i < count; ++i) {
    const InstanceIn& in = ins[i];
    if (in.n < 1 || in.m < 0 || in.m_eq < 0 || in.m_eq > in.m)
      throw Fail{PDQP_ERR_INVALID, "sizes: need n >= 1, 0 <= m_eq <= m"};
    if (!in.Q_rowptr || !in.c || !in.l || !in.u) throw Fail{PDQP_ERR_INVALID, "null Q_rowptr, c, l or u"};
    if (in.m > 0 && (!in.A_rowptr || !in.b)) throw Fail{PDQP_ERR_INVALID, "null A_rowptr or b with m > 0"};
    xoff[i] = N;
    yoff[i] = M;
    N += in.n;
    M += in.m;
  }
  if (N > (1LL << 30) || M > (1LL << 30)) throw Fail{PDQP_ERR_INVALID, "total n or m exceeds 2^30"};
  S.N = N;
  S.M = M;
  std::vector<Piece> pieces(count);
  parallel_instances(count, [&](int i) { pieces[i] = make_piece(ins[i], xoff[i], yoff[i], N, mem, s); });
  // offsets of every instance's nonzeros and row blocks; the instances' records
  std::vector<int64_t> pe(count + 1, 0), ae(count + 1, 0);
  std::vector<int> pb(count + 1, 0), ab(count + 1, 0);
  S.insts.resize(count);
  for (int i = 0; i < count; ++i) {
    const Piece& P = pieces[i];
    pe[i + 1] = pe[i] + (int64_t)P.pcol.size();
    ae[i + 1] = ae[i] + (int64_t)P.acol.size();
    pb[i + 1] = pb[i] + (int)P.pbl.size() - 1;
    ab[i + 1] = ab[i] + (int)P.abl.size() - 1;
    Inst& I = S.insts[i];
    I.n = (int)ins[i].n;
    I.m = (int)ins[i].m;
    I.m_eq = (int)ins[i].m_eq;
    I.xoff = (int)xoff[i];
    I.yoff = (int)yoff[i];
    I.bP0 = pb[i];
    I.bP1 = pb[i + 1];
    I.bA0 = ab[i];
    I.bA1 = ab[i + 1];
    I.cP0 = i == 0 ? 0 : S.insts[i - 1].cP0 + kkt_chunks(S.insts[i - 1].bP0, S.insts[i - 1].bP1);
    I.cA0 = i == 0 ? 0 : S.insts[i - 1].cA0 + kkt_chunks(S.insts[i - 1].bA0, S.insts[i - 1].bA1);
  }
  if (pe[count] > (int64_t)INT32_MAX - 16) throw Fail{PDQP_ERR_INVALID, "nnz(Q) + nnz(A) exceeds 2^31"};
  if (ae[count] > (int64_t)INT32_MAX - 16) throw Fail{PDQP_ERR_INVALID, "nnz(A) exceeds 2^31"};
  S.prp.assign(N + 1, 0);
  S.psplit.resize(N);
  S.pcol.resize(pe[count]);
  S.pval.resize(pe[count]);
  S.arp.assign(M + 1, 0);
  S.acol.resize(ae[count]);
  S.aval.resize(ae[count]);
  S.pblk.assign(pb[count] + 1, 0);
  S.binst_p.resize(pb[count]);
  S.ablk.assign(ab[count] + 1, 0);
  S.binst_a.resize(ab[count]);
  S.hc.resize(N);
  S.hl.resize(N);
  S.hu.resize(N);
  S.hb.resize(M);
  S.rinst_n.resize(N);
  S.rinst_m.resize(M);
  S.ineq.resize(M);
  parallel_instances(count, [&](int i) {
    Piece& P = pieces[i];
    const int64_t x0 = xoff[i], y0 = yoff[i], n = ins[i].n, m = ins[i].m;
    for (int64_t j = 0; j < n; ++j) {
      S.prp[x0 + j + 1] = (int32_t)(pe[i] + P.prp[j + 1]);
      S.psplit[x0 + j] = (int32_t)(pe[i] + P.psplit[j]);
    }
    std::copy(P.pcol.begin(), P.pcol.end(), S.pcol.begin() + pe[i]);
    std::copy(P.pval.begin(), P.pval.end(), S.pval.begin() + pe[i]);
    for (int64_t r = 0; r < m; ++r) S.arp[y0 + r + 1] = (int32_t)(ae[i] + P.arp[r + 1]);
    std::copy(P.acol.begin(), P.acol.end(), S.acol.begin() + ae[i]);
    std::copy(P.aval.begin(), P.aval.end(), S.aval.begin() + ae[i]);
    for (size_t q = 1; q < P.pbl.size(); ++q) {
      S.pblk[pb[i] + q] = (int32_t)(x0 + P.pbl[q]);
      S.binst_p[pb[i] + q - 1] = i;
    }
    for (size_t q = 1; q < P.abl.size(); ++q) {
      S.ablk[ab[i] + q] = (int32_t)(y0 + P.abl[q]);
      S.binst_a[ab[i] + q - 1] = i;
    }
    std::copy(P.c.begin(), P.c.end(), S.hc.begin() + x0);
    std::copy(P.l.begin(), P.l.end(), S.hl.begin() + x0);
    std::copy(P.u.begin(), P.u.end(), S.hu.begin() + x0);
    std::copy(P.b.begin(), P.b.end(), S.hb.begin() + y0);
    std::fill(S.rinst_n.begin() + x0, S.rinst_n.begin() + x0 + n, i);
    std::fill(S.rinst_m.begin() + y0, S.rinst_m.begin() + y0 + m, i);
    for (int64_t r = 0; r < m; ++r) S.ineq[y0 + r] = r >= ins[i].m_eq ? 1 : 0;
    P = Piece();   // free the piece as soon as it is placed
  });
  return S;
}

void begin_work(pdqp_problem* h, int64_t N, int64_t M, int m_eq, int count, const std::vector<Inst>& insts) {
  Work& w = h->w;
  w.n = (int)N;
  w.m = (int)M;
  w.m_eq = m_eq;
  w.count = count;
  w.inst_host = insts;
  w.nchunk_m = w.nchunk_n = w.maxchunk_m = w.maxchunk_n = 0;
  for (const Inst& I : insts) {
    const int cn = kkt_chunks(I.bP0, I.bP1), cm = kkt_chunks(I.bA0, I.bA1);
    w.nchunk_n += cn;
    w.nchunk_m += cm;
    w.maxchunk_n = std::max(w.maxchunk_n, cn);
    w.maxchunk_m = std::max(w.maxchunk_m, cm);
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&w.num_sms, cudaDevAttrMultiProcessorCount, dev));
}

// Upload the structure and data of a host stack.
void upload_stack(pdqp_problem* h, const Stack& S, cudaStream_t s) {
  Work& w = h->w;
  const size_t n = (size_t)S.N, m = (size_t)S.M;
  upload_csr(h, w.P, (int)S.N, S.prp, S.pcol, S.pval, &S.psplit, S.pblk, s);
  upload_csr(h, w.A, (int)S.M, S.arp, S.acol, S.aval, nullptr, S.ablk, s);
  w.inst = dalloc<Inst>(h, S.count);
  to_device(w.inst, S.insts.data(), S.count, s);
  w.blk_inst_P = dalloc<int>(h, S.binst_p.size());
  to_device(w.blk_inst_P, S.binst_p.data(), S.binst_p.size(), s);
  w.blk_inst_A = dalloc<int>(h, S.binst_a.size());
  to_device(w.blk_inst_A, S.binst_a.data(), S.binst_a.size(), s);
  w.row_inst_n = dalloc<int>(h, n);
  to_device(w.row_inst_n, S.rinst_n.data(), n, s);
  w.row_inst_m = dalloc<int>(h, m);
  to_device(w.row_inst_m, S.rinst_m.data(), m, s);
  w.row_ineq = dalloc<unsigned char>(h, m);
  to_device(w.row_ineq, S.ineq.data(), m, s);
  w.c = dalloc<double>(h, n);
  w.l = dalloc<double>(h, n);
  w.u = dalloc<double>(h, n);
  w.b = dalloc<double>(h, m);
  to_device(w.c, S.hc.data(), n, s);
  to_device(w.l, S.hl.data(), n, s);
  to_device(w.u, S.hu.data(), n, s);
  to_device(w.b, S.hb.data(), m, s);
  CK(cudaStreamSynchronize(s));   // the host vectors die with the caller
}

// Everything else a handle needs, sized from w.n, w.m, w.count and the blocks.
void alloc_work(pdqp_problem* h, cudaStream_t s) {
  Work& w = h->w;
  const size_t n = (size_t)w.n, m = (size_t)w.m;
  const int count = w.count;
  w.cs = dalloc<double>(h, n); w.ls = dalloc<double>(h, n); w.us = dalloc<double>(h, n); w.bs = dalloc<double>(h, m);
  w.dsc = dalloc<double>(h, n + m); w.idsc = dalloc<double>(h, n + m); w.nu = dalloc<double>(h, n + m);
  w.D2 = w.dsc; w.D1 = w.dsc + n; w.iD2 = w.idsc; w.iD1 = w.idsc + n;
  w.x = dalloc<double>(h, n); w.xbar = dalloc<double>(h, n); w.xt = dalloc<double>(h, n);
  w.Z[0] = dalloc<double>(h, n + m); w.Z[1] = dalloc<double>(h, n + m); w.ax = dalloc<double>(h, n);
  w.y = w.Z[1] + n;
  w.ybar = dalloc<double>(h, m); w.ay = dalloc<double>(h, m);
  w.pu[0] = dalloc<double>(h, n); w.pu[1] = dalloc<double>(h, n);
  w.pz[0] = dalloc<double>(h, n + m); w.pz[1] = dalloc<double>(h, n + m);
  w.lw[0] = dalloc<double>(h, n); w.lw[1] = dalloc<double>(h, n);
  w.lz_al = dalloc<double>(h, (size_t)count * 2 * 512); w.lz_be = dalloc<double>(h, (size_t)count * 2 * 512);
  w.part = dalloc<double>(h, (size_t)PDQP_RED_BLOCKS * 32);
  w.part_m = dalloc<double>(h, (size_t)9 * (w.A.nblk > 0 ? w.A.nblk : 1));
  w.part_n = dalloc<double>(h, (size_t)15 * (w.P.nblk > 0 ? w.P.nblk : 1));
  w.act_A = dalloc<int>(h, (size_t)std::max(w.A.nblk, 1));
  w.act_P = dalloc<int>(h, (size_t)std::max(w.P.nblk, 1));
  w.cpart_m = dalloc<double>(h, (size_t)9 * std::max(w.nchunk_m, 1));
  w.cpart_n = dalloc<double>(h, (size_t)15 * std::max(w.nchunk_n, 1));
  {  // the L2 prefetch of the row blocks' streams pays where every instance is small
    long long big = 0;
    for (const Inst& I : w.inst_host) big = std::max(big, (long long)I.n + I.m);
    w.P.pf = w.A.pf = big <= 32768 ? 1 : 0;
  }
  {  // relKKT groups: KKT_GROUP consecutive row blocks of one instance each
    const int count = (int)w.inst_host.size();
    std::vector<int> gi[2], gf[2];
    for (int side = 0; side < 2; ++side) {
      gf[side].assign((size_t)count + 1, 0);
      for (int i = 0; i < count; ++i) {
        const Inst& I = w.inst_host[i];
        const int nb = side ? I.bP1 - I.bP0 : I.bA1 - I.bA0;
        gf[side][i] = (int)gi[side].size();
        gi[side].insert(gi[side].end(), (size_t)((nb + KKT_GROUP - 1) / KKT_GROUP), i);
      }
      gf[side][count] = (int)gi[side].size();
    }
    w.ngrp_A = (int)gi[0].size();
    w.ngrp_P = (int)gi[1].size();
    w.grp_inst_A = dalloc<int>(h, std::max<size_t>(gi[0].size(), 1));
    w.grp_inst_P = dalloc<int>(h, std::max<size_t>(gi[1].size(), 1));
    w.grp_first_A = dalloc<int>(h, gf[0].size());
    w.grp_first_P = dalloc<int>(h, gf[1].size());
    if (!gi[0].empty()) to_device(w.grp_inst_A, gi[0].data(), gi[0].size(), s);
    if (!gi[1].empty()) to_device(w.grp_inst_P, gi[1].data(), gi[1].size(), s);
    to_device(w.grp_first_A, gf[0].data(), gf[0].size(), s);
    to_device(w.grp_first_P, gf[1].data(), gf[1].size(), s);
    CK(cudaStreamSynchronize(s));   // the host vectors go out of scope
  }
  w.lz_ticket = dalloc<unsigned>(h, (size_t)std::max(w.nchunk_n, 1));
  CK(cudaMemsetAsync(w.lz_ticket, 0, sizeof(unsigned) * std::max(w.nchunk_n, 1), s));
  w.st = dalloc<DevState>(h, count);
  w.bst = dalloc<BatchState>(h, 1);
  w.stage_n = dalloc<double>(h, n); w.stage_m = dalloc<double>(h, m);
  CK(cudaMallocHost(&w.st_host, sizeof(DevState) * count));
  CK(cudaMallocHost(&w.bst_host, sizeof(BatchState)));
  for (auto& e : h->ev) CK(cudaEventCreate(&e));
  CK(cudaMemsetAsync(w.st, 0, sizeof(DevState) * count, s));
  CK(cudaMemsetAsync(w.bst, 0, sizeof(BatchState), s));
  CK(cudaStreamSynchronize(s));
}

pdqp_problem* build_problem(int count, const InstanceIn* ins, int mem, cudaStream_t s) {
  const Stack S = stack_instances(count, ins, mem, s);
  pdqp_problem* h = new pdqp_problem();
  h->alloc_stream = s;
  try {
    begin_work(h, S.N, S.M, (int)ins[0].m_eq, count, S.insts);
    upload_stack(h, S, s);
    alloc_work(h, s);
  } catch (...) {
    pdqp_destroy(h);
    throw;
  }
  return h;
}

// ---------------------------------------------------------------- families
// Device-side replication of a one-instance stack into `count` copies.
__global__ void k_rep_rowptr(const int* __restrict__ trp, int rows_t, long long nnz_t, int count, int* __restrict__ rp) {
  const long long total = (long long)count * rows_t;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i <= total; i += (long long)gridDim.x * blockDim.x)
    rp[i] = i == total ? (int)(count * nnz_t) : (int)((i / rows_t) * nnz_t + trp[i % rows_t]);
}

// P mode: template columns j < n_t are x columns (instance offset inst * n_t),
// j >= n_t are y columns (global N + inst * m_t + j - n_t); A mode: x columns.
__global__ void k_rep_cols(const int* __restrict__ tcol, const double* __restrict__ tval, long long nnz_t, int count,
                           int n_t, int m_t, long long N, int pmode, int* __restrict__ col, double* __restrict__ val) {
  const long long total = (long long)count * nnz_t;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
    const long long inst = k / nnz_t, q = k % nnz_t;
    const int c = tcol[q];
    col[k] = (pmode && c >= n_t) ? (int)(N + inst * m_t + (c - n_t)) : (int)(inst * n_t + c);
    val[k] = tval[q];
  }
}

__global__ void k_rep_split(const int* __restrict__ tsplit, int n_t, long long nnz_t, int count, int* __restrict__ split) {
  const long long total = (long long)count * n_t;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    split[i] = (int)((i / n_t) * nnz_t + tsplit[i % n_t]);
}

// blk[0] = 0, blk[1 + inst*nb + q] = inst*rows_t + tblk[q+1]; meta per block
__global__ void k_rep_blocks(const int* __restrict__ tblk, int nb, int rows_t, int count, const int* __restrict__ rp,
                             int* __restrict__ blk, int* __restrict__ binst, int* __restrict__ meta) {
  const long long total = (long long)count * nb;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < total; b += (long long)gridDim.x * blockDim.x) {
    const long long inst = b / nb;
    const int q = (int)(b % nb);
    const int r0 = (int)(inst * rows_t + tblk[q]), r1 = (int)(inst * rows_t + tblk[q + 1]);
    if (b == 0) blk[0] = 0;
    blk[b + 1] = r1;
    binst[b] = (int)inst;
    meta[4 * b + 0] = r0;
    meta[4 * b + 1] = r1;
    meta[4 * b + 2] = rp[r0];
    meta[4 * b + 3] = rp[r1];
  }
}

__global__ void k_rep_rows(int n_t, int m_t, int m_eq, int count, int* __restrict__ rinst_n, int* __restrict__ rinst_m,
                           unsigned char* __restrict__ ineq) {
  const long long tn = (long long)count * n_t, tm = (long long)count * m_t;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tn + tm; i += (long long)gridDim.x * blockDim.x) {
    if (i < tn) {
      rinst_n[i] = (int)(i / n_t);
    } else {
      const long long r = i - tn;
      rinst_m[r] = (int)(r / m_t);
      ineq[r] = (r % m_t) >= m_eq ? 1 : 0;
    }
  }
}

__global__ void k_rep_vec(const double* __restrict__ t, int len, long long total, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    out[i] = t[i % len];
}

__global__ void k_count_nonfinite(const double* __restrict__ v, long long n, unsigned long long* __restrict__ cnt) {
  unsigned long long c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c += !isfinite(v[i]);
  if (c) atomicAdd(cnt, c);
}

int rep_grid(long long total) { return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 4096)); }

// Replicate a device CSR of one instance (template handle t) `count` times.
void replicate_csr(pdqp_problem* h, DCsr& M, const DCsr& T, int count, int n_t, int m_t, long long N, bool pmode,
                   cudaStream_t s) {
  const long long rows = (long long)count * T.rows, nnz = (long long)count * T.nnz;
  M.rows = (int)rows;
  M.nnz = nnz;
  M.rp = dalloc<int>(h, rows + 1 + 8);
  M.col = dalloc<int>(h, nnz + 8);
  M.val = dalloc<double>(h, nnz + 8);
  M.sval = dalloc<double>(h, nnz + 8);
  // k_rep_cols writes every index and value: only the padding past the end
  // needs zeros (the row pointers are small and cleared whole: no rows, no launch)
  CK(cudaMemsetAsync(M.rp, 0, (rows + 1 + 8) * sizeof(int), s));
  CK(cudaMemsetAsync(M.col + nnz, 0, 8 * sizeof(int), s));
  CK(cudaMemsetAsync(M.val + nnz, 0, 8 * sizeof(double), s));
  CK(cudaMemsetAsync(M.sval, 0, (nnz + 8) * sizeof(double), s));
  if (T.rows > 0) k_rep_rowptr<<<rep_grid(rows + 1), 256, 0, s>>>(T.rp, T.rows, T.nnz, count, M.rp);
  if (T.nnz > 0)
    k_rep_cols<<<rep_grid(nnz), 256, 0, s>>>(T.col, T.val, T.nnz, count, n_t, m_t, N, pmode ? 1 : 0, M.col, M.val);
  M.nblk = count * T.nblk;
  M.blk = dalloc<int>(h, (size_t)M.nblk + 1);
  M.meta = dalloc<int>(h, 4 * (size_t)(M.nblk > 0 ? M.nblk : 1));
  CK(cudaMemsetAsync(M.blk, 0, ((size_t)M.nblk + 1) * sizeof(int), s));
  int* binst = dalloc<int>(h, (size_t)std::max(M.nblk, 1));
  if (T.nblk > 0) k_rep_blocks<<<rep_grid(M.nblk), 256, 0, s>>>(T.blk, T.nblk, T.rows, count, M.rp, M.blk, binst, M.meta);
  if (pmode) {
    h->w.blk_inst_P = binst;
    M.split = dalloc<int>(h, rows);
    if (T.rows > 0) k_rep_split<<<rep_grid(rows), 256, 0, s>>>(T.split, T.rows, T.nnz, count, M.split);
  } else {
    h->w.blk_inst_A = binst;
  }
  CK(cudaGetLastError());
}

pdqp_problem* build_family(const InstanceIn& base, int count, const double* C, const double* B, int mem,
                           cudaStream_t s) {
  if (count < 1) throw Fail{PDQP_ERR_INVALID, "count must be >= 1"};
  if (!C || (base.m > 0 && !B)) throw Fail{PDQP_ERR_INVALID, "null C or B"};
  check_space(C, mem, "C");
  check_space(B, mem, "B");
  pdqp_problem* t = build_problem(1, &base, mem, s);   // validates the base problem
  pdqp_problem* h = nullptr;
  try {
    const Work& tw = t->w;
    const long long n_t = tw.n, m_t = tw.m;
    if ((long long)count * tw.P.nnz > INT32_MAX - 16 || (long long)count * tw.A.nnz > INT32_MAX - 16)
      throw Fail{PDQP_ERR_INVALID, "count * nnz exceeds 2^31"};
    if ((long long)count * n_t > (1LL << 30) || (long long)count * m_t > (1LL << 30))
      throw Fail{PDQP_ERR_INVALID, "total n or m exceeds 2^30"};
    std::vector<Inst> insts(count);
    const Inst& I0 = tw.inst_host[0];
    const int nbP = tw.P.nblk, nbA = tw.A.nblk;
    for (int i = 0; i < count; ++i) {
      Inst& I = insts[i];
      I = I0;
      I.xoff = (int)(i * n_t);
      I.yoff = (int)(i * m_t);
      I.bP0 = i * nbP;
      I.bP1 = (i + 1) * nbP;
      I.bA0 = i * nbA;
      I.bA1 = (i + 1) * nbA;
      I.cP0 = i * kkt_chunks(0, nbP);
      I.cA0 = i * kkt_chunks(0, nbA);
    }
    h = new pdqp_problem();
    h->alloc_stream = s;
    const long long N = count * n_t, M = count * m_t;
    begin_work(h, N, M, tw.m_eq, count, insts);
    Work& w = h->w;
    replicate_csr(h, w.P, tw.P, count, (int)n_t, (int)m_t, N, true, s);
    replicate_csr(h, w.A, tw.A, count, (int)n_t, (int)m_t, N, false, s);
    for (int side = 0; side < 2; ++side) {   // long-row segments: the template's, offset per member
      const DCsr& T = side == 0 ? tw.P : tw.A;
      DCsr& Mr = side == 0 ? w.P : w.A;
      if (T.nlseg == 0) continue;
      std::vector<int4> ts(T.nlseg);
      std::vector<int2> tb(T.nblk);
      CK(cudaMemcpy(ts.data(), T.lseg, ts.size() * sizeof(int4), cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(tb.data(), T.blk_seg, tb.size() * sizeof(int2), cudaMemcpyDeviceToHost));
      std::vector<int4> seg;
      std::vector<int2> bseg((size_t)count * T.nblk);
      for (int i = 0; i < count; ++i) {
        for (int b = 0; b < T.nblk; ++b)
          bseg[(size_t)i * T.nblk + b] = tb[b].y ? make_int2(tb[b].x + i * T.nlseg, tb[b].y) : make_int2(0, 0);
        for (const int4& q : ts)
          seg.push_back(make_int4(q.x + i * T.rows, (int)(q.y + (long long)i * T.nnz), (int)(q.z + (long long)i * T.nnz),
                                  q.w + i * T.nblk));
      }
      Mr.nlseg = (int)seg.size();
      Mr.lseg = dalloc<int4>(h, seg.size());
      to_device(Mr.lseg, seg.data(), seg.size(), s);
      Mr.blk_seg = dalloc<int2>(h, bseg.size());
      to_device(Mr.blk_seg, bseg.data(), bseg.size(), s);
      Mr.lpart_d = dalloc<double>(h, seg.size());
      Mr.lpart_f = dalloc<float>(h, seg.size());
      CK(cudaStreamSynchronize(s));
    }
    w.inst = dalloc<Inst>(h, count);
    to_device(w.inst, insts.data(), count, s);
    w.row_inst_n = dalloc<int>(h, N);
    w.row_inst_m = dalloc<int>(h, M);
    w.row_ineq = dalloc<unsigned char>(h, M);
    k_rep_rows<<<rep_grid(N + M), 256, 0, s>>>((int)n_t, (int)m_t, tw.m_eq, count, w.row_inst_n, w.row_inst_m,
                                               w.row_ineq);
    w.c = dalloc<double>(h, N);
    w.l = dalloc<double>(h, N);
    w.u = dalloc<double>(h, N);
    w.b = dalloc<double>(h, M);
    const cudaMemcpyKind kind = mem == PDQP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(w.c, C, (size_t)N * sizeof(double), kind, s));
    if (M > 0) CK(cudaMemcpyAsync(w.b, B, (size_t)M * sizeof(double), kind, s));
    k_rep_vec<<<rep_grid(N), 256, 0, s>>>(tw.l, (int)n_t, N, w.l);
    k_rep_vec<<<rep_grid(N), 256, 0, s>>>(tw.u, (int)n_t, N, w.u);
    unsigned long long* cnt = dalloc<unsigned long long>(h, 1);
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    k_count_nonfinite<<<rep_grid(N), 256, 0, s>>>(w.c, N, cnt);
    if (M > 0) k_count_nonfinite<<<rep_grid(M), 256, 0, s>>>(w.b, M, cnt);
    CK(cudaGetLastError());
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&bad, cnt, sizeof(bad), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (bad) throw Fail{PDQP_ERR_INVALID, "C or B: non-finite entry"};
    alloc_work(h, s);
    // one member's structure for the member-interleaved iteration kernels
    w.fam_count = count;
    w.fam_n = (int)n_t;
    w.fam_m = (int)m_t;
    w.fam_ld = (count + 127) / 128 * 128;   // whole warps of 4 float (2 double) members per lane
    w.fam_nnzP = tw.P.nnz;
    w.fam_nnzA = tw.A.nnz;
    w.fam_il = tw.P.nlseg == 0 && tw.A.nlseg == 0 && n_t > 0;
    if (w.fam_il) {
      w.famP_col = dalloc<int>(h, tw.P.nnz + 8);
      CK(cudaMemcpyAsync(w.famP_col, tw.P.col, (size_t)tw.P.nnz * sizeof(int), cudaMemcpyDeviceToDevice, s));
      CK(cudaStreamSynchronize(s));
    }
  } catch (...) {
    if (h) pdqp_destroy(h);
    pdqp_destroy(t);
    throw;
  }
  h->tmpl = t;
  return h;
}

// ---------------------------------------------------------------- one problem, built on the device
// pdqp_create of a single problem: the CSR input is copied to the device as
// given, validated there, A is transposed by a column count, scan, scatter
// and a per-column sort by row (the same A' as the stable counting sort of
// the host path), and P = [Q | -A'] is assembled row by row.  Only the greedy
// row blocks are formed on the host (from the row pointers), so the handle is
// the one build_problem makes.
enum : unsigned {
  VE_RP = 1u, VE_COL = 2u, VE_ORDER = 4u, VE_VAL = 8u, VE_C = 16u, VE_BOUNDS = 32u, VE_B = 64u, VE_LONG = 128u
};

// Row pointers outside [0, nnz] or decreasing are flagged first (thread per
// row); the entries are then checked per nonzero (its row by binary search), so
// long rows spread over the grid.
__global__ void k_validate_rowptr(const int* __restrict__ rp, int rows, long long nnz, unsigned* __restrict__ err) {
  unsigned e = 0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const int a = rp[r], b = rp[r + 1];
    if (a < 0 || b < a || b > nnz) e |= VE_RP;
  }
  if (e) atomicOr(err, e);
}

__device__ __forceinline__ int row_of(const int* __restrict__ rp, int rows, long long k) {
  int lo = 0, hi = rows - 1;   // last row with rp[row] <= k
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rp[mid] <= k) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// A nonzero of row r belongs to the instance rinst[r]: its column must lie in
// that instance's variables [ioff[inst], ioff[inst + 1]).
__global__ void k_validate_entries(const int* __restrict__ rp, const int* __restrict__ col,
                                   const double* __restrict__ val, int rows, long long nnz,
                                   const int* __restrict__ rinst, const int* __restrict__ ioff,
                                   unsigned* __restrict__ err) {
  unsigned e = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
    const int r = row_of(rp, rows, k);
    const int inst = rinst[r];
    const int c = col[k];
    if (c < ioff[inst] || c >= ioff[inst + 1]) e |= VE_COL;
    if (!isfinite(val[k])) e |= VE_VAL;
    if (k > rp[r] && c <= col[k - 1]) e |= VE_ORDER;
  }
  if (e) atomicOr(err, e);
}

__global__ void k_validate_vecs(const double* __restrict__ c, const double* __restrict__ l, const double* __restrict__ u,
                                int n, const double* __restrict__ b, int m, unsigned* __restrict__ err) {
  unsigned e = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n || i < m; i += gridDim.x * blockDim.x) {
    if (i < n) {
      if (!isfinite(c[i])) e |= VE_C;
      const double lo = l[i], hi = u[i];
      if (isnan(lo) || isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY) e |= VE_BOUNDS;
    }
    if (i < m && !isfinite(b[i])) e |= VE_B;
  }
  if (e) atomicOr(err, e);
}

__global__ void k_col_count(const int* __restrict__ col, long long nnz, int* __restrict__ cnt) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[k]], 1);
}

// exclusive scan of cnt[0..len) into out[0..len] (out[len] = total), three
// phases: per-block scans of 1024 elements, a one-block scan of the block
// totals, the offsets added back
__global__ void __launch_bounds__(1024) k_scan_blocks(const int* __restrict__ in, int len, int* __restrict__ out,
                                                      int* __restrict__ sums) {
  __shared__ int sh[1024];
  const int i = blockIdx.x * 1024 + threadIdx.x;
  const int v = i < len ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < len) out[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == 1023) sums[blockIdx.x] = sh[1023];
}

__global__ void __launch_bounds__(1024) k_scan_sums(int* __restrict__ sums, int nb, int* __restrict__ total) {
  __shared__ int sh[1024];
  int carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? sums[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) sums[i] = carry + sh[threadIdx.x] - v;
    const int blk_total = sh[1023];
    __syncthreads();
    carry += blk_total;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int* __restrict__ out, int len, const int* __restrict__ sums, const int* __restrict__ total) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) out[i] += sums[i / 1024];
  if (blockIdx.x == 0 && threadIdx.x == 0) out[len] = *total;
}

// scatter A's entries into the column segments of A' (per nonzero, its row by
// binary search; order within a segment decided by the atomics, sorted after)
__global__ void k_col_scatter(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
                              int rows, long long nnz, const int* __restrict__ trp, int* __restrict__ cur,
                              int* __restrict__ tcol, double* __restrict__ tval) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
    const int c = col[k];
    const int p = trp[c] + atomicAdd(&cur[c], 1);
    tcol[p] = row_of(rp, rows, k);
    tval[p] = val[k];
  }
}

// sort each segment of A' by row (insertion sort; segments longer than
// SEG_MAX are flagged and the problem is built on the host instead)
constexpr int SEG_MAX = 4096;
__global__ void k_seg_sort(const int* __restrict__ trp, int segs, int* __restrict__ tcol, double* __restrict__ tval,
                           unsigned* __restrict__ err) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < segs; j += gridDim.x * blockDim.x) {
    const int a = trp[j], b = trp[j + 1];
    if (b - a > SEG_MAX) { atomicOr(err, VE_LONG); continue; }
    for (int k = a + 1; k < b; ++k) {
      const int key = tcol[k];
      const double v = tval[k];
      int q = k - 1;
      while (q >= a && tcol[q] > key) {
        tcol[q + 1] = tcol[q];
        tval[q + 1] = tval[q];
        --q;
      }
      tcol[q + 1] = key;
      tval[q + 1] = v;
    }
  }
}

__global__ void k_row_len(const int* __restrict__ qrp, const int* __restrict__ trp, int n, int* __restrict__ len) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    len[j] = (qrp[j + 1] - qrp[j]) + (trp[j + 1] - trp[j]);
}

// row j of P: Q's row (columns j'), then -A' row (columns n + i)
__global__ void k_assemble_P(const int* __restrict__ qrp, const int* __restrict__ qcol, const double* __restrict__ qval,
                             const int* __restrict__ trp, const int* __restrict__ tcol, const double* __restrict__ tval,
                             int n, const int* __restrict__ prp, int* __restrict__ pcol, double* __restrict__ pval,
                             int* __restrict__ split) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < n; j += nw) {
    const int p0 = prp[j], q0 = qrp[j], ql = qrp[j + 1] - q0, t0 = trp[j], tl = trp[j + 1] - t0;
    for (int k = lane; k < ql; k += 32) {
      pcol[p0 + k] = qcol[q0 + k];
      pval[p0 + k] = qval[q0 + k];
    }
    for (int k = lane; k < tl; k += 32) {
      pcol[p0 + ql + k] = n + tcol[t0 + k];
      pval[p0 + ql + k] = -tval[t0 + k];
    }
    if (lane == 0) split[j] = p0 + ql;
  }
}

__global__ void k_block_meta(const int* __restrict__ blk, int nblk, const int* __restrict__ rp, int* __restrict__ meta) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
    const int r0 = blk[b], r1 = blk[b + 1];
    meta[4 * b + 0] = r0;
    meta[4 * b + 1] = r1;
    meta[4 * b + 2] = rp[r0];
    meta[4 * b + 3] = rp[r1];
  }
}

// The instance of every variable and row -- the last instance whose first
// variable (ioff) or first row (joff) is at or before it; instances without
// rows repeat a joff entry and are passed over -- and the inequality flags.
__global__ void k_batch_rows(const int* __restrict__ ioff, const int* __restrict__ joff, const int* __restrict__ meq,
                             int count, int N, int M, int* __restrict__ rinst_n, int* __restrict__ rinst_m,
                             unsigned char* __restrict__ ineq) {
  const long long total = (long long)N + M;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const bool var = i < N;
    const int r = var ? (int)i : (int)(i - N);
    const int* __restrict__ off = var ? ioff : joff;
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= r) lo = mid; else hi = mid - 1;
    }
    if (var) {
      rinst_n[r] = lo;
    } else {
      rinst_m[r] = lo;
      ineq[r] = r - off[lo] >= meq[lo] ? 1 : 0;
    }
  }
}

// device copy of a caller array (or the array itself when it is on the device)
template <typename T>
const T* on_device(pdqp_problem* h, const T* p, size_t count, int mem, std::vector<void*>& tmp, cudaStream_t s) {
  if (mem == PDQP_MEM_DEVICE || count == 0) return p;
  T* d = (T*)pool_alloc(count * sizeof(T), s);
  tmp.push_back(d);
  CK(cudaMemcpyAsync(d, p, count * sizeof(T), cudaMemcpyHostToDevice, s));
  return d;
}

// build temporaries, freed in stream order after the kernels that use them
struct TmpFree {
  std::vector<void*> v;
  cudaStream_t s = nullptr;
  ~TmpFree() {
    for (void* p : v) cudaFreeAsync(p, s);
  }
};

// Grid for `total` items, capped at 8192 blocks: every kernel launched with it
// loops over its items with the grid's stride.
int grid_of(long long total, int threads = 256) {
  return (int)std::max<long long>(1, std::min<long long>((total + threads - 1) / threads, 8192));
}

// exclusive scan on the device: out[0..len] from in[0..len)
void device_scan(const int* in, int len, int* out, std::vector<void*>& tmp, cudaStream_t s) {
  const int nb = std::max(1, (len + 1023) / 1024);
  int* sums = (int*)pool_alloc((size_t)nb * sizeof(int), s);
  tmp.push_back(sums);
  int* total = (int*)pool_alloc(sizeof(int), s);
  tmp.push_back(total);
  k_scan_blocks<<<nb, 1024, 0, s>>>(in, len, out, sums);
  k_scan_sums<<<1, 1024, 0, s>>>(sums, nb, total);
  k_scan_add<<<grid_of(std::max(len, 1)), 256, 0, s>>>(out, len, sums, total);
  CK(cudaGetLastError());
}

// A batch handed over as one block-diagonal problem: instance i owns the
// variables [xoff_i, xoff_i + n_i) and the rows [yoff_i, yoff_i + m_i), in
// order; Q (N rows) and A (M rows) are CSR over the whole stack with global
// column indices, and c, l, u (N) and b (M) are the instances' vectors
// concatenated.  A single problem is the case count = 1.
struct PackedIn {
  int count = 0;
  const int64_t *n = nullptr, *m = nullptr, *m_eq = nullptr;
  const int32_t *Q_rowptr = nullptr, *Q_col = nullptr;
  const double* Q_val = nullptr;
  const int32_t *A_rowptr = nullptr, *A_col = nullptr;
  const double* A_val = nullptr;
  const double *c = nullptr, *b = nullptr, *l = nullptr, *u = nullptr;
};

// The instances of a packed batch as the host path takes them: pointers into
// the packed arrays, with row pointers and columns rebased to the instance.
std::vector<InstanceIn> unpack_instances(const PackedIn& in, const std::vector<int64_t>& xoff,
                                         const std::vector<int64_t>& yoff, const std::vector<int32_t>& qrp,
                                         const std::vector<int32_t>& arp) {
  std::vector<InstanceIn> ins(in.count);
  for (int i = 0; i < in.count; ++i) {
    const int64_t q0 = qrp[xoff[i]], a0 = arp[yoff[i]];
    InstanceIn& t = ins[i];
    t.n = in.n[i];
    t.m = in.m[i];
    t.m_eq = in.m_eq[i];
    t.Q_rowptr = in.Q_rowptr + xoff[i];
    t.Q_col = in.Q_col ? in.Q_col + q0 : nullptr;
    t.Q_val = in.Q_val ? in.Q_val + q0 : nullptr;
    t.A_rowptr = in.A_rowptr ? in.A_rowptr + yoff[i] : nullptr;
    t.A_col = in.A_col ? in.A_col + a0 : nullptr;
    t.A_val = in.A_val ? in.A_val + a0 : nullptr;
    t.c = in.c + xoff[i];
    t.b = in.b ? in.b + yoff[i] : nullptr;
    t.l = in.l + xoff[i];
    t.u = in.u + xoff[i];
    t.rebase = true;
    t.col_base = xoff[i];
  }
  return ins;
}

// Build on the device: the packed input is copied as given and validated
// there, A is transposed by a column count, scan, scatter and a per-column
// sort by row (the same A' as the stable counting sort of the host path), and
// P = [Q | -A'] is assembled row by row.  Only the greedy row blocks are formed
// on the host, per instance, from the row pointers, so the handle is the one
// build_problem makes from the same instances.  Returns nullptr, with the
// instances for the host path in *fallback, when a column of A is longer than
// SEG_MAX; throws Fail on invalid input.
pdqp_problem* build_device(const PackedIn& in, int mem, cudaStream_t s, std::vector<InstanceIn>* fallback) {
  if (mem != PDQP_MEM_HOST && mem != PDQP_MEM_DEVICE) throw Fail{PDQP_ERR_INVALID, "mem_space"};
  const int count = in.count;
  if (count < 1 || !in.n || !in.m || !in.m_eq) throw Fail{PDQP_ERR_INVALID, "null argument or count < 1"};
  std::vector<int64_t> xoff((size_t)count + 1, 0), yoff((size_t)count + 1, 0);
  for (int i = 0; i < count; ++i) {
    if (in.n[i] < 1 || in.m[i] < 0 || in.m_eq[i] < 0 || in.m_eq[i] > in.m[i])
      throw Fail{PDQP_ERR_INVALID, "sizes: need n >= 1, 0 <= m_eq <= m"};
    if (in.n[i] > (1LL << 30) || in.m[i] > (1LL << 30)) throw Fail{PDQP_ERR_INVALID, "total n or m exceeds 2^30"};
    xoff[i + 1] = xoff[i] + in.n[i];
    yoff[i + 1] = yoff[i] + in.m[i];
    if (xoff[i + 1] > (1LL << 30) || yoff[i + 1] > (1LL << 30))
      throw Fail{PDQP_ERR_INVALID, "total n or m exceeds 2^30"};
  }
  const int N = (int)xoff[count], M = (int)yoff[count];
  if (!in.Q_rowptr || !in.c || !in.l || !in.u) throw Fail{PDQP_ERR_INVALID, "null Q_rowptr, c, l or u"};
  if (M > 0 && (!in.A_rowptr || !in.b)) throw Fail{PDQP_ERR_INVALID, "null A_rowptr or b with m > 0"};
  for (auto pr : {(const void*)in.Q_rowptr, (const void*)in.Q_col, (const void*)in.Q_val, (const void*)in.A_rowptr,
                  (const void*)in.A_col, (const void*)in.A_val, (const void*)in.c, (const void*)in.b,
                  (const void*)in.l, (const void*)in.u})
    check_space(pr, mem, "input array");
  // row pointers on the host (the greedy row blocks are formed there)
  std::vector<int32_t> qrp = fetch(in.Q_rowptr, (size_t)N + 1, mem, s);
  std::vector<int32_t> arp = M > 0 ? fetch(in.A_rowptr, (size_t)M + 1, mem, s) : std::vector<int32_t>(1, 0);
  if (qrp[0] != 0) throw Fail{PDQP_ERR_INVALID, "Q: rowptr[0] != 0"};
  if (arp[0] != 0) throw Fail{PDQP_ERR_INVALID, "A: rowptr[0] != 0"};
  const long long nnzQ = qrp[N], nnzA = arp[M];
  if (nnzQ < 0 || (nnzQ > 0 && (!in.Q_col || !in.Q_val))) throw Fail{PDQP_ERR_INVALID, "Q: bad nnz or null arrays"};
  if (nnzA < 0 || (nnzA > 0 && (!in.A_col || !in.A_val))) throw Fail{PDQP_ERR_INVALID, "A: bad nnz or null arrays"};
  if (nnzQ + nnzA > (long long)INT32_MAX - 16) throw Fail{PDQP_ERR_INVALID, "nnz(Q) + nnz(A) exceeds 2^31"};
  TmpFree tmp;
  tmp.s = s;
  const int* dqrp = on_device(nullptr, in.Q_rowptr, (size_t)N + 1, mem, tmp.v, s);
  const int* dqcol = on_device(nullptr, in.Q_col, (size_t)nnzQ, mem, tmp.v, s);
  const double* dqval = on_device(nullptr, in.Q_val, (size_t)nnzQ, mem, tmp.v, s);
  const int* darp = M > 0 ? on_device(nullptr, in.A_rowptr, (size_t)M + 1, mem, tmp.v, s) : nullptr;
  const int* dacol = on_device(nullptr, in.A_col, (size_t)nnzA, mem, tmp.v, s);
  const double* daval = on_device(nullptr, in.A_val, (size_t)nnzA, mem, tmp.v, s);
  unsigned* derr = (unsigned*)pool_alloc(sizeof(unsigned), s);
  tmp.v.push_back(derr);
  CK(cudaMemsetAsync(derr, 0, sizeof(unsigned), s));
  // instance tables: first variable and first row of every instance (then
  // the totals), equality rows per instance
  std::vector<int32_t> itab(3 * (size_t)count + 2);
  for (int i = 0; i <= count; ++i) {
    itab[i] = (int32_t)xoff[i];
    itab[count + 1 + i] = (int32_t)yoff[i];
    if (i < count) itab[2 * (size_t)count + 2 + i] = (int32_t)in.m_eq[i];
  }
  int* ditab = (int*)pool_alloc(itab.size() * sizeof(int), s);
  tmp.v.push_back(ditab);
  to_device(ditab, itab.data(), itab.size(), s);
  const int *dioff = ditab, *djoff = ditab + count + 1, *dmeq = ditab + 2 * (size_t)count + 2;

  pdqp_problem* h = new pdqp_problem();
  h->alloc_stream = s;
  try {
    Work& w = h->w;
    // vectors straight into the handle
    w.c = dalloc<double>(h, N); w.l = dalloc<double>(h, N); w.u = dalloc<double>(h, N); w.b = dalloc<double>(h, M);
    const cudaMemcpyKind kind = mem == PDQP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(w.c, in.c, (size_t)N * sizeof(double), kind, s));
    CK(cudaMemcpyAsync(w.l, in.l, (size_t)N * sizeof(double), kind, s));
    CK(cudaMemcpyAsync(w.u, in.u, (size_t)N * sizeof(double), kind, s));
    if (M > 0) CK(cudaMemcpyAsync(w.b, in.b, (size_t)M * sizeof(double), kind, s));
    w.row_inst_n = dalloc<int>(h, N);
    w.row_inst_m = dalloc<int>(h, M);
    w.row_ineq = dalloc<unsigned char>(h, M);
    k_batch_rows<<<grid_of((long long)N + M), 256, 0, s>>>(dioff, djoff, dmeq, count, N, M, w.row_inst_n,
                                                           w.row_inst_m, w.row_ineq);
    k_validate_rowptr<<<grid_of(N), 256, 0, s>>>(dqrp, N, nnzQ, derr);
    if (M > 0) k_validate_rowptr<<<grid_of(M), 256, 0, s>>>(darp, M, nnzA, derr);
    k_validate_vecs<<<grid_of(std::max(N, M)), 256, 0, s>>>(w.c, w.l, w.u, N, w.b, M, derr);
    CK(cudaGetLastError());
    unsigned herr = 0;
    CK(cudaMemcpyAsync(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (herr & VE_RP) throw Fail{PDQP_ERR_INVALID, "Q or A: rowptr decreases"};
    // the row pointers are sound: check the entries
    if (nnzQ > 0)
      k_validate_entries<<<grid_of(nnzQ), 256, 0, s>>>(dqrp, dqcol, dqval, N, nnzQ, w.row_inst_n, dioff, derr);
    if (nnzA > 0)
      k_validate_entries<<<grid_of(nnzA), 256, 0, s>>>(darp, dacol, daval, M, nnzA, w.row_inst_m, dioff, derr);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (herr & VE_COL) throw Fail{PDQP_ERR_INVALID, "Q or A: column index out of range (of its instance)"};
    if (herr & VE_ORDER) throw Fail{PDQP_ERR_INVALID, "Q or A: column indices not strictly increasing in a row"};
    if (herr & VE_VAL) throw Fail{PDQP_ERR_INVALID, "Q or A: non-finite value"};
    if (herr & VE_C) throw Fail{PDQP_ERR_INVALID, "c: non-finite entry"};
    if (herr & VE_BOUNDS) throw Fail{PDQP_ERR_INVALID, "bounds: need l <= u, l < +inf, u > -inf"};
    if (herr & VE_B) throw Fail{PDQP_ERR_INVALID, "b: non-finite entry"};
    // A' by column count, scan, scatter, per-column sort (A is block-diagonal,
    // so A' is too, with the instances in the same order)
    int* cnt = (int*)pool_alloc((size_t)N * sizeof(int), s); tmp.v.push_back(cnt);
    int* trp = (int*)pool_alloc(((size_t)N + 1) * sizeof(int), s); tmp.v.push_back(trp);
    int* cur = (int*)pool_alloc((size_t)N * sizeof(int), s); tmp.v.push_back(cur);
    int* tcol = (int*)pool_alloc(std::max<size_t>((size_t)nnzA, 1) * sizeof(int), s); tmp.v.push_back(tcol);
    double* tval = (double*)pool_alloc(std::max<size_t>((size_t)nnzA, 1) * sizeof(double), s);
    tmp.v.push_back(tval);
    CK(cudaMemsetAsync(cnt, 0, (size_t)N * sizeof(int), s));
    CK(cudaMemsetAsync(cur, 0, (size_t)N * sizeof(int), s));
    if (nnzA > 0) k_col_count<<<grid_of(nnzA), 256, 0, s>>>(dacol, nnzA, cnt);
    device_scan(cnt, N, trp, tmp.v, s);
    if (nnzA > 0) {
      k_col_scatter<<<grid_of(nnzA), 256, 0, s>>>(darp, dacol, daval, M, nnzA, trp, cur, tcol, tval);
      k_seg_sort<<<grid_of(N), 256, 0, s>>>(trp, N, tcol, tval, derr);
    }
    // P = [Q | -A']
    int* plen = cnt;   // reuse
    k_row_len<<<grid_of(N), 256, 0, s>>>(dqrp, trp, N, plen);
    const long long nnzP = nnzQ + nnzA;
    w.P.rows = N;
    w.P.nnz = nnzP;
    w.P.rp = dalloc<int>(h, (size_t)N + 1 + 8);
    w.P.col = dalloc<int>(h, (size_t)nnzP + 8);
    w.P.val = dalloc<double>(h, (size_t)nnzP + 8);
    w.P.sval = dalloc<double>(h, (size_t)nnzP + 8);
    w.P.split = dalloc<int>(h, N);
    CK(cudaMemsetAsync(w.P.rp, 0, ((size_t)N + 1 + 8) * sizeof(int), s));
    CK(cudaMemsetAsync(w.P.col + nnzP, 0, 8 * sizeof(int), s));
    CK(cudaMemsetAsync(w.P.val + nnzP, 0, 8 * sizeof(double), s));
    CK(cudaMemsetAsync(w.P.sval, 0, ((size_t)nnzP + 8) * sizeof(double), s));
    device_scan(plen, N, w.P.rp, tmp.v, s);
    k_assemble_P<<<grid_of((long long)N * 32), 256, 0, s>>>(dqrp, dqcol, dqval, trp, tcol, tval, N, w.P.rp, w.P.col,
                                                            w.P.val, w.P.split);
    // A as given
    w.A.rows = M;
    w.A.nnz = nnzA;
    w.A.rp = dalloc<int>(h, (size_t)M + 1 + 8);
    w.A.col = dalloc<int>(h, (size_t)nnzA + 8);
    w.A.val = dalloc<double>(h, (size_t)nnzA + 8);
    w.A.sval = dalloc<double>(h, (size_t)nnzA + 8);
    CK(cudaMemsetAsync(w.A.rp, 0, ((size_t)M + 1 + 8) * sizeof(int), s));
    CK(cudaMemsetAsync(w.A.col, 0, ((size_t)nnzA + 8) * sizeof(int), s));
    CK(cudaMemsetAsync(w.A.val, 0, ((size_t)nnzA + 8) * sizeof(double), s));
    CK(cudaMemsetAsync(w.A.sval, 0, ((size_t)nnzA + 8) * sizeof(double), s));
    if (M > 0) {
      CK(cudaMemcpyAsync(w.A.rp, darp, ((size_t)M + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
      if (nnzA > 0) {
        CK(cudaMemcpyAsync(w.A.col, dacol, (size_t)nnzA * sizeof(int), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(w.A.val, daval, (size_t)nnzA * sizeof(double), cudaMemcpyDeviceToDevice, s));
      }
    }
    CK(cudaGetLastError());
    // greedy row blocks on the host from the row pointers
    std::vector<int32_t> prp((size_t)N + 1);
    CK(cudaMemcpyAsync(prp.data(), w.P.rp, ((size_t)N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (herr & VE_LONG) {   // a column of A longer than the device sort handles
      pdqp_destroy(h);
      if (fallback) *fallback = unpack_instances(in, xoff, yoff, qrp, arp);
      return nullptr;
    }
    // each instance's blocks in its own rows, as build_problem forms them
    std::vector<int32_t> pblk{0}, ablk{0}, binst_p, binst_a;
    std::vector<Inst> insts(count);
    for (int i = 0; i < count; ++i) {
      Inst& I = insts[i];
      I.n = (int)in.n[i];
      I.m = (int)in.m[i];
      I.m_eq = (int)in.m_eq[i];
      I.xoff = (int)xoff[i];
      I.yoff = (int)yoff[i];
      I.bP0 = (int)pblk.size() - 1;
      append_row_blocks(xoff[i], xoff[i + 1], prp, pblk);
      I.bP1 = (int)pblk.size() - 1;
      I.bA0 = (int)ablk.size() - 1;
      append_row_blocks(yoff[i], yoff[i + 1], arp, ablk);
      I.bA1 = (int)ablk.size() - 1;
      binst_p.resize(I.bP1, i);
      binst_a.resize(I.bA1, i);
      I.cP0 = i == 0 ? 0 : insts[i - 1].cP0 + kkt_chunks(insts[i - 1].bP0, insts[i - 1].bP1);
      I.cA0 = i == 0 ? 0 : insts[i - 1].cA0 + kkt_chunks(insts[i - 1].bA0, insts[i - 1].bA1);
    }
    begin_work(h, N, M, (int)in.m_eq[0], count, insts);
    for (int side = 0; side < 2; ++side) {
      DCsr& C = side == 0 ? w.P : w.A;
      const std::vector<int32_t>& blk = side == 0 ? pblk : ablk;
      const std::vector<int32_t>& bin = side == 0 ? binst_p : binst_a;
      C.nblk = (int)blk.size() - 1;
      C.blk = dalloc<int>(h, blk.size());
      to_device(C.blk, blk.data(), blk.size(), s);
      C.meta = dalloc<int>(h, 4 * (size_t)std::max(C.nblk, 1));
      int* binst = dalloc<int>(h, (size_t)std::max(C.nblk, 1));
      to_device(binst, bin.data(), bin.size(), s);
      if (C.nblk > 0) k_block_meta<<<grid_of(C.nblk), 256, 0, s>>>(C.blk, C.nblk, C.rp, C.meta);
      (side == 0 ? w.blk_inst_P : w.blk_inst_A) = binst;
      build_long_segments(h, C, side == 0 ? prp : arp, blk, s);
    }
    w.inst = dalloc<Inst>(h, count);
    to_device(w.inst, insts.data(), count, s);
    CK(cudaGetLastError());
    alloc_work(h, s);
  } catch (...) {
    cudaStreamSynchronize(s);
    pdqp_destroy(h);
    throw;
  }
  return h;
}

pdqp_status create_packed(pdqp_handle* out, const PackedIn& in, int mem, cudaStream_t s) {
  if (!out) return PDQP_ERR_INVALID;
  *out = nullptr;
  try {
    std::vector<InstanceIn> fallback;
    pdqp_problem* h = build_device(in, mem, s, &fallback);
    *out = h ? h : build_problem((int)fallback.size(), fallback.data(), mem, s);
    // the pool allocations are stream-ordered: complete them before the handle
    // is used on any other stream
    CK(cudaStreamSynchronize(s));
    return PDQP_OK;
  } catch (const Fail& f) {
    g_create_error = f.msg;
    return f.st;
  } catch (const std::bad_alloc&) {
    g_create_error = "host allocation failed";
    return PDQP_ERR_OOM;
  }
}

pdqp_status create_common(pdqp_handle* out, int count, const InstanceIn* ins, int mem, cudaStream_t s) {
  if (!out) return PDQP_ERR_INVALID;
  *out = nullptr;
  if (count == 1) {   // a single problem is built on the device
    PackedIn p;
    p.count = 1;
    p.n = &ins[0].n;
    p.m = &ins[0].m;
    p.m_eq = &ins[0].m_eq;
    p.Q_rowptr = ins[0].Q_rowptr; p.Q_col = ins[0].Q_col; p.Q_val = ins[0].Q_val;
    p.A_rowptr = ins[0].A_rowptr; p.A_col = ins[0].A_col; p.A_val = ins[0].A_val;
    p.c = ins[0].c; p.b = ins[0].b; p.l = ins[0].l; p.u = ins[0].u;
    return create_packed(out, p, mem, s);
  }
  try {
    *out = build_problem(count, ins, mem, s);
    CK(cudaStreamSynchronize(s));
    return PDQP_OK;
  } catch (const Fail& f) {
    g_create_error = f.msg;
    return f.st;
  } catch (const std::bad_alloc&) {
    g_create_error = "host allocation failed";
    return PDQP_ERR_OOM;
  }
}

}  // namespace

// ==========================================================================
// --------------------------------------------------------------------------
// Solver state for a resume (pdqp_get_state / pdqp_set_state): an opaque blob
// of a fixed header and the device sections below, in this order.  Every
// section is a whole device array, so a resumed solve continues bit for bit
// where the saved one stopped.
// --------------------------------------------------------------------------
namespace {

constexpr char STATE_MAGIC[8] = {'P', 'D', 'Q', 'P', 'S', 'T', 'A', 'T'};
constexpr uint32_t STATE_VERSION = 1;

struct StateHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int64_t n, m, count, r, nnz_P, nnz_A;
  int64_t check_period, pos, k_total;
  int32_t mixed, y_in_z1, fy_in_z1, pad;
  SolveParams params;
  uint64_t total_bytes;
};

// (device pointer, bytes) of each section after the header and the step table
std::vector<std::pair<void*, size_t>> state_sections(Work& w, bool mixed) {
  const size_t n = (size_t)w.n, m = (size_t)w.m, c = (size_t)w.count;
  std::vector<std::pair<void*, size_t>> v = {
      {w.st, c * sizeof(DevState)}, {w.dsc, (n + m) * sizeof(double)},
      {w.x, n * sizeof(double)},    {w.xbar, n * sizeof(double)},       {w.xt, n * sizeof(double)},
      {w.Z[0], (n + m) * sizeof(double)}, {w.Z[1], (n + m) * sizeof(double)},
      {w.ybar, m * sizeof(double)}, {w.ax, n * sizeof(double)},        {w.ay, m * sizeof(double)}};
  if (mixed) {
    const std::pair<void*, size_t> f[] = {
        {w.fx, n * 4},     {w.fxbar, n * 4}, {w.fxt, n * 4}, {w.fZ[0], (n + m) * 4}, {w.fZ[1], (n + m) * 4},
        {w.fybar, m * 4},  {w.fc, n * 4},    {w.fl, n * 4},  {w.fu, n * 4},          {w.fb, m * 4},
        {w.fylo, m * 4},   {w.xhi, n * 8},   {w.yhi, m * 8}, {w.yk, m * 8}};
    v.insert(v.end(), std::begin(f), std::end(f));
  }
  return v;
}

size_t state_bytes(Work& w, bool mixed, int C) {
  size_t b = sizeof(StateHeader) + (size_t)w.count * C * sizeof(StepEntry);
  for (auto& sec : state_sections(w, mixed)) b += sec.second;
  return b;
}

}  // namespace

extern "C" {

void pdqp_default_options(pdqp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = PDQP_PREC_FP64;
  o->step_rule = PDQP_STEP_ADAPTIVE;
  o->restart_rule = PDQP_RESTART_PDQP;
  o->accelerate = 1;
  o->scaling = 1;
  o->ruiz_iters = 10;
  o->l2_scaling = 1;
  o->pock_chambolle = 1;
  o->fixed_K = 64;
  o->check_period = 64;
  o->max_iter = 200000;
  o->eps = 1e-6;
  o->time_limit = 3600.0;
  o->beta_suff = 0.2;
  o->beta_nec = 0.8;
  o->beta_art = 0.36;
  o->pw_theta = 0.2;
  o->eps_zero = 1e-10;
  o->norm_A = 0.0;
  o->norm_Q = 0.0;
  o->norm_iters = 500;
  o->norm_tol = 1e-6;
  o->spmv_threads = 0;
  o->no_graphs = 0;
  o->detect_infeasibility = 0;
  o->eps_infeasible = 1e-8;
  o->maintained_products = 0;
}

const char* pdqp_status_string(int32_t st) {
  switch (st) {
    case PDQP_OK: return "optimal";
    case PDQP_ERR_INVALID: return "invalid input";
    case PDQP_ERR_CUDA: return "CUDA error";
    case PDQP_ERR_OOM: return "out of memory";
    case PDQP_ITER_LIMIT: return "iteration limit";
    case PDQP_TIME_LIMIT: return "time limit";
    case PDQP_NUMERICAL: return "numerical error";
    case PDQP_DEVICE_TIMEOUT: return "device timeout";
    case PDQP_PRIMAL_INFEASIBLE: return "primal infeasible";
    case PDQP_DUAL_INFEASIBLE: return "dual infeasible";
    default: return "unknown status";
  }
}

pdqp_status pdqp_create(pdqp_handle* out, int64_t n, int64_t m, int64_t m_eq, const int32_t* Q_rowptr,
                        const int32_t* Q_col, const double* Q_val, const int32_t* A_rowptr, const int32_t* A_col,
                        const double* A_val, const double* c, const double* b, const double* l, const double* u,
                        int32_t mem, void* stream) {
  InstanceIn in{n, m, m_eq, Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, c, b, l, u};
  return create_common(out, 1, &in, mem, (cudaStream_t)stream);
}

pdqp_status pdqp_create_batch(pdqp_handle* out, int32_t count, const int64_t* n, const int64_t* m,
                              const int64_t* m_eq, const int32_t* const* Q_rowptr, const int32_t* const* Q_col,
                              const double* const* Q_val, const int32_t* const* A_rowptr,
                              const int32_t* const* A_col, const double* const* A_val, const double* const* c,
                              const double* const* b, const double* const* l, const double* const* u, int32_t mem,
                              void* stream) {
  if (!out || count < 1 || !n || !m || !m_eq || !Q_rowptr || !Q_col || !Q_val || !A_rowptr || !A_col || !A_val ||
      !c || !b || !l || !u) {
    if (out) *out = nullptr;
    g_create_error = "null argument or count < 1";
    return PDQP_ERR_INVALID;
  }
  std::vector<InstanceIn> ins(count);
  for (int i = 0; i < count; ++i)
    ins[i] = InstanceIn{n[i], m[i], m_eq[i], Q_rowptr[i], Q_col[i], Q_val[i], A_rowptr[i], A_col[i], A_val[i],
                        c[i], b[i], l[i], u[i]};
  return create_common(out, count, ins.data(), mem, (cudaStream_t)stream);
}

pdqp_status pdqp_create_batch_packed(pdqp_handle* out, int32_t count, const int64_t* n, const int64_t* m,
                                     const int64_t* m_eq, const int32_t* Q_rowptr, const int32_t* Q_col,
                                     const double* Q_val, const int32_t* A_rowptr, const int32_t* A_col,
                                     const double* A_val, const double* c, const double* b, const double* l,
                                     const double* u, int32_t mem, void* stream) {
  PackedIn p;
  p.count = count;
  p.n = n; p.m = m; p.m_eq = m_eq;
  p.Q_rowptr = Q_rowptr; p.Q_col = Q_col; p.Q_val = Q_val;
  p.A_rowptr = A_rowptr; p.A_col = A_col; p.A_val = A_val;
  p.c = c; p.b = b; p.l = l; p.u = u;
  return create_packed(out, p, mem, (cudaStream_t)stream);
}

pdqp_status pdqp_create_family(pdqp_handle* out, int32_t count, int64_t n, int64_t m, int64_t m_eq,
                               const int32_t* Q_rowptr, const int32_t* Q_col, const double* Q_val,
                               const int32_t* A_rowptr, const int32_t* A_col, const double* A_val, const double* C,
                               const double* B, const double* l, const double* u, int32_t mem, void* stream) {
  if (!out) return PDQP_ERR_INVALID;
  *out = nullptr;
  try {
    if (count < 1) throw Fail{PDQP_ERR_INVALID, "count must be >= 1"};
    InstanceIn base{n, m, m_eq, Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, C, B, l, u};
    *out = build_family(base, count, C, B, mem, (cudaStream_t)stream);
    CK(cudaStreamSynchronize((cudaStream_t)stream));   // complete the stream-ordered allocations
    return PDQP_OK;
  } catch (const Fail& f) {
    g_create_error = f.msg;
    return f.st;
  } catch (const std::bad_alloc&) {
    g_create_error = "host allocation failed";
    return PDQP_ERR_OOM;
  }
}

pdqp_status pdqp_set_lowrank_Q(pdqp_handle h, int32_t r, const float* F, int32_t mem, void* stream) {
  if (!h) return PDQP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  Work& w = h->w;
  h->alloc_stream = s;
  try {
    if (r < 1 || r > 256) throw Fail{PDQP_ERR_INVALID, "low-rank: need 1 <= r <= 256"};
    if (!F) throw Fail{PDQP_ERR_INVALID, "low-rank: null F"};
    if (w.count != 1) throw Fail{PDQP_ERR_INVALID, "low-rank: only for single-problem handles"};
    if (w.r != 0) throw Fail{PDQP_ERR_INVALID, "low-rank: already set"};
    check_space(F, mem, "F");
    const size_t N = (size_t)w.n * r;
    std::vector<float> hf = fetch(F, N, mem, s);
    for (float v : hf)
      if (!std::isfinite(v)) throw Fail{PDQP_ERR_INVALID, "low-rank: non-finite entry of F"};
    std::vector<double> hd(hf.begin(), hf.end());
    w.F = dalloc<float>(h, N);
    w.Fo = dalloc<double>(h, N);
    w.Fs = dalloc<float>(h, N);
    w.Fd = dalloc<double>(h, N);
    w.wlr = dalloc<double>(h, 2 * (size_t)r);
    w.wlr_f = dalloc<float>(h, 2 * (size_t)r);
    w.lr_part = dalloc<double>(h, (size_t)((w.n + LR_ROWS - 1) / LR_ROWS) * 2 * r);
    to_device(w.F, hf.data(), N, s);
    to_device(w.Fo, hd.data(), N, s);
    CK(cudaStreamSynchronize(s));
    w.r = r;
    drop_graphs(h);
    return PDQP_OK;
  } catch (const Fail& f) {
    h->err = f.msg;
    return f.st;
  }
}

pdqp_status pdqp_solve(pdqp_handle h, const pdqp_options* opt, const double* x0, const double* y0, double* x_out,
                       double* y_out, pdqp_info* info, int32_t mem, void* stream) {
  if (!h) return PDQP_ERR_INVALID;
  pdqp_options o;
  if (opt) o = *opt; else pdqp_default_options(&o);
  try {
    h->err.clear();
    return solve_impl(h, o, x0, y0, x_out, y_out, info, mem, (cudaStream_t)stream);
  } catch (const Fail& f) {
    h->err = f.msg;
    if (info) { std::memset(info, 0, sizeof(*info)); info->status = f.st; }
    return f.st;
  }
}

pdqp_status pdqp_solve_batch(int32_t count, const pdqp_handle* hs, const pdqp_options* opt,
                             const double* const* x0, const double* const* y0, double* const* x_out,
                             double* const* y_out, pdqp_info* infos, int32_t mem, void* stream) {
  if (count < 0 || (count > 0 && !hs)) return PDQP_ERR_INVALID;
  pdqp_status worst = PDQP_OK;
  for (int32_t i = 0; i < count; ++i) {
    pdqp_status st = pdqp_solve(hs[i], opt, x0 ? x0[i] : nullptr, y0 ? y0[i] : nullptr,
                                x_out ? x_out[i] : nullptr, y_out ? y_out[i] : nullptr,
                                infos ? infos + i : nullptr, mem, stream);
    if (st > worst) worst = st;
  }
  return worst;
}

pdqp_status pdqp_get_iterates(pdqp_handle h, double* x, double* y, double* xbar, double* ybar, int32_t mem,
                           void* stream) {
  if (!h) return PDQP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  Work& w = h->w;
  try {
    for (auto p : {x, y, xbar, ybar}) check_space(p, mem, "state output");
    if (mem == PDQP_MEM_DEVICE) {
      pdqp::write_state(w, x, y, xbar, ybar, s);
    } else {
      double* outs[4] = {x, y, xbar, ybar};
      for (int k = 0; k < 2; ++k) {
        double* hx = outs[2 * k];
        double* hy = outs[2 * k + 1];
        if (!hx && !hy) continue;
        if (k == 0) pdqp::write_state(w, w.stage_n, w.stage_m, nullptr, nullptr, s);
        else pdqp::write_state(w, nullptr, nullptr, w.stage_n, w.stage_m, s);
        if (hx) CK(cudaMemcpyAsync(hx, w.stage_n, w.n * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (hy && w.m) CK(cudaMemcpyAsync(hy, w.stage_m, w.m * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
      }
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return PDQP_OK;
  } catch (const Fail& f) {
    h->err = f.msg;
    return f.st;
  }
}

pdqp_status pdqp_get_state(pdqp_handle h, void* buf, size_t* bytes, void* stream) {
  if (!h || !bytes) return PDQP_ERR_INVALID;
  try {
    h->err.clear();
    if (!h->solved) throw Fail{PDQP_ERR_INVALID, "pdqp_get_state: no solve has run on this handle"};
    if (h->end_mp)
      throw Fail{PDQP_ERR_INVALID, "pdqp_get_state: the last solve maintained its products (no resumable state)"};
    Work& w = h->w;
    const bool mixed = h->end_p.mixed != 0;
    const int C = h->end_p.check_period;
    const size_t need = state_bytes(w, mixed, C);
    if (!buf) { *bytes = need; return PDQP_OK; }
    if (*bytes < need) throw Fail{PDQP_ERR_INVALID, "pdqp_get_state: buffer smaller than the state"};
    cudaStream_t s = (cudaStream_t)stream;
    StateHeader hd{};
    std::memcpy(hd.magic, STATE_MAGIC, 8);
    hd.version = STATE_VERSION;
    hd.header_bytes = sizeof(StateHeader);
    hd.n = w.n; hd.m = w.m; hd.count = w.count; hd.r = w.r; hd.nnz_P = w.P.nnz; hd.nnz_A = w.A.nnz;
    hd.check_period = C; hd.pos = h->end_pos; hd.k_total = h->end_k_total;
    hd.mixed = mixed;
    hd.y_in_z1 = w.y == w.Z[1] + w.n;
    hd.fy_in_z1 = mixed && w.fy == w.fZ[1] + w.n;
    hd.params = h->end_p;
    hd.total_bytes = need;
    unsigned char* out = static_cast<unsigned char*>(buf);
    std::memcpy(out, &hd, sizeof hd);
    size_t off = sizeof hd;
    // the step table, [count][C] out of its [count][tab_stride] layout
    CK(cudaMemcpy2DAsync(out + off, C * sizeof(StepEntry), w.tab, (size_t)w.tab_stride * sizeof(StepEntry),
                         C * sizeof(StepEntry), w.count, cudaMemcpyDeviceToHost, s));
    off += (size_t)w.count * C * sizeof(StepEntry);
    for (auto& sec : state_sections(w, mixed)) {
      if (sec.second) CK(cudaMemcpyAsync(out + off, sec.first, sec.second, cudaMemcpyDeviceToHost, s));
      off += sec.second;
    }
    CK(cudaStreamSynchronize(s));
    *bytes = need;
    return PDQP_OK;
  } catch (const Fail& f) {
    h->err = f.msg;
    return f.st;
  }
}

pdqp_status pdqp_set_state(pdqp_handle h, const void* buf, size_t bytes, void* stream) {
  if (!h || !buf) return PDQP_ERR_INVALID;
  try {
    h->err.clear();
    Work& w = h->w;
    StateHeader hd{};
    if (bytes < sizeof hd) throw Fail{PDQP_ERR_INVALID, "pdqp_set_state: buffer shorter than the state header"};
    std::memcpy(&hd, buf, sizeof hd);
    if (std::memcmp(hd.magic, STATE_MAGIC, 8) != 0 || hd.version != STATE_VERSION ||
        hd.header_bytes != sizeof(StateHeader))
      throw Fail{PDQP_ERR_INVALID, "pdqp_set_state: not a state of this library version"};
    if (hd.n != w.n || hd.m != w.m || hd.count != w.count || hd.r != w.r || hd.nnz_P != w.P.nnz ||
        hd.nnz_A != w.A.nnz)
      throw Fail{PDQP_ERR_INVALID, "pdqp_set_state: the state belongs to a problem of other sizes"};
    const int C = (int)hd.check_period;
    if (C < 2 || C > PDQP_MAX_CHECK || hd.pos < 0 || hd.pos >= C || hd.k_total < 0 || hd.params.check_period != C ||
        hd.params.mixed != hd.mixed)
      throw Fail{PDQP_ERR_INVALID, "pdqp_set_state: inconsistent state header"};
    const bool mixed = hd.mixed != 0;
    cudaStream_t s = (cudaStream_t)stream;
    h->alloc_stream = s;
    if (mixed) alloc_mixed(h);
    const size_t need = state_bytes(w, mixed, C);
    if (bytes < need || hd.total_bytes != need)
      throw Fail{PDQP_ERR_INVALID, "pdqp_set_state: buffer shorter than the state it describes"};
    if (w.tab_stride < C) {
      w.tab = dalloc<StepEntry>(h, (size_t)w.count * C);
      w.tab_stride = C;
      drop_graphs(h);
    }
    const unsigned char* in = static_cast<const unsigned char*>(buf);
    size_t off = sizeof hd;
    CK(cudaMemcpy2DAsync(w.tab, (size_t)w.tab_stride * sizeof(StepEntry), in + off, C * sizeof(StepEntry),
                         C * sizeof(StepEntry), w.count, cudaMemcpyHostToDevice, s));
    off += (size_t)w.count * C * sizeof(StepEntry);
    // instances the iteration limit stopped run on; the others keep their status
    std::vector<DevState> sts((size_t)w.count);
    std::memcpy(sts.data(), in + off, sts.size() * sizeof(DevState));
    int limit_stopped = 0;
    for (DevState& S : sts)
      if (S.status == ST_ITER_LIMIT) { S.status = ST_RUNNING; ++limit_stopped; }
    bool first = true;
    for (auto& sec : state_sections(w, mixed)) {
      const void* src = first ? static_cast<const void*>(sts.data()) : static_cast<const void*>(in + off);
      if (sec.second) CK(cudaMemcpyAsync(sec.first, src, sec.second, cudaMemcpyHostToDevice, s));
      off += sec.second;
      first = false;
    }
    CK(cudaStreamSynchronize(s));   // the host copy of the statuses goes out of scope
    w.y = hd.y_in_z1 ? w.Z[1] + w.n : w.Z[0] + w.n;
    if (mixed) {
      w.fy = hd.fy_in_z1 ? w.fZ[1] + w.n : w.fZ[0] + w.n;
      w.y = w.yk;
    }
    h->resume = true;
    h->resume_p = hd.params;
    h->resume_pos = (int)hd.pos;
    h->resume_k_total = hd.k_total;
    h->resume_recheck = hd.pos == 0 && limit_stopped > 0;
    h->solved = false;
    return PDQP_OK;
  } catch (const Fail& f) {
    h->err = f.msg;
    return f.st;
  }
}

pdqp_status pdqp_kkt(pdqp_handle h, const double* x, const double* y, double* parts, int32_t mem, void* stream) {
  if (!h || !x || !parts || (h->w.m > 0 && !y)) return PDQP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  Work& w = h->w;
  try {
    check_space(x, mem, "x");
    check_space(y, mem, "y");
    const double* dx = x;
    const double* dy = y;
    if (mem == PDQP_MEM_HOST) {
      to_device(w.stage_n, x, w.n, s);
      dx = w.stage_n;
      if (w.m) { to_device(w.stage_m, y, w.m, s); dy = w.stage_m; }
    }
    pdqp::eval_kkt_user(w, dx, dy ? dy : w.stage_m, s);
    CK(cudaGetLastError());
    sync_state(h, s);
    for (int k = 0; k < 6; ++k) parts[k] = w.st_host->out_parts[k];
    return PDQP_OK;
  } catch (const Fail& f) {
    h->err = f.msg;
    return f.st;
  }
}

pdqp_status pdqp_batch_info(pdqp_handle h, pdqp_info* infos, int32_t count) {
  if (!h || !infos || count != h->w.count || (int)h->infos.size() != count) return PDQP_ERR_INVALID;
  for (int i = 0; i < count; ++i) infos[i] = h->infos[i];
  return PDQP_OK;
}

int32_t pdqp_batch_count(pdqp_handle h) { return h ? h->w.count : 0; }

pdqp_status pdqp_get_sizes(pdqp_handle h, int64_t* n, int64_t* m, int64_t* m_eq, int64_t* nnz_Q, int64_t* nnz_A) {
  if (!h) return PDQP_ERR_INVALID;
  if (n) *n = h->w.n;
  if (m) *m = h->w.m;
  if (m_eq) *m_eq = h->w.m_eq;
  if (nnz_Q) *nnz_Q = h->w.P.nnz - h->w.A.nnz;
  if (nnz_A) *nnz_A = h->w.A.nnz;
  return PDQP_OK;
}

const char* pdqp_last_error(pdqp_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void pdqp_destroy(pdqp_handle h) {
  if (!h) return;
  // nothing may still run on the handle's memory (cudaFree used to imply this
  // wait); the blocks then go back to the pool without a device-wide free
  cudaDeviceSynchronize();
  for (void* p : h->allocs) cudaFreeAsync(p, free_stream());
  if (h->w.st_host) cudaFreeHost(h->w.st_host);
  if (h->w.bst_host) cudaFreeHost(h->w.bst_host);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->tune_ev)
    if (e) cudaEventDestroy(e);
  if (h->graph.exec) cudaGraphExecDestroy(h->graph.exec);
  for (auto& c : h->cgraphs)
    if (c.exec) cudaGraphExecDestroy(c.exec);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->tmpl) pdqp_destroy(h->tmpl);
  delete h;
}

int64_t pdqp_launch_count(void) { return pdqp::g_launches.load(std::memory_order_relaxed); }

pdqp_status pdqp_profile_enable(pdqp_handle h, int32_t on) {
  if (!h) return PDQP_ERR_INVALID;
  h->w.prof.reset();
  h->w.prof.on = on != 0;
  return PDQP_OK;
}

pdqp_status pdqp_profile_read(pdqp_handle h, pdqp_profile* out) {
  if (!h || !out) return PDQP_ERR_INVALID;
  std::memset(out, 0, sizeof(*out));
  const Work& w = h->w;
  for (int k = 0; k < 4; ++k) {
    out->launches[k] = w.prof.launches[k];
    out->ms[k] = w.prof.ms[k];
  }
  // algorithmic bytes per launch: the mean of each timed launch's bytes (the
  // instances running at that launch); without timed launches, the whole problem
  const double sv = h->last_precision == PDQP_PREC_MIXED ? 4.0 : 8.0;
  const double n = w.n, m = w.m;
  const double full[2] = {(double)w.A.nnz * (sv + 4.0) + 4.0 * (m + 1) + sv * (n + 5.0 * m),
                          (double)w.P.nnz * (sv + 4.0) + 4.0 * (n + 1) + sv * (10.0 * n + m)};
  for (int k = 0; k < 2; ++k)
    out->bytes[k] = w.prof.launches[k] > 0 ? w.prof.bytes[k] / (double)w.prof.launches[k] : full[k];
  if (w.prof.launches[3] > 0) out->bytes[3] = w.prof.bytes[3] / (double)w.prof.launches[3];
  return PDQP_OK;
}

}  // extern "C"
