// Internal structures shared by the host-side translation units.
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/qtt.h"
#include "common.cuh"

// Kernel classes for the built-in profiler (qtt_ctx_profile*).
enum { PK_GEMM = 0, PK_QR = 1, PK_JACOBI = 2, PK_ELEM = 3, PK_N = 4 };

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
  double flops, bytes;
  int sweep_idx;         // Jacobi: index of the device sweep counter, else -1
  double per_sweep;      // Jacobi: model flops of one sweep
  int64_t shape[4];      // GEMM: M, N, K, batch; QR: m, n, 0, batch; Jacobi: p, q, 0, batch
  int variant;           // GEMM: tile edge (32, 64; 128 = tensor cores) x 100 + split-K; else 0
};

struct qtt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t launches = 0;
  bool prof = false;
  int prof_mode = 0;         // 0 off, 1 every launch, 2 timed iterations of ms_homogenize only
  std::vector<ProfRec> recs;
  int* d_sweeps = nullptr;   // device counters written by profiled Jacobi launches
  int sweeps_cap = 0, sweeps_used = 0;
  bool tc = false;           // route large float contractions to the tensor cores (3 TF32 passes)
  bool tc_sketch = false;    // the sketch contractions of sketched roundings on the tensor cores, 1 pass
  bool in_sketch = false;    // set while those contractions are issued
  int* d_tcerr = nullptr;    // bounded-wait failure flag of the tensor-core GEMM
  int64_t fail_alloc_after = -1;  // test hook: allocations left before dalloc fails (-1: off)
  // profiler totals handed over by contexts that worked for this one (the
  // load-case workers of ms_homogenize), per kernel class
  double ext_ms[PK_N] = {0, 0, 0, 0}, ext_flops[PK_N] = {0, 0, 0, 0}, ext_bytes[PK_N] = {0, 0, 0, 0};
  int64_t ext_launches[PK_N] = {0, 0, 0, 0};
};

// Scoped switch of the single-pass tensor-core route of the sketch contractions.
struct TcSketchScope {
  qtt_ctx* c;
  bool old;
  TcSketchScope(qtt_ctx* ctx, bool on) : c(ctx), old(ctx->tc_sketch) { ctx->tc_sketch = on; }
  ~TcSketchScope() { c->tc_sketch = old; }
};
struct InSketch {
  qtt_ctx* c;
  bool old;
  explicit InSketch(qtt_ctx* ctx) : c(ctx), old(ctx->in_sketch) { ctx->in_sketch = true; }
  ~InSketch() { c->in_sketch = old; }
};

// Scoped switch of the tensor-core route for one ABI call.
struct TcScope {
  qtt_ctx* c;
  bool old;
  TcScope(qtt_ctx* ctx, bool on) : c(ctx), old(ctx->tc) { ctx->tc = on; }
  ~TcScope() { c->tc = old; }
};

inline cudaEvent_t prof_begin(qtt_ctx* c) {
  if (!c->prof) return nullptr;
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, c->stream);
  return e;
}
inline void prof_end(qtt_ctx* c, cudaEvent_t a, int cls, double flops, double bytes, int sweep_idx = -1,
                     double per_sweep = 0.0) {
  if (!c->prof || !a) return;
  cudaEvent_t b;
  cudaEventCreate(&b);
  cudaEventRecord(b, c->stream);
  c->recs.push_back(ProfRec{cls, a, b, flops, bytes, sweep_idx, per_sweep, {0, 0, 0, 0}, 0});
}
// Shape of the launch that the last prof_end(c, a, ...) recorded (a = its start event).
inline void prof_shape(qtt_ctx* c, cudaEvent_t a, int64_t d0, int64_t d1, int64_t d2, int64_t batch,
                       int variant = 0) {
  if (!c->prof || !a || c->recs.empty() || c->recs.back().a != a) return;
  ProfRec& r = c->recs.back();
  r.shape[0] = d0;
  r.shape[1] = d1;
  r.shape[2] = d2;
  r.shape[3] = batch;
  r.variant = variant;
}
inline int* prof_sweep_slot(qtt_ctx* c, int* idx) {
  *idx = -1;
  if (!c->prof || !c->d_sweeps || c->sweeps_used >= c->sweeps_cap) return nullptr;
  *idx = c->sweeps_used++;
  return c->d_sweeps + *idx;
}

struct qtt_tt {
  qtt_ctx* ctx = nullptr;
  int d = 0;
  std::vector<int> n, r;          // modes (d), ranks (d + 1)
  qtt_dtype dtype = QTT_C128;
  void* data = nullptr;           // one allocation holding every core
  std::vector<size_t> off;        // byte offset of each core
  size_t bytes = 0;
};

struct qtt_mpo {
  qtt_ctx* ctx = nullptr;
  int d = 0;
  std::vector<int> no, ni, g;     // output modes, input modes, bond ranks (d + 1)
  std::vector<char> diag;         // per core: zero unless in == out index (a diagonal
                                  // operator core; the contractions then skip the zeros)
  qtt_dtype dtype = QTT_C128;
  void* data = nullptr;
  std::vector<size_t> off;
  size_t bytes = 0;
};

size_t dtype_size(qtt_dtype t);
int dalloc(qtt_ctx* c, void** p, size_t bytes);
void dfree(qtt_ctx* c, void* p);
int sync_read(qtt_ctx* c, void* host, const void* dev, size_t bytes);
qtt_tt* tt_alloc(qtt_ctx* c, int d, const std::vector<int>& n, const std::vector<int>& r, qtt_dtype dt, int* st);
void tt_free(qtt_tt* x);
qtt_mpo* mpo_alloc(qtt_ctx* c, int d, const std::vector<int>& no, const std::vector<int>& ni,
                   const std::vector<int>& g, qtt_dtype dt, int* st);
void mpo_free(qtt_mpo* A);

template <class R>
int round_det(qtt_ctx* c, const qtt_tt* x, double eps, int max_rank, const int* forced, qtt_round_info* info,
              qtt_tt** yout, bool left_orth = false, bool polar = false);
template <class R>
int round_det_batch(qtt_ctx* c, int B, const qtt_tt* const* xs, double eps, int max_rank, qtt_round_info* infos,
                    qtt_tt** ys);
template <class R>
int round_sketched(qtt_ctx* c, int T, const qtt_complex* coef, const qtt_mpo* const* ops, const qtt_tt* const* xs,
                   const qtt_tt* S, double eps, int max_rank, qtt_round_info* info, qtt_tt** yout);
// <y, s> for s = sum_t coef_t A_t x_t (A_t may be NULL), without forming s
template <class R>
int structured_dot(qtt_ctx* c, int T, const qtt_complex* coef, const qtt_mpo* const* ops, const qtt_tt* const* xs,
                   const qtt_tt* y, double out[2]);
template <class R>
int tt_svd_dev(qtt_ctx* c, int d, const std::vector<int>& modes, const cplx<R>* dense, double eps, int max_rank,
               qtt_dtype dt, qtt_tt** out);
template <class R>
int dot_dev(qtt_ctx* c, const qtt_tt* x, const qtt_tt* y, double out[2]);
template <class R>
int norm_dev(qtt_ctx* c, const qtt_tt* x, double* out);

// RAII device buffer on the context stream
struct DBuf {
  qtt_ctx* c = nullptr;
  void* p = nullptr;
  DBuf() {}
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : c(o.c), p(o.p) { o.p = nullptr; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      dfree(c, p);
      c = o.c;
      p = o.p;
      o.p = nullptr;
    }
    return *this;
  }
  ~DBuf() { dfree(c, p); }
  int alloc(qtt_ctx* ctx, size_t bytes) {
    dfree(c, p);
    c = ctx;
    return dalloc(ctx, &p, bytes);
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// C = alpha op(A) op(B) + beta C for a general multi-index descriptor
template <class R>
int gemm_ab(qtt_ctx* c, const GemmDesc& g, cplx<R> alpha, cplx<R> beta, const cplx<R>* A, const cplx<R>* B,
            cplx<R>* C);

// z = a x + b y (ranks add) and a synchronous host -> device copy (engine.cu)
template <class R>
int add_dev(qtt_ctx* c, cplx<R> a, const qtt_tt* x, cplx<R> b, const qtt_tt* y, qtt_tt** out);
int upload(qtt_ctx* c, void* dst, const void* src, size_t bytes);

// TT-cross (cross.cu): the sweep with an FP64 rounding of the result at eps;
// seeds are extra starting points (site values) for the right index sets
struct CrossOut {
  int half_sweeps = 0;
  int64_t evaluations = 0;
  double rel_change = 0.0;
  int max_rank = 1;
};
int cross_rounded(qtt_ctx* c, const CrossFn& f, const std::vector<int>& modes, double eps, int max_rank, int kick,
                  int max_half_sweeps, uint64_t seed, const std::vector<std::vector<uint8_t>>& seeds, qtt_tt** out,
                  CrossOut* st);
// the voxel of every box (stride 6) or ellipsoid (stride 15) centre as site
// values (position convention)
std::vector<std::vector<uint8_t>> centre_seeds(const SiteMap& m, const double* rows, int nrows, int stride);

// AMEn y ~ A x (amen.cu)
template <class R>
int amen_mv_dev(qtt_ctx* c, const qtt_mpo* A, const qtt_tt* x, const qtt_tt* y0, double eps, int kick,
                int max_sweeps, uint64_t seed, int max_rank, qtt_tt** yout, int* sweeps_out, double* dx_out);

// Left singular vectors (rows x min(rows, cols), row-major, by decreasing
// singular value) and singular values of the row-major rows x cols C
// (leading dimension ld); *nsv = min(rows, cols).
template <class R>
int left_svd(qtt_ctx* c, const cplx<R>* Cm, int64_t rows, int64_t cols, int64_t ld, cplx<R>* U, R* sigma,
             int64_t* nsv);

template <class T>
inline T* core_ptr(const qtt_tt* x, int k) {
  return reinterpret_cast<T*>(static_cast<char*>(x->data) + x->off[k]);
}
template <class T>
inline T* core_ptr(const qtt_mpo* A, int k) {
  return reinterpret_cast<T*>(static_cast<char*>(A->data) + A->off[k]);
}
