// Host side of the library: contexts, train handles, and the tensor-train
// algorithms (rounding, sketched rounding, TT-SVD, inner products) composed
// from the device kernels.  Everything numeric runs in kernels on the
// context's stream; the host only sizes buffers and reads back the ranks that
// the truncations choose.
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <float.h>

#include <algorithm>
#include <numeric>
#include <map>
#include <mutex>
#include <chrono>
#include <new>
#include <vector>

#include "../../include/qtt.h"
#include "common.cuh"
#include "engine.h"
#include "kernels.h"

// ------------------------------------------------------------------ basics

size_t dtype_size(qtt_dtype t) { return t == QTT_C128 ? 16 : 8; }

int dalloc(qtt_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return QTT_OK;
  if (c->fail_alloc_after >= 0) {
    if (c->fail_alloc_after == 0) return QTT_ERR_OOM;  // injected failure (qtt_ctx_fail_alloc_after)
    --c->fail_alloc_after;
  }
  if (cudaMallocAsync(p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return QTT_ERR_OOM;
  }
  return QTT_OK;
}
void dfree(qtt_ctx* c, void* p) {
  if (p) cudaFreeAsync(p, c->stream);
}

int sync_read(qtt_ctx* c, void* host, const void* dev, size_t bytes) {
  if (cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return QTT_ERR_CUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return QTT_ERR_CUDA;
  return QTT_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

qtt_tt* tt_alloc(qtt_ctx* c, int d, const std::vector<int>& n, const std::vector<int>& r, qtt_dtype dt, int* st) {
  qtt_tt* x = new (std::nothrow) qtt_tt();
  if (!x) {
    *st = QTT_ERR_OOM;
    return nullptr;
  }
  x->ctx = c;
  x->d = d;
  x->n = n;
  x->r = r;
  x->dtype = dt;
  x->off.resize(d);
  size_t tot = 0;
  for (int k = 0; k < d; ++k) {
    x->off[k] = tot;
    tot += align256((size_t)r[k] * n[k] * r[k + 1] * dtype_size(dt));
  }
  x->bytes = tot;
  *st = dalloc(c, &x->data, tot ? tot : 256);
  if (*st) {
    delete x;
    return nullptr;
  }
  return x;
}

void tt_free(qtt_tt* x) {
  if (!x) return;
  dfree(x->ctx, x->data);
  delete x;
}

qtt_mpo* mpo_alloc(qtt_ctx* c, int d, const std::vector<int>& no, const std::vector<int>& ni,
                   const std::vector<int>& g, qtt_dtype dt, int* st) {
  qtt_mpo* A = new (std::nothrow) qtt_mpo();
  if (!A) {
    *st = QTT_ERR_OOM;
    return nullptr;
  }
  A->ctx = c;
  A->d = d;
  A->no = no;
  A->ni = ni;
  A->g = g;
  A->diag.assign(d, 0);
  A->dtype = dt;
  A->off.resize(d);
  size_t tot = 0;
  for (int k = 0; k < d; ++k) {
    A->off[k] = tot;
    tot += align256((size_t)g[k] * no[k] * ni[k] * g[k + 1] * dtype_size(dt));
  }
  A->bytes = tot;
  *st = dalloc(c, &A->data, tot ? tot : 256);
  if (*st) {
    delete A;
    return nullptr;
  }
  return A;
}

void mpo_free(qtt_mpo* A) {
  if (!A) return;
  dfree(A->ctx, A->data);
  delete A;
}

static inline MIdx L1(int64_t n, int64_t s) { return MIdx{n, 1, s, 0}; }
static inline MIdx L2(int64_t n1, int64_t s1, int64_t n2, int64_t s2) { return MIdx{n1, n2, s1, s2}; }
static inline MIdx B0() { return MIdx{1, 1, 0, 0}; }

// Tensor-core route for one float contraction (batch handled by a loop);
// returns QTT_ERR_UNSUPPORTED when the contraction is too small to pay for
// the packing, so that the caller falls back to the CUDA-core kernel.
// A batch whose A (or B) operand is the same for every entry (batch stride 0)
// is one GEMM with the batch folded into N (or M) as the outer part of a
// two-level index: C[:, (b, n)] = A B[:, (b, n)].
static GemmDesc fold_shared_batch(const GemmDesc& g) {
  GemmDesc f = g;
  if (g.batch <= 1 || g.bA.n2 != 1 || g.bB.n2 != 1 || g.bC.n2 != 1) return f;
  if (g.bA.s1 == 0 && g.nB.n2 == 1 && g.nC.n2 == 1) {
    f.nB = MIdx{g.batch, g.N, g.bB.s1, g.nB.s1};
    f.nC = MIdx{g.batch, g.N, g.bC.s1, g.nC.s1};
    f.N = g.batch * g.N;
  } else if (g.bB.s1 == 0 && g.mA.n2 == 1 && g.mC.n2 == 1) {
    f.mA = MIdx{g.batch, g.M, g.bA.s1, g.mA.s1};
    f.mC = MIdx{g.batch, g.M, g.bC.s1, g.mC.s1};
    f.M = g.batch * g.M;
  } else {
    return f;
  }
  f.batch = 1;
  f.bA = f.bB = f.bC = MIdx{1, 1, 0, 0};
  return f;
}

static int tc_route(qtt_ctx* c, const GemmDesc& g0, cc alpha, cc beta, const cc* A, const cc* B, cc* C) {
  const bool sketch = c->tc_sketch && c->in_sketch;
  if (!c->tc && !sketch) return QTT_ERR_UNSUPPORTED;
  const GemmDesc g = fold_shared_batch(g0);
  if (g.M < 64 || g.N < 16 || g.K < 32 || (double)g.M * g.N * g.K * g.batch < 2.0e5) return QTT_ERR_UNSUPPORTED;
  if (!c->d_tcerr) {
    if (cudaMalloc(&c->d_tcerr, sizeof(int)) != cudaSuccess) return QTT_ERR_OOM;
    cudaMemsetAsync(c->d_tcerr, 0, sizeof(int), c->stream);
  }
  // three passes in both routes: a single TF32 pass in the sketch
  // contractions leaves errors outside the range the sketch should capture
  // (measured: the 16^3 sphere's iterates then settle at 1e-4, not 2e-5)
  const int passes = 3;
  // batched in one launch per chunk of entries (the packed operands of a
  // chunk stay within about 1 GiB)
  const size_t per = qtt_tc_gemm_workspace_ex(g.M, g.N, g.K, 1, passes);
  int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(g.batch, ((int64_t)1 << 30) / (int64_t)per));
  // a chunk starts at a multiple of every two-level batch index's inner
  // size, so that the offsets of its entries are those of a batch from 0
  const int64_t inner = std::lcm(std::lcm(std::max<int64_t>(1, g.bA.n2), std::max<int64_t>(1, g.bB.n2)),
                                 std::max<int64_t>(1, g.bC.n2));
  chunk = std::min<int64_t>(chunk, 65535 / inner * inner);   // grid z limit
  if (chunk < g.batch) chunk = std::max<int64_t>(inner, chunk / inner * inner);
  void* ws = nullptr;
  if (dalloc(c, &ws, qtt_tc_gemm_workspace_ex(g.M, g.N, g.K, chunk, passes))) return QTT_ERR_OOM;
  int st = QTT_OK;
  for (int64_t b0 = 0; b0 < g.batch && !st; b0 += chunk) {
    GemmDesc part = g;
    part.batch = std::min<int64_t>(chunk, g.batch - b0);
    c->launches += 4;
    cudaEvent_t ev = prof_begin(c);
    st = qtt_tc_gemm_ex(part, alpha, beta, A + midx_off(g.bA, b0), B + midx_off(g.bB, b0), C + midx_off(g.bC, b0),
                        ws, c->d_tcerr, c->stream, passes);
    prof_end(c, ev, PK_GEMM, 8.0 * g.M * g.N * g.K * part.batch,
             (double)(g.M * g.K + g.K * g.N + g.M * g.N) * part.batch * sizeof(cc));
    prof_shape(c, ev, g.M, g.N, g.K, part.batch, 128 * 100 + passes);
  }
  dfree(c, ws);
  return st;
}

// ------------------------------------------------------ GEMM tile autotuner
// The first CUDA-core GEMM of a shape (element size, M, N, K, batch and which
// operand indices are contiguous) with enough work times the two tile edges
// (32, 64) once, at the split count the rule gives the shape, with CUDA
// events on the caller's stream into a scratch output, and caches the
// faster; later GEMMs of the shape use it.  The choice only changes speed:
// both edges give the same result bit for bit, so results are reproducible
// across contexts, threads and processes.  GEMMs that accumulate into C
// (beta != 0) or are too small to matter keep the rule's choice.
struct TuneKey {
  int64_t v[7];
  bool operator<(const TuneKey& o) const { return std::lexicographical_compare(v, v + 7, o.v, o.v + 7); }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tune;  // -> (tile, splits)

static bool unit_inner(const MIdx& m) { return (m.n2 == 1 ? m.s1 : m.s2) == 1; }

template <class R>
static int tune_gemm(qtt_ctx* c, const GemmDesc& g, const cplx<R>* A, const cplx<R>* B, int* tile, int* splits) {
  GemmDesc d = g;  // dense scratch output
  d.bC = MIdx{g.batch, 1, g.M * g.N, 0};
  d.mC = MIdx{g.M, 1, g.N, 0};
  d.nC = MIdx{g.N, 1, 1, 0};
  // The split count is fixed by the shape (the rule at tile edge 64), only
  // the tile edge is timed: both edges sum every element over K in the same
  // order (K tiles of the same depth, then the fixed-order split reduction),
  // so whichever edge a process picks, the results are the same bit for bit
  // in every process.
  std::vector<std::pair<int, int>> cand;
  const int s0 = std::min(qtt_gemm_splits_for(g, 64), (int)std::max<int64_t>(1, 65535 / std::max<int64_t>(1, g.batch)));
  for (int t : {32, 64}) cand.emplace_back(t, s0);
  int maxs = 1;
  for (auto& cs : cand) maxs = std::max(maxs, cs.second);
  void* buf = nullptr;
  const size_t outb = (size_t)g.batch * g.M * g.N * sizeof(cplx<R>);
  if (dalloc(c, &buf, outb * (1 + (maxs > 1 ? maxs : 0)))) return QTT_ERR_OOM;
  cplx<R>* Cs = reinterpret_cast<cplx<R>*>(buf);
  cplx<R>* Ps = Cs + (size_t)g.batch * g.M * g.N;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int st = QTT_OK;
  for (auto& cs : cand) {
    float ms = 0.f;
    for (int rep = 0; rep < 2 && st == QTT_OK; ++rep) {  // first run warms up
      cudaEventRecord(e0, c->stream);
      st = qtt_gemm_ex<R>(d, cplx<R>(1, 0), cplx<R>(0, 0), A, B, Cs, cs.second, Ps, c->stream, cs.first);
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = QTT_ERR_CUDA;
      cudaEventElapsedTime(&ms, e0, e1);
    }
    c->launches += 2 * (cs.second > 1 ? 2 : 1);
    if (st == QTT_OK && ms < best) {
      best = ms;
      *tile = cs.first;
      *splits = cs.second;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dfree(c, buf);
  return st;
}

// CUDA-core GEMM: tile edge and split-K from the tuner (or the rule)
template <class R>
static int simt_gemm(qtt_ctx* c, const GemmDesc& g, cplx<R> alpha, cplx<R> beta, const cplx<R>* A, const cplx<R>* B,
                     cplx<R>* C) {
  int tile = 0, splits = qtt_gemm_splits(g);
  const bool beta0 = beta.re == R(0) && beta.im == R(0);
  if (beta0 && (double)g.M * g.N * g.K * g.batch >= 4.0e6) {
    const bool a_kfast = unit_inner(g.kA) && !unit_inner(g.mA);
    const bool b_kfast = unit_inner(g.kB) && !unit_inner(g.nB);
    const TuneKey key{{(int64_t)sizeof(R), g.M, g.N, g.K, g.batch, (int64_t)a_kfast, (int64_t)b_kfast}};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) {
      int t = qtt_gemm_tile_rule(g), sp = splits;
      const int ts = tune_gemm<R>(c, g, A, B, &t, &sp);
      if (ts != QTT_OK) return ts;
      it = g_tune.emplace(key, std::make_pair(t, sp)).first;
    }
    tile = it->second.first;
    splits = it->second.second;
  }
  void* P = nullptr;
  if (splits > 1 && dalloc(c, &P, (size_t)splits * g.batch * g.M * g.N * sizeof(cplx<R>))) return QTT_ERR_OOM;
  c->launches += splits > 1 ? 2 : 1;
  cudaEvent_t ev = prof_begin(c);
  int st = qtt_gemm_ex<R>(g, alpha, beta, A, B, C, splits, reinterpret_cast<cplx<R>*>(P), c->stream, tile);
  prof_end(c, ev, PK_GEMM, 8.0 * g.M * g.N * g.K * g.batch,
           (double)(g.M * g.K + g.K * g.N + g.M * g.N) * g.batch * sizeof(cplx<R>));
  prof_shape(c, ev, g.M, g.N, g.K, g.batch, (tile ? tile : qtt_gemm_tile_rule(g)) * 100 + splits);
  dfree(c, P);
  return st;
}

// C (M x N) = alpha op(A) op(B) + beta C, single batch, general strides
template <class R>
int mm(qtt_ctx* c, int64_t M, int64_t N, int64_t K, const cplx<R>* A, int64_t sAm, int64_t sAk, int conjA,
       const cplx<R>* B, int64_t sBk, int64_t sBn, int conjB, cplx<R>* C, int64_t sCm, int64_t sCn,
       cplx<R> alpha = cplx<R>(1, 0), cplx<R> beta = cplx<R>(0, 0)) {
  GemmDesc g;
  g.bA = B0();
  g.bB = B0();
  g.bC = B0();
  g.mA = L1(M, sAm);
  g.kA = L1(K, sAk);
  g.kB = L1(K, sBk);
  g.nB = L1(N, sBn);
  g.mC = L1(M, sCm);
  g.nC = L1(N, sCn);
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = 1;
  g.conjA = conjA;
  g.conjB = conjB;
  if (K == 0) {
    // C = beta C (only used with beta = 0 here): zero the output
    if (sCn == 1 && sCm == N) return cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(cplx<R>), c->stream) == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
  }
  if (sizeof(R) == 4) {
    int st = tc_route(c, g, cc((float)alpha.re, (float)alpha.im), cc((float)beta.re, (float)beta.im),
                      reinterpret_cast<const cc*>(A), reinterpret_cast<const cc*>(B), reinterpret_cast<cc*>(C));
    if (st != QTT_ERR_UNSUPPORTED) return st;
  }
  return simt_gemm<R>(c, g, alpha, beta, A, B, C);
}

// C = alpha op(A) op(B) + beta C for a general descriptor
template <class R>
int gemm_ab(qtt_ctx* c, const GemmDesc& g, cplx<R> alpha, cplx<R> beta, const cplx<R>* A, const cplx<R>* B,
            cplx<R>* C) {
  if (sizeof(R) == 4) {
    int st = tc_route(c, g, cc((float)alpha.re, (float)alpha.im), cc((float)beta.re, (float)beta.im),
                      reinterpret_cast<const cc*>(A), reinterpret_cast<const cc*>(B), reinterpret_cast<cc*>(C));
    if (st != QTT_ERR_UNSUPPORTED) return st;
  }
  return simt_gemm<R>(c, g, alpha, beta, A, B, C);
}
template int gemm_ab<double>(qtt_ctx*, const GemmDesc&, zc, zc, const zc*, const zc*, zc*);
template int gemm_ab<float>(qtt_ctx*, const GemmDesc&, cc, cc, const cc*, const cc*, cc*);

template <class R>
int gemm(qtt_ctx* c, const GemmDesc& g, const cplx<R>* A, const cplx<R>* B, cplx<R>* C) {
  if (sizeof(R) == 4) {
    int st = tc_route(c, g, cc(1, 0), cc(0, 0), reinterpret_cast<const cc*>(A), reinterpret_cast<const cc*>(B),
                      reinterpret_cast<cc*>(C));
    if (st != QTT_ERR_UNSUPPORTED) return st;
  }
  return simt_gemm<R>(c, g, cplx<R>(1, 0), cplx<R>(0, 0), A, B, C);
}

#define TRY(expr)                 \
  do {                            \
    int _st = (expr);             \
    if (_st != QTT_OK) return _st; \
  } while (0)

static bool dbg_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("QTT_DEBUG_CHECKS");
    v = (e && *e && *e != '0') ? 1 : 0;
  }
  return v == 1;
}

// Debug-only non-finite scan of an intermediate buffer (QTT_DEBUG_CHECKS=1).
template <class R>
static int dbg_finite(qtt_ctx* c, const cplx<R>* p, int64_t count, const char* tag, int k) {
  if (!dbg_enabled() || count <= 0) return QTT_OK;
  void* flag;
  if (dalloc(c, &flag, sizeof(int))) return QTT_ERR_OOM;
  cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
  qtt_isfinite<R>(p, count, reinterpret_cast<int*>(flag), c->stream);
  int h = 0;
  int s = sync_read(c, &h, flag, sizeof(int));
  dfree(c, flag);
  if (s) return s;
  if (h) {
    fprintf(stderr, "qtt-debug: non-finite in %s (core %d, %lld elements)\n", tag, k, (long long)count);
    return QTT_ERR_NAN;
  }
  return QTT_OK;
}

// model flops of a complex Householder QR of an m x n panel (R only, or R and Q)
static double qr_flops(double m, double n, bool with_q) {
  double k = m < n ? m : n;
  double f = 8.0 * (2.0 * m * n * k - (m + n) * k * k + 2.0 * k * k * k / 3.0);
  return with_q ? 2.0 * f : f;
}
// one sweep of one-sided Jacobi on p x q: q(q-1)/2 pairs, each three complex
// dot products of length p and two rotations of p- and q-long column pairs
static double jacobi_sweep_flops(double p, double q) { return 0.5 * q * (q - 1) * (40.0 * p + 24.0 * q); }

template <class R>
static int qr_launch(qtt_ctx* c, const cplx<R>* in, MIdx inB, MIdx rowI, MIdx colI, int conj_in, int64_t m,
                     int64_t n, int64_t rows_total, int64_t rows_per_batch, int64_t batch, cplx<R>* W, cplx<R>* out,
                     int64_t out_bstride, int64_t ldr, cplx<R>* tauws = nullptr, cplx<R>* Qout = nullptr,
                     int64_t q_bstride = 0, int64_t ldq = 0) {
  c->launches++;
  void* qws = nullptr;
  if (Qout) TRY(dalloc(c, &qws, (size_t)batch * m * std::min(m, n) * sizeof(cplx<R>)));
  cudaEvent_t ev = prof_begin(c);
  int st = qtt_qr_r<R>(in, inB, rowI, colI, conj_in, m, n, rows_total, rows_per_batch, batch, W, out, out_bstride,
                       ldr, c->stream, tauws, Qout, q_bstride, ldq, reinterpret_cast<cplx<R>*>(qws));
  dfree(c, qws);
  prof_end(c, ev, PK_QR, batch * qr_flops((double)m, (double)n, Qout != nullptr),
           (double)batch * m * n * sizeof(cplx<R>) * 2.0);
  prof_shape(c, ev, m, n, 0, batch, Qout ? 1 : 0);
  return st;
}

template <class R>
static int jacobi_launch(qtt_ctx* c, cplx<R>* G, cplx<R>* Vwork, R* sigma, cplx<R>* Vsorted, int p, int q,
                         int max_sweeps, cplx<R>* Usorted = nullptr) {
  // Routing.  Without rotations wanted (Vsorted null) and q >= 32: the
  // block-cyclic cluster kernel (columns split over 4 or 8 CTAs, a cluster
  // barrier only per block exchange), in FP32 and FP64 alike.  Otherwise:
  // FP32 matrices too large for one CTA's shared memory go to the row-split
  // cluster kernel; FP64 with q >= 32 and anything with q > 256 to the
  // multi-launch kernel over all SMs (FP64 runs at 2 DFMA/clk/SM on this
  // part); the rest to the single-CTA shared-memory kernel.
  int bs = 0;
  if (!Vsorted && qtt_jacobi_block_plan<R>(p, q, &bs)) {
    int idx;
    int* slot = prof_sweep_slot(c, &idx);
    c->launches++;
    cudaEvent_t ev = prof_begin(c);
    int st = qtt_jacobi_block<R>(G, sigma, Usorted, p, q, max_sweeps, slot, c->stream);
    prof_end(c, ev, PK_JACOBI, 0.0, (double)p * q * sizeof(cplx<R>) * 2.0, idx, jacobi_sweep_flops(p, q));
    prof_shape(c, ev, p, q, 0, 1);
    return st;
  }
  // Vsorted may be null (rotations not wanted): the single-CTA, cluster and
  // multi-launch kernels then skip the rotation updates, the global-memory
  // kernel writes them to scratch space
  const bool cluster = sizeof(R) == 4 && q >= 48 && qtt_jacobi_smem_bytes<R>(p, q) > 200 * 1024 &&
                       qtt_jacobi_cluster_bytes<R>(p, q, q <= 160 ? 4 : 8) <= 200 * 1024;
  const bool wide = !cluster && ((sizeof(R) == 8 && q >= 32) || q > 256);
  const bool smem = !cluster && !wide && qtt_jacobi_smem_bytes<R>(p, q) <= 200 * 1024;
  DBuf vtmp;
  if (!smem && !wide && !cluster && (!Vsorted || !Vwork)) {
    TRY(vtmp.alloc(c, (size_t)2 * q * q * sizeof(cplx<R>)));
    if (!Vsorted) Vsorted = vtmp.as<cplx<R>>();
    if (!Vwork) Vwork = vtmp.as<cplx<R>>() + (size_t)q * q;
  }
  if (cluster) {
    const int nc = q <= 160 ? 4 : 8;
    {
      int idx;
      int* slot = prof_sweep_slot(c, &idx);
      c->launches++;
      cudaEvent_t ev = prof_begin(c);
      int st = qtt_jacobi_cluster<R>(G, sigma, Vsorted, Usorted, p, q, nc, max_sweeps, slot, c->stream);
      prof_end(c, ev, PK_JACOBI, 0.0, (double)(p + 2.0 * q) * q * sizeof(cplx<R>), idx, jacobi_sweep_flops(p, q));
      prof_shape(c, ev, p, q, 0, 1);
      (void)Vwork;
      return st;
    }
  }
  if (smem) {
    int idx;
    int* slot = prof_sweep_slot(c, &idx);
    c->launches++;
    cudaEvent_t ev = prof_begin(c);
    int st = qtt_jacobi_smem<R>(G, Vwork, sigma, Vsorted, Usorted, p, q, max_sweeps, slot, c->stream);
    prof_end(c, ev, PK_JACOBI, 0.0, (double)(p + 2.0 * q) * q * sizeof(cplx<R>), idx, jacobi_sweep_flops(p, q));
    prof_shape(c, ev, p, q, 0, 1);
    return st;
  }
  if (wide) {
    void* buf = nullptr;
    size_t gb = (size_t)p * q * sizeof(cplx<R>), vb = Vsorted ? (size_t)q * q * sizeof(cplx<R>) : 0;
    TRY(dalloc(c, &buf, gb + vb + 256));
    cplx<R>* Gw = reinterpret_cast<cplx<R>*>(buf);
    cplx<R>* Vw = reinterpret_cast<cplx<R>*>(static_cast<char*>(buf) + gb);
    int* flag = reinterpret_cast<int*>(static_cast<char*>(buf) + gb + vb);
    int sweeps = 0;
    cudaEvent_t ev = prof_begin(c);
    int st = qtt_jacobi_wide<R>(G, Gw, Vw, sigma, Vsorted, Usorted, p, q, max_sweeps, flag, &sweeps, &c->launches,
                                c->stream);
    prof_end(c, ev, PK_JACOBI, jacobi_sweep_flops(p, q) * std::max(1, sweeps), (double)(p + 2.0 * q) * q * sizeof(cplx<R>));
    prof_shape(c, ev, p, q, 0, 1);
    dfree(c, buf);
    (void)Vwork;
    return st;
  }
  c->launches++;
  int idx;
  int* slot = prof_sweep_slot(c, &idx);
  cudaEvent_t ev = prof_begin(c);
  int st = qtt_jacobi<R>(G, Vwork, sigma, Vsorted, p, q, 1, max_sweeps, slot, c->stream, Usorted);
  prof_end(c, ev, PK_JACOBI, 0.0, (double)(p + 2.0 * q) * q * sizeof(cplx<R>), idx, jacobi_sweep_flops(p, q));
  prof_shape(c, ev, p, q, 0, 1);
  return st;
}

// ------------------------------------------------------------ TSQR (R only)
// R factor of an m x n matrix whose element (i, c) is in[rowI(i) + colI(c)]
// (conjugated if conj_in): row blocks of max(2n, 256) rows are factored in
// parallel (one CTA each), their R factors stacked and factored again until
// one block remains.  Output: min(m, n) x n, row-major, leading dimension n.
template <class R>
int tsqr_r(qtt_ctx* c, const cplx<R>* in, MIdx rowI, MIdx colI, int conj_in, int64_t m, int64_t n, cplx<R>* Rout,
           int64_t* rows_out) {
  const int64_t chunk = std::max<int64_t>(2 * n, 256);
  if (m <= chunk) {
    DBuf W;
    TRY(W.alloc(c, (size_t)m * n * sizeof(cplx<R>)));
    TRY(qr_launch<R>(c, in, B0(), rowI, colI, conj_in, m, n, m, m, 1, W.as<cplx<R>>(), Rout, 0, n));
    *rows_out = std::min(m, n);
    return QTT_OK;
  }
  const int64_t nch = (m + chunk - 1) / chunk;
  DBuf W, Rs;
  TRY(W.alloc(c, (size_t)nch * chunk * n * sizeof(cplx<R>)));
  TRY(Rs.alloc(c, (size_t)nch * n * n * sizeof(cplx<R>)));
  // batch b reads rows [b*chunk, (b+1)*chunk): the batch stride is chunk rows;
  // at most 65535 batches per launch, so very tall inputs go in slabs
  if (rowI.n2 != 1) return QTT_ERR_UNSUPPORTED;
  MIdx rows = L1(chunk, rowI.s1);
  const int64_t max_batch = 65535;
  for (int64_t b0 = 0; b0 < nch; b0 += max_batch) {
    const int64_t nb = std::min(max_batch, nch - b0), r0 = b0 * chunk;
    TRY(qr_launch<R>(c, in + r0 * rowI.s1, L1(nb, chunk * rowI.s1), rows, colI, conj_in, chunk, n, m - r0, chunk,
                     nb, W.as<cplx<R>>() + b0 * chunk * n, Rs.as<cplx<R>>() + b0 * n * n, n * n, n));
  }
  return tsqr_r<R>(c, Rs.as<cplx<R>>(), L1(nch * n, n), L1(n, 1), 0, nch * n, n, Rout, rows_out);
}

// Left singular vectors and singular values of a (rows x cols) row-major
// matrix C (leading dimension ld): C^H = Q R by TSQR (R only, got x rows,
// got = min(rows, cols)), then one-sided Jacobi on R^H (rows x got), whose
// normalised rotated columns are the left singular vectors of C (no rotation
// accumulation).  U: rows x got, row-major (leading dimension got), columns
// by decreasing singular value; sigma: got values; *nsv = got.
template <class R>
int left_svd(qtt_ctx* c, const cplx<R>* Cm, int64_t rows, int64_t cols, int64_t ld, cplx<R>* U, R* sigma,
             int64_t* nsv) {
  const int64_t p = std::min(rows, cols);
  DBuf Rc, G;
  TRY(Rc.alloc(c, (size_t)std::max<int64_t>(p, 1) * rows * sizeof(cplx<R>)));
  int64_t got = 0;
  // C^H is cols x rows: element (i, j) = conj(C[j, i]) -> row stride 1, column stride ld
  TRY(tsqr_r<R>(c, Cm, L1(cols, 1), L1(rows, ld), 1, cols, rows, Rc.as<cplx<R>>(), &got));
  // G = R^H (rows x got): element (i, j) = conj(R[j, i])
  TRY(G.alloc(c, (size_t)rows * std::max<int64_t>(got, 1) * sizeof(cplx<R>)));
  c->launches++;
  TRY(qtt_copy_strided<R>(Rc.as<cplx<R>>(), L1(rows, 1), L1(got, rows), rows, got, 1, G.as<cplx<R>>(), got,
                          c->stream));
  TRY(jacobi_launch<R>(c, G.as<cplx<R>>(), nullptr, sigma, nullptr, (int)rows, (int)got, 60, U));
  *nsv = got;
  return QTT_OK;
}

// ------------------------------------------------- polar-based truncation
// Compression via polar decomposition (Sec. 2.2) of A (m x q, row-major):
// the polar factor U of A by the Newton-Schulz iteration X <- X (3I - X^H X)/2
// from X0 = A / ||A||_F; H = U^H A (Hermitian part); the sign function S of
// H - dt I by the same iteration on S0 = (H - dt I) / ||.||_F; P+ = (I + S)/2
// and l = round(tr P+); an orthonormal basis C+ of range P+ by two steps of
// subspace iteration from a Gaussian block (Philox, seeded by `stream_id`),
// each orthonormalised by Newton-Schulz; F = U C+ (m x l, orthonormal
// columns).  Only GEMMs and elementwise kernels: under QTT_PREC_TC32 every
// product runs on the tensor cores.  The iteration counts cover the dynamic
// range min(||A|| / dt, 1 / machine epsilon) at a growth of 1.5 per step for
// the smallest scaled values, plus 12 steps to finish (quadratic convergence).
// tail = sqrt(||A||^2 - ||C+^H H||^2), the discarded mass.
template <class R>
static int ns_iterate(qtt_ctx* c, cplx<R>*& X, cplx<R>*& Xn, cplx<R>* G, int64_t m, int64_t q, int iters,
                      bool hermitian) {
  typedef cplx<R> C;
  for (int it = 0; it < iters; ++it) {
    // G = X^H X (or X X for a Hermitian X), Xn = 1.5 X - 0.5 X G
    if (hermitian)
      TRY(mm<R>(c, q, q, q, X, q, 1, 0, X, q, 1, 0, G, q, 1));
    else
      TRY(mm<R>(c, q, q, m, X, 1, q, 1, X, q, 1, 0, G, q, 1));
    if (cudaMemcpyAsync(Xn, X, (size_t)m * q * sizeof(C), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
      return QTT_ERR_CUDA;
    TRY(mm<R>(c, m, q, q, X, q, 1, 0, G, q, 1, 0, Xn, q, 1, C(-0.5, 0), C(1.5, 0)));
    std::swap(X, Xn);
  }
  return QTT_OK;
}

template <class R>
static int polar_truncate_dev(qtt_ctx* c, const cplx<R>* A, int64_t m, int64_t q, double dt, uint64_t stream_id,
                              DBuf* Fout, int64_t* l_out, double* tail_out) {
  typedef cplx<R> C;
  DBuf scal;
  TRY(scal.alloc(c, 64));
  double* ds = scal.as<double>();
  double s2 = 0;
  c->launches++;
  TRY(qtt_sumsq<R>(A, m * q, ds, c->stream));
  TRY(sync_read(c, &s2, ds, sizeof(double)));
  const double an = sqrt(s2);
  const double ueps = sizeof(R) == 8 ? DBL_EPSILON : FLT_EPSILON;
  if (!(an > 0)) {
    // zero centre: any unit vector spans the (empty) kept part
    TRY(Fout->alloc(c, (size_t)m * sizeof(C)));
    if (cudaMemsetAsync(Fout->p, 0, (size_t)m * sizeof(C), c->stream) != cudaSuccess) return QTT_ERR_CUDA;
    const C one(1, 0);
    if (cudaMemcpyAsync(Fout->p, &one, sizeof(C), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return QTT_ERR_CUDA;
    *l_out = 1;
    *tail_out = 0;
    return QTT_OK;
  }
  const double range = std::min(an / std::max(dt, 1e-300), 1.0 / ueps);
  const int iters = std::max(12, std::min(120, (int)ceil(log(std::max(range, 1.0)) / log(1.5)) + 12));
  // polar factor of A
  DBuf Xa, Xb, G;
  TRY(Xa.alloc(c, (size_t)m * q * sizeof(C)));
  TRY(Xb.alloc(c, (size_t)m * q * sizeof(C)));
  TRY(G.alloc(c, (size_t)q * q * sizeof(C)));
  if (cudaMemcpyAsync(Xa.p, A, (size_t)m * q * sizeof(C), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return QTT_ERR_CUDA;
  c->launches++;
  TRY(qtt_scale<R>(Xa.as<C>(), m * q, C((R)(1.0 / an), 0), c->stream));
  C* X = Xa.as<C>();
  C* Xn = Xb.as<C>();
  TRY(ns_iterate<R>(c, X, Xn, G.as<C>(), m, q, iters, false));
  // H = U^H A (Hermitian part) and B = H - dt I, scaled
  DBuf Hr, Hh, Sa, Sb, S2;
  TRY(Hr.alloc(c, (size_t)q * q * sizeof(C)));
  TRY(Hh.alloc(c, (size_t)q * q * sizeof(C)));
  TRY(Sa.alloc(c, (size_t)q * q * sizeof(C)));
  TRY(Sb.alloc(c, (size_t)q * q * sizeof(C)));
  TRY(S2.alloc(c, (size_t)q * q * sizeof(C)));
  TRY(mm<R>(c, q, q, m, X, 1, q, 1, A, q, 1, 0, Hr.as<C>(), q, 1));
  c->launches += 2;
  TRY(qtt_herm_shift<R>(Hr.as<C>(), q, 0.0, Hh.as<C>(), c->stream));
  TRY(qtt_herm_shift<R>(Hr.as<C>(), q, dt, Sa.as<C>(), c->stream));
  double b2 = 0;
  c->launches++;
  TRY(qtt_sumsq<R>(Sa.as<C>(), q * q, ds, c->stream));
  TRY(sync_read(c, &b2, ds, sizeof(double)));
  if (!(b2 > 0)) b2 = 1;
  c->launches++;
  TRY(qtt_scale<R>(Sa.as<C>(), q * q, C((R)(1.0 / sqrt(b2)), 0), c->stream));
  // sign function, P+ = (I + S) / 2, l = round(tr P+)
  C* S = Sa.as<C>();
  C* Sn = Sb.as<C>();
  TRY(ns_iterate<R>(c, S, Sn, S2.as<C>(), q, q, iters, true));
  double tr = 0;
  c->launches++;
  TRY(qtt_half_identity_plus<R>(S, q, ds + 1, c->stream));
  TRY(sync_read(c, &tr, ds + 1, sizeof(double)));
  const int64_t l = std::max<int64_t>(1, std::min<int64_t>(std::min(m, q), (int64_t)llround(tr)));
  // basis of range P+: two subspace-iteration steps, each orthonormalised
  DBuf Om, Ya, Yb, Gl;
  TRY(Om.alloc(c, (size_t)q * l * sizeof(C)));
  TRY(Ya.alloc(c, (size_t)q * l * sizeof(C)));
  TRY(Yb.alloc(c, (size_t)q * l * sizeof(C)));
  TRY(Gl.alloc(c, (size_t)l * l * sizeof(C)));
  c->launches++;
  TRY(qtt_fill_gaussian<R>(Om.as<C>(), q * l, 0x706f6c6172ULL, stream_id, 1.0, c->stream));
  C* Y = Ya.as<C>();
  C* Yn = Yb.as<C>();
  for (int pass = 0; pass < 2; ++pass) {
    TRY(mm<R>(c, q, l, q, S, q, 1, 0, pass == 0 ? Om.as<C>() : Y, l, 1, 0, Yn, l, 1));
    std::swap(Y, Yn);
    double y2 = 0;
    c->launches++;
    TRY(qtt_sumsq<R>(Y, q * l, ds + 2, c->stream));
    TRY(sync_read(c, &y2, ds + 2, sizeof(double)));
    c->launches++;
    TRY(qtt_scale<R>(Y, q * l, C((R)(1.0 / sqrt(std::max(y2, 1e-300))), 0), c->stream));
    // the starting block's condition enters only the first pass; the second starts near orthonormal
    TRY(ns_iterate<R>(c, Y, Yn, Gl.as<C>(), q, l, pass == 0 ? 40 : 16, false));
  }
  // F = U C+, tail from G = C+^H H
  TRY(Fout->alloc(c, (size_t)m * l * sizeof(C)));
  TRY(mm<R>(c, m, l, q, X, q, 1, 0, Y, l, 1, 0, Fout->as<C>(), l, 1));
  DBuf Gm;
  TRY(Gm.alloc(c, (size_t)l * q * sizeof(C)));
  TRY(mm<R>(c, l, q, q, Y, 1, l, 1, Hh.as<C>(), q, 1, 0, Gm.as<C>(), q, 1));
  double g2 = 0;
  c->launches++;
  TRY(qtt_sumsq<R>(Gm.as<C>(), l * q, ds + 3, c->stream));
  TRY(sync_read(c, &g2, ds + 3, sizeof(double)));
  *l_out = l;
  *tail_out = sqrt(std::max(0.0, s2 - g2));
  return QTT_OK;
}

// ------------------------------------------------------- deterministic round
// R-only variant of the QR-then-SVD rounding (Sec. 2.2): the left sweep keeps
// only the triangular factors R_k of R_{k-1} A_k; the right sweep factors
// C_k = R_{k-1} T_k with T_k = A_k (T_{k+1} V_{k+1}), keeps V_k^H as core k and
// never needs the Q factors.  In exact arithmetic this equals keeping Q_k and
// absorbing U_k S_k into it.
//
// left_orth: cores 0..d-2 of x are already left-orthogonal (their (r_k n_k) x
// r_{k+1} unfoldings have orthonormal columns), so every R factor is the
// identity and the left sweep is skipped.
//
// The SVD of C_k is taken by one-sided Jacobi on C_k^H itself (C^H V = W,
// right singular vectors W / |W|): its Gram matrix equals that of the
// triangular factor of a QR of C_k^H, so a QR first would not shorten the
// sweeps; it pays only when C_k is far wider than tall.  The right vectors
// come from the rotated data, not from the accumulated rotations V, whose
// rounding error would leak into the kept subspace (about 10x larger rounding
// error in FP32).
template <class R>
int round_det(qtt_ctx* c, const qtt_tt* x, double eps, int max_rank, const int* forced, qtt_round_info* info,
              qtt_tt** yout, bool left_orth, bool polar) {
  const int d = x->d;
  std::vector<int> n = x->n, r = x->r;
  auto A = [&](int k) { return reinterpret_cast<const cplx<R>*>(static_cast<const char*>(x->data) + x->off[k]); };
  if (d == 1) {
    int st;
    qtt_tt* y = tt_alloc(c, 1, n, r, x->dtype, &st);
    if (!y) return st;
    cudaMemcpyAsync(y->data, x->data, (size_t)n[0] * sizeof(cplx<R>), cudaMemcpyDeviceToDevice, c->stream);
    double s2 = 0;
    DBuf db;
    TRY(db.alloc(c, sizeof(double)));
    c->launches++;
    TRY(qtt_sumsq<R>(A(0), n[0], db.as<double>(), c->stream));
    TRY(sync_read(c, &s2, db.p, sizeof(double)));
    if (info) {
      info->norm = sqrt(s2);
      info->delta = 0;
      info->tail = 0;
      info->err = 0;
      info->capped = 0;
      info->max_rank_out = 1;
    }
    *yout = y;
    return QTT_OK;
  }
  // ---- sweep 1: R factors
  std::vector<DBuf> Rf(d);
  std::vector<int64_t> rp(d + 1, 1);
  if (left_orth)
    for (int k = 0; k < d; ++k) rp[k] = r[k];
  for (int k = 0; k < d - 1 && !left_orth; ++k) {
    const int64_t a0 = r[k], nk = n[k], a1 = r[k + 1];
    DBuf Mb;
    const cplx<R>* M = A(k);
    if (k > 0) {
      TRY(Mb.alloc(c, (size_t)rp[k] * nk * a1 * sizeof(cplx<R>)));
      TRY(mm<R>(c, rp[k], nk * a1, a0, Rf[k - 1].as<cplx<R>>(), a0, 1, 0, A(k), nk * a1, 1, 0, Mb.as<cplx<R>>(),
                nk * a1, 1));
      M = Mb.as<cplx<R>>();
    }
    const int64_t m = rp[k] * nk;
    rp[k + 1] = std::min(m, a1);
    TRY(Rf[k].alloc(c, (size_t)rp[k + 1] * a1 * sizeof(cplx<R>)));
    int64_t got = 0;
    TRY(tsqr_r<R>(c, M, L1(m, a1), L1(a1, 1), 0, m, a1, Rf[k].as<cplx<R>>(), &got));
    TRY(dbg_finite<R>(c, M, m * a1, "round sweep1 M", k));
    TRY(dbg_finite<R>(c, Rf[k].as<cplx<R>>(), rp[k + 1] * a1, "round sweep1 R", k));
  }
  // ---- norm from the orthogonality centre R_{d-2} A_{d-1}
  DBuf scal;
  TRY(scal.alloc(c, 64));
  double* dscal = scal.as<double>();
  int* dint = reinterpret_cast<int*>(dscal + 4);
  {
    const int64_t a0 = r[d - 1], nk = n[d - 1];
    DBuf Cb;
    const cplx<R>* centre = A(d - 1);
    if (!left_orth) {
      TRY(Cb.alloc(c, (size_t)rp[d - 1] * nk * sizeof(cplx<R>)));
      TRY(mm<R>(c, rp[d - 1], nk, a0, Rf[d - 2].as<cplx<R>>(), a0, 1, 0, A(d - 1), nk, 1, 0, Cb.as<cplx<R>>(), nk,
                1));
      centre = Cb.as<cplx<R>>();
    }
    c->launches++;
    TRY(qtt_sumsq<R>(centre, rp[d - 1] * nk, dscal, c->stream));
  }
  double nrm2 = 0;
  TRY(sync_read(c, &nrm2, dscal, sizeof(double)));
  if (!std::isfinite(nrm2)) return QTT_ERR_NAN;  // a non-finite input: nothing to truncate
  const double nrm = sqrt(nrm2);
  const double delta = d > 1 ? eps * nrm / sqrt((double)(d - 1)) : 0.0;
  // ---- sweep 2
  std::vector<DBuf> newc(d);
  std::vector<int> nr(d + 1, 1);
  DBuf Tb;
  const cplx<R>* T = A(d - 1);
  int64_t Trows = r[d - 1];
  double tail2 = 0;
  int capped = 0;
  for (int k = d - 1; k >= 1; --k) {
    const int64_t nk = n[k], tk = nr[k + 1], Tcols = nk * tk;
    const int64_t rk = rp[k];  // rows of R_{k-1}
    const int64_t a0 = r[k];
    DBuf Cb, U, UG, sig, Rc, Qc, Wq, tau, Vw;
    // Jacobi on G = C^H (Tcols x rk, row-major) unless C is so wide that a QR
    // of C^H first pays for itself
    const int64_t jp = Tcols;
    int64_t jq = rk;
    // Jacobi on C^H directly only where one of the fast single-launch
    // kernels takes the (jp x jq) shape (the block-cyclic cluster kernel or
    // the one-CTA shared-memory kernel; FP64 goes to the all-SM kernel
    // anyway); otherwise, e.g. 512 x 256 in FP32, the QR first leaves a
    // jq x jq factor that they do take
    int bsd = 0;
    const bool direct_fast = sizeof(R) == 8 || jq < 32 || qtt_jacobi_block_plan<R>((int)jp, (int)jq, &bsd) != 0 ||
                             qtt_jacobi_smem_bytes<R>((int)jp, (int)jq) <= 200 * 1024;
    if (polar || jp * jq <= 4096 || (jp <= 4 * jq && (jp < jq || direct_fast))) {
      TRY(Cb.alloc(c, (size_t)rk * Tcols * sizeof(cplx<R>)));
      if (left_orth) {
        c->launches++;
        TRY(qtt_copy_strided<R>(T, L1(Tcols, 1), L1(rk, Tcols), Tcols, rk, 1, Cb.as<cplx<R>>(), rk, c->stream));
      } else {
        // element (j, i) = sum_a conj(R[i, a]) conj(T[a, j]), written transposed
        TRY(mm<R>(c, rk, Tcols, a0, Rf[k - 1].as<cplx<R>>(), a0, 1, 1, T, Tcols, 1, 1, Cb.as<cplx<R>>(), 1, rk));
      }
      TRY(dbg_finite<R>(c, Cb.as<cplx<R>>(), rk * Tcols, "round sweep2 G", k));
      // X (Tcols x jq): right singular vectors of C, columns by decreasing singular value
      DBuf X;
      if (polar) {
        // polar-based compression of the centre C^H at dt = delta / q, q its number of singular values
        int64_t l = 0;
        double tl = 0;
        TRY(polar_truncate_dev<R>(c, Cb.as<cplx<R>>(), Tcols, rk, delta / (double)std::min(Tcols, rk),
                                  (uint64_t)k, &X, &l, &tl));
        jq = l;
        nr[k] = (int)l;
        tail2 += tl * tl;
      } else if (Tcols < rk) {
        // C taller than wide (rank <= Tcols): C = Q_c R_c with R_c square
        // (R only), and Jacobi on R_c^H (Tcols x Tcols) gives the same right
        // vectors as normalised rotated columns, in Tcols - 1 rounds a sweep
        // instead of rk - 1
        DBuf Rq, Gq;
        TRY(Rq.alloc(c, (size_t)Tcols * Tcols * sizeof(cplx<R>)));
        int64_t got = 0;
        // Cb holds C^H (Tcols x rk, row-major): C (rk x Tcols) is read through the transposed view, conjugated
        TRY(tsqr_r<R>(c, Cb.as<cplx<R>>(), L1(rk, 1), L1(Tcols, rk), 1, rk, Tcols, Rq.as<cplx<R>>(), &got));
        TRY(Gq.alloc(c, (size_t)Tcols * Tcols * sizeof(cplx<R>)));
        c->launches++;
        // G = R_c^H: element (i, j) = conj(R_c[j, i])
        TRY(qtt_copy_strided<R>(Rq.as<cplx<R>>(), L1(Tcols, 1), L1(Tcols, Tcols), Tcols, Tcols, 1, Gq.as<cplx<R>>(),
                                Tcols, c->stream));
        TRY(X.alloc(c, (size_t)Tcols * Tcols * sizeof(cplx<R>)));
        TRY(sig.alloc(c, (size_t)Tcols * sizeof(R)));
        TRY(jacobi_launch<R>(c, Gq.as<cplx<R>>(), nullptr, sig.as<R>(), nullptr, (int)Tcols, (int)Tcols, 60,
                             X.as<cplx<R>>()));
        jq = Tcols;
      } else {
        TRY(X.alloc(c, (size_t)Tcols * jq * sizeof(cplx<R>)));
        TRY(sig.alloc(c, (size_t)jq * sizeof(R)));
        TRY(jacobi_launch<R>(c, Cb.as<cplx<R>>(), nullptr, sig.as<R>(), nullptr, (int)jp, (int)jq, 60,
                             X.as<cplx<R>>()));
      }
      TRY(dbg_finite<R>(c, X.as<cplx<R>>(), Tcols * jq, "round sweep2 X", k));
      int t;
      if (polar) {
        t = (int)jq;  // the rank polar_truncate_dev found; no cap in this variant
      } else {
        c->launches++;
        if (forced) {
          t = (int)std::min<int64_t>(forced[k], jq);
          TRY(qtt_trunc_rank<R>(sig.as<R>(), (int)jq, -1.0, t, dint, reinterpret_cast<double*>(dint + 2),
                                c->stream));
        } else {
          TRY(qtt_trunc_rank<R>(sig.as<R>(), (int)jq, delta, max_rank, dint, reinterpret_cast<double*>(dint + 2),
                                c->stream));
        }
        int hv[4];
        TRY(sync_read(c, hv, dint, sizeof(hv)));
        double tl;
        memcpy(&tl, hv + 2, sizeof(double));
        t = hv[0];
        if (!forced) capped |= hv[1];
        tail2 += tl * tl;
        nr[k] = t;
      }
      // new core k = X[:, :t]^H (t x Tcols)
      TRY(newc[k].alloc(c, (size_t)t * Tcols * sizeof(cplx<R>)));
      cplx<R>* core = newc[k].as<cplx<R>>();
      c->launches++;
      TRY(qtt_copy_strided<R>(X.as<cplx<R>>(), L1(t, 1), L1(Tcols, jq), t, Tcols, 1, core, Tcols, c->stream));
      // P = T X[:, :t] (a0 x t); T_{k-1} = A_{k-1} P
      DBuf P, Tn;
      TRY(P.alloc(c, (size_t)a0 * t * sizeof(cplx<R>)));
      TRY(mm<R>(c, a0, t, Tcols, T, Tcols, 1, 0, X.as<cplx<R>>(), jq, 1, 0, P.as<cplx<R>>(), t, 1));
      const int64_t pr = (int64_t)r[k - 1] * n[k - 1];
      TRY(Tn.alloc(c, (size_t)pr * t * sizeof(cplx<R>)));
      TRY(mm<R>(c, pr, t, a0, A(k - 1), a0, 1, 0, P.as<cplx<R>>(), t, 1, 0, Tn.as<cplx<R>>(), t, 1));
      Tb = std::move(Tn);
      T = Tb.as<cplx<R>>();
      Trows = r[k - 1];
      continue;
    }
    const cplx<R>* Cm = T;  // R factor is the identity for a left-orthogonal train
    if (!left_orth) {
      TRY(Cb.alloc(c, (size_t)rk * Tcols * sizeof(cplx<R>)));
      TRY(mm<R>(c, rk, Tcols, a0, Rf[k - 1].as<cplx<R>>(), a0, 1, 0, T, Tcols, 1, 0, Cb.as<cplx<R>>(), Tcols, 1));
      Cm = Cb.as<cplx<R>>();
    }
    // SVD of C (rk x Tcols): C^H = Q_c R_c (Householder, explicit Q_c), then
    // one-sided Jacobi R_c V = U_G S.  Left vectors of C: V; right: Q_c U_G.
    const int64_t pq = std::min(rk, Tcols);
    TRY(Rc.alloc(c, (size_t)pq * rk * sizeof(cplx<R>)));
    TRY(Qc.alloc(c, (size_t)Tcols * pq * sizeof(cplx<R>)));
    TRY(Wq.alloc(c, (size_t)Tcols * rk * sizeof(cplx<R>)));
    TRY(tau.alloc(c, (size_t)2 * rk * sizeof(cplx<R>)));
    TRY(qr_launch<R>(c, Cm, B0(), L1(Tcols, 1), L1(rk, Tcols), 1, Tcols, rk, Tcols, Tcols, 1,
                     Wq.as<cplx<R>>(), Rc.as<cplx<R>>(), 0, rk, tau.as<cplx<R>>(), Qc.as<cplx<R>>(), 0, pq));
    TRY(U.alloc(c, (size_t)rk * rk * sizeof(cplx<R>)));
    TRY(UG.alloc(c, (size_t)pq * rk * sizeof(cplx<R>)));
    TRY(Vw.alloc(c, (size_t)rk * rk * sizeof(cplx<R>)));
    TRY(sig.alloc(c, (size_t)rk * sizeof(R)));
    c->launches++;
    TRY(dbg_finite<R>(c, Cm, rk * Tcols, "round sweep2 C", k));
    TRY(dbg_finite<R>(c, Rc.as<cplx<R>>(), pq * rk, "round sweep2 Rc", k));
    TRY(dbg_finite<R>(c, Qc.as<cplx<R>>(), Tcols * pq, "round sweep2 Qc", k));
    TRY(jacobi_launch<R>(c, Rc.as<cplx<R>>(), Vw.as<cplx<R>>(), sig.as<R>(), U.as<cplx<R>>(), (int)pq, (int)rk, 60,
                         UG.as<cplx<R>>()));
    TRY(dbg_finite<R>(c, U.as<cplx<R>>(), rk * rk, "round sweep2 U", k));
    TRY(dbg_finite<R>(c, UG.as<cplx<R>>(), pq * rk, "round sweep2 UG", k));
    int t;
    if (forced) {
      t = (int)std::min<int64_t>(forced[k], rk);
      c->launches++;
      TRY(qtt_trunc_rank<R>(sig.as<R>(), (int)rk, -1.0, t, dint, dscal + 1, c->stream));
      // trunc with delta < 0 keeps everything then caps at t
    } else {
      c->launches++;
      TRY(qtt_trunc_rank<R>(sig.as<R>(), (int)rk, delta, max_rank, dint, dscal + 1, c->stream));
    }
    int hv[2];
    double tl = 0;
    TRY(sync_read(c, hv, dint, sizeof(hv)));
    TRY(sync_read(c, &tl, dscal + 1, sizeof(double)));
    t = hv[0];
    if (!forced) capped |= hv[1];
    tail2 += tl * tl;
    nr[k] = t;
    // new core k = (Q_c U_G[:, :t])^H = U_G[:, :t]^H Q_c^H  (t x Tcols)
    TRY(newc[k].alloc(c, (size_t)t * Tcols * sizeof(cplx<R>)));
    cplx<R>* core = newc[k].as<cplx<R>>();
    TRY(mm<R>(c, t, Tcols, pq, UG.as<cplx<R>>(), 1, rk, 1, Qc.as<cplx<R>>(), 1, pq, 1, core, Tcols, 1));
    TRY(dbg_finite<R>(c, core, t * Tcols, "round sweep2 core", k));
    // P = T core^H (a0 x t); T_{k-1} = A_{k-1} P (r_{k-2} n_{k-1} x t)
    DBuf P, Tn;
    TRY(P.alloc(c, (size_t)a0 * t * sizeof(cplx<R>)));
    TRY(mm<R>(c, a0, t, Tcols, T, Tcols, 1, 0, core, 1, Tcols, 1, P.as<cplx<R>>(), t, 1));
    const int64_t pr = (int64_t)r[k - 1] * n[k - 1];
    TRY(Tn.alloc(c, (size_t)pr * t * sizeof(cplx<R>)));
    TRY(mm<R>(c, pr, t, a0, A(k - 1), a0, 1, 0, P.as<cplx<R>>(), t, 1, 0, Tn.as<cplx<R>>(), t, 1));
    Tb = std::move(Tn);
    T = Tb.as<cplx<R>>();
    Trows = r[k - 1];
  }
  // core 0 = T_0 (1 x n_0 x t_1)
  int st;
  qtt_tt* y = tt_alloc(c, d, n, nr, x->dtype, &st);
  if (!y) return st;
  for (int k = 0; k < d; ++k) {
    const void* src = (k == 0) ? (const void*)T : newc[k].p;
    size_t bytes = (size_t)nr[k] * n[k] * nr[k + 1] * sizeof(cplx<R>);
    if (cudaMemcpyAsync(static_cast<char*>(y->data) + y->off[k], src, bytes, cudaMemcpyDeviceToDevice, c->stream) !=
        cudaSuccess) {
      tt_free(y);
      return QTT_ERR_CUDA;
    }
  }
  (void)Trows;
  if (info) {
    info->norm = nrm;
    info->delta = delta;
    info->tail = sqrt(tail2);
    info->err = -1;
    info->capped = capped;
    info->max_rank_out = *std::max_element(nr.begin(), nr.end());
  }
  *yout = y;
  return QTT_OK;
}

template int round_det<double>(qtt_ctx*, const qtt_tt*, double, int, const int*, qtt_round_info*, qtt_tt**,
                                bool, bool);
template int round_det<float>(qtt_ctx*, const qtt_tt*, double, int, const int*, qtt_round_info*, qtt_tt**,
                               bool, bool);

// ------------------------------------------------ batched deterministic round
// B trains of one shape (same modes and ranks) rounded in lockstep by the
// algorithm of round_det: every step of either sweep is one launch per kernel
// for the whole batch -- batched GEMMs, one QR CTA per train, one Jacobi
// cluster per train -- and the truncation sweep needs one host
// synchronisation per core for all trains.  Each train keeps its own
// truncation: a bond is carried at the largest rank of the batch, the
// singular vectors beyond a train's own rank are zeroed, so that its padded
// rows and columns stay exactly zero, and the outputs are cropped to each
// train's ranks.  QTT_ERR_UNSUPPORTED for shapes it does not take (the
// caller then rounds the trains one by one).
template <class R>
static GemmDesc bgemm(int64_t B, int64_t M, int64_t N, int64_t K, int64_t bA, MIdx mA, MIdx kA, int64_t bB, MIdx kB,
                      MIdx nB, int64_t bC, MIdx mC, MIdx nC, int conjA = 0, int conjB = 0) {
  GemmDesc g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = B;
  g.bA = L1(B, bA);
  g.mA = mA;
  g.kA = kA;
  g.bB = L1(B, bB);
  g.kB = kB;
  g.nB = nB;
  g.bC = L1(B, bC);
  g.mC = mC;
  g.nC = nC;
  g.conjA = conjA;
  g.conjB = conjB;
  return g;
}

template <class R>
int round_det_batch(qtt_ctx* c, int B, const qtt_tt* const* xs, double eps, int max_rank, qtt_round_info* infos,
                    qtt_tt** ys) {
  typedef cplx<R> C;
  const qtt_tt* x0 = xs[0];
  const int d = x0->d;
  for (int b = 1; b < B; ++b)
    if (xs[b]->d != d || xs[b]->n != x0->n || xs[b]->r != x0->r || xs[b]->dtype != x0->dtype) return QTT_ERR_ARG;
  if (d < 2 || B > 65535) return QTT_ERR_UNSUPPORTED;
  const std::vector<int>& n = x0->n;
  const std::vector<int>& r = x0->r;
  // the trains side by side: train b at X + b * xst, core k at offset off[k]
  const int64_t xst = (int64_t)(x0->bytes / sizeof(C));
  DBuf Xall;
  TRY(Xall.alloc(c, (size_t)B * x0->bytes));
  for (int b = 0; b < B; ++b)
    if (cudaMemcpyAsync(Xall.as<char>() + (size_t)b * x0->bytes, xs[b]->data, x0->bytes, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess)
      return QTT_ERR_CUDA;
  auto A = [&](int k) { return Xall.as<C>() + x0->off[k] / sizeof(C); };
  // ---- sweep 1: R factors, B per core
  std::vector<DBuf> Rf(d);
  std::vector<int64_t> rp(d + 1, 1);
  for (int k = 0; k < d - 1; ++k) {
    const int64_t a0 = r[k], nk = n[k], a1 = r[k + 1];
    const C* M = A(k);
    int64_t mst = xst;
    DBuf Mb;
    if (k > 0) {
      TRY(Mb.alloc(c, (size_t)B * rp[k] * nk * a1 * sizeof(C)));
      TRY(gemm<R>(c, bgemm<R>(B, rp[k], nk * a1, a0, rp[k] * a0, L1(rp[k], a0), L1(a0, 1), xst, L1(a0, nk * a1),
                              L1(nk * a1, 1), rp[k] * nk * a1, L1(rp[k], nk * a1), L1(nk * a1, 1)),
                  Rf[k - 1].as<C>(), A(k), Mb.as<C>()));
      M = Mb.as<C>();
      mst = rp[k] * nk * a1;
    }
    const int64_t m = rp[k] * nk;
    rp[k + 1] = std::min(m, a1);
    DBuf W;
    TRY(Rf[k].alloc(c, (size_t)B * rp[k + 1] * a1 * sizeof(C)));
    TRY(W.alloc(c, (size_t)B * m * a1 * sizeof(C)));
    TRY(qr_launch<R>(c, M, L1(B, mst), L1(m, a1), L1(a1, 1), 0, m, a1, m, 0, B, W.as<C>(), Rf[k].as<C>(),
                     rp[k + 1] * a1, a1));
  }
  // ---- norms from the orthogonality centres, thresholds per train
  DBuf scal;
  TRY(scal.alloc(c, (size_t)B * (sizeof(double) + 4 * sizeof(int))));
  double* dnorm = scal.as<double>();
  int* dtr = reinterpret_cast<int*>(dnorm + B);
  std::vector<double> nrm(B), delta(B);
  {
    const int64_t M = rp[d - 1], N = n[d - 1], K = r[d - 1];
    DBuf Cc;
    TRY(Cc.alloc(c, (size_t)B * M * N * sizeof(C)));
    TRY(gemm<R>(c, bgemm<R>(B, M, N, K, M * K, L1(M, K), L1(K, 1), xst, L1(K, N), L1(N, 1), M * N, L1(M, N),
                            L1(N, 1)),
                Rf[d - 2].as<C>(), A(d - 1), Cc.as<C>()));
    for (int b = 0; b < B; ++b) {
      c->launches++;
      TRY(qtt_sumsq<R>(Cc.as<C>() + (size_t)b * M * N, M * N, dnorm + b, c->stream));
    }
    TRY(sync_read(c, nrm.data(), dnorm, (size_t)B * sizeof(double)));
    for (int b = 0; b < B; ++b) {
      nrm[b] = sqrt(nrm[b]);
      delta[b] = eps * nrm[b] / sqrt((double)(d - 1));
    }
    if (cudaMemcpyAsync(dnorm, delta.data(), (size_t)B * sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess)
      return QTT_ERR_CUDA;
  }
  // ---- sweep 2
  std::vector<DBuf> newc(d);
  std::vector<int> tmax(d + 1, 1);
  std::vector<std::vector<int>> tb(B, std::vector<int>(d + 1, 1));
  std::vector<double> tail2(B, 0.0);
  std::vector<int> capped(B, 0);
  std::vector<int> hv((size_t)4 * B);
  DBuf Tb;
  const C* T = A(d - 1);
  int64_t tst = xst;
  for (int k = d - 1; k >= 1; --k) {
    const int64_t nk = n[k], Tcols = nk * tmax[k + 1], rk = rp[k], a0 = r[k];
    if (!(Tcols <= 4 * rk || Tcols * rk <= 4096)) return QTT_ERR_UNSUPPORTED;
    // C_b^H (Tcols x rk) = (R_{k-1,b} T_b)^H, written transposed
    DBuf Cb, Rq, Gq, W2, X, sig;
    TRY(Cb.alloc(c, (size_t)B * rk * Tcols * sizeof(C)));
    TRY(gemm<R>(c, bgemm<R>(B, rk, Tcols, a0, rk * a0, L1(rk, a0), L1(a0, 1), tst, L1(a0, Tcols), L1(Tcols, 1),
                            rk * Tcols, L1(rk, 1), L1(Tcols, rk), 1, 1),
                Rf[k - 1].as<C>(), T, Cb.as<C>()));
    C* G = Cb.as<C>();
    int64_t gq = rk;
    if (Tcols < rk) {
      // C taller than wide: R-only QR of C_b (read conjugated through C_b^H), Jacobi on R_b^H
      TRY(Rq.alloc(c, (size_t)B * Tcols * Tcols * sizeof(C)));
      TRY(W2.alloc(c, (size_t)B * rk * Tcols * sizeof(C)));
      TRY(qr_launch<R>(c, Cb.as<C>(), L1(B, rk * Tcols), L1(rk, 1), L1(Tcols, rk), 1, rk, Tcols, rk, 0, B,
                       W2.as<C>(), Rq.as<C>(), Tcols * Tcols, Tcols));
      TRY(Gq.alloc(c, (size_t)B * Tcols * Tcols * sizeof(C)));
      c->launches++;
      TRY(qtt_copy_batch<R>(Rq.as<C>(), Tcols * Tcols, L1(Tcols, 1), L1(Tcols, Tcols), Tcols, Tcols, 1, Gq.as<C>(),
                            Tcols, Tcols * Tcols, B, c->stream));
      G = Gq.as<C>();
      gq = Tcols;
    }
    const int64_t jq = gq;
    TRY(X.alloc(c, (size_t)B * Tcols * jq * sizeof(C)));
    TRY(sig.alloc(c, (size_t)B * jq * sizeof(R)));
    int bsz = 0;
    if (qtt_jacobi_block_plan<R>((int)Tcols, (int)jq, &bsz)) {
      int idx;
      int* slot = prof_sweep_slot(c, &idx);
      c->launches++;
      cudaEvent_t ev = prof_begin(c);
      TRY(qtt_jacobi_block<R>(G, sig.as<R>(), X.as<C>(), (int)Tcols, (int)jq, 60, slot, c->stream, B));
      prof_end(c, ev, PK_JACOBI, 0.0, (double)B * Tcols * jq * sizeof(C) * 2.0, idx,
               B * jacobi_sweep_flops((double)Tcols, (double)jq));
      prof_shape(c, ev, Tcols, jq, 0, B);
    } else {
      for (int b = 0; b < B; ++b)
        TRY(jacobi_launch<R>(c, G + (size_t)b * Tcols * jq, nullptr, sig.as<R>() + (size_t)b * jq, nullptr,
                             (int)Tcols, (int)jq, 60, X.as<C>() + (size_t)b * Tcols * jq));
    }
    c->launches++;
    TRY(qtt_trunc_rank_batch<R>(sig.as<R>(), (int)jq, dnorm, max_rank, dtr, B, c->stream));
    TRY(sync_read(c, hv.data(), dtr, (size_t)4 * B * sizeof(int)));
    int tm = 1;
    for (int b = 0; b < B; ++b) {
      double tl;
      memcpy(&tl, &hv[(size_t)4 * b + 2], sizeof(double));
      tb[b][k] = hv[(size_t)4 * b];
      capped[b] |= hv[(size_t)4 * b + 1];
      tail2[b] += tl * tl;
      tm = std::max(tm, tb[b][k]);
    }
    tmax[k] = tm;
    // singular vectors beyond each train's own rank -> 0
    c->launches++;
    TRY(qtt_mask_cols_batch<R>(X.as<C>(), Tcols * jq, Tcols, jq, jq, dtr, 4, B, c->stream));
    // padded core k of train b = X_b[:, :tm]^H (tm x Tcols)
    TRY(newc[k].alloc(c, (size_t)B * tm * Tcols * sizeof(C)));
    c->launches++;
    TRY(qtt_copy_batch<R>(X.as<C>(), Tcols * jq, L1(tm, 1), L1(Tcols, jq), tm, Tcols, 1, newc[k].as<C>(), Tcols,
                          tm * Tcols, B, c->stream));
    // P_b = T_b X_b[:, :tm] (a0 x tm); T_{k-1,b} = A_{k-1,b} P_b
    DBuf P, Tn;
    TRY(P.alloc(c, (size_t)B * a0 * tm * sizeof(C)));
    TRY(gemm<R>(c, bgemm<R>(B, a0, tm, Tcols, tst, L1(a0, Tcols), L1(Tcols, 1), Tcols * jq, L1(Tcols, jq),
                            L1(tm, 1), a0 * tm, L1(a0, tm), L1(tm, 1)),
                T, X.as<C>(), P.as<C>()));
    const int64_t pr = (int64_t)r[k - 1] * n[k - 1];
    TRY(Tn.alloc(c, (size_t)B * pr * tm * sizeof(C)));
    TRY(gemm<R>(c, bgemm<R>(B, pr, tm, a0, xst, L1(pr, a0), L1(a0, 1), a0 * tm, L1(a0, tm), L1(tm, 1), pr * tm,
                            L1(pr, tm), L1(tm, 1)),
                A(k - 1), P.as<C>(), Tn.as<C>()));
    Tb = std::move(Tn);
    T = Tb.as<C>();
    tst = pr * tm;
  }
  // ---- outputs cropped to each train's ranks
  std::vector<C*> ptrs((size_t)d * B);
  std::vector<int> t01((size_t)2 * d * B);
  for (int b = 0; b < B; ++b) {
    std::vector<int> rb(d + 1, 1);
    for (int k = 1; k < d; ++k) rb[k] = tb[b][k];
    int st;
    ys[b] = tt_alloc(c, d, n, rb, x0->dtype, &st);
    if (!ys[b]) {
      for (int e = 0; e < b; ++e) {
        tt_free(ys[e]);
        ys[e] = nullptr;
      }
      return st;
    }
    for (int k = 0; k < d; ++k) {
      ptrs[(size_t)k * B + b] = reinterpret_cast<C*>(static_cast<char*>(ys[b]->data) + ys[b]->off[k]);
      t01[(size_t)k * B + b] = rb[k];
      t01[(size_t)d * B + (size_t)k * B + b] = rb[k + 1];
    }
    if (infos) {
      infos[b].norm = nrm[b];
      infos[b].delta = delta[b];
      infos[b].tail = sqrt(tail2[b]);
      infos[b].err = -1;
      infos[b].capped = capped[b];
      infos[b].max_rank_out = *std::max_element(rb.begin(), rb.end());
    }
  }
  DBuf meta;
  TRY(meta.alloc(c, ptrs.size() * sizeof(C*) + t01.size() * sizeof(int)));
  C** dptrs = meta.as<C*>();
  int* dt01 = reinterpret_cast<int*>(dptrs + ptrs.size());
  if (cudaMemcpyAsync(dptrs, ptrs.data(), ptrs.size() * sizeof(C*), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(dt01, t01.data(), t01.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return QTT_ERR_CUDA;
  tmax[0] = tmax[d] = 1;
  for (int k = 0; k < d; ++k) {
    const C* src = k == 0 ? T : newc[k].as<C>();
    c->launches++;
    TRY(qtt_crop_batch<R>(src, (int64_t)tmax[k] * n[k] * tmax[k + 1], tmax[k], n[k], tmax[k + 1],
                          dptrs + (size_t)k * B, dt01 + (size_t)k * B, dt01 + (size_t)d * B + (size_t)k * B, B,
                          c->stream));
  }
  // the host arrays above were copied from pageable memory (staged before return)
  return QTT_OK;
}

template int round_det_batch<double>(qtt_ctx*, int, const qtt_tt* const*, double, int, qtt_round_info*, qtt_tt**);
template int round_det_batch<float>(qtt_ctx*, int, const qtt_tt* const*, double, int, qtt_round_info*, qtt_tt**);

// -------------------------------------------------------------- TT sum
// z = a x + b y: block-diagonal placement of the cores (ranks add; a and b
// scale the first core's blocks).
template <class R>
int add_dev(qtt_ctx* c, cplx<R> a, const qtt_tt* x, cplx<R> b, const qtt_tt* y, qtt_tt** out) {
  const int d = x->d;
  std::vector<int> r(d + 1, 1);
  for (int k = 1; k < d; ++k) r[k] = x->r[k] + y->r[k];
  int st;
  qtt_tt* z = tt_alloc(c, d, x->n, r, x->dtype, &st);
  if (!z) return st;
  cudaMemsetAsync(z->data, 0, z->bytes, c->stream);
  typedef cplx<R> C;
  const C one(1, 0);
  for (int k = 0; k < d; ++k) {
    const int64_t n = x->n[k];
    const int64_t xa = x->r[k], xb = x->r[k + 1], ya = y->r[k], yb = y->r[k + 1];
    C* Z = core_ptr<C>(z, k);
    const int64_t zb = r[k + 1];
    if (d == 1) {
      // z = a x + b y elementwise (single core)
      c->launches += 2;
      int s1 = qtt_place_block<R>(core_ptr<C>(x, 0), 1, n, 1, Z, 1, 0, 0, a, c->stream);
      if (s1) {
        tt_free(z);
        return s1;
      }
      // accumulate b*y with a rank-1 GEMM: Z (1 x n) += b * [1] (1 x 1) * y (1 x n)
      void* onep;
      if (dalloc(c, &onep, sizeof(C))) {
        tt_free(z);
        return QTT_ERR_OOM;
      }
      cudaMemcpyAsync(onep, &one, sizeof(C), cudaMemcpyHostToDevice, c->stream);
      GemmDesc g;
      g.bA = g.bB = g.bC = MIdx{1, 1, 0, 0};
      g.M = 1;
      g.N = n;
      g.K = 1;
      g.batch = 1;
      g.mA = MIdx{1, 1, 1, 0};
      g.kA = MIdx{1, 1, 1, 0};
      g.kB = MIdx{1, 1, n, 0};
      g.nB = MIdx{n, 1, 1, 0};
      g.mC = MIdx{1, 1, n, 0};
      g.nC = MIdx{n, 1, 1, 0};
      g.conjA = g.conjB = 0;
      int s2 = qtt_gemm<R>(g, b, one, reinterpret_cast<C*>(onep), core_ptr<C>(y, 0), Z, c->stream);
      dfree(c, onep);
      if (s2) {
        tt_free(z);
        return s2;
      }
      break;
    }
    const int64_t xoff0 = 0, xoff1 = 0;
    const int64_t yoff0 = (k == 0) ? 0 : xa;
    const int64_t yoff1 = (k == d - 1) ? 0 : xb;
    c->launches += 2;
    int s1 = qtt_place_block<R>(core_ptr<C>(x, k), xa, n, xb, Z, zb, xoff0, xoff1, k == 0 ? a : one, c->stream);
    int s2 = qtt_place_block<R>(core_ptr<C>(y, k), ya, n, yb, Z, zb, yoff0, yoff1, k == 0 ? b : one, c->stream);
    if (s1 || s2) {
      tt_free(z);
      return s1 ? s1 : s2;
    }
  }
  *out = z;
  return QTT_OK;
}

template int add_dev<double>(qtt_ctx*, zc, const qtt_tt*, zc, const qtt_tt*, qtt_tt**);
template int add_dev<float>(qtt_ctx*, cc, const qtt_tt*, cc, const qtt_tt*, qtt_tt**);

// host -> device copy on the context stream, then wait for it
int upload(qtt_ctx* c, void* dst, const void* src, size_t bytes) {
  if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) return QTT_ERR_CUDA;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

// ------------------------------------------------------------------- TT-SVD
template <class R>
int tt_svd_dev(qtt_ctx* c, int d, const std::vector<int>& modes, const cplx<R>* dense, double eps, int max_rank,
               qtt_dtype dt, qtt_tt** out) {
  int64_t total = 1;
  for (int k = 0; k < d; ++k) total *= modes[k];
  DBuf scal;
  TRY(scal.alloc(c, 64));
  double* dscal = scal.as<double>();
  int* dint = reinterpret_cast<int*>(dscal + 4);
  c->launches++;
  TRY(qtt_sumsq<R>(dense, total, dscal, c->stream));
  double n2 = 0;
  TRY(sync_read(c, &n2, dscal, sizeof(double)));
  if (!std::isfinite(n2)) return QTT_ERR_NAN;
  const double delta = d > 1 ? eps * sqrt(n2) / sqrt((double)(d - 1)) : 0.0;
  std::vector<DBuf> cores(d);
  std::vector<int> ranks(d + 1, 1);
  DBuf Cown;
  const cplx<R>* C = dense;
  int64_t rest = total;
  int64_t rprev = 1;
  for (int k = 0; k < d - 1; ++k) {
    const int64_t m = rprev * modes[k];
    rest /= modes[k];
    // C viewed as m x rest (row-major)
    DBuf U, sig;
    TRY(U.alloc(c, (size_t)m * m * sizeof(cplx<R>)));
    TRY(sig.alloc(c, (size_t)m * sizeof(R)));
    int64_t nsv = 0;
    TRY(left_svd<R>(c, C, m, rest, rest, U.as<cplx<R>>(), sig.as<R>(), &nsv));
    c->launches++;
    TRY(qtt_trunc_rank<R>(sig.as<R>(), (int)nsv, delta, max_rank, dint, dscal + 1, c->stream));
    int hv[2];
    TRY(sync_read(c, hv, dint, sizeof(hv)));
    const int t = hv[0];
    ranks[k + 1] = t;
    // core k = U[:, :t] as (rprev, n_k, t)
    TRY(cores[k].alloc(c, (size_t)m * t * sizeof(cplx<R>)));
    c->launches++;
    TRY(qtt_copy_strided<R>(U.as<cplx<R>>(), L1(m, nsv), L1(t, 1), m, t, 0, cores[k].as<cplx<R>>(), t, c->stream));
    // next C = U_t^H C  (t x rest)
    DBuf Cn;
    TRY(Cn.alloc(c, (size_t)t * rest * sizeof(cplx<R>)));
    TRY(mm<R>(c, t, rest, m, U.as<cplx<R>>(), 1, nsv, 1, C, rest, 1, 0, Cn.as<cplx<R>>(), rest, 1));
    Cown = std::move(Cn);
    C = Cown.as<cplx<R>>();
    rprev = t;
  }
  int st;
  std::vector<int> md(modes.begin(), modes.begin() + d);
  qtt_tt* y = tt_alloc(c, d, md, ranks, dt, &st);
  if (!y) return st;
  for (int k = 0; k < d; ++k) {
    const void* src = (k == d - 1) ? (const void*)C : cores[k].p;
    size_t bytes = (size_t)ranks[k] * modes[k] * ranks[k + 1] * sizeof(cplx<R>);
    cudaMemcpyAsync(static_cast<char*>(y->data) + y->off[k], src, bytes, cudaMemcpyDeviceToDevice, c->stream);
  }
  *out = y;
  return QTT_OK;
}

template int tt_svd_dev<double>(qtt_ctx*, int, const std::vector<int>&, const zc*, double, int, qtt_dtype, qtt_tt**);
template int tt_svd_dev<float>(qtt_ctx*, int, const std::vector<int>&, const cc*, double, int, qtt_dtype, qtt_tt**);
template int left_svd<double>(qtt_ctx*, const zc*, int64_t, int64_t, int64_t, zc*, double*, int64_t*);
template int left_svd<float>(qtt_ctx*, const cc*, int64_t, int64_t, int64_t, cc*, float*, int64_t*);

// ----------------------------------------------------------- inner product
template <class R>
int dot_dev(qtt_ctx* c, const qtt_tt* x, const qtt_tt* y, double out[2]) {
  const int d = x->d;
  DBuf W, T;
  // W_0 = [1]
  int64_t wa = 1, wb = 1;
  TRY(W.alloc(c, sizeof(cplx<R>)));
  cplx<R> one(1, 0);
  cudaMemcpyAsync(W.p, &one, sizeof(one), cudaMemcpyHostToDevice, c->stream);
  for (int k = 0; k < d; ++k) {
    const int64_t a0 = x->r[k], a1 = x->r[k + 1], b0 = y->r[k], b1 = y->r[k + 1], nk = x->n[k];
    const cplx<R>* Ak = reinterpret_cast<const cplx<R>*>(static_cast<const char*>(x->data) + x->off[k]);
    const cplx<R>* Bk = reinterpret_cast<const cplx<R>*>(static_cast<const char*>(y->data) + y->off[k]);
    // T[a0, (i, b1)] = W[a0, b0] B[b0, (i, b1)]
    DBuf Tn;
    TRY(Tn.alloc(c, (size_t)a0 * nk * b1 * sizeof(cplx<R>)));
    TRY(mm<R>(c, a0, nk * b1, b0, W.as<cplx<R>>(), wb, 1, 0, Bk, nk * b1, 1, 0, Tn.as<cplx<R>>(), nk * b1, 1));
    // W'[a1, b1] = sum_{(a0, i)} conj(A[(a0, i), a1]) T[(a0, i), b1]
    DBuf Wn;
    TRY(Wn.alloc(c, (size_t)a1 * b1 * sizeof(cplx<R>)));
    TRY(mm<R>(c, a1, b1, a0 * nk, Ak, 1, a1, 1, Tn.as<cplx<R>>(), b1, 1, 0, Wn.as<cplx<R>>(), b1, 1));
    W = std::move(Wn);
    wa = a1;
    wb = b1;
  }
  (void)wa;
  cplx<R> h;
  TRY(sync_read(c, &h, W.p, sizeof(h)));
  out[0] = (double)h.re;
  out[1] = (double)h.im;
  return QTT_OK;
}

template int dot_dev<double>(qtt_ctx*, const qtt_tt*, const qtt_tt*, double*);
template int dot_dev<float>(qtt_ctx*, const qtt_tt*, const qtt_tt*, double*);

// Frobenius norm: R factor sweep, then the norm of the centre.
template <class R>
int norm_dev(qtt_ctx* c, const qtt_tt* x, double* out) {
  const int d = x->d;
  auto A = [&](int k) { return reinterpret_cast<const cplx<R>*>(static_cast<const char*>(x->data) + x->off[k]); };
  DBuf Rprev;
  int64_t rp = 1;
  DBuf scal;
  TRY(scal.alloc(c, 64));
  for (int k = 0; k < d; ++k) {
    const int64_t a0 = x->r[k], nk = x->n[k], a1 = x->r[k + 1];
    DBuf Mb;
    const cplx<R>* M = A(k);
    if (k > 0) {
      TRY(Mb.alloc(c, (size_t)rp * nk * a1 * sizeof(cplx<R>)));
      TRY(mm<R>(c, rp, nk * a1, a0, Rprev.as<cplx<R>>(), a0, 1, 0, A(k), nk * a1, 1, 0, Mb.as<cplx<R>>(), nk * a1, 1));
      M = Mb.as<cplx<R>>();
    }
    const int64_t m = rp * nk;
    if (k == d - 1) {
      c->launches++;
      TRY(qtt_sumsq<R>(M, m * a1, scal.as<double>(), c->stream));
      break;
    }
    DBuf Rn;
    const int64_t rn = std::min(m, a1);
    TRY(Rn.alloc(c, (size_t)rn * a1 * sizeof(cplx<R>)));
    int64_t got;
    TRY(tsqr_r<R>(c, M, L1(m, a1), L1(a1, 1), 0, m, a1, Rn.as<cplx<R>>(), &got));
    Rprev = std::move(Rn);
    rp = rn;
  }
  double s2;
  TRY(sync_read(c, &s2, scal.p, sizeof(double)));
  *out = sqrt(s2);
  return QTT_OK;
}

template int norm_dev<double>(qtt_ctx*, const qtt_tt*, double*);
template int norm_dev<float>(qtt_ctx*, const qtt_tt*, double*);

// ------------------------------------------------------- sketched rounding
// Randomize-then-orthogonalize for s = sum_t coef_t A_t x_t (A_t may be NULL).
// With dot_out set, only the right partial contractions are run, down to the
// first core, and the bilinear form sum_i S(i) s(i) is returned in dot_out
// (no projection, no rounding).
template <class R>
static int sketch_core(qtt_ctx* c, int T, const qtt_complex* coef, const qtt_mpo* const* ops,
                       const qtt_tt* const* xs, const qtt_tt* S, double eps, int max_rank, qtt_round_info* info,
                       qtt_tt** yout, double* dot_out) {
  const int d = S->d;
  typedef cplx<R> C;
  // identity operators for terms without one
  std::vector<qtt_mpo*> own(T, nullptr);
  std::vector<const qtt_mpo*> A(T);
  struct Cleanup {
    std::vector<qtt_mpo*>& v;
    ~Cleanup() {
      for (auto* p : v) mpo_free(p);
    }
  } cleanup{own};
  for (int t = 0; t < T; ++t) {
    if (xs[t]->d != d) return QTT_ERR_ARG;
    if (ops && ops[t]) {
      if (ops[t]->d != d) return QTT_ERR_ARG;
      A[t] = ops[t];
    } else {
      int st;
      std::vector<int> g(d + 1, 1);
      own[t] = mpo_alloc(c, d, xs[t]->n, xs[t]->n, g, S->dtype, &st);
      if (!own[t]) return st;
      for (int k = 0; k < d; ++k) {
        c->launches++;
        TRY(qtt_identity_core<R>(1, xs[t]->n[k],
                                 reinterpret_cast<C*>(static_cast<char*>(own[t]->data) + own[t]->off[k]), c->stream));
        own[t]->diag[k] = 1;
      }
      A[t] = own[t];
    }
    for (int k = 0; k < d; ++k) {
      if (A[t]->ni[k] != xs[t]->n[k] || A[t]->no[k] != S->n[k]) return QTT_ERR_ARG;
    }
  }
  auto Dk = [&](int t, int k) {
    return reinterpret_cast<const C*>(static_cast<const char*>(A[t]->data) + A[t]->off[k]);
  };
  auto Xk = [&](int t, int k) {
    return reinterpret_cast<const C*>(static_cast<const char*>(xs[t]->data) + xs[t]->off[k]);
  };
  auto Sk = [&](int k) { return reinterpret_cast<const C*>(static_cast<const char*>(S->data) + S->off[k]); };
  // stacked bond sizes and offsets
  std::vector<std::vector<int64_t>> boff(d + 1, std::vector<int64_t>(T + 1, 0));
  for (int k = 0; k <= d; ++k)
    for (int t = 0; t < T; ++t) boff[k][t + 1] = boff[k][t] + (int64_t)A[t]->g[k] * xs[t]->r[k];
  auto Bt = [&](int k) { return boff[k][T]; };
  // ---- right partial contractions W_k (Bt_k x l_k), k = 1..d
  std::vector<DBuf> W(d + 1);
  {
    TRY(W[d].alloc(c, (size_t)T * sizeof(C)));
    std::vector<C> ones(T, C(1, 0));
    cudaMemcpyAsync(W[d].p, ones.data(), T * sizeof(C), cudaMemcpyHostToDevice, c->stream);
  }
  for (int k = d - 1; k >= (dot_out ? 0 : 1); --k) {
    const int64_t l0 = S->r[k], l1 = S->r[k + 1], no = S->n[k];
    TRY(W[k].alloc(c, (size_t)Bt(k) * l0 * sizeof(C)));
    // the sketch side: under QTT_PREC_TF32S these contractions run on the
    // tensor cores, batched (not for an exact inner product)
    InSketch in_sketch(c);
    if (dot_out) c->in_sketch = false;
    for (int t = 0; t < T; ++t) {
      const int64_t g0 = A[t]->g[k], g1 = A[t]->g[k + 1], ni = A[t]->ni[k];
      const int64_t a0 = xs[t]->r[k], a1 = xs[t]->r[k + 1];
      const C* Wn = W[k + 1].as<C>() + boff[k + 1][t] * l1;  // (g1 a1) x l1
      // U1[g1, a1, i, l0] = sum_l1 Wn[(g1 a1), l1] S[l0, i, l1]
      DBuf U1, U2;
      TRY(U1.alloc(c, (size_t)g1 * a1 * no * l0 * sizeof(C)));
      {
        GemmDesc g;
        g.bA = g.bB = g.bC = B0();
        g.M = g1 * a1;
        g.N = no * l0;
        g.K = l1;
        g.batch = 1;
        g.mA = L1(g.M, l1);
        g.kA = L1(l1, 1);
        g.kB = L1(l1, 1);
        g.nB = L2(no, l1, l0, no * l1);
        g.mC = L1(g.M, no * l0);
        g.nC = L1(g.N, 1);
        g.conjA = g.conjB = 0;
        TRY(gemm<R>(c, g, Wn, Sk(k), U1.as<C>()));
      }
      TRY(dbg_finite<R>(c, U1.as<C>(), g1 * a1 * no * l0, "sketch U1", k));
      // U2[a1, g0, j, l0] = sum_{i, g1} D[g0, i, j, g1] U1[g1, a1, i, l0]   (batch a1)
      TRY(U2.alloc(c, (size_t)a1 * g0 * ni * l0 * sizeof(C)));
      const bool dg = A[t]->diag[k] && ni == no;
      if (dg) {
        // diagonal core (D[g0, i, j, g1] = 0 for i != j): batch (a1, i),
        // U2[a1, g0, i, l0] = sum_g1 D[g0, i, i, g1] U1[g1, a1, i, l0]
        GemmDesc g;
        g.M = g0;
        g.N = l0;
        g.K = g1;
        g.batch = a1 * ni;
        g.bA = L2(a1, 0, ni, (ni + 1) * g1);
        g.mA = L1(g0, no * ni * g1);
        g.kA = L1(g1, 1);
        g.bB = L2(a1, no * l0, ni, l0);
        g.kB = L1(g1, a1 * no * l0);
        g.nB = L1(l0, 1);
        g.bC = L2(a1, g0 * ni * l0, ni, l0);
        g.mC = L1(g0, ni * l0);
        g.nC = L1(l0, 1);
        g.conjA = g.conjB = 0;
        TRY(gemm<R>(c, g, Dk(t, k), U1.as<C>(), U2.as<C>()));
      } else {
        GemmDesc g;
        g.M = g0 * ni;
        g.N = l0;
        g.K = no * g1;
        g.batch = a1;
        g.bA = L1(a1, 0);
        g.mA = L2(g0, no * ni * g1, ni, g1);
        g.kA = L2(no, ni * g1, g1, 1);
        g.bB = L1(a1, no * l0);
        g.kB = L2(no, l0, g1, a1 * no * l0);
        g.nB = L1(l0, 1);
        g.bC = L1(a1, g0 * ni * l0);
        g.mC = L1(g.M, l0);
        g.nC = L1(l0, 1);
        g.conjA = g.conjB = 0;
        TRY(gemm<R>(c, g, Dk(t, k), U1.as<C>(), U2.as<C>()));
      }
      TRY(dbg_finite<R>(c, U2.as<C>(), a1 * g0 * ni * l0, "sketch U2", k));
      // W_k[g0, a0, l0] = sum_{j, a1} X[a0, j, a1] U2[a1, g0, j, l0]   (batch g0)
      {
        GemmDesc g;
        g.M = a0;
        g.N = l0;
        g.K = ni * a1;
        g.batch = g0;
        g.bA = L1(g0, 0);
        g.mA = L1(a0, ni * a1);
        g.kA = L1(g.K, 1);
        g.bB = L1(g0, ni * l0);
        g.kB = L2(ni, l0, a1, g0 * ni * l0);
        g.nB = L1(l0, 1);
        g.bC = L1(g0, a0 * l0);
        g.mC = L1(a0, l0);
        g.nC = L1(l0, 1);
        g.conjA = g.conjB = 0;
        TRY(gemm<R>(c, g, Xk(t, k), U2.as<C>(), W[k].as<C>() + boff[k][t] * l0));
      }
    }
    TRY(dbg_finite<R>(c, W[k].as<C>(), Bt(k) * l0, "sketch W", k));
  }
  if (dot_out) {
    // W_0 holds one entry per term (bond 0 has rank 1 for every term)
    std::vector<C> w0(T);
    TRY(sync_read(c, w0.data(), W[0].p, (size_t)T * sizeof(C)));
    double re = 0, im = 0;
    for (int t = 0; t < T; ++t) {
      re += coef[t].re * (double)w0[t].re - coef[t].im * (double)w0[t].im;
      im += coef[t].re * (double)w0[t].im + coef[t].im * (double)w0[t].re;
    }
    dot_out[0] = re;
    dot_out[1] = im;
    return QTT_OK;
  }
  // ---- left-to-right projection
  std::vector<DBuf> outc(d);
  std::vector<int> orank(d + 1, 1);
  DBuf M;  // l_k x Bt_k
  {
    TRY(M.alloc(c, (size_t)T * sizeof(C)));
    std::vector<C> cf(T);
    for (int t = 0; t < T; ++t) cf[t] = C((R)coef[t].re, (R)coef[t].im);
    cudaMemcpyAsync(M.p, cf.data(), T * sizeof(C), cudaMemcpyHostToDevice, c->stream);
  }
  int64_t lk = 1;
  for (int k = 0; k < d; ++k) {
    const int64_t no = S->n[k];
    const int64_t Bn = Bt(k + 1);
    DBuf Y;
    TRY(Y.alloc(c, (size_t)lk * no * Bn * sizeof(C)));
    for (int t = 0; t < T; ++t) {
      const int64_t g0 = A[t]->g[k], g1 = A[t]->g[k + 1], ni = A[t]->ni[k];
      const int64_t a0 = xs[t]->r[k], a1 = xs[t]->r[k + 1];
      // T1[l, g0, j, a1] = sum_a0 M[l, off + g0 a0 + a0] X[a0, j, a1]
      DBuf T1;
      TRY(T1.alloc(c, (size_t)lk * g0 * ni * a1 * sizeof(C)));
      {
        GemmDesc g;
        g.bA = g.bB = g.bC = B0();
        g.M = lk * g0;
        g.N = ni * a1;
        g.K = a0;
        g.batch = 1;
        g.mA = L2(lk, Bt(k), g0, a0);
        g.kA = L1(a0, 1);
        g.kB = L1(a0, ni * a1);
        g.nB = L1(g.N, 1);
        g.mC = L1(g.M, ni * a1);
        g.nC = L1(g.N, 1);
        g.conjA = g.conjB = 0;
        TRY(gemm<R>(c, g, M.as<C>() + boff[k][t], Xk(t, k), T1.as<C>()));
      }
      TRY(dbg_finite<R>(c, T1.as<C>(), lk * g0 * ni * a1, "left T1", k));
      // Y[l, i, off' + g1 a1 + a1] = sum_{g0, j} D[g0, i, j, g1] T1[l, g0, j, a1]  (batch l)
      if (A[t]->diag[k] && ni == no) {
        // diagonal core: batch (l, i), sum over g0 only with j = i
        GemmDesc g;
        g.M = g1;
        g.N = a1;
        g.K = g0;
        g.batch = lk * no;
        g.bA = L2(lk, 0, no, (ni + 1) * g1);
        g.mA = L1(g1, 1);
        g.kA = L1(g0, no * ni * g1);
        g.bB = L2(lk, g0 * ni * a1, no, a1);
        g.kB = L1(g0, ni * a1);
        g.nB = L1(a1, 1);
        g.bC = L2(lk, no * Bn, no, Bn);
        g.mC = L1(g1, a1);
        g.nC = L1(a1, 1);
        g.conjA = g.conjB = 0;
        TRY(gemm<R>(c, g, Dk(t, k), T1.as<C>(), Y.as<C>() + boff[k + 1][t]));
      } else {
        GemmDesc g;
        g.M = no * g1;
        g.N = a1;
        g.K = g0 * ni;
        g.batch = lk;
        g.bA = L1(lk, 0);
        g.mA = L2(no, ni * g1, g1, 1);
        g.kA = L2(g0, no * ni * g1, ni, g1);
        g.bB = L1(lk, g0 * ni * a1);
        g.kB = L1(g.K, a1);
        g.nB = L1(a1, 1);
        g.bC = L1(lk, no * Bn);
        g.mC = L2(no, Bn, g1, a1);
        g.nC = L1(a1, 1);
        g.conjA = g.conjB = 0;
        TRY(gemm<R>(c, g, Dk(t, k), T1.as<C>(), Y.as<C>() + boff[k + 1][t]));
      }
    }
    const int64_t l1 = S->r[k + 1];
    // Z = Y (lk no x Bn) W_{k+1} (Bn x l1)
    DBuf Z;
    TRY(Z.alloc(c, (size_t)lk * no * l1 * sizeof(C)));
    TRY(dbg_finite<R>(c, Y.as<C>(), lk * no * Bn, "left Y", k));
    TRY(mm<R>(c, lk * no, l1, Bn, Y.as<C>(), Bn, 1, 0, W[k + 1].as<C>(), l1, 1, 0, Z.as<C>(), l1, 1));
    TRY(dbg_finite<R>(c, Z.as<C>(), lk * no * l1, "left Z", k));
    if (k == d - 1) {
      outc[k] = std::move(Z);
      break;
    }
    // Q of Z (lk no x l1): new core (lk, no, q)
    const int64_t m = lk * no, q = std::min(m, l1);
    DBuf Wq, tau;
    TRY(outc[k].alloc(c, (size_t)m * q * sizeof(C)));
    TRY(Wq.alloc(c, (size_t)m * l1 * sizeof(C)));
    TRY(tau.alloc(c, (size_t)2 * l1 * sizeof(C)));
    TRY(qr_launch<R>(c, Z.as<C>(), B0(), L1(m, l1), L1(l1, 1), 0, m, l1, m, m, 1, Wq.as<C>(), nullptr, 0, 0,
                     tau.as<C>(), outc[k].as<C>(), 0, q));
    TRY(dbg_finite<R>(c, outc[k].as<C>(), m * q, "left Q", k));
    orank[k + 1] = (int)q;
    // M_{k+1} = Q^H Y  (q x Bn)
    DBuf Mn;
    TRY(Mn.alloc(c, (size_t)q * Bn * sizeof(C)));
    TRY(mm<R>(c, q, Bn, m, outc[k].as<C>(), 1, q, 1, Y.as<C>(), Bn, 1, 0, Mn.as<C>(), Bn, 1));
    M = std::move(Mn);
    lk = q;
  }
  // assemble the projected train, then round it deterministically
  int st;
  qtt_tt* P = tt_alloc(c, d, S->n, orank, S->dtype, &st);
  if (!P) return st;
  for (int k = 0; k < d; ++k) {
    size_t bytes = (size_t)orank[k] * S->n[k] * orank[k + 1] * sizeof(C);
    cudaMemcpyAsync(static_cast<char*>(P->data) + P->off[k], outc[k].p, bytes, cudaMemcpyDeviceToDevice, c->stream);
  }
  int rs = round_det<R>(c, P, eps, max_rank, nullptr, info, yout, true);
  tt_free(P);
  return rs;
}

template <class R>
int round_sketched(qtt_ctx* c, int T, const qtt_complex* coef, const qtt_mpo* const* ops, const qtt_tt* const* xs,
                   const qtt_tt* S, double eps, int max_rank, qtt_round_info* info, qtt_tt** yout) {
  return sketch_core<R>(c, T, coef, ops, xs, S, eps, max_rank, info, yout, nullptr);
}

// <y, s> = sum_i conj(y(i)) s(i) for the structured sum s = sum_t coef_t A_t x_t,
// by the right partial contractions of the sketched rounding with the
// conjugated train of y in the place of the sketch.
template <class R>
int structured_dot(qtt_ctx* c, int T, const qtt_complex* coef, const qtt_mpo* const* ops, const qtt_tt* const* xs,
                   const qtt_tt* y, double out[2]) {
  int st;
  qtt_tt* yc = tt_alloc(c, y->d, y->n, y->r, y->dtype, &st);
  if (!yc) return st;
  for (int k = 0; k < y->d; ++k) {
    const int64_t rows = (int64_t)y->r[k] * y->n[k], cols = y->r[k + 1];
    c->launches++;
    st = qtt_copy_strided<R>(core_ptr<cplx<R>>(y, k), L1(rows, cols), L1(cols, 1), rows, cols, 1,
                             core_ptr<cplx<R>>(yc, k), cols, c->stream);
    if (st) {
      tt_free(yc);
      return st;
    }
  }
  st = sketch_core<R>(c, T, coef, ops, xs, yc, 0.0, 0, nullptr, nullptr, out);
  tt_free(yc);
  return st;
}

template int structured_dot<double>(qtt_ctx*, int, const qtt_complex*, const qtt_mpo* const*, const qtt_tt* const*,
                                    const qtt_tt*, double*);
template int structured_dot<float>(qtt_ctx*, int, const qtt_complex*, const qtt_mpo* const*, const qtt_tt* const*,
                                   const qtt_tt*, double*);
template int round_sketched<double>(qtt_ctx*, int, const qtt_complex*, const qtt_mpo* const*, const qtt_tt* const*,
                                    const qtt_tt*, double, int, qtt_round_info*, qtt_tt**);
template int round_sketched<float>(qtt_ctx*, int, const qtt_complex*, const qtt_mpo* const*, const qtt_tt* const*,
                                   const qtt_tt*, double, int, qtt_round_info*, qtt_tt**);
