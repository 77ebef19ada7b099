// AMEn approximation of y = A x on the device (Sec. 2.1: the optimisation-
// based alternative to forming A x and rounding it; Sec. 3.2: how the Green
// operator is applied), after Dolgov & Savostyanov's alternating minimal
// energy method with residual enrichment, matrix-vector form.
//
// Before every sweep y and the residual train z are right-orthogonalised and
// the right interfaces Psi (y^H A x), Psi^z (z^H A x) and Psi^zy (z^H y) are
// built from the last core down.  Sweeping k = 0..d-1, core k of y becomes
// the projection Phi_k A_k X_k Psi_{k+1} (the optimal core with the others
// fixed), is truncated by SVD at eps ||Y_k|| / sqrt(d - 1) (at most max_rank
// kept, 0: no cap), z's core k
// becomes the leading left singular vectors of the residual A x - y
// projected on z's interfaces, and the kept basis of y's core k is enriched
// by the residual projected on y's left and z's right interface before it is
// orthonormalised (the enrichment directions get zero weight in core k+1, so
// y is unchanged).  Sweeps stop when no core changed by more than eps; the
// result is rounded at eps.  Every contraction is one strided GEMM
// (two-level multi-indices, no permutation passes); the factorisations are
// the library's TSQR + one-sided Jacobi SVD.
#include <float.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "engine.h"
#include "kernels.h"

namespace {

#define TRY(expr)                  \
  do {                             \
    int _st = (expr);              \
    if (_st != QTT_OK) return _st; \
  } while (0)

inline MIdx L1(int64_t n, int64_t s) { return MIdx{n, 1, s, 0}; }
inline MIdx L2(int64_t n1, int64_t s1, int64_t n2, int64_t s2) { return MIdx{n1, n2, s1, s2}; }
inline MIdx B0() { return MIdx{1, 1, 0, 0}; }

// out = a x + b y, elementwise
template <class R>
__global__ void axpby_kernel(const cplx<R>* __restrict__ x, const cplx<R>* __restrict__ y, int64_t n, R a, R b,
                             cplx<R>* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = cplx<R>(a * x[e].re + b * y[e].re, a * x[e].im + b * y[e].im);
}

template <class R>
int axpby(qtt_ctx* c, const cplx<R>* x, const cplx<R>* y, int64_t n, R a, R b, cplx<R>* out) {
  if (n <= 0) return QTT_OK;
  c->launches++;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 1 << 20);
  axpby_kernel<R><<<(unsigned)blocks, 256, 0, c->stream>>>(x, y, n, a, b, out);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

GemmDesc desc(int64_t M, int64_t N, int64_t K, int64_t batch, MIdx bA, MIdx mA, MIdx kA, int conjA, MIdx bB,
              MIdx kB, MIdx nB, MIdx bC, MIdx mC, MIdx nC) {
  GemmDesc g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = batch;
  g.bA = bA;
  g.mA = mA;
  g.kA = kA;
  g.bB = bB;
  g.kB = kB;
  g.nB = nB;
  g.bC = bC;
  g.mC = mC;
  g.nC = nC;
  g.conjA = conjA;
  g.conjB = 0;
  return g;
}

// Row-major matrix product C (M x N) = alpha A (M x K, ld lda, conj) B (K x N, ld ldb) + beta C.
template <class R>
int mmr(qtt_ctx* c, int64_t M, int64_t N, int64_t K, const cplx<R>* A, int64_t lda, int conjA, const cplx<R>* B,
        int64_t ldb, cplx<R>* C, cplx<R> alpha = cplx<R>(1, 0), cplx<R> beta = cplx<R>(0, 0)) {
  if (M <= 0 || N <= 0) return QTT_OK;
  if (K <= 0) return cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(cplx<R>), c->stream) == cudaSuccess ? QTT_OK
                                                                                             : QTT_ERR_CUDA;
  GemmDesc g = desc(M, N, K, 1, B0(), L1(M, lda), L1(K, 1), conjA, B0(), L1(K, ldb), L1(N, 1), B0(), L1(M, N),
                    L1(N, 1));
  return gemm_ab<R>(c, g, alpha, beta, A, B, C);
}

// C (M x N) = alpha A^H B: A is K x M row-major (ld lda), B K x N (ld ldb).
template <class R>
int mmh(qtt_ctx* c, int64_t M, int64_t N, int64_t K, const cplx<R>* A, int64_t lda, const cplx<R>* B, int64_t ldb,
        cplx<R>* C) {
  if (M <= 0 || N <= 0) return QTT_OK;
  GemmDesc g = desc(M, N, K, 1, B0(), L1(M, 1), L1(K, lda), 1, B0(), L1(K, ldb), L1(N, 1), B0(), L1(M, N),
                    L1(N, 1));
  return gemm_ab<R>(c, g, cplx<R>(1, 0), cplx<R>(0, 0), A, B, C);
}

template <class R>
struct Buf {
  DBuf b;
  int d0 = 0, d1 = 0, d2 = 0;   // shape (a train core (r0, n, r1) or an interface (ry, ra, rx))
  cplx<R>* p() const { return b.as<cplx<R>>(); }
  int64_t size() const { return (int64_t)d0 * d1 * d2; }
  int make(qtt_ctx* c, int a, int n, int r) {
    d0 = a;
    d1 = n;
    d2 = r;
    return b.alloc(c, (size_t)std::max<int64_t>(size(), 1) * sizeof(cplx<R>));
  }
};

// The operator's core k: (g0, m, n, g1).
struct OpCore {
  const void* p;
  int g0, m, n, g1;
};

// T2[a, b', i, g'] = sum_{g, j} (phi X)[a, g, j, b'] A[g, i, j, g'] for phi (ry, ra, rx).
template <class R>
int phi_ax(qtt_ctx* c, const Buf<R>& phi, const OpCore& A, const cplx<R>* X, int rx1, DBuf* T2) {
  const int64_t ry = phi.d0, ra = phi.d1, rx = phi.d2, n = A.n, m = A.m, ra1 = A.g1;
  DBuf T1;
  TRY(T1.alloc(c, (size_t)ry * ra * n * rx1 * sizeof(cplx<R>)));
  TRY(mmr<R>(c, ry * ra, n * rx1, rx, phi.p(), rx, 0, X, n * rx1, T1.as<cplx<R>>()));
  TRY(T2->alloc(c, (size_t)ry * rx1 * m * ra1 * sizeof(cplx<R>)));
  GemmDesc g = desc(rx1, m * ra1, ra * n, ry, L1(ry, ra * n * rx1), L1(rx1, 1), L2(ra, n * rx1, n, rx1), 0, B0(),
                    L2(ra, m * n * ra1, n, ra1), L2(m, n * ra1, ra1, 1), L1(ry, rx1 * m * ra1), L1(rx1, m * ra1),
                    L1(m * ra1, 1));
  return gemm_ab<R>(c, g, cplx<R>(1, 0), cplx<R>(0, 0), T1.as<cplx<R>>(),
                    reinterpret_cast<const cplx<R>*>(A.p), T2->as<cplx<R>>());
}

// out[a, i, a'] (+)= alpha sum T2[a, b', i, g'] psi[a', g', b']
template <class R>
int contract_psi(qtt_ctx* c, const cplx<R>* T2, int64_t ry, int64_t rx1, int64_t m, int64_t ra1, const Buf<R>& psi,
                 cplx<R>* out, cplx<R> alpha, cplx<R> beta) {
  const int64_t ry1 = psi.d0;
  GemmDesc g = desc(ry * m, ry1, rx1 * ra1, 1, B0(), L2(ry, rx1 * m * ra1, m, ra1), L2(rx1, m * ra1, ra1, 1), 0,
                    B0(), L2(rx1, 1, ra1, rx1), L1(ry1, ra1 * rx1), B0(), L1(ry * m, ry1), L1(ry1, 1));
  return gemm_ab<R>(c, g, alpha, beta, T2, psi.p(), out);
}

// Local projection Phi A_k X_k Psi -> out (ry, m, ry1)
template <class R>
int proj(qtt_ctx* c, const Buf<R>& phi, const OpCore& A, const cplx<R>* X, int rx1, const Buf<R>& psi,
         Buf<R>* out) {
  DBuf T2;
  TRY(phi_ax<R>(c, phi, A, X, rx1, &T2));
  TRY(out->make(c, phi.d0, A.m, psi.d0));
  return contract_psi<R>(c, T2.as<cplx<R>>(), phi.d0, rx1, A.m, A.g1, psi, out->p(), cplx<R>(1, 0),
                         cplx<R>(0, 0));
}

// Phi_{k+1}[a', g', b'] = sum conj(Y[a, i, a']) T2[a, b', i, g']
template <class R>
int phi_next(qtt_ctx* c, const Buf<R>& phi, const OpCore& A, const cplx<R>* X, int rx1, const Buf<R>& Y,
             Buf<R>* out) {
  DBuf T2;
  TRY(phi_ax<R>(c, phi, A, X, rx1, &T2));
  const int64_t ry = Y.d0, m = Y.d1, ry1 = Y.d2, ra1 = A.g1;
  TRY(out->make(c, (int)ry1, (int)ra1, rx1));
  GemmDesc g = desc(ry1, ra1 * rx1, ry * m, 1, B0(), L1(ry1, 1), L2(ry, m * ry1, m, ry1), 1, B0(),
                    L2(ry, (int64_t)rx1 * m * ra1, m, ra1), L2(ra1, 1, rx1, m * ra1), B0(), L1(ry1, ra1 * rx1),
                    L1(ra1 * rx1, 1));
  return gemm_ab<R>(c, g, cplx<R>(1, 0), cplx<R>(0, 0), Y.p(), T2.as<cplx<R>>(), out->p());
}

// Psi_k[a, g, b] = sum conj(Y[a, i, a']) A[g, i, j, g'] X[b, j, b'] psi[a', g', b']
template <class R>
int psi_prev(qtt_ctx* c, const Buf<R>& psi, const OpCore& A, const cplx<R>* X, int rx, const Buf<R>& Y,
             Buf<R>* out) {
  const int64_t ry1 = psi.d0, ra1 = psi.d1, rx1 = psi.d2, n = A.n, m = A.m, ra = A.g0, ry = Y.d0;
  DBuf S1, S2;
  TRY(S1.alloc(c, (size_t)rx * n * ry1 * ra1 * sizeof(cplx<R>)));
  GemmDesc g1 = desc(rx * n, ry1 * ra1, rx1, 1, B0(), L1(rx * n, rx1), L1(rx1, 1), 0, B0(), L1(rx1, 1),
                     L1(ry1 * ra1, rx1), B0(), L1(rx * n, ry1 * ra1), L1(ry1 * ra1, 1));
  TRY(gemm_ab<R>(c, g1, cplx<R>(1, 0), cplx<R>(0, 0), X, psi.p(), S1.as<cplx<R>>()));
  TRY(S2.alloc(c, (size_t)rx * ra * m * ry1 * sizeof(cplx<R>)));
  GemmDesc g2 = desc(ra * m, ry1, n * ra1, rx, B0(), L1(ra * m, n * ra1), L1(n * ra1, 1), 0,
                     L1(rx, n * ry1 * ra1), L2(n, ry1 * ra1, ra1, 1), L1(ry1, ra1), L1(rx, ra * m * ry1),
                     L1(ra * m, ry1), L1(ry1, 1));
  TRY(gemm_ab<R>(c, g2, cplx<R>(1, 0), cplx<R>(0, 0), reinterpret_cast<const cplx<R>*>(A.p), S1.as<cplx<R>>(),
                 S2.as<cplx<R>>()));
  TRY(out->make(c, (int)ry, (int)ra, rx));
  GemmDesc g3 = desc(ry, ra * rx, m * ry1, 1, B0(), L1(ry, m * ry1), L1(m * ry1, 1), 1, B0(), L1(m * ry1, 1),
                     L2(ra, m * ry1, rx, ra * m * ry1), B0(), L1(ry, ra * rx), L1(ra * rx, 1));
  return gemm_ab<R>(c, g3, cplx<R>(1, 0), cplx<R>(0, 0), Y.p(), S2.as<cplx<R>>(), out->p());
}

// [c', a'] = sum conj(Z[c, i, c']) phi[c, a] Y[a, i, a']   (phi: rz x ry stored in d0 x d1)
template <class R>
int phi_zy_next(qtt_ctx* c, const Buf<R>& phi, const Buf<R>& Z, const Buf<R>& Y, Buf<R>* out) {
  const int64_t rz = Z.d0, m = Z.d1, rz1 = Z.d2, ry = Y.d0, ry1 = Y.d2;
  DBuf W;
  TRY(W.alloc(c, (size_t)rz * m * ry1 * sizeof(cplx<R>)));
  TRY(mmr<R>(c, rz, m * ry1, ry, phi.p(), ry, 0, Y.p(), m * ry1, W.as<cplx<R>>()));
  TRY(out->make(c, (int)rz1, (int)ry1, 1));
  return mmh<R>(c, rz1, ry1, rz * m, Z.p(), rz1, W.as<cplx<R>>(), ry1, out->p());
}

// [c, a] = sum conj(Z[c, i, c']) Y[a, i, a'] psi[c', a']
template <class R>
int psi_zy_prev(qtt_ctx* c, const Buf<R>& psi, const Buf<R>& Z, const Buf<R>& Y, Buf<R>* out) {
  const int64_t rz = Z.d0, m = Z.d1, rz1 = Z.d2, ry = Y.d0, ry1 = Y.d2;
  DBuf W;
  TRY(W.alloc(c, (size_t)ry * m * rz1 * sizeof(cplx<R>)));
  GemmDesc g1 = desc(ry * m, rz1, ry1, 1, B0(), L1(ry * m, ry1), L1(ry1, 1), 0, B0(), L1(ry1, 1), L1(rz1, ry1),
                     B0(), L1(ry * m, rz1), L1(rz1, 1));
  TRY(gemm_ab<R>(c, g1, cplx<R>(1, 0), cplx<R>(0, 0), Y.p(), psi.p(), W.as<cplx<R>>()));
  TRY(out->make(c, (int)rz, (int)ry, 1));
  GemmDesc g2 = desc(rz, ry, m * rz1, 1, B0(), L1(rz, m * rz1), L1(m * rz1, 1), 1, B0(), L1(m * rz1, 1),
                     L1(ry, m * rz1), B0(), L1(rz, ry), L1(ry, 1));
  return gemm_ab<R>(c, g2, cplx<R>(1, 0), cplx<R>(0, 0), Z.p(), W.as<cplx<R>>(), out->p());
}

template <class R>
int sumsq_host(qtt_ctx* c, const cplx<R>* p, int64_t n, DBuf& scal, double* out) {
  c->launches++;
  TRY(qtt_sumsq<R>(p, n, scal.as<double>(), c->stream));
  return sync_read(c, out, scal.p, sizeof(double));
}

// Orthonormal basis of the columns of A (rows x cols, row-major): the left
// singular vectors whose discarded tail is at most delta (all if delta < 0),
// at most max_rank (0: no cap).  Q: rows x t.
template <class R>
int col_basis(qtt_ctx* c, const cplx<R>* A, int64_t rows, int64_t cols, double delta, int max_rank, DBuf& scal,
              DBuf* Q, int* t_out) {
  const int64_t p = std::min(rows, cols);
  DBuf U, sig;
  TRY(U.alloc(c, (size_t)rows * p * sizeof(cplx<R>)));
  TRY(sig.alloc(c, (size_t)p * sizeof(R)));
  int64_t nsv = 0;
  TRY(left_svd<R>(c, A, rows, cols, cols, U.as<cplx<R>>(), sig.as<R>(), &nsv));
  int* dint = reinterpret_cast<int*>(scal.as<double>() + 4);
  c->launches++;
  TRY(qtt_trunc_rank<R>(sig.as<R>(), (int)nsv, delta, max_rank, dint, scal.as<double>() + 1, c->stream));
  int t = 0;
  TRY(sync_read(c, &t, dint, sizeof(int)));
  t = std::max(1, t);
  TRY(Q->alloc(c, (size_t)rows * t * sizeof(cplx<R>)));
  c->launches++;
  TRY(qtt_copy_strided<R>(U.as<cplx<R>>(), L1(rows, nsv), L1(t, 1), rows, t, 0, Q->as<cplx<R>>(), t, c->stream));
  *t_out = t;
  return QTT_OK;
}

// Right-orthogonalise a train held as cores (all but core 0 get orthonormal rows).
template <class R>
int right_orth(qtt_ctx* c, std::vector<Buf<R>>& y, DBuf& scal) {
  const double u = sizeof(R) == 8 ? DBL_EPSILON : FLT_EPSILON;
  for (int k = (int)y.size() - 1; k >= 1; --k) {
    Buf<R>& Y = y[k];
    const int64_t r0 = Y.d0, n = Y.d1, r1 = Y.d2;
    // M^H ((n r1) x r0), materialised
    DBuf MH;
    TRY(MH.alloc(c, (size_t)n * r1 * r0 * sizeof(cplx<R>)));
    c->launches++;
    TRY(qtt_copy_strided<R>(Y.p(), L1(n * r1, 1), L1(r0, n * r1), n * r1, r0, 1, MH.as<cplx<R>>(), r0, c->stream));
    double n2 = 0;
    TRY(sumsq_host<R>(c, Y.p(), Y.size(), scal, &n2));
    DBuf Q;
    int t = 0;
    TRY(col_basis<R>(c, MH.as<cplx<R>>(), n * r1, r0, 100.0 * u * sqrt(n2), 0, scal, &Q, &t));
    // carry = M Q (r0 x t); core k = Q^H as (t, n, r1)
    DBuf carry;
    TRY(carry.alloc(c, (size_t)r0 * t * sizeof(cplx<R>)));
    TRY(mmr<R>(c, r0, t, n * r1, Y.p(), n * r1, 0, Q.as<cplx<R>>(), t, carry.as<cplx<R>>()));
    Buf<R> nk;
    TRY(nk.make(c, t, (int)n, (int)r1));
    c->launches++;
    TRY(qtt_copy_strided<R>(Q.as<cplx<R>>(), L1(t, 1), L1(n * r1, t), t, n * r1, 1, nk.p(), n * r1, c->stream));
    Buf<R>& P = y[k - 1];
    Buf<R> np;
    TRY(np.make(c, P.d0, P.d1, t));
    TRY(mmr<R>(c, (int64_t)P.d0 * P.d1, t, r0, P.p(), r0, 0, carry.as<cplx<R>>(), t, np.p()));
    y[k] = std::move(nk);
    y[k - 1] = std::move(np);
  }
  return QTT_OK;
}

template <class R>
int gauss_train(qtt_ctx* c, const std::vector<int>& modes, int r, uint64_t seed, uint64_t stream0,
                std::vector<Buf<R>>* out) {
  const int d = (int)modes.size();
  out->clear();
  out->resize(d);
  for (int k = 0; k < d; ++k) {
    const int r0 = k == 0 ? 1 : r, r1 = k == d - 1 ? 1 : r;
    TRY((*out)[k].make(c, r0, modes[k], r1));
    c->launches++;
    TRY(qtt_fill_gaussian<R>((*out)[k].p(), (*out)[k].size(), seed, stream0 + k, 1.0, c->stream));
  }
  return QTT_OK;
}

}  // namespace

template <class R>
int amen_mv_dev(qtt_ctx* c, const qtt_mpo* A, const qtt_tt* x, const qtt_tt* y0, double eps, int kick,
                int max_sweeps, uint64_t seed, int max_rank, qtt_tt** yout, int* sweeps_out, double* dx_out) {
  typedef cplx<R> C;
  const int d = x->d;
  const double u = sizeof(R) == 8 ? DBL_EPSILON : FLT_EPSILON;
  std::vector<OpCore> Ak(d);
  std::vector<int> modes(d);
  for (int k = 0; k < d; ++k) {
    Ak[k] = OpCore{core_ptr<const char>(A, k), A->g[k], A->no[k], A->ni[k], A->g[k + 1]};
    modes[k] = A->no[k];
  }
  auto X = [&](int k) { return core_ptr<const C>(x, k); };
  DBuf scal;
  TRY(scal.alloc(c, 64));
  std::vector<Buf<R>> y(d), z;
  if (y0) {
    for (int k = 0; k < d; ++k) {
      TRY(y[k].make(c, y0->r[k], y0->n[k], y0->r[k + 1]));
      if (cudaMemcpyAsync(y[k].p(), core_ptr<const C>(y0, k), y[k].size() * sizeof(C), cudaMemcpyDeviceToDevice,
                          c->stream) != cudaSuccess)
        return QTT_ERR_CUDA;
    }
  } else {
    TRY(gauss_train<R>(c, modes, 4, seed, 1u << 20, &y));
  }
  TRY(gauss_train<R>(c, modes, std::max(kick, 1), seed, 2u << 20, &z));
  Buf<R> one3, one2;
  {
    TRY(one3.make(c, 1, 1, 1));
    TRY(one2.make(c, 1, 1, 1));
    const C o(1, 0);
    if (cudaMemcpyAsync(one3.p(), &o, sizeof(C), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(one2.p(), &o, sizeof(C), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return QTT_ERR_CUDA;
    cudaStreamSynchronize(c->stream);   // the host sources above are stack values
  }
  const double sq = sqrt((double)std::max(d - 1, 1));
  double dx = INFINITY;
  int sweep = 0;
  uint64_t zs = 3u << 20;
  for (sweep = 1; sweep <= max_sweeps; ++sweep) {
    TRY(right_orth<R>(c, y, scal));
    TRY(right_orth<R>(c, z, scal));
    std::vector<Buf<R>> psi(d + 1), psiz(d + 1), psizy(d + 1);
    auto set_one = [&](Buf<R>& b, const Buf<R>& src) -> int {
      TRY(b.make(c, 1, 1, 1));
      return cudaMemcpyAsync(b.p(), src.p(), sizeof(C), cudaMemcpyDeviceToDevice, c->stream) == cudaSuccess
                 ? QTT_OK
                 : QTT_ERR_CUDA;
    };
    TRY(set_one(psi[d], one3));
    TRY(set_one(psiz[d], one3));
    TRY(set_one(psizy[d], one2));
    for (int k = d - 1; k >= 1; --k) {
      TRY(psi_prev<R>(c, psi[k + 1], Ak[k], X(k), x->r[k], y[k], &psi[k]));
      TRY(psi_prev<R>(c, psiz[k + 1], Ak[k], X(k), x->r[k], z[k], &psiz[k]));
      TRY(psi_zy_prev<R>(c, psizy[k + 1], z[k], y[k], &psizy[k]));
    }
    Buf<R> phi, phiz, phizy;
    TRY(set_one(phi, one3));
    TRY(set_one(phiz, one3));
    TRY(set_one(phizy, one2));
    dx = 0.0;
    for (int k = 0; k < d; ++k) {
      Buf<R> Yn;
      TRY(proj<R>(c, phi, Ak[k], X(k), x->r[k + 1], psi[k + 1], &Yn));
      double n2 = 0, dd = 0;
      TRY(sumsq_host<R>(c, Yn.p(), Yn.size(), scal, &n2));
      if (y[k].d0 == Yn.d0 && y[k].d1 == Yn.d1 && y[k].d2 == Yn.d2) {
        DBuf D;
        TRY(D.alloc(c, (size_t)Yn.size() * sizeof(C)));
        TRY(axpby<R>(c, Yn.p(), y[k].p(), Yn.size(), R(1), R(-1), D.as<C>()));
        TRY(sumsq_host<R>(c, D.as<C>(), Yn.size(), scal, &dd));
        if (n2 > 0) dx = std::max(dx, sqrt(dd / n2));
      } else {
        dx = INFINITY;
      }
      if (k == d - 1) {
        y[k] = std::move(Yn);
        break;
      }
      const int64_t r0 = Yn.d0, m = Yn.d1, r1 = Yn.d2;
      // truncation of the new core
      DBuf Ut;
      int t = 0;
      TRY(col_basis<R>(c, Yn.p(), r0 * m, r1, eps * sqrt(n2) / sq, max_rank, scal, &Ut, &t));
      DBuf Rt, Ycur;
      TRY(Rt.alloc(c, (size_t)t * r1 * sizeof(C)));
      TRY(mmh<R>(c, t, r1, r0 * m, Ut.as<C>(), t, Yn.p(), r1, Rt.as<C>()));
      TRY(Ycur.alloc(c, (size_t)r0 * m * r1 * sizeof(C)));
      TRY(mmr<R>(c, r0 * m, r1, t, Ut.as<C>(), t, 0, Rt.as<C>(), r1, Ycur.as<C>()));
      Buf<R> Yc;   // Ycur with its shape, for the z^H y interfaces
      Yc.b = std::move(Ycur);
      Yc.d0 = (int)r0;
      Yc.d1 = (int)m;
      Yc.d2 = (int)r1;
      // residual core of z: projection on z's interfaces minus phi^zy Ycur psi^zy
      Buf<R> Zk;
      TRY(proj<R>(c, phiz, Ak[k], X(k), x->r[k + 1], psiz[k + 1], &Zk));
      {
        const int64_t rz = phizy.d0, rz1 = psizy[k + 1].d0;
        DBuf W;
        TRY(W.alloc(c, (size_t)rz * m * r1 * sizeof(C)));
        TRY(mmr<R>(c, rz, m * r1, r0, phizy.p(), r0, 0, Yc.p(), m * r1, W.as<C>()));
        GemmDesc g = desc(rz * m, rz1, r1, 1, B0(), L1(rz * m, r1), L1(r1, 1), 0, B0(), L1(r1, 1), L1(rz1, r1),
                          B0(), L1(rz * m, rz1), L1(rz1, 1));
        TRY(gemm_ab<R>(c, g, C(-1, 0), C(1, 0), W.as<C>(), psizy[k + 1].p(), Zk.p()));
      }
      {
        double z2 = 0;
        TRY(sumsq_host<R>(c, Zk.p(), Zk.size(), scal, &z2));
        if (!(z2 > 0)) {   // exact so far: random directions keep z full rank
          c->launches++;
          TRY(qtt_fill_gaussian<R>(Zk.p(), Zk.size(), seed, zs++, 1.0, c->stream));
        }
        DBuf Qz;
        int kz = 0;
        TRY(col_basis<R>(c, Zk.p(), (int64_t)Zk.d0 * Zk.d1, Zk.d2, -1.0, std::max(kick, 1), scal, &Qz, &kz));
        Buf<R> nz;
        nz.b = std::move(Qz);
        nz.d0 = Zk.d0;
        nz.d1 = Zk.d1;
        nz.d2 = kz;
        z[k] = std::move(nz);
        if (z[k + 1].d0 != kz) {
          // only the shape of core k+1 matters (it is recomputed next)
          Buf<R> nn;
          TRY(nn.make(c, kz, z[k + 1].d1, z[k + 1].d2));
          c->launches++;
          TRY(qtt_fill_gaussian<R>(nn.p(), nn.size(), seed, zs++, 1.0, c->stream));
          z[k + 1] = std::move(nn);
        }
      }
      // enrichment: projection on y's left and z's right interface minus Ycur psi^zy
      Buf<R> Ek;
      TRY(proj<R>(c, phi, Ak[k], X(k), x->r[k + 1], psiz[k + 1], &Ek));
      {
        const int64_t rz1 = psizy[k + 1].d0;
        GemmDesc g = desc(r0 * m, rz1, r1, 1, B0(), L1(r0 * m, r1), L1(r1, 1), 0, B0(), L1(r1, 1), L1(rz1, r1),
                          B0(), L1(r0 * m, rz1), L1(rz1, 1));
        TRY(gemm_ab<R>(c, g, C(-1, 0), C(1, 0), Yc.p(), psizy[k + 1].p(), Ek.p()));
      }
      const int64_t ez = Ek.d2, wa = t + ez;
      DBuf Uaug;
      TRY(Uaug.alloc(c, (size_t)r0 * m * wa * sizeof(C)));
      c->launches += 2;
      TRY(qtt_copy_strided<R>(Ut.as<C>(), L1(r0 * m, t), L1(t, 1), r0 * m, t, 0, Uaug.as<C>(), wa, c->stream));
      TRY(qtt_copy_strided<R>(Ek.p(), L1(r0 * m, ez), L1(ez, 1), r0 * m, ez, 0, Uaug.as<C>() + t, wa, c->stream));
      double a2 = 0;
      TRY(sumsq_host<R>(c, Uaug.as<C>(), r0 * m * wa, scal, &a2));
      DBuf Q;
      int keep = 0;
      TRY(col_basis<R>(c, Uaug.as<C>(), r0 * m, wa, 100.0 * u * sqrt(a2), 0, scal, &Q, &keep));
      // carry = Q^H Ycur (keep x r1), core k+1 <- carry core k+1
      DBuf carry;
      TRY(carry.alloc(c, (size_t)keep * r1 * sizeof(C)));
      TRY(mmh<R>(c, keep, r1, r0 * m, Q.as<C>(), keep, Yc.p(), r1, carry.as<C>()));
      Buf<R> nextc;
      TRY(nextc.make(c, keep, y[k + 1].d1, y[k + 1].d2));
      TRY(mmr<R>(c, keep, (int64_t)y[k + 1].d1 * y[k + 1].d2, r1, carry.as<C>(), r1, 0, y[k + 1].p(),
                 (int64_t)y[k + 1].d1 * y[k + 1].d2, nextc.p()));
      Buf<R> yk;
      yk.b = std::move(Q);
      yk.d0 = (int)r0;
      yk.d1 = (int)m;
      yk.d2 = keep;
      y[k] = std::move(yk);
      y[k + 1] = std::move(nextc);
      Buf<R> phin, phizn, phizyn;
      TRY(phi_next<R>(c, phi, Ak[k], X(k), x->r[k + 1], y[k], &phin));
      TRY(phi_next<R>(c, phiz, Ak[k], X(k), x->r[k + 1], z[k], &phizn));
      TRY(phi_zy_next<R>(c, phizy, z[k], y[k], &phizyn));
      phi = std::move(phin);
      phiz = std::move(phizn);
      phizy = std::move(phizyn);
    }
    if (dx <= eps) break;
  }
  // assemble and round
  std::vector<int> r(d + 1, 1);
  for (int k = 0; k < d; ++k) r[k + 1] = y[k].d2;
  r[d] = 1;
  int st = 0;
  qtt_tt* yt = tt_alloc(c, d, modes, r, x->dtype, &st);
  if (!yt) return st;
  for (int k = 0; k < d; ++k)
    cudaMemcpyAsync(core_ptr<char>(yt, k), y[k].p(), (size_t)y[k].size() * sizeof(C), cudaMemcpyDeviceToDevice,
                    c->stream);
  qtt_round_info ri;
  st = round_det<R>(c, yt, eps, max_rank, nullptr, &ri, yout);
  tt_free(yt);
  if (sweeps_out) *sweeps_out = std::min(sweep, max_sweeps);
  if (dx_out) *dx_out = dx;
  return st;
}

template int amen_mv_dev<double>(qtt_ctx*, const qtt_mpo*, const qtt_tt*, const qtt_tt*, double, int, int, uint64_t,
                                 int, qtt_tt**, int*, double*);
template int amen_mv_dev<float>(qtt_ctx*, const qtt_mpo*, const qtt_tt*, const qtt_tt*, double, int, int, uint64_t,
                                int, qtt_tt**, int*, double*);
