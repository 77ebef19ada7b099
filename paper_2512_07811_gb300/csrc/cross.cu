// TT-cross on the device (Sec. 3, operator setup: the cores of the phase and
// Green operator trains are separated by the TT-cross approximation of
// Oseledets & Tyrtyshnikov, here in its rank-adaptive two-site form): the
// superblock sampler, the maximum-volume row selection and the index-set
// bookkeeping.  The sweep itself is driven from the host (capi.cu).
#include <limits.h>

#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "engine.h"
#include "kernels.h"

namespace {

constexpr int TPB = 256;

inline unsigned nblocks(int64_t count) {
  int64_t b = (count + TPB - 1) / TPB;
  if (b > (int64_t)1 << 20) b = (int64_t)1 << 20;
  return (unsigned)(b < 1 ? 1 : b);
}

#define TRYK(e)                      \
  do {                               \
    int _s = (e);                    \
    if (_s != QTT_OK) return _s;     \
  } while (0)
#define CHECK_LAUNCH() return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA

// Coordinates of one multi-index, accumulated site by site.
struct CrossAcc {
  int ctrl;
  int64_t v[3];
};

__device__ __forceinline__ void cross_put(const CrossFn& f, int site, int val, CrossAcc& a) {
  if (f.kind == CROSS_GREEN) {
    if (site == 0) {
      a.ctrl = val;
      return;
    }
    const int p = site - 1;
    a.v[f.m.dim[p]] |= (int64_t)val << f.m.pos[p];
  } else {
    const int dm = f.m.dim[site];
    a.v[dm] |= (int64_t)val << (f.m.nb[dm] - 1 - f.m.pos[site]);
  }
}

__device__ double cross_value(const CrossFn& f, const CrossAcc& a) {
  if (f.kind == CROSS_GREEN) {
    double xi[3];
    for (int d = 0; d < 3; ++d) {
      const int64_t N = (int64_t)1 << f.m.nb[d];
      xi[d] = (double)(a.v[d] < (N + 1) / 2 ? a.v[d] : a.v[d] - N);
    }
    return green_entry(xi, a.ctrl / f.ncomp, a.ctrl % f.ncomp, f.ncomp, f.k0, f.lam0, f.mu0);
  }
  double c[3];
  for (int d = 0; d < 3; ++d) c[d] = ((double)a.v[d] + 0.5) / (double)((int64_t)1 << f.m.nb[d]);
  if (f.kind == CROSS_ELLIPSOIDS) {
    for (int e = 0; e < f.nells; ++e) {
      const double* E = f.ells + 15 * e;
      double D[3];
      for (int d = 0; d < 3; ++d) {
        const double t = __dsub_rn(c[d], E[d]);
        D[d] = __dsub_rn(t, rint(t));   // round half to even, as the host voxelisation
      }
      double q = 0.0;
      for (int i = 0; i < 3; ++i) {
        double u = __dadd_rn(__dmul_rn(E[6 + i], D[0]), __dmul_rn(E[9 + i], D[1]));
        u = __dadd_rn(u, __dmul_rn(E[12 + i], D[2]));
        const double t = __ddiv_rn(u, E[3 + i]);
        q = i == 0 ? __dmul_rn(t, t) : __dadd_rn(q, __dmul_rn(t, t));
      }
      if (q <= 1.0) return 1.0;
    }
    return 0.0;
  }
  for (int b = 0; b < f.nboxes; ++b) {
    const double* B = f.boxes + 6 * b;
    bool in = true;
    for (int d = 0; d < 3 && in; ++d) {
      // (c - centre + 1/2) mod 1, the result taking the sign of the divisor
      double t = fmod(c[d] - B[d] + 0.5, 1.0);
      if (t < 0) t += 1.0;
      in = fabs(t - 0.5) <= B[3 + d];
    }
    if (in) return 1.0;
  }
  return 0.0;
}

// S[(a, i), (j, b)] = f(Il[a], i, j, Jr[b]) for the bond between sites k and
// k+1: Il holds rl left rows of k site values, Jr rr right rows of d-k-2
// values.  Row-major (rl n0) x (n1 rr), or its conjugate transpose (herm).
// With k + 1 == d (a one-site train) n1 = rr = 1 and no second site.
template <class R>
__global__ void cross_eval_kernel(CrossFn f, int d, int k, const uint8_t* __restrict__ Il, int rl,
                                  const uint8_t* __restrict__ Jr, int rr, int n0, int n1, int herm,
                                  cplx<R>* __restrict__ out) {
  const int64_t total = (int64_t)rl * n0 * n1 * rr;
  const int nr = d - k - 2;
  const int64_t rows = (int64_t)rl * n0, cols = (int64_t)n1 * rr;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = e;
    const int b = (int)(t % rr);
    t /= rr;
    const int j = (int)(t % n1);
    t /= n1;
    const int i = (int)(t % n0);
    const int a = (int)(t / n0);
    CrossAcc acc{0, {0, 0, 0}};
    for (int s = 0; s < k; ++s) cross_put(f, s, Il[(int64_t)a * k + s], acc);
    cross_put(f, k, i, acc);
    if (k + 1 < d) cross_put(f, k + 1, j, acc);
    for (int s = 0; s < nr; ++s) cross_put(f, k + 2 + s, Jr[(int64_t)b * nr + s], acc);
    const cplx<R> v((R)cross_value(f, acc), R(0));
    const int64_t row = (int64_t)a * n0 + i, col = (int64_t)j * rr + b;
    if (herm)
      out[col * rows + row] = v;   // the values are real: conjugation is a no-op
    else
      out[row * cols + col] = v;
  }
}

// Block-wide argmax of (value, index) pairs: the largest value, ties to the
// smallest index.  Every thread receives the result.
__device__ void block_argmax(double v, long long idx, double* sv, long long* si, double* out_v, long long* out_i) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, o);
    const long long oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
  if (lane == 0) {
    sv[w] = v;
    si[w] = idx;
  }
  __syncthreads();
  if (w == 0) {
    v = lane < nw ? sv[lane] : -1.0;
    idx = lane < nw ? si[lane] : LLONG_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, v, o);
      const long long oi = __shfl_down_sync(0xffffffffu, idx, o);
      if (ov > v || (ov == v && oi < idx)) {
        v = ov;
        idx = oi;
      }
    }
    if (lane == 0) {
      sv[32] = v;
      si[32] = idx;
    }
  }
  __syncthreads();
  *out_v = sv[32];
  *out_i = si[32];
  __syncthreads();
}

// Maximum-volume rows of the tall A (m x r, row-major, full column rank), in
// place, one CTA.  Phase 1: Gauss-Jordan elimination by column operations
// with partial pivoting over rows, which leaves A A[piv]^-1 (the pivot rows
// become unit rows).  Phase 2: while the largest |B_ij| of B = A A[piv]^-1
// exceeds sqrt(tol2), row i replaces piv[j] and B takes the rank-one update
// B -= B[:, j] (B[i, :] - e_j) / B[i, j] (Sherman-Morrison), at most
// max_iters times.  status: 1 if a pivot column was zero (rank deficient),
// else the number of swaps + 2 (so that 0 means "not run").
template <class R>
__global__ void __launch_bounds__(1024) maxvol_kernel(cplx<R>* __restrict__ A, int m, int r, int* __restrict__ piv,
                                                      double tol2, int max_iters, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char mv_smem[];
  cplx<R>* rowv = reinterpret_cast<cplx<R>*>(mv_smem);
  cplx<R>* colv = rowv + r;
  unsigned char* chosen = reinterpret_cast<unsigned char*>(colv + m);
  __shared__ double sv[33];
  __shared__ long long si[33];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t mr = (int64_t)m * r;
  for (int i = tid; i < m; i += nt) chosen[i] = 0;
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    double bv = -1.0;
    long long bi = LLONG_MAX;
    for (int i = tid; i < m; i += nt)
      if (!chosen[i]) {
        const double v = (double)abs2(A[(int64_t)i * r + j]);
        if (v > bv) {
          bv = v;
          bi = i;
        }
      }
    double best;
    long long bidx;
    block_argmax(bv, bi, sv, si, &best, &bidx);
    if (!(best > 0.0)) {
      if (tid == 0) *status = 1;
      return;
    }
    const int p = (int)bidx;
    for (int l = tid; l < r; l += nt) rowv[l] = A[(int64_t)p * r + l];
    if (tid == 0) {
      piv[j] = p;
      chosen[p] = 1;
    }
    __syncthreads();
    const cplx<R> pv = rowv[j];
    const R den = pv.re * pv.re + pv.im * pv.im;
    const cplx<R> inv(pv.re / den, -pv.im / den);
    for (int i = tid; i < m; i += nt) {
      const cplx<R> x = i == p ? cplx<R>(1, 0) : A[(int64_t)i * r + j] * inv;
      colv[i] = x;
      A[(int64_t)i * r + j] = x;
    }
    __syncthreads();
    for (int64_t e = tid; e < mr; e += nt) {
      const int i = (int)(e / r), l = (int)(e - (int64_t)i * r);
      if (l == j) continue;
      if (i == p) {
        A[e] = cplx<R>(0, 0);
      } else {
        cplx<R> x = A[e];
        cfma(x, -rowv[l], colv[i]);
        A[e] = x;
      }
    }
    __syncthreads();
  }
  int swaps = 0;
  for (int it = 0; it < max_iters; ++it) {
    double bv = -1.0;
    long long bi = LLONG_MAX;
    for (int64_t e = tid; e < mr; e += nt) {
      const double v = (double)abs2(A[e]);
      if (v > bv) {
        bv = v;
        bi = e;
      }
    }
    double best;
    long long bidx;
    block_argmax(bv, bi, sv, si, &best, &bidx);
    if (!(best > tol2)) break;
    const int i = (int)(bidx / r), j = (int)(bidx - (long long)i * r);
    for (int l = tid; l < r; l += nt) {
      cplx<R> x = A[(int64_t)i * r + l];
      if (l == j) x.re -= R(1);
      rowv[l] = x;
    }
    for (int q = tid; q < m; q += nt) colv[q] = A[(int64_t)q * r + j];
    __syncthreads();
    const cplx<R> pv = colv[i];
    const R den = pv.re * pv.re + pv.im * pv.im;
    const cplx<R> inv(pv.re / den, -pv.im / den);
    for (int64_t e = tid; e < mr; e += nt) {
      const int q = (int)(e / r), l = (int)(e - (int64_t)q * r);
      cplx<R> x = A[e];
      cfma(x, -(colv[q] * inv), rowv[l]);
      A[e] = x;
    }
    if (tid == 0) piv[j] = i;
    ++swaps;
    __syncthreads();
  }
  if (tid == 0) *status = 2 + swaps;
}

// New left rows: row a extends Iprev[piv[a] / n0] (k values) by piv[a] % n0.
__global__ void cross_left_index_kernel(const uint8_t* __restrict__ Iprev, int k, int n0, const int* __restrict__ piv,
                                        int t, uint8_t* __restrict__ Inew) {
  const int w = k + 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)t * w;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / w), s = (int)(e - (int64_t)a * w);
    const int p = piv[a];
    Inew[e] = s < k ? Iprev[(int64_t)(p / n0) * k + s] : (uint8_t)(p % n0);
  }
}

// New right rows: row a is piv[a] / rr followed by Jnext[piv[a] % rr] (nr values).
__global__ void cross_right_index_kernel(const uint8_t* __restrict__ Jnext, int nr, int rr,
                                         const int* __restrict__ piv, int t, uint8_t* __restrict__ Jnew) {
  const int w = nr + 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)t * w;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / w), s = (int)(e - (int64_t)a * w);
    const int c = piv[a];
    Jnew[e] = s == 0 ? (uint8_t)(c / rr) : Jnext[(int64_t)(c % rr) * nr + s - 1];
  }
}

// Rows piv of S (ld columns, len copied): out[a, c] = S[piv[a], c], or the
// conjugate transpose out[c, a] = conj(S[piv[a], c]).
template <class R>
__global__ void cross_gather_kernel(const cplx<R>* __restrict__ S, int64_t ld, const int* __restrict__ piv, int t,
                                    int64_t len, int trans, cplx<R>* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)t * len;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / len);
    const int64_t c = e - (int64_t)a * len;
    const cplx<R> v = S[(int64_t)piv[a] * ld + c];
    if (trans)
      out[c * t + a] = conjg(v);
    else
      out[e] = v;
  }
}

}  // namespace

template <class R>
int qtt_cross_eval(const CrossFn& f, int d, int k, const uint8_t* Il, int rl, const uint8_t* Jr, int rr, int n0,
                   int n1, int herm, cplx<R>* out, cudaStream_t s) {
  const int64_t total = (int64_t)rl * n0 * n1 * rr;
  if (total <= 0) return QTT_OK;
  cross_eval_kernel<R><<<nblocks(total), TPB, 0, s>>>(f, d, k, Il, rl, Jr, rr, n0, n1, herm, out);
  CHECK_LAUNCH();
}

template <class R>
size_t qtt_maxvol_smem(int m, int r) {
  return (size_t)(m + r) * sizeof(cplx<R>) + (size_t)m + 16;
}

template <class R>
int qtt_maxvol(cplx<R>* A, int m, int r, int* piv, double tol, int max_iters, int* status, cudaStream_t s) {
  if (r < 1 || m < r) return QTT_ERR_ARG;
  const size_t smem = qtt_maxvol_smem<R>(m, r);
  if (smem > 200 * 1024) return QTT_ERR_UNSUPPORTED;
  if (smem > 48 * 1024) TRYK(qtt_allow_max_smem((const void*)maxvol_kernel<R>));
  maxvol_kernel<R><<<1, 1024, smem, s>>>(A, m, r, piv, tol * tol, max_iters, status);
  CHECK_LAUNCH();
}

int qtt_cross_left_index(const uint8_t* Iprev, int k, int n0, const int* piv, int t, uint8_t* Inew, cudaStream_t s) {
  const int64_t total = (int64_t)t * (k + 1);
  if (total <= 0) return QTT_OK;
  cross_left_index_kernel<<<nblocks(total), TPB, 0, s>>>(Iprev, k, n0, piv, t, Inew);
  CHECK_LAUNCH();
}

int qtt_cross_right_index(const uint8_t* Jnext, int nr, int rr, const int* piv, int t, uint8_t* Jnew, cudaStream_t s) {
  const int64_t total = (int64_t)t * (nr + 1);
  if (total <= 0) return QTT_OK;
  cross_right_index_kernel<<<nblocks(total), TPB, 0, s>>>(Jnext, nr, rr, piv, t, Jnew);
  CHECK_LAUNCH();
}

template <class R>
int qtt_cross_gather(const cplx<R>* S, int64_t ld, const int* piv, int t, int64_t len, int trans, cplx<R>* out,
                     cudaStream_t s) {
  const int64_t total = (int64_t)t * len;
  if (total <= 0) return QTT_OK;
  cross_gather_kernel<R><<<nblocks(total), TPB, 0, s>>>(S, ld, piv, t, len, trans, out);
  CHECK_LAUNCH();
}

template int qtt_cross_eval<double>(const CrossFn&, int, int, const uint8_t*, int, const uint8_t*, int, int, int, int,
                                    zc*, cudaStream_t);
template size_t qtt_maxvol_smem<double>(int, int);
template int qtt_maxvol<double>(zc*, int, int, int*, double, int, int*, cudaStream_t);
template int qtt_cross_gather<double>(const zc*, int64_t, const int*, int, int64_t, int, zc*, cudaStream_t);

#define TRY(expr)                  \
  do {                             \
    int _st = (expr);              \
    if (_st != QTT_OK) return _st; \
  } while (0)

// ------------------------------------------------------------ TT-cross
// Rank-adaptive two-site TT-cross (Sec. 3 operator setup; Oseledets &
// Tyrtyshnikov, two-site form of Savostyanov & Oseledets).  Index sets live
// on the device as byte rows: I[k] holds rI[k] left rows of k site values
// (sites 0..k-1), J[k] holds rJ[k] right rows of d-k values (sites k..d-1).
// A forward half-sweep samples at bond k (sites k, k+1) the superblock
// S = f(I[k], i, j, J[k+2]), keeps the leading left singular vectors whose
// tail is at most eps ||S|| / sqrt(d-1), appends `kick` Gaussian columns,
// picks their maximum-volume rows, which give I[k+1] and the interpolation
// core A A[rows]^-1; at the last bond core d-1 is S[rows, :].  A backward
// half-sweep does the same on S^H, giving J[k+1], the cores
// (A A[rows]^-1)^H and at bond 0 core 0 = S[:, rows].
static uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Site values (position convention) of the voxel holding each box (or
// ellipsoid) centre: starting points inside the phase-2 region, which random
// points may miss.  Rows of `stride` values, the centre first.
std::vector<std::vector<uint8_t>> centre_seeds(const SiteMap& m, const double* rows, int nrows, int stride) {
  std::vector<std::vector<uint8_t>> out;
  for (int b = 0; b < nrows; ++b) {
    int64_t x[3];
    for (int a = 0; a < 3; ++a) {
      const int64_t N = (int64_t)1 << m.nb[a];
      double cf = rows[stride * b + a] - floor(rows[stride * b + a]);
      x[a] = std::min<int64_t>((int64_t)(cf * (double)N), N - 1);
    }
    std::vector<uint8_t> p(m.d);
    for (int q = 0; q < m.d; ++q) p[q] = (uint8_t)((x[m.dim[q]] >> (m.nb[m.dim[q]] - 1 - m.pos[q])) & 1);
    out.push_back(p);
  }
  return out;
}

static int cross_dev(qtt_ctx* c, const CrossFn& f, const std::vector<int>& modes, double eps, int max_rank, int kick,
              int max_half_sweeps, uint64_t seed, const std::vector<std::vector<uint8_t>>& seeds, qtt_tt** out,
              CrossOut* st) {
  const int d = (int)modes.size();
  for (int k = 0; k < d; ++k)
    if (modes[k] < 1 || modes[k] > 255) return QTT_ERR_ARG;
  int s = 0;
  if (d == 1) {
    qtt_tt* y = tt_alloc(c, 1, modes, std::vector<int>{1, 1}, QTT_C128, &s);
    if (!y) return s;
    c->launches++;
    s = qtt_cross_eval<double>(f, 1, 0, nullptr, 1, nullptr, 1, modes[0], 1, 0, core_ptr<zc>(y, 0), c->stream);
    if (s) {
      tt_free(y);
      return s;
    }
    st->evaluations = modes[0];
    *out = y;
    return QTT_OK;
  }
  // initial right index sets: the suffixes of 8 random points and of the
  // caller's seed points, duplicates removed
  const int npts = 8;
  uint64_t rs = seed ^ 0x5DEECE66Dull;
  std::vector<std::vector<uint8_t>> pts(npts, std::vector<uint8_t>(d));
  for (auto& p : pts)
    for (int k = 0; k < d; ++k) p[k] = (uint8_t)(splitmix64(rs) % (uint64_t)modes[k]);
  for (const auto& p : seeds)
    if ((int)p.size() == d) pts.push_back(p);
  std::vector<DBuf> I(d + 1), J(d + 1);
  std::vector<int> rI(d + 1, 1), rJ(d + 1, 1);
  for (int k = 1; k < d; ++k) {
    std::vector<std::vector<uint8_t>> rows;
    for (auto& p : pts) rows.emplace_back(p.begin() + k, p.end());
    std::sort(rows.begin(), rows.end());
    rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
    std::vector<uint8_t> flat;
    for (auto& r : rows) flat.insert(flat.end(), r.begin(), r.end());
    TRY(J[k].alloc(c, flat.size()));
    TRY(upload(c, J[k].p, flat.data(), flat.size()));
    rJ[k] = (int)rows.size();
  }
  DBuf scal, pivb, Zb;
  TRY(scal.alloc(c, 64));
  double* dscal = scal.as<double>();
  int* dint = reinterpret_cast<int*>(dscal + 4);
  std::vector<DBuf> cores(d);
  struct Held {
    qtt_tt* p = nullptr;
    ~Held() {
      if (p) tt_free(p);
    }
  } held;   // the train of the previous half-sweep
  qtt_tt*& prev = held.p;
  uint64_t gauss_stream = 1;
  const double sq = sqrt((double)(d - 1));
  int h = 0;
  double rel = INFINITY;
  for (h = 1; h <= std::max(2, max_half_sweeps); ++h) {
    const bool fwd = (h & 1) == 1;
    for (int step = 0; step < d - 1; ++step) {
      const int k = fwd ? step : d - 2 - step;
      const int rl = rI[k], rr = rJ[k + 2], n0 = modes[k], n1 = modes[k + 1];
      const int64_t rows = (int64_t)rl * n0, cols = (int64_t)n1 * rr;
      DBuf S;
      TRY(S.alloc(c, (size_t)rows * cols * sizeof(zc)));
      c->launches++;
      TRY(qtt_cross_eval<double>(f, d, k, I[k].as<uint8_t>(), rl, J[k + 2].as<uint8_t>(), rr, n0, n1, fwd ? 0 : 1,
                                 S.as<zc>(), c->stream));
      st->evaluations += rows * cols;
      // basis side: rows of S (forward) or of S^H (backward)
      const int64_t M = fwd ? rows : cols, Nn = fwd ? cols : rows;
      c->launches++;
      TRY(qtt_sumsq<double>(S.as<zc>(), rows * cols, dscal, c->stream));
      double n2 = 0;
      TRY(sync_read(c, &n2, dscal, sizeof(double)));
      int t = 0;
      DBuf U, sig;
      int64_t nsv = 0;
      if (n2 > 0) {
        const int64_t p = std::min(M, Nn);
        TRY(U.alloc(c, (size_t)M * p * sizeof(zc)));
        TRY(sig.alloc(c, (size_t)p * sizeof(double)));
        TRY(left_svd<double>(c, S.as<zc>(), M, Nn, Nn, U.as<zc>(), sig.as<double>(), &nsv));
        c->launches++;
        TRY(qtt_trunc_rank<double>(sig.as<double>(), (int)nsv, eps * sqrt(n2) / sq, max_rank, dint,
                                   dscal + 1, c->stream));
        TRY(sync_read(c, &t, dint, sizeof(int)));
      }
      // a zero superblock keeps only random directions (exploration)
      const int tk = (int)std::min<int64_t>(std::max(t + kick, 1), M);
      DBuf A;
      TRY(A.alloc(c, (size_t)M * tk * sizeof(zc)));
      if (t > 0) {
        c->launches++;
        TRY(qtt_copy_strided<double>(U.as<zc>(), MIdx{M, 1, nsv, 0}, MIdx{t, 1, 1, 0}, M, t, 0, A.as<zc>(), tk,
                                     c->stream));
      }
      if (tk > t) {
        const int e = tk - t;
        TRY(Zb.alloc(c, (size_t)M * e * sizeof(zc)));
        c->launches += 2;
        TRY(qtt_fill_gaussian<double>(Zb.as<zc>(), M * e, seed, gauss_stream++, 1.0, c->stream));
        TRY(qtt_copy_strided<double>(Zb.as<zc>(), MIdx{M, 1, e, 0}, MIdx{e, 1, 1, 0}, M, e, 0, A.as<zc>() + t, tk,
                                     c->stream));
      }
      TRY(pivb.alloc(c, (size_t)tk * sizeof(int)));
      cudaMemsetAsync(dint + 2, 0, sizeof(int), c->stream);
      c->launches++;
      TRY(qtt_maxvol<double>(A.as<zc>(), (int)M, tk, pivb.as<int>(), 1.05, 100, dint + 2, c->stream));
      int mvst = 0;
      TRY(sync_read(c, &mvst, dint + 2, sizeof(int)));
      if (mvst == 1) return QTT_ERR_RANK;
      if (mvst < 2) return QTT_ERR_CUDA;
      if (fwd) {
        cores[k] = std::move(A);
        DBuf In;
        TRY(In.alloc(c, (size_t)tk * (k + 1)));
        c->launches++;
        TRY(qtt_cross_left_index(I[k].as<uint8_t>(), k, n0, pivb.as<int>(), tk, In.as<uint8_t>(), c->stream));
        I[k + 1] = std::move(In);
        rI[k + 1] = tk;
        if (k == d - 2) {
          TRY(cores[d - 1].alloc(c, (size_t)tk * cols * sizeof(zc)));
          c->launches++;
          TRY(qtt_cross_gather<double>(S.as<zc>(), cols, pivb.as<int>(), tk, cols, 0, cores[d - 1].as<zc>(),
                                       c->stream));
        }
      } else {
        DBuf Cn;
        TRY(Cn.alloc(c, (size_t)tk * M * sizeof(zc)));
        c->launches++;
        TRY(qtt_copy_strided<double>(A.as<zc>(), MIdx{tk, 1, 1, 0}, MIdx{M, 1, tk, 0}, tk, M, 1, Cn.as<zc>(), M,
                                     c->stream));
        cores[k + 1] = std::move(Cn);
        DBuf Jn;
        TRY(Jn.alloc(c, (size_t)tk * (d - k - 1)));
        c->launches++;
        TRY(qtt_cross_right_index(J[k + 2].as<uint8_t>(), d - k - 2, rr, pivb.as<int>(), tk, Jn.as<uint8_t>(),
                                  c->stream));
        J[k + 1] = std::move(Jn);
        rJ[k + 1] = tk;
        if (k == 0) {
          // core 0 (1, n0, tk): S[i, piv[a]] = conj(S^H[piv[a], i])
          TRY(cores[0].alloc(c, (size_t)rows * tk * sizeof(zc)));
          c->launches++;
          TRY(qtt_cross_gather<double>(S.as<zc>(), rows, pivb.as<int>(), tk, rows, 1, cores[0].as<zc>(),
                                       c->stream));
        }
      }
    }
    std::vector<int> r(d + 1, 1);
    for (int k = 1; k < d; ++k) r[k] = fwd ? rI[k] : rJ[k];
    qtt_tt* y = tt_alloc(c, d, modes, r, QTT_C128, &s);
    if (!y) return s;
    for (int k = 0; k < d; ++k)
      cudaMemcpyAsync(core_ptr<char>(y, k), cores[k].p, (size_t)r[k] * modes[k] * r[k + 1] * sizeof(zc),
                      cudaMemcpyDeviceToDevice, c->stream);
    st->max_rank = *std::max_element(r.begin(), r.end());
    st->half_sweeps = h;
    if (prev) {
      qtt_tt* diff = nullptr;
      double nd = 0, ny = 0;
      s = add_dev<double>(c, zc(1, 0), y, zc(-1, 0), prev, &diff);
      if (!s) s = norm_dev<double>(c, diff, &nd);
      if (diff) tt_free(diff);
      if (!s) s = norm_dev<double>(c, y, &ny);
      tt_free(prev);
      prev = nullptr;
      if (s) {
        tt_free(y);
        return s;
      }
      rel = ny > 0 ? nd / ny : 0.0;
    }
    prev = y;
    st->rel_change = rel;
    if (h >= 2 && rel <= 10.0 * eps) break;
  }
  *out = prev;
  prev = nullptr;
  return QTT_OK;
}

// TT-cross, then an FP64 SVD rounding at eps (the interpolation ranks carry
// the kick columns and some redundancy).
int cross_rounded(qtt_ctx* c, const CrossFn& f, const std::vector<int>& modes, double eps, int max_rank, int kick,
                  int max_half_sweeps, uint64_t seed, const std::vector<std::vector<uint8_t>>& seeds, qtt_tt** out,
                  CrossOut* st) {
  qtt_tt* x = nullptr;
  TRY(cross_dev(c, f, modes, eps, max_rank, kick, max_half_sweeps, seed, seeds, &x, st));
  qtt_round_info ri;
  int s = round_det<double>(c, x, eps, 0, nullptr, &ri, out);
  tt_free(x);
  return s;
}

