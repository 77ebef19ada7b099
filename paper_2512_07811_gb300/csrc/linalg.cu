// Small dense factorisations on the device, one CTA per matrix, batched over
// blockIdx.x:
//   * Householder QR returning only R (the orthogonalisation sweep of TT
//     rounding needs only the triangular factor; TSQR trees stack R factors);
//   * one-sided (Hestenes) Jacobi SVD with accumulated right rotations;
//   * the truncation-rank rule on sorted singular values.
// Arithmetic is in the storage precision R (double or float); reductions of
// the truncation tail are always in double.
#include <cooperative_groups.h>
#include <float.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <utility>

#include "common.cuh"
#include "kernels.h"

namespace {

template <class R>
__device__ R block_sum(R v, R* red) {
  // red: shared scratch of blockDim.x/32 entries
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  R s = R(0);
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// --------------------------------------------------------------- QR (R only)
// Input element (i, c) of batch b sits at in[in_b + rowI(i) + colI(c)] (optionally
// conjugated); rows at or beyond rows_valid(b) read as zero.  W is a per-batch
// workspace of m*n elements (row-major, ld = n).  Output R_b is min(m, n) x n,
// upper trapezoidal, row-major with leading dimension ldr, at out + b*out_bstride.
template <class R>
__device__ __forceinline__ R warp_sum(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Householder QR, one CTA of 1024 threads per matrix.  The matrix is copied
// into a column-major workspace (W + c*m + i holds element (i, c)) so that a
// warp streams a column with consecutive lanes on consecutive rows; every
// trailing column is handled by one warp (dot product with the reflector by
// shuffles, then the rank-1 update).  Two barriers per column: thread 0 forms
// reflector j from the norm that the warp owning column j computed while it
// applied reflector j-1, then all warps apply reflector j.  Reflectors are
// stored unscaled below the diagonal, v = (1, x_{j+1} / v0, ...), with 1/v0
// kept per column, and scaled on the fly.
template <class R>
__global__ void __launch_bounds__(1024)
qr_r_kernel(const cplx<R>* __restrict__ in, MIdx inB, MIdx rowI, MIdx colI, int conj_in,
            int64_t m, int64_t n, int64_t rows_total, int64_t rows_per_batch,
            cplx<R>* __restrict__ Wbase, cplx<R>* __restrict__ out, int64_t out_bstride, int64_t ldr,
            cplx<R>* __restrict__ tauws, cplx<R>* __restrict__ Qout, int64_t q_bstride, int64_t ldq,
            cplx<R>* __restrict__ Qws) {
  __shared__ double red[32];
  __shared__ double s_nrm2[2];
  __shared__ cplx<R> s_iv;
  __shared__ R s_tau;
  __shared__ int s_zero;
  const int64_t b = blockIdx.x;
  cplx<R>* W = Wbase + b * m * n;
  const int64_t row0 = b * rows_per_batch;
  int64_t valid = rows_total - row0;
  if (valid > m) valid = m;
  const int64_t ib = midx_off(inB, b);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  double part = 0.0, part0 = 0.0;
  for (int64_t e = threadIdx.x; e < m * n; e += blockDim.x) {
    int64_t i = e / n, c = e - i * n;
    cplx<R> v(0, 0);
    if (i < valid) {
      v = in[ib + midx_off(rowI, i) + midx_off(colI, c)];
      if (conj_in) v.im = -v.im;
    }
    W[c * m + i] = v;
    const double a2 = (double)v.re * v.re + (double)v.im * v.im;
    part += a2;
    if (c == 0) part0 += a2;
  }
  // columns whose remaining norm is below eps * ||A||_F are numerically zero:
  // they are cleared instead of reflected (a perturbation within the
  // backward error of the factorisation), which keeps every reflector
  // away from underflow
  const double anorm2 = block_sum(part, red);
  const double col0 = block_sum(part0, red);
  if (threadIdx.x == 0) s_nrm2[0] = col0;
  const double eps = sizeof(R) == 8 ? (double)DBL_EPSILON : (double)FLT_EPSILON;
  const double zero_thresh2 = eps * eps * anorm2;
  const int64_t kmax = m < n ? m : n;
  __syncthreads();
  for (int64_t j = 0; j < kmax; ++j) {
    cplx<R>* colj = W + j * m;
    if (threadIdx.x == 0) {
      const double nrm2 = s_nrm2[j & 1];
      cplx<R> x0 = colj[j];
      double ax2 = (double)x0.re * x0.re + (double)x0.im * x0.im;
      double below = nrm2 - ax2;
      cplx<R> iv(0, 0);
      if (nrm2 <= zero_thresh2 || below <= zero_thresh2) {
        s_tau = R(0);
        s_zero = 1;
        if (nrm2 <= zero_thresh2) colj[j] = cplx<R>(0, 0);
      } else {
        // H = I - tau v v^H, v0 = x0 - alpha, alpha = -e^{i arg x0} ||x||,
        // tau = 2 |v0|^2 / ||x - alpha e1||^2 in [1, 2]
        double ax0 = sqrt(ax2), nrm = sqrt(nrm2);
        double phr = ax0 > 0 ? x0.re / ax0 : 1.0, phi = ax0 > 0 ? x0.im / ax0 : 0.0;
        double alr = -phr * nrm, ali = -phi * nrm;
        double v0r = x0.re - alr, v0i = x0.im - ali;
        double v02 = v0r * v0r + v0i * v0i;
        s_tau = (R)(2.0 * v02 / (below + v02));
        iv = cplx<R>((R)(v0r / v02), (R)(-v0i / v02));
        s_zero = 0;
        colj[j] = cplx<R>((R)alr, (R)ali);
      }
      s_iv = iv;
      if (tauws) {
        tauws[b * 2 * n + 2 * j] = iv;
        tauws[b * 2 * n + 2 * j + 1] = cplx<R>(s_tau, R(0));
      }
    }
    __syncthreads();
    const R tau = s_tau;
    const cplx<R> iv = s_iv;
    if (s_zero) {
      for (int64_t i = j + 1 + threadIdx.x; i < m; i += blockDim.x) colj[i] = cplx<R>(0, 0);
    }
    for (int64_t c = j + 1 + warp; c < n; c += nwarps) {
      cplx<R>* colc = W + c * m;
      if (tau != R(0)) {
        cplx<R> w(0, 0);
        if (lane == 0) w = colc[j];
        for (int64_t i = j + 1 + lane; i < m; i += 32) cfma_conj(w, colj[i] * iv, colc[i]);
        w.re = warp_sum(w.re);
        w.im = warp_sum(w.im);
        w = tau * w;
        if (lane == 0) colc[j] = colc[j] - w;
        for (int64_t i = j + 1 + lane; i < m; i += 32) colc[i] = colc[i] - (colj[i] * iv) * w;
      }
      if (c == j + 1) {
        // norm of the next column below (and at) the next diagonal, for the next step
        __syncwarp();
        double p2 = 0.0;
        for (int64_t i = j + 1 + lane; i < m; i += 32) {
          cplx<R> v = colc[i];
          p2 += (double)v.re * v.re + (double)v.im * v.im;
        }
        for (int o = 16; o > 0; o >>= 1) p2 += __shfl_xor_sync(0xffffffffu, p2, o);
        if (lane == 0) s_nrm2[(j + 1) & 1] = p2;
      }
    }
    __syncthreads();
  }
  if (out) {
    cplx<R>* Rb = out + b * out_bstride;
    for (int64_t e = threadIdx.x; e < kmax * n; e += blockDim.x) {
      int64_t i = e / n, c = e - i * n;
      Rb[i * ldr + c] = (c >= i) ? W[c * m + i] : cplx<R>(0, 0);
    }
  }
  if (Qout) {
    // Q = H_0 H_1 ... H_{kmax-1} [I; 0], accumulated from the last reflector
    // in the column-major workspace Qws (one warp per column of Q, rows on
    // the lanes), then written out row-major
    cplx<R>* Qc = Qws + b * m * kmax;
    for (int64_t e = threadIdx.x; e < m * kmax; e += blockDim.x) {
      int64_t c = e / m, i = e - c * m;
      Qc[e] = cplx<R>(i == c ? R(1) : R(0), R(0));
    }
    __syncthreads();
    for (int64_t j = kmax - 1; j >= 0; --j) {
      const R tau = tauws[b * 2 * n + 2 * j + 1].re;
      const cplx<R> iv = tauws[b * 2 * n + 2 * j];
      const cplx<R>* colj = W + j * m;
      if (tau != R(0)) {
        for (int64_t c = j + warp; c < kmax; c += nwarps) {
          cplx<R>* qc = Qc + c * m;
          cplx<R> w(0, 0);
          if (lane == 0) w = qc[j];
          for (int64_t i = j + 1 + lane; i < m; i += 32) cfma_conj(w, colj[i] * iv, qc[i]);
          w.re = warp_sum(w.re);
          w.im = warp_sum(w.im);
          w = tau * w;
          if (lane == 0) qc[j] = qc[j] - w;
          for (int64_t i = j + 1 + lane; i < m; i += 32) qc[i] = qc[i] - (colj[i] * iv) * w;
        }
      }
      __syncthreads();
    }
    cplx<R>* Q = Qout + b * q_bstride;
    for (int64_t e = threadIdx.x; e < m * kmax; e += blockDim.x) {
      int64_t i = e / kmax, c = e - i * kmax;
      Q[i * ldq + c] = Qc[c * m + i];
    }
  }
}

// ------------------------------------------------------- one-sided Jacobi
// G (p x q, row-major ld = q, per batch at G + b*p*q) is rotated in place so
// that its columns become mutually orthogonal; V (q x q, row-major, per batch
// at V + b*q*q) accumulates the rotations (G_in V = G_out).  On exit the
// columns are sorted by decreasing norm: sigma[b*q + j] = ||G_out[:, j]||,
// V columns permuted alike; G columns are left unsorted (callers use V).
template <class R>
__global__ void __launch_bounds__(256)
jacobi_kernel(cplx<R>* __restrict__ Gbase, cplx<R>* __restrict__ Vbase, R* __restrict__ sigma_out,
              cplx<R>* __restrict__ Vsorted_base, cplx<R>* __restrict__ Usorted_base, int p, int q, int max_sweeps,
              int* __restrict__ sweeps_out) {
  extern __shared__ unsigned char smem_raw[];
  const int64_t b = blockIdx.x;
  cplx<R>* G = Gbase + b * (int64_t)p * q;
  cplx<R>* V = Vbase + b * (int64_t)q * q;
  const int qe = q + (q & 1);            // even number of players (one virtual)
  int* order = reinterpret_cast<int*>(smem_raw);          // qe entries
  R* norms = reinterpret_cast<R*>(order + qe + (qe & 1)); // q entries (aligned for double)
  __shared__ int s_rot;
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
    int i = e / q, c = e - i * q;
    V[e] = cplx<R>(i == c ? R(1) : R(0), R(0));
  }
  for (int e = threadIdx.x; e < qe; e += blockDim.x) order[e] = e;
  __syncthreads();
  // stop when every column pair has |cos| <= sqrt(p) eps; the sweep count is bounded by max_sweeps
  const R tol = (sizeof(R) == 8 ? R(DBL_EPSILON) : R(FLT_EPSILON)) * sqrt(R(p > 1 ? p : 1));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < qe - 1; ++round) {
      for (int pr = warp; pr < qe / 2; pr += nwarps) {
        int a = order[pr], c = order[qe - 1 - pr];
        if (a >= q || c >= q) continue;
        if (a > c) { int t = a; a = c; c = t; }
        R al = 0, be = 0;
        cplx<R> ga(0, 0);
        for (int i = lane; i < p; i += 32) {
          cplx<R> x = G[(int64_t)i * q + a], y = G[(int64_t)i * q + c];
          al += abs2(x);
          be += abs2(y);
          cfma_conj(ga, x, y);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga.re += __shfl_xor_sync(0xffffffffu, ga.re, o);
          ga.im += __shfl_xor_sync(0xffffffffu, ga.im, o);
        }
        R ag = sqrt(abs2(ga));
        if (!(al > R(0) && be > R(0)) || !(ag > tol * sqrt(al) * sqrt(be))) continue;
        // rotation making columns a, c orthogonal (complex Hestenes step)
        cplx<R> ph(ga.re / ag, ga.im / ag);       // e^{i phi}
        R zeta = (be - al) / (R(2) * ag);
        R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
        R cs = R(1) / sqrt(R(1) + t * t);
        R sn = cs * t;
        // new_a = cs*a - sn*conj(ph)*c ; new_c = sn*ph*a + cs*c
        cplx<R> f1 = sn * conjg(ph);
        cplx<R> f2 = sn * ph;
        for (int i = lane; i < p; i += 32) {
          cplx<R> x = G[(int64_t)i * q + a], y = G[(int64_t)i * q + c];
          G[(int64_t)i * q + a] = cs * x - f1 * y;
          G[(int64_t)i * q + c] = f2 * x + cs * y;
        }
        for (int i = lane; i < q; i += 32) {
          cplx<R> x = V[(int64_t)i * q + a], y = V[(int64_t)i * q + c];
          V[(int64_t)i * q + a] = cs * x - f1 * y;
          V[(int64_t)i * q + c] = f2 * x + cs * y;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
      // rotate the tournament: keep order[0], cycle the rest
      if (threadIdx.x == 0) {
        int last = order[qe - 1];
        for (int i = qe - 1; i > 1; --i) order[i] = order[i - 1];
        order[1] = last;
      }
      __syncthreads();
    }
    int any = s_rot;
    __syncthreads();
    if (!any) break;
  }
  if (threadIdx.x == 0 && sweeps_out) sweeps_out[b] = sweep;
  // column norms
  for (int c = warp; c < q; c += nwarps) {
    R s = 0;
    for (int i = lane; i < p; i += 32) s += abs2(G[(int64_t)i * q + c]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) norms[c] = sqrt(s);
  }
  __syncthreads();
  // rank of each column by decreasing norm (ties by index) and scatter
  cplx<R>* Vs = Vsorted_base + b * (int64_t)q * q;
  for (int c = threadIdx.x; c < q; c += blockDim.x) {
    R v = norms[c];
    int rk = 0;
    for (int i = 0; i < q; ++i) {
      R u = norms[i];
      rk += (u > v) || (u == v && i < c);
    }
    sigma_out[b * (int64_t)q + rk] = v;
    for (int i = 0; i < q; ++i) Vs[(int64_t)i * q + rk] = V[(int64_t)i * q + c];
    if (Usorted_base) {
      // normalised rotated column: G_in V = U S, so U[:, rk] = G_out[:, c] / sigma
      cplx<R>* Us = Usorted_base + b * (int64_t)p * q;
      // columns with a subnormal norm carry no usable direction
      R f = v > (sizeof(R) == 8 ? R(DBL_MIN) : R(FLT_MIN)) * R(4) ? R(1) / v : R(0);
      for (int i = 0; i < p; ++i) {
        cplx<R> g = G[(int64_t)i * q + c];
        Us[(int64_t)i * q + rk] = cplx<R>(g.re * f, g.im * f);
      }
    }
  }
}

// Truncation rule on sorted singular values: smallest t >= 1 with
// sqrt(sum_{j >= t} s_j^2) <= delta, then capped at max_rank.  Writes t and
// whether the cap cut a rank the tolerance asked for, plus the discarded tail.
template <class R>
__device__ void trunc_rank_body(const R* __restrict__ s, int q, double delta, int max_rank,
                                int* __restrict__ out /* [t, capped] */, double* __restrict__ tail_out) {
  double tail2 = 0.0;
  int t = q;
  // walk from the end: tail2 after including s[j] is sum_{i >= j} s_i^2
  for (int j = q - 1; j >= 1; --j) {
    double v = (double)s[j];
    double nt = tail2 + v * v;
    if (sqrt(nt) <= delta) {
      tail2 = nt;
      t = j;
    } else {
      break;
    }
  }
  if (q == 0) t = 0;
  int capped = 0;
  if (max_rank > 0 && t > max_rank) {
    t = max_rank;
    capped = 1;
  }
  double tl = 0.0;
  for (int j = t; j < q; ++j) tl += (double)s[j] * (double)s[j];
  out[0] = t;
  out[1] = capped;
  if (tail_out) *tail_out = sqrt(tl);
}

template <class R>
__global__ void trunc_rank_kernel(const R* __restrict__ s, int q, double delta, int max_rank,
                                  int* __restrict__ out, double* __restrict__ tail_out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) trunc_rank_body<R>(s, q, delta, max_rank, out, tail_out);
}

// ------------------------------------------- one-sided Jacobi over many CTAs
// Same rotations as jacobi_kernel, one launch per round of the round-robin
// tournament (q/2 disjoint column pairs, one warp per pair, all SMs), on a
// column-major copy Gc (q columns of length p) and Vc (q columns of length q).
// Round r pairs position i with position qe-1-i of the order
// [0, 1 + (r mod (qe-1)), ...]: order[0] = 0, order[i] = 1 + (i - 1 + r) mod (qe - 1).
template <class R>
__global__ void __launch_bounds__(256)
jacobi_round_kernel(cplx<R>* __restrict__ Gc, cplx<R>* __restrict__ Vc, int p, int q, int round,
                    int* __restrict__ rotated) {
  const int qe = q + (q & 1);
  const int lane = threadIdx.x & 31;
  const int pr = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (pr >= qe / 2) return;
  auto ord = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + round) % (qe - 1); };
  int a = ord(pr), c = ord(qe - 1 - pr);
  if (a >= q || c >= q) return;
  if (a > c) { int t = a; a = c; c = t; }
  cplx<R>* ga = Gc + (int64_t)a * p;
  cplx<R>* gc = Gc + (int64_t)c * p;
  R al = 0, be = 0;
  cplx<R> g(0, 0);
  for (int i = lane; i < p; i += 32) {
    cplx<R> x = ga[i], y = gc[i];
    al += abs2(x);
    be += abs2(y);
    cfma_conj(g, x, y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    g.re += __shfl_xor_sync(0xffffffffu, g.re, o);
    g.im += __shfl_xor_sync(0xffffffffu, g.im, o);
  }
  const R tol = (sizeof(R) == 8 ? R(DBL_EPSILON) : R(FLT_EPSILON)) * sqrt(R(p > 1 ? p : 1));
  R ag = sqrt(abs2(g));
  if (!(al > R(0) && be > R(0)) || !(ag > tol * sqrt(al) * sqrt(be))) return;
  cplx<R> ph(g.re / ag, g.im / ag);
  R zeta = (be - al) / (R(2) * ag);
  R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
  R cs = R(1) / sqrt(R(1) + t * t);
  R sn = cs * t;
  cplx<R> f1 = sn * conjg(ph), f2 = sn * ph;
  for (int i = lane; i < p; i += 32) {
    cplx<R> x = ga[i], y = gc[i];
    ga[i] = cs * x - f1 * y;
    gc[i] = f2 * x + cs * y;
  }
  if (Vc) {
    cplx<R>* va = Vc + (int64_t)a * q;
    cplx<R>* vc = Vc + (int64_t)c * q;
    for (int i = lane; i < q; i += 32) {
      cplx<R> x = va[i], y = vc[i];
      va[i] = cs * x - f1 * y;
      vc[i] = f2 * x + cs * y;
    }
  }
  if (lane == 0) *rotated = 1;
}

// column norms of Gc, then the sorted outputs in the row-major layout of jacobi_kernel
template <class R>
__global__ void __launch_bounds__(256)
jacobi_finish_kernel(const cplx<R>* __restrict__ Gc, const cplx<R>* __restrict__ Vc, int p, int q,
                     R* __restrict__ sigma_out, cplx<R>* __restrict__ Vs, cplx<R>* __restrict__ Us) {
  extern __shared__ unsigned char smem_raw[];
  R* norms = reinterpret_cast<R*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int c = warp; c < q; c += nwarps) {
    R s = 0;
    for (int i = lane; i < p; i += 32) s += abs2(Gc[(int64_t)c * p + i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) norms[c] = sqrt(s);
  }
  __syncthreads();
  for (int c = warp; c < q; c += nwarps) {
    R v = norms[c];
    int rk = 0;
    for (int i = 0; i < q; ++i) {
      R u = norms[i];
      rk += (u > v) || (u == v && i < c);
    }
    if (lane == 0) sigma_out[rk] = v;
    if (Vs)
      for (int i = lane; i < q; i += 32) Vs[(int64_t)i * q + rk] = Vc[(int64_t)c * q + i];
    if (Us) {
      R f = v > (sizeof(R) == 8 ? R(DBL_MIN) : R(FLT_MIN)) * R(4) ? R(1) / v : R(0);
      for (int i = lane; i < p; i += 32) {
        cplx<R> g = Gc[(int64_t)c * p + i];
        Us[(int64_t)i * q + rk] = cplx<R>(g.re * f, g.im * f);
      }
    }
  }
}

// G (p x q row-major) -> Gc column-major; Vc = identity (column-major)
template <class R>
__global__ void jacobi_setup_kernel(const cplx<R>* __restrict__ G, int p, int q, cplx<R>* __restrict__ Gc,
                                    cplx<R>* __restrict__ Vc) {
  const int64_t tg = (int64_t)p * q, tv = (int64_t)q * q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tg + tv;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < tg) {
      int64_t c = e / p, i = e - c * p;
      Gc[e] = G[i * q + c];
    } else if (Vc) {
      int64_t f = e - tg;
      int64_t c = f / q, i = f - c * q;
      Vc[f] = cplx<R>(i == c ? R(1) : R(0), R(0));
    }
  }
}

// ------------------------------------------- one-sided Jacobi in shared memory
// One CTA of 1024 threads.  G (p x q, row-major input, ld q) is held
// column-major in shared memory.  Each round of the round-robin tournament
// pairs order[i] with order[qe-1-i] (order[0] = 0, order[i] = 1 + (i - 1 + r)
// mod (qe - 1)); each half-warp takes one pair of a round (its 16 lanes the
// rows), so the 64 pairs of a 128-column round run side by side.  Outputs as
// in jacobi_kernel: sigma sorted decreasingly, normalised columns of the
// rotated G (row-major p x q) and, when Vs is given, the accumulated rotations
// (row-major q x q, accumulated column-major in the global workspace Vws) in
// the same order.  Without Vs no rotation touches global memory.
// Rotation of one column pair from al = |g_a|^2, be = |g_c|^2, g = g_a^H g_c:
// false if the pair is already orthogonal to tol (|g|^2 <= tol2 al be, a zero
// column, or |g|^2 below the normal range), else the unitary [cs, -f1; f2, cs] (f1 = sn conj(ph), f2 = sn
// ph, ph = g / |g|, tan = t from the usual smaller root of t^2 + 2 zeta t - 1
// = 0, zeta = (be - al) / (2 |g|)).  1/|g| and cos come from a reciprocal
// square root refined by one Newton step, y <- y (3 - x y^2) / 2, which keeps
// cs^2 (1 + t^2) and |ph| within a few units in the last place of 1.
template <class R>
__device__ __forceinline__ R rsqrt_refined(R x) {
  R y = rsqrt(x);
  return y * (R(1.5) - R(0.5) * x * y * y);
}

template <class R>
__device__ __forceinline__ bool jacobi_rotation(R al, R be, cplx<R> g, R tol2, R& cs, cplx<R>& f1, cplx<R>& f2) {
  const R ag2 = abs2(g);
  // an inner product whose square is below the normal range is rounding noise of two tiny columns
  const R tiny = sizeof(R) == 8 ? R(DBL_MIN) : R(FLT_MIN);
  if (!(al > R(0) && be > R(0)) || !(ag2 > tol2 * al * be) || !(ag2 >= tiny)) return false;
  const R inv = rsqrt_refined(ag2);
  const R zeta = (be - al) * (R(0.5) * inv);
  const R az = fabs(zeta);
  // for |zeta| beyond 1e18 the root is 1 / (2 zeta) to working precision (and zeta^2 could overflow)
  R t;
  if constexpr (sizeof(R) == 4) {
    // the tangent only steers the rotation (cos and sin below are consistent
    // with whatever t is, so the rotation stays orthogonal); hardware
    // approximations of the square root and the quotient leave a residual
    // inner product of a few ulp, far below the stopping tolerance
    const R u = R(1) + az * az;
    t = az < R(1e18) ? __fdividef(R(1), az + u * rsqrtf(u)) : __fdividef(R(0.5), az);
  } else {
    t = az < R(1e18) ? R(1) / (az + sqrt(R(1) + az * az)) : R(0.5) / az;
  }
  if (zeta < R(0)) t = -t;
  cs = rsqrt_refined(R(1) + t * t);
  const R sn = cs * t;
  const cplx<R> ph(g.re * inv, g.im * inv);
  f1 = sn * conjg(ph);
  f2 = sn * ph;
  return true;
}

template <class R>
__device__ __forceinline__ R half_sum(R v, unsigned mask) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, 16);
  return v;
}

template <class R>
__global__ void __launch_bounds__(1024)
jacobi_smem_kernel(const cplx<R>* __restrict__ Gin, cplx<R>* __restrict__ Vws, R* __restrict__ sigma_out,
                   cplx<R>* __restrict__ Vs, cplx<R>* __restrict__ Us, int p, int q, int max_sweeps,
                   int* __restrict__ sweeps_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* Gs = reinterpret_cast<cplx<R>*>(smem_raw);
  R* norms = reinterpret_cast<R*>(Gs + (size_t)p * q);
  __shared__ int s_rot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int hl = lane & 15, hw = warp * 2 + (lane >> 4), nhw = nwarps * 2;
  const unsigned hmask = (lane >> 4) ? 0xffff0000u : 0x0000ffffu;
  const bool wantV = Vs != nullptr;
  for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
    int i = e / q, c = e - i * q;
    Gs[c * p + i] = Gin[e];
  }
  if (wantV)
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
      int c = e / q, i = e - c * q;
      Vws[e] = cplx<R>(i == c ? R(1) : R(0), R(0));
    }
  __syncthreads();
  const int qe = q + (q & 1);
  const R tol = (sizeof(R) == 8 ? R(DBL_EPSILON) : R(FLT_EPSILON)) * sqrt(R(p > 1 ? p : 1));
  const R tol2 = tol * tol;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < qe - 1; ++round) {
      for (int pr = hw; pr < qe / 2; pr += nhw) {
        int a = pr == 0 ? 0 : 1 + (pr - 1 + round) % (qe - 1);
        int qi = qe - 1 - pr;
        int c = qi == 0 ? 0 : 1 + (qi - 1 + round) % (qe - 1);
        if (a >= q || c >= q) continue;
        if (a > c) { int t = a; a = c; c = t; }
        cplx<R>* ga = Gs + (size_t)a * p;
        cplx<R>* gc = Gs + (size_t)c * p;
        R al = 0, be = 0;
        cplx<R> g(0, 0);
#pragma unroll 4
        for (int i = hl; i < p; i += 16) {
          cplx<R> x = ga[i], y = gc[i];
          al += abs2(x);
          be += abs2(y);
          cfma_conj(g, x, y);
        }
        al = half_sum(al, hmask);
        be = half_sum(be, hmask);
        g.re = half_sum(g.re, hmask);
        g.im = half_sum(g.im, hmask);
        cplx<R> f1, f2;
        R cs;
        if (!jacobi_rotation(al, be, g, tol2, cs, f1, f2)) continue;
#pragma unroll 4
        for (int i = hl; i < p; i += 16) {
          cplx<R> x = ga[i], y = gc[i];
          ga[i] = cs * x - f1 * y;
          gc[i] = f2 * x + cs * y;
        }
        if (wantV) {
          cplx<R>* va = Vws + (size_t)a * q;
          cplx<R>* vc = Vws + (size_t)c * q;
          for (int i0 = hl; i0 < q; i0 += 64) {
            cplx<R> x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int i = i0 + 16 * u;
              if (i < q) {
                x[u] = va[i];
                y[u] = vc[i];
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int i = i0 + 16 * u;
              if (i < q) {
                va[i] = cs * x[u] - f1 * y[u];
                vc[i] = f2 * x[u] + cs * y[u];
              }
            }
          }
        }
        if (hl == 0) s_rot = 1;
      }
      __syncthreads();
    }
    int any = s_rot;
    __syncthreads();
    if (!any) {
      ++sweep;
      break;
    }
  }
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
  for (int c = warp; c < q; c += nwarps) {
    R sacc = 0;
    for (int i = lane; i < p; i += 32) sacc += abs2(Gs[(size_t)c * p + i]);
    sacc = warp_sum(sacc);
    if (lane == 0) norms[c] = sqrt(sacc);
  }
  __syncthreads();
  for (int c = warp; c < q; c += nwarps) {
    R v = norms[c];
    int rk = 0;
    for (int i = 0; i < q; ++i) {
      R u = norms[i];
      rk += (u > v) || (u == v && i < c);
    }
    if (lane == 0) sigma_out[rk] = v;
    if (wantV)
      for (int i = lane; i < q; i += 32) Vs[(size_t)i * q + rk] = Vws[(size_t)c * q + i];
    if (Us) {
      R f = v > (sizeof(R) == 8 ? R(DBL_MIN) : R(FLT_MIN)) * R(4) ? R(1) / v : R(0);
      for (int i = lane; i < p; i += 32) {
        cplx<R> g = Gs[(size_t)c * p + i];
        Us[(size_t)i * q + rk] = cplx<R>(g.re * f, g.im * f);
      }
    }
  }
}

// ----------------------------------------- one-sided Jacobi over a CTA cluster
// The rows of G (p x q) and of the rotation matrix V (q x q) are split over the
// NC CTAs of one thread-block cluster; each CTA keeps its rows of every
// column in shared memory.  A round of the round-robin tournament (order[0] =
// 0, order[i] = 1 + (i - 1 + r) mod (qe - 1), pairs (order[i], order[qe-1-i]))
// runs in three steps: every CTA computes its partial inner products of the
// round's column pairs (||g_a||^2, ||g_c||^2, g_a^H g_c over its rows) and
// writes them into slot [its rank] of every CTA's exchange buffer (distributed
// shared memory, double-buffered by round parity); one cluster barrier; every
// CTA sums the NC slots in rank order -- identical totals, hence identical
// rotation decisions in all CTAs -- and rotates its own rows of G and, when
// Vs_out is given, of V.  A half-warp takes one column pair in both steps.
template <class R, int NC>
__global__ void __launch_bounds__(1024)
jacobi_cluster_kernel(const cplx<R>* __restrict__ Gin, R* __restrict__ sigma_out, cplx<R>* __restrict__ Vs_out,
                      cplx<R>* __restrict__ Us_out, int p, int q, int max_sweeps, int* __restrict__ sweeps_out) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int qe = q + (q & 1);
  const int npairs = qe / 2;
  const bool wantV = Vs_out != nullptr;
  const int chunk = (p + NC - 1) / NC;                   // G rows per CTA
  const int chunkv = wantV ? (q + NC - 1) / NC : 0;      // V rows per CTA
  const int r0 = rank * chunk, r1 = min(p, r0 + chunk);
  const int v0 = rank * chunkv, v1 = min(q, v0 + chunkv);
  const int nr = max(r1 - r0, 0), nv = max(v1 - v0, 0);
  // layout: slots[2][NC][npairs] x 4 R | nsum[NC][q] R | norms[q] R | G[q][chunk] | V[q][chunkv]
  R* slots = reinterpret_cast<R*>(smem_raw);
  R* nsum = slots + 2 * NC * npairs * 4;
  R* norms = nsum + NC * q;
  size_t off = (size_t)(2 * NC * npairs * 4 + NC * q + q) * sizeof(R);
  off = (off + 15) & ~(size_t)15;
  cplx<R>* G = reinterpret_cast<cplx<R>*>(smem_raw + off);
  cplx<R>* V = G + (size_t)q * chunk;
  __shared__ int s_rot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int hl = lane & 15, hw = warp * 2 + (lane >> 4), nhw = nwarps * 2;
  const unsigned hmask = (lane >> 4) ? 0xffff0000u : 0x0000ffffu;
  for (int e = threadIdx.x; e < q * chunk; e += blockDim.x) {
    int c = e / chunk, i = e - c * chunk;
    G[e] = (r0 + i < p) ? Gin[(int64_t)(r0 + i) * q + c] : cplx<R>(0, 0);
  }
  for (int e = threadIdx.x; e < q * chunkv; e += blockDim.x) {
    int c = e / chunkv, i = e - c * chunkv;
    V[e] = cplx<R>((v0 + i == c) ? R(1) : R(0), R(0));
  }
  cluster.sync();
  const R tol = (sizeof(R) == 8 ? R(DBL_EPSILON) : R(FLT_EPSILON)) * sqrt(R(p > 1 ? p : 1));
  const R tol2 = tol * tol;
  int sweep = 0, round_count = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < qe - 1; ++round, ++round_count) {
      const int buf = round_count & 1;
      // 1. partial inner products of this round's pairs over the local rows (a half-warp per pair)
      for (int pr = hw; pr < npairs; pr += nhw) {
        int a = pr == 0 ? 0 : 1 + (pr - 1 + round) % (qe - 1);
        int qi = qe - 1 - pr;
        int c = qi == 0 ? 0 : 1 + (qi - 1 + round) % (qe - 1);
        R al = 0, be = 0;
        cplx<R> g(0, 0);
        if (a < q && c < q) {
          if (a > c) { int t = a; a = c; c = t; }
          const cplx<R>* ga = G + (size_t)a * chunk;
          const cplx<R>* gc = G + (size_t)c * chunk;
#pragma unroll 4
          for (int i = hl; i < nr; i += 16) {
            cplx<R> x = ga[i], y = gc[i];
            al += abs2(x);
            be += abs2(y);
            cfma_conj(g, x, y);
          }
          al = half_sum(al, hmask);
          be = half_sum(be, hmask);
          g.re = half_sum(g.re, hmask);
          g.im = half_sum(g.im, hmask);
        }
        if (hl < NC) {
          R* dst = cluster.map_shared_rank(slots, hl) + ((size_t)(buf * NC + rank) * npairs + pr) * 4;
          dst[0] = al;
          dst[1] = be;
          dst[2] = g.re;
          dst[3] = g.im;
        }
      }
      cluster.sync();
      // 2. totals (same order in every CTA) and the rotation of the local rows
      for (int pr = hw; pr < npairs; pr += nhw) {
        int a = pr == 0 ? 0 : 1 + (pr - 1 + round) % (qe - 1);
        int qi = qe - 1 - pr;
        int c = qi == 0 ? 0 : 1 + (qi - 1 + round) % (qe - 1);
        if (a >= q || c >= q) continue;
        if (a > c) { int t = a; a = c; c = t; }
        R al = 0, be = 0;
        cplx<R> g(0, 0);
#pragma unroll
        for (int rr = 0; rr < NC; ++rr) {
          const R* src = slots + ((size_t)(buf * NC + rr) * npairs + pr) * 4;
          al += src[0];
          be += src[1];
          g.re += src[2];
          g.im += src[3];
        }
        cplx<R> f1, f2;
        R cs;
        if (!jacobi_rotation(al, be, g, tol2, cs, f1, f2)) continue;
        cplx<R>* ga = G + (size_t)a * chunk;
        cplx<R>* gc = G + (size_t)c * chunk;
#pragma unroll 4
        for (int i = hl; i < nr; i += 16) {
          cplx<R> x = ga[i], y = gc[i];
          ga[i] = cs * x - f1 * y;
          gc[i] = f2 * x + cs * y;
        }
        if (wantV) {
          cplx<R>* va = V + (size_t)a * chunkv;
          cplx<R>* vc = V + (size_t)c * chunkv;
          for (int i = hl; i < nv; i += 16) {
            cplx<R> x = va[i], y = vc[i];
            va[i] = cs * x - f1 * y;
            vc[i] = f2 * x + cs * y;
          }
        }
        if (hl == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int any = s_rot;  // identical in every CTA: the decisions come from identical totals
    __syncthreads();
    if (!any) {
      ++sweep;
      break;
    }
  }
  if (rank == 0 && threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
  // column norms: local partial sums exchanged, then summed in rank order
  for (int c = warp; c < q; c += nwarps) {
    R sacc = 0;
    for (int i = lane; i < nr; i += 32) sacc += abs2(G[(size_t)c * chunk + i]);
    sacc = warp_sum(sacc);
    if (lane < NC) cluster.map_shared_rank(nsum, lane)[rank * q + c] = sacc;
  }
  cluster.sync();
  for (int c = threadIdx.x; c < q; c += blockDim.x) {
    R sacc = 0;
    for (int rr = 0; rr < NC; ++rr) sacc += nsum[rr * q + c];
    norms[c] = sqrt(sacc);
  }
  __syncthreads();
  for (int c = warp; c < q; c += nwarps) {
    R v = norms[c];
    int rk = 0;
    for (int i = 0; i < q; ++i) {
      R u = norms[i];
      rk += (u > v) || (u == v && i < c);
    }
    if (rank == 0 && lane == 0) sigma_out[rk] = v;
    if (wantV)
      for (int i = lane; i < nv; i += 32) Vs_out[(size_t)(v0 + i) * q + rk] = V[(size_t)c * chunkv + i];
    if (Us_out) {
      R f = v > (sizeof(R) == 8 ? R(DBL_MIN) : R(FLT_MIN)) * R(4) ? R(1) / v : R(0);
      for (int i = lane; i < nr; i += 32) {
        cplx<R> g = G[(size_t)c * chunk + i];
        Us_out[(size_t)(r0 + i) * q + rk] = cplx<R>(g.re * f, g.im * f);
      }
    }
  }
  // keep every CTA's shared memory alive until all remote writes are done
  cluster.sync();
}

}  // namespace

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum
// (minus its static shared memory), once per (kernel, device).  The limit is
// never lowered afterwards, so launches from several host threads with
// different dynamic sizes cannot invalidate one another.
int qtt_allow_max_smem(const void* func) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QTT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({func, dev})) return QTT_OK;
  int optin = 0;
  cudaFuncAttributes fa;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, func) != cudaSuccess)
    return QTT_ERR_CUDA;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) !=
      cudaSuccess)
    return QTT_ERR_CUDA;
  done.insert({func, dev});
  return QTT_OK;
}

// Compensated sums in working precision: each partial sum carries its
// rounding error (Knuth's TwoSum), so a sum of squares over a column is
// accurate to a few units in the last place however many terms it has,
// without FP64 arithmetic (slow on this part).
template <class R>
__device__ __forceinline__ void two_sum_acc(R& hi, R& lo, R t) {
  const R s = hi + t;
  const R bb = s - hi;
  lo += (hi - (s - bb)) + (t - bb);
  hi = s;
}

template <class R>
__device__ __forceinline__ R warp_sum_compensated(R hi, R lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const R ohi = __shfl_xor_sync(0xffffffffu, hi, o);
    const R olo = __shfl_xor_sync(0xffffffffu, lo, o);
    lo += olo;
    two_sum_acc(hi, lo, ohi);
  }
  return hi + lo;
}

// Reflector of a shared-memory column whose diagonal is row j, formed by one
// warp (lane 0 computes, the warp clears a numerically zero column):
// alpha = -e^{i arg x0} ||x||, v0 = x0 - alpha, stored as 1/v0 and tau; the
// scaled reflector (0 above row j, 1 at j, x_i / v0 below, 0 in the padding
// up to MP rows) is also written to vs, so that its users need no scaling.
template <class R, int MP>
__device__ __forceinline__ void qr_reflector_warp(cplx<R>* col, int j, int m, R below, R zero_thresh2, int lane,
                                                  R* s_taus, cplx<R>* s_ivs, cplx<R>* tauws, cplx<R>* vs) {
  __syncwarp();
  int zero = 0;
  cplx<R> iv(0, 0);
  if (lane == 0) {
    const cplx<R> x0 = col[j];
    const R ax2 = abs2(x0);
    const R nrm2 = below + ax2;
    R tau = R(0);
    if (nrm2 <= zero_thresh2 || below <= zero_thresh2) {
      zero = 1;
      if (nrm2 <= zero_thresh2) col[j] = cplx<R>(0, 0);
    } else {
      const R ax0 = sqrt(ax2), nrm = sqrt(nrm2);
      const R phr = ax0 > R(0) ? x0.re / ax0 : R(1), phi = ax0 > R(0) ? x0.im / ax0 : R(0);
      const R s0 = ax0 + nrm;
      const R v02 = s0 * s0;
      tau = R(2) * v02 / (below + v02);
      iv = cplx<R>(phr / s0, -phi / s0);
      col[j] = cplx<R>(-phr * nrm, -phi * nrm);
    }
    s_taus[j] = tau;
    s_ivs[j] = iv;
    if (tauws) {
      tauws[2 * j] = iv;
      tauws[2 * j + 1] = cplx<R>(tau, R(0));
    }
  }
  zero = __shfl_sync(0xffffffffu, zero, 0);
  iv.re = __shfl_sync(0xffffffffu, iv.re, 0);
  iv.im = __shfl_sync(0xffffffffu, iv.im, 0);
  if (zero)
    for (int i = j + 1 + lane; i < m; i += 32) col[i] = cplx<R>(0, 0);
  for (int i = lane; i < MP; i += 32)
    vs[i] = i > j && i < m ? col[i] * iv : cplx<R>(i == j ? R(1) : R(0), R(0));
}

// ------------------------------------------------- left-looking panel QR
// Householder QR, one CTA per matrix, for m <= 32 * RPL rows.  Columns are
// taken in panels of NW (= warps per CTA) columns.  For a panel, each warp
// loads one column into registers (rows on the lanes) and applies every
// earlier reflector to it on its own -- no barrier, the reflectors read from
// the workspace W through L1 -- then the panel is factored in shared memory
// (all warps apply reflector j, the warp owning column j + 1 meanwhile
// computes that column's norm and reflector, one barrier per column) and
// written back to W.  Earlier reflectors
// are staged in shared memory one panel at a time.  The explicit Q, when
// wanted, is formed column by column in registers, one warp per column
// (Q e_c = H_0 ... H_c e_c).  Same inputs, outputs, zero-column rule and
// reflector format (v = (1, x_{j+1} / v0, ...) with 1/v0 and tau kept per
// column) as qr_r_kernel.
// warps per CTA of qr_panel_kernel: 16 where two register columns would not fit 64 registers
template <class R, int RPL>
constexpr int qr_panel_warps() { return sizeof(R) * RPL > 32 ? 16 : 32; }

template <class R, int RPL>
__global__ void __launch_bounds__(32 * qr_panel_warps<R, RPL>())
qr_panel_kernel(const cplx<R>* __restrict__ in, MIdx inB, MIdx rowI, MIdx colI, int conj_in, int m, int n,
                int64_t rows_total, int64_t rows_per_batch, cplx<R>* __restrict__ Wbase, cplx<R>* __restrict__ out,
                int64_t out_bstride, int64_t ldr, cplx<R>* __restrict__ tauws, cplx<R>* __restrict__ Qout,
                int64_t q_bstride, int64_t ldq) {
  constexpr int MP = 32 * RPL;  // rows padded to whole warps
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NW = blockDim.x >> 5;
  const int kmax = m < n ? m : n;
  cplx<R>* P = reinterpret_cast<cplx<R>*>(smem_raw);           // panel, NW columns of m
  cplx<R>* S = P + (size_t)NW * m;                              // NW scaled reflectors of MP rows
  cplx<R>* Vc = S + (size_t)NW * MP;                            // the current scaled reflector, 2 x MP
  cplx<R>* s_ivs = Vc + 2 * MP;                                 // 1/v0 per reflector
  R* s_taus = reinterpret_cast<R*>(s_ivs + kmax);               // tau per reflector
  __shared__ R red[32];
  const int64_t b = blockIdx.x;
  cplx<R>* W = Wbase + b * (int64_t)m * n;
  cplx<R>* tw = tauws ? tauws + b * 2 * n : nullptr;
  const int64_t row0 = b * rows_per_batch;
  int64_t valid = rows_total - row0;
  if (valid > m) valid = m;
  const int64_t ib = midx_off(inB, b);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // Frobenius norm of the input, for the numerically-zero threshold
  R part = 0;
  for (int c = warp; c < n; c += NW)
    for (int i = lane; i < valid; i += 32) part += abs2(in[ib + midx_off(rowI, i) + midx_off(colI, c)]);
  const R anorm2 = block_sum(part, red);
  const R eps = sizeof(R) == 8 ? R(DBL_EPSILON) : R(FLT_EPSILON);
  const R zero_thresh2 = eps * eps * anorm2;
  // stage reflectors q0 .. q0+qn-1 from W into S, scaled
  auto stage = [&](int q0, int qn) {
    for (int e = threadIdx.x; e < qn * MP; e += blockDim.x) {
      const int jj = e / MP, i = e - jj * MP;
      const int j = q0 + jj;
      const cplx<R> v = i > j && i < m ? W[(int64_t)j * m + i] * s_ivs[j] : cplx<R>(i == j ? R(1) : R(0), R(0));
      S[e] = s_taus[j] != R(0) ? v : cplx<R>(0, 0);
    }
  };
  // x <- (I - tau v v^H) x for a register column and the scaled reflector j
  // in shared memory; v is zero above row j and below row m, so only the
  // 32-row slices that meet rows j .. m-1 are touched (a warp-uniform test)
  auto reflect = [&](cplx<R>(&x)[RPL], const cplx<R>* v, R tau, int j) {
    cplx<R> w(0, 0), w1(0, 0);
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      if (32 * u + 31 < j || 32 * u >= m) continue;
      if (u & 1) cfma_conj(w1, v[lane + 32 * u], x[u]); else cfma_conj(w, v[lane + 32 * u], x[u]);
    }
    w = w + w1;
    w.re = warp_sum(w.re);
    w.im = warp_sum(w.im);
    w = tau * w;
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      if (32 * u + 31 < j || 32 * u >= m) continue;
      x[u] = x[u] - v[lane + 32 * u] * w;
    }
  };
  for (int p0 = 0; p0 < n; p0 += NW) {
    const int pcols = min(NW, n - p0);
    const int pw = max(0, min(NW, kmax - p0));  // reflectors formed in this panel
    // 1. column p0 + warp: load, apply reflectors 0 .. p0-1 (staged one
    // earlier panel at a time), store into the panel
    const int c = p0 + warp;
    cplx<R> x[RPL];
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      const int i = lane + 32 * u;
      cplx<R> v(0, 0);
      if (warp < pcols && i < valid) {
        v = in[ib + midx_off(rowI, i) + midx_off(colI, c)];
        if (conj_in) v.im = -v.im;
      }
      x[u] = v;
    }
    for (int q0 = 0; q0 < p0 && q0 < kmax; q0 += NW) {
      const int qn = min(NW, kmax - q0);
      stage(q0, qn);
      __syncthreads();
      if (warp < pcols)
        for (int jj = 0; jj < qn; ++jj) {
          const R tau = s_taus[q0 + jj];
          if (tau != R(0)) reflect(x, S + (size_t)jj * MP, tau, q0 + jj);
        }
      __syncthreads();
    }
    if (warp < pcols) {
      cplx<R>* pc = P + (size_t)warp * m;
      R hi = 0, lo = 0;
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        const int i = lane + 32 * u;
        if (i < m) {
          pc[i] = x[u];
          if (warp == 0 && i > p0) two_sum_acc(hi, lo, abs2(x[u]));
        }
      }
      if (warp == 0 && pw > 0) {
        const R below = warp_sum_compensated(hi, lo);
        qr_reflector_warp<R, MP>(pc, p0, m, below, zero_thresh2, lane, s_taus, s_ivs, tw, Vc + (p0 & 1) * MP);
      }
    }
    __syncthreads();
    // 2. factor the panel in shared memory: reflector j is ready; every warp
    // applies it to one later panel column, and the warp holding column j + 1
    // also forms reflector j + 1 from that column's fresh norm -- one barrier
    // per column
    for (int jj = 0; jj < pw; ++jj) {
      const int j = p0 + jj;
      const R tau = s_taus[j];
      const int cl = jj + 1 + warp;  // one panel column per warp, rows in registers
      if (cl < pcols) {
        cplx<R>* colc = P + (size_t)cl * m;
        cplx<R> xr[RPL];
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int i = lane + 32 * u;
          xr[u] = i < m ? colc[i] : cplx<R>(0, 0);
        }
        if (tau != R(0)) {
          reflect(xr, Vc + (j & 1) * MP, tau, j);
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int i = lane + 32 * u;
            if (i >= j && i < m) colc[i] = xr[u];
          }
        }
        if (cl == jj + 1 && jj + 1 < pw) {
          R hi = 0, lo = 0;
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int i = lane + 32 * u;
            if (i >= j + 2 && i < m) two_sum_acc(hi, lo, abs2(xr[u]));
          }
          const R below = warp_sum_compensated(hi, lo);
          qr_reflector_warp<R, MP>(colc, j + 1, m, below, zero_thresh2, lane, s_taus, s_ivs, tw,
                                   Vc + ((j + 1) & 1) * MP);
        }
      }
      __syncthreads();
    }
    // 3. panel back to the workspace (R above, reflectors below the diagonal)
    for (int e = threadIdx.x; e < pcols * m; e += blockDim.x) {
      const int cc = e / m, i = e - cc * m;
      W[(int64_t)(p0 + cc) * m + i] = P[(size_t)cc * m + i];
    }
    __syncthreads();
  }
  if (out) {
    cplx<R>* Rb = out + b * out_bstride;
    for (int64_t e = threadIdx.x; e < (int64_t)kmax * n; e += blockDim.x) {
      const int64_t i = e / n, c = e - i * n;
      Rb[i * ldr + c] = (c >= i) ? W[c * m + i] : cplx<R>(0, 0);
    }
  }
  if (Qout) {
    // NW columns of Q at a time, one per warp; the reflectors they need
    // (j <= c) are staged panel by panel, last panel first
    cplx<R>* Q = Qout + b * q_bstride;
    for (int g0 = 0; g0 < kmax; g0 += NW) {
      const int c = g0 + warp;
      cplx<R> x[RPL];
#pragma unroll
      for (int u = 0; u < RPL; ++u) x[u] = cplx<R>(lane + 32 * u == c ? R(1) : R(0), R(0));
      const int jmax = min(kmax - 1, g0 + NW - 1);
      for (int q0 = (jmax / NW) * NW; q0 >= 0; q0 -= NW) {
        const int qn = min(NW, kmax - q0);
        __syncthreads();
        stage(q0, qn);
        __syncthreads();
        if (c < kmax)
          for (int jj = qn - 1; jj >= 0; --jj) {
            const int j = q0 + jj;
            const R tau = s_taus[j];
            if (j <= c && tau != R(0)) reflect(x, S + (size_t)jj * MP, tau, j);
          }
      }
      if (c < kmax) {
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int i = lane + 32 * u;
          if (i < m) Q[(int64_t)i * ldq + c] = x[u];
        }
      }
    }
  }
}

template <class R, int RPL>
static int launch_qr_panel(const cplx<R>* in, MIdx inB, MIdx rowI, MIdx colI, int conj_in, int64_t m, int64_t n,
                           int64_t rows_total, int64_t rows_per_batch, int64_t batch, cplx<R>* W, cplx<R>* out,
                           int64_t out_bstride, int64_t ldr, cplx<R>* tauws, cplx<R>* Qout, int64_t q_bstride,
                           int64_t ldq, cudaStream_t s) {
  const int nw = qr_panel_warps<R, RPL>();
  const int64_t kmax = std::min(m, n);
  const size_t sm = ((size_t)nw * m + (size_t)(nw + 2) * 32 * RPL + kmax) * sizeof(cplx<R>) + (size_t)kmax * sizeof(R) +
                    16;
  if (sm > 200 * 1024) return QTT_ERR_UNSUPPORTED;
  if (qtt_allow_max_smem((const void*)qr_panel_kernel<R, RPL>) != QTT_OK) return QTT_ERR_CUDA;
  qr_panel_kernel<R, RPL><<<(unsigned)batch, 32 * nw, sm, s>>>(in, inB, rowI, colI, conj_in, (int)m, (int)n,
                                                                rows_total, rows_per_batch, W, out, out_bstride, ldr,
                                                                tauws, Qout, q_bstride, ldq);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

// ------------------------------------------------ blocked left-looking QR
// Householder QR, one CTA of 16 warps per matrix, m <= 32 * RPL rows, in
// panels of QB = 16 columns with the compact WY form of each panel's
// reflectors: H_{p0} ... H_{p0+15} = I - V T V^H, T upper triangular
// (T_kk = tau_k, T_{0:k,k} = -tau_k T_{0:k,0:k} V_{:,0:k}^H v_k).
//   * A panel (all m rows, in shared memory) first receives every earlier
//     panel q as one block update P <- P - V_q (T_q^H (V_q^H P)): the
//     reflectors of q staged from the workspace W, T_q kept in shared memory;
//     three small products instead of sixteen rank-1 updates with a warp
//     reduction each.
//   * The panel is then factored in shared memory column by column (every
//     warp applies reflector j to one later panel column, the warp holding
//     column j + 1 forms reflector j + 1; one barrier per column), written
//     back to W (R above, reflectors below the diagonal), and T of the panel
//     built from the Gram matrix of its reflectors.
//   * The explicit Q is formed backwards from [I; 0]: for the panels from the
//     last to the first, Q[p0:, c0:c0+16] <- X - V (T (V^H X)) for every
//     16-column chunk c0 >= p0 (read from and written to Qout).
// Same inputs, outputs, reflector format (W, 1/v0 and tau per column) and
// zero-column rule as qr_panel_kernel.
constexpr int QB = 16;

// Building blocks of the blocked QR kernels (512 threads; S, X: QB columns of
// ldp complex values in shared memory, column-major).
//
// S <- the scaled reflectors q0 .. q0+qn-1 (column k: 0 above row q0+k, 1
// there, x_i / v0 below; zero for tau = 0 and for k >= qn), whose unscaled
// entries are column k of src (stride ld); taus / ivs indexed by reflector.
template <class R>
__device__ __forceinline__ void qb_stage(cplx<R>* S, int ldp, const cplx<R>* src, int ld, int q0, int qn, int m,
                                         const R* taus, const cplx<R>* ivs) {
  for (int e = threadIdx.x; e < QB * m; e += blockDim.x) {
    const int k = e / m, i = e - k * m, j = q0 + k;
    cplx<R> v(0, 0);
    if (k < qn && taus[j] != R(0))
      v = i > j ? src[(size_t)k * ld + i] * ivs[j] : cplx<R>(i == j ? R(1) : R(0), R(0));
    S[(size_t)k * ldp + i] = v;
  }
}

// Yb[k][c] = sum over rows i >= r0 of conj(S[k][i]) X[c][i]: each thread sums
// the outputs (k, c), (k, c+8), (k+8, c), (k+8, c+8) over every eighth row,
// the eight row groups of an output being adjacent lanes (reduced by shuffles)
template <class R>
__device__ __forceinline__ void qb_vhx(const cplx<R>* S, const cplx<R>* X, int ldp, int r0, int m, cplx<R>* Yb) {
  const int tid = threadIdx.x, g = tid & 7, q = tid >> 3, kq = q >> 3, cq = q & 7;
  const cplx<R>* s0 = S + (size_t)kq * ldp;
  const cplx<R>* s1 = S + (size_t)(kq + 8) * ldp;
  const cplx<R>* x0 = X + (size_t)cq * ldp;
  const cplx<R>* x1 = X + (size_t)(cq + 8) * ldp;
  cplx<R> a00(0, 0), a01(0, 0), a10(0, 0), a11(0, 0);
  for (int i = r0 + g; i < m; i += 8) {
    const cplx<R> u0 = s0[i], u1 = s1[i], y0 = x0[i], y1 = x1[i];
    cfma_conj(a00, u0, y0);
    cfma_conj(a01, u0, y1);
    cfma_conj(a10, u1, y0);
    cfma_conj(a11, u1, y1);
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    a00.re += __shfl_xor_sync(0xffffffffu, a00.re, o);
    a00.im += __shfl_xor_sync(0xffffffffu, a00.im, o);
    a01.re += __shfl_xor_sync(0xffffffffu, a01.re, o);
    a01.im += __shfl_xor_sync(0xffffffffu, a01.im, o);
    a10.re += __shfl_xor_sync(0xffffffffu, a10.re, o);
    a10.im += __shfl_xor_sync(0xffffffffu, a10.im, o);
    a11.re += __shfl_xor_sync(0xffffffffu, a11.re, o);
    a11.im += __shfl_xor_sync(0xffffffffu, a11.im, o);
  }
  if (g == 0) {
    Yb[kq * QB + cq] = a00;
    Yb[kq * QB + cq + 8] = a01;
    Yb[(kq + 8) * QB + cq] = a10;
    Yb[(kq + 8) * QB + cq + 8] = a11;
  }
}

// X[c][i] -= sum_k S[k][i] Zb[k][c] for rows i >= r0 and columns c < ncols,
// one row per thread (its QB reflector entries in registers, Zb broadcast)
template <class R>
__device__ __forceinline__ void qb_update(const cplx<R>* S, const cplx<R>* Zb, cplx<R>* X, int ldp, int r0, int m,
                                          int ncols) {
  for (int i = r0 + threadIdx.x; i < m; i += blockDim.x) {
    cplx<R> sv[QB];
#pragma unroll
    for (int kk = 0; kk < QB; ++kk) sv[kk] = S[(size_t)kk * ldp + i];
#pragma unroll
    for (int c = 0; c < QB; ++c) {
      if (c >= ncols) break;
      cplx<R> acc(0, 0);
#pragma unroll
      for (int kk = 0; kk < QB; ++kk) cfma(acc, sv[kk], Zb[kk * QB + c]);
      X[(size_t)c * ldp + i] = X[(size_t)c * ldp + i] - acc;
    }
  }
}

template <class R, int RPL>
static size_t qr_blocked_bytes(int m, int n) {
  const int kmax = m < n ? m : n, npan = (kmax + QB - 1) / QB, ldp = m | 1;
  return ((size_t)2 * QB * ldp + (size_t)npan * QB * QB + (size_t)2 * QB * QB + 2 * 32 * RPL + kmax) *
             sizeof(cplx<R>) + (size_t)kmax * sizeof(R) + 16;
}

template <class R, int RPL>
__global__ void __launch_bounds__(32 * QB, 1)
qr_blocked_kernel(const cplx<R>* __restrict__ in, MIdx inB, MIdx rowI, MIdx colI, int conj_in, int m, int n,
                  int64_t rows_total, int64_t rows_per_batch, cplx<R>* __restrict__ Wbase, cplx<R>* __restrict__ out,
                  int64_t out_bstride, int64_t ldr, cplx<R>* __restrict__ tauws, cplx<R>* __restrict__ Qout,
                  int64_t q_bstride, int64_t ldq, cplx<R>* __restrict__ Tg) {
  constexpr int MP = 32 * RPL;  // rows padded to whole warps (the panel factorisation's registers)
  constexpr int NT = 32 * QB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int kmax = m < n ? m : n;
  const int npan = (kmax + QB - 1) / QB;
  const int ldp = m | 1;  // odd column stride: lanes on different columns of one row hit different banks
  cplx<R>* P = reinterpret_cast<cplx<R>*>(smem_raw);  // QB columns of ldp: the panel, or a chunk of Q
  cplx<R>* S = P + (size_t)QB * ldp;                   // QB staged scaled reflectors
  cplx<R>* Tall = S + (size_t)QB * ldp;                // npan x QB x QB, T_q[l][k] row-major
  cplx<R>* Yb = Tall + (size_t)npan * QB * QB;         // QB x QB: V^H X
  cplx<R>* Zb = Yb + QB * QB;                          // QB x QB
  cplx<R>* Vc = Zb + QB * QB;                          // 2 x MP reflector being applied in the panel
  cplx<R>* s_ivs = Vc + 2 * MP;                        // 1/v0 per reflector
  R* s_taus = reinterpret_cast<R*>(s_ivs + kmax);      // tau per reflector
  __shared__ R red[32];
  const int64_t b = blockIdx.x;
  cplx<R>* W = Wbase + b * (int64_t)m * n;
  cplx<R>* tw = tauws ? tauws + b * 2 * n : nullptr;
  const int64_t row0 = b * rows_per_batch;
  int64_t valid = rows_total - row0;
  if (valid > m) valid = m;
  const int64_t ib = midx_off(inB, b);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  R part = 0;
  for (int c = warp; c < n; c += QB)
    for (int i = lane; i < valid; i += 32) part += abs2(in[ib + midx_off(rowI, i) + midx_off(colI, c)]);
  const R anorm2 = block_sum(part, red);
  const R eps = sizeof(R) == 8 ? R(DBL_EPSILON) : R(FLT_EPSILON);
  const R zero_thresh2 = eps * eps * anorm2;
  // x <- (I - tau v v^H) x for a register column and the scaled reflector in
  // shared memory (zero above its diagonal row and from row m; the row count
  // is padded only to whole warps, so every slice is processed -- measured
  // faster than testing which slices meet the nonzero rows)
  auto reflect = [&](cplx<R>(&x)[RPL], const cplx<R>* v, R tau) {
    cplx<R> w(0, 0), w1(0, 0);
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      if (u & 1) cfma_conj(w1, v[lane + 32 * u], x[u]); else cfma_conj(w, v[lane + 32 * u], x[u]);
    }
    w = w + w1;
    w.re = warp_sum(w.re);
    w.im = warp_sum(w.im);
    w = tau * w;
#pragma unroll
    for (int u = 0; u < RPL; ++u) x[u] = x[u] - v[lane + 32 * u] * w;
  };
  // ---------------- R
  for (int p0 = 0, pi = 0; p0 < n; p0 += QB, ++pi) {
    const int pcols = min(QB, n - p0);
    const int pw = max(0, min(QB, kmax - p0));  // reflectors formed in this panel
    __syncthreads();  // the previous panel's reads of P are done
    for (int e = tid; e < pcols * m; e += NT) {
      const int c = e / m, i = e - c * m;
      cplx<R> v(0, 0);
      if (i < valid) {
        v = in[ib + midx_off(rowI, i) + midx_off(colI, p0 + c)];
        if (conj_in) v.im = -v.im;
      }
      P[(size_t)c * ldp + i] = v;
    }
    // every earlier panel as one block update: P <- P - V (T^H (V^H P))
    for (int q0 = 0, qi = 0; q0 < p0 && q0 < kmax; q0 += QB, ++qi) {
      const int qn = min(QB, kmax - q0);
      __syncthreads();
      qb_stage(S, ldp, W + (size_t)q0 * m, m, q0, qn, m, s_taus, s_ivs);
      __syncthreads();
      qb_vhx(S, P, ldp, q0, m, Yb);
      __syncthreads();
      if (tid < QB * QB) {
        const int k = tid / QB, c = tid - k * QB;
        const cplx<R>* T = Tall + (size_t)qi * QB * QB;
        cplx<R> z(0, 0);
        for (int l = 0; l <= k; ++l) cfma_conj(z, T[l * QB + k], Yb[l * QB + c]);
        Zb[tid] = z;
      }
      __syncthreads();
      qb_update(S, Zb, P, ldp, q0, m, pcols);
    }
    __syncthreads();
    // factor the panel: warp w keeps panel column w in registers (rows on
    // lanes).  Step jj: warp jj forms reflector p0 + jj from its column (norm
    // below the diagonal, scalars in every lane), writes the finished column
    // to P and the scaled reflector to Vc; after the barrier the warps of the
    // later columns apply it.  The warp that forms the next reflector thus
    // goes straight from applying this one to forming its own.
    cplx<R> xr[RPL];
    {
      const cplx<R>* col = P + (size_t)warp * ldp;
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        const int i = lane + 32 * u;
        xr[u] = warp < pcols && i < m ? col[i] : cplx<R>(0, 0);
      }
    }
    for (int jj = 0; jj < pw; ++jj) {
      const int j = p0 + jj;
      if (warp == jj) {
        R hi = 0, lo = 0;
        cplx<R> x0(0, 0);
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int i = lane + 32 * u;
          if (i > j && i < m) two_sum_acc(hi, lo, abs2(xr[u]));
          if (i == j) x0 = xr[u];
        }
        const R below = warp_sum_compensated(hi, lo);
        x0.re = warp_sum(x0.re);  // one lane holds row j, the others add zeros
        x0.im = warp_sum(x0.im);
        const R ax2 = abs2(x0), nrm2 = below + ax2;
        const bool zero = nrm2 <= zero_thresh2 || below <= zero_thresh2;
        R tau = R(0);
        cplx<R> iv(0, 0), diag = nrm2 <= zero_thresh2 ? cplx<R>(0, 0) : x0;
        if (!zero) {
          const R ax0 = sqrt(ax2), nrm = sqrt(nrm2);
          const R phr = ax0 > R(0) ? x0.re / ax0 : R(1), phi = ax0 > R(0) ? x0.im / ax0 : R(0);
          const R s0 = ax0 + nrm;
          const R v02 = s0 * s0;
          tau = R(2) * v02 / (below + v02);
          iv = cplx<R>(phr / s0, -phi / s0);
          diag = cplx<R>(-phr * nrm, -phi * nrm);
        }
        cplx<R>* col = P + (size_t)jj * ldp;
        cplx<R>* vs = Vc + (j & 1) * MP;
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int i = lane + 32 * u;
          if (32 * u >= m) {
            vs[i] = cplx<R>(0, 0);
            continue;
          }
          const cplx<R> x = i == j ? diag : (i > j && zero ? cplx<R>(0, 0) : xr[u]);
          if (i < m) col[i] = x;
          vs[i] = i > j && i < m ? x * iv : cplx<R>(i == j ? R(1) : R(0), R(0));
        }
        if (lane == 0) {
          s_taus[j] = tau;
          s_ivs[j] = iv;
          if (tw) {
            tw[2 * j] = iv;
            tw[2 * j + 1] = cplx<R>(tau, R(0));
          }
        }
      }
      __syncthreads();
      if (warp > jj && warp < pcols) {
        const R tau = s_taus[j];
        if (tau != R(0)) reflect(xr, Vc + (j & 1) * MP, tau);
      }
    }
    // columns past the last reflector (n > m) go back as they are
    if (warp >= pw && warp < pcols) {
      cplx<R>* col = P + (size_t)warp * ldp;
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        const int i = lane + 32 * u;
        if (i < m) col[i] = xr[u];
      }
    }
    __syncthreads();
    // panel back to W; T of the panel from the Gram matrix of its reflectors
    for (int e = tid; e < pcols * m; e += NT) {
      const int c = e / m, i = e - c * m;
      W[(size_t)(p0 + c) * m + i] = P[(size_t)c * ldp + i];
    }
    if (pw > 0) {
      qb_stage(S, ldp, P, ldp, p0, pw, m, s_taus, s_ivs);
      __syncthreads();
      qb_vhx(S, S, ldp, p0, m, Yb);
      cplx<R>* T = Tall + (size_t)pi * QB * QB;
      if (tid < QB * QB) {
        const int l = tid / QB, k = tid - l * QB;
        T[tid] = l == k && k < pw ? cplx<R>(s_taus[p0 + k], R(0)) : cplx<R>(0, 0);
      }
      __syncthreads();
      for (int k = 1; k < pw; ++k) {
        if (tid < k) {
          const int l = tid;
          cplx<R> acc(0, 0);
          for (int jx = l; jx < k; ++jx) cfma(acc, T[l * QB + jx], Yb[jx * QB + k]);
          const R tk = s_taus[p0 + k];
          T[l * QB + k] = cplx<R>(-tk * acc.re, -tk * acc.im);
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();
  if (out) {
    cplx<R>* Rb = out + b * out_bstride;
    for (int64_t e = tid; e < (int64_t)kmax * n; e += NT) {
      const int64_t i = e / n, c = e - i * n;
      Rb[i * ldr + c] = (c >= i) ? W[c * m + i] : cplx<R>(0, 0);
    }
  }
  if (!Qout) return;
  if (Tg) {
    // Q is formed by qr_form_q_kernel, one CTA per 16-column chunk: hand the T factors over
    cplx<R>* Tb = Tg + b * (int64_t)npan * QB * QB;
    for (int e = tid; e < npan * QB * QB; e += NT) Tb[e] = Tall[e];
    return;
  }
  // ---------------- explicit Q, backwards from [I; 0]
  cplx<R>* Q = Qout + b * q_bstride;
  for (int64_t e = tid; e < (int64_t)m * kmax; e += NT) {
    const int64_t i = e / kmax, c = e - i * kmax;
    Q[i * ldq + c] = cplx<R>(i == c ? R(1) : R(0), R(0));
  }
  for (int pi = npan - 1; pi >= 0; --pi) {
    const int p0 = pi * QB, qn = min(QB, kmax - p0);
    __syncthreads();
    qb_stage(S, ldp, W + (size_t)p0 * m, m, p0, qn, m, s_taus, s_ivs);
    const cplx<R>* T = Tall + (size_t)pi * QB * QB;
    for (int c0 = p0; c0 < kmax; c0 += QB) {
      const int ncols = min(QB, kmax - c0);
      __syncthreads();
      for (int e = tid; e < (m - p0) * QB; e += NT) {
        const int i = p0 + (e >> 4), c = e & (QB - 1);
        P[(size_t)c * ldp + i] = c < ncols ? Q[(int64_t)i * ldq + c0 + c] : cplx<R>(0, 0);
      }
      __syncthreads();
      qb_vhx(S, P, ldp, p0, m, Yb);
      __syncthreads();
      if (tid < QB * QB) {
        const int k = tid / QB, c = tid - k * QB;
        cplx<R> z(0, 0);
        for (int l = k; l < QB; ++l) cfma(z, T[k * QB + l], Yb[l * QB + c]);
        Zb[tid] = z;
      }
      __syncthreads();
      qb_update(S, Zb, P, ldp, p0, m, ncols);
      __syncthreads();
      for (int e = tid; e < (m - p0) * QB; e += NT) {
        const int i = p0 + (e >> 4), c = e & (QB - 1);
        if (c < ncols) Q[(int64_t)i * ldq + c0 + c] = P[(size_t)c * ldp + i];
      }
    }
  }
}

// Explicit Q of the blocked QR, m x min(m, n): CTA ci forms columns 16 ci ..
// 16 ci + 15 in shared memory, starting from the identity columns and
// applying the block reflectors of panels ci, ci - 1, ..., 0 in that order
// (X <- X - V_p (T_p (V_p^H X)) on rows >= 16 p).  The chunks are independent,
// so the backward accumulation runs on as many SMs as there are panels.
// Reads the reflectors (W), the (1/v0, tau) pairs (tauws) and the T factors
// (Tg, npan x 16 x 16 per matrix) that qr_blocked_kernel left.
template <class R>
__global__ void __launch_bounds__(32 * QB, 1)
qr_form_q_kernel(const cplx<R>* __restrict__ Wbase, int m, int n, const cplx<R>* __restrict__ Tg,
                 const cplx<R>* __restrict__ tauws, cplx<R>* __restrict__ Qout, int64_t q_bstride, int64_t ldq) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int kmax = m < n ? m : n, npan = (kmax + QB - 1) / QB, ldp = m | 1;
  const int tid = threadIdx.x, ci = blockIdx.x, c0 = ci * QB, ncols = min(QB, kmax - c0);
  const int64_t b = blockIdx.y;
  cplx<R>* X = reinterpret_cast<cplx<R>*>(smem_raw);  // QB x ldp
  cplx<R>* S = X + (size_t)QB * ldp;                   // QB x ldp
  cplx<R>* Yb = S + (size_t)QB * ldp;
  cplx<R>* Zb = Yb + QB * QB;
  cplx<R>* T = Zb + QB * QB;
  cplx<R>* ivs = T + QB * QB;                          // kmax
  R* taus = reinterpret_cast<R*>(ivs + kmax);          // kmax
  const cplx<R>* W = Wbase + b * (int64_t)m * n;
  const cplx<R>* tw = tauws + b * 2 * n;
  const cplx<R>* Tb = Tg + b * (int64_t)npan * QB * QB;
  for (int j = tid; j < kmax; j += blockDim.x) {
    ivs[j] = tw[2 * j];
    taus[j] = tw[2 * j + 1].re;
  }
  for (int e = tid; e < QB * m; e += blockDim.x) {
    const int c = e / m, i = e - c * m;
    X[(size_t)c * ldp + i] = cplx<R>(c < ncols && i == c0 + c ? R(1) : R(0), R(0));
  }
  for (int p = ci; p >= 0; --p) {
    const int p0 = p * QB, qn = min(QB, kmax - p0);
    __syncthreads();
    qb_stage(S, ldp, W + (size_t)p0 * m, m, p0, qn, m, taus, ivs);
    for (int e = tid; e < QB * QB; e += blockDim.x) T[e] = Tb[(size_t)p * QB * QB + e];
    __syncthreads();
    qb_vhx(S, X, ldp, p0, m, Yb);
    __syncthreads();
    if (tid < QB * QB) {
      const int k = tid / QB, c = tid - k * QB;
      cplx<R> z(0, 0);
      for (int l = k; l < QB; ++l) cfma(z, T[k * QB + l], Yb[l * QB + c]);
      Zb[tid] = z;
    }
    __syncthreads();
    qb_update(S, Zb, X, ldp, p0, m, ncols);
  }
  __syncthreads();
  cplx<R>* Q = Qout + b * q_bstride;
  for (int e = tid; e < m * QB; e += blockDim.x) {
    const int i = e / QB, c = e - i * QB;
    if (c < ncols) Q[(int64_t)i * ldq + c0 + c] = X[(size_t)c * ldp + i];
  }
}

template <class R>
static size_t qr_form_q_bytes(int m, int n) {
  const int kmax = m < n ? m : n, ldp = m | 1;
  return ((size_t)2 * QB * ldp + (size_t)3 * QB * QB + kmax) * sizeof(cplx<R>) + (size_t)kmax * sizeof(R) + 16;
}

template <class R, int RPL>
static int launch_qr_blocked(const cplx<R>* in, MIdx inB, MIdx rowI, MIdx colI, int conj_in, int64_t m, int64_t n,
                             int64_t rows_total, int64_t rows_per_batch, int64_t batch, cplx<R>* W, cplx<R>* out,
                             int64_t out_bstride, int64_t ldr, cplx<R>* tauws, cplx<R>* Qout, int64_t q_bstride,
                             int64_t ldq, cplx<R>* Qws, cudaStream_t s) {
  const size_t sm = qr_blocked_bytes<R, RPL>((int)m, (int)n);
  if (sm > 200 * 1024) return QTT_ERR_UNSUPPORTED;
  const int64_t kmax = std::min(m, n), npan = (kmax + QB - 1) / QB;
  // the explicit Q by the chunk-parallel kernel where the workspace can hold
  // the T factors and the (1/v0, tau) pairs are kept
  const bool split_q = Qout && tauws && Qws && npan * QB * QB <= m * kmax &&
                       qr_form_q_bytes<R>((int)m, (int)n) <= 200 * 1024;
  if (qtt_allow_max_smem((const void*)qr_blocked_kernel<R, RPL>) != QTT_OK) return QTT_ERR_CUDA;
  qr_blocked_kernel<R, RPL><<<(unsigned)batch, 32 * QB, sm, s>>>(in, inB, rowI, colI, conj_in, (int)m, (int)n,
                                                                  rows_total, rows_per_batch, W, out, out_bstride,
                                                                  ldr, tauws, Qout, q_bstride, ldq,
                                                                  split_q ? Qws : nullptr);
  if (split_q) {
    if (qtt_allow_max_smem((const void*)qr_form_q_kernel<R>) != QTT_OK) return QTT_ERR_CUDA;
    qr_form_q_kernel<R><<<dim3((unsigned)npan, (unsigned)batch), 32 * QB, qr_form_q_bytes<R>((int)m, (int)n), s>>>(
        W, (int)m, (int)n, Qws, tauws, Qout, q_bstride, ldq);
  }
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template <class R>
int qtt_qr_r(const cplx<R>* in, MIdx inB, MIdx rowI, MIdx colI, int conj_in, int64_t m, int64_t n,
             int64_t rows_total, int64_t rows_per_batch, int64_t batch, cplx<R>* W, cplx<R>* out,
             int64_t out_bstride, int64_t ldr, cudaStream_t s, cplx<R>* tauws, cplx<R>* Qout,
             int64_t q_bstride, int64_t ldq, cplx<R>* Qws) {
  if (batch <= 0 || m <= 0 || n <= 0) return QTT_OK;
  if (batch > 65535 || m > INT32_MAX || n > INT32_MAX) return QTT_ERR_ARG;
  // FP32: the blocked kernel where its shared memory fits; else the panel
  // kernel for up to 512 rows (256 in FP64); else the workspace kernel
  if constexpr (sizeof(R) == 4) {
    int st = QTT_ERR_UNSUPPORTED;
    if (m <= 128)
      st = launch_qr_blocked<R, 4>(in, inB, rowI, colI, conj_in, m, n, rows_total, rows_per_batch, batch, W, out,
                                   out_bstride, ldr, tauws, Qout, q_bstride, ldq, Qws, s);
    else if (m <= 256)
      st = launch_qr_blocked<R, 8>(in, inB, rowI, colI, conj_in, m, n, rows_total, rows_per_batch, batch, W, out,
                                   out_bstride, ldr, tauws, Qout, q_bstride, ldq, Qws, s);
    else if (m <= 288)  // 2 x 136 rows: the projection QR of sketch width 136
      st = launch_qr_blocked<R, 9>(in, inB, rowI, colI, conj_in, m, n, rows_total, rows_per_batch, batch, W, out,
                                   out_bstride, ldr, tauws, Qout, q_bstride, ldq, Qws, s);
    else if (m <= 512)
      st = launch_qr_blocked<R, 16>(in, inB, rowI, colI, conj_in, m, n, rows_total, rows_per_batch, batch, W, out,
                                    out_bstride, ldr, tauws, Qout, q_bstride, ldq, Qws, s);
    if (st != QTT_ERR_UNSUPPORTED) return st;
  }
  {
    int st = QTT_ERR_UNSUPPORTED;
    if (m <= 128)
      st = launch_qr_panel<R, 4>(in, inB, rowI, colI, conj_in, m, n, rows_total, rows_per_batch, batch, W, out,
                                 out_bstride, ldr, tauws, Qout, q_bstride, ldq, s);
    else if (m <= 256)
      st = launch_qr_panel<R, 8>(in, inB, rowI, colI, conj_in, m, n, rows_total, rows_per_batch, batch, W, out,
                                 out_bstride, ldr, tauws, Qout, q_bstride, ldq, s);
    else if constexpr (sizeof(R) == 4) {
      if (m <= 512)
        st = launch_qr_panel<R, 16>(in, inB, rowI, colI, conj_in, m, n, rows_total, rows_per_batch, batch, W, out,
                                    out_bstride, ldr, tauws, Qout, q_bstride, ldq, s);
    }
    if (st != QTT_ERR_UNSUPPORTED) return st;
  }
  if (Qout && (!tauws || !Qws)) return QTT_ERR_ARG;
  qr_r_kernel<R><<<(unsigned)batch, 1024, 0, s>>>(in, inB, rowI, colI, conj_in, m, n, rows_total,
                                                 rows_per_batch, W, out, out_bstride, ldr, tauws, Qout,
                                                 q_bstride, ldq, Qws);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template <class R>
int qtt_jacobi(cplx<R>* G, cplx<R>* Vwork, R* sigma, cplx<R>* Vsorted, int p, int q, int batch,
               int max_sweeps, int* sweeps, cudaStream_t s, cplx<R>* Usorted) {
  if (batch <= 0 || q <= 0) return QTT_OK;
  int qe = q + (q & 1);
  size_t sm = (size_t)(qe + (qe & 1)) * sizeof(int) + (size_t)q * sizeof(R) + 16;
  if (sm > 48 * 1024 && qtt_allow_max_smem((const void*)jacobi_kernel<R>) != QTT_OK) return QTT_ERR_CUDA;
  jacobi_kernel<R><<<(unsigned)batch, 256, sm, s>>>(G, Vwork, sigma, Vsorted, Usorted, p, q, max_sweeps, sweeps);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

// one block per matrix of a batch: sigma q apart, delta per matrix, out[4 b
// .. 4 b + 3] = (t, capped, tail as a double)
template <class R>
__global__ void trunc_rank_batch_kernel(const R* __restrict__ s, int q, const double* __restrict__ delta,
                                        int max_rank, int* __restrict__ out) {
  const int b = blockIdx.x;
  if (threadIdx.x == 0)
    trunc_rank_body<R>(s + (size_t)b * q, q, delta[b], max_rank, out + 4 * b,
                       reinterpret_cast<double*>(out + 4 * b + 2));
}

template <class R>
int qtt_trunc_rank_batch(const R* sigma, int q, const double* delta, int max_rank, int* out, int batch,
                         cudaStream_t s) {
  if (batch < 1) return QTT_OK;
  trunc_rank_batch_kernel<R><<<batch, 32, 0, s>>>(sigma, q, delta, max_rank, out);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}
template int qtt_trunc_rank_batch<double>(const double*, int, const double*, int, int*, int, cudaStream_t);
template int qtt_trunc_rank_batch<float>(const float*, int, const double*, int, int*, int, cudaStream_t);

template <class R>
int qtt_trunc_rank(const R* sigma, int q, double delta, int max_rank, int* out, double* tail, cudaStream_t s) {
  trunc_rank_kernel<R><<<1, 32, 0, s>>>(sigma, q, delta, max_rank, out, tail);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template int qtt_qr_r<double>(const zc*, MIdx, MIdx, MIdx, int, int64_t, int64_t, int64_t, int64_t, int64_t,
                              zc*, zc*, int64_t, int64_t, cudaStream_t, zc*, zc*, int64_t, int64_t, zc*);
template int qtt_qr_r<float>(const cc*, MIdx, MIdx, MIdx, int, int64_t, int64_t, int64_t, int64_t, int64_t,
                             cc*, cc*, int64_t, int64_t, cudaStream_t, cc*, cc*, int64_t, int64_t, cc*);
template int qtt_jacobi<double>(zc*, zc*, double*, zc*, int, int, int, int, int*, cudaStream_t, zc*);
template int qtt_jacobi<float>(cc*, cc*, float*, cc*, int, int, int, int, int*, cudaStream_t, cc*);
template int qtt_trunc_rank<double>(const double*, int, double, int, int*, double*, cudaStream_t);
template int qtt_trunc_rank<float>(const float*, int, double, int, int*, double*, cudaStream_t);

// Multi-CTA one-sided Jacobi (batch 1): one launch per round, a device flag
// per sweep read by the host (one synchronisation per sweep, at most
// max_sweeps sweeps).  Gwork needs p*q elements, Vwork q*q.
template <class R>
int qtt_jacobi_wide(const cplx<R>* G, cplx<R>* Gwork, cplx<R>* Vwork, R* sigma, cplx<R>* Vsorted, cplx<R>* Usorted,
                    int p, int q, int max_sweeps, int* dflag, int* sweeps_done, int64_t* launches, cudaStream_t s) {
  if (q <= 0) return QTT_OK;
  if (!Vsorted) Vwork = nullptr;  // rotations not wanted
  if (Vsorted && !Vwork) return QTT_ERR_ARG;
  const int64_t tot = (int64_t)p * q + (int64_t)q * q;
  jacobi_setup_kernel<R><<<(unsigned)std::min<int64_t>((tot + 255) / 256, 65535), 256, 0, s>>>(G, p, q, Gwork, Vwork);
  *launches += 1;
  const int qe = q + (q & 1);
  const int pairs = qe / 2;
  const unsigned blocks = (unsigned)((pairs * 32 + 255) / 256);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (cudaMemsetAsync(dflag, 0, sizeof(int), s) != cudaSuccess) return QTT_ERR_CUDA;
    for (int r = 0; r < qe - 1; ++r)
      jacobi_round_kernel<R><<<blocks, 256, 0, s>>>(Gwork, Vwork, p, q, r, dflag);
    *launches += qe - 1;
    int h = 0;
    if (cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return QTT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return QTT_ERR_CUDA;
    if (!h) {
      ++sweep;
      break;
    }
  }
  if (sweeps_done) *sweeps_done = sweep;
  size_t sm = (size_t)q * sizeof(R);
  if (sm > 48 * 1024 && qtt_allow_max_smem((const void*)jacobi_finish_kernel<R>) != QTT_OK) return QTT_ERR_CUDA;
  jacobi_finish_kernel<R><<<1, 256, sm, s>>>(Gwork, Vwork, p, q, sigma, Vsorted, Usorted);
  *launches += 1;
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template int qtt_jacobi_wide<double>(const zc*, zc*, zc*, double*, zc*, zc*, int, int, int, int*, int*, int64_t*,
                                     cudaStream_t);
template int qtt_jacobi_wide<float>(const cc*, cc*, cc*, float*, cc*, cc*, int, int, int, int*, int*, int64_t*,
                                    cudaStream_t);

template <class R>
size_t qtt_jacobi_smem_bytes(int p, int q) { return (size_t)p * q * sizeof(cplx<R>) + (size_t)q * sizeof(R) + 16; }

template <class R>
int qtt_jacobi_smem(const cplx<R>* G, cplx<R>* Vws, R* sigma, cplx<R>* Vsorted, cplx<R>* Usorted, int p, int q,
                    int max_sweeps, int* sweeps, cudaStream_t s) {
  if (q <= 0) return QTT_OK;
  size_t sm = qtt_jacobi_smem_bytes<R>(p, q);
  if (sm > 227 * 1024) return QTT_ERR_RANK;
  if (qtt_allow_max_smem((const void*)jacobi_smem_kernel<R>) != QTT_OK) return QTT_ERR_CUDA;
  jacobi_smem_kernel<R><<<1, 1024, sm, s>>>(G, Vws, sigma, Vsorted, Usorted, p, q, max_sweeps, sweeps);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template size_t qtt_jacobi_smem_bytes<double>(int, int);
template size_t qtt_jacobi_smem_bytes<float>(int, int);
template int qtt_jacobi_smem<double>(const zc*, zc*, double*, zc*, zc*, int, int, int, int*, cudaStream_t);
template int qtt_jacobi_smem<float>(const cc*, cc*, float*, cc*, cc*, int, int, int, int*, cudaStream_t);

template <class R, int NC>
static size_t jacobi_cluster_bytes(int p, int q) {
  const int qe = q + (q & 1);
  const int chunk = (p + NC - 1) / NC, chunkv = (q + NC - 1) / NC;
  size_t off = (size_t)(2 * NC * (qe / 2) * 4 + NC * q + q) * sizeof(R);
  off = (off + 15) & ~(size_t)15;
  return off + (size_t)q * (chunk + chunkv) * sizeof(cplx<R>);
}

template <class R, int NC>
static int launch_jacobi_cluster(const cplx<R>* G, R* sigma, cplx<R>* Vs, cplx<R>* Us, int p, int q, int max_sweeps,
                                 int* sweeps, cudaStream_t s) {
  const size_t sm = jacobi_cluster_bytes<R, NC>(p, q);
  if (qtt_allow_max_smem((const void*)jacobi_cluster_kernel<R, NC>) != QTT_OK) return QTT_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(NC, 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = NC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<R, NC>, G, sigma, Vs, Us, p, q, max_sweeps, sweeps) !=
      cudaSuccess)
    return QTT_ERR_CUDA;
  return QTT_OK;
}

// Shared-memory bytes per CTA of the cluster Jacobi for the given cluster size
// (0 if that size is not compiled).
template <class R>
size_t qtt_jacobi_cluster_bytes(int p, int q, int nc) {
  switch (nc) {
    case 4: return jacobi_cluster_bytes<R, 4>(p, q);
    case 8: return jacobi_cluster_bytes<R, 8>(p, q);
    default: return 0;
  }
}

template <class R>
int qtt_jacobi_cluster(const cplx<R>* G, R* sigma, cplx<R>* Vsorted, cplx<R>* Usorted, int p, int q, int nc,
                       int max_sweeps, int* sweeps, cudaStream_t s) {
  if (q <= 0) return QTT_OK;
  int st;
  switch (nc) {
    case 4: st = launch_jacobi_cluster<R, 4>(G, sigma, Vsorted, Usorted, p, q, max_sweeps, sweeps, s); break;
    case 8: st = launch_jacobi_cluster<R, 8>(G, sigma, Vsorted, Usorted, p, q, max_sweeps, sweeps, s); break;
    default: return QTT_ERR_ARG;
  }
  if (st) return st;
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template size_t qtt_jacobi_cluster_bytes<double>(int, int, int);
template size_t qtt_jacobi_cluster_bytes<float>(int, int, int);
template int qtt_jacobi_cluster<double>(const zc*, double*, zc*, zc*, int, int, int, int, int*, cudaStream_t);
template int qtt_jacobi_cluster<float>(const cc*, float*, cc*, cc*, int, int, int, int, int*, cudaStream_t);

// ------------------------------------- block-cyclic one-sided Jacobi (cluster)
// Columns split, not rows: the q columns (padded with zero columns to
// 2*NC*bs, bs even) form NB = 2*NC blocks of bs whole columns, and CTA i of
// the cluster holds the blocks at tournament positions i ("top") and NB-1-i
// ("bottom"); at block-round r of a sweep position j holds block 0 (j = 0) or
// 1 + (j - 1 + r) mod (NB - 1), the round-robin tournament of the blocks.  In
// a block-round every CTA rotates all bs*bs cross pairs of its two blocks (bs
// rounds of bs disjoint pairs: top column w with bottom column (w + s) mod
// bs, one warp per pair, the top column kept in registers); in the first
// block-round of a sweep also the pairs inside each block (bs - 1 rounds of
// the round-robin of bs columns).  A sweep thus rotates every column pair
// once, like the scalar orderings, but needs a cluster barrier only at the
// NB - 1 block exchanges (each block moves one position down the tournament,
// copied into the receiving CTA's spare slots through distributed shared
// memory), not at every round.  NB - 1 exchanges bring every block back to
// its starting CTA, so at a sweep boundary CTA i holds blocks i and NB-1-i.
// Rotation parameters and the stopping rule are those of the other Jacobi
// kernels; the rotations are not accumulated (callers that need V use the
// other kernels).  Outputs: sigma sorted decreasingly and the normalised
// rotated columns (row-major p x q) in the same order.
template <class R, int RPL>
__device__ __forceinline__ bool warp_pair_rotate(cplx<R> (&x)[RPL], cplx<R> (&y)[RPL], R tol2, int p) {
  // two independent accumulator sets (even / odd rows) halve the FMA chains;
  // 32-row slices at or below row p hold zeros and are skipped (warp-uniform)
  R al = 0, be = 0, al1 = 0, be1 = 0;
  cplx<R> g(0, 0), g1(0, 0);
#pragma unroll
  for (int u = 0; u < RPL; u += 2) {
    if (32 * u >= p) break;
    al += abs2(x[u]);
    be += abs2(y[u]);
    cfma_conj(g, x[u], y[u]);
    if (u + 1 < RPL && 32 * (u + 1) < p) {
      al1 += abs2(x[u + 1]);
      be1 += abs2(y[u + 1]);
      cfma_conj(g1, x[u + 1], y[u + 1]);
    }
  }
  al += al1;
  be += be1;
  g = g + g1;
  al = warp_sum(al);
  be = warp_sum(be);
  g.re = warp_sum(g.re);
  g.im = warp_sum(g.im);
  cplx<R> f1, f2;
  R cs;
  if (!jacobi_rotation(al, be, g, tol2, cs, f1, f2)) return false;
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    if (32 * u >= p) break;
    const cplx<R> a = x[u], b = y[u];
    x[u] = cs * a - f1 * b;
    y[u] = f2 * a + cs * b;
  }
  return true;
}

template <class R, int RPL>
__device__ __forceinline__ void col_load(cplx<R> (&x)[RPL], const cplx<R>* col, int p, int lane) {
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const int i = lane + 32 * u;
    x[u] = i < p ? col[i] : cplx<R>(0, 0);
  }
}

template <class R, int RPL>
__device__ __forceinline__ void col_store(const cplx<R> (&x)[RPL], cplx<R>* col, int p, int lane) {
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const int i = lane + 32 * u;
    if (i < p) col[i] = x[u];
  }
}

// shared-memory bytes of jacobi_block_kernel: four block slots, all column norms, the cluster's flags
template <class R>
static size_t jacobi_block_bytes(int p, int bs, int nc) {
  return (size_t)4 * bs * p * sizeof(cplx<R>) + (size_t)2 * nc * bs * sizeof(R) + 2 * nc * sizeof(int) + 16;
}

template <class R, int NC, int RPL>
__global__ void __launch_bounds__(512, 1)
jacobi_block_kernel(const cplx<R>* __restrict__ Gin, R* __restrict__ sigma_out, cplx<R>* __restrict__ Us_out, int p,
                    int q, int bs, int max_sweeps, int* __restrict__ sweeps_out) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  constexpr int NB = 2 * NC;
  const int rank = (int)cluster.block_rank();
  // one cluster per matrix of a batch (blockIdx.y): matrices p*q apart, sigma q apart
  Gin += (size_t)blockIdx.y * p * q;
  sigma_out += (size_t)blockIdx.y * q;
  if (Us_out) Us_out += (size_t)blockIdx.y * p * q;
  if (blockIdx.y != 0) sweeps_out = nullptr;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* slots = reinterpret_cast<cplx<R>*>(smem_raw);  // [4][bs][p]
  R* norms = reinterpret_cast<R*>(slots + (size_t)4 * bs * p);  // [NB * bs]
  int* flags = reinterpret_cast<int*>(norms + (size_t)NB * bs);  // [2][NC]
  __shared__ int s_rot;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int top = 0, bot = 1, in_top = 2, in_bot = 3;
  auto col = [&](int slot, int j) { return slots + ((size_t)slot * bs + j) * p; };
  // initial blocks: rank (top) and NB-1-rank (bottom)
  for (int e = threadIdx.x; e < 2 * bs * p; e += blockDim.x) {
    const int half = e / (bs * p), f = e - half * bs * p;
    const int j = f / p, i = f - j * p;
    const int blk = half == 0 ? rank : NB - 1 - rank;
    const int c = blk * bs + j;
    col(half == 0 ? top : bot, j)[i] = c < q ? Gin[(int64_t)i * q + c] : cplx<R>(0, 0);
  }
  if (threadIdx.x == 0) s_rot = 0;
  cluster.sync();
  const R tol = (sizeof(R) == 8 ? R(DBL_EPSILON) : R(FLT_EPSILON)) * sqrt(R(p > 1 ? p : 1));
  const R tol2 = tol * tol;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int br = 0; br < NB - 1; ++br) {
      if (br == 0) {
        // pairs inside each block: round-robin of bs columns, warps < bs/2 on the top block
        for (int s = 0; s + 1 < bs; ++s) {
          const int k = w < bs / 2 ? w : w - bs / 2;
          const int slot = w < bs / 2 ? top : bot;
          const int a = k == 0 ? 0 : 1 + (k - 1 + s) % (bs - 1);
          const int kk = bs - 1 - k;
          const int c = kk == 0 ? 0 : 1 + (kk - 1 + s) % (bs - 1);
          cplx<R> x[RPL], y[RPL];
          col_load(x, col(slot, a), p, lane);
          col_load(y, col(slot, c), p, lane);
          if (warp_pair_rotate(x, y, tol2, p)) {
            col_store(x, col(slot, a), p, lane);
            col_store(y, col(slot, c), p, lane);
            if (lane == 0) s_rot = 1;
          }
          __syncthreads();
        }
      }
      // cross pairs: top column w (in registers) with bottom column (w + s) mod bs
      cplx<R> x[RPL];
      col_load(x, col(top, w), p, lane);
      bool xr = false;
      for (int s = 0; s < bs; ++s) {
        const int c = (w + s) % bs;
        cplx<R> y[RPL];
        col_load(y, col(bot, c), p, lane);
        if (warp_pair_rotate(x, y, tol2, p)) {
          col_store(y, col(bot, c), p, lane);
          xr = true;
        }
        __syncthreads();
      }
      if (xr) {
        col_store(x, col(top, w), p, lane);
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
      // exchange: the block at position j moves to j - 1 (j >= 2), position 1 to NB - 1, position 0 stays
      const int pos[2] = {rank, NB - 1 - rank};
      const int src[2] = {top, bot};
      for (int h = 0; h < 2; ++h) {
        int np = pos[h] == 0 ? 0 : (pos[h] == 1 ? NB - 1 : pos[h] - 1);
        const int dcta = np < NC ? np : NB - 1 - np;
        const int drole = np < NC ? in_top : in_bot;  // slot indices agree in every CTA
        cplx<R>* dst = cluster.map_shared_rank(col(drole, 0), dcta);
        const cplx<R>* sp = col(src[h], 0);
        for (int e = threadIdx.x; e < bs * p; e += blockDim.x) dst[e] = sp[e];
      }
      if (br == NB - 2 && threadIdx.x == 0) {
        const int any = s_rot;
        for (int rr = 0; rr < NC; ++rr) cluster.map_shared_rank(flags, rr)[(sweep & 1) * NC + rank] = any;
      }
      cluster.sync();
      int t = top;
      top = in_top;
      in_top = t;
      t = bot;
      bot = in_bot;
      in_bot = t;
    }
    int any = 0;
    for (int rr = 0; rr < NC; ++rr) any |= flags[(sweep & 1) * NC + rr];
    __syncthreads();
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    if (!any) {
      ++sweep;
      break;
    }
  }
  if (rank == 0 && threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
  // column norms (whole columns are local), gathered in every CTA
  for (int j = w; j < 2 * bs; j += blockDim.x >> 5) {
    const int slot = j < bs ? top : bot;
    const int blk = j < bs ? rank : NB - 1 - rank;
    const cplx<R>* cp = col(slot, j < bs ? j : j - bs);
    R sacc = 0;
    for (int i = lane; i < p; i += 32) sacc += abs2(cp[i]);
    sacc = warp_sum(sacc);
    if (lane < NC) cluster.map_shared_rank(norms, lane)[blk * bs + (j < bs ? j : j - bs)] = sqrt(sacc);
  }
  cluster.sync();
  const int qp = NB * bs;
  for (int j = w; j < 2 * bs; j += blockDim.x >> 5) {
    const int blk = j < bs ? rank : NB - 1 - rank;
    const int c = blk * bs + (j < bs ? j : j - bs);
    if (c >= q) continue;
    const R v = norms[c];
    int rk = 0;
    for (int i = 0; i < qp; ++i) {
      const R u = norms[i];
      rk += (u > v) || (u == v && i < c);
    }
    if (lane == 0) sigma_out[rk] = v;
    if (Us_out) {
      const cplx<R>* cp = col(j < bs ? top : bot, j < bs ? j : j - bs);
      const R f = v > (sizeof(R) == 8 ? R(DBL_MIN) : R(FLT_MIN)) * R(4) ? R(1) / v : R(0);
      for (int i = lane; i < p; i += 32) {
        const cplx<R> g = cp[i];
        Us_out[(size_t)i * q + rk] = cplx<R>(g.re * f, g.im * f);
      }
    }
  }
}

template <class R, int NC, int RPL>
static int launch_jacobi_block(const cplx<R>* G, R* sigma, cplx<R>* Us, int p, int q, int bs, int max_sweeps,
                               int* sweeps, cudaStream_t s, int batch) {
  const size_t sm = jacobi_block_bytes<R>(p, bs, NC);
  if (qtt_allow_max_smem((const void*)jacobi_block_kernel<R, NC, RPL>) != QTT_OK) return QTT_ERR_CUDA;
  if (batch < 1 || batch > 65535) return QTT_ERR_ARG;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(NC, (unsigned)batch, 1);
  cfg.blockDim = dim3(32 * bs, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = NC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, jacobi_block_kernel<R, NC, RPL>, G, sigma, Us, p, q, bs, max_sweeps, sweeps) !=
      cudaSuccess)
    return QTT_ERR_CUDA;
  return QTT_OK;
}

// Cluster size and block width of the block-cyclic Jacobi for a p x q matrix,
// or 0 when it does not apply (q < 32, p > 512, more than 16 columns per block
// or too much shared memory).
template <class R>
int qtt_jacobi_block_plan(int p, int q, int* bs_out) {
  if (q < 32 || p < 1 || p > (sizeof(R) == 8 ? 256 : 512)) return 0;
  // 4 CTAs below q = 64, else 8 (4 CTAs of 16 warps at q = 128 measured 1.4x
  // slower than 8 of 8: each round's pair chain, not the number of warps,
  // sets the time)
  auto width = [&](int nc) {
    int bs = (q + 2 * nc - 1) / (2 * nc);
    return bs + (bs & 1);
  };
  auto fits = [&](int nc) { return width(nc) <= 16 && jacobi_block_bytes<R>(p, width(nc), nc) <= 200 * 1024; };
  int nc = q < 64 && fits(4) ? 4 : 8;
  if (!fits(nc)) return 0;
  *bs_out = width(nc);
  return nc;
}

template <class R>
int qtt_jacobi_block(const cplx<R>* G, R* sigma, cplx<R>* Usorted, int p, int q, int max_sweeps, int* sweeps,
                     cudaStream_t s, int batch) {
  int bs = 0;
  const int nc = qtt_jacobi_block_plan<R>(p, q, &bs);
  if (!nc) return QTT_ERR_UNSUPPORTED;
  const int rpl = p <= 128 ? 4 : (p <= 256 ? 8 : 16);
  if (sizeof(R) == 8 && rpl > 8) return QTT_ERR_UNSUPPORTED;
  int st;
  constexpr int RMAX = sizeof(R) == 8 ? 8 : 16;  // rows per lane: two columns of them live in registers
  if (nc == 8)
    st = rpl == 4 ? launch_jacobi_block<R, 8, 4>(G, sigma, Usorted, p, q, bs, max_sweeps, sweeps, s, batch)
       : rpl == 8 ? launch_jacobi_block<R, 8, 8>(G, sigma, Usorted, p, q, bs, max_sweeps, sweeps, s, batch)
                  : launch_jacobi_block<R, 8, RMAX>(G, sigma, Usorted, p, q, bs, max_sweeps, sweeps, s, batch);
  else
    st = rpl == 4 ? launch_jacobi_block<R, 4, 4>(G, sigma, Usorted, p, q, bs, max_sweeps, sweeps, s, batch)
       : rpl == 8 ? launch_jacobi_block<R, 4, 8>(G, sigma, Usorted, p, q, bs, max_sweeps, sweeps, s, batch)
                  : launch_jacobi_block<R, 4, RMAX>(G, sigma, Usorted, p, q, bs, max_sweeps, sweeps, s, batch);
  if (st != QTT_OK) return st;
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template int qtt_jacobi_block_plan<double>(int, int, int*);
template int qtt_jacobi_block_plan<float>(int, int, int*);
template int qtt_jacobi_block<double>(const zc*, double*, zc*, int, int, int, int*, cudaStream_t, int);
template int qtt_jacobi_block<float>(const cc*, float*, cc*, int, int, int, int*, cudaStream_t, int);
