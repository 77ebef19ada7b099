// Elementwise and placement kernels of the tensor-train path, plus the dense
// operator fills used when building the Fourier and Green trains on the device.
//
// Core layout: (r_{k-1}, n_k, r_k) row-major.  Combined bonds put the first
// operand's index first (major).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int TPB = 256;

inline unsigned nblocks(int64_t count) {
  int64_t b = (count + TPB - 1) / TPB;
  if (b > (int64_t)1 << 30) b = (int64_t)1 << 30;
  return (unsigned)(b < 1 ? 1 : b);
}

// complex product with separately rounded terms (no contraction to FMA), so
// that scaling by exactly representable factors reproduces the host result.
__device__ __forceinline__ zc mul_rn(zc a, zc b) {
  return zc(__dsub_rn(__dmul_rn(a.re, b.re), __dmul_rn(a.im, b.im)),
            __dadd_rn(__dmul_rn(a.re, b.im), __dmul_rn(a.im, b.re)));
}
__device__ __forceinline__ cc mul_rn(cc a, cc b) {
  return cc(__fsub_rn(__fmul_rn(a.re, b.re), __fmul_rn(a.im, b.im)),
            __fadd_rn(__fmul_rn(a.re, b.im), __fmul_rn(a.im, b.re)));
}

// dst[(off0 + a), j, (off1 + c)] = scale * src[a, j, c];  dst row length n*d1
template <class R>
__global__ void place_block_kernel(const cplx<R>* __restrict__ src, int64_t s0, int64_t n, int64_t s1,
                                   cplx<R>* __restrict__ dst, int64_t d1, int64_t off0, int64_t off1,
                                   cplx<R> scale, int unit) {
  const int64_t total = s0 * n * s1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = e % s1;
    int64_t t = e / s1;
    int64_t j = t % n;
    int64_t a = t / n;
    cplx<R> v = src[e];
    if (!unit) v = mul_rn(scale, v);
    dst[((off0 + a) * n + j) * d1 + off1 + c] = v;
  }
}

// out[(a0i, b0i), i, (a1i, b1i)] = x[a0i, i, a1i] * y[b0i, i, b1i]
template <class R>
__global__ void hadamard_kernel(const cplx<R>* __restrict__ x, int64_t a0, int64_t a1,
                                const cplx<R>* __restrict__ y, int64_t b0, int64_t b1, int64_t n,
                                cplx<R>* __restrict__ out) {
  const int64_t o1 = a1 * b1;
  const int64_t total = a0 * b0 * n * o1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = e % o1;
    int64_t t = e / o1;
    int64_t i = t % n;
    int64_t r = t / n;
    int64_t ra = r / b0, rb = r - ra * b0;
    int64_t ca = c / b1, cb = c - ca * b1;
    out[e] = mul_rn(x[(ra * n + i) * a1 + ca], y[(rb * n + i) * b1 + cb]);
  }
}

// out[(g0i, a0i), i, (g1i, a1i)] = sum_j D[g0i, i, j, g1i] * X[a0i, j, a1i]
template <class R>
__global__ void mpo_core_kernel(const cplx<R>* __restrict__ D, int64_t g0, int64_t no, int64_t ni,
                                int64_t g1, const cplx<R>* __restrict__ X, int64_t a0, int64_t a1,
                                cplx<R>* __restrict__ out) {
  const int64_t o1 = g1 * a1;
  const int64_t total = g0 * a0 * no * o1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = e % o1;
    int64_t t = e / o1;
    int64_t i = t % no;
    int64_t r = t / no;
    int64_t gr = r / a0, ar = r - gr * a0;
    int64_t gc = c / a1, ac = c - gc * a1;
    cplx<R> acc(0, 0);
    for (int64_t j = 0; j < ni; ++j)
      cfma(acc, D[((gr * no + i) * ni + j) * g1 + gc], X[(ar * ni + j) * a1 + ac]);
    out[e] = acc;
  }
}

template <class R>
__global__ void scale_kernel(cplx<R>* x, int64_t count, cplx<R> s) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    x[e] = mul_rn(s, x[e]);
}

// single-block sum of squared moduli in double (deterministic order per launch shape)
template <class R>
__global__ void sumsq_kernel(const cplx<R>* __restrict__ x, int64_t count, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < count; e += blockDim.x) {
    double re = (double)x[e].re, im = (double)x[e].im;
    acc = fma(re, re, acc);
    acc = fma(im, im, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    *out = s;
  }
}

__global__ void z2c_kernel(const zc* __restrict__ in, cc* __restrict__ out, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = cc((float)in[e].re, (float)in[e].im);
}
__global__ void c2z_kernel(const cc* __restrict__ in, zc* __restrict__ out, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = zc((double)in[e].re, (double)in[e].im);
}

template <class R>
__global__ void copy_strided_kernel(const cplx<R>* __restrict__ in, MIdx rows, MIdx cols, int64_t nrows,
                                    int64_t ncols, int conj_in, cplx<R>* __restrict__ out, int64_t ldo) {
  const int64_t total = nrows * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / ncols, c = e - i * ncols;
    cplx<R> v = in[midx_off(rows, i) + midx_off(cols, c)];
    if (conj_in) v.im = -v.im;
    out[i * ldo + c] = v;
  }
}

// x[i, :] *= sv[i]  (or /= sv[i] when invert; rows with sv[i] == 0 are zeroed)
template <class R>
__global__ void scale_rows_kernel(cplx<R>* x, int64_t rows, int64_t cols, int64_t ld, const R* sv, int invert) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / cols, c = e - i * cols;
    R s = sv[i];
    R f = invert ? (s > R(0) ? R(1) / s : R(0)) : s;
    cplx<R>& v = x[i * ld + c];
    v = cplx<R>(v.re * f, v.im * f);
  }
}

template <class R>
__global__ void isfinite_kernel(const cplx<R>* __restrict__ x, int64_t count, int* flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (!isfinite(x[e].re) || !isfinite(x[e].im)) atomicExch(flag, 1);
  }
}

// Q_n of the superfast Fourier transform in site order: entry index
// s = sum_a (m_a*2 + j_a) 4^(n-1-a), value exp(sign 2 pi i sum_{b<=a} j_a m_b 2^(b-a-1)) / sqrt(2^n).
template <class R>
__global__ void qft_dense_kernel(cplx<R>* out, int n, double sign) {
  const int64_t total = (int64_t)1 << (2 * n);
  const double norm = pow(2.0, -0.5 * n);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    double phase = 0.0;  // in units of full turns
    for (int a = 0; a < n; ++a) {
      int ja = (int)((e >> (2 * (n - 1 - a))) & 1);
      if (!ja) continue;
      for (int b = 0; b <= a; ++b) {
        int mb = (int)((e >> (2 * (n - 1 - b) + 1)) & 1);
        if (mb) phase += ldexp(1.0, b - a - 1);
      }
    }
    phase -= floor(phase);
    double sn, cs;
    sincospi(2.0 * sign * phase, &sn, &cs);
    out[e] = cplx<R>((R)(cs * norm), (R)(sn * norm));
  }
}

// Dense Green operator in momentum site order: out[IJ * 2^d + s], s the site
// multi-index (site 0 slowest).  In momentum space site (dim, pos) carries
// the bit of weight 2^pos of the frequency index k_dim (Sec. 3.2: bits
// reversed per dimension).  Frequencies xi = k below the Nyquist index, else
// k - N (a one-voxel dimension has the single frequency 0).
template <class R>
__global__ void green_dense_kernel(cplx<R>* out, SiteMap m, int ncomp, double k0, double lam0, double mu0) {
  const int d = m.d;
  const int64_t total = (int64_t)1 << d;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total;
       s += (int64_t)gridDim.x * blockDim.x) {
    int64_t k[3] = {0, 0, 0};
    for (int p = 0; p < d; ++p) {
      const int bit = (int)((s >> (d - 1 - p)) & 1);
      k[m.dim[p]] |= (int64_t)bit << m.pos[p];
    }
    double xi[3];
    for (int a = 0; a < 3; ++a) {
      const int64_t N = (int64_t)1 << m.nb[a];
      xi[a] = (double)(k[a] < (N + 1) / 2 ? k[a] : k[a] - N);
    }
    for (int I = 0; I < ncomp; ++I)
      for (int J = 0; J < ncomp; ++J)
        out[(int64_t)(I * ncomp + J) * total + s] = cplx<R>((R)green_entry(xi, I, J, ncomp, k0, lam0, mu0), R(0));
  }
}

// Phase indicator (Nx x Ny x Nz doubles, x slowest, MSB-first bits) to site order.
template <class R>
__global__ void indicator_sites_kernel(const double* __restrict__ ind, SiteMap m, cplx<R>* __restrict__ out) {
  const int d = m.d;
  const int64_t total = (int64_t)1 << d;
  const int64_t Ny = (int64_t)1 << m.nb[1], Nz = (int64_t)1 << m.nb[2];
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total;
       s += (int64_t)gridDim.x * blockDim.x) {
    int64_t x[3] = {0, 0, 0};
    for (int p = 0; p < d; ++p) {
      const int bit = (int)((s >> (d - 1 - p)) & 1);
      const int dm = m.dim[p];
      x[dm] |= (int64_t)bit << (m.nb[dm] - 1 - m.pos[p]);
    }
    out[s] = cplx<R>((R)ind[(x[0] * Ny + x[1]) * Nz + x[2]], R(0));
  }
}

// Full tensor of a train (control index c slowest, then the site multi-index
// s with site 0 most significant) to the voxel field out[c][x][y][z]: site p
// holds bit nb[dim[p]] - 1 - pos[p] of coordinate dim[p] (position space).
template <class R>
__global__ void sites_to_voxels_kernel(const cplx<R>* __restrict__ in, SiteMap m, int ncomp,
                                       cplx<R>* __restrict__ out) {
  const int d = m.d;
  const int64_t nv = (int64_t)1 << d;
  const int64_t total = nv * ncomp;
  const int64_t Ny = (int64_t)1 << m.nb[1], Nz = (int64_t)1 << m.nb[2];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e >> d, s = e & (nv - 1);
    int64_t x[3] = {0, 0, 0};
    for (int p = 0; p < d; ++p) {
      const int bit = (int)((s >> (d - 1 - p)) & 1);
      const int dm = m.dim[p];
      x[dm] |= (int64_t)bit << (m.nb[dm] - 1 - m.pos[p]);
    }
    out[c * nv + (x[0] * Ny + x[1]) * Nz + x[2]] = in[e];
  }
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): counter-based generator, 10 rounds with the published
// multipliers and Weyl key increments.
__device__ __forceinline__ void philox4x32_10(uint32_t ctr[4], uint32_t key[2]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, ctr[0]), lo0 = M0 * ctr[0];
    uint32_t hi1 = __umulhi(M1, ctr[2]), lo1 = M1 * ctr[2];
    uint32_t n0 = hi1 ^ ctr[1] ^ key[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ ctr[3] ^ key[1];
    uint32_t n3 = lo0;
    ctr[0] = n0; ctr[1] = n1; ctr[2] = n2; ctr[3] = n3;
    key[0] += W0;
    key[1] += W1;
  }
}

// Real Gaussian entries N(0, scale^2) stored as complex with zero imaginary
// part: Box-Muller on two 32-bit uniforms per entry; counter = (index, stream).
template <class R>
__global__ void gaussian_kernel(cplx<R>* out, int64_t count, uint64_t seed, uint64_t stream, double scale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t ctr[4] = {(uint32_t)e, (uint32_t)((uint64_t)e >> 32), (uint32_t)stream, (uint32_t)(stream >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    philox4x32_10(ctr, key);
    double u1 = ((double)ctr[0] + 0.5) * 2.3283064365386963e-10;   // (0, 1)
    double u2 = ((double)ctr[1] + 0.5) * 2.3283064365386963e-10;
    double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[e] = cplx<R>((R)(scale * rad * cs), R(0));
  }
}

// D[a, i, i, b] = X[a, i, b], zero elsewhere (Sec. 2.1, Eq. tt_to_tto)
template <class R>
__global__ void diag_mpo_kernel(const cplx<R>* __restrict__ X, int64_t r0, int64_t n, int64_t r1,
                                cplx<R>* __restrict__ D) {
  const int64_t total = r0 * n * n * r1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = e % r1;
    int64_t t = e / r1;
    int64_t j = t % n;
    t /= n;
    int64_t i = t % n;
    int64_t a = t / n;
    D[e] = (i == j) ? X[(a * n + i) * r1 + b] : cplx<R>(0, 0);
  }
}

// identity operator core carrying a bond of size g: D[c, i, j, c'] = delta_ij delta_cc'
template <class R>
__global__ void identity_core_kernel(int64_t g, int64_t n, cplx<R>* __restrict__ D) {
  const int64_t total = g * n * n * g;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c2 = e % g;
    int64_t t = e / g;
    int64_t j = t % n;
    t /= n;
    int64_t i = t % n;
    int64_t c = t / n;
    D[e] = cplx<R>((i == j && c == c2) ? R(1) : R(0), R(0));
  }
}

// adjoint operator core: out[c, j, i, c'] = conj(D[c, i, j, c'])
template <class R>
__global__ void adjoint_core_kernel(const cplx<R>* __restrict__ D, int64_t g0, int64_t no, int64_t ni,
                                    int64_t g1, cplx<R>* __restrict__ out) {
  const int64_t total = g0 * no * ni * g1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c2 = e % g1;
    int64_t t = e / g1;
    int64_t j = t % ni;
    t /= ni;
    int64_t i = t % no;
    int64_t c = t / no;
    out[((c * ni + j) * no + i) * g1 + c2] = conjg(D[e]);
  }
}

}  // namespace

#define CHECK_LAUNCH() return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA

template <class R>
__global__ void copy_batch_kernel(const cplx<R>* __restrict__ in, int64_t ib, MIdx rows, MIdx cols, int64_t nrows,
                                  int64_t ncols, int conj_in, cplx<R>* __restrict__ out, int64_t ldo, int64_t ob) {
  const int64_t b = blockIdx.y, tot = nrows * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols, j = e - i * ncols;
    cplx<R> v = in[b * ib + midx_off(rows, i) + midx_off(cols, j)];
    if (conj_in) v.im = -v.im;
    out[b * ob + i * ldo + j] = v;
  }
}

template <class R>
__global__ void mask_cols_kernel(cplx<R>* __restrict__ X, int64_t bs, int64_t rows, int64_t cols, int64_t ld,
                                 const int* __restrict__ t, int tstride) {
  const int64_t b = blockIdx.y, tot = rows * cols;
  const int tb = t[b * tstride];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    if (j >= tb) X[b * bs + i * ld + j] = cplx<R>(0, 0);
  }
}

template <class R>
__global__ void crop_kernel(const cplx<R>* __restrict__ src, int64_t sb, int64_t r0, int64_t n, int64_t r1,
                            cplx<R>* const* __restrict__ dst, const int* __restrict__ t0, const int* __restrict__ t1) {
  const int64_t b = blockIdx.y;
  const int64_t a0 = t0[b], a1 = t1[b], tot = a0 * n * a1;
  cplx<R>* d = dst[b];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / (n * a1), rem = e - i * n * a1, k = rem / a1, j = rem - k * a1;
    d[e] = src[b * sb + (i * n + k) * r1 + j];
  }
}

// out = (H + H^H) / 2 - shift I (q x q, row-major), and the identity-plus
// helpers of the polar compression
template <class R>
__global__ void herm_shift_kernel(const cplx<R>* __restrict__ H, int64_t q, double shift, cplx<R>* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < q * q; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / q, j = e - i * q;
    const cplx<R> a = H[e], b = H[j * q + i];
    cplx<R> v(R(0.5) * (a.re + b.re), R(0.5) * (a.im - b.im));
    if (i == j) v.re -= (R)shift;
    out[e] = v;
  }
}

// P = (I + S) / 2 in place, and the real part of its trace into *tr
template <class R>
__global__ void half_identity_plus_kernel(cplx<R>* __restrict__ S, int64_t q, double* __restrict__ tr) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < q * q; e += blockDim.x) {
    const int64_t i = e / q, j = e - i * q;
    cplx<R> v = S[e];
    v.re *= R(0.5);
    v.im *= R(0.5);
    if (i == j) {
      v.re += R(0.5);
      acc += (double)v.re;
    }
    S[e] = v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *tr = t;
  }
}

template <class R>
int qtt_place_block(const cplx<R>* src, int64_t s0, int64_t n, int64_t s1, cplx<R>* dst, int64_t d1,
                    int64_t off0, int64_t off1, cplx<R> scale, cudaStream_t s) {
  int64_t total = s0 * n * s1;
  if (total <= 0) return QTT_OK;
  int unit = (scale.re == R(1) && scale.im == R(0));
  place_block_kernel<R><<<nblocks(total), TPB, 0, s>>>(src, s0, n, s1, dst, d1, off0, off1, scale, unit);
  CHECK_LAUNCH();
}
template <class R>
int qtt_hadamard_core(const cplx<R>* x, int64_t a0, int64_t a1, const cplx<R>* y, int64_t b0, int64_t b1,
                      int64_t n, cplx<R>* out, cudaStream_t s) {
  int64_t total = a0 * b0 * n * a1 * b1;
  if (total <= 0) return QTT_OK;
  hadamard_kernel<R><<<nblocks(total), TPB, 0, s>>>(x, a0, a1, y, b0, b1, n, out);
  CHECK_LAUNCH();
}
template <class R>
int qtt_mpo_core(const cplx<R>* D, int64_t g0, int64_t no, int64_t ni, int64_t g1, const cplx<R>* X,
                 int64_t a0, int64_t a1, cplx<R>* out, cudaStream_t s) {
  int64_t total = g0 * a0 * no * g1 * a1;
  if (total <= 0) return QTT_OK;
  mpo_core_kernel<R><<<nblocks(total), TPB, 0, s>>>(D, g0, no, ni, g1, X, a0, a1, out);
  CHECK_LAUNCH();
}
template <class R>
int qtt_scale(cplx<R>* x, int64_t count, cplx<R> sc, cudaStream_t s) {
  if (count <= 0) return QTT_OK;
  scale_kernel<R><<<nblocks(count), TPB, 0, s>>>(x, count, sc);
  CHECK_LAUNCH();
}
template <class R>
int qtt_sumsq(const cplx<R>* x, int64_t count, double* out, cudaStream_t s) {
  sumsq_kernel<R><<<1, 1024, 0, s>>>(x, count, out);
  CHECK_LAUNCH();
}
int qtt_convert_z2c(const zc* in, cc* out, int64_t count, cudaStream_t s) {
  if (count <= 0) return QTT_OK;
  z2c_kernel<<<nblocks(count), TPB, 0, s>>>(in, out, count);
  CHECK_LAUNCH();
}
int qtt_convert_c2z(const cc* in, zc* out, int64_t count, cudaStream_t s) {
  if (count <= 0) return QTT_OK;
  c2z_kernel<<<nblocks(count), TPB, 0, s>>>(in, out, count);
  CHECK_LAUNCH();
}
template <class R>
int qtt_copy_strided(const cplx<R>* in, MIdx rows, MIdx cols, int64_t nrows, int64_t ncols, int conj_in,
                     cplx<R>* out, int64_t ldo, cudaStream_t s) {
  int64_t total = nrows * ncols;
  if (total <= 0) return QTT_OK;
  copy_strided_kernel<R><<<nblocks(total), TPB, 0, s>>>(in, rows, cols, nrows, ncols, conj_in, out, ldo);
  CHECK_LAUNCH();
}
template <class R>
int qtt_scale_rows(cplx<R>* x, int64_t rows, int64_t cols, int64_t ld, const R* sv, int invert, cudaStream_t s) {
  int64_t total = rows * cols;
  if (total <= 0) return QTT_OK;
  scale_rows_kernel<R><<<nblocks(total), TPB, 0, s>>>(x, rows, cols, ld, sv, invert);
  CHECK_LAUNCH();
}
template <class R>
int qtt_isfinite(const cplx<R>* x, int64_t count, int* flag, cudaStream_t s) {
  if (count <= 0) return QTT_OK;
  isfinite_kernel<R><<<nblocks(count), TPB, 0, s>>>(x, count, flag);
  CHECK_LAUNCH();
}
template <class R>
int qtt_fill_qft_dense(cplx<R>* out, int n, double sign, cudaStream_t s) {
  int64_t total = (int64_t)1 << (2 * n);
  qft_dense_kernel<R><<<nblocks(total), TPB, 0, s>>>(out, n, sign);
  CHECK_LAUNCH();
}
template <class R>
int qtt_fill_green_dense(cplx<R>* out, const SiteMap& m, int ncomp, double k0, double lam0, double mu0,
                         cudaStream_t s) {
  const int64_t total = (int64_t)1 << m.d;
  green_dense_kernel<R><<<nblocks(total), TPB, 0, s>>>(out, m, ncomp, k0, lam0, mu0);
  CHECK_LAUNCH();
}
template <class R>
int qtt_fill_indicator_sites(const double* ind, const SiteMap& m, cplx<R>* out, cudaStream_t s) {
  const int64_t total = (int64_t)1 << m.d;
  indicator_sites_kernel<R><<<nblocks(total), TPB, 0, s>>>(ind, m, out);
  CHECK_LAUNCH();
}

template <class R>
int qtt_sites_to_voxels(const cplx<R>* in, const SiteMap& m, int ncomp, cplx<R>* out, cudaStream_t s) {
  const int64_t total = ((int64_t)1 << m.d) * ncomp;
  sites_to_voxels_kernel<R><<<nblocks(total), TPB, 0, s>>>(in, m, ncomp, out);
  CHECK_LAUNCH();
}

template <class R>
int qtt_fill_gaussian(cplx<R>* out, int64_t count, uint64_t seed, uint64_t stream, double scale, cudaStream_t s) {
  if (count <= 0) return QTT_OK;
  gaussian_kernel<R><<<nblocks(count), TPB, 0, s>>>(out, count, seed, stream, scale);
  CHECK_LAUNCH();
}
template <class R>
int qtt_diag_mpo_core(const cplx<R>* X, int64_t r0, int64_t n, int64_t r1, cplx<R>* D, cudaStream_t s) {
  int64_t total = r0 * n * n * r1;
  if (total <= 0) return QTT_OK;
  diag_mpo_kernel<R><<<nblocks(total), TPB, 0, s>>>(X, r0, n, r1, D);
  CHECK_LAUNCH();
}
template <class R>
int qtt_identity_core(int64_t g, int64_t n, cplx<R>* D, cudaStream_t s) {
  int64_t total = g * n * n * g;
  if (total <= 0) return QTT_OK;
  identity_core_kernel<R><<<nblocks(total), TPB, 0, s>>>(g, n, D);
  CHECK_LAUNCH();
}
template <class R>
int qtt_adjoint_core(const cplx<R>* D, int64_t g0, int64_t no, int64_t ni, int64_t g1, cplx<R>* out,
                     cudaStream_t s) {
  int64_t total = g0 * no * ni * g1;
  if (total <= 0) return QTT_OK;
  adjoint_core_kernel<R><<<nblocks(total), TPB, 0, s>>>(D, g0, no, ni, g1, out);
  CHECK_LAUNCH();
}

#define INST(R)                                                                                          \
  template int qtt_place_block<R>(const cplx<R>*, int64_t, int64_t, int64_t, cplx<R>*, int64_t, int64_t,  \
                                  int64_t, cplx<R>, cudaStream_t);                                        \
  template int qtt_hadamard_core<R>(const cplx<R>*, int64_t, int64_t, const cplx<R>*, int64_t, int64_t,  \
                                    int64_t, cplx<R>*, cudaStream_t);                                    \
  template int qtt_mpo_core<R>(const cplx<R>*, int64_t, int64_t, int64_t, int64_t, const cplx<R>*,        \
                               int64_t, int64_t, cplx<R>*, cudaStream_t);                                \
  template int qtt_scale<R>(cplx<R>*, int64_t, cplx<R>, cudaStream_t);                                   \
  template int qtt_sumsq<R>(const cplx<R>*, int64_t, double*, cudaStream_t);                             \
  template int qtt_copy_strided<R>(const cplx<R>*, MIdx, MIdx, int64_t, int64_t, int, cplx<R>*, int64_t, \
                                   cudaStream_t);                                                        \
  template int qtt_scale_rows<R>(cplx<R>*, int64_t, int64_t, int64_t, const R*, int, cudaStream_t);       \
  template int qtt_isfinite<R>(const cplx<R>*, int64_t, int*, cudaStream_t);                             \
  template int qtt_fill_qft_dense<R>(cplx<R>*, int, double, cudaStream_t);                               \
  template int qtt_fill_green_dense<R>(cplx<R>*, const SiteMap&, int, double, double, double, cudaStream_t);   \
  template int qtt_fill_indicator_sites<R>(const double*, const SiteMap&, cplx<R>*, cudaStream_t);              \
  template int qtt_sites_to_voxels<R>(const cplx<R>*, const SiteMap&, int, cplx<R>*, cudaStream_t);            \
  template int qtt_fill_gaussian<R>(cplx<R>*, int64_t, uint64_t, uint64_t, double, cudaStream_t);          \
  template int qtt_diag_mpo_core<R>(const cplx<R>*, int64_t, int64_t, int64_t, cplx<R>*, cudaStream_t);    \
  template int qtt_identity_core<R>(int64_t, int64_t, cplx<R>*, cudaStream_t);                             \
  template int qtt_adjoint_core<R>(const cplx<R>*, int64_t, int64_t, int64_t, int64_t, cplx<R>*, cudaStream_t);
INST(double)
INST(float)

static unsigned grid_for(int64_t tot) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 4096)); }

template <class R>
int qtt_copy_batch(const cplx<R>* in, int64_t ib, MIdx rows, MIdx cols, int64_t nrows, int64_t ncols, int conj_in,
                   cplx<R>* out, int64_t ldo, int64_t ob, int batch, cudaStream_t s) {
  if (batch < 1 || nrows * ncols == 0) return QTT_OK;
  if (batch > 65535) return QTT_ERR_ARG;
  copy_batch_kernel<R><<<dim3(grid_for(nrows * ncols), batch), 256, 0, s>>>(in, ib, rows, cols, nrows, ncols, conj_in,
                                                                            out, ldo, ob);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template <class R>
int qtt_mask_cols_batch(cplx<R>* X, int64_t bs, int64_t rows, int64_t cols, int64_t ld, const int* t, int tstride,
                        int batch, cudaStream_t s) {
  if (batch < 1 || rows * cols == 0) return QTT_OK;
  if (batch > 65535) return QTT_ERR_ARG;
  mask_cols_kernel<R><<<dim3(grid_for(rows * cols), batch), 256, 0, s>>>(X, bs, rows, cols, ld, t, tstride);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template <class R>
int qtt_crop_batch(const cplx<R>* src, int64_t sb, int64_t r0, int64_t n, int64_t r1, cplx<R>* const* dst,
                   const int* t0, const int* t1, int batch, cudaStream_t s) {
  if (batch < 1) return QTT_OK;
  if (batch > 65535) return QTT_ERR_ARG;
  crop_kernel<R><<<dim3(grid_for(r0 * n * r1), batch), 256, 0, s>>>(src, sb, r0, n, r1, dst, t0, t1);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template int qtt_copy_batch<double>(const zc*, int64_t, MIdx, MIdx, int64_t, int64_t, int, zc*, int64_t, int64_t, int,
                                    cudaStream_t);
template int qtt_copy_batch<float>(const cc*, int64_t, MIdx, MIdx, int64_t, int64_t, int, cc*, int64_t, int64_t, int,
                                   cudaStream_t);
template int qtt_mask_cols_batch<double>(zc*, int64_t, int64_t, int64_t, int64_t, const int*, int, int, cudaStream_t);
template int qtt_mask_cols_batch<float>(cc*, int64_t, int64_t, int64_t, int64_t, const int*, int, int, cudaStream_t);
template int qtt_crop_batch<double>(const zc*, int64_t, int64_t, int64_t, int64_t, zc* const*, const int*,
                                    const int*, int, cudaStream_t);
template int qtt_crop_batch<float>(const cc*, int64_t, int64_t, int64_t, int64_t, cc* const*, const int*, const int*,
                                   int, cudaStream_t);

template <class R>
int qtt_herm_shift(const cplx<R>* H, int64_t q, double shift, cplx<R>* out, cudaStream_t s) {
  if (q <= 0) return QTT_OK;
  herm_shift_kernel<R><<<grid_for(q * q), 256, 0, s>>>(H, q, shift, out);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}
template <class R>
int qtt_half_identity_plus(cplx<R>* S, int64_t q, double* tr, cudaStream_t s) {
  if (q <= 0) return QTT_OK;
  half_identity_plus_kernel<R><<<1, 1024, 0, s>>>(S, q, tr);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}
template int qtt_herm_shift<double>(const zc*, int64_t, double, zc*, cudaStream_t);
template int qtt_herm_shift<float>(const cc*, int64_t, double, cc*, cudaStream_t);
template int qtt_half_identity_plus<double>(zc*, int64_t, double*, cudaStream_t);
template int qtt_half_identity_plus<float>(cc*, int64_t, double*, cudaStream_t);
