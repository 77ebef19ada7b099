// Shared device helpers for the QTT kernels: complex arithmetic over double and
// float, launch-error plumbing.  Complex numbers are stored interleaved
// (re, im), 8- or 16-byte aligned, exactly like C99 `double _Complex` /
// `float _Complex`.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define QTT_HD __host__ __device__ __forceinline__

template <class R>
struct alignas(2 * sizeof(R)) cplx {
  R re, im;
  QTT_HD cplx() {}
  QTT_HD cplx(R r, R i = R(0)) : re(r), im(i) {}
};

typedef cplx<double> zc;   // complex double
typedef cplx<float> cc;    // complex float

template <class R> QTT_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return cplx<R>(a.re + b.re, a.im + b.im); }
template <class R> QTT_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return cplx<R>(a.re - b.re, a.im - b.im); }
template <class R> QTT_HD cplx<R> operator-(cplx<R> a) { return cplx<R>(-a.re, -a.im); }
template <class R> QTT_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return cplx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R> QTT_HD cplx<R> operator*(R s, cplx<R> a) { return cplx<R>(s * a.re, s * a.im); }
template <class R> QTT_HD cplx<R> conjg(cplx<R> a) { return cplx<R>(a.re, -a.im); }
template <class R> QTT_HD R abs2(cplx<R> a) { return a.re * a.re + a.im * a.im; }
// a += b * c   (fused where the hardware fuses)
template <class R> QTT_HD void cfma(cplx<R>& a, cplx<R> b, cplx<R> c) {
  a.re = fma(b.re, c.re, a.re);
  a.re = fma(-b.im, c.im, a.re);
  a.im = fma(b.re, c.im, a.im);
  a.im = fma(b.im, c.re, a.im);
}
// a += conj(b) * c
template <class R> QTT_HD void cfma_conj(cplx<R>& a, cplx<R> b, cplx<R> c) {
  a.re = fma(b.re, c.re, a.re);
  a.re = fma(b.im, c.im, a.re);
  a.im = fma(b.re, c.im, a.im);
  a.im = fma(-b.im, c.re, a.im);
}

// Status codes shared with the C-ABI (qtt.h).
#define QTT_OK 0
#define QTT_ERR_ARG -1
#define QTT_ERR_OOM -2
#define QTT_ERR_RANK -3
#define QTT_ERR_TIMEOUT -4
#define QTT_ERR_NOT_CONVERGED -5
#define QTT_ERR_NAN -6
#define QTT_ERR_CUDA -7
#define QTT_ERR_UNSUPPORTED -8

// Multi-index GEMM descriptor.  Every logical index of a contraction is a
// pair of sub-indices (outer, inner) with sizes (n1, n2) and element strides
// (s1, s2): logical value v maps to offset (v / n2) * s1 + (v % n2) * s2.
struct MIdx {
  int64_t n1, n2;   // sizes
  int64_t s1, s2;   // strides (elements)
};

QTT_HD int64_t midx_off(const MIdx& m, int64_t v) {
  if (m.n2 == 1) return v * m.s1;
  int64_t a = v / m.n2;
  int64_t b = v - a * m.n2;
  return a * m.s1 + b * m.s2;
}
QTT_HD int64_t midx_size(const MIdx& m) { return m.n1 * m.n2; }

// Spatial QTT sites of a grid with 2^nb[dim] voxels along dimension dim:
// site p (0-based, control site excluded) holds bit pos[p] (0 = most
// significant in position space) of dimension dim[p].  Passed to kernels by
// value.
struct SiteMap {
  int d;                 // number of spatial sites, nb[0] + nb[1] + nb[2]
  int nb[3];
  signed char dim[64];
  signed char pos[64];
};

// Green operator component (I, J) at the frequency vector xi (Sec. 3.1):
// scalar conductivity (ncomp 3) xi_I xi_J / (k0 |xi|^2); isotropic elasticity
// (ncomp 6, Voigt order 11, 22, 33, 23, 13, 12 on engineering strains) the
// Moulinec-Suquet operator scaled by the Voigt weights of I and J; 0 at xi = 0.
__device__ __forceinline__ double green_entry(const double xi[3], int I, int J, int ncomp, double k0, double lam0,
                                              double mu0) {
  const double q2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
  if (!(q2 > 0)) return 0.0;
  if (ncomp == 3) return xi[I] * xi[J] / (k0 * q2);
  const int vi[6] = {0, 1, 2, 1, 0, 0};
  const int vj[6] = {0, 1, 2, 2, 2, 1};
  const double vw[6] = {1, 1, 1, 2, 2, 2};
  const double coef = (lam0 + mu0) / (mu0 * (lam0 + 2 * mu0));
  const int i = vi[I], j = vj[I], kk = vi[J], h = vj[J];
  double t = 0.0;
  if (kk == i) t += xi[h] * xi[j];
  if (h == i) t += xi[kk] * xi[j];
  if (kk == j) t += xi[h] * xi[i];
  if (h == j) t += xi[kk] * xi[i];
  double g = t / (4.0 * mu0 * q2) - coef * xi[i] * xi[j] * xi[kk] * xi[h] / (q2 * q2);
  return g * (vw[I] * vw[J]);
}

// A function sampled by the TT-cross (Sec. 3, operator setup).
//  CROSS_GREEN: the Green operator train, site 0 the control index I*ncomp+J
//    (ncomp^2 values), then the spatial sites of `m` in the momentum
//    convention (site (dim, pos) holds the bit of weight 2^pos of k_dim);
//  CROSS_BOXES: the phase indicator of a union of axis-aligned boxes (rows
//    cx, cy, cz, hx, hy, hz of `boxes`, device memory), spatial sites only,
//    position convention (site (dim, pos) holds bit nb[dim]-1-pos of x_dim);
//    a voxel is inside a box when the periodic distance of its centre
//    (x + 1/2)/N from the box centre is at most the half width on every axis.
//  CROSS_ELLIPSOIDS: the phase indicator of a union of ellipsoids (rows of
//    15: centre, semi-axes a_i (may be +inf: a fibre), rotation R row-major,
//    column i the direction of semi-axis i; device memory), spatial sites
//    only, position convention: with the periodic offsets
//    D_j = (c_j - centre_j) - rint(c_j - centre_j) of the voxel centre, the
//    voxel is inside when sum_i (u_i / a_i)^2 <= 1, u_i = sum_j R[j][i] D_j,
//    every operation rounded separately in that order (no fused multiply-add).
enum { CROSS_GREEN = 1, CROSS_BOXES = 2, CROSS_ELLIPSOIDS = 3 };
struct CrossFn {
  int kind;
  SiteMap m;
  int ncomp;
  double k0, lam0, mu0;
  const double* boxes;
  int nboxes;
  const double* ells;
  int nells;
};

// C[b][m][n] = alpha * sum_k opA(A)[b][m][k] * opB(B)[b][k][n] + beta * C[b][m][n]
// with every one of b, m, n, k a two-level multi-index per operand.
struct GemmDesc {
  MIdx bA, mA, kA;   // A strides for batch, m, k
  MIdx bB, kB, nB;   // B strides for batch, k, n
  MIdx bC, mC, nC;   // C strides for batch, m, n
  int64_t M, N, K, batch;
  int conjA, conjB;  // conjugate A / B elements
};
