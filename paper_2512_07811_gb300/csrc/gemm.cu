// Batched complex GEMM over two-level multi-indices (CUDA cores, FP64 / FP32).
//
// Every core contraction of the tensor-train path (absorbing R or U*S into a
// neighbouring core, transfer matrices of inner products, the structured
// sketch contractions of operator-times-train products) is one call of this
// kernel with suitable index strides, so no contraction needs an explicit
// permutation pass.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace {

// With splits > 1 every CTA sums only its share of K and stores the raw
// partial tile to P[split][batch][m][n] (dense); a second kernel reduces the
// partials in split order and applies alpha, beta and the output strides.
//
// Index arithmetic: the element offsets of the tile's BM rows of A and BN
// columns of B are computed once per CTA, those of each K-tile's BK values
// once per tile (two tiles ahead, in a ring of three), so the loads do no
// division.  Threads walk a tile along whichever index is contiguous in
// memory (k or m for A, k or n for B) so that neighbouring threads read
// neighbouring elements.  The main loop is software-pipelined: the next
// tile is loaded into registers while the current one is multiplied from
// shared memory.
QTT_HD bool midx_unit_inner(const MIdx& m) { return (m.n2 == 1 ? m.s1 : m.s2) == 1; }

template <class R, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_midx_kernel(GemmDesc g, cplx<R> alpha, cplx<R> beta,
                 const cplx<R>* __restrict__ A, const cplx<R>* __restrict__ B,
                 cplx<R>* __restrict__ C, int splits, int64_t kchunk, cplx<R>* __restrict__ P) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int TX = BN / TN;
  constexpr int LA = BM * BK / NT, LB = BN * BK / NT;  // tile elements each thread loads
  static_assert(2 * BK <= NT && LA * NT == BM * BK && LB * NT == BN * BK, "tile shape");
  __shared__ cplx<R> As[BK][BM + 1];
  __shared__ cplx<R> Bs[BK][BN + 1];
  __shared__ int64_t rowA[BM], colB[BN], kOffA[3][BK], kOffB[3][BK];

  const int64_t b = blockIdx.z / splits;
  const int split = blockIdx.z - (int)(b * splits);
  const int64_t kbeg = (int64_t)split * kchunk;
  const int64_t kend = min(g.K, kbeg + kchunk);
  const int64_t m0 = (int64_t)blockIdx.y * BM;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int ntiles = kend > kbeg ? (int)((kend - kbeg + BK - 1) / BK) : 0;

  const int64_t offA = midx_off(g.bA, b), offB = midx_off(g.bB, b), offC = midx_off(g.bC, b);
  for (int i = tid; i < BM; i += NT) rowA[i] = (m0 + i < g.M) ? offA + midx_off(g.mA, m0 + i) : -1;
  for (int i = tid; i < BN; i += NT) colB[i] = (n0 + i < g.N) ? offB + midx_off(g.nB, n0 + i) : -1;
  // K offsets of tile t live in slot t mod 3, computed two tiles ahead
  auto koffs = [&](int t) {
    const int sl = t % 3;
    if (tid < BK) {
      const int64_t k = kbeg + (int64_t)t * BK + tid;
      kOffA[sl][tid] = k < kend ? midx_off(g.kA, k) : -1;
    } else if (tid < 2 * BK) {
      const int64_t k = kbeg + (int64_t)t * BK + tid - BK;
      kOffB[sl][tid - BK] = k < kend ? midx_off(g.kB, k) : -1;
    }
  };
  koffs(0);
  koffs(1);
  const bool a_kfast = midx_unit_inner(g.kA) && !midx_unit_inner(g.mA);
  const bool b_kfast = midx_unit_inner(g.kB) && !midx_unit_inner(g.nB);
  __syncthreads();

  // global -> registers for tile t (this thread's LA + LB elements)
  cplx<R> ra[LA], rb[LB];
  auto fetch = [&](int t) {
    const int sl = t % 3;
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int e = tid + l * NT;
      const int mm = a_kfast ? e / BK : e % BM;
      const int kk = a_kfast ? e % BK : e / BM;
      const int64_t r = rowA[mm], k = kOffA[sl][kk];
      cplx<R> v(0, 0);
      if (r >= 0 && k >= 0) {
        v = A[r + k];
        if (g.conjA) v.im = -v.im;
      }
      ra[l] = v;
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int e = tid + l * NT;
      const int nn = b_kfast ? e / BK : e % BN;
      const int kk = b_kfast ? e % BK : e / BN;
      const int64_t c = colB[nn], k = kOffB[sl][kk];
      cplx<R> v(0, 0);
      if (c >= 0 && k >= 0) {
        v = B[c + k];
        if (g.conjB) v.im = -v.im;
      }
      rb[l] = v;
    }
  };

  cplx<R> acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = cplx<R>(0, 0);

  if (ntiles > 0) fetch(0);
  for (int t = 0; t < ntiles; ++t) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int e = tid + l * NT;
      As[a_kfast ? e % BK : e / BM][a_kfast ? e / BK : e % BM] = ra[l];
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int e = tid + l * NT;
      Bs[b_kfast ? e % BK : e / BN][b_kfast ? e / BK : e % BN] = rb[l];
    }
    __syncthreads();
    // the next tile's loads are in flight while this one is multiplied
    if (t + 1 < ntiles) fetch(t + 1);
    koffs(t + 2);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplx<R> a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + j * TX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cfma(acc[i][j], a[i], bb[j]);
    }
    __syncthreads();
  }
  const bool use_beta = (beta.re != R(0) || beta.im != R(0));
  if (splits > 1) {
    cplx<R>* Pt = P + ((int64_t)split * g.batch + b) * g.M * g.N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int64_t m = m0 + ty + i * (BM / TM);
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int64_t n = n0 + tx + j * TX;
        if (n < g.N) Pt[m * g.N + n] = acc[i][j];
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t m = m0 + ty + i * (BM / TM);
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t n = n0 + tx + j * TX;
      if (n >= g.N) continue;
      int64_t o = offC + midx_off(g.mC, m) + midx_off(g.nC, n);
      cplx<R> v = alpha * acc[i][j];
      if (use_beta) v = v + beta * C[o];
      C[o] = v;
    }
  }
}

// C[b][m][n] = alpha sum_s P[s][b][m][n] + beta C[b][m][n], summed in split order
template <class R>
__global__ void splitk_reduce_kernel(GemmDesc g, cplx<R> alpha, cplx<R> beta, const cplx<R>* __restrict__ P,
                                     int splits, cplx<R>* __restrict__ C) {
  const int64_t mn = g.M * g.N, total = g.batch * mn;
  const bool use_beta = (beta.re != R(0) || beta.im != R(0));
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = e / mn, r = e - b * mn;
    int64_t m = r / g.N, n = r - m * g.N;
    cplx<R> acc(0, 0);
    for (int s = 0; s < splits; ++s) acc = acc + P[(int64_t)s * total + e];
    int64_t o = midx_off(g.bC, b) + midx_off(g.mC, m) + midx_off(g.nC, n);
    cplx<R> v = alpha * acc;
    if (use_beta) v = v + beta * C[o];
    C[o] = v;
  }
}

}  // namespace

// Tile edge of qtt_gemm_ex: 64, or 32 for thin shapes and for grids of
// 64 x 64 tiles that would not fill a quarter of the SMs.
static int64_t gemm_tile(const GemmDesc& g) {
  if (g.M <= 32 || g.N <= 32) return 32;
  const int64_t t64 = ((g.M + 63) / 64) * ((g.N + 63) / 64) * g.batch;
  return t64 < 38 ? 32 : 64;
}

// Number of K splits worth using for this shape (1 = no split): GEMMs whose
// output tiles cannot occupy half the SMs and whose K is at least 128 get
// their K range cut into chunks of 64 or more, about one CTA per SM.
int qtt_gemm_splits(const GemmDesc& g) {
  const int64_t tile = gemm_tile(g);
  const int64_t tiles = ((g.M + tile - 1) / tile) * ((g.N + tile - 1) / tile) * g.batch;
  if (tiles >= 76 || g.K < 128) return 1;
  int64_t s = std::min<int64_t>((g.K + 63) / 64, std::max<int64_t>(1, 152 / tiles));
  return (int)std::min<int64_t>(s, 32);
}

template <class R>
int qtt_gemm_ex(const GemmDesc& g, cplx<R> alpha, cplx<R> beta, const cplx<R>* A, const cplx<R>* B, cplx<R>* C,
                int splits, cplx<R>* P, cudaStream_t s, int tile) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return QTT_OK;
  if (splits < 1 || (splits > 1 && !P)) return QTT_ERR_ARG;
  const int64_t kchunk = splits > 1 ? (g.K + splits - 1) / splits : std::max<int64_t>(g.K, 1);
  const bool thin = (tile ? tile : gemm_tile(g)) == 32;
  constexpr int BK = sizeof(R) == 8 ? 8 : 16;
  const int64_t zdim = g.batch * splits;
  if (zdim > 65535) return QTT_ERR_ARG;
  if (thin) {
    dim3 grid((unsigned)((g.N + 31) / 32), (unsigned)((g.M + 31) / 32), (unsigned)zdim);
    if (grid.y > 65535) return QTT_ERR_ARG;
    gemm_midx_kernel<R, 32, 32, BK, 2, 2><<<grid, 256, 0, s>>>(g, alpha, beta, A, B, C, splits, kchunk, P);
  } else {
    dim3 grid((unsigned)((g.N + 63) / 64), (unsigned)((g.M + 63) / 64), (unsigned)zdim);
    if (grid.y > 65535) return QTT_ERR_ARG;
    gemm_midx_kernel<R, 64, 64, BK, 4, 4><<<grid, 256, 0, s>>>(g, alpha, beta, A, B, C, splits, kchunk, P);
  }
  if (splits > 1) {
    const int64_t total = g.batch * g.M * g.N;
    splitk_reduce_kernel<R><<<(unsigned)std::min<int64_t>((total + 255) / 256, 65535), 256, 0, s>>>(g, alpha, beta, P,
                                                                                                     splits, C);
  }
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template int qtt_gemm_ex<double>(const GemmDesc&, zc, zc, const zc*, const zc*, zc*, int, zc*, cudaStream_t, int);
template int qtt_gemm_ex<float>(const GemmDesc&, cc, cc, const cc*, const cc*, cc*, int, cc*, cudaStream_t, int);

// the rule's tile edge and the split count the rule would take with a given tile
int qtt_gemm_tile_rule(const GemmDesc& g) { return (int)gemm_tile(g); }
int qtt_gemm_splits_for(const GemmDesc& g, int tile) {
  const int64_t tiles = ((g.M + tile - 1) / tile) * ((g.N + tile - 1) / tile) * g.batch;
  if (tiles >= 76 || g.K < 128) return 1;
  int64_t s = std::min<int64_t>((g.K + 63) / 64, std::max<int64_t>(1, 152 / tiles));
  return (int)std::min<int64_t>(s, 32);
}

template <class R>
int qtt_gemm(const GemmDesc& g, cplx<R> alpha, cplx<R> beta, const cplx<R>* A,
             const cplx<R>* B, cplx<R>* C, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return QTT_OK;
  if (g.K <= 0) {
    // C = beta * C; scale through the kernel with K = 0 (loop body skipped)
  }
  constexpr int BM = 64, BN = 64, TM = 4, TN = 4;
  constexpr int BK = sizeof(R) == 8 ? 8 : 16;
  dim3 grid((unsigned)((g.N + BN - 1) / BN), (unsigned)((g.M + BM - 1) / BM), (unsigned)g.batch);
  if (grid.y > 65535 || grid.z > 65535) return QTT_ERR_ARG;
  gemm_midx_kernel<R, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(g, alpha, beta, A, B, C, 1,
                                                                                std::max<int64_t>(g.K, 1), nullptr);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template int qtt_gemm<double>(const GemmDesc&, zc, zc, const zc*, const zc*, zc*, cudaStream_t);
template int qtt_gemm<float>(const GemmDesc&, cc, cc, const cc*, const cc*, cc*, cudaStream_t);
