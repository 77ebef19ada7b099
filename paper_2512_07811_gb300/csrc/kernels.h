// Internal kernel launchers (C++ linkage; not part of the C-ABI).
#pragma once

#include "common.cuh"

// raise a kernel's dynamic shared-memory limit to the maximum once per device (linalg.cu)
int qtt_allow_max_smem(const void* func);

template <class R>
int qtt_gemm(const GemmDesc& g, cplx<R> alpha, cplx<R> beta, const cplx<R>* A, const cplx<R>* B,
             cplx<R>* C, cudaStream_t s);

// split-K aware variant: `splits` K ranges, partials in P (splits x batch x M x N), see qtt_gemm_splits
int qtt_gemm_splits(const GemmDesc& g);
// tile: 0 = the rule (gemm_tile), else 32 or 64
template <class R>
int qtt_gemm_ex(const GemmDesc& g, cplx<R> alpha, cplx<R> beta, const cplx<R>* A, const cplx<R>* B, cplx<R>* C,
                int splits, cplx<R>* P, cudaStream_t s, int tile = 0);
int qtt_gemm_tile_rule(const GemmDesc& g);
int qtt_gemm_splits_for(const GemmDesc& g, int tile);

template <class R>
int qtt_qr_r(const cplx<R>* in, MIdx inB, MIdx rowI, MIdx colI, int conj_in, int64_t m, int64_t n,
             int64_t rows_total, int64_t rows_per_batch, int64_t batch, cplx<R>* W, cplx<R>* out,
             int64_t out_bstride, int64_t ldr, cudaStream_t s, cplx<R>* tauws = nullptr,
             cplx<R>* Qout = nullptr, int64_t q_bstride = 0, int64_t ldq = 0, cplx<R>* Qws = nullptr);

template <class R>
size_t qtt_jacobi_smem_bytes(int p, int q);
template <class R>
int qtt_jacobi_smem(const cplx<R>* G, cplx<R>* Vws, R* sigma, cplx<R>* Vsorted, cplx<R>* Usorted, int p, int q,
                    int max_sweeps, int* sweeps, cudaStream_t s);

template <class R>
int qtt_jacobi(cplx<R>* G, cplx<R>* Vwork, R* sigma, cplx<R>* Vsorted, int p, int q, int batch,
               int max_sweeps, int* sweeps, cudaStream_t s, cplx<R>* Usorted = nullptr);

template <class R>
int qtt_jacobi_wide(const cplx<R>* G, cplx<R>* Gwork, cplx<R>* Vwork, R* sigma, cplx<R>* Vsorted, cplx<R>* Usorted,
                    int p, int q, int max_sweeps, int* dflag, int* sweeps_done, int64_t* launches, cudaStream_t s);

template <class R>
int qtt_trunc_rank(const R* sigma, int q, double delta, int max_rank, int* out, double* tail,
                   cudaStream_t s);

// ---- elementwise / placement kernels (elem.cu)
template <class R>
int qtt_place_block(const cplx<R>* src, int64_t s0, int64_t n, int64_t s1, cplx<R>* dst, int64_t d1,
                    int64_t off0, int64_t off1, cplx<R> scale, cudaStream_t s);
template <class R>
int qtt_hadamard_core(const cplx<R>* x, int64_t a0, int64_t a1, const cplx<R>* y, int64_t b0,
                      int64_t b1, int64_t n, cplx<R>* out, cudaStream_t s);
template <class R>
int qtt_mpo_core(const cplx<R>* D, int64_t g0, int64_t no, int64_t ni, int64_t g1, const cplx<R>* X,
                 int64_t a0, int64_t a1, cplx<R>* out, cudaStream_t s);
template <class R>
int qtt_scale(cplx<R>* x, int64_t count, cplx<R> scale, cudaStream_t s);
template <class R>
int qtt_sumsq(const cplx<R>* x, int64_t count, double* out, cudaStream_t s);
int qtt_convert_z2c(const zc* in, cc* out, int64_t count, cudaStream_t s);
int qtt_convert_c2z(const cc* in, zc* out, int64_t count, cudaStream_t s);
template <class R>
int qtt_copy_strided(const cplx<R>* in, MIdx rows, MIdx cols, int64_t nrows, int64_t ncols, int conj_in,
                     cplx<R>* out, int64_t ldo, cudaStream_t s);
template <class R>
int qtt_scale_rows(cplx<R>* x, int64_t rows, int64_t cols, int64_t ld, const R* sv, int invert,
                   cudaStream_t s);
template <class R>
int qtt_isfinite(const cplx<R>* x, int64_t count, int* flag, cudaStream_t s);

// ---- operator construction on the device (elem.cu)
template <class R>
int qtt_fill_qft_dense(cplx<R>* out, int n, double sign, cudaStream_t s);
template <class R>
int qtt_fill_green_dense(cplx<R>* out, const SiteMap& m, int ncomp, double k0, double lam0, double mu0,
                         cudaStream_t s);
template <class R>
int qtt_fill_indicator_sites(const double* ind, const SiteMap& m, cplx<R>* out, cudaStream_t s);
template <class R>
int qtt_fill_gaussian(cplx<R>* out, int64_t count, uint64_t seed, uint64_t stream, double scale, cudaStream_t s);
template <class R>
int qtt_diag_mpo_core(const cplx<R>* X, int64_t r0, int64_t n, int64_t r1, cplx<R>* D, cudaStream_t s);
template <class R>
int qtt_identity_core(int64_t g, int64_t n, cplx<R>* D, cudaStream_t s);
template <class R>
int qtt_adjoint_core(const cplx<R>* D, int64_t g0, int64_t no, int64_t ni, int64_t g1, cplx<R>* out,
                     cudaStream_t s);

// tensor-core complex64 GEMM (tc_gemm.cu), batch 1
size_t qtt_tc_gemm_workspace(int64_t M, int64_t N, int64_t K);
size_t qtt_tc_gemm_workspace_ex(int64_t M, int64_t N, int64_t K, int64_t batch, int passes);
int qtt_tc_gemm_ex(const GemmDesc& g, cc alpha, cc beta, const cc* A, const cc* B, cc* C, void* ws, int* err,
                   cudaStream_t s, int passes);
int qtt_tc_gemm(const GemmDesc& g, cc alpha, cc beta, const cc* A, const cc* B, cc* C, void* ws, int* err,
                cudaStream_t s);

// one-sided Jacobi over a thread-block cluster of nc CTAs (4 or 8), rows split over the CTAs (linalg.cu)
template <class R>
size_t qtt_jacobi_cluster_bytes(int p, int q, int nc);
template <class R>
int qtt_jacobi_cluster(const cplx<R>* G, R* sigma, cplx<R>* Vsorted, cplx<R>* Usorted, int p, int q, int nc,
                       int max_sweeps, int* sweeps, cudaStream_t s);

// block-cyclic one-sided Jacobi over a cluster (columns split into blocks, linalg.cu); no rotations output
template <class R>
int qtt_jacobi_block_plan(int p, int q, int* bs_out);
// batch: that many p x q matrices back to back (sigma q apart, Usorted p*q apart), one cluster each
template <class R>
int qtt_jacobi_block(const cplx<R>* G, R* sigma, cplx<R>* Usorted, int p, int q, int max_sweeps, int* sweeps,
                     cudaStream_t s, int batch = 1);
// truncation rule for a batch of sorted singular-value vectors (q apart), delta per vector;
// out[4b] = t, out[4b+1] = capped, out[4b+2..3] = discarded tail (double)
template <class R>
int qtt_trunc_rank_batch(const R* sigma, int q, const double* delta, int max_rank, int* out, int batch,
                         cudaStream_t s);
// ---- batched copies (elem.cu)
// out[b*ob + i*ldo + j] = op(in[b*ib + rows(i) + cols(j)]), op = conj if conj_in
template <class R>
int qtt_copy_batch(const cplx<R>* in, int64_t ib, MIdx rows, MIdx cols, int64_t nrows, int64_t ncols, int conj_in,
                   cplx<R>* out, int64_t ldo, int64_t ob, int batch, cudaStream_t s);
// zero columns j >= t[b * tstride] of each rows x cols matrix (leading dimension ld, matrices bs apart)
template <class R>
int qtt_mask_cols_batch(cplx<R>* X, int64_t bs, int64_t rows, int64_t cols, int64_t ld, const int* t, int tstride,
                        int batch, cudaStream_t s);
// dst[b] (t0[b] x n x t1[b]) = src[b][:t0[b], :, :t1[b]] of the padded r0 x n x r1 cores (src cores sb apart)
template <class R>
int qtt_crop_batch(const cplx<R>* src, int64_t sb, int64_t r0, int64_t n, int64_t r1, cplx<R>* const* dst,
                   const int* t0, const int* t1, int batch, cudaStream_t s);
// polar compression helpers (elem.cu): out = (H + H^H)/2 - shift I; S <- (I + S)/2 with Re tr into *tr
template <class R>
int qtt_herm_shift(const cplx<R>* H, int64_t q, double shift, cplx<R>* out, cudaStream_t s);
template <class R>
int qtt_half_identity_plus(cplx<R>* S, int64_t q, double* tr, cudaStream_t s);

// TT-cross (cross.cu): superblock sampler, maximum-volume rows, index sets
template <class R>
int qtt_cross_eval(const CrossFn& f, int d, int k, const uint8_t* Il, int rl, const uint8_t* Jr, int rr, int n0,
                   int n1, int herm, cplx<R>* out, cudaStream_t s);
template <class R>
size_t qtt_maxvol_smem(int m, int r);
template <class R>
int qtt_maxvol(cplx<R>* A, int m, int r, int* piv, double tol, int max_iters, int* status, cudaStream_t s);
int qtt_cross_left_index(const uint8_t* Iprev, int k, int n0, const int* piv, int t, uint8_t* Inew, cudaStream_t s);
int qtt_cross_right_index(const uint8_t* Jnext, int nr, int rr, const int* piv, int t, uint8_t* Jnew, cudaStream_t s);
template <class R>
int qtt_cross_gather(const cplx<R>* S, int64_t ld, const int* piv, int t, int64_t len, int trans, cplx<R>* out,
                     cudaStream_t s);

// full tensor in site order (control first) -> voxel field (elem.cu)
template <class R>
int qtt_sites_to_voxels(const cplx<R>* in, const SiteMap& m, int ncomp, cplx<R>* out, cudaStream_t s);
