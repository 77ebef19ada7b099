/*
 * qtt.h - C-ABI of the GB300 library for the quantized-tensor-train (QTT)
 * Moulinec-Suquet hot path of arXiv 2512.07811 ("Performance Benchmarking of
 * Tensor Trains for Quantum-Inspired Homogenization on TPU, GPU, and CPU
 * Architectures").
 *
 * General conventions
 *  - Every call returns QTT_OK (0) or a negative status (see below); no C++
 *    exception crosses this boundary.  qtt_status_string() names a status.
 *  - A tensor train (TT) with d cores stores core k as a row-major array of
 *    shape (r_{k-1}, n_k, r_k), r_0 = r_d = 1 (Sec. 2, Eq. tt_format; the
 *    paper writes (r_k x p x r_{k-1}), the index order is immaterial).
 *    Elements are interleaved complex numbers: QTT_C128 = two doubles
 *    (C99 double _Complex), QTT_C64 = two floats.
 *  - An operator train (TTO / MPO) stores core k as (g_{k-1}, m_k, n_k, g_k):
 *    output mode m_k, input mode n_k (Sec. 2, Eq. tto_format).
 *  - Combined bonds put the first operand's bond index first (major):
 *    Hadamard (alpha_x, alpha_y), operator application (gamma, alpha),
 *    addition [x block | y block].
 *  - Trains and operators are library-owned device memory on the device of
 *    the context; callers release them with qtt_tt_destroy / qtt_mpo_destroy.
 *    Inputs are never modified and never aliased into outputs; outputs are
 *    freshly allocated and owned by the caller.
 *  - All work is enqueued on the context's stream.  Calls that return host
 *    scalars (tt_dot, tt_norm, ranks chosen by rounding, ms_homogenize)
 *    synchronise that stream.
 *  - The library has no CPU fallback: every operation runs in its CUDA
 *    kernels on an sm_103a device; creating a context fails without one.
 */
#ifndef QTT_H
#define QTT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QTT_API __attribute__((visibility("default")))
#else
#define QTT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ statuses */
#define QTT_OK 0
#define QTT_ERR_ARG -1           /* invalid argument, shape or dtype mismatch   */
#define QTT_ERR_OOM -2           /* device allocation failed                    */
#define QTT_ERR_RANK -3          /* a rank exceeds a fixed workspace limit      */
#define QTT_ERR_TIMEOUT -4       /* a bounded device wait gave up               */
#define QTT_ERR_NOT_CONVERGED -5 /* iteration limit reached before the tolerance */
#define QTT_ERR_NAN -6           /* non-finite values detected in a result      */
#define QTT_ERR_CUDA -7          /* a CUDA runtime call failed                  */
#define QTT_ERR_UNSUPPORTED -8   /* combination not implemented                 */

typedef struct qtt_ctx qtt_ctx;
typedef struct qtt_tt qtt_tt;
typedef struct qtt_mpo qtt_mpo;
typedef struct qtt_mlp qtt_mlp;

typedef enum { QTT_C128 = 0, QTT_C64 = 1 } qtt_dtype;

/* Arithmetic used inside an operation.  QTT_PREC_F64 needs QTT_C128 storage
 * and computes everything in double.  QTT_PREC_F32 (QTT_C64 storage) runs the
 * core contractions and the small factorisations in float, norms, rounding
 * thresholds and residuals in double.  QTT_PREC_TC32 (QTT_C64 storage) is
 * QTT_PREC_F32 with the larger core contractions on the tensor cores
 * (tcgen05.mma kind::tf32, three-term TF32 split, FP32 accumulation in
 * tensor memory): about 1e-5 relative per contraction at K ~ 10^3.
 * QTT_PREC_TF32S (QTT_C64 storage) is QTT_PREC_F32 with the sketch
 * contractions of the sketched roundings (the right partial contractions of
 * the random sketch with the structured sum) on the tensor cores, three-term
 * TF32 split, every batch entry of a contraction in one launch; all other
 * contractions stay on the CUDA cores. */
typedef enum { QTT_PREC_F64 = 0, QTT_PREC_F32 = 1, QTT_PREC_TC32 = 2, QTT_PREC_TF32S = 3 } qtt_prec;

typedef struct {
  double re, im;
} qtt_complex;

/* Outcome of one rounding (Sec. 2.2, Compression via SVD). */
typedef struct {
  double norm;      /* ||x||_F of the (possibly structured) input train          */
  double delta;     /* per-bond threshold eps ||x||_F / sqrt(d - 1)             */
  double tail;      /* sqrt(sum over bonds of squared discarded singular values) */
  double err;       /* exact relative error ||x - y|| / ||x|| when computed, else -1 */
  int32_t capped;   /* 1 if max_rank cut a rank that the tolerance asked for    */
  int32_t max_rank_out;
} qtt_round_info;

/* ------------------------------------------------------------- context */
/* Bind a context to CUDA device `device` and stream `cuda_stream` (a
 * cudaStream_t, or NULL for a new non-blocking stream owned by the context).
 * Fails with QTT_ERR_CUDA if the device is absent or is not sm_103. */
QTT_API int qtt_ctx_create(int device, void* cuda_stream, qtt_ctx** out);
QTT_API void qtt_ctx_destroy(qtt_ctx* ctx);
QTT_API int qtt_ctx_sync(qtt_ctx* ctx);
/* Number of kernels this library has launched on the context so far. */
QTT_API int64_t qtt_ctx_launch_count(const qtt_ctx* ctx);
/* Built-in profiler: with `enable` != 0 every launch of the GEMM (class 0),
 * Householder QR (1), one-sided Jacobi (2) and elementwise (3) kernels is
 * bracketed by CUDA events on the context stream and its model flops and
 * bytes are recorded; enabling or disabling clears the records.  enable = 2
 * records inside ms_homogenize only the iterations of its timed region
 * (report->timed_ms), including those of its load-case workers. */
QTT_API int qtt_ctx_profile(qtt_ctx* ctx, int enable);
/* Totals of one kernel class since profiling was enabled: summed event time
 * (ms), launches, model flops (Jacobi: per-sweep model times the sweeps the
 * kernel ran) and model bytes.  Synchronises the stream. */
QTT_API int qtt_ctx_profile_read(qtt_ctx* ctx, int kclass, double* total_ms, int64_t* launches, double* flops,
                                 double* bytes);
/* The same records of one kernel class grouped by launch shape, this
 * context's own launches only (not those of ms_homogenize's load-case
 * workers: profile a solve with lc_workers = 1 to see its shapes).  Writes up
 * to `max_rows` rows of 8 doubles to `rows` (host, caller-owned, 8 *
 * max_rows), by decreasing total time: d0, d1, d2, batch, variant, launches,
 * total ms, model flops -- GEMM: M, N, K, batch and variant = tile edge x 100
 * + split-K count (tile edge 128: the tensor-core kernel, + its TF32
 * passes); QR: m, n, 0, batch, variant 1 when the explicit Q was formed;
 * Jacobi: rows p, columns q, 0, batch, 0.  *n_rows = the number of distinct
 * shapes (may exceed max_rows).  Synchronises the stream.  QTT_ERR_ARG on a
 * bad class or null pointers. */
QTT_API int qtt_ctx_profile_shapes(qtt_ctx* ctx, int kclass, double* rows, int64_t max_rows, int64_t* n_rows);
/* Failure injection for tests of the error paths (not in the paper): after
 * `n` more successful device allocations of this context, every allocation
 * fails as if the device were out of memory, so the call in progress
 * returns QTT_ERR_OOM after releasing what it holds.  n < 0 switches the
 * injection off again.  Host-side only: no kernel is affected. */
QTT_API int qtt_ctx_fail_alloc_after(qtt_ctx* ctx, int64_t n);

/* Arithmetic peak of the context's GPU in TFLOP/s, measured by the
 * library's own kernels (not in the paper; the rooflines are quoted against
 * them): QTT_PEAK_FP32_FMA / QTT_PEAK_FP64_FMA, a full grid of independent
 * fused-multiply-add chains (two flops each), best of five timed launches;
 * QTT_PEAK_TF32_MMA / QTT_PEAK_BF16_MMA, one CTA per SM issuing tcgen05.mma
 * (M 128, N 256, FP32 accumulation in tensor memory) from operand tiles held
 * in shared memory, best of three, no loads (the tensor pipe's issue rate).
 * Synchronises the stream; QTT_ERR_ARG for another `which`, QTT_ERR_TIMEOUT
 * if a bounded wait gave up. */
#define QTT_PEAK_FP32_FMA 0
#define QTT_PEAK_FP64_FMA 1
#define QTT_PEAK_TF32_MMA 2
#define QTT_PEAK_BF16_MMA 3
QTT_API int qtt_measure_peak(qtt_ctx* ctx, int which, double* tflops);

/* --------------------------------------------------------------- trains */
/* New train with the given modes (d entries) and ranks (d + 1 entries,
 * ranks[0] = ranks[d] = 1), zero-filled. */
QTT_API int qtt_tt_create(qtt_ctx* ctx, int ncores, const int32_t* modes, const int32_t* ranks, qtt_dtype dtype,
                  qtt_tt** out);
QTT_API void qtt_tt_destroy(qtt_tt* x);
QTT_API int qtt_tt_ncores(const qtt_tt* x);
QTT_API int qtt_tt_ranks(const qtt_tt* x, int32_t* ranks /* ncores + 1 */);
QTT_API int qtt_tt_modes(const qtt_tt* x, int32_t* modes /* ncores */);
QTT_API int qtt_tt_dtype(const qtt_tt* x);
/* Device address of core k (valid until the train is destroyed). */
QTT_API void* qtt_tt_core_ptr(const qtt_tt* x, int core);
/* Copy core k from / to host memory (r_{k-1} * n_k * r_k complex elements). */
QTT_API int qtt_tt_from_host(qtt_tt* x, int core, const void* buf);
QTT_API int qtt_tt_to_host(const qtt_tt* x, int core, void* buf);
/* Copy core k from device memory of the same device (stream-ordered). */
QTT_API int qtt_tt_from_device(qtt_tt* x, int core, const void* dev_buf);
/* y = x stored in another dtype (rounds to nearest when narrowing). */
QTT_API int qtt_tt_convert(qtt_ctx* ctx, const qtt_tt* x, qtt_dtype dtype, qtt_tt** y);

/* ------------------------------------------------------------ operators */
QTT_API int qtt_mpo_create(qtt_ctx* ctx, int ncores, const int32_t* modes_out, const int32_t* modes_in,
                   const int32_t* ranks, qtt_dtype dtype, qtt_mpo** out);
QTT_API void qtt_mpo_destroy(qtt_mpo* A);
QTT_API int qtt_mpo_ranks(const qtt_mpo* A, int32_t* ranks /* ncores + 1 */);
QTT_API int qtt_mpo_from_host(qtt_mpo* A, int core, const void* buf);
QTT_API int qtt_mpo_to_host(const qtt_mpo* A, int core, void* buf);

/* --------------------------------------------------------- TT algebra */
/* z = a x + b y by block placement (Sec. 2.1, Addition; constant
 * multiplication rescales the first cores, Eq. tt_const_multiplication).
 * Ranks add.  x and y need equal modes and dtypes. */
QTT_API int tt_add(qtt_ctx* ctx, qtt_complex a, const qtt_tt* x, qtt_complex b, const qtt_tt* y, qtt_tt** z);

/* z = x (elementwise) y: C_k(i) = A_k(i) (kron) B_k(i) (Sec. 2.1, Hadamard
 * product).  Ranks multiply. */
QTT_API int tt_hadamard(qtt_ctx* ctx, const qtt_tt* x, const qtt_tt* y, qtt_tt** z);

/* y = A x: B_k(i) = sum_j D_k(i, j) (kron) A_k(j) (Sec. 2.1, TT-TTO
 * contraction).  Ranks multiply. */
QTT_API int tt_mpo_apply(qtt_ctx* ctx, const qtt_mpo* A, const qtt_tt* x, qtt_tt** y);

/* SVD-based rounding (Sec. 2.2, Orthogonalization and Compression via SVD):
 * a left-to-right QR sweep, ||x|| from the orthogonality centre, the
 * threshold delta = eps ||x|| / sqrt(d - 1) (Eq. optimal_delta, read with
 * sqrt(d-1)), then a right-to-left sweep of truncated SVDs keeping the
 * smallest rank whose discarded tail is <= delta, capped at max_rank (<= 0:
 * no cap).  The output's cores 2..d are right-orthonormal.  `prec` must
 * match the dtype (F64 for C128, F32 for C64).  `info` may be NULL. */
QTT_API int tt_round(qtt_ctx* ctx, const qtt_tt* x, double eps, int max_rank, qtt_prec prec, qtt_round_info* info,
             qtt_tt** y);

/* Compression via polar decomposition (Sec. 2.2): the sweeps of tt_round
 * with the truncated SVD of each centre replaced by its polar
 * decomposition T = U H, the sign function of H - dt I (dt = delta / q, q the
 * centre's number of singular values), the projector P+ = (I + sign) / 2,
 * whose trace is the kept rank, and an orthonormal basis C+ of its range
 * (subspace iteration): new core = (U C+)^H.  Computed by Newton-Schulz
 * iterations, i.e. matrix products only (on the tensor cores under
 * QTT_PREC_TC32).  The bound ||x - y|| <= eps ||x|| holds with ranks at
 * least those of tt_round; no rank cap.  info->capped is 0. */
QTT_API int tt_round_polar(qtt_ctx* ctx, const qtt_tt* x, double eps, qtt_prec prec, qtt_round_info* info,
                           qtt_tt** y);

/* Batched SVD-based rounding: count trains of one shape (equal modes, ranks
 * and dtype), each rounded exactly as tt_round would (its own ||x||, delta,
 * truncation ranks and cap), in lockstep: each step of either sweep is one
 * launch per kernel for the whole batch (one QR block and one Jacobi
 * cluster per train), so many independent roundings share the device instead
 * of queueing.  An addition for many RVEs or load cases (the grouped
 * batching the paper lists as future work, Sec. 6); results agree with
 * tt_round to rounding error (the Jacobi sweeps may visit pairs in another
 * order).  x: count input handles; y: count outputs (new handles owned by
 * the caller); info: NULL or count entries.  QTT_ERR_ARG if the shapes
 * differ; trains with a single core are rounded one by one. */
QTT_API int tt_round_batch(qtt_ctx* ctx, int count, const qtt_tt* const* x, double eps, int max_rank, qtt_prec prec,
                           qtt_round_info* info, qtt_tt** y);

/* Randomize-then-orthogonalize rounding of a structured sum
 *     s = sum_t coef[t] * A_t x_t     (A_t = NULL means the identity)
 * without forming s: with the Gaussian sketch train `sketch` (modes = the
 * output modes, ranks l_k) the right partial contractions of s with the
 * sketch are built term by term, then a left-to-right sweep of QR
 * factorisations of the sketched cores projects s onto rank l_k, and a
 * deterministic rounding (tt_round) of that projection applies eps and
 * max_rank.  Not in the paper (Al Daas et
 * al., SIAM J. Sci. Comput. 45, 2023).  All trains share one dtype. */
QTT_API int tt_round_sketched(qtt_ctx* ctx, int nterms, const qtt_complex* coef, const qtt_mpo* const* ops,
                      const qtt_tt* const* xs, const qtt_tt* sketch, double eps, int max_rank, qtt_prec prec,
                      qtt_round_info* info, qtt_tt** y);

/* <y, s> = sum_i conj(y(i)) s(i) for the structured sum s = sum_t coef_t A_t x_t
 * (ops[t] NULL: the identity) without forming s (Sec. 2.1: operator-train
 * application; the transfer products run core by core from the right).
 * All trains and operators of one dtype; FP64 result; synchronises.  Used
 * for the FP64 a-posteriori error of roundings with learned sketch widths. */
QTT_API int tt_dot_structured(qtt_ctx* ctx, int nterms, const qtt_complex* coef, const qtt_mpo* const* ops,
                              const qtt_tt* const* xs, const qtt_tt* y, double out[2]);
/* out = <x, y> = sum_i conj(x(i)) y(i) through the transfer-matrix chain
 * W_k = sum_i A_k(i)^H W_{k-1} B_k(i); out[0] = real, out[1] = imaginary
 * part.  Accumulates in the storage precision; returns a double. */
QTT_API int tt_dot(qtt_ctx* ctx, const qtt_tt* x, const qtt_tt* y, double out[2]);

/* ||x||_F as the norm of the orthogonality centre after the QR sweep
 * (Sec. 2.2), which avoids the cancellation of <x, x> for differences. */
QTT_API int tt_norm(qtt_ctx* ctx, const qtt_tt* x, double* out);

/* Dense tensor (device memory, modes[0] slowest) to a train by sequential
 * truncated SVDs of the unfoldings (TT-SVD, Oseledets 2011), threshold
 * eps ||A|| / sqrt(d - 1) per bond, computed in double (QTT_C128 output). */
QTT_API int tt_from_dense(qtt_ctx* ctx, int ncores, const int32_t* modes, const void* dense_c128, double eps,
                  int max_rank, qtt_tt** out);

/* Q_n of QFT_n = R_n Q_n (Sec. 3.2, Fig. 1): the unitary DFT with sign
 * `sign` (-1: exp(-2 pi i jk/N)) whose output bits are left in reversed
 * order, as an operator train of `nbits` sites (site a: output bit of weight
 * 2^(a-1), input bit of weight 2^(nbits-a)), rounded at `tol`, QTT_C128.
 * Up to 12 bits: TT-SVD of the closed-form matrix; beyond: product of the
 * circuit's layers (Hadamard, then the controlled phases of one qubit),
 * rounded after every layer. */
QTT_API int qtt_qft_mpo(qtt_ctx* ctx, int nbits, int sign, double tol, qtt_mpo** out);

/* C = A B for row-major complex64 device matrices A (M x K), B (K x N),
 * C (M x N): engine 0 on the CUDA cores (float FMA), engine 1 on the tensor
 * cores (tcgen05.mma kind::tf32 with the three-term TF32 split, which keeps
 * FP32-level accuracy).  The same routines serve every core contraction of
 * the float path.  QTT_ERR_TIMEOUT if a bounded device wait gave up. */
QTT_API int qtt_cgemm(qtt_ctx* ctx, int64_t M, int64_t N, int64_t K, const void* A, const void* B, void* C,
                      int engine);

/* The same product as qtt_cgemm with engine 1 (tensor cores), for callers
 * that may not allocate device memory: for example a host application that
 * reserves the whole device memory for itself at start-up and forbids its
 * libraries to call cudaMalloc afterwards, or code that must not block on
 * the allocator while it runs.  This call allocates nothing: its working
 * space is a fixed 16 MiB array that the library reserves on every device
 * it is loaded on, kept until the process exits.  The paper has no
 * counterpart; it is a service of this library.
 *  - A, B, C: row-major complex64 device matrices (M x K, K x N, M x N);
 *    `stream` is a cudaStream_t (NULL: the legacy default stream).
 *  - Sizes whose packed operands do not fit the array are rejected with
 *    QTT_ERR_RANK before any GPU work (the working space is
 *    4 (Mp K3 + Np K3 + Mp Np) bytes plus alignment, Mp = M rounded up to
 *    128, Np = 2N rounded up to 128, K3 = 6K rounded up to 32; M = N = K = 384
 *    fits).
 *  - The first call on a device looks up the array's device address (and
 *    checks the device is sm_103); make that first call before any stream
 *    capture.  Every call synchronises `stream`.
 *  - All calls share the one array, which keeps the last call's contents:
 *    calls whose GPU work overlaps (other streams, other host threads) race
 *    on it, so serialise them.
 *  - QTT_ERR_TIMEOUT if a bounded device wait gave up. */
QTT_API int qtt_cgemm_noalloc(void* stream, int64_t M, int64_t N, int64_t K, const void* A, const void* B,
                              void* C);

/* The train x lifted to the operator D(i, j) = x(i) delta(i, j) (Sec. 2.1,
 * Eq. tt_to_tto): applying it is the Hadamard product with x, which lets
 * tt_round_sketched round x (elementwise) y without forming it. */
QTT_API int qtt_mpo_diag(qtt_ctx* ctx, const qtt_tt* x, qtt_mpo** out);
/* B = A stored in another dtype. */
QTT_API int qtt_mpo_convert(qtt_ctx* ctx, const qtt_mpo* A, qtt_dtype dtype, qtt_mpo** out);

/* Algorithm 2's final contract(): the full tensor of x written as a voxel
 * field.  x has the homogenisation's site convention: either a control core
 * (ncomp components) followed by the spatial sites, or spatial sites only
 * (ncomp = 1); nbits_dim and interleaved as in qtt_rve (position space, most
 * significant bit first), 1 to 40 bits in all.  out: host, ncomp x Nx x Ny x
 * Nz complex values of x's dtype, component slowest, z fastest. */
QTT_API int tt_contract_voxels(qtt_ctx* ctx, const qtt_tt* x, const int32_t* nbits_dim, int32_t interleaved,
                               void* out);

/* ---------------------------------------------------------------- AMEn */
typedef struct {
  int32_t sweeps;   /* sweeps made                                                     */
  double dx;        /* largest relative change of a core in the last sweep             */
} qtt_amen_info;

/* y ~ A x by AMEn (Sec. 2.1, the optimisation-based product that the paper
 * applies to the Green operator, Sec. 3.2; Dolgov & Savostyanov's
 * alternating minimal energy with residual enrichment, matrix-vector form):
 * sweeps over the cores replace each core of y by the projection of A x on
 * the interfaces of the others (right-orthogonalised before every sweep),
 * truncate it by SVD at eps ||y|| / sqrt(d - 1), and enrich its basis with
 * the residual A x - y projected on a rank-`kick` residual train z, updated
 * alongside; sweeps stop when no core changes by more than eps (relative),
 * or after max_sweeps; the result is rounded at eps.  A x is never formed:
 * every step contracts the cores of A and x with interfaces of rank
 * (r_y, r_A, r_x).  y0: initial guess (NULL: a Gaussian train of rank 4
 * drawn with `seed`), same modes as A's outputs and x's dtype.  A and x of
 * one dtype (complex128: FP64 arithmetic; complex64: FP32).  QTT_ERR_ARG on
 * mismatched shapes or dtypes. */
QTT_API int tt_amen_mv(qtt_ctx* ctx, const qtt_mpo* A, const qtt_tt* x, const qtt_tt* y0, double eps, int32_t kick,
                       int32_t max_sweeps, uint64_t seed, qtt_tt** y, qtt_amen_info* info);

/* The spatial site order of a grid of 2^nbits_dim[a] voxels per dimension
 * (the order every homogenisation train uses after its control site): for
 * each site p (0-based), dim[p] the dimension and pos[p] the bit level it
 * holds (0 = most significant in position space, least significant in
 * momentum space).  interleaved: level by level (bit a of x, y, z in turn,
 * skipping a dimension whose bits are used up), else grouped by dimension.
 * Host only (no context, no device); dim and pos take at least
 * nbits_dim[0] + nbits_dim[1] + nbits_dim[2] entries; returns that count,
 * or QTT_ERR_ARG. */
QTT_API int qtt_site_order(const int32_t* nbits_dim, int32_t interleaved, int32_t* dim, int32_t* pos);

/* ------------------------------------------------------------ TT-cross */
/* Functions the TT-cross samples (Sec. 3, operator setup: the discretised
 * operands are separated into cores by the TT-cross approximation instead of
 * a TT-SVD of the dense array, so the grid is never stored densely).
 *  QTT_CROSS_GREEN: the Green operator train of the reference medium, modes
 *    (ncomp^2, 2, ..., 2): site 0 the component I * ncomp + J, then the
 *    spatial bits in the momentum convention (every dimension's bits least
 *    significant first, Sec. 3.2); ncomp 3: xi_I xi_J / (k0 |xi|^2); ncomp 6:
 *    the isotropic elastic operator of (lam0, mu0) in Voigt form on
 *    engineering strains; 0 at xi = 0; frequencies xi = k below the Nyquist
 *    index, else k - N.
 *  QTT_CROSS_BOXES: the phase indicator of a union of axis-aligned boxes,
 *    modes (2, ..., 2), position convention (most significant bit first); a
 *    voxel is in phase 2 (value 1) when, on every axis, the periodic distance
 *    |((c - cx + 1/2) mod 1) - 1/2| of its centre c = (x + 1/2) / N from some
 *    box centre is at most that box's half width.
 *  QTT_CROSS_ELLIPSOIDS: the phase indicator of a union of ellipsoids (the
 *    spheres, random ellipsoids and aligned fibres of the 3D workloads),
 *    modes (2, ..., 2), position convention; rows of 15 doubles (cx, cy, cz,
 *    a0, a1, a2, R00, R01, R02, R10, R11, R12, R20, R21, R22): the centre,
 *    the semi-axes (+inf allowed: a cylinder, i.e. a fibre) and the rotation
 *    R (row-major) whose column i is the direction of semi-axis i.  With the
 *    voxel centre c = (x + 1/2) / N, the periodic offsets
 *    D_j = (c_j - centre_j) - rint(c_j - centre_j) (half to even), the
 *    body-frame coordinates u_i = (R[0][i] D_0 + R[1][i] D_1) + R[2][i] D_2
 *    and t_i = u_i / a_i, a voxel is in phase 2 when
 *    (t_0 t_0 + t_1 t_1) + t_2 t_2 <= 1 for some row, each operation an IEEE
 *    double operation in that order.
 * The spatial sites are ordered as in qtt_rve (interleaved level by level,
 * or grouped by dimension). */
typedef enum { QTT_CROSS_GREEN = 1, QTT_CROSS_BOXES = 2, QTT_CROSS_ELLIPSOIDS = 3 } qtt_cross_kind;
typedef struct {
  int32_t kind;          /* qtt_cross_kind                                                 */
  int32_t nbits_dim[3];  /* 2^nbits_dim[a] voxels along x, y, z: 0 to 20 each, 1 to 60 in all */
  int32_t interleaved;
  int32_t ncomp;         /* GREEN: 3 or 6                                                  */
  double k0, lam0, mu0;  /* GREEN: reference conductivity / Lame constants                 */
  const double* boxes;   /* BOXES: host, nboxes rows (cx, cy, cz, hx, hy, hz)             */
  int32_t nboxes;
  const double* ellipsoids; /* ELLIPSOIDS: host, nellipsoids rows of 15 (see above)        */
  int32_t nellipsoids;
} qtt_cross_fn;

typedef struct {
  int32_t half_sweeps;   /* half-sweeps made                                               */
  int64_t evaluations;   /* function samples taken                                         */
  double rel_change;     /* ||x_h - x_{h-1}|| / ||x_h|| over the last half-sweep           */
  int32_t max_rank;      /* largest bond rank before the final rounding                    */
} qtt_cross_info;

/* TT-cross approximation of the function `fn` (rank-adaptive two-site cross
 * with maximum-volume index sets, Oseledets & Tyrtyshnikov; Savostyanov &
 * Oseledets): half-sweeps alternate left to right and right to left; at
 * every bond the sampled two-site superblock is truncated by SVD at
 * eps ||S||_F / sqrt(d - 1) (at most max_rank singular vectors, 0 = no cap),
 * `kick` Gaussian columns are appended so that the index sets keep
 * exploring, and the maximum-volume rows (tolerance 1.05, at most 100 swaps)
 * become the next index set.  The sweep stops once the train changes by at
 * most 10 eps (relative) over a half-sweep, or after max_half_sweeps (at
 * least 2); the result is then rounded at eps (FP64 SVD rounding).  Every
 * step runs on the device; complex128 train.  seed: the initial index sets
 * (8 random points, plus the voxel of every box centre for a box geometry)
 * and the Gaussian columns.  Inside ms_homogenize: kick 4 for the Green
 * operator, 8 for a box geometry, at most 24 half-sweeps.  QTT_ERR_ARG for an invalid
 * description, QTT_ERR_RANK if a superblock's kept basis is rank deficient. */
QTT_API int tt_cross(qtt_ctx* ctx, const qtt_cross_fn* fn, double eps, int32_t max_rank, int32_t kick,
                     int32_t max_half_sweeps, uint64_t seed, qtt_tt** out, qtt_cross_info* info);

/* ---------------------------------------------------- homogenisation */
typedef struct {
  int32_t ncomp;        /* 3: scalar conductivity, 6: elasticity (Voigt 11,22,33,23,13,12) */
  int32_t nbits;        /* N = 2^nbits voxels per side (a cube; see nbits_dim)             */
  const double* indicator; /* host, Nx*Ny*Nz values 0/1 (1 = phase 2), x slowest, z fastest */
  double k1, k2;        /* scalar: phase conductivities                                    */
  double lam1, mu1, lam2, mu2; /* elasticity: Lame constants of phases 1 and 2             */
  int32_t interleaved;  /* site order: 1 = x1 y1 z1 x2 ... (level by level), 0 = grouped   */
  int32_t nbits_dim[3]; /* if any is nonzero: 2^nbits_dim[a] voxels along x, y, z (0 to 15
                         * each, 1 to 27 in all; nbits is then ignored).  A dimension of
                         * 2^0 = 1 voxel has no sites: every field is uniform along it, the
                         * plane problem (plane strain for elasticity) for nbits_dim[2] = 0. */
  const double* boxes;  /* host; used when indicator is NULL: nboxes rows (cx, cy, cz, hx,
                         * hy, hz) of axis-aligned boxes in unit-cell coordinates (the
                         * phase-2 region, see qtt_cross_fn), the phase train then built by
                         * tt_cross; the grid may then have 0 to 20 bits per dimension and
                         * 1 to 60 in all                                                   */
  int32_t nboxes;
  int32_t op_cross;     /* 1: build the Green operator train by tt_cross; 0: by a dense
                         * TT-SVD up to 27 bits in all, by tt_cross above               */
  const double* ellipsoids; /* host; used when indicator and boxes are NULL: nellipsoids
                         * rows of 15 (centre, semi-axes, rotation; see qtt_cross_fn) of
                         * a union of ellipsoids, the phase train then built by tt_cross
                         * (grids as for boxes)                                           */
  int32_t nellipsoids;
} qtt_rve;

/* Per-bond rank features of one rounding inside ms_homogenize (the rank
 * predictor's input), QTT_MLP_FEATURES floats per bond k = 1..d-1:
 *  0 k/d                      1 log2(1 + structured input rank at bond k)/10
 *  2 log2(1 + previous output rank at k, same step)/10 (0 on the first iteration)
 *  3, 4 the same at k-1 and k+1       5 -log10(eps)/10
 *  6 log2(1 + max_rank)/10            7 step id/8 (0 contrast, 1-3 SFFT x,y,z,
 *                                       4 Green, 5-7 inverse SFFT z,y,x)
 *  8 min(iteration, 20)/20            9 log2 of the smaller mode product on
 *                                       either side of the bond / 20
 * target: log2(output rank at bond k). */
#define QTT_MLP_FEATURES 10

typedef struct {
  qtt_prec prec;        /* arithmetic of the iteration                                    */
  double eps;           /* rounding tolerance of every step                               */
  double op_tol;        /* tolerance of the operator trains (phase, Green); float paths
                           with op_tol >= 1e-7 build them in float (ms_setup)             */
  int32_t max_iter;
  int32_t oversample;   /* sketch width = max_rank + oversample                           */
  int32_t load_mask;    /* bit k set: solve load case E = e_k (column k of C_eff)        */
  int32_t min_iter;
  uint64_t seed;        /* counter-based generator seed for the sketches                 */
  const qtt_mlp* predictor; /* NULL: every sketch has width max_rank + oversample; else the
                            per-bond widths are 1.25 * predicted rank + oversample and the
                            result is judged: the SFFT and update roundings by their FP64
                            a-posteriori error ||s - y|| (exact, from FP64 inner products;
                            above (2 eps + 1e-5 on the float path) ||s|| they are redone at
                            the full width, then by the deterministic SVD rounding of the
                            explicit sum when its rank is at most 4096), the contrast and
                            Green roundings by saturation (a bond whose rank comes within the
                            oversampling of its narrowed width is widened)                 */
  float* trace;          /* NULL or host buffer receiving (features, target) rows of every
                            sketched rounding: QTT_MLP_FEATURES + 1 floats per bond          */
  int64_t trace_cap;     /* capacity of `trace` in rows                                     */
  int32_t green_amen;    /* 1: the Green step eps^ = Gamma0 tau^ by AMEn (tt_amen_mv, kick 4,
                            at most 12 sweeps, warm-started from the previous iteration's
                            eps^) instead of the MPO x TT product with a sketched rounding  */
  qtt_tt** strain;       /* NULL, or receives the converged strain train of the last solved
                            load case (control core first, site order of the RVE, the
                            iteration's dtype); *strain must be NULL or a train the call
                            may destroy; ms_homogenize_batch ignores it                    */
  int32_t lc_workers;    /* load cases solved at the same time, each on its own stream and
                            host thread, all sharing the one set of operator trains (0 or 1:
                            one after another; ignored when trace or strain is requested)  */
  int32_t warm_iter;     /* iterations of every load case before report->timed_ms starts */
} ms_opts;

typedef struct {
  int32_t iterations[6];
  double residual[6];      /* last relative change ||eps_{m+1} - eps_m|| / ||E 1|| (FP64) */
  double sigma_imag_max;   /* max |Im sigma_eff| (diagnostic)                             */
  int32_t max_rank_seen;
  double setup_ms, iterate_ms;
  int64_t kernel_launches;
  int64_t trace_len;       /* rows written to opts->trace                                 */
  int64_t sketch_width_sum;/* sum over roundings and bonds of the sketch ranks used      */
  int32_t fallbacks;       /* sketched roundings redone at the full width                */
  int32_t green_rank;      /* largest bond rank of the Green operator train              */
  int32_t phase_rank;      /* largest bond rank of the phase indicator train             */
  int32_t fp64_residuals;  /* float path: stop tests evaluated from FP64 inner products  */
  double timed_ms;         /* wall time from the moment every load case running at the
                              start has made opts->warm_iter iterations (streams synchronised)
                              until every load case has finished                          */
  int32_t timed_iter;      /* iterations (summed over load cases) inside timed_ms          */
  int64_t timed_launches;  /* kernel launches of those iterations                          */
  int32_t post_checks;     /* learned widths: roundings judged by their FP64 a-posteriori
                              error (the SFFT steps and the update)                        */
  int32_t svd_fallbacks;   /* judged roundings redone by deterministic SVD rounding of the
                              explicit sum (the full-width sketch still above the bound)   */
  double post_err_max;     /* largest a-posteriori error / ||s|| of the judged roundings    */
} ms_report;

/* Moulinec-Suquet homogenisation in QTT form (Sec. 3.2, Algorithm 2):
 *   tau = round((C - C0) eps_m);  tau^ = S tau;  eps^ = round(Gamma0 tau^);
 *   eps_{m+1} = round(E - S^{-1} eps^);  stop when
 *   ||eps_{m+1} - eps_m||_F / ||E 1||_F < tol (Algorithm 2; Appendix A for the
 * effective tensor, sigma_eff = <C eps>).  C0 is the isotropic reference
 * (3x3 k0*I or Voigt 6x6, row-major).  Each rounding uses the sketched
 * rounding with width max_rank + oversample.  S is applied one dimension at
 * a time for interleaved sites, and as one operator train (the product of
 * the three, whose bonds do not multiply) for sites grouped by dimension;
 * the last inverse transform is applied inside the update's rounding,
 * round(E - S^{-1} eps^) as one two-term sketched rounding.  The stop test
 * is evaluated in FP64 on both paths: by a QR sweep of the difference train
 * on the FP64 path, and from FP64 inner products of the exactly widened
 * iterates, <a,a> + <b,b> - 2 Re <a,b>, on the float path (absolute error
 * about 1e-8 relative to ||E 1||, so float-path tolerances below 1e-6 are
 * not meaningful; its iterates' own noise is larger).  C_eff (ncomp x
 * ncomp, row-major, real part) receives the columns of the load cases in
 * opts->load_mask; `report` may be NULL. */
QTT_API int ms_homogenize(qtt_ctx* ctx, const qtt_rve* rve, const double* C0, double tol, int max_rank,
                  const ms_opts* opts, double* C_eff, ms_report* report);

/* The same solve in two parts, so that one RVE's operator trains serve many
 * solves (precisions, tolerances, load cases):
 *  ms_setup builds the trains of `rve` and C0 (what ms_homogenize does before
 *  its iterations; op_tol as opts->op_tol), on ctx's stream, and returns a
 *  handle owning them; the host arrays of `rve` are not kept.  op_prec
 *  QTT_PREC_F64: every factorisation in FP64; QTT_PREC_F32 (op_tol >= 1e-7
 *  only, else QTT_ERR_ARG): the dense TT-SVDs (phase image, Green
 *  operator) in complex64, the TT-cross samplings in FP64.  ms_homogenize
 *  itself takes QTT_PREC_F32 for the float paths when opts->op_tol >= 1e-7.
 *  ms_homogenize_ops runs the iterations of ms_homogenize on a handle, on
 *  any context of the same device (the trains are only read);
 *  report->setup_ms is 0 there.
 *  ms_ops_destroy frees the trains on the stream of the setup's context,
 *  which must still exist; ms_ops_ranks reports the largest bond ranks of
 *  the Green operator and phase trains.  Not in the paper as an interface;
 *  the paper builds the operators once per RVE as well (Sec. 3.2). */
typedef struct ms_ops ms_ops;
QTT_API int ms_setup(qtt_ctx* ctx, const qtt_rve* rve, const double* C0, double op_tol, qtt_prec op_prec,
                     ms_ops** out);
QTT_API int ms_homogenize_ops(qtt_ctx* ctx, const ms_ops* ops, double tol, int max_rank, const ms_opts* opts,
                              double* C_eff, ms_report* report);
QTT_API void ms_ops_destroy(ms_ops* ops);
QTT_API int ms_ops_ranks(const ms_ops* ops, int32_t* green_rank, int32_t* phase_rank);

QTT_API /* Many RVEs at once: the operator trains of every RVE are built once
 * (ms_setup, RVEs spread over the workers), then the (RVE, load case) pairs
 * of rves[0..n-1] (load cases from opts->load_mask) are solved by `workers`
 * host threads, each with its own context and stream, largest RVE first, so
 * that independent rounding chains run concurrently on different SMs.  C0s holds n reference tensors
 * at a stride of 36 doubles (3x3 or 6x6 row-major at the start of each
 * slot); C_effs receives the effective tensors back to back (ncomp^2 each);
 * reports (nullable) one report per RVE.  Every pair gives the same result
 * as its own ms_homogenize call.  Trace recording is off in this call. */
QTT_API int ms_homogenize_batch(qtt_ctx* ctx, int n, const qtt_rve* rves, const double* C0s, double tol,
                                int max_rank, const ms_opts* opts, int workers, double* C_effs,
                                ms_report* reports);

/* ------------------------------------------------ rank predictor (MLP) */
/* A multilayer perceptron with three hidden layers of width 64 and ReLU, FP16
 * weights, FP32 accumulation, FP32 master weights and Adam moments; it maps
 * QTT_MLP_FEATURES (or any n_features <= 32) per-bond features to a predicted
 * log2 rank.  Not in the paper (nearest
 * relative: the coarse-grained ranks of Sec. 5.1).  Packed parameter order:
 * W0 (64 x F), b0 (64), W1 (64 x 64), b1, W2 (64 x 64), b2, W3 (64), b3 (1),
 * weights row-major (out, in).  Host buffers throughout; every call
 * synchronises the context stream. */
QTT_API int qtt_mlp_create(qtt_ctx* ctx, int n_features, uint64_t seed, qtt_mlp** out);
QTT_API void qtt_mlp_destroy(qtt_mlp* m);
QTT_API int64_t qtt_mlp_param_count(const qtt_mlp* m);
/* Replace the FP32 master parameters (the FP16 weights are rounded from them)
 * and reset the Adam moments. */
QTT_API int qtt_mlp_set_params(qtt_mlp* m, const float* params, int64_t count);
QTT_API int qtt_mlp_get_params(const qtt_mlp* m, float* params, int64_t count);
/* y[b] for the B rows of X (B x F, row-major). */
QTT_API int qtt_mlp_forward(qtt_mlp* m, const float* X, int64_t B, float* y);
/* One training step on the batch: the asymmetric loss
 * (1/B) sum w_b (y_b - t_b)^2, w_b = alpha where y_b < t_b, else 1; its
 * gradient by the hand-written backward kernel; one Adam update with rate lr.
 * Returns the loss before the update; `grads` (nullable) receives the packed
 * gradient. */
QTT_API int qtt_mlp_train_step(qtt_mlp* m, const float* X, const float* t, int64_t B, float alpha, float lr,
                               double* loss, float* grads);

QTT_API const char* qtt_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* QTT_H */
