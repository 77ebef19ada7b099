// Complex GEMM on the 5th-generation tensor cores (tcgen05, kind::tf32) for
// the FP32 path.
//
// C = alpha op(A) op(B) + beta C with complex64 operands given through
// two-level strided views (any contraction of the tensor-train path) is
// computed as ONE real GEMM C3 = A3 B3^T on packed operands:
//   A2 = [Ar | Ai]                       (M x 2K, K contiguous)
//   B2 = [[Br^T | -Bi^T]; [Bi^T | Br^T]] (2N x 2K)   =>  A2 B2^T = [Cr | Ci]
// and, for FP32-level accuracy, the split x = hi + lo with hi = tf32(x),
// lo = tf32(x - hi): A3 = [A2hi | A2hi | A2lo], B3 = [B2hi | B2lo | B2hi]
// (K3 = 6K, padded to 32), so A3 B3^T = A2hi B2hi^T + A2hi B2lo^T + A2lo B2hi^T
// (three passes); or the single pass A3 = A2hi, B3 = B2hi (K3 = 2K), TF32's
// 11-bit significand (available to callers; the library's own routes use
// three passes).
// A batch of such products runs as one launch: the packed operands are
// stacked [batch][rows][K3] and read through 3D tensor maps, blockIdx.z
// being the batch entry.
//
// The tensor-core kernel: one CTA (128 threads) per 128 x 128 tile of C3;
// TMA (128-byte swizzle, 32 fp32 of K per row) fills a 4-stage ring of A and
// B tiles guarded by mbarriers; one thread issues tcgen05.mma (M = 128,
// N = 128, K = 8 per instruction) into a 128-column FP32 accumulator in
// tensor memory and commits each stage back to the producer; after the last
// stage the four warps read their 32 accumulator lanes with tcgen05.ld and
// store C3.  Every mbarrier wait is bounded: on timeout the kernel records
// the failure in `err`, stops issuing work, still frees its tensor memory and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/qtt.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 32, STAGES = 4;
constexpr int TILE_A_BYTES = TBM * TBK * 4;   // 16 KB
constexpr int TILE_B_BYTES = TBN * TBK * 4;   // 16 KB
constexpr int STAGE_BYTES = TILE_A_BYTES + TILE_B_BYTES;
constexpr uint32_t WAIT_LIMIT = 1u << 26;     // bounded spin (~ seconds), then give up

// ----------------------------------------------------------- packing kernels
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// A3 row m (m < Mp): columns [part*2K + c], c < 2K: c < K -> Re A[m, c], else Im A[m, c-K]
template <int PART_LO>
__device__ __forceinline__ float split_part(float x) {
  float hi = to_tf32(x);
  return PART_LO ? to_tf32(x - hi) : hi;
}

// Packing and unpacking move one 32 x 32 tile of complex values per CTA
// (32 x 8 threads) through shared memory: the reads run along whichever index
// of the source is contiguous, the writes along the packed rows, so both are
// coalesced; the element offsets of the tile's 32 rows and 32 K values are
// computed once per CTA.  The packed buffers are zeroed beforehand, so only
// the valid entries are written.
constexpr int PT = 32;

// A3 row m of batch entry b: [part 0: Re | Im (hi)] [part 1: the same] [part 2: Re | Im (lo)]
// (passes 3; passes 1: part 0 only), each half K wide.  B3 rows n and N + n:
// [Br | -Bi] and [Bi | Br] with parts (hi, lo, hi).
template <int IS_B>
__global__ void __launch_bounds__(256) pack_tile_kernel(const cc* __restrict__ src, MIdx bI, MIdx rI, MIdx kI,
                                                         int conj, int64_t R, int64_t K, int64_t rows_out,
                                                         int64_t K3p, int passes, int r_contig,
                                                         float* __restrict__ out) {
  __shared__ cc tile[PT][PT + 1];
  __shared__ int64_t roff[PT], koff[PT];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * PT + tx;
  const int64_t k0 = (int64_t)blockIdx.x * PT, b = blockIdx.z, base = midx_off(bI, b);
  if (tid < PT) koff[tid] = k0 + tid < K ? midx_off(kI, k0 + tid) : -1;
  // row tiles grid-stride over y (the loop bounds are the same for the whole CTA)
  for (int64_t r0 = (int64_t)blockIdx.y * PT; r0 < R; r0 += (int64_t)gridDim.y * PT) {
    __syncthreads();
    if (tid >= PT && tid < 2 * PT) roff[tid - PT] = r0 + tid - PT < R ? midx_off(rI, r0 + tid - PT) : -1;
    __syncthreads();
    for (int i = ty; i < PT; i += 8) {
      const int rr = r_contig ? tx : i, kk = r_contig ? i : tx;
      cc v(0.f, 0.f);
      if (roff[rr] >= 0 && koff[kk] >= 0) {
        v = src[base + roff[rr] + koff[kk]];
        if (conj) v.im = -v.im;
      }
      tile[rr][kk] = v;
    }
    __syncthreads();
    const int64_t k = k0 + tx;
    if (k >= K) continue;
    for (int i = ty; i < PT; i += 8) {
      const int64_t r = r0 + i;
      if (r >= R) break;
      const cc v = tile[i][tx];
      if (!IS_B) {
        float* row = out + (b * rows_out + r) * K3p;
        const float hr = split_part<0>(v.re), hi = split_part<0>(v.im);
        row[k] = hr;
        row[K + k] = hi;
        if (passes == 3) {
          row[2 * K + k] = hr;
          row[3 * K + k] = hi;
          row[4 * K + k] = split_part<1>(v.re);
          row[5 * K + k] = split_part<1>(v.im);
        }
      } else {
        float* rn = out + (b * rows_out + r) * K3p;      // [Br | -Bi]
        float* rm = out + (b * rows_out + R + r) * K3p;  // [Bi |  Br]
        const float hr = split_part<0>(v.re), hi = split_part<0>(v.im), hmi = split_part<0>(-v.im);
        rn[k] = hr;
        rn[K + k] = hmi;
        rm[k] = hi;
        rm[K + k] = hr;
        if (passes == 3) {
          const float lr = split_part<1>(v.re), li = split_part<1>(v.im), lmi = split_part<1>(-v.im);
          rn[2 * K + k] = lr;
          rn[3 * K + k] = lmi;
          rm[2 * K + k] = li;
          rm[3 * K + k] = lr;
          rn[4 * K + k] = hr;
          rn[5 * K + k] = hmi;
          rm[4 * K + k] = hi;
          rm[5 * K + k] = hr;
        }
      }
    }
  }
}

// C[m, n] = alpha (C3[m, n] + i C3[m, N + n]) + beta C[m, n], one 32 x 32
// tile per CTA step: C3 read along n, C written along its contiguous index
__global__ void __launch_bounds__(256) unpack_tile_kernel(const float* __restrict__ C3, int64_t ldc3,
                                                           int64_t c3_batch, GemmDesc g, cc alpha, cc beta,
                                                           int m_contig, cc* __restrict__ C) {
  __shared__ cc tile[PT][PT + 1];
  __shared__ int64_t moff[PT], noff[PT];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * PT + tx;
  const int64_t n0 = (int64_t)blockIdx.x * PT, b = blockIdx.z, base = midx_off(g.bC, b);
  if (tid < PT) noff[tid] = n0 + tid < g.N ? midx_off(g.nC, n0 + tid) : -1;
  const float* c3 = C3 + b * c3_batch;
  const bool use_beta = beta.re != 0.f || beta.im != 0.f;
  for (int64_t m0 = (int64_t)blockIdx.y * PT; m0 < g.M; m0 += (int64_t)gridDim.y * PT) {
    __syncthreads();
    if (tid >= PT && tid < 2 * PT) moff[tid - PT] = m0 + tid - PT < g.M ? midx_off(g.mC, m0 + tid - PT) : -1;
    for (int i = ty; i < PT; i += 8) {
      const int64_t m = m0 + i, n = n0 + tx;
      cc v(0.f, 0.f);
      if (m < g.M && n < g.N) v = cc(c3[m * ldc3 + n], c3[m * ldc3 + g.N + n]);
      tile[i][tx] = v;
    }
    __syncthreads();
    for (int i = ty; i < PT; i += 8) {
      const int mm = m_contig ? tx : i, nn = m_contig ? i : tx;
      if (moff[mm] < 0 || noff[nn] < 0) continue;
      const int64_t o = base + moff[mm] + noff[nn];
      cc r = alpha * tile[mm][nn];
      if (use_beta) r = r + beta * C[o];
      C[o] = r;
    }
  }
}

// ------------------------------------------------------- PTX helper wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes));
}
// bounded wait on the phase with the given parity; returns false on timeout,
// or as soon as *stop (a CTA-wide abort flag, read through a volatile
// pointer so every poll reloads it) is set, when stop is given
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* stop = nullptr) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
    if (stop && *stop) return false;
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// tile (x, y) of batch entry z of a 3D tensor map (x innermost)
__device__ __forceinline__ void tma_load_3d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// shared-memory matrix descriptor (K-major, 128-byte swizzle): start >> 4,
// leading byte offset 16 (unused with swizzling), stride byte offset 1024
// (eight 128-byte rows), descriptor version 1, swizzle mode 2 (128 B)
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, N, M
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4)                       // D format F32
         | (2u << 7)                     // A format TF32
         | (2u << 10)                    // B format TF32
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__global__ void __launch_bounds__(128, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, float* __restrict__ C3,
               int64_t ldc3, int64_t c3_batch, int k_tiles, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    // 128 columns of FP32 accumulator for the 128 x 128 tile
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  volatile int* abort_v = &abort_sh;
  if (warp == 0 && lane == 0) {
    // producer: TMA loads into the ring
    int issued = 0;
    for (int kt = 0; kt < k_tiles; ++kt) {
      const int s = kt % STAGES;
      const uint32_t round = kt / STAGES;
      if (kt >= STAGES) {
        if (!mbar_wait(&empty_bar[s], (round - 1) & 1, abort_v)) {
          atomicExch(err, 1);
          atomicExch(&abort_sh, 1);
          break;
        }
      }
      if (*abort_v) break;
      unsigned char* a = smem + s * STAGE_BYTES;
      unsigned char* b = a + TILE_A_BYTES;
      mbar_expect_tx(&full_bar[s], STAGE_BYTES);
      tma_load_3d(&mapA, &full_bar[s], a, kt * TBK, m0, (int)blockIdx.z);
      tma_load_3d(&mapB, &full_bar[s], b, kt * TBK, n0, (int)blockIdx.z);
      issued = kt + 1;
    }
    // Drain: every load this thread issued must have landed before the CTA
    // may exit (normally the MMA issuer has consumed them already and these
    // waits return at once).  A stage's latest issued load is the only one
    // that can still be in flight (the stage was refilled only after its
    // previous load was consumed), and a TMA load completes by itself, so
    // these waits end; they are bounded all the same.
    for (int kt = issued - 1; kt >= 0 && kt >= issued - STAGES; --kt) {
      if (!mbar_wait(&full_bar[kt % STAGES], (kt / STAGES) & 1)) atomicExch(err, 4);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = idesc_tf32(TBM, TBN);
    for (int kt = 0; kt < k_tiles; ++kt) {
      const int s = kt % STAGES;
      if (!mbar_wait(&full_bar[s], (kt / STAGES) & 1, abort_v)) {
        atomicExch(err, 2);
        atomicExch(&abort_sh, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = smem_u32(smem + s * STAGE_BYTES);
      const uint32_t b = a + TILE_A_BYTES;
#pragma unroll
      for (int kk = 0; kk < TBK / 8; ++kk) {
        // K advances 8 tf32 = 32 bytes inside the 128-byte swizzle atom
        const uint64_t da = smem_desc_sw128(a + kk * 32);
        const uint64_t db = smem_desc_sw128(b + kk * 32);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      // free the stage once these MMAs have read it
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&empty_bar[s])));
    }
    // issued on every exit path, abort included: done_bar completes once
    // every MMA this thread issued has finished, so the epilogue's wait also
    // orders the tensor-memory release after the last MMA
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(&done_bar)));
  }
  // epilogue: every warp waits for the accumulator, then reads its 32 lanes
  __syncwarp();
  bool ok = mbar_wait(&done_bar, 0);
  if (!ok && lane == 0) atomicExch(err, 3);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    float* crow = C3 + (int64_t)blockIdx.z * c3_batch + (int64_t)row * ldc3 + n0;
#pragma unroll 1
    for (int c0 = 0; c0 < TBN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) crow[c0 + j] = __uint_as_float(v[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TBN));
  }
}

// ------------------------------------------------------ tensor-map encoding
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// batch x rows x cols fp32, row-major (cols contiguous), box 32 (cols) x 128
// (rows) x 1, 128-byte swizzle
bool make_map(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t batch) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)cols * sizeof(float), (cuuint64_t)(rows * cols) * sizeof(float)};
  cuuint32_t box[3] = {(cuuint32_t)TBK, (cuuint32_t)TBM, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// grid.y of the tile kernels: one CTA per 32 rows, at most 65535 (the kernels loop over the rest)
inline unsigned tiles_y(int64_t rows) { return (unsigned)std::min<int64_t>((rows + PT - 1) / PT, 65535); }

}  // namespace

static int64_t k3_pad(int64_t K, int passes) { return ((passes == 3 ? 6 : 2) * K + TBK - 1) / TBK * TBK; }

// Workspace bytes for a batched call (passes 1 or 3).
size_t qtt_tc_gemm_workspace_ex(int64_t M, int64_t N, int64_t K, int64_t batch, int passes) {
  const int64_t Mp = (M + TBM - 1) / TBM * TBM;
  const int64_t Np = (2 * N + TBN - 1) / TBN * TBN;
  const int64_t K3p = k3_pad(K, passes);
  return (size_t)batch * (Mp * K3p + Np * K3p + Mp * Np) * sizeof(float) + 3 * 1024 + 16;
}

// Workspace bytes for one call with the given sizes.
size_t qtt_tc_gemm_workspace(int64_t M, int64_t N, int64_t K) { return qtt_tc_gemm_workspace_ex(M, N, K, 1, 3); }

// Batched complex64 GEMM through the tensor cores, every batch entry of g in
// one launch, 1 or 3 TF32 passes.  `ws` needs qtt_tc_gemm_workspace_ex bytes
// (device), `err` one device int (set non-zero when a bounded wait gave up).
int qtt_tc_gemm_ex(const GemmDesc& g, cc alpha, cc beta, const cc* A, const cc* B, cc* C, void* ws, int* err,
                   cudaStream_t s, int passes) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0 || g.batch > 65535) return QTT_ERR_ARG;
  if ((g.M + TBM - 1) / TBM > 65535 || (g.K + PT - 1) / PT > INT32_MAX) return QTT_ERR_ARG;
  if (passes != 1 && passes != 3) return QTT_ERR_ARG;
  const int64_t Mp = (g.M + TBM - 1) / TBM * TBM;
  const int64_t Np = (2 * g.N + TBN - 1) / TBN * TBN;
  const int64_t K3p = k3_pad(g.K, passes);
  uintptr_t p = (reinterpret_cast<uintptr_t>(ws) + 1023) & ~(uintptr_t)1023;
  float* A3 = reinterpret_cast<float*>(p);
  p = (reinterpret_cast<uintptr_t>(A3 + g.batch * Mp * K3p) + 1023) & ~(uintptr_t)1023;
  float* B3 = reinterpret_cast<float*>(p);
  p = (reinterpret_cast<uintptr_t>(B3 + g.batch * Np * K3p) + 1023) & ~(uintptr_t)1023;
  float* C3 = reinterpret_cast<float*>(p);
  if (cudaMemsetAsync(A3, 0, (size_t)g.batch * Mp * K3p * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(B3, 0, (size_t)g.batch * Np * K3p * sizeof(float), s) != cudaSuccess)
    return QTT_ERR_CUDA;
  const auto unit = [](const MIdx& m) { return (m.n2 == 1 ? m.s1 : m.s2) == 1; };
  {
    dim3 blk(PT, 8), grd((unsigned)((g.K + PT - 1) / PT), tiles_y(g.M), (unsigned)g.batch);
    pack_tile_kernel<0><<<grd, blk, 0, s>>>(A, g.bA, g.mA, g.kA, g.conjA, g.M, g.K, Mp, K3p, passes,
                                            unit(g.mA) && !unit(g.kA) ? 1 : 0, A3);
  }
  {
    dim3 blk(PT, 8), grd((unsigned)((g.K + PT - 1) / PT), tiles_y(g.N), (unsigned)g.batch);
    pack_tile_kernel<1><<<grd, blk, 0, s>>>(B, g.bB, g.nB, g.kB, g.conjB, g.N, g.K, Np, K3p, passes,
                                            unit(g.nB) && !unit(g.kB) ? 1 : 0, B3);
  }
  CUtensorMap ma, mb;
  if (!make_map(&ma, A3, Mp, K3p, g.batch) || !make_map(&mb, B3, Np, K3p, g.batch)) return QTT_ERR_CUDA;
  const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024;
  if (qtt_allow_max_smem((const void*)tc_gemm_kernel) != QTT_OK) return QTT_ERR_CUDA;
  dim3 grid((unsigned)(Np / TBN), (unsigned)(Mp / TBM), (unsigned)g.batch);
  tc_gemm_kernel<<<grid, 128, smem, s>>>(ma, mb, C3, Np, Mp * Np, (int)(K3p / TBK), err);
  {
    dim3 blk(PT, 8), grd((unsigned)((g.N + PT - 1) / PT), tiles_y(g.M), (unsigned)g.batch);
    unpack_tile_kernel<<<grd, blk, 0, s>>>(C3, Np, Mp * Np, g, alpha, beta, unit(g.mC) && !unit(g.nC) ? 1 : 0, C);
  }
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

// Single-batch complex64 GEMM through the tensor cores, three TF32 passes.
int qtt_tc_gemm(const GemmDesc& g, cc alpha, cc beta, const cc* A, const cc* B, cc* C, void* ws, int* err,
                cudaStream_t s) {
  if (g.batch != 1) return QTT_ERR_UNSUPPORTED;
  return qtt_tc_gemm_ex(g, alpha, beta, A, B, C, ws, err, s, 3);
}

// --------------------------------------------- allocation-free entry point
// Scratch of qtt_cgemm_noalloc: the packed operands, the real product and the
// wait-failure flag of one call live in this file-scope device array, so the
// call itself never allocates.  Every device that loads the library holds it
// (16 MiB) until the process exits.  Calls share it: a call overwrites what
// the previous one left, and two calls in flight on the GPU at the same time
// (different streams, or different host threads) would race on it.
#define QTT_NOALLOC_SCRATCH_BYTES (16u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[QTT_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[128] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device address).
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return QTT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return QTT_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return QTT_ERR_UNSUPPORTED;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return QTT_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return QTT_OK;
}
}  // namespace

extern "C" int qtt_cgemm_noalloc(void* stream, int64_t M, int64_t N, int64_t K, const void* A, const void* B,
                                 void* C) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return QTT_ERR_ARG;
  // no operand dimension of a problem that fits the array comes near 2^22;
  // refusing larger ones first keeps the workspace arithmetic below from
  // overflowing
  if (M > (1 << 22) || N > (1 << 22) || K > (1 << 22)) return QTT_ERR_RANK;
  const size_t need = qtt_tc_gemm_workspace(M, N, K);
  if (need + 256 > QTT_NOALLOC_SCRATCH_BYTES) return QTT_ERR_RANK;
  void* base = nullptr;
  int st = noalloc_scratch(&base);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the flag must start at zero; everything else is overwritten by the call
  int* err = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + QTT_NOALLOC_SCRATCH_BYTES - 256);
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return QTT_ERR_CUDA;
  GemmDesc g;
  g.bA = g.bB = g.bC = MIdx{1, 1, 0, 0};
  g.mA = MIdx{M, 1, K, 0};
  g.kA = MIdx{K, 1, 1, 0};
  g.kB = MIdx{K, 1, N, 0};
  g.nB = MIdx{N, 1, 1, 0};
  g.mC = MIdx{M, 1, N, 0};
  g.nC = MIdx{N, 1, 1, 0};
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = 1;
  g.conjA = g.conjB = 0;
  st = qtt_tc_gemm(g, cc(1.f, 0.f), cc(0.f, 0.f), reinterpret_cast<const cc*>(A), reinterpret_cast<const cc*>(B),
                   reinterpret_cast<cc*>(C), base, err, s);
  if (st) return st;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return QTT_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return QTT_ERR_CUDA;
  return h ? QTT_ERR_TIMEOUT : QTT_OK;
}
