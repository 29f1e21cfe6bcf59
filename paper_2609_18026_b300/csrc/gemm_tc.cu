// Dense BF16 GEMM on the 5th-generation tensor cores for the learned surrogate's
// training (no counterpart in the paper):
//   C[m][n] (+)= sum_k A(m, k) B(n, k)       m < M, n < N, k < K
// A: P BF16 parts, K-major, stored [P][Ma][Kp] (row stride Kp elements); with
//    P = 3 they are the split x_hi + x_mid + x_lo of an FP32 operand (FP32-level
//    accuracy on the BF16 pipe), with P = 1 a plain BF16 operand.
// B: one BF16 part, K-major, stored [Nb][Kp].
// C: FP32 row-major [M][N]; with atomic != 0 the tile adds into C (split K over
//    gridDim.z; C zeroed by the caller), else it is stored.
// Tile 128 rows x BN columns; both operands are brought into shared memory by TMA
// (2-D / 3-D tensor maps, 128-byte swizzle, 64-wide K boxes) through an S-stage
// mbarrier ring that one thread keeps full while it issues the
// tcgen05.mma.cta_group::1.kind::f16 instructions (M = 128, N = BN, K = 16) into
// FP32 TMEM accumulators: hi * B in one, the correction parts in a second (P = 3),
// added in the epilogue.  Every wait is bounded; on expiry bit 16 is set in the
// status word, the tile skips its remaining work, waits (bounded) for what it
// issued, frees its TMEM and returns.
#include "mlx_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

namespace {

constexpr int G_BM = 128;
constexpr int G_BK = 64;
constexpr int G_THREADS = 128;
template <int P>
__global__ void __launch_bounds__(G_THREADS, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
          int nchunk_total, int chunks_per_split, int BN, int stages, int tmem_cols, float* __restrict__ C,
          int atomic, const float* __restrict__ bias, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar_tma[8], bar_mma[8];
  __shared__ unsigned tmem_slot;
  __shared__ int bad_flag;
  const unsigned raw = tcx::smem_u32(smem_raw);
  const unsigned pad = (1024u - (raw & 1023u)) & 1023u;
  const unsigned a_bytes = (unsigned)P * G_BM * 128u;
  const unsigned b_bytes = (unsigned)BN * 128u;
  const unsigned stage_bytes = a_bytes + b_bytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * G_BM;
  const int kc0 = blockIdx.z * chunks_per_split;
  const int nk = min(chunks_per_split, nchunk_total - kc0);

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tcx::smem_u32(&bar_tma[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tcx::smem_u32(&bar_mma[s])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bad_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tcx::smem_u32(&tmem_slot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;
  // D f32, A bf16, B bf16, both K-major; N >> 3 and M >> 4
  const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) |
                         ((unsigned)(G_BM >> 4) << 24);

  if (tid == 0 && nk > 0) {
    auto issue = [&](int j) {   // TMA of local chunk j into stage j % stages
      const int s = j % stages;
      const unsigned sA = raw + pad + (unsigned)s * stage_bytes;
      const unsigned sB = sA + a_bytes;
      const unsigned bt = tcx::smem_u32(&bar_tma[s]);
      const int kx = (kc0 + j) * G_BK;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bt), "r"(stage_bytes) : "memory");
      for (int p = 0; p < P; ++p)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(sA + (unsigned)p * G_BM * 128u),
            "l"(&tmA), "r"(kx), "r"(m0), "r"(p), "r"(bt)
            : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
          ::"r"(sB), "l"(&tmB), "r"(kx), "r"(n0), "r"(bt)
          : "memory");
    };
    const int pre = nk < stages ? nk : stages;
    for (int j = 0; j < pre; ++j) issue(j);
    int issued = pre;
    bool ok = true;
    int last_commit = -1;
    for (int j = 0; j < nk && ok; ++j) {
      const int s = j % stages;
      const unsigned sA = raw + pad + (unsigned)s * stage_bytes;
      const unsigned sB = sA + a_bytes;
      if (!tcx::mbar_wait(tcx::smem_u32(&bar_tma[s]), (unsigned)((j / stages) & 1))) { ok = false; atomicOr(err, 16); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < G_BK / 16; ++ks) {
        const uint64_t db = tcx::desc_sw128(sB) + (uint64_t)(2 * ks);
        for (int p = 0; p < P; ++p) {
          const uint64_t da = tcx::desc_sw128(sA + (unsigned)p * G_BM * 128u) + (uint64_t)(2 * ks);
          const unsigned dt = tmem + (p == 0 ? 0u : (unsigned)BN);
          const unsigned acc = (j | ks) ? 1u : (p > 1 ? 1u : 0u);
          tcx::mma_bf16(dt, da, db, idesc, acc);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tcx::smem_u32(&bar_mma[s]))
                   : "memory");
      last_commit = j;
      if (issued < nk) {
        // stage s is refilled once the MMAs that read it have completed
        if (!tcx::mbar_wait(tcx::smem_u32(&bar_mma[s]), (unsigned)((j / stages) & 1))) { ok = false; atomicOr(err, 16); break; }
        issue(issued);
        ++issued;
      }
    }
    // the last commit covers every MMA issued before it; TMA still in flight on
    // failure is waited for (bounded) so that no copy lands after the CTA exits
    if (last_commit >= 0)
      if (!tcx::mbar_wait(tcx::smem_u32(&bar_mma[last_commit % stages]), (unsigned)((last_commit / stages) & 1))) {
        ok = false;
        atomicOr(err, 16);
      }
    if (!ok) {
      for (int j = last_commit + 1; j < issued; ++j)
        tcx::mbar_wait(tcx::smem_u32(&bar_tma[j % stages]), (unsigned)((j / stages) & 1));
      bad_flag = 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (!bad_flag && nk > 0) {
    // Each warp owns TMEM lanes (rows) 32 warp .. 32 warp + 31.  Per 16-column slice
    // the values pass through a per-warp shared tile so that the global stores run
    // along rows (two rows of 16 consecutive columns per instruction).  The stage
    // buffers are free: every MMA that read them has completed.
    float* tile = reinterpret_cast<float*>(smem_raw + pad) + warp * (32 * 17);
    const unsigned tbase = tmem + ((unsigned)(warp * 32) << 16);
    for (int c0 = 0; c0 < BN; c0 += 16) {
      unsigned r[16], q[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tbase + (unsigned)c0));
      if (P > 1) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
              "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
            : "r"(tbase + (unsigned)(BN + c0)));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float v = __uint_as_float(r[j]);
        if (P > 1) v += __uint_as_float(q[j]);
        tile[lane * 17 + j] = v;
      }
      __syncwarp();
      const int col = n0 + c0 + (lane & 15);
      const float bv = (bias && col < N) ? bias[col] : 0.f;
#pragma unroll 4
      for (int rr = 0; rr < 16; ++rr) {
        const int lr = rr * 2 + (lane >> 4);
        const int row = m0 + warp * 32 + lr;
        if (row < M && col < N) {
          float* p = C + (long long)row * N + col;
          const float v = tile[lr * 17 + (lane & 15)];
          if (atomic) atomicAdd(p, v); else *p = v + bv;
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

typedef CUresult (*EncodeTiledFnG)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFnG encoder() {
  static EncodeTiledFnG fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = (EncodeTiledFnG)p;
  }
  return fn;
}

size_t gemm_smem(int P, int BN, int stages) {
  return (size_t)stages * ((size_t)P * G_BM * 128 + (size_t)BN * 128) + 1024;
}

}  // namespace

// C[M][N] (+)= A(M x K, P BF16 parts [P][Ma][Kp]) * B(N x K, [Nb][Kp])^T on the tensor
// cores (contract above).  Kp: row stride of both operands in elements, a multiple
// of 8 (16-byte rows for TMA); K <= Kp and the elements k in [K, Kp) must be zero.
// Ma >= M and Nb >= N are the allocated row counts (reads beyond are zero-filled).
// split > 1 splits K over CTAs and adds into C, which the caller has zeroed.
// bias (device, N floats, or NULL) is added to every row; only without split.
int mlx_gemm_tc(int P, const void* A, long long Ma, const void* B, long long Nb, long long Kp, int M, int N, int K,
                float* C, int split, int* err, cudaStream_t st, const float* bias) {
  if ((P != 1 && P != 3) || M < 1 || N < 1 || K < 1 || K > Kp || (Kp % 8) != 0 || split < 1) return MLX_EINVAL;
  if ((((uintptr_t)A) & 15u) || (((uintptr_t)B) & 15u)) return MLX_EINVAL;
  EncodeTiledFnG fn = encoder();
  if (!fn) return MLX_ECUDA;
  const int BN = N >= 256 ? 256 : (N > 128 ? 256 : (N > 64 ? 128 : 64));
  CUtensorMap ta, tb;
  {
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)Ma, (cuuint64_t)P};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)(Kp * Ma * 2)};
    cuuint32_t box[3] = {G_BK, G_BM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (fn(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(A), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return MLX_ECUDA;
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)Nb};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {G_BK, (cuuint32_t)BN};
    cuuint32_t estr[2] = {1, 1};
    if (fn(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(B), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return MLX_ECUDA;
  }
  const int nchunks = (K + G_BK - 1) / G_BK;
  const int cps = (nchunks + split - 1) / split;
  const int nsplit = (nchunks + cps - 1) / cps;
  // stages: at most 4 and within 200 KB; a tile with fewer chunks keeps 2 (the
  // shared-memory request then also caps co-resident CTAs so that their TMEM
  // accumulators fit the SM's 512 columns)
  int stages = 4;
  while (stages > 2 && gemm_smem(P, BN, stages) > 200 * 1024) --stages;
  if (cps < stages) stages = cps < 2 ? 2 : cps;
  int cols = 32;
  while (cols < (P > 1 ? 2 : 1) * BN) cols <<= 1;
  const size_t smem = gemm_smem(P, BN, stages);
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 201 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(k_gemm_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 201 * 1024) != cudaSuccess)
      return MLX_ECUDA;
    attr_set = true;
  }
  dim3 grid((N + BN - 1) / BN, (M + G_BM - 1) / G_BM, nsplit);
  const int atomic = (nsplit > 1) ? 1 : 0;
  if (atomic && bias) return MLX_EINVAL;   // a bias is added by the single tile that owns an element
  if (P == 1)
    k_gemm_tc<1><<<grid, G_THREADS, smem, st>>>(ta, tb, M, N, nchunks, cps, BN, stages, cols, C, atomic, bias, err);
  else
    k_gemm_tc<3><<<grid, G_THREADS, smem, st>>>(ta, tb, M, N, nchunks, cps, BN, stages, cols, C, atomic, bias, err);
  return cudaGetLastError() == cudaSuccess ? MLX_OK : MLX_ECUDA;
}
