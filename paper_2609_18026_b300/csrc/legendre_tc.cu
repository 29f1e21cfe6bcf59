// K4 (tensor-core form): the ragged per-m Legendre contraction of the transform
// pair (Eq. (2) and its Gauss-quadrature inverse, Sec. 3.1) on the 5th-generation
// tensor cores, split-BF16 with FP32 accumulation.
//
// Every FP32/FP64 operand x is split into three BF16 parts
//   x_hi = bf16(x), x_mid = bf16(x - x_hi), x_lo = bf16(x - x_hi - x_mid)
// and a*b is formed from the products hi*hi, hi*mid, mid*hi, hi*lo, lo*hi, mid*mid
// (six; with eight also mid*lo and lo*mid).  hi*hi accumulates in one FP32 TMEM
// accumulator and the correction products in a second one, so that the small
// terms are not rounded against the large running sum; the epilogue adds the two.
// This reaches FP32-level accuracy (<= 1e-6 relative per transform) on the BF16
// tensor pipe.
//
// Per output tile (m, 128 rows, BN <= 256 columns):
//   A (basis, static): BF16 split tables in global memory, staged into shared
//     memory by TMA (3-D tensor map [split][row][k], 128-byte swizzle, box
//     64 k x 128 rows), one 64-wide K chunk at a time;
//   B (data): converted in the kernel from FP32 (mixed layout, forward) or FP64
//     (spectral state, backward) into the three BF16 parts and written into the
//     same 128-byte-swizzled K-major layout by all threads;
//   D: 128 lanes x BN columns of TMEM (FP32) per accumulator, issued by one
//     thread as tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = BN, K = 16),
//     4 K-steps x 6 products per chunk, completion tracked by tcgen05.commit ->
//     mbarrier; two shared-memory stages so the B conversion of chunk k+1 runs
//     while the tensor core works on chunk k;
//   epilogue: each of the 4 warps reads its 32 TMEM lanes with tcgen05.ld and
//     writes its rows (FP64 spectral coefficients, or FP32 mixed values).
// Forward  D[n - m][c] = sum_i W_m[n][i] X_c[i]     (W = w_i Pbar_n^m(x_i))
// Backward D[i][c]     = sum_n P_m[n][i] S_c[n]     (A = P_m^T, stored [m][i][n])
// Column c < K is the real part of wavenumber slot c, c >= K the imaginary part.
// Every wait on an mbarrier is bounded; on expiry the kernel records an error
// code in a device word, still waits (bounded) for its issued work, frees its
// TMEM and returns.
#include "mlx_internal.cuh"

#include <cuda_bf16.h>

namespace {

constexpr int TC_BM = 128;     // tile rows = TMEM lanes
constexpr int TC_BK = 64;      // K chunk: one 128-byte swizzle atom of BF16
constexpr int TC_THREADS = 128;
constexpr long long kSpinLimit = 1LL << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned phase) {
  for (long long it = 0; it < kSpinLimit; ++it)
    if (mbar_try(bar, phase)) return true;
  return false;
}

// K-major operand in 128-byte-swizzled layout: rows of 128 bytes (64 BF16),
// 8-row groups 1024 bytes apart, 16-byte chunk index XOR (row mod 8).
__device__ __forceinline__ uint64_t sw128_desc(unsigned saddr) {
  return ((uint64_t)((saddr >> 4) & 0x3FFF)) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ unsigned sw128_offset(int row, int k) {
  return (unsigned)(row * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) + ((k & 7) << 1));
}

template <typename T>
__device__ __forceinline__ void split3(T x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn((float)x);
  const T r1 = x - (T)__bfloat162float(h);
  m = __float2bfloat16_rn((float)r1);
  const T r2 = r1 - (T)__bfloat162float(m);
  l = __float2bfloat16_rn((float)r2);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem, uint64_t da, uint64_t db, unsigned idesc,
                                         unsigned acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
      ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void store_split4(unsigned char* pB, int BN, int col, int k, const float* v) {
  // four consecutive k (same 16-byte chunk, k % 4 == 0) of one column, three parts
  __nv_bfloat16 h[4], md[4], lo[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) split3<float>(v[j], h[j], md[j], lo[j]);
  const unsigned off = sw128_offset(col, k);
  uint2 a, b, c;
  a.x = (unsigned)__bfloat16_as_ushort(h[0]) | ((unsigned)__bfloat16_as_ushort(h[1]) << 16);
  a.y = (unsigned)__bfloat16_as_ushort(h[2]) | ((unsigned)__bfloat16_as_ushort(h[3]) << 16);
  b.x = (unsigned)__bfloat16_as_ushort(md[0]) | ((unsigned)__bfloat16_as_ushort(md[1]) << 16);
  b.y = (unsigned)__bfloat16_as_ushort(md[2]) | ((unsigned)__bfloat16_as_ushort(md[3]) << 16);
  c.x = (unsigned)__bfloat16_as_ushort(lo[0]) | ((unsigned)__bfloat16_as_ushort(lo[1]) << 16);
  c.y = (unsigned)__bfloat16_as_ushort(lo[2]) | ((unsigned)__bfloat16_as_ushort(lo[3]) << 16);
  *reinterpret_cast<uint2*>(pB + off) = a;
  *reinterpret_cast<uint2*>(pB + (size_t)BN * 128 + off) = b;
  *reinterpret_cast<uint2*>(pB + (size_t)2 * BN * 128 + off) = c;
}

// Columns of a tile are interleaved: column c is (slot c / 2, Re if c even, Im if
// odd), so one 16-byte complex load feeds two columns and the epilogue writes
// whole complex values.
template <bool FWD>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_leg_tc(const __grid_constant__ CUtensorMap tmapA, const LegTile* __restrict__ tiles, int nc, int nr,
         int M, int K, int BN, int tmem_cols, int nprod, int stages, const long long* __restrict__ soff,
         const long long* __restrict__ arow_base, const float* __restrict__ mixed_in,
         const double2* __restrict__ spec_in, double2* __restrict__ spec_out,
         float* __restrict__ mixed_out, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar_tma[2], bar_mma[2];
  __shared__ unsigned tmem_slot;
  const unsigned raw = smem_u32(smem_raw);
  const unsigned pad = (1024u - (raw & 1023u)) & 1023u;
  const unsigned stage_bytes = 3u * TC_BM * 128u + 3u * (unsigned)BN * 128u;

  const LegTile tile = tiles[blockIdx.x];
  const int m = tile.m;
  const int Nm = nc - m;
  const int rows = FWD ? Nm : nr;
  const int kdim = FWD ? nr : Nm;
  const int ncol = 2 * K;
  const long long plane = (long long)K * M * nr;
  const long long so = soff[m];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_tma[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma[s])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;

  const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) |
                         ((unsigned)(TC_BM >> 4) << 24);
  const int nchunks = (kdim + TC_BK - 1) / TC_BK;
  const int arow = (int)arow_base[m] + tile.row0;
  const int kslot0 = tile.col0 >> 1;            // first wavenumber slot of this tile
  const int nslot = BN >> 1;
  bool bad = false;

  for (int kc = 0; kc < nchunks; ++kc) {
    const int s = kc % stages;
    const unsigned sA = raw + pad + (unsigned)s * stage_bytes;
    const unsigned sB = sA + 3u * TC_BM * 128u;
    unsigned char* pB = smem_raw + pad + (size_t)s * stage_bytes + 3 * TC_BM * 128;
    // stage reuse: the MMAs of chunk kc - stages must have finished reading it
    if (kc >= stages) {
      const bool ok = mbar_wait_bounded(smem_u32(&bar_mma[s]), (unsigned)(((kc / stages) - 1) & 1));
      if (__syncthreads_or(!ok)) { bad = true; if (tid == 0) atomicOr(err, 2); break; }
    }
    if (tid == 0) {
      const unsigned bt = smem_u32(&bar_tma[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bt), "r"(3 * TC_BM * 128)
                   : "memory");
      for (int sp = 0; sp < 3; ++sp)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
            ::"r"(sA + (unsigned)sp * TC_BM * 128u), "l"(&tmapA), "r"(kc * TC_BK), "r"(arow), "r"(sp), "r"(bt)
            : "memory");
    }
    // B chunk: (slot, 4 consecutive k) per thread step
    const int k0 = kc * TC_BK;
    for (int e = tid; e < nslot * (TC_BK / 4); e += TC_THREADS) {
      const int sl = e / (TC_BK / 4), kq = (e - sl * (TC_BK / 4)) * 4;
      const int kidx = kslot0 + sl;
      float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
      if (kidx < K) {
        if (FWD) {
          const float* pr = mixed_in + ((long long)kidx * M + m) * nr + k0 + kq;
          const float* pi = pr + plane;
          if (((nr & 3) == 0) && k0 + kq + 3 < kdim) {
            const float4 a = *reinterpret_cast<const float4*>(pr);
            const float4 b = *reinterpret_cast<const float4*>(pi);
            re[0] = a.x; re[1] = a.y; re[2] = a.z; re[3] = a.w;
            im[0] = b.x; im[1] = b.y; im[2] = b.z; im[3] = b.w;
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (k0 + kq + j < kdim) { re[j] = pr[j]; im[j] = pi[j]; }
          }
        } else {
          const double2* ps = spec_in + so + (long long)kidx * Nm + k0 + kq;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (k0 + kq + j < kdim) { const double2 v = ps[j]; re[j] = (float)v.x; im[j] = (float)v.y; }
        }
      }
      store_split4(pB, BN, 2 * sl, kq, re);
      store_split4(pB, BN, 2 * sl + 1, kq, im);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      if (!mbar_wait_bounded(smem_u32(&bar_tma[s]), (unsigned)((kc / stages) & 1))) {
        atomicOr(err, 1);
        bad = true;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int pa[8] = {0, 0, 1, 0, 2, 1, 1, 2};
        const int pb[8] = {0, 1, 0, 2, 0, 1, 2, 1};
#pragma unroll
        for (int ks = 0; ks < TC_BK / 16; ++ks) {
          for (int q = 0; q < nprod; ++q) {
            const uint64_t da = sw128_desc(sA + (unsigned)pa[q] * TC_BM * 128u) + (uint64_t)(2 * ks);
            const uint64_t db = sw128_desc(sB + (unsigned)pb[q] * BN * 128u) + (uint64_t)(2 * ks);
            const unsigned dt = tmem + (q == 0 ? 0u : (unsigned)BN);
            const unsigned acc = (kc | ks) ? 1u : (q > 1 ? 1u : 0u);
            mma_bf16(dt, da, db, idesc, acc);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar_mma[s]))
                     : "memory");
      }
    }
    if (__syncthreads_or(bad)) { bad = true; break; }
  }
  // the last commit covers every MMA issued before it
  if (!bad && nchunks > 0) {
    const int kl = nchunks - 1;
    const bool ok = mbar_wait_bounded(smem_u32(&bar_mma[kl % stages]), (unsigned)((kl / stages) & 1));
    if (__syncthreads_or(!ok)) { bad = true; if (tid == 0) atomicOr(err, 4); }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (!bad) {
    const int row = tile.row0 + warp * 32 + lane;
    const unsigned tbase = tmem + ((unsigned)(warp * 32) << 16);
    for (int c0 = 0; c0 < BN; c0 += 16) {
      unsigned r[16], q[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tbase + (unsigned)c0));
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
            "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
          : "r"(tbase + (unsigned)(BN + c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < rows) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int kidx = kslot0 + ((c0 + j) >> 1);
          if (kidx >= K) break;
          const float vr = __uint_as_float(r[j]) + __uint_as_float(q[j]);
          const float vi = __uint_as_float(r[j + 1]) + __uint_as_float(q[j + 1]);
          if (FWD) {
            spec_out[so + (long long)kidx * Nm + row] = make_double2((double)vr, (double)vi);
          } else {
            const long long o = ((long long)kidx * M + m) * nr + row;
            mixed_out[o] = vr;
            mixed_out[plane + o] = vi;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// BF16 split tables from the FP64 basis.
//  Wb[sp][t][k]  t = row (m, n - m) of W, k = i < Nr (zero up to Kp)
//  Pb[sp][m * Nr + i][k]  k = n - m < Nc - m (zero up to Kq)
__global__ void k_split_tables(int M, int nc, int nr, int Kp, int Kq, long long trows,
                               const long long* __restrict__ boff, const double* __restrict__ W64,
                               const double* __restrict__ P64, __nv_bfloat16* __restrict__ Wb,
                               __nv_bfloat16* __restrict__ Pb) {
  const long long nW = trows * Kp;
  const long long nP = (long long)M * nr * Kq;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nW) {
    const long long t = idx / Kp;
    const int k = (int)(idx - t * Kp);
    double v = 0.0;
    if (k < nr) v = W64[t * nr + k];   // W rows are contiguous across m
    __nv_bfloat16 h, md, lo;
    split3<double>(v, h, md, lo);
    Wb[idx] = h;
    Wb[nW + idx] = md;
    Wb[2 * nW + idx] = lo;
  } else if (idx < nW + nP) {
    const long long j = idx - nW;
    const long long r = j / Kq;
    const int k = (int)(j - r * Kq);
    const int m = (int)(r / nr), i = (int)(r - (long long)m * nr);
    double v = 0.0;
    if (k < nc - m) v = P64[boff[m] + (long long)k * nr + i];
    __nv_bfloat16 h, md, lo;
    split3<double>(v, h, md, lo);
    Pb[j] = h;
    Pb[nP + j] = md;
    Pb[2 * nP + j] = lo;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_map(mlx_ctx* c, CUtensorMap* map, void* base, long long kpad, long long rows) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    MLX_CUDA_TRY(c, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) { c->last_err = "cuTensorMapEncodeTiled unavailable"; return MLX_ECUDA; }
    fn = (EncodeTiledFn)p;
  }
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, 3};
  cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)(kpad * rows * 2)};
  cuuint32_t box[3] = {TC_BK, TC_BM, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { c->last_err = "cuTensorMapEncodeTiled failed"; return MLX_ECUDA; }
  return MLX_OK;
}

size_t tc_smem(int BN, int stages) {
  return (size_t)stages * (3 * TC_BM * 128 + (size_t)3 * BN * 128) + 1024;
}

}  // namespace

// Build the split tables, tensor maps and tile lists for the tensor-core form.
int mlx_tc_prepare(mlx_ctx* c, cudaStream_t st) {
  const long long Kp = (c->nr + TC_BK - 1) / TC_BK * TC_BK;
  const long long Kq = (c->nc + TC_BK - 1) / TC_BK * TC_BK;
  const long long nW = c->tri * Kp, nP = (long long)c->M * c->nr * Kq;
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_Wb, sizeof(__nv_bfloat16) * 3 * nW));
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_Pb, sizeof(__nv_bfloat16) * 3 * nP));
  const long long tot = nW + nP;
  k_split_tables<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(c->M, c->nc, c->nr, (int)Kp, (int)Kq, c->tri,
                                                                c->d_boff, c->d_W64, c->d_P64,
                                                                (__nv_bfloat16*)c->d_Wb, (__nv_bfloat16*)c->d_Pb);
  MLX_LAUNCH_CHECK(c);
  int rc = encode_map(c, &c->tmapW, c->d_Wb, Kp, c->tri);
  if (rc) return rc;
  rc = encode_map(c, &c->tmapP, c->d_Pb, Kq, (long long)c->M * c->nr);
  if (rc) return rc;
  // A-row bases: W rows of m start at sum_{m'<m}(Nc - m'); P^T rows at m * Nr
  std::vector<long long> aw(c->M), ap(c->M);
  long long t = 0;
  for (int m = 0; m < c->M; ++m) { aw[m] = t; ap[m] = (long long)m * c->nr; t += c->nc - m; }
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_arowW, sizeof(long long) * c->M));
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_arowP, sizeof(long long) * c->M));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(c->d_arowW, aw.data(), sizeof(long long) * c->M, cudaMemcpyHostToDevice, st));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(c->d_arowP, ap.data(), sizeof(long long) * c->M, cudaMemcpyHostToDevice, st));
  // columns per tile (interleaved Re/Im pairs, multiple of 16): narrow tiles when
  // the grid would otherwise leave SMs idle
  const int ncol = 2 * c->K;
  int bn = 256;
  {
    int rt = 0;
    for (int m = 0; m < c->M; ++m) rt += (c->nc - m + TC_BM - 1) / TC_BM;
    while (bn > 32 && (long long)rt * ((ncol + bn - 1) / bn) < 148) bn -= 16;
  }
  return mlx_tc_retile(c, bn, st);
}

// Tile lists for a requested column-tile width (the autotuner's knob).
int mlx_tc_retile(mlx_ctx* c, int bn_req, cudaStream_t st) {
  const int ncol = 2 * c->K;
  if (bn_req < 16 || bn_req > 256) return MLX_EINVAL;
  const int nct = (ncol + bn_req - 1) / bn_req;
  c->tc_bn = ((ncol + nct - 1) / nct + 15) / 16 * 16;
  if (c->tc_bn > 256) c->tc_bn = 256;
  cudaFree(c->d_tc_fwd);
  cudaFree(c->d_tc_bwd);
  c->d_tc_fwd = c->d_tc_bwd = nullptr;
  std::vector<LegTile> tf, tb;
  for (int m = 0; m < c->M; ++m) {
    for (int r0 = 0; r0 < c->nc - m; r0 += TC_BM)
      for (int c0 = 0; c0 < ncol; c0 += c->tc_bn) tf.push_back(LegTile{m, r0, c0, 0});
    for (int r0 = 0; r0 < c->nr; r0 += TC_BM)
      for (int c0 = 0; c0 < ncol; c0 += c->tc_bn) tb.push_back(LegTile{m, r0, c0, 0});
  }
  c->ntc_fwd = (int)tf.size();
  c->ntc_bwd = (int)tb.size();
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_tc_fwd, sizeof(LegTile) * tf.size()));
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_tc_bwd, sizeof(LegTile) * tb.size()));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(c->d_tc_fwd, tf.data(), sizeof(LegTile) * tf.size(), cudaMemcpyHostToDevice, st));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(c->d_tc_bwd, tb.data(), sizeof(LegTile) * tb.size(), cudaMemcpyHostToDevice, st));
  int cols = 32;
  while (cols < 2 * c->tc_bn) cols <<= 1;   // two accumulators of BN columns
  c->tc_tmem_cols = cols;
  c->tc_stages = tc_smem(c->tc_bn, 2) <= 220 * 1024 ? 2 : 1;
  // the attribute is a per-function ceiling shared by every context: set it to
  // the largest size any tile width uses
  const int smem = 220 * 1024 + 1024;
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_leg_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_leg_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return MLX_OK;
}

int mlx_legendre_tc_forward(mlx_ctx* c, double2* spec, cudaStream_t st) {
  TimedLaunch tl(c, KID_LEG_FWD, st);
  k_leg_tc<true><<<c->ntc_fwd, TC_THREADS, tc_smem(c->tc_bn, c->tc_stages), st>>>(
      c->tmapW, c->d_tc_fwd, c->nc, c->nr, c->M, c->K, c->tc_bn, c->tc_tmem_cols, c->tc_products, c->tc_stages,
      c->d_soff, c->d_arowW,
      (const float*)c->d_mixed, nullptr, spec, nullptr, c->d_err);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

int mlx_legendre_tc_backward(mlx_ctx* c, const double2* spec, cudaStream_t st) {
  TimedLaunch tl(c, KID_LEG_BWD, st);
  k_leg_tc<false><<<c->ntc_bwd, TC_THREADS, tc_smem(c->tc_bn, c->tc_stages), st>>>(
      c->tmapP, c->d_tc_bwd, c->nc, c->nr, c->M, c->K, c->tc_bn, c->tc_tmem_cols, c->tc_products, c->tc_stages,
      c->d_soff, c->d_arowP,
      nullptr, spec, nullptr, (float*)c->d_mixed, c->d_err);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}
