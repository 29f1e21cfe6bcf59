// K4 (tensor-core form): the ragged per-m Legendre contraction of the transform
// pair (Eq. (2) and its Gauss-quadrature inverse, Sec. 3.1) on the 5th-generation
// tensor cores, split-BF16 with FP32 accumulation.
//
// Every operand value x is split into three BF16 parts
//   x_hi = bf16(x), x_mid = bf16(x - x_hi), x_lo = bf16(x - x_hi - x_mid)
// and a*b is formed from the products hi*hi, hi*mid, mid*hi, hi*lo, lo*hi, mid*mid
// (six; with eight also mid*lo and lo*mid).  hi*hi accumulates in one FP32 TMEM
// accumulator and the correction products in a second one, so that the small
// terms are not rounded against the large running sum; the epilogue adds the two.
// This reaches FP32-level accuracy (<= 1e-6 relative per transform) on the BF16
// tensor pipe.
//
// Forward  D[n - m][c] = sum_i W_m[n][i] X_c[i]     (W = w_i Pbar_n^m(x_i))
// Backward D[i][c]     = sum_n P_m[n][i] S_c[n]     (A = P_m^T, stored [m][i][n])
// Column c of a tile is (wavenumber slot c / 2, Re if c even, Im if odd).
//
// The data operand arrives as three BF16 planes in global memory, K-major:
// Bs[part][m * 2K + c][k] (forward: written by the FFT kernel that produces the
// mixed values; backward: by k_split_spec from the FP64 spectral field).  One
// persistent CTA per SM walks its share of the work items (m, 128-row tile,
// BN-column tile) with warp-specialised roles:
//   warps 0-3  epilogue: TMEM -> registers -> global (each warp owns its 32 TMEM
//              lanes), on two TMEM accumulator pairs so that the epilogue of one
//              tile runs while the tensor core works on the next;
//   warp 4     TMA producer: three BF16 parts of the basis chunk (128 x 32) and of
//              the data chunk (BN x 32), 64-byte swizzle, into a four-stage ring;
//   warp 5     one thread issues tcgen05.mma (M = 128, N = BN, K = 16) and commits
//              each stage back to the ring.
// Every wait on an mbarrier is bounded.  A role that gives up records an error
// bit in the device word and raises a CTA-wide abort flag; every role then
// leaves its loop, the producer waits (bounded) for the tensor copies it issued
// and the MMA thread for the MMAs it issued, and the TMEM is freed only after
// that.  `expire` (a test hook) makes the producer's first stage-reuse wait
// report expiry at once.
#include "mlx_internal.cuh"
#include "bf16_split.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>
#include <string.h>
#include <algorithm>

namespace {

constexpr int TC_BM = 128;                 // tile rows = TMEM lanes
constexpr int TC_BK = 32;                  // K chunk: one 64-byte swizzled row of BF16
constexpr int TC_STAGES = 4;
constexpr int TC_PROD_WARP = 4;
constexpr int TC_MMA_WARP = 5;
constexpr int TC_THREADS = 32 * 6;
constexpr int TC_MAX_BN = 128;
constexpr unsigned TC_A_PART = TC_BM * 64;                         // one BF16 part of a 128 x 32 chunk
constexpr unsigned TC_A_BYTES = 3 * TC_A_PART;

__host__ __device__ constexpr unsigned tc_stage_bytes(int bn) { return TC_A_BYTES + 3u * (unsigned)bn * 64u; }

// split3 and f64w_to_f32: bf16_split.cuh

// FP32 -> FP64 (exact) by integer operations; FP32 subnormals (< 1.2e-38) flush to zero
__device__ __forceinline__ double f32_to_f64(float v) {
  const unsigned b = __float_as_uint(v);
  const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xffu, mant = b & 0x7fffffu;
  const unsigned eh = (e == 255u) ? 2047u : e + 896u;
  const unsigned hi = (e == 0u) ? sign : (sign | (eh << 20) | (mant >> 3));
  const unsigned lo = (e == 0u) ? 0u : (mant << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// Sizes and outputs of one member of a launch (one context, or one member of a
// batched launch).
struct TcArgs {
  int nc, nr, M, K, bn, pad_;
  const long long* soff;
  const long long* arow;      // first A row of each m
  double2* spec_out;          // forward output
  float* mixed_out;           // backward output (planar [2][K][M][Nr])
  long long pad2_;
};
// Launch parameters: NB members' operand maps and sizes (NB = 1 for one context;
// a batched launch indexes them by the item's member).
template <int NB>
struct TcParams {
  CUtensorMap a[NB];
  CUtensorMap b[NB];
  TcArgs g[NB];
};

// Walk of one CTA's work: items blockIdx.x, blockIdx.x + gridDim.x, ...; chunks of
// 32 along the contraction within each item.  Every role walks the same sequence.
// An item's member is its pad field (0 for a single context).
struct Walk {
  int t, kc, nch, tl;
  __device__ __forceinline__ bool valid(int nitems) const { return t < nitems; }
};
template <int NB>
__device__ __forceinline__ int item_member(const LegTile& tile) { return NB == 1 ? 0 : tile.pad; }
template <bool FWD, int NB>
__device__ __forceinline__ int item_chunks(const TcParams<NB>& P, const LegTile* items, int t) {
  const LegTile tile = items[t];
  const TcArgs& g = P.g[item_member<NB>(tile)];
  const int kdim = FWD ? g.nr : g.nc - tile.m;
  return (kdim + TC_BK - 1) / TC_BK;
}
template <bool FWD, int NB>
__device__ __forceinline__ Walk walk_begin(const TcParams<NB>& P, const LegTile* items, int nitems) {
  Walk w{(int)blockIdx.x, 0, 0, 0};
  if (w.t < nitems) w.nch = item_chunks<FWD, NB>(P, items, w.t);
  return w;
}
template <bool FWD, int NB>
__device__ __forceinline__ void walk_next(Walk& w, const TcParams<NB>& P, const LegTile* items, int nitems) {
  if (++w.kc < w.nch) return;
  w.kc = 0;
  w.t += gridDim.x;
  ++w.tl;
  if (w.t < nitems) w.nch = item_chunks<FWD, NB>(P, items, w.t);
}

// 1 = completed, 0 = left because another role raised the abort flag, -1 = expired
__device__ __forceinline__ int wait3(unsigned bar, unsigned parity, volatile int* abort) {
  for (long long it = 0; it < tcx::kSpinLimit; ++it) {
    if (tcx::mbar_try(bar, parity)) return 1;
    if ((it & 63) == 63 && *abort) return 0;
  }
  return -1;
}

// bnmax: the widest column tile of the launch's members (the ring's stage size and
// the TMEM accumulator stride follow it; each item uses its member's width).
template <bool FWD, int NPROD, int NB>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_leg_tc(const __grid_constant__ TcParams<NB> P, const LegTile* __restrict__ items, int nitems, int bnmax,
         int tmem_cols, int expire, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full_a[TC_STAGES], empty[TC_STAGES], tfull[2], tempty[2], drain;
  __shared__ unsigned tmem_slot;
  __shared__ int abort_flag;
  volatile int* abortp = &abort_flag;
  const unsigned raw = tcx::smem_u32(smem_raw);
  const unsigned pad = (1024u - (raw & 1023u)) & 1023u;
  const unsigned sbytes = tc_stage_bytes(bnmax);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pdl_wait();      // (a no-op unless launched with programmatic serialisation)
  pdl_trigger();

  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      tcx::mbar_init(tcx::smem_u32(&full_a[s]), 1);
      tcx::mbar_init(tcx::smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tcx::mbar_init(tcx::smem_u32(&tfull[b]), 1);
      tcx::mbar_init(tcx::smem_u32(&tempty[b]), 4);
    }
    tcx::mbar_init(tcx::smem_u32(&drain), 1);
    abort_flag = 0;
    tcx::fence_mbar_init();
  }
  if (warp == 0) tcx::tmem_alloc(tcx::smem_u32(&tmem_slot), (unsigned)tmem_cols);
  tcx::tc_fence_before();
  __syncthreads();
  tcx::tc_fence_after();
  const unsigned tmem = tmem_slot;

  if (warp == TC_PROD_WARP) {
    // ---- basis operand A by TMA
    if (lane == 0) {
      unsigned fills[TC_STAGES] = {0u, 0u, 0u, 0u};
      int g = 0;
      for (Walk w = walk_begin<FWD, NB>(P, items, nitems); w.valid(nitems); walk_next<FWD, NB>(w, P, items, nitems), ++g) {
        const int s = g % TC_STAGES, u = g / TC_STAGES;
        if (u > 0) {
          if (expire && g == TC_STAGES) { atomicOr(err, 2); *abortp = 1; break; }
          const int r = wait3(tcx::smem_u32(&empty[s]), (unsigned)((u - 1) & 1), abortp);
          if (r < 0) { atomicOr(err, 2); *abortp = 1; }
          if (r <= 0) break;
        }
        const LegTile tile = items[w.t];
        const int mem = item_member<NB>(tile);
        const TcArgs& ga = P.g[mem];
        const int bn = ga.bn;
        const unsigned sA = raw + pad + (unsigned)s * sbytes;
        const unsigned sB = sA + TC_A_BYTES;
        if (w.kc == 0 && w.t + (int)gridDim.x < nitems) {
          // warm the next item's tile record and basis-row base into L1
          asm volatile("prefetch.global.L1 [%0];" ::"l"(items + w.t + gridDim.x));
        }
        const unsigned bar = tcx::smem_u32(&full_a[s]);
        tcx::mbar_expect_tx(bar, TC_A_BYTES + 3u * (unsigned)bn * 64u);
        const int arow = (int)ga.arow[tile.m] + tile.row0;
        const int brow = tile.m * 2 * ga.K + tile.col0;
        for (int p = 0; p < 3; ++p) {
          tcx::tma_load_3d(sA + (unsigned)p * TC_A_PART, &P.a[mem], w.kc * TC_BK, arow, p, bar);
          tcx::tma_load_3d(sB + (unsigned)p * (unsigned)bn * 64u, &P.b[mem], w.kc * TC_BK, brow, p, bar);
        }
        ++fills[s];
      }
      // drain: every tensor copy issued must land before the CTA leaves
      for (int s = 0; s < TC_STAGES; ++s)
        if (fills[s] && !tcx::mbar_wait(tcx::smem_u32(&full_a[s]), (fills[s] - 1u) & 1u)) atomicOr(err, 1);
    }
  } else if (warp == TC_MMA_WARP) {
    // ---- tensor-core issue
    if (lane == 0) {
      bool issued = false, ok = true;
      int g = 0, tl_cur = -1, bn = 0;
      unsigned idesc = 0u;
      for (Walk w = walk_begin<FWD, NB>(P, items, nitems); w.valid(nitems) && ok;) {
        const int buf = w.tl & 1;
        if (w.tl != tl_cur) {
          tl_cur = w.tl;
          bn = P.g[item_member<NB>(items[w.t])].bn;
          idesc = tcx::idesc_bf16(TC_BM, bn);
          if (w.tl >= 2) {
            const int r = wait3(tcx::smem_u32(&tempty[buf]), (unsigned)(((w.tl >> 1) - 1) & 1), abortp);
            if (r < 0) { atomicOr(err, 4); *abortp = 1; }
            if (r <= 0) { ok = false; break; }
            tcx::tc_fence_after();
          }
        }
        const int s = g % TC_STAGES, u = g / TC_STAGES;
        const int r = wait3(tcx::smem_u32(&full_a[s]), (unsigned)(u & 1), abortp);
        if (r < 0) { atomicOr(err, 1); *abortp = 1; }
        if (r <= 0) { ok = false; break; }
        tcx::tc_fence_after();
        const unsigned sA = raw + pad + (unsigned)s * sbytes;
        const unsigned sB = sA + TC_A_BYTES;
        const unsigned dhi = tmem + (unsigned)(buf * 2 * bnmax), dco = dhi + (unsigned)bnmax;
        // descriptors of the three parts of each operand, once per chunk
        const uint64_t a0 = tcx::desc_sw64(sA), a1 = tcx::desc_sw64(sA + TC_A_PART),
                       a2 = tcx::desc_sw64(sA + 2 * TC_A_PART);
        const uint64_t b0 = tcx::desc_sw64(sB), b1 = tcx::desc_sw64(sB + (unsigned)bn * 64u),
                       b2 = tcx::desc_sw64(sB + 2u * (unsigned)bn * 64u);
#pragma unroll
        for (int ks = 0; ks < TC_BK / 16; ++ks) {
          const uint64_t o = (uint64_t)(2 * ks);           // 32 bytes per 16-wide K step
          const unsigned first = (w.kc | ks) ? 1u : 0u;    // 0: the tile's first step overwrites
          tcx::mma_bf16(dhi, a0 + o, b0 + o, idesc, first);   // hi * hi
          tcx::mma_bf16(dco, a0 + o, b1 + o, idesc, first);   // hi * mid
          tcx::mma_bf16(dco, a1 + o, b0 + o, idesc, 1u);      // mid * hi
          tcx::mma_bf16(dco, a0 + o, b2 + o, idesc, 1u);      // hi * lo
          tcx::mma_bf16(dco, a2 + o, b0 + o, idesc, 1u);      // lo * hi
          tcx::mma_bf16(dco, a1 + o, b1 + o, idesc, 1u);      // mid * mid
          if (NPROD == 8) {
            tcx::mma_bf16(dco, a1 + o, b2 + o, idesc, 1u);    // mid * lo
            tcx::mma_bf16(dco, a2 + o, b1 + o, idesc, 1u);    // lo * mid
          }
        }
        tcx::mma_commit(tcx::smem_u32(&empty[s]));
        issued = true;
        const bool last = w.kc + 1 == w.nch;
        if (last) tcx::mma_commit(tcx::smem_u32(&tfull[buf]));
        walk_next<FWD, NB>(w, P, items, nitems);
        ++g;
      }
      // drain: every MMA issued must complete before the TMEM is freed
      if (issued) {
        tcx::mma_commit(tcx::smem_u32(&drain));
        if (!tcx::mbar_wait(tcx::smem_u32(&drain), 0u)) atomicOr(err, 4);
      }
    }
  } else if (warp < 4) {
    // ---- epilogue (warps 0-3): TMEM lanes 32 warp .. 32 warp + 31
    for (Walk w = walk_begin<FWD, NB>(P, items, nitems); w.valid(nitems);) {
      const int buf = w.tl & 1;
      int r = 0;
      if (lane == 0) {
        r = wait3(tcx::smem_u32(&tfull[buf]), (unsigned)((w.tl >> 1) & 1), abortp);
        if (r < 0) { atomicOr(err, 4); *abortp = 1; }
      }
      r = __shfl_sync(0xffffffffu, r, 0);
      if (r <= 0) break;
      tcx::tc_fence_after();
      const LegTile tile = items[w.t];
      const TcArgs& ga = P.g[item_member<NB>(tile)];
      const int nc = ga.nc, nr = ga.nr, M = ga.M, K = ga.K, bn = ga.bn;
      const long long plane = (long long)K * M * nr;
      double2* __restrict__ spec_out = ga.spec_out;
      float* __restrict__ mixed_out = ga.mixed_out;
      const int m = tile.m, Nm = nc - m;
      const int rows = FWD ? Nm : nr;
      const int row = tile.row0 + warp * 32 + lane;
      const int kslot0 = tile.col0 >> 1;
      const long long so = ga.soff[m];
      const unsigned tb = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(buf * 2 * bnmax);
      for (int c0 = 0; c0 < bn; c0 += 16) {
        unsigned hi[16], co[16];
        tcx::tmem_ld16(tb + (unsigned)c0, hi);
        tcx::tmem_ld16(tb + (unsigned)(bnmax + c0), co);
        tcx::tmem_wait_ld();
        if (row < rows) {
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int kidx = kslot0 + ((c0 + j) >> 1);
            if (kidx >= K) break;
            const float vr = __uint_as_float(hi[j]) + __uint_as_float(co[j]);
            const float vi = __uint_as_float(hi[j + 1]) + __uint_as_float(co[j + 1]);
            if (FWD) {
              spec_out[so + (long long)kidx * Nm + row] = make_double2(f32_to_f64(vr), f32_to_f64(vi));
            } else {
              const long long o = ((long long)kidx * M + m) * nr + row;
              mixed_out[o] = vr;
              mixed_out[plane + o] = vi;
            }
          }
        }
      }
      tcx::tc_fence_before();
      __syncwarp();
      if (lane == 0) tcx::mbar_arrive(tcx::smem_u32(&tempty[buf]));
      // next tile of this CTA
      do { walk_next<FWD, NB>(w, P, items, nitems); } while (w.valid(nitems) && w.kc != 0);
    }
  }
  tcx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tcx::tc_fence_after();
    tcx::tmem_dealloc(tmem, (unsigned)tmem_cols);
  }
}

// Backward data operand: the FP64 spectral field split into three BF16 parts,
// Bs[part][m * 2K + 2 k + (0 Re, 1 Im)][n - m] (row length Kq; the rows' tails
// n - m >= Nc - m stay zero from allocation).  FP64 -> FP32 by integer rounding,
// then FP32 residuals.  One thread per complex coefficient.
__global__ void k_split_spec(int nc, int K, int Kq, long long part, const long long* __restrict__ soff,
                             const double2* __restrict__ spec, unsigned short* __restrict__ bs) {
  const int m = blockIdx.z, kidx = blockIdx.y;
  const int Nm = nc - m;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Nm) return;
  const long long idx = soff[m] + (long long)kidx * Nm + a;
  const uint4 wv = __ldg(reinterpret_cast<const uint4*>(spec) + idx);
  const float v[2] = {f64w_to_f32(wv.y, wv.x), f64w_to_f32(wv.w, wv.z)};
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    __nv_bfloat16 h, md, l;
    split3<float>(v[p], h, md, l);
    const long long o = ((long long)m * 2 * K + 2 * kidx + p) * Kq + a;
    bs[o] = __bfloat16_as_ushort(h);
    bs[part + o] = __bfloat16_as_ushort(md);
    bs[2 * part + o] = __bfloat16_as_ushort(l);
  }
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

// 3-D map [part][row][k] of BF16 values: kdim valid elements per row (TMA fills
// zeros beyond), row length kpad elements, `rows` rows, box 32 x box_rows x 1.
int encode_map(mlx_ctx* c, CUtensorMap* map, void* base, long long kdim, long long kpad, long long rows,
               int box_rows) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    MLX_CUDA_TRY(c, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) { c->last_err = "cuTensorMapEncodeTiled unavailable"; return MLX_ECUDA; }
    fn = (EncodeTiledFn)p;
  }
  cuuint64_t dims[3] = {(cuuint64_t)kdim, (cuuint64_t)rows, 3};
  cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)(kpad * rows * 2)};
  cuuint32_t box[3] = {TC_BK, (cuuint32_t)box_rows, 1};   // 32 BF16 = one 64-byte swizzled row
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { c->last_err = "cuTensorMapEncodeTiled failed"; return MLX_ECUDA; }
  return MLX_OK;
}

size_t tc_smem(int bn) { return (size_t)TC_STAGES * tc_stage_bytes(bn) + 1024; }

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
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
  int rc = encode_map(c, &c->tmapW, c->d_Wb, Kp, Kp, c->tri, TC_BM);
  if (rc) return rc;
  rc = encode_map(c, &c->tmapP, c->d_Pb, Kq, Kq, (long long)c->M * c->nr, TC_BM);
  if (rc) return rc;
  // data-operand planes [3][M * 2K][K pad]: forward (written by the FFT kernels,
  // rows of Nr radii; the map reads zeros beyond Nr) and backward (written by
  // k_split_spec, rows of Nc - m coefficients; the tails stay zero from here)
  c->tc_kp = Kp;
  c->tc_kq = Kq;
  const long long brows = (long long)c->M * 2 * c->K;
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_bsf, sizeof(__nv_bfloat16) * 3 * brows * Kp));
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_bsb, sizeof(__nv_bfloat16) * 3 * brows * Kq));
  MLX_CUDA_TRY(c, cudaMemsetAsync(c->d_bsf, 0, sizeof(__nv_bfloat16) * 3 * brows * Kp, st));
  MLX_CUDA_TRY(c, cudaMemsetAsync(c->d_bsb, 0, sizeof(__nv_bfloat16) * 3 * brows * Kq, st));
  // A-row bases: W rows of m start at sum_{m'<m}(Nc - m'); P^T rows at m * Nr
  std::vector<long long> aw(c->M), ap(c->M);
  long long t = 0;
  for (int m = 0; m < c->M; ++m) { aw[m] = t; ap[m] = (long long)m * c->nr; t += c->nc - m; }
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_arowW, sizeof(long long) * c->M));
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_arowP, sizeof(long long) * c->M));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(c->d_arowW, aw.data(), sizeof(long long) * c->M, cudaMemcpyHostToDevice, st));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(c->d_arowP, ap.data(), sizeof(long long) * c->M, cudaMemcpyHostToDevice, st));
  // columns per tile (interleaved Re/Im pairs, multiple of 16, at most 128): the
  // widest tile whose item list still gives every SM work, else 32
  const int ncol = 2 * c->K;
  int bn = 32;
  {
    int rt = 0;
    for (int m = 0; m < c->M; ++m) rt += (c->nc - m + TC_BM - 1) / TC_BM;
    for (int cand = TC_MAX_BN; cand >= 32; cand -= 16)
      if ((long long)rt * ((ncol + cand - 1) / cand) >= sm_count()) { bn = cand; break; }
  }
  return mlx_tc_retile(c, bn, st);
}

// Tile lists for a requested column-tile width (the autotuner's knob).
int mlx_tc_retile(mlx_ctx* c, int bn_req, cudaStream_t st) {
  const int ncol = 2 * c->K;
  if (bn_req < 16 || bn_req > 256) return MLX_EINVAL;
  if (bn_req > TC_MAX_BN) bn_req = TC_MAX_BN;
  const int nct = (ncol + bn_req - 1) / bn_req;
  c->tc_bn = ((ncol + nct - 1) / nct + 15) / 16 * 16;
  if (c->tc_bn > TC_MAX_BN) c->tc_bn = TC_MAX_BN;
  cudaFree(c->d_tc_fwd);
  cudaFree(c->d_tc_bwd);
  c->d_tc_fwd = c->d_tc_bwd = nullptr;
  // items ordered (m, row tile, column tile): consecutive CTAs share the basis
  // chunks of one (m, row tile) through L2
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
  while (cols < 4 * c->tc_bn) cols <<= 1;   // two tiles in flight x two accumulators of BN columns
  c->tc_tmem_cols = cols;
  // data-operand maps: boxes of BN rows (columns of the tile)
  const long long brows = (long long)c->M * 2 * c->K;
  int rc = encode_map(c, &c->tmapBf, c->d_bsf, c->nr, c->tc_kp, brows, c->tc_bn);
  if (rc) return rc;
  rc = encode_map(c, &c->tmapBb, c->d_bsb, c->tc_kq, c->tc_kq, brows, c->tc_bn);
  if (rc) return rc;
  if (c->d_bsv)
    for (int f = 0; f < 6; ++f) {
      unsigned short* base = reinterpret_cast<unsigned short*>(c->d_bsv) + (long long)f * 3 * brows * c->tc_kq;
      if ((rc = encode_map(c, &c->tmapBv[f], base, c->tc_kq, c->tc_kq, brows, c->tc_bn))) return rc;
    }
  // the attribute is a per-function ceiling shared by every context: the largest
  // size any tile width uses
  const int smem = (int)tc_smem(TC_MAX_BN);
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_leg_tc<true, 6, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_leg_tc<false, 6, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_leg_tc<true, 8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_leg_tc<false, 8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_leg_tc<true, 6, kTcBatchMax>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_leg_tc<false, 6, kTcBatchMax>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return MLX_OK;
}

namespace {

TcParams<1> single_params(mlx_ctx* c, const CUtensorMap& a, const CUtensorMap& b, bool fwd, double2* spec,
                          float* mixed) {
  TcParams<1> P;
  P.a[0] = a;
  P.b[0] = b;
  TcArgs& g = P.g[0];
  memset(&g, 0, sizeof(g));
  g.nc = c->nc; g.nr = c->nr; g.M = c->M; g.K = c->K; g.bn = c->tc_bn;
  g.soff = c->d_soff;
  g.arow = fwd ? c->d_arowW : c->d_arowP;
  g.spec_out = spec;
  g.mixed_out = mixed;
  return P;
}

int launch_single(mlx_ctx* c, bool fwd, const TcParams<1>& P, cudaStream_t st) {
  const int n = fwd ? c->ntc_fwd : c->ntc_bwd;
  const LegTile* items = fwd ? c->d_tc_fwd : c->d_tc_bwd;
  const int grid = n < sm_count() ? n : sm_count();
  const size_t smem = tc_smem(c->tc_bn);
  if (fwd) {
    auto kern = c->tc_products == 8 ? k_leg_tc<true, 8, 1> : k_leg_tc<true, 6, 1>;
    MLX_CUDA_TRY(c, launch_pdl(kern, dim3(grid), dim3(TC_THREADS), smem, st, P, items, n, c->tc_bn,
                               c->tc_tmem_cols, c->tc_expire, c->d_err));
  } else {
    auto kern = c->tc_products == 8 ? k_leg_tc<false, 8, 1> : k_leg_tc<false, 6, 1>;
    MLX_CUDA_TRY(c, launch_pdl(kern, dim3(grid), dim3(TC_THREADS), smem, st, P, items, n, c->tc_bn,
                               c->tc_tmem_cols, c->tc_expire, c->d_err));
  }
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

}  // namespace

int mlx_legendre_tc_forward(mlx_ctx* c, double2* spec, cudaStream_t st) {
  TimedLaunch tl(c, KID_LEG_FWD, st);
  return launch_single(c, true, single_params(c, c->tmapW, c->tmapBf, true, spec, nullptr), st);
}

int mlx_tc_vortex_planes(mlx_ctx* c, cudaStream_t st) {
  if (c->d_bsv) return MLX_OK;
  const long long brows = (long long)c->M * 2 * c->K;
  const size_t bytes = sizeof(__nv_bfloat16) * 6 * 3 * brows * c->tc_kq;
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_bsv, bytes));
  MLX_CUDA_TRY(c, cudaMemsetAsync(c->d_bsv, 0, bytes, st));   // row tails n - m >= Nc - m stay zero
  return mlx_tc_retile(c, c->tc_bn, st);                       // encodes the six maps
}

int mlx_legendre_tc_backward_field(mlx_ctx* c, int f, cudaStream_t st) {
  TimedLaunch tl(c, KID_LEG_BWD, st);
  return launch_single(c, false, single_params(c, c->tmapP, c->tmapBv[f], false, nullptr, (float*)c->d_mixed), st);
}

int mlx_legendre_tc_backward(mlx_ctx* c, const double2* spec, cudaStream_t st, bool planes_ready) {
  if (!planes_ready) {   // (planes_ready: the solve that wrote spec also wrote its split planes)
    TimedLaunch tl(c, KID_LEG_SPLIT, st);
    const int tb = c->nc >= 128 ? 128 : 64;
    k_split_spec<<<dim3((c->nc + tb - 1) / tb, c->K, c->M), tb, 0, st>>>(
        c->nc, c->K, (int)c->tc_kq, (long long)c->M * 2 * c->K * c->tc_kq, c->d_soff, spec,
        (unsigned short*)c->d_bsb);
    MLX_LAUNCH_CHECK(c);
  }
  TimedLaunch tl(c, KID_LEG_BWD, st);
  return launch_single(c, false, single_params(c, c->tmapP, c->tmapBb, false, nullptr, (float*)c->d_mixed), st);
}

// ---- batched persistent contraction (batch.cu) ----
// One launch serves up to kTcBatchMax MLX_BF16X3 members: their maps and sizes are
// the launch parameters, the work items (m, row tile, column tile, member) of all
// members one list sorted by decreasing length (chunks), walked round-robin by the
// persistent CTAs as in the single-context launch.  Each item uses its member's
// column-tile width; the ring stages and TMEM accumulators are sized for the
// widest.  A bounded wait that expires is reported in the first member's status
// word.
struct TcBatchPlan {
  TcParams<kTcBatchMax> P;
  LegTile* d_items = nullptr;
  int nitems = 0, bnmax = 16, tmem_cols = 32, grid = 0;
  bool fwd = true;
  int* err = nullptr;
  // backward split of the members' spectral states into their planes
  SplitJob* d_split = nullptr;
  int4* d_split_items = nullptr;
  int nsplit = 0, split_grid = 0;
  int* d_ctr = nullptr;
};

namespace {

// Batched split (backward direction): items (member, m, k slot); a CTA of 128
// threads splits the Nc - m coefficients of that column, as k_split_spec does.
__global__ void __launch_bounds__(128) kb_split_spec(const SplitJob* __restrict__ jobs, const int4* __restrict__ items,
                                                    int nitems, int* __restrict__ ctr) {
  __shared__ int s_it;
  for (;;) {
    if (threadIdx.x == 0) s_it = atomicAdd(ctr, 1);
    __syncthreads();
    const int it = s_it;
    if (it >= nitems) break;
    const int4 w = items[it];
    const SplitJob j = jobs[w.x];
    const int m = w.y, kidx = w.z;
    const int Nm = j.nc - m;
    for (int a = threadIdx.x; a < Nm; a += blockDim.x) {
      const long long idx = j.soff[m] + (long long)kidx * Nm + a;
      const uint4 wv = __ldg(reinterpret_cast<const uint4*>(j.spec) + idx);
      const float v[2] = {f64w_to_f32(wv.y, wv.x), f64w_to_f32(wv.w, wv.z)};
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        __nv_bfloat16 h, md, l;
        split3<float>(v[p], h, md, l);
        const long long o = ((long long)m * 2 * j.K + 2 * kidx + p) * j.Kq + a;
        j.bs[o] = __bfloat16_as_ushort(h);
        j.bs[j.part + o] = __bfloat16_as_ushort(md);
        j.bs[2 * j.part + o] = __bfloat16_as_ushort(l);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) bq_finish(ctr, gridDim.x);
}

}  // namespace

// Plan of one batched contraction launch over members[0..n) (n <= kTcBatchMax,
// every one MLX_BF16X3).  Forward: mixed planes (already split) -> specs[i];
// backward: specs[i] split into the members' planes (those with need_split[i],
// or all when need_split is NULL; the others' planes are already written), then
// -> their mixed buffers.
int mlx_tc_batch_plan(mlx_ctx* const* members, int n, bool fwd, double2* const* specs, const char* need_split,
                      TcBatchPlan** out) {
  *out = nullptr;
  if (n <= 0 || n > kTcBatchMax) return MLX_EINVAL;
  TcBatchPlan* pl = new TcBatchPlan();
  memset(&pl->P, 0, sizeof(pl->P));
  pl->fwd = fwd;
  pl->err = members[0]->d_err;
  std::vector<LegTile> items;
  std::vector<double> cost;
  std::vector<SplitJob> sj;
  std::vector<int4> si;
  for (int i = 0; i < n; ++i) {
    mlx_ctx* c = members[i];
    if (c->precision != MLX_BF16X3) { delete pl; return MLX_EINVAL; }
    pl->P.a[i] = fwd ? c->tmapW : c->tmapP;
    pl->P.b[i] = fwd ? c->tmapBf : c->tmapBb;
    TcArgs& g = pl->P.g[i];
    g.nc = c->nc; g.nr = c->nr; g.M = c->M; g.K = c->K; g.bn = c->tc_bn;
    g.soff = c->d_soff;
    g.arow = fwd ? c->d_arowW : c->d_arowP;
    g.spec_out = fwd ? specs[i] : nullptr;
    g.mixed_out = fwd ? nullptr : (float*)c->d_mixed;
    if (c->tc_bn > pl->bnmax) pl->bnmax = c->tc_bn;
    const int ncol = 2 * c->K;
    for (int m = 0; m < c->M; ++m) {
      const int rows = fwd ? c->nc - m : c->nr;
      const int kdim = fwd ? c->nr : c->nc - m;
      for (int r0 = 0; r0 < rows; r0 += TC_BM)
        for (int c0 = 0; c0 < ncol; c0 += c->tc_bn) {
          items.push_back(LegTile{m, r0, c0, i});
          cost.push_back((double)((kdim + TC_BK - 1) / TC_BK));
        }
    }
    if (!fwd && (!need_split || need_split[i])) {
      SplitJob j;
      j.nc = c->nc; j.K = c->K; j.Kq = (int)c->tc_kq;
      j.part = (long long)c->M * 2 * c->K * c->tc_kq;
      j.soff = c->d_soff;
      j.spec = specs[i];
      j.bs = (unsigned short*)c->d_bsb;
      const int js = (int)sj.size();
      sj.push_back(j);
      for (int m = 0; m < c->M; ++m)
        for (int k = 0; k < c->K; ++k) si.push_back(make_int4(js, m, k, 0));
    }
  }
  // decreasing length; members' items stay in their (m, row tile, column tile)
  // order within one length, so that neighbouring CTAs share basis chunks in L2
  std::vector<int> ord(items.size());
  for (size_t t = 0; t < ord.size(); ++t) ord[t] = (int)t;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<LegTile> sorted(items.size());
  for (size_t t = 0; t < ord.size(); ++t) sorted[t] = items[ord[t]];
  pl->nitems = (int)sorted.size();
  pl->grid = pl->nitems < sm_count() ? pl->nitems : sm_count();
  int cols = 32;
  while (cols < 4 * pl->bnmax) cols <<= 1;
  pl->tmem_cols = cols;
  auto fail = [&](cudaError_t) { mlx_tc_batch_free(pl); return MLX_ECUDA; };
  cudaError_t e;
  if ((e = cudaMalloc(&pl->d_items, sizeof(LegTile) * sorted.size())) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(pl->d_items, sorted.data(), sizeof(LegTile) * sorted.size(), cudaMemcpyHostToDevice)) !=
      cudaSuccess) return fail(e);
  if (!si.empty()) {
    pl->nsplit = (int)si.size();
    pl->split_grid = pl->nsplit < 8 * sm_count() ? pl->nsplit : 8 * sm_count();
    if ((e = cudaMalloc(&pl->d_split, sizeof(SplitJob) * sj.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&pl->d_split_items, sizeof(int4) * si.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&pl->d_ctr, 2 * sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(pl->d_split, sj.data(), sizeof(SplitJob) * sj.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(e);
    if ((e = cudaMemcpy(pl->d_split_items, si.data(), sizeof(int4) * si.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess) return fail(e);
    if ((e = cudaMemset(pl->d_ctr, 0, 2 * sizeof(int))) != cudaSuccess) return fail(e);
  }
  *out = pl;
  return MLX_OK;
}

int mlx_tc_batch_launch(TcBatchPlan* pl, cudaStream_t st) {
  if (!pl->fwd && pl->nsplit > 0) {
    kb_split_spec<<<pl->split_grid, 128, 0, st>>>(pl->d_split, pl->d_split_items, pl->nsplit, pl->d_ctr);
    if (cudaGetLastError() != cudaSuccess) return MLX_ECUDA;
  }
  const size_t smem = tc_smem(pl->bnmax);
  if (pl->fwd)
    k_leg_tc<true, 6, kTcBatchMax><<<pl->grid, TC_THREADS, smem, st>>>(pl->P, pl->d_items, pl->nitems, pl->bnmax,
                                                                      pl->tmem_cols, 0, pl->err);
  else
    k_leg_tc<false, 6, kTcBatchMax><<<pl->grid, TC_THREADS, smem, st>>>(pl->P, pl->d_items, pl->nitems, pl->bnmax,
                                                                       pl->tmem_cols, 0, pl->err);
  return cudaGetLastError() == cudaSuccess ? MLX_OK : MLX_ECUDA;
}

void mlx_tc_batch_free(TcBatchPlan* pl) {
  if (!pl) return;
  if (pl->d_items) cudaFree(pl->d_items);
  if (pl->d_split) cudaFree(pl->d_split);
  if (pl->d_split_items) cudaFree(pl->d_split_items);
  if (pl->d_ctr) cudaFree(pl->d_ctr);
  delete pl;
}
