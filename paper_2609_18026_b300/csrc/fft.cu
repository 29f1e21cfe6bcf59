// K2/K3: azimuthal (real) and axial (complex) Fourier transforms of the
// transform pair (Eq. (2)), as batched warp-shuffle FFTs.
//
// Global layouts (planar complex, r fastest so that a warp reads consecutive radii):
//   physical  [Nz][Nphi][Nr] real
//   zm        [2][Nz][M][Nr]      after the phi transform (Re plane, Im plane)
//   mixed     [2][K][M][Nr]       after the z transform; for Nz == 1 zm == mixed
// A CTA of the phi kernel owns one z-plane and a tile of R radii; two real radial
// lines (r and r + R/2) are packed into one complex line of length Nphi.  A CTA of
// the z kernel owns one m and a tile of R radii (one complex line per radius).
// Tiles are staged through shared memory as [line][point] rows of stride N + 1
// (coalesced global access along r; conflict-free per-line reads; the global-load
// loops are unrolled so that every thread keeps several loads in flight, which
// the memory latency needs at these occupancies).  Each line is
// transformed by one warp (or a group of N lanes when N < 32): lane l holds
// points l + 32 e, e < E = N/32, in registers; butterflies at distance >= 32 are
// in-lane, below 32 they use __shfl_xor_sync.  DIF (natural in, bit-reversed
// out) and DIT (bit-reversed in, natural out) radix-2 stages; the fused Fisher-KPP
// kernel runs inverse DIF -> gamma u (1 - u) -> forward DIT without leaving
// registers.
#include "mlx_internal.cuh"

#include <cuda_bf16.h>
#include <string.h>

namespace {

template <typename T> struct C2T;
template <> struct C2T<float> { typedef float2 type; };
template <> struct C2T<double> { typedef double2 type; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C shfl_xor(C v, int d) {
  C r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, d);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, d);
  return r;
}
// twiddle exp(-+ 2 pi i t / N) from the table exp(-2 pi i t / N), t < N/2
template <typename C> __device__ __forceinline__ C twid(const C* __restrict__ tw, int t, bool inv) {
  C w = tw[t];
  if (inv) w.y = -w.y;
  return w;
}

__device__ __forceinline__ int bitrev(int p, int logn) {
  return logn ? (int)(__brev((unsigned)p) >> (32 - logn)) : 0;
}

template <typename T> __device__ __forceinline__ T fmaT(T a, T b, T c);
template <> __device__ __forceinline__ float fmaT<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <> __device__ __forceinline__ double fmaT<double>(double a, double b, double c) { return fma(a, b, c); }

// The CTA's per-stage twiddle tables in shared memory (staged once per CTA, before
// the tile's first barrier): the butterflies at distance d (d = N/2, ..., 1) use
// exp(-2 pi i t (N / 2d) / N) for t < d, stored contiguously at offset N - 2d (N - 1
// entries in all), so that the lanes of a stage read consecutive entries or one
// entry (a strided read of the single table exp(-2 pi i t / N) conflicts on the
// banks).  tw: the global table exp(-2 pi i t / N), t < N/2.
template <typename C>
__device__ __forceinline__ void stage_twiddles(C* __restrict__ tws, const C* __restrict__ tw, int N) {
  for (int u = threadIdx.x; u < N - 1; u += blockDim.x) {
    int d = N >> 1, off = 0;
    while (u >= off + d) { off += d; d >>= 1; }
    tws[u] = tw[(u - off) * (N / (2 * d))];
  }
}
// twiddle of stage d, index t < d, from the per-stage tables (conjugated for inverse)
template <typename C>
__device__ __forceinline__ C stw(const C* __restrict__ tws, int N, int d, int t, bool inv) {
  return twid(tws, N - 2 * d + t, inv);
}

// asynchronous global -> shared copy of one element (4 or 8 bytes): the tile loads
// keep every element in flight at once instead of staging them through registers
template <typename T>
__device__ __forceinline__ void cp_async_el(T* smem_dst, const T* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
// the same with the shared-memory address already converted
template <typename T>
__device__ __forceinline__ void cp_async_el_s(unsigned d, const T* gsrc) {
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Decimation in frequency: natural order in, bit-reversed order out.
// j = lj + 32 e is the point held in v[e]; N = 32 E when E > 1 (all strides then
// compile-time constants), else N <= 32.  tw: the shared-memory twiddle copy.
// Lane-exchange stage at distance d (the partner holds p): the lower lane keeps
// v + p, the upper lane (p - v) w.  Both are written as (p + sgn v) weff with
// sgn = +-1 and weff = 1 or w chosen once per stage, with no select per point.
template <typename C, int E>
__device__ __forceinline__ void dif(C (&v)[E], int N, int lj, const C* __restrict__ tw, bool inv) {
  typedef decltype(C().x) T;
#pragma unroll
  for (int de = E / 2; de >= 1; de >>= 1) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if ((e & de) == 0) {
        const C w = stw(tw, 32 * E, 32 * de, lj + 32 * (e & (de - 1)), inv);
        const C a = v[e], b = v[e + de];
        v[e] = cadd(a, b);
        v[e + de] = cmul(csub(a, b), w);
      }
    }
  }
  auto stage = [&](int d) {
    const bool upper = (lj & d) != 0;
    C w = stw(tw, N, d, lj & (d - 1), inv);
    if (!upper) { w.x = (T)1; w.y = (T)0; }
    const T sg = upper ? (T)-1 : (T)1;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const C p = shfl_xor(v[e], d);
      C t;
      t.x = fmaT(sg, v[e].x, p.x);
      t.y = fmaT(sg, v[e].y, p.y);
      v[e] = cmul(t, w);
    }
  };
  if constexpr (E > 1) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) stage(d);
  } else {
    for (int d = N >> 1; d >= 1; d >>= 1) stage(d);
  }
}

// Decimation in time: bit-reversed order in, natural order out.  Lane-exchange
// stage: the lower lane keeps v + w p, the upper lane p - w v.  The upper lane
// multiplies its own value by w before the exchange (the lower lane by 1), so
// that both write a + sgn b with the received value: no select per point.
template <typename C, int E>
__device__ __forceinline__ void dit(C (&v)[E], int N, int lj, const C* __restrict__ tw, bool inv) {
  typedef decltype(C().x) T;
  auto stage = [&](int d) {
    const bool upper = (lj & d) != 0;
    C w = stw(tw, N, d, lj & (d - 1), inv);
    if (!upper) { w.x = (T)1; w.y = (T)0; }
    const T sg = upper ? (T)-1 : (T)1;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const C a = cmul(w, v[e]);          // lower: v; upper: w v
      const C p = shfl_xor(a, d);         // lower: w v_upper; upper: v_lower
      v[e].x = fmaT(sg, a.x, p.x);
      v[e].y = fmaT(sg, a.y, p.y);
    }
  };
  if constexpr (E > 1) {
#pragma unroll
    for (int d = 1; d <= 16; d <<= 1) stage(d);
  } else {
    for (int d = 1; d < N; d <<= 1) stage(d);
  }
#pragma unroll
  for (int de = 1; de <= E / 2; de <<= 1) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if ((e & de) == 0) {
        const C w = stw(tw, 32 * E, 32 * de, lj + 32 * (e & (de - 1)), inv);
        const C a = v[e], b = cmul(w, v[e + de]);
        v[e] = cadd(a, b);
        v[e + de] = csub(a, b);
      }
    }
  }
}

// Iterate the lines of a CTA tile warp by warp; calls f(line, lj, active).
// All 32 lanes of a warp take part in every call (the shuffles need them).
template <typename F>
__device__ __forceinline__ void for_lines(int N, int nlines, F f) {
  const int lpl = N < 32 ? N : 32;         // lanes per line
  const int lpw = 32 / lpl;                 // lines per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b0 = warp * lpw; b0 < nlines; b0 += nw * lpw) {
    const int b = b0 + lane / lpl;
    f(b, lane % lpl, b < nlines);
  }
}

enum PhiMode { PHI_FWD = 0, PHI_BWD = 1, PHI_FKPP = 2 };

// Forward output for the MLX_BF16X3 contraction: the value of (m, slot kk, part p
// = Re/Im, radius r) as three BF16 parts hi, mid, lo (round to nearest, FP32
// residuals) in the planes bs[part][(m * 2K + 2 kk + p) * Kp + r], the K-major data
// operand that the tensor-core kernel loads by TMA.
struct SplitOut {
  unsigned short* bs = nullptr;   // null: write the FP32 planes instead
  long long part;                 // elements per part plane
  int Kp, K2;                     // row length (padded K-dim) and columns per m (2K)
};
template <typename T>
__device__ __forceinline__ void split_store(const SplitOut& so, int m, int kk, int p, int r, T vt) {
  if constexpr (sizeof(T) == 4) {
    const float v = (float)vt;
    const unsigned short h = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    const float r1 = v - __bfloat162float(__ushort_as_bfloat16(h));
    const unsigned short md = __bfloat16_as_ushort(__float2bfloat16_rn(r1));
    const float r2 = r1 - __bfloat162float(__ushort_as_bfloat16(md));
    const unsigned short lo = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
    const long long o = ((long long)m * so.K2 + 2 * kk + p) * so.Kp + r;
    so.bs[o] = h;
    so.bs[so.part + o] = md;
    so.bs[2 * so.part + o] = lo;
  }
}

// Real analysis of packed line pairs held in L[b][m] (natural order, forward
// DFT), scaled by 1/N, written to zm for this (z, r-tile).
// With brev the line holds frequency p at position bitrev(p) (DIF output kept in
// register order), so only the M retained frequencies are looked up scattered.
template <typename T, typename C>
__device__ void phi_unpack_store(const C* L, int ld, int N, int B, int M, int Nr, int r0, int z,
                                 T* __restrict__ zre, T* __restrict__ zim, bool brev, int logN,
                                 const SplitOut& so) {
  const T inv = (T)1 / (T)N;
  const int R = 2 * B;
  const int lR = __ffs(R) - 1;          // tiles are powers of two: shifts, not divisions
  // blockDim.x is a multiple of R: each thread keeps one radius and steps through m
  const int rr = threadIdx.x & (R - 1), mstep = (int)blockDim.x >> lR;
  const int b = rr & (B - 1);
  if (r0 + rr >= Nr) return;
#pragma unroll 2
  for (int m = threadIdx.x >> lR; m < M; m += mstep) {
    const int pm = m, pc = (N - m) & (N - 1);
    const C zm = L[b * ld + (brev ? bitrev(pm, logN) : pm)];
    const C zc = L[b * ld + (brev ? bitrev(pc, logN) : pc)];
    T re, im;
    if (rr < B) {  // X_m = (Z_m + conj(Z_{N-m})) / 2
      re = (zm.x + zc.x) * (T)0.5;
      im = (zm.y - zc.y) * (T)0.5;
    } else {       // Y_m = (Z_m - conj(Z_{N-m})) / (2i)
      re = (zm.y + zc.y) * (T)0.5;
      im = (zc.x - zm.x) * (T)0.5;
    }
    // Nyquist chop: m = +-N/2 share the grid function (-1)^j, and each stored
    // member takes half of the (real) bin
    if (m == (N >> 1)) re *= (T)0.5;
    const int r = r0 + rr;
    if (so.bs) {
      split_store<T>(so, m, 0, 0, r, re * inv);
      split_store<T>(so, m, 0, 1, r, im * inv);
    } else {
      const long long o = ((long long)z * M + m) * Nr + r;
      zre[o] = re * inv;
      zim[o] = im * inv;
    }
  }
}

// One CTA tile of the phi transform: radii bx R .. bx R + R - 1 of z-plane z.
template <typename T, int MODE, int E>
__device__ __forceinline__ void phi_tile(int N, int logN, int M, int Nr, int R, int bx, int z,
                                         T* __restrict__ phys, T* __restrict__ zre, T* __restrict__ zim,
                                         const typename C2T<T>::type* __restrict__ tw, T gamma,
                                         int* __restrict__ err, const SplitOut& so,
                                         unsigned char* __restrict__ smem_raw) {
  typedef typename C2T<T>::type C;
  C* L = reinterpret_cast<C*>(smem_raw);
  const int B = R / 2;
  const int lR = __ffs(R) - 1;          // R and B are powers of two
  const int ld = N + 1;
  const int r0 = bx * R;
  const long long plane = (long long)z * N * Nr;
  C* tws = L + (size_t)B * ld;          // the twiddle tables after the tile
  stage_twiddles(tws, tw, N);

  // blockDim.x is a multiple of R: each thread keeps one radius of the tile
  const int rr = threadIdx.x & (R - 1), rstep = (int)blockDim.x >> lR;
  if constexpr (MODE == PHI_FWD) {
    {
      const int r = r0 + rr;
      T* srow = reinterpret_cast<T*>(&L[(rr & (B - 1)) * ld]) + (rr < B ? 0 : 1);   // point j at srow[2 j]
      if (r < Nr) {
        const T* g = phys + plane + r;
        const unsigned s0 = (unsigned)__cvta_generic_to_shared(srow);
#pragma unroll 4
        for (int j = threadIdx.x >> lR; j < N; j += rstep)
          cp_async_el_s(s0 + (unsigned)(j * (int)sizeof(C)), g + (long long)j * Nr);
      } else {
        for (int j = threadIdx.x >> lR; j < N; j += rstep) srow[2 * j] = (T)0;
      }
    }
    cp_async_all();
    __syncthreads();
    for_lines(N, B, [&](int b, int lj, bool act) {
      C v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = act ? L[b * ld + lj + 32 * e] : C{};
      dif<C, E>(v, N, lj, tws, false);
      if (act) {
#pragma unroll
        for (int e = 0; e < E; ++e) L[b * ld + lj + 32 * e] = v[e];   // bit-reversed order
      }
    });
    __syncthreads();
    phi_unpack_store<T, C>(L, ld, N, B, M, Nr, r0, z, zre, zim, true, logN, so);
  } else {
    // packed Hermitian spectrum of each line pair: Zhat[m] = A_m + i B_m,
    // Zhat[N-m] = conj(A_m) + i conj(B_m), Zhat[0] = Re A_0 + i Re B_0
    for (int t = threadIdx.x; t < B * ld; t += blockDim.x) L[t] = C{};
    __syncthreads();
    const int b = threadIdx.x & (B - 1), mstep = (int)blockDim.x >> (lR - 1);
    const int ra = r0 + b, rb = r0 + b + B;
    const bool va = ra < Nr, vb = rb < Nr;
    const T* __restrict__ zr = zre + (long long)z * M * Nr;
    const T* __restrict__ zi = zim + (long long)z * M * Nr;
#pragma unroll 4
    for (int m = threadIdx.x >> (lR - 1); m < M; m += mstep) {
      T ar = 0, ai = 0, br = 0, bi = 0;
      const long long oa = (long long)m * Nr;
      if (va) { ar = zr[oa + ra]; ai = zi[oa + ra]; }
      if (vb) { br = zr[oa + rb]; bi = zi[oa + rb]; }
      // the synthesis-only transform takes its input bit-reversed (DIT), the fused
      // Fisher-KPP transform in natural order (DIF, product, DIT)
      const int p1 = (MODE == PHI_BWD) ? bitrev(m, logN) : m;
      const int p2 = (MODE == PHI_BWD) ? bitrev(N - m, logN) : N - m;
      if (m == 0) {
        C v; v.x = ar; v.y = br;
        L[b * ld] = v;
      } else if (m == (N >> 1)) {
        // Nyquist chop: the m and N - m slots coincide; the bin receives both
        // members of the pair, A_m + conj(A_m) + i (B_m + conj(B_m))
        C v; v.x = ar + ar; v.y = br + br;
        L[b * ld + p1] = v;
      } else {
        C v1; v1.x = ar - bi; v1.y = ai + br;
        C v2; v2.x = ar + bi; v2.y = br - ai;
        L[b * ld + p1] = v1;
        L[b * ld + p2] = v2;
      }
    }
    __syncthreads();
    for_lines(N, B, [&](int b, int lj, bool act) {
      C v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = act ? L[b * ld + lj + 32 * e] : C{};
      if constexpr (MODE == PHI_BWD) {
        dit<C, E>(v, N, lj, tws, true);   // bit-reversed spectrum in, physical values in natural order
        if (act) {
#pragma unroll
          for (int e = 0; e < E; ++e) L[b * ld + lj + 32 * e] = v[e];
        }
        return;
      }
      dif<C, E>(v, N, lj, tws, true);   // physical values, bit-reversed positions
      if constexpr (MODE == PHI_FKPP) {
        bool finite = true;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          v[e].x = gamma * v[e].x * ((T)1 - v[e].x);
          v[e].y = gamma * v[e].y * ((T)1 - v[e].y);
          finite = finite && isfinite(v[e].x) && isfinite(v[e].y);
        }
        // a non-finite product (blow-up or NaN in the state) sets the status bit
        // that mlx_device_status reports as MLX_ENUMERIC
        if (__any_sync(0xffffffffu, !finite) && (threadIdx.x & 31) == 0) atomicOr(err, 16);
        dit<C, E>(v, N, lj, tws, false);   // forward DFT, natural order
        if (act) {
#pragma unroll
          for (int e = 0; e < E; ++e) L[b * ld + lj + 32 * e] = v[e];
        }
      }
    });
    __syncthreads();
    if constexpr (MODE == PHI_BWD) {
      const int r = r0 + rr;
      if (r < Nr) {
        const T* srow = reinterpret_cast<const T*>(&L[(rr & (B - 1)) * ld]) + (rr < B ? 0 : 1);
        T* g = phys + plane + r;
#pragma unroll 4
        for (int j = threadIdx.x >> lR; j < N; j += rstep) g[(long long)j * Nr] = srow[2 * j];
      }
    } else {
      phi_unpack_store<T, C>(L, ld, N, B, M, Nr, r0, z, zre, zim, false, logN, so);
    }
  }
}

template <typename T, int MODE, int E>
__global__ void __launch_bounds__(256) k_phi(int N, int logN, int M, int Nr, int R,
                                             T* __restrict__ phys, T* __restrict__ zre,
                                             T* __restrict__ zim,
                                             const typename C2T<T>::type* __restrict__ tw, T gamma,
                                             int* __restrict__ err, SplitOut so) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  phi_tile<T, MODE, E>(N, logN, M, Nr, R, blockIdx.x, blockIdx.y, phys, zre, zim, tw, gamma, err, so, smem_raw);
  pdl_trigger();
}

// Axial transform for one m and a tile of R radii: lines are radii.
template <typename T, bool INVERSE, int E>
__device__ __forceinline__ void z_tile(int Nz, int logN, int Kz, int K, int M, int Nr, int R, int bx, int m,
                                       T* __restrict__ zre, T* __restrict__ zim,
                                       T* __restrict__ mre, T* __restrict__ mim,
                                       const typename C2T<T>::type* __restrict__ tw, const SplitOut& so,
                                       unsigned char* __restrict__ smem_raw) {
  typedef typename C2T<T>::type C;
  C* L = reinterpret_cast<C*>(smem_raw);
  const int ld = Nz + 1;
  const int r0 = bx * R;
  const int lR = __ffs(R) - 1;          // R is a power of two
  C* tws = L + (size_t)R * ld;          // the twiddle tables after the tile
  stage_twiddles(tws, tw, Nz);
  // blockDim.x is a multiple of R: each thread keeps one radius (line b) of the
  // tile in the loads and stores (recomputed per phase, so that nothing stays
  // live across the transform)
#define MLX_Z_LINE                                                       \
  const int b = threadIdx.x & (R - 1), lstep = (int)blockDim.x >> lR;    \
  const int r = r0 + b;                                                  \
  const long long rs = (long long)M * Nr;   /* stride of a z (or k) row */ \
  const long long mo = (long long)m * Nr + r;                            \
  C* Lb = L + (size_t)b * ld;
  if (!INVERSE) {
    MLX_Z_LINE
    if (r < Nr) {
      const unsigned s0 = (unsigned)__cvta_generic_to_shared(Lb);
#pragma unroll 4
      for (int l = threadIdx.x >> lR; l < Nz; l += lstep) {
        const long long o = (long long)l * rs + mo;
        const unsigned d = s0 + (unsigned)(l * (int)sizeof(C));
        cp_async_el_s(d, zre + o);
        cp_async_el_s(d + (unsigned)sizeof(T), zim + o);
      }
    } else {
      for (int l = threadIdx.x >> lR; l < Nz; l += lstep) Lb[l] = C{};
    }
    cp_async_all();
  } else {
    for (int t = threadIdx.x; t < R * ld; t += blockDim.x) L[t] = C{};
    __syncthreads();
    // Nyquist chop (K = Nz + 1): rows k = +Nz/2 (kk = Kz - 1) and k = -Nz/2
    // (kk = Kz) feed the same bin, which receives their sum
    const bool nyq = K == Nz + 1;
    MLX_Z_LINE
    if (r < Nr) {
      const unsigned s0 = (unsigned)__cvta_generic_to_shared(Lb);
#pragma unroll 2
      for (int kk = threadIdx.x >> lR; kk < K; kk += lstep) {
        const int pos = (kk < Kz) ? kk : Nz - (K - kk);
        if (nyq && kk == Kz) continue;
        const long long o = (long long)kk * rs + mo;
        const int q = bitrev(pos, logN);            // bit-reversed input of the DIT below
        if (nyq && kk == Kz - 1) {
          const long long o2 = (long long)Kz * rs + mo;
          C v;
          v.x = mre[o] + mre[o2];
          v.y = mim[o] + mim[o2];
          Lb[q] = v;
        } else {
          const unsigned d = s0 + (unsigned)(q * (int)sizeof(C));
          cp_async_el_s(d, mre + o);
          cp_async_el_s(d + (unsigned)sizeof(T), mim + o);
        }
      }
    }
    cp_async_all();
  }
  __syncthreads();
  for_lines(Nz, R, [&](int b, int lj, bool act) {
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = act ? L[b * ld + lj + 32 * e] : C{};
    // forward: DIF, output kept in register (bit-reversed) order; inverse: DIT
    // from the bit-reversed input, natural output.  Either way the dense line is
    // written back in register order, and only the K retained wavenumbers are
    // addressed through the bit reversal.
    if (INVERSE) dit<C, E>(v, Nz, lj, tws, true);
    else dif<C, E>(v, Nz, lj, tws, false);
    if (act) {
#pragma unroll
      for (int e = 0; e < E; ++e) L[b * ld + lj + 32 * e] = v[e];
    }
  });
  __syncthreads();
  MLX_Z_LINE
#undef MLX_Z_LINE
  if (r >= Nr) return;
  if (!INVERSE) {
    const T inv = (T)1 / (T)Nz;
    const bool nyq = K == Nz + 1;     // Nyquist chop: rows k = +-Nz/2 take half the bin each
#pragma unroll 4
    for (int kk = threadIdx.x >> lR; kk < K; kk += lstep) {
      const int pos = (kk < Kz) ? kk : Nz - (K - kk);
      C v = Lb[bitrev(pos, logN)];
      if (nyq && (kk == Kz - 1 || kk == Kz)) { v.x *= (T)0.5; v.y *= (T)0.5; }
      if (so.bs) {
        split_store<T>(so, m, kk, 0, r, v.x * inv);
        split_store<T>(so, m, kk, 1, r, v.y * inv);
      } else {
        const long long o = (long long)kk * rs + mo;
        mre[o] = v.x * inv;
        mim[o] = v.y * inv;
      }
    }
  } else {
#pragma unroll 2
    for (int l = threadIdx.x >> lR; l < Nz; l += lstep) {
      const C v = Lb[l];
      const long long o = (long long)l * rs + mo;
      zre[o] = v.x;
      zim[o] = v.y;
    }
  }
}

template <typename T, bool INVERSE, int E>
__global__ void __launch_bounds__(256) k_z(int Nz, int logN, int Kz, int K, int M, int Nr, int R,
                                           T* __restrict__ zre, T* __restrict__ zim,
                                           T* __restrict__ mre, T* __restrict__ mim,
                                           const typename C2T<T>::type* __restrict__ tw, SplitOut so) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  z_tile<T, INVERSE, E>(Nz, logN, Kz, K, M, Nr, R, blockIdx.x, blockIdx.y, zre, zim, mre, mim, tw, so, smem_raw);
  pdl_trigger();
}

// Batched persistent forms of the stages (batch.cu): every CTA takes (member,
// radius tile, plane) items from the queue until it is empty; the member's job
// gives the sizes and buffers and E (1..8: transforms of at most 256 points) the
// register width of its lines.  The tile
// functions are those of the single-context kernels, so each member's values are
// bitwise those of its own launches.
__device__ __forceinline__ SplitOut job_split(const BFftJob& j) {
  SplitOut so;
  if (j.bs) { so.bs = j.bs; so.part = j.part; so.Kp = j.kp; so.K2 = j.k2; }
  return so;
}

template <typename T>
__global__ void __launch_bounds__(256) kb_phi_fkpp(const BFftJob* __restrict__ jobs, const int4* __restrict__ items,
                                                  int nitems, int* __restrict__ ctr) {
  typedef typename C2T<T>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_it;
  for (;;) {
    if (threadIdx.x == 0) s_it = atomicAdd(ctr, 1);
    __syncthreads();
    const int it = s_it;
    if (it >= nitems) break;
    const int4 w = items[it];
    const BFftJob j = jobs[w.x];
    const SplitOut so = job_split(j);
    T* zre = (T*)j.b;
    T* zim = (T*)j.c;
    const C* tw = (const C*)j.tw;
    switch (j.E) {
      case 1: phi_tile<T, PHI_FKPP, 1>(j.N, j.logN, j.M, j.Nr, j.R, w.y, w.z, nullptr, zre, zim, tw, (T)j.gamma, j.err, so, smem_raw); break;
      case 2: phi_tile<T, PHI_FKPP, 2>(j.N, j.logN, j.M, j.Nr, j.R, w.y, w.z, nullptr, zre, zim, tw, (T)j.gamma, j.err, so, smem_raw); break;
      case 4: phi_tile<T, PHI_FKPP, 4>(j.N, j.logN, j.M, j.Nr, j.R, w.y, w.z, nullptr, zre, zim, tw, (T)j.gamma, j.err, so, smem_raw); break;
      default: phi_tile<T, PHI_FKPP, 8>(j.N, j.logN, j.M, j.Nr, j.R, w.y, w.z, nullptr, zre, zim, tw, (T)j.gamma, j.err, so, smem_raw); break;
    }
    __syncthreads();   // the tile's shared memory and s_it are reused by the next item
  }
  if (threadIdx.x == 0) bq_finish(ctr, gridDim.x);
}

template <typename T, bool INV>
__global__ void __launch_bounds__(256) kb_z(const BFftJob* __restrict__ jobs, const int4* __restrict__ items,
                                           int nitems, int* __restrict__ ctr) {
  typedef typename C2T<T>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_it;
  for (;;) {
    if (threadIdx.x == 0) s_it = atomicAdd(ctr, 1);
    __syncthreads();
    const int it = s_it;
    if (it >= nitems) break;
    const int4 w = items[it];
    const BFftJob j = jobs[w.x];
    const SplitOut so = job_split(j);
    T* zre = (T*)j.a;
    T* zim = (T*)j.b;
    T* mre = (T*)j.c;
    T* mim = (T*)j.d;
    const C* tw = (const C*)j.tw;
    switch (j.E) {
      case 1: z_tile<T, INV, 1>(j.N, j.logN, j.Kz, j.K, j.M, j.Nr, j.R, w.y, w.z, zre, zim, mre, mim, tw, so, smem_raw); break;
      case 2: z_tile<T, INV, 2>(j.N, j.logN, j.Kz, j.K, j.M, j.Nr, j.R, w.y, w.z, zre, zim, mre, mim, tw, so, smem_raw); break;
      case 4: z_tile<T, INV, 4>(j.N, j.logN, j.Kz, j.K, j.M, j.Nr, j.R, w.y, w.z, zre, zim, mre, mim, tw, so, smem_raw); break;
      default: z_tile<T, INV, 8>(j.N, j.logN, j.Kz, j.K, j.M, j.Nr, j.R, w.y, w.z, zre, zim, mre, mim, tw, so, smem_raw); break;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) bq_finish(ctr, gridDim.x);
}

int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

// Radii per CTA when not set: the largest tile (32 down to 4) whose grid still
// has `target` CTAs.  These kernels are bound by memory latency at small sizes
// (one short wave), so more, smaller CTAs hide it better: at 128 x 128 x 64 the z
// kernels take 14.3 us with 32 radii per CTA and 10.2 us with 8, the phi kernel
// 15.3 us with 32 and 14.4 us with 16 (fewer radii per CTA lose more to the
// per-CTA staging).  Large grids keep 32.
int auto_tile(int nr, int lines, int target) {
  for (int R = 32; R > 4; R /= 2)
    if ((long long)((nr + R - 1) / R) * lines >= target) return R;
  return 4;
}

constexpr int kSmemLimit = 200 * 1024;

template <typename T, int MODE, int E>
void phi_go(dim3 grid, size_t smem, cudaStream_t st, int N, int M, int Nr, int R, T* phys, T* zre,
            T* zim, const void* tw, double gamma, int* err, const SplitOut& so) {
  typedef typename C2T<T>::type C;
  launch_pdl(k_phi<T, MODE, E>, grid, dim3(256), smem, st, N, ilog2(N), M, Nr, R, phys, zre, zim,
             reinterpret_cast<const C*>(tw), (T)gamma, err, so);
}

template <typename T, int MODE>
void phi_dispatch(int E, dim3 grid, size_t smem, cudaStream_t st, int N, int M, int Nr, int R,
                  T* phys, T* zre, T* zim, const void* tw, double gamma, int* err, const SplitOut& so) {
  switch (E) {
    case 1: phi_go<T, MODE, 1>(grid, smem, st, N, M, Nr, R, phys, zre, zim, tw, gamma, err, so); break;
    case 2: phi_go<T, MODE, 2>(grid, smem, st, N, M, Nr, R, phys, zre, zim, tw, gamma, err, so); break;
    case 4: phi_go<T, MODE, 4>(grid, smem, st, N, M, Nr, R, phys, zre, zim, tw, gamma, err, so); break;
    case 8: phi_go<T, MODE, 8>(grid, smem, st, N, M, Nr, R, phys, zre, zim, tw, gamma, err, so); break;
    default: phi_go<T, MODE, 16>(grid, smem, st, N, M, Nr, R, phys, zre, zim, tw, gamma, err, so); break;
  }
}

// the split-plane output of the BF16X3 context (forward data of the contraction)
SplitOut split_out(mlx_ctx* c) {
  SplitOut so;
  if (c->precision != MLX_BF16X3 || !c->d_bsf) return so;
  so.bs = reinterpret_cast<unsigned short*>(c->d_bsf);
  so.Kp = (int)c->tc_kp;
  so.K2 = 2 * c->K;
  so.part = (long long)c->M * so.K2 * so.Kp;
  return so;
}

template <typename T>
int phi_launch(mlx_ctx* c, int mode, T* phys, T* zbase, const void* tw, double gamma,
               cudaStream_t st, const SplitOut& so = SplitOut()) {
  typedef typename C2T<T>::type C;
  const int N = c->nphi;
  int R = c->phi_tile ? c->phi_tile : auto_tile(c->nr, c->nz, 2 * 148);
  auto need = [&](int R_) { return ((size_t)(R_ / 2) * (N + 1) + N) * sizeof(C); };   // tile + twiddles
  while (need(R) > kSmemLimit && R > 2) R /= 2;
  const size_t smem = need(R);
  dim3 grid((c->nr + R - 1) / R, c->nz);
  const long long pl = (long long)c->nz * c->M * c->nr;
  T* zre = zbase;
  T* zim = zbase + pl;
  const int E = N >= 32 ? N / 32 : 1;
  TimedLaunch tl(c, mode == PHI_FWD ? KID_PHI_FWD : (mode == PHI_BWD ? KID_PHI_BWD : KID_PHI_FKPP), st);
  int* err = c->d_err;
  if (mode == PHI_FWD) phi_dispatch<T, PHI_FWD>(E, grid, smem, st, N, c->M, c->nr, R, phys, zre, zim, tw, gamma, err, so);
  else if (mode == PHI_BWD) phi_dispatch<T, PHI_BWD>(E, grid, smem, st, N, c->M, c->nr, R, phys, zre, zim, tw, gamma, err, so);
  else phi_dispatch<T, PHI_FKPP>(E, grid, smem, st, N, c->M, c->nr, R, phys, zre, zim, tw, gamma, err, so);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

template <typename T, bool INV, int E>
void z_go(dim3 grid, size_t smem, cudaStream_t st, mlx_ctx* c, int R, T* zb, T* mb, const void* tw,
          const SplitOut& so) {
  typedef typename C2T<T>::type C;
  const long long plz = (long long)c->nz * c->M * c->nr;
  const long long plm = (long long)c->K * c->M * c->nr;
  launch_pdl(k_z<T, INV, E>, grid, dim3(256), smem, st, c->nz, ilog2(c->nz), c->Kz, c->K, c->M, c->nr, R, zb,
             zb + plz, mb, mb + plm, reinterpret_cast<const C*>(tw), so);
}

template <typename T, bool INV>
void z_dispatch(int E, dim3 grid, size_t smem, cudaStream_t st, mlx_ctx* c, int R, T* zb, T* mb,
                const void* tw, const SplitOut& so) {
  switch (E) {
    case 1: z_go<T, INV, 1>(grid, smem, st, c, R, zb, mb, tw, so); break;
    case 2: z_go<T, INV, 2>(grid, smem, st, c, R, zb, mb, tw, so); break;
    case 4: z_go<T, INV, 4>(grid, smem, st, c, R, zb, mb, tw, so); break;
    case 8: z_go<T, INV, 8>(grid, smem, st, c, R, zb, mb, tw, so); break;
    default: z_go<T, INV, 16>(grid, smem, st, c, R, zb, mb, tw, so); break;
  }
}

template <typename T>
int z_launch(mlx_ctx* c, bool inverse, T* zbase, T* mbase, const void* tw, cudaStream_t st,
             const SplitOut& so = SplitOut()) {
  typedef typename C2T<T>::type C;
  int R = c->z_tile ? c->z_tile : auto_tile(c->nr, c->M, 4 * 148);
  auto need = [&](int R_) { return ((size_t)R_ * (c->nz + 1) + c->nz) * sizeof(C); };   // tile + twiddles
  while (need(R) > kSmemLimit && R > 1) R /= 2;
  // automatic tiles keep at least 6 CTAs per SM (tiles <= 34 KB): at 256^3 the z
  // kernels take 47.3 / 57.0 us (inverse / forward) with 66 KB tiles of 32 radii
  // and 40.6 / 44.6 us with 16
  if (!c->z_tile)
    while (R > 8 && need(R) > 34 * 1024) R /= 2;
  const size_t smem = need(R);
  dim3 grid((c->nr + R - 1) / R, c->M);
  const int E = c->nz >= 32 ? c->nz / 32 : 1;
  TimedLaunch tl(c, inverse ? KID_Z_BWD : KID_Z_FWD, st);
  if (!inverse) z_dispatch<T, false>(E, grid, smem, st, c, R, zbase, mbase, tw, so);
  else z_dispatch<T, true>(E, grid, smem, st, c, R, zbase, mbase, tw, SplitOut());
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

template <typename T>
int fft_forward_t(mlx_ctx* c, const void* phys, cudaStream_t st, const void* twphi, const void* twz) {
  T* mixed = reinterpret_cast<T*>(c->d_mixed);
  const SplitOut so = split_out(c);
  if (c->nz == 1) return phi_launch<T>(c, PHI_FWD, (T*)phys, mixed, twphi, 0.0, st, so);
  T* zm = reinterpret_cast<T*>(c->d_zm);
  int rc = phi_launch<T>(c, PHI_FWD, (T*)phys, zm, twphi, 0.0, st);
  if (rc) return rc;
  return z_launch<T>(c, false, zm, mixed, twz, st, so);
}

template <typename T>
int fft_backward_t(mlx_ctx* c, void* phys, cudaStream_t st, const void* twphi, const void* twz) {
  T* mixed = reinterpret_cast<T*>(c->d_mixed);
  if (c->nz == 1) return phi_launch<T>(c, PHI_BWD, (T*)phys, mixed, twphi, 0.0, st);
  T* zm = reinterpret_cast<T*>(c->d_zm);
  int rc = z_launch<T>(c, true, zm, mixed, twz, st);
  if (rc) return rc;
  return phi_launch<T>(c, PHI_BWD, (T*)phys, zm, twphi, 0.0, st);
}

template <typename T>
int fft_fkpp_t(mlx_ctx* c, double gamma, cudaStream_t st, const void* twphi, const void* twz) {
  T* mixed = reinterpret_cast<T*>(c->d_mixed);
  const SplitOut so = split_out(c);
  if (c->nz == 1) return phi_launch<T>(c, PHI_FKPP, nullptr, mixed, twphi, gamma, st, so);
  T* zm = reinterpret_cast<T*>(c->d_zm);
  int rc = z_launch<T>(c, true, zm, mixed, twz, st);
  if (rc) return rc;
  rc = phi_launch<T>(c, PHI_FKPP, nullptr, zm, twphi, gamma, st);
  if (rc) return rc;
  return z_launch<T>(c, false, zm, mixed, twz, st, so);
}

template <typename T, int MODE, int E>
int attr_phi(mlx_ctx* c) {
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_phi<T, MODE, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
  return MLX_OK;
}
template <typename T, bool INV, int E>
int attr_z(mlx_ctx* c) {
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_z<T, INV, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
  return MLX_OK;
}
template <typename T, int E>
int attr_all(mlx_ctx* c) {
  int rc = attr_phi<T, PHI_FWD, E>(c);
  if (!rc) rc = attr_phi<T, PHI_BWD, E>(c);
  if (!rc) rc = attr_phi<T, PHI_FKPP, E>(c);
  if (!rc) rc = attr_z<T, false, E>(c);
  if (!rc) rc = attr_z<T, true, E>(c);
  return rc;
}

}  // namespace

const void* mlx_fft_batch_kernel(int stage, bool dbl);

// Opt every FFT kernel into the shared memory the launch helpers may ask for
// (each launch stays below 200 KB).
int mlx_fft_prepare(mlx_ctx* c) {
  int rc = MLX_OK;
  if (!rc) rc = attr_all<float, 1>(c);
  if (!rc) rc = attr_all<float, 2>(c);
  if (!rc) rc = attr_all<float, 4>(c);
  if (!rc) rc = attr_all<float, 8>(c);
  if (!rc) rc = attr_all<float, 16>(c);
  if (!rc) rc = attr_all<double, 1>(c);
  if (!rc) rc = attr_all<double, 2>(c);
  if (!rc) rc = attr_all<double, 4>(c);
  if (!rc) rc = attr_all<double, 8>(c);
  if (!rc) rc = attr_all<double, 16>(c);
  for (int stage = 0; stage < 3 && !rc; ++stage)
    for (int d = 0; d < 2 && !rc; ++d)
      if (cudaFuncSetAttribute(mlx_fft_batch_kernel(stage, d != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSmemLimit) != cudaSuccess) {
        c->last_err = "cudaFuncSetAttribute (batched FFT stage)";
        rc = MLX_ECUDA;
      }
  return rc;
}

int mlx_fft_forward(mlx_ctx* c, const void* phys, cudaStream_t st) {
  if (c->precision == MLX_FP64) return fft_forward_t<double>(c, phys, st, c->d_twphi64, c->d_twz64);
  return fft_forward_t<float>(c, phys, st, c->d_twphi32, c->d_twz32);
}

int mlx_fft_backward(mlx_ctx* c, void* phys, cudaStream_t st) {
  if (c->precision == MLX_FP64) return fft_backward_t<double>(c, phys, st, c->d_twphi64, c->d_twz64);
  return fft_backward_t<float>(c, phys, st, c->d_twphi32, c->d_twz32);
}

int mlx_fft_fkpp(mlx_ctx* c, double gamma, cudaStream_t st) {
  if (c->precision == MLX_FP64) return fft_fkpp_t<double>(c, gamma, st, c->d_twphi64, c->d_twz64);
  return fft_fkpp_t<float>(c, gamma, st, c->d_twphi32, c->d_twz32);
}

// ---- batched persistent Fisher-KPP stages (batch.cu) ----
// Job and work items of member c (index inst) for one stage of the fused
// Fisher-KPP transform sequence: stage 0 the inverse z transform (mixed -> zm),
// 1 the phi synthesis / product / analysis, 2 the forward z transform (zm ->
// mixed or the split planes).  Stages 0 and 2 exist for Nz > 1 only (returns
// false otherwise).  cost[i]: relative work of items[i]; *smem: the shared memory
// one of its CTAs needs.  The tiles are the member's own (its phi_tile / z_tile).
bool mlx_fft_batch_member(mlx_ctx* c, int stage, double gamma, int inst, BFftJob* job,
                          std::vector<int4>& items, std::vector<double>& cost, size_t* smem) {
  const bool dbl = c->precision == MLX_FP64;
  const size_t es = dbl ? 8 : 4, cs = 2 * es;
  if ((stage == 0 || stage == 2) && c->nz == 1) return false;
  BFftJob j;
  memset(&j, 0, sizeof(j));
  j.M = c->M;
  j.Nr = c->nr;
  j.Kz = c->Kz;
  j.K = c->K;
  j.gamma = gamma;
  j.err = c->d_err;
  char* mixed = (char*)c->d_mixed;
  const long long plm = (long long)c->K * c->M * c->nr;
  const SplitOut so = split_out(c);
  if (stage == 1) {
    const int N = c->nphi;
    int R = c->phi_tile ? c->phi_tile : auto_tile(c->nr, c->nz, 2 * 148);
    auto need = [&](int R_) { return ((size_t)(R_ / 2) * (N + 1) + N) * cs; };
    while (need(R) > kSmemLimit && R > 2) R /= 2;
    *smem = need(R);
    j.N = N; j.logN = ilog2(N); j.R = R; j.E = N >= 32 ? N / 32 : 1;
    j.tw = dbl ? (const void*)c->d_twphi64 : (const void*)c->d_twphi32;
    if (c->nz == 1) {
      j.b = mixed; j.c = mixed + plm * es;
      if (so.bs) { j.bs = so.bs; j.part = so.part; j.kp = so.Kp; j.k2 = so.K2; }
    } else {
      const long long pl = (long long)c->nz * c->M * c->nr;
      j.b = c->d_zm; j.c = (char*)c->d_zm + pl * es;
    }
    const double w = (double)N * (j.logN + 2) * R;
    for (int z = 0; z < c->nz; ++z)
      for (int bx = 0; bx < (c->nr + R - 1) / R; ++bx) { items.push_back(make_int4(inst, bx, z, 0)); cost.push_back(w); }
  } else {
    const int N = c->nz;
    int R = c->z_tile ? c->z_tile : auto_tile(c->nr, c->M, 4 * 148);
    auto need = [&](int R_) { return ((size_t)R_ * (N + 1) + N) * cs; };
    while (need(R) > kSmemLimit && R > 1) R /= 2;
    if (!c->z_tile)
      while (R > 8 && need(R) > 34 * 1024) R /= 2;
    *smem = need(R);
    j.N = N; j.logN = ilog2(N); j.R = R; j.E = N >= 32 ? N / 32 : 1;
    j.tw = dbl ? (const void*)c->d_twz64 : (const void*)c->d_twz32;
    const long long plz = (long long)c->nz * c->M * c->nr;
    j.a = c->d_zm; j.b = (char*)c->d_zm + plz * es;
    j.c = mixed; j.d = mixed + plm * es;
    if (stage == 2 && so.bs) { j.bs = so.bs; j.part = so.part; j.kp = so.Kp; j.k2 = so.K2; }
    const double w = (double)N * (j.logN + 2) * R;
    for (int m = 0; m < c->M; ++m)
      for (int bx = 0; bx < (c->nr + R - 1) / R; ++bx) { items.push_back(make_int4(inst, bx, m, 0)); cost.push_back(w); }
  }
  *job = j;
  return true;
}

// The kernel of a batched stage launch (stage as above, dbl: FP64 members).
const void* mlx_fft_batch_kernel(int stage, bool dbl) {
  if (dbl) {
    if (stage == 0) return (const void*)kb_z<double, true>;
    if (stage == 1) return (const void*)kb_phi_fkpp<double>;
    return (const void*)kb_z<double, false>;
  }
  if (stage == 0) return (const void*)kb_z<float, true>;
  if (stage == 1) return (const void*)kb_phi_fkpp<float>;
  return (const void*)kb_z<float, false>;
}

int mlx_fft_batch_launch(int stage, bool dbl, const BFftJob* jobs, const int4* items, int nitems, int* ctr,
                         size_t smem, int grid, cudaStream_t st) {
  if (dbl) {
    if (stage == 0) kb_z<double, true><<<grid, 256, smem, st>>>(jobs, items, nitems, ctr);
    else if (stage == 1) kb_phi_fkpp<double><<<grid, 256, smem, st>>>(jobs, items, nitems, ctr);
    else kb_z<double, false><<<grid, 256, smem, st>>>(jobs, items, nitems, ctr);
  } else {
    if (stage == 0) kb_z<float, true><<<grid, 256, smem, st>>>(jobs, items, nitems, ctr);
    else if (stage == 1) kb_phi_fkpp<float><<<grid, 256, smem, st>>>(jobs, items, nitems, ctr);
    else kb_z<float, false><<<grid, 256, smem, st>>>(jobs, items, nitems, ctr);
  }
  return cudaGetLastError() == cudaSuccess ? MLX_OK : MLX_ECUDA;
}
