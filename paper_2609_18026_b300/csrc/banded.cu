// K6: FP64 banded implicit radial solves per harmonic (m, k) (Sec. 3.1, Sec. 3.3).
//
// Operator of Eq. (11) on harmonic (m, k), kappa = 2 pi |k| / Lz:
//   L = nu (D_m - kappa^2 I) - nu_h (-(D_m - kappa^2 I))^{p/2}
// with D_m the pentadiagonal Laplacian band (half width 2).  The power is a
// product of truncated band matrices (half width grows by 2 per factor, p in
// total).  Every matrix depends on (m, |k|) only, so one set of factors serves
// the wavenumbers k and -k.
//
// Storage per (m, |k|) system of size N = Nc - m, rows i = 0..N-1:
//   Bplus [N][2kl+1]  band of I + dt/2 L (column i + o at slot o + kl), kept
//                     for reference and tests; the solve does not read it
//   LU of I - c L, c = dt/2 (half) and dt (full), partial pivoting over the kl
//   rows below the diagonal: U row i holds U_ii then columns i+1..i+2kl divided
//   by U_ii (slot t = column - i), L multipliers [N][kl], pivot rows, 1/U_ii.
// One thread per system factorises.  The solve variants (staged, segmented, lean)
// are described at their kernels; all use these FP64 factors.
#include "mlx_internal.cuh"
#include "df.cuh"
#include "bf16_split.cuh"

#include <string.h>

#include <algorithm>
#include <type_traits>

namespace {

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_s(unsigned sa, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8_s(unsigned sa, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Right-hand sides of the implicit steps in one explicit rounding order, so that
// every solve variant forms bit-identical values: AB-CN 2 s + (3/2) dt A -
// (1/2) dt A_prev, FE-BE s + h A.  The recurrences below likewise spell out each
// fused multiply-add and each product (__fma_rn, __dmul_rn): a product feeding a
// later subtraction could otherwise be fused either way, and the choice would
// differ between kernels of different shape.
// 2 v exactly: for normal v with a finite double, an exponent increment (integer
// pipe); zero, subnormal, overflowing, infinite and NaN inputs take the FP64 product
__device__ __forceinline__ double twice(double v) {
  const long long b = __double_as_longlong(v);
  const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
  if (e - 1u < 2045u) return __longlong_as_double(b + (1LL << 52));
  if (((unsigned long long)b << 1) == 0) return v;
  return __dmul_rn(2.0, v);
}
__device__ __forceinline__ double rhs_abcn(double sv, double a, double ap, bool hasA, bool hasAp, double dt) {
  double r = twice(sv);
  if (hasA) r = __fma_rn(1.5 * dt, a, r);
  if (hasAp) r = __fma_rn(-0.5 * dt, ap, r);
  return r;
}
__device__ __forceinline__ double rhs_febe(double sv, double a, bool hasA, double h) {
  return hasA ? __fma_rn(h, a, sv) : sv;
}

// Copy nrows rows of row_bytes bytes (a multiple of 4) from global memory (row stride
// src_stride bytes) to shared memory (row stride dst_stride bytes) with cp.async,
// in 16-byte pieces when every address, stride and length allows, else 8 or 4.
// Each lane owns one piece position and walks the rows with fixed strides (one
// division per call, none per piece).
template <int CH>
__device__ __forceinline__ void stage_rows_ch(unsigned char* d0, int dst_stride, const unsigned char* s0,
                                              long long src_stride, int nrows, int per_row, int lane) {
  if (per_row <= 32) {
    const int rpp = 32 / per_row;                      // rows per pass of the warp
    const int r0 = lane / per_row, j = lane - r0 * per_row;
    if (r0 >= rpp) return;
    unsigned char* d = d0 + (size_t)r0 * dst_stride + (size_t)j * CH;
    const unsigned char* g = s0 + (long long)r0 * src_stride + (long long)j * CH;
    const size_t dstep = (size_t)rpp * dst_stride;
    const long long gstep = (long long)rpp * src_stride;
    for (int i = r0; i < nrows; i += rpp, d += dstep, g += gstep) {
      if (CH == 16) cp_async16(d, g);
      else if (CH == 8) cp_async8(d, g);
      else cp_async4(d, g);
    }
  } else {
    for (int e = lane; e < nrows * per_row; e += 32) {
      const int i = e / per_row, j = e - i * per_row;
      unsigned char* d = d0 + (size_t)i * dst_stride + (size_t)j * CH;
      const unsigned char* g = s0 + (long long)i * src_stride + (long long)j * CH;
      if (CH == 16) cp_async16(d, g);
      else if (CH == 8) cp_async8(d, g);
      else cp_async4(d, g);
    }
  }
}
__device__ __forceinline__ void stage_rows(void* dst, int dst_stride, const void* src, long long src_stride,
                                           int nrows, int row_bytes, int lane) {
  const unsigned long long a = (unsigned long long)(uintptr_t)src | (unsigned long long)src_stride |
                               (unsigned long long)row_bytes | (unsigned long long)dst_stride |
                               (unsigned long long)__cvta_generic_to_shared(dst);
  unsigned char* d0 = reinterpret_cast<unsigned char*>(dst);
  const unsigned char* s0 = reinterpret_cast<const unsigned char*>(src);
  if ((a & 15) == 0) stage_rows_ch<16>(d0, dst_stride, s0, src_stride, nrows, row_bytes / 16, lane);
  else if ((a & 7) == 0) stage_rows_ch<8>(d0, dst_stride, s0, src_stride, nrows, row_bytes / 8, lane);
  else stage_rows_ch<4>(d0, dst_stride, s0, src_stride, nrows, row_bytes / 4, lane);
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Factor rows of one m are interleaved by |k|: row (m, i, kabs) has index
// band_off[m] + i * Kz + kabs, so the threads of a warp (consecutive k) read
// neighbouring rows.
__device__ __forceinline__ void sys_of(int idx, int M, int nc, int Kz, const long long* band_off,
                                       int& m, int& kabs, long long& row0) {
  // idx enumerates (m, kabs) m-major
  m = idx / Kz;
  kabs = idx % Kz;
  row0 = band_off[m] + kabs;
}

// Build the band of L (half width kl) for system (m, kabs) into Lb[N][2kl+1]
// using two scratch buffers of the same shape.
__device__ void build_L(int m, int N, double kappa2, double nu, double nu_h, int p, int kl,
                        const double* __restrict__ lap_m, double* Lb, double* Q, double* T1) {
  const int W = 2 * kl + 1;
  for (long long t = 0; t < (long long)N * W; ++t) { Lb[t] = 0.0; Q[t] = 0.0; }
  // -(D - kappa^2) into Q (half width 2), nu (D - kappa^2) into Lb
  for (int i = 0; i < N; ++i) {
    for (int o = -2; o <= 2; ++o) {
      const int j = i + o;
      if (j < 0 || j >= N) continue;
      double d = lap_m[i * 5 + (o + 2)];
      if (o == 0) d -= kappa2;
      Lb[i * W + o + kl] = nu * d;
      Q[i * W + o + kl] = -d;
    }
  }
  if (nu_h == 0.0) return;
  // T1 = Q^{p/2}: start with Q, multiply by Q (half width 2) p/2 - 1 times
  for (long long t = 0; t < (long long)N * W; ++t) T1[t] = Q[t];
  int hw = 2;
  for (int f = 1; f < p / 2; ++f) {
    // T1 <- T1 * Q ; result half width hw + 2, written row by row via Lb's
    // slack: use a small per-row temporary of width W
    for (int i = 0; i < N; ++i) {
      double rowtmp[2 * 16 + 1];
      for (int o = 0; o < W; ++o) rowtmp[o] = 0.0;
      for (int a = -hw; a <= hw; ++a) {
        const int k = i + a;
        if (k < 0 || k >= N) continue;
        const double tv = T1[i * W + a + kl];
        if (tv == 0.0) continue;
        for (int b = -2; b <= 2; ++b) {
          const int j = k + b;
          if (j < 0 || j >= N) continue;
          rowtmp[j - i + kl] += tv * Q[k * W + b + kl];
        }
      }
      // row i of the product only depends on rows of Q, not on T1 rows other
      // than i, so it can overwrite T1 row i in place
      for (int o = 0; o < W; ++o) T1[i * W + o] = rowtmp[o];
    }
    hw += 2;
  }
  for (long long t = 0; t < (long long)N * W; ++t) Lb[t] -= nu_h * T1[t];
}

// Banded LU with partial pivoting of A = alpha I + beta Lb.  work: [N][3kl+1] row
// windows (column j of row i at slot j - i + kl).  Factor row i is stored at row
// index i * rs of U / Lm / piv / invd (rs = Kz: systems of one m are interleaved by
// |k|; rs = 1 for the kappa-independent Laplacian factors).
__device__ void band_lu(int N, int kl, double alpha, double beta, const double* Lb, double* work,
                        double* U, double* Lm, int* piv, double* invd, int rs) {
  const int W = 2 * kl + 1;     // band of L
  const int WW = 3 * kl + 1;    // window: columns i-kl .. i+2kl
  for (long long t = 0; t < (long long)N * WW; ++t) work[t] = 0.0;
  for (int i = 0; i < N; ++i)
    for (int o = -kl; o <= kl; ++o) {
      const int j = i + o;
      if (j < 0 || j >= N) continue;
      double v = beta * Lb[i * W + o + kl];
      if (o == 0) v += alpha;
      work[i * WW + o + kl] = v;
    }
  for (int j = 0; j < N; ++j) {
    const int last = min(N - 1, j + kl);
    int pr = j;
    double best = fabs(work[j * WW + kl]);
    for (int i = j + 1; i <= last; ++i) {
      const double v = fabs(work[i * WW + (j - i) + kl]);
      if (v > best) { best = v; pr = i; }
    }
    piv[(long long)j * rs] = pr;
    const int cend = min(N - 1, j + 2 * kl);
    if (pr != j) {
      for (int cc = j; cc <= cend; ++cc) {
        double* a = &work[j * WW + (cc - j) + kl];
        double* b = &work[pr * WW + (cc - pr) + kl];
        const double t = *a; *a = *b; *b = t;
      }
    }
    const double d = work[j * WW + kl];
    const double inv = 1.0 / d;
    for (int i = j + 1; i <= last; ++i) {
      const double l = work[i * WW + (j - i) + kl] * inv;
      Lm[(long long)j * rs * kl + (i - j - 1)] = l;
      work[i * WW + (j - i) + kl] = 0.0;
      for (int cc = j + 1; cc <= cend; ++cc) work[i * WW + (cc - i) + kl] -= l * work[j * WW + (cc - j) + kl];
    }
    for (int i = last + 1; i <= j + kl; ++i) Lm[(long long)j * rs * kl + (i - j - 1)] = 0.0;
  }
  // U row i is stored as (U_ii, U_i,i+1 / U_ii, ..., U_i,i+2kl / U_ii) so that the
  // back substitution is x_i = y_i / U_ii - sum_t (U_i,i+t / U_ii) x_{i+t}
  for (int i = 0; i < N; ++i) {
    double* Ui = U + (long long)i * rs * (2 * kl + 1);
    const double dinv = 1.0 / work[i * WW + kl];
    Ui[0] = work[i * WW + kl];
    for (int t = 1; t <= 2 * kl; ++t) {
      const int cc = i + t;
      Ui[t] = (cc < N) ? work[i * WW + t + kl] * dinv : 0.0;
    }
    invd[(long long)i * rs] = dinv;
  }
}

__global__ void k_band_setup(int M, int nc, int Kz, double lz, const long long* __restrict__ band_off,
                             const long long* __restrict__ lap_rows, const double* __restrict__ lap,
                             double nu, double nu_h, int p, double dt, int kl,
                             double* __restrict__ Bplus,
                             double* __restrict__ Uh, double* __restrict__ Lh, int* __restrict__ Ph, double* __restrict__ Dh,
                             double* __restrict__ Uf, double* __restrict__ Lf, int* __restrict__ Pf, double* __restrict__ Df,
                             double* __restrict__ scratch, long long scratch_stride) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * Kz) return;
  int m, kabs;
  long long row0;
  sys_of(idx, M, nc, Kz, band_off, m, kabs, row0);
  const int N = nc - m;
  const double kappa = 2.0 * M_PI * kabs / lz;
  const int W = 2 * kl + 1;
  double* Lb = scratch + (long long)idx * scratch_stride;
  double* Q = Lb + (long long)N * W;
  double* T1 = Q + (long long)N * W;
  double* work = T1 + (long long)N * W;
  build_L(m, N, kappa * kappa, nu, nu_h, p, kl, lap + lap_rows[m] * 5, Lb, Q, T1);
  for (int i = 0; i < N; ++i)
    for (int o = 0; o < W; ++o) {
      double v = 0.5 * dt * Lb[i * W + o];
      if (o == kl) v += 1.0;
      Bplus[(row0 + (long long)i * Kz) * W + o] = v;
    }
  band_lu(N, kl, 1.0, -0.5 * dt, Lb, work, Uh + row0 * W, Lh + row0 * kl, Ph + row0, Dh + row0, Kz);
  band_lu(N, kl, 1.0, -dt, Lb, work, Uf + row0 * W, Lf + row0 * kl, Pf + row0, Df + row0, Kz);
}

// Factors of the horizontal Laplacian D_m (family "lap", one system per m) and of
// the Helmholtz operator D_m - kappa^2 (family "helm", per (m, |k|)), both with
// half bandwidth 2.  At m = 0 the Laplacian is singular (its column 0 vanishes:
// the constant has zero Laplacian); its system drops row and column 0 and the
// solve recovers x_0 from the far-field decay condition.
__global__ void k_lap_setup(int M, int nc, int Kz, double lz, int helm, const long long* __restrict__ fac_off,
                            const long long* __restrict__ lap_rows, const double* __restrict__ lap,
                            double* __restrict__ U, double* __restrict__ Lm, int* __restrict__ piv,
                            double* __restrict__ invd, double* __restrict__ scratch, long long stride) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int per_m = helm ? Kz : 1;
  if (idx >= M * per_m) return;
  const int m = idx / per_m, kabs = idx % per_m;
  const int shift = (!helm && m == 0) ? 1 : 0;
  const int N = nc - m - shift;
  const int kl = 2, W = 5;
  double* Lb = scratch + (long long)idx * stride;
  double* work = Lb + (long long)nc * W;
  const double* lm = lap + (lap_rows[m] + shift) * 5;
  for (int i = 0; i < N; ++i)
    for (int o = 0; o < W; ++o) {
      const int j = i + o - kl;
      Lb[i * W + o] = (j >= 0 && j < N) ? lm[i * 5 + o] : 0.0;
    }
  const double kappa = 2.0 * M_PI * kabs / lz;
  const int rs = helm ? Kz : 1;
  const long long row0 = fac_off[m] + (helm ? kabs : 0);
  band_lu(N, kl, helm ? -kappa * kappa : 0.0, 1.0, Lb, work, U + row0 * W, Lm + row0 * kl, piv + row0,
          invd + row0, rs);
}

// Projection operators of the vortex term on order-m coefficients, with
// J = multiplication by x (J_{i,i+1} = J_{i+1,i} = e_i = a_{m+i+1},
// a_n = sqrt((n^2 - m^2)/(4 n^2 - 1))) and d_i = -n(n+1):
//   family 0: Q = (I - J^2) diag(d)            = r^2 lap_h        (per m, decay row at m = 0)
//   family 1: H = (I - J) Q                    = (1 - x) r^2 lap_h (per m, decay row at m = 0)
//   family 2: G = H - kappa^2 ell^2 (I + J)                        (per (m, |k|), |k| >= 1)
// built as half-bandwidth-3 bands and factorised with partial pivoting.
__device__ __forceinline__ double jac_e(int m, int i) {
  const double n = (double)(m + i + 1), mm = (double)m;
  return sqrt((n * n - mm * mm) / (4.0 * n * n - 1.0));
}

__global__ void k_proj_setup(int M, int nc, int Kz, double lz, double ell, int family,
                             const long long* __restrict__ fac_off, double* __restrict__ U,
                             double* __restrict__ Lm, int* __restrict__ piv, double* __restrict__ invd,
                             double* __restrict__ scratch, long long stride) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int per_m = (family == 2) ? Kz : 1;
  if (idx >= M * per_m) return;
  const int m = idx / per_m, kabs = idx % per_m;
  const int Nf = nc - m;                       // full system size
  const int shift = (family < 2 && m == 0) ? 1 : 0;
  const int N = Nf - shift;
  constexpr int kl = 3, W = 7;
  double* Qb = scratch + (long long)idx * stride;   // [Nf][W] full-size bands
  double* Hb = Qb + (long long)Nf * W;
  double* work = Hb + (long long)Nf * W;            // [Nf][3 kl + 1]
  for (long long t = 0; t < (long long)Nf * W; ++t) { Qb[t] = 0.0; Hb[t] = 0.0; }
  auto e = [&](int i) -> double { return (i >= 0 && i + 1 < Nf) ? jac_e(m, i) : 0.0; };
  auto d = [&](int j) -> double { const double n = (double)(m + j); return -n * (n + 1.0); };
  // Q[i][j] = (delta_ij - (J^2)_ij) d_j
  for (int i = 0; i < Nf; ++i) {
    const double j2d = e(i - 1) * e(i - 1) + e(i) * e(i);
    Qb[i * W + kl] = (1.0 - j2d) * d(i);
    if (i + 2 < Nf) Qb[i * W + kl + 2] = -e(i) * e(i + 1) * d(i + 2);
    if (i - 2 >= 0) Qb[i * W + kl - 2] = -e(i - 1) * e(i - 2) * d(i - 2);
  }
  if (family >= 1) {
    // H[i][j] = Q[i][j] - e_{i-1} Q[i-1][j] - e_i Q[i+1][j]
    for (int i = 0; i < Nf; ++i)
      for (int o = -kl; o <= kl; ++o) {
        const int j = i + o;
        if (j < 0 || j >= Nf) continue;
        double v = (o >= -2 && o <= 2) ? Qb[i * W + kl + o] : 0.0;
        if (i - 1 >= 0) { const int oo = j - (i - 1); if (oo >= -2 && oo <= 2) v -= e(i - 1) * Qb[(i - 1) * W + kl + oo]; }
        if (i + 1 < Nf) { const int oo = j - (i + 1); if (oo >= -2 && oo <= 2) v -= e(i) * Qb[(i + 1) * W + kl + oo]; }
        Hb[i * W + kl + o] = v;
      }
  }
  double* src = (family == 0) ? Qb : Hb;
  if (family == 2) {
    const double kappa = 2.0 * M_PI * kabs / lz;
    const double c = kappa * kappa * ell * ell;
    for (int i = 0; i < Nf; ++i) {
      src[i * W + kl] -= c;
      if (i + 1 < Nf) src[i * W + kl + 1] -= c * e(i);
      if (i - 1 >= 0) src[i * W + kl - 1] -= c * e(i - 1);
    }
    if (kabs == 0) {   // unused slot: keep it well defined (identity)
      for (long long t = 0; t < (long long)Nf * W; ++t) src[t] = 0.0;
      for (int i = 0; i < Nf; ++i) src[i * W + kl] = 1.0;
    }
  }
  // drop row and column 0 at m = 0 for the decay-row families (column 0 is zero
  // there): the band rows start one row later and band_lu skips entries that
  // would reach column -1
  const double* band = src + (long long)shift * W;
  const int rs = (family == 2) ? Kz : 1;
  const long long row0 = fac_off[m] + ((family == 2) ? kabs : 0);
  band_lu(N, kl, 0.0, 1.0, band, work, U + row0 * W, Lm + row0 * kl, piv + row0, invd + row0, rs);
}

// Solve kernel.  The substitution is a sequential recurrence in the row index, and
// on this GPU FP64 throughput per SM sub-partition is the limit, so the work is
// spread as widely as possible: every real chain (one of Re / Im of one system)
// is one lane, a warp owns CPW chains = CPW/4 values of |k| for one m (the four
// chains +|k| Re/Im, -|k| Re/Im share one set of real factors), and each warp
// stages its factors and right-hand sides in its own shared-memory slab, so warps
// never wait on one another.  For AB-CN the right-hand side uses the identity
//   (I - c L)^{-1} ((I + c L) s + r) = (I - c L)^{-1} (2 s + r) - s,   c = dt/2,
// which needs no band product: rhs = 2 s + dt/2 (3 A - A_prev), and s is
// subtracted after the back substitution.
template <int KL>
struct SolveSmem {
  static constexpr int W = 2 * KL + 1;
  // per |k| and row: U (W), L (KL), 1/diag (1) doubles + pivot row (int)
  // keep_s: the AB-CN "- s" term is read from a shared-memory copy of s made while
  // staging (saves a global re-read at the end, costs N CPW doubles per warp)
  __host__ __device__ static size_t per_warp(int nc, int CPW, int keep_s) {
    const int G = CPW / 4;
    const size_t b = (size_t)nc * G * (W + KL + 1) * sizeof(double) +
                     (size_t)(keep_s ? 2 : 1) * nc * CPW * sizeof(double) + (size_t)nc * G * sizeof(int);
    return (b + 15) / 16 * 16;   // keeps every warp's slab 16-byte aligned
  }
};

// The work of one warp: systems (m, |k| = k0 .. k0 + G - 1), gw = m groups_per_m
// + group; base: the warp's shared-memory slab.
template <int KL>
__device__ __forceinline__ void band_solve_warp(int gw, unsigned char* __restrict__ base, int M, int nc, int Kz,
                                                int K, int CPW, int groups_per_m, int step, int keep_s,
                                                double dt, const long long* __restrict__ soff,
                                                const long long* __restrict__ band_off, int kz_fac, int m0_shift,
                                                const double* __restrict__ U,
                                                const double* __restrict__ Lm, const int* __restrict__ piv,
                                                const double* __restrict__ invd, const double* __restrict__ s,
                                                const double* __restrict__ A, const double* __restrict__ Ap,
                                                double* __restrict__ out, double* __restrict__ Az = nullptr) {
  constexpr int W = 2 * KL + 1;
  const int lane = threadIdx.x & 31;
  if (gw >= M * groups_per_m) return;
  const int m = gw / groups_per_m;
  const int G = CPW / 4;
  const int k0 = (gw % groups_per_m) * G;
  const int gcnt = min(G, Kz - k0);
  const int sh = (m == 0) ? m0_shift : 0;   // Laplacian at m = 0: unknowns n >= 1
  const int Nm = nc - m;
  const int N = Nm - sh;
  double* Us = reinterpret_cast<double*>(base);              // [N][G][W]
  double* Ls = Us + (size_t)N * G * W;                       // [N][G][KL]
  double* Ds = Ls + (size_t)N * G * KL;                      // [N][G]
  double* Y = Ds + (size_t)N * G;                            // [N][CPW]
  double* S = Y + (size_t)N * CPW;                           // [N][CPW] s, for the AB-CN "- s" (keep_s)
  int* Pi = reinterpret_cast<int*>(S + (keep_s ? (size_t)N * CPW : 0));   // [N][G] pivot rows
  const long long fb = band_off[m];
  const long long sm = soff[m];
  // stage factors with asynchronous copies: the rows of the warp's gcnt values of
  // |k| are contiguous for every i (interleaved storage), so each i is one span
  if (kz_fac != 1) {
    const long long r0 = fb + k0;
    stage_rows(Us, G * W * 8, U + r0 * W, (long long)kz_fac * W * 8, N, gcnt * W * 8, lane);
    stage_rows(Ls, G * KL * 8, Lm + r0 * KL, (long long)kz_fac * KL * 8, N, gcnt * KL * 8, lane);
    stage_rows(Ds, G * 8, invd + r0, (long long)kz_fac * 8, N, gcnt * 8, lane);
    stage_rows(Pi, G * 4, piv + r0, (long long)kz_fac * 4, N, gcnt * 4, lane);
  } else {
    // one factor set per m, shared by every |k|: replicated into each slot
    for (int kq = 0; kq < gcnt; ++kq) {
      stage_rows(Us + kq * W, G * W * 8, U + fb * W, (long long)W * 8, N, W * 8, lane);
      stage_rows(Ls + kq * KL, G * KL * 8, Lm + fb * KL, (long long)KL * 8, N, KL * 8, lane);
      stage_rows(Ds + kq, G * 8, invd + fb, 8, N, 8, lane);
      stage_rows(Pi + kq, G * 4, piv + fb, 4, N, 4, lane);
    }
  }
  cp_async_commit();
  // stage right-hand sides, one complex value per step (chain c = kk * 4 + sgn * 2 + part)
  const double h = (step == MLX_STEP_FEBE_FULL) ? dt : 0.5 * dt;
  const double2* s2 = reinterpret_cast<const double2*>(s);
  const double2* A2 = reinterpret_cast<const double2*>(A);
  const double2* Ap2 = reinterpret_cast<const double2*>(Ap);
  // lane -> complex piece cp = lane / LP (cp = kq * 2 + sg) and rows lane % LP + LP t
  const int LP = 16 / G;
  const int cpl = lane / LP, il = lane - cpl * LP;
  const int kql = cpl >> 1, sgl = cpl & 1, kabsl = k0 + kql;
  const bool lane_piece = cpl < 2 * gcnt && !(sgl && kabsl == 0);
  const long long pbase = sm + (long long)(sgl ? K - kabsl : kabsl) * Nm + sh;
  // RB rows per lane per batch: their loads are all in flight before any is used
  constexpr int RB = 8;
  for (int i = il; i < (lane_piece ? N : 0); i += RB * LP) {
    double2 sv[RB], av[RB], apv[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int ii = i + u * LP;
      const bool in = ii < N;
      const long long o = pbase + (in ? ii : i);
      sv[u] = s2[o];
      av[u] = (step != MLX_STEP_PLAIN && A) ? A2[o] : make_double2(0.0, 0.0);
      apv[u] = (step == MLX_STEP_ABCN && Ap) ? Ap2[o] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int ii = i + u * LP;
      if (ii >= N) break;
      double2 r;
      if (step == MLX_STEP_PLAIN) {
        r = sv[u];
      } else if (step == MLX_STEP_ABCN) {
        r = make_double2(rhs_abcn(sv[u].x, av[u].x, apv[u].x, A, Ap, dt),
                         rhs_abcn(sv[u].y, av[u].y, apv[u].y, A, Ap, dt));
        if (keep_s) {
          S[(size_t)ii * CPW + cpl * 2] = sv[u].x;
          S[(size_t)ii * CPW + cpl * 2 + 1] = sv[u].y;
        }
      } else {
        r = sv[u];
        if (A) r = make_double2(rhs_febe(sv[u].x, av[u].x, true, h), rhs_febe(sv[u].y, av[u].y, true, h));
      }
      Y[(size_t)ii * CPW + cpl * 2] = r.x;
      Y[(size_t)ii * CPW + cpl * 2 + 1] = r.y;
    }
  }
  cp_async_wait_all();
  __syncwarp();

  const int c = lane;
  const int kk = c >> 2, sgn = (c >> 1) & 1, part = c & 1;
  const bool valid = c < 4 * gcnt && !(sgn && k0 + kk == 0);
  if (c < 4 * gcnt) {
    double* y = Y + c;
    // forward elimination, rows j..j+KL of the chain in registers
    double w[KL + 1];
#pragma unroll
    for (int q = 0; q < KL; ++q) w[q + 1] = (q < N) ? y[(size_t)q * CPW] : 0.0;
#pragma unroll 2
    for (int j = 0; j < N; ++j) {
#pragma unroll
      for (int q = 0; q < KL; ++q) w[q] = w[q + 1];
      w[KL] = (j + KL < N) ? y[(size_t)(j + KL) * CPW] : 0.0;
      const int d = Pi[(size_t)j * G + kk] - j;
#pragma unroll
      for (int q = 1; q <= KL; ++q)
        if (q == d) { const double t = w[0]; w[0] = w[q]; w[q] = t; }
      y[(size_t)j * CPW] = w[0];
      const double* l = Ls + ((size_t)j * G + kk) * KL;
#pragma unroll
      for (int q = 1; q <= KL; ++q) w[q] = __fma_rn(-l[q - 1], w[0], w[q]);
    }
  }
  __syncwarp();
  // y_r / U_rr for every row and chain with all lanes busy (an FP64 instruction
  // costs the pipe as much with 8 active lanes as with 32): the back substitution
  // takes these products as they are, the same rounded values it would form
  for (int i = il; i < (lane_piece ? N : 0); i += LP) {
    const double dv = Ds[(size_t)i * G + kql];
    Y[(size_t)i * CPW + cpl * 2] = __dmul_rn(Y[(size_t)i * CPW + cpl * 2], dv);
    Y[(size_t)i * CPW + cpl * 2 + 1] = __dmul_rn(Y[(size_t)i * CPW + cpl * 2 + 1], dv);
  }
  __syncwarp();
  if (c < 4 * gcnt) {
    double* y = Y + c;
    // back substitution x_r = y_r / U_rr - sum_{q=1..2KL} (U_r,r+q / U_rr) x_{r+q},
    // software-pipelined: acc[t] is the partial sum of row i - t, and at step i
    // every pending row takes its term with x_{i+1} (row r the term q = i + 1 - r).
    // The 2KL multiply-adds of a step are independent of one another; only x_i
    // waits for x_{i+1}.  Each row still adds its terms from q = 2KL down to 1.
    double acc[2 * KL];
#pragma unroll
    for (int t = 0; t < 2 * KL; ++t) {
      const int r = N - 1 - t;
      acc[t] = (r >= 0) ? y[(size_t)r * CPW] : 0.0;
    }
    double xn = 0.0;   // x_{i+1}
#pragma unroll 2
    for (int i = N - 1; i >= 0; --i) {
      const double xi = __fma_rn(-Us[((size_t)i * G + kk) * W + 1], xn, acc[0]);
#pragma unroll
      for (int t = 1; t < 2 * KL; ++t)
        if (i - t >= 0) acc[t] = __fma_rn(-Us[((size_t)(i - t) * G + kk) * W + t + 1], xn, acc[t]);
      y[(size_t)i * CPW] = xi;
#pragma unroll
      for (int t = 0; t < 2 * KL - 1; ++t) acc[t] = acc[t + 1];
      const int rn = i - 2 * KL;
      acc[2 * KL - 1] = (rn >= 0) ? y[(size_t)rn * CPW] : 0.0;
      xn = xi;
    }
  }
  __syncwarp();
  (void)valid;
  if (sh) {
    // x_0 from the decay condition sum_n Pbar_n^0(1) x_n = 0, Pbar_n^0(1) = sqrt((2n+1)/2)
    if (c < 4 * gcnt && valid) {
      double acc = 0.0;
      for (int i = 0; i < N; ++i) acc = __fma_rn(sqrt((2.0 * (i + 1) + 1.0) * 0.5), Y[(size_t)i * CPW + c], acc);
      const int kabs = k0 + kk;
      const int kidx = sgn ? K - kabs : kabs;
      out[2 * (sm + (long long)kidx * Nm) + part] = -acc / sqrt(0.5);
    }
  }
  double2* out2 = reinterpret_cast<double2*>(out);
#pragma unroll 4
  for (int i = il; i < (lane_piece ? N : 0); i += LP) {
    const int cp = cpl;
    double2 v = make_double2(Y[(size_t)i * CPW + cp * 2], Y[(size_t)i * CPW + cp * 2 + 1]);
    if (step == MLX_STEP_ABCN) {
      if (keep_s) {
        v.x -= S[(size_t)i * CPW + cp * 2];
        v.y -= S[(size_t)i * CPW + cp * 2 + 1];
      } else {
        const double2 sv = s2[pbase + i];
        v.x -= sv.x;
        v.y -= sv.y;
      }
    }
    out2[pbase + i] = v;
    // a batched member without a nonlinear term: its A^j (zero) written where
    // the single-context step clears it
    if (Az) reinterpret_cast<double2*>(Az)[pbase + i] = make_double2(0.0, 0.0);
  }
}

// gw0: the first warp task (m gw0 / groups_per_m onwards; 0 for a whole family)
template <int KL>
__global__ void k_band_solve(int M, int nc, int Kz, int K, int CPW, int groups_per_m, int step, int keep_s,
                             double dt, const long long* __restrict__ soff,
                             const long long* __restrict__ band_off, int kz_fac, int m0_shift,
                             const double* __restrict__ U,
                             const double* __restrict__ Lm, const int* __restrict__ piv,
                             const double* __restrict__ invd, const double* __restrict__ s,
                             const double* __restrict__ A, const double* __restrict__ Ap,
                             double* __restrict__ out, int gw0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5;
  const int gw = gw0 + blockIdx.x * (blockDim.x >> 5) + wib;   // global warp = (m, group)
  unsigned char* base = smem_raw + (size_t)wib * SolveSmem<KL>::per_warp(nc, CPW, keep_s);
  band_solve_warp<KL>(gw, base, M, nc, Kz, K, CPW, groups_per_m, step, keep_s, dt, soff, band_off, kz_fac,
                      m0_shift, U, Lm, piv, invd, s, A, Ap, out);
}

// Batched persistent form (batch.cu): every warp takes (member, warp task) items
// from the queue into its own slab of `slab` bytes (the largest any member needs).
template <int KL>
__global__ void kb_band_solve(const BSolveJob* __restrict__ jobs, const int2* __restrict__ items, int nitems,
                              int slab, int* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* base = smem_raw + (size_t)wib * slab;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(ctr, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= nitems) break;
    const int2 w = items[it];
    const BSolveJob j = jobs[w.x];
    band_solve_warp<KL>(w.y, base, j.M, j.nc, j.Kz, j.K, j.CPW, j.gpm, j.step, 0, j.dt, j.soff, j.band_off,
                        j.kz_fac, 0, j.U, j.L, j.piv, j.invd, j.s, j.A, j.Ap, j.out, j.Az);
    __syncwarp();   // the slab is restaged by the next item
  }
  if (lane == 0) bq_finish(ctr, gridDim.x * (blockDim.x >> 5));
}


// Segmented variant for narrow bands (the diffusion / Fisher-KPP operators): each
// real chain is cut into SEG row segments that run side by side on SEG lanes.
// An FP64 instruction holds its sub-partition's unit for the same time with 8 or
// 32 active lanes, and the recurrences of the staged kernel run one row at a time
// with 8 of 32 lanes busy, so their cost is (rows) x (FP64 instructions per row);
// here every lane works and a warp walks N / SEG rows.  With the factors fixed,
// both substitutions are linear recurrences, and a segment's result is its
// "particular" run from a zero entry state plus a precomputed linear function of
// the entry state (k_seg_setup):
//   forward: y_j = y^p_j + PHf[j] . w,   exit window = E^p + PSf . w,
//            w = the KL pending rows that enter the segment (exact for segment 0);
//   back:    x_i = x^p_i + PHb[i] . v,   v = x of the 2KL rows after the segment
//            (zero for the last).
// A short sequential pass over the segments (one state component per lane) then
// fixes every entry state, and a full-lane pass adds the corrections.  The sums are
// ordered differently from k_band_solve: results agree to rounding, not bitwise.

template <int KL, int SEG>
struct SegSmem {
  static constexpr int W = 2 * KL + 1;
  static constexpr int CPW = 32 / SEG, G = CPW / 4;
  // pivot-free record: L (KL), 1/diag, U upper (KL), PHf (KL), PHb (KL), padded to
  // an even count (16-byte records)
  static constexpr int RW = (4 * KL + 1 + 1) & ~1;
  static constexpr int RO_L = 0, RO_D = KL, RO_U = KL + 1, RO_F = 2 * KL + 1, RO_B = 3 * KL + 1;
  // doubles per row and |k|: U (W), L (KL), 1/diag, PHf (KL), PHb (2 KL); or the
  // pivot-free record (RW, no pivot rows)
  __host__ __device__ static size_t per_warp(int nc, int keep_s, bool np = false) {
    const size_t rowd = np ? (size_t)RW : (size_t)(W + KL + 1 + KL + 2 * KL);
    const size_t d = (size_t)nc * G * rowd + (size_t)G * SEG * KL * KL +
                     (size_t)nc * CPW * (keep_s ? 2 : 1) + (size_t)SEG * CPW * (3 * KL + 2 * KL);
    return (d * sizeof(double) + (np ? 0 : (size_t)nc * G * sizeof(int)) + 15) / 16 * 16;
  }
};

// Pivot-free records of one family (see BandLU::RNP): thread = (m, |k| x row).
template <int KL>
__global__ void k_pack_seg_np(int nc, int Kz, const long long* __restrict__ off, const double* __restrict__ U,
                              const double* __restrict__ Lm, const double* __restrict__ invd,
                              const double* __restrict__ PHf, const double* __restrict__ PHb,
                              double* __restrict__ RNP) {
  using SM = SegSmem<KL, 8>;
  constexpr int W = 2 * KL + 1, RW = SM::RW;
  const int m = blockIdx.y;
  const int Nm = nc - m;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)Kz * Nm) return;
  const int kabs = (int)(t / Nm), i = (int)(t % Nm);
  const long long R = off[m] + (long long)i * Kz + kabs;       // factor row
  double* rec = RNP + (off[m] + (long long)kabs * Nm + i) * RW;
#pragma unroll
  for (int q = 0; q < KL; ++q) {
    rec[SM::RO_L + q] = Lm[R * KL + q];
    rec[SM::RO_U + q] = U[R * W + q + 1];
    rec[SM::RO_F + q] = PHf[R * KL + q];
    rec[SM::RO_B + q] = PHb[R * 2 * KL + q];
  }
  rec[SM::RO_D] = invd[R];
  for (int q = 4 * KL + 1; q < RW; ++q) rec[q] = 0.0;
}

// rows [j0, j1) of segment s of an N-row chain: SEG - 1 segments of floor(N / SEG)
// rows, the last takes the rest
template <int SEG>
__host__ __device__ __forceinline__ void seg_range(int N, int s, int& j0, int& j1) {
  const int L = N / SEG;
  j0 = s * L;
  j1 = (s == SEG - 1) ? N : j0 + L;
}

// Influence data of the segmented solve for one factor family (rows off[m] + r Kz + k):
// thread = (system m * Kz + k, segment, unit u); u < KL: forward entry-window unit,
// else back entry unit t = u - KL.
template <int KL, int SEG>
__global__ void k_seg_setup(int M, int nc, int Kz, const long long* __restrict__ off,
                            const double* __restrict__ U, const double* __restrict__ Lm,
                            const int* __restrict__ piv, double* __restrict__ PHf, double* __restrict__ PHb,
                            double* __restrict__ PSf) {
  constexpr int W = 2 * KL + 1, NU = 3 * KL;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)M * Kz * SEG * NU) return;
  const int u = (int)(t % NU);
  const int s = (int)((t / NU) % SEG);
  const long long sys = t / ((long long)NU * SEG);
  const int m = (int)(sys / Kz), kabs = (int)(sys % Kz);
  const int N = nc - m;
  int j0, j1;
  seg_range<SEG>(N, s, j0, j1);
  auto row = [&](int r) -> long long { return off[m] + (long long)r * Kz + kabs; };
  if (u < KL) {
    // forward: unit entry window w[1 + u] = 1, no right-hand side
    double w[KL + 1];
#pragma unroll
    for (int q = 0; q <= KL; ++q) w[q] = (q == u + 1) ? 1.0 : 0.0;
    for (int j = j0; j < j1; ++j) {
      const long long R = row(j);
#pragma unroll
      for (int q = 0; q < KL; ++q) w[q] = w[q + 1];
      w[KL] = 0.0;
      const int d = piv[R] - j;
#pragma unroll
      for (int q = 1; q <= KL; ++q)
        if (q == d) { const double x = w[0]; w[0] = w[q]; w[q] = x; }
      PHf[R * KL + u] = w[0];
#pragma unroll
      for (int q = 1; q <= KL; ++q) w[q] = __fma_rn(-Lm[R * KL + q - 1], w[0], w[q]);
    }
#pragma unroll
    for (int q = 0; q < KL; ++q) PSf[((sys * SEG + s) * KL + q) * KL + u] = w[q + 1];
  } else {
    // back: unit value of x at row j1 + tu, zero y; x_i = -sum_q U_{i,i+q}/U_ii x_{i+q}
    const int tu = u - KL;
    double xv[2 * KL];                                 // x_{i+1} .. x_{i+2KL}
#pragma unroll
    for (int q = 0; q < 2 * KL; ++q) xv[q] = (q == tu) ? 1.0 : 0.0;   // at i = j1 - 1
    for (int i = j1 - 1; i >= j0; --i) {
      const long long R = row(i);
      double x = 0.0;
#pragma unroll
      for (int q = 2 * KL; q >= 1; --q) x = __fma_rn(-U[R * W + q], xv[q - 1], x);
      PHb[R * 2 * KL + tu] = x;
#pragma unroll
      for (int q = 2 * KL - 1; q >= 1; --q) xv[q] = xv[q - 1];
      xv[0] = x;
    }
  }
}

// Arithmetic of the segmented recurrences: FP64, or (DF) double-float on the FP32
// pipe (df.cuh) for the FP32 and BF16x3 forms, whose factor records and entry-window
// data were converted to hi + lo pairs at setup.  Both representations take 8 bytes,
// so the shared-memory layout is the same.  The right-hand side is formed in FP64
// (as in every variant) and converted once; the output is rounded back to FP64 and
// the AB-CN "- s" taken there (the FP64 pipe has room; fewer instructions than the
// double-float subtraction).
template <bool DF>
struct SegAr;
template <>
struct SegAr<false> {
  using R = double;
  __device__ static R zero() { return 0.0; }
  __device__ static R from(double v) { return v; }
  __device__ static R fma(R a, R b, R c) { return __fma_rn(a, b, c); }
  __device__ static R nfma(R a, R b, R c) { return __fma_rn(-a, b, c); }   // c - a b
  __device__ static R mul(R a, R b) { return __dmul_rn(a, b); }
  __device__ static double sub_out(R y, double sv) { return y - sv; }
  __device__ static double out(R y) { return y; }
};
template <>
struct SegAr<true> {
  using R = dfl;
  __device__ static R zero() { return df_make(0.0f, 0.0f); }
  __device__ static R from(double v) { return df_from_double(v); }
  __device__ static R fma(R a, R b, R c) { return df_madd(a, b, c); }
  __device__ static R nfma(R a, R b, R c) { return df_nmadd(a, b, c); }
  __device__ static R mul(R a, R b) { return df_mul(a, b); }
  __device__ static double sub_out(R y, double sv) { return __dsub_rn(df_to_double(y), sv); }
  __device__ static double out(R y) { return df_to_double(y); }
};
static_assert(sizeof(dfl) == sizeof(double), "double-float records keep the FP64 layout");

// NP (no pivoting): the factorisation made no row interchange in any system of
// the family, so the pivoted U rows carry exact zeros beyond the KL-th upper
// entry; the recurrences then skip the swaps and those zero terms (the same
// products in the same order: bitwise equal results, up to the sign of zero).
// The work of one warp (gw = m groups_per_m + group) in its shared-memory slab
// `base`; Az (may be NULL) as in band_solve_warp.
template <int KL, int SEG, bool NP, bool DF = false>
__device__ __forceinline__ void band_solve_seg_warp(int gw, unsigned char* __restrict__ base, int M, int nc,
                                                    int Kz, int K, int groups_per_m, int step, int keep_s,
                                                    double dt, const long long* __restrict__ soff,
                                                    const long long* __restrict__ band_off,
                                                    const double* __restrict__ U,
                                                    const double* __restrict__ Lm, const int* __restrict__ piv,
                                                    const double* __restrict__ invd,
                                                    const double* __restrict__ PHf,
                                                    const double* __restrict__ PHb,
                                                    const double* __restrict__ PSf,
                                                    const double* __restrict__ RNP,
                                                    const double* __restrict__ s, const double* __restrict__ A,
                                                    const double* __restrict__ Ap, double* __restrict__ out,
                                                    const SplitPlanes& sp, double* __restrict__ Az = nullptr,
                                                    bool pdl = false) {
  using SM = SegSmem<KL, SEG>;
  using AR = SegAr<DF>;
  using R = typename AR::R;                                  // double, or dfl when DF
  static_assert(NP || !DF, "the double-float form is pivot-free only");
  constexpr int W = SM::W, CPW = SM::CPW, G = SM::G, RW = SM::RW;
  constexpr int UW = NP ? KL : 2 * KL;                      // upper entries the substitution reads
  const int lane = threadIdx.x & 31;
  if (gw >= M * groups_per_m) return;
  const int m = gw / groups_per_m;
  const int k0 = (gw % groups_per_m) * G;
  const int gcnt = min(G, Kz - k0);
  const int N = nc - m;
  // pivoting form: U [N][G][W], L [N][G][KL], 1/diag [N][G], PHf [N][G][KL],
  // PHb [N][G][2KL]; pivot-free form: the records [G][N][RW]
  double* Us = reinterpret_cast<double*>(base);
  double* Ls = Us + (size_t)N * G * W;
  double* Ds = Ls + (size_t)N * G * KL;
  double* Pf = Ds + (size_t)N * G;
  double* Pb = Pf + (size_t)N * G * KL;
  R* Rs = reinterpret_cast<R*>(base);
  R* PS = NP ? Rs + (size_t)G * N * RW : reinterpret_cast<R*>(Pb + (size_t)N * G * 2 * KL);   // [G][SEG][KL][KL]
  R* Y = PS + (size_t)G * SEG * KL * KL;                     // [N][CPW]
  double* Sv = reinterpret_cast<double*>(Y + (size_t)N * CPW);   // [N][CPW] (keep_s)
  R* BH = reinterpret_cast<R*>(Sv + (keep_s ? (size_t)N * CPW : 0));   // [SEG][KL][CPW] right-hand side heads
  R* EP = BH + SEG * KL * CPW;                               // [SEG][KL][CPW] particular exit windows
  R* SF = EP + SEG * KL * CPW;                               // [SEG][KL][CPW] entry windows
  R* SB = SF + SEG * KL * CPW;                               // [SEG][2KL][CPW] back entry values
  int* Pi = reinterpret_cast<int*>(SB + SEG * 2 * KL * CPW); // [N][G]
  const long long fb = band_off[m];
  const long long sm = soff[m];
  if constexpr (NP) {
    // the warp's gcnt systems are consecutive blocks of N records
    const int bytes = gcnt * N * RW * 8;
    stage_rows(Rs, bytes, RNP + (fb + (long long)k0 * N) * RW, bytes, 1, bytes, lane);
    stage_rows(PS, G * SEG * KL * KL * 8, PSf + ((long long)m * Kz + k0) * SEG * KL * KL, 0, 1,
               gcnt * SEG * KL * KL * 8, lane);
  } else {
    const long long r0 = fb + k0;
    stage_rows(Us, G * W * 8, U + r0 * W, (long long)Kz * W * 8, N, gcnt * W * 8, lane);
    stage_rows(Ls, G * KL * 8, Lm + r0 * KL, (long long)Kz * KL * 8, N, gcnt * KL * 8, lane);
    stage_rows(Ds, G * 8, invd + r0, (long long)Kz * 8, N, gcnt * 8, lane);
    stage_rows(Pf, G * KL * 8, PHf + r0 * KL, (long long)Kz * KL * 8, N, gcnt * KL * 8, lane);
    stage_rows(Pb, G * 2 * KL * 8, PHb + r0 * 2 * KL, (long long)Kz * 2 * KL * 8, N, gcnt * 2 * KL * 8, lane);
    stage_rows(PS, G * SEG * KL * KL * 8, PSf + ((long long)m * Kz + k0) * SEG * KL * KL, 0, 1,
               gcnt * SEG * KL * KL * 8, lane);
    stage_rows(Pi, G * 4, piv + r0, (long long)Kz * 4, N, gcnt * 4, lane);
  }
  // operand accessors: row i of system kq (R is double whenever NP is false)
  auto Lrow = [&](int i, int kq) -> const R* {
    return NP ? Rs + ((size_t)kq * N + i) * RW + SM::RO_L : reinterpret_cast<const R*>(Ls + ((size_t)i * G + kq) * KL);
  };
  auto Dval = [&](int i, int kq) -> R {
    return NP ? Rs[((size_t)kq * N + i) * RW + SM::RO_D] : reinterpret_cast<const R*>(Ds)[(size_t)i * G + kq];
  };
  auto Uup = [&](int i, int kq, int t) -> R {     // U_{i, i+1+t}
    return NP ? Rs[((size_t)kq * N + i) * RW + SM::RO_U + t]
              : reinterpret_cast<const R*>(Us)[((size_t)i * G + kq) * W + t + 1];
  };
  auto PFrow = [&](int i, int kq) -> const R* {
    return NP ? Rs + ((size_t)kq * N + i) * RW + SM::RO_F : reinterpret_cast<const R*>(Pf + ((size_t)i * G + kq) * KL);
  };
  auto PBrow = [&](int i, int kq) -> const R* {
    return NP ? Rs + ((size_t)kq * N + i) * RW + SM::RO_B
              : reinterpret_cast<const R*>(Pb + ((size_t)i * G + kq) * 2 * KL);
  };
  cp_async_commit();
  // pdl: launched as a programmatic dependent; the staged factors and influence data
  // were written at setup, so their copies above may overlap the predecessor's tail,
  // and the wait comes before the first read of s, A, A_prev and the first write
  if (pdl) {
    pdl_wait();
    pdl_trigger();
  }
  // right-hand sides, every lane busy (as in k_band_solve)
  const double h = (step == MLX_STEP_FEBE_FULL) ? dt : 0.5 * dt;
  const double2* s2 = reinterpret_cast<const double2*>(s);
  const double2* A2 = reinterpret_cast<const double2*>(A);
  const double2* Ap2 = reinterpret_cast<const double2*>(Ap);
  const int LP = 16 / G;
  const int cpl = lane / LP, il = lane - cpl * LP;
  const int kql = cpl >> 1, sgl = cpl & 1, kabsl = k0 + kql;
  const bool lane_piece = cpl < 2 * gcnt && !(sgl && kabsl == 0);
  const long long pbase = sm + (long long)(sgl ? K - kabsl : kabsl) * N;
  // rows per unrolled batch and unroll depths: the double-float bodies are about 15
  // times longer, so their loops stay short to keep the code in the instruction cache
  constexpr int RB = DF ? 4 : 8;
  constexpr int UR = DF ? 1 : 2, UO = DF ? 2 : 4;
  for (int i = il; i < (lane_piece ? N : 0); i += RB * LP) {
    double2 sv[RB], av[RB], apv[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int ii = i + u * LP;
      const long long o = pbase + (ii < N ? ii : i);
      sv[u] = s2[o];
      av[u] = (step != MLX_STEP_PLAIN && A) ? A2[o] : make_double2(0.0, 0.0);
      apv[u] = (step == MLX_STEP_ABCN && Ap) ? Ap2[o] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int ii = i + u * LP;
      if (ii >= N) break;
      double2 r;
      if (step == MLX_STEP_PLAIN) {
        r = sv[u];
      } else if (step == MLX_STEP_ABCN) {
        r = make_double2(rhs_abcn(sv[u].x, av[u].x, apv[u].x, A, Ap, dt),
                         rhs_abcn(sv[u].y, av[u].y, apv[u].y, A, Ap, dt));
        if (keep_s) {
          Sv[(size_t)ii * CPW + cpl * 2] = sv[u].x;
          Sv[(size_t)ii * CPW + cpl * 2 + 1] = sv[u].y;
        }
      } else {
        r = sv[u];
        if (A) r = make_double2(rhs_febe(sv[u].x, av[u].x, true, h), rhs_febe(sv[u].y, av[u].y, true, h));
      }
      Y[(size_t)ii * CPW + cpl * 2] = AR::from(r.x);
      Y[(size_t)ii * CPW + cpl * 2 + 1] = AR::from(r.y);
    }
  }
  cp_async_wait_all();
  __syncwarp();
  // lane = segment sg x chain c
  const int c = lane % CPW, sg = lane / CPW;
  const int kk = c >> 2;
  const bool act = kk < gcnt;
  int j0, j1;
  seg_range<SEG>(N, sg, j0, j1);
  // heads of the right-hand side of every segment after the first: the previous
  // segment's window reads them after their owner has overwritten them
  for (int e = lane; e < SEG * KL * CPW; e += 32) {
    const int ss = e / (KL * CPW), q = (e / CPW) % KL, cc = e % CPW;
    int a0, a1;
    seg_range<SEG>(N, ss, a0, a1);
    BH[e] = (ss > 0) ? Y[(size_t)(a0 + q) * CPW + cc] : AR::zero();
  }
  __syncwarp();
  R* y = Y + c;
  // ---- forward, particular run of this segment ----
  if (act) {
    R w[KL + 1];
    w[0] = AR::zero();
#pragma unroll
    for (int q = 0; q < KL; ++q) w[q + 1] = (sg == 0 && q < N) ? y[(size_t)q * CPW] : AR::zero();
#pragma unroll UR
    for (int j = j0; j < j1; ++j) {
#pragma unroll
      for (int q = 0; q < KL; ++q) w[q] = w[q + 1];
      const int jn = j + KL;
      w[KL] = (jn >= N) ? AR::zero() : (jn >= j1 ? BH[((sg + 1) * KL + (jn - j1)) * CPW + c] : y[(size_t)jn * CPW]);
      if (!NP) {
        const int d = Pi[(size_t)j * G + kk] - j;
#pragma unroll
        for (int q = 1; q <= KL; ++q)
          if (q == d) { const R t = w[0]; w[0] = w[q]; w[q] = t; }
      }
      y[(size_t)j * CPW] = w[0];
      const R* l = Lrow(j, kk);
#pragma unroll
      for (int q = 1; q <= KL; ++q) w[q] = AR::nfma(l[q - 1], w[0], w[q]);
    }
#pragma unroll
    for (int q = 0; q < KL; ++q) EP[(sg * KL + q) * CPW + c] = w[q + 1];
  }
  __syncwarp();
  // ---- entry windows, one component per lane: SF[1] = EP[0], SF[s] = EP[s-1] + PSf[s-1] SF[s-1] ----
  for (int ss = 1; ss < SEG; ++ss) {
    for (int q = sg; q < KL; q += SEG) {
      if (act) {
        R v = EP[((ss - 1) * KL + q) * CPW + c];
        if (ss > 1) {
          const R* ps = PS + ((size_t)(kk * SEG + ss - 1) * KL + q) * KL;
#pragma unroll
          for (int q2 = 0; q2 < KL; ++q2) v = AR::fma(ps[q2], SF[((ss - 1) * KL + q2) * CPW + c], v);
        }
        SF[(ss * KL + q) * CPW + c] = v;
      }
    }
    __syncwarp();
  }
  // ---- forward corrections, then y / U_rr for every row and chain ----
  if (act && sg > 0) {
    R wv[KL];
#pragma unroll
    for (int q = 0; q < KL; ++q) wv[q] = SF[(sg * KL + q) * CPW + c];
    for (int j = j0; j < j1; ++j) {
      const R* pf = PFrow(j, kk);
      R v = y[(size_t)j * CPW];
#pragma unroll
      for (int q = 0; q < KL; ++q) v = AR::fma(pf[q], wv[q], v);
      y[(size_t)j * CPW] = v;
    }
  }
  __syncwarp();
  for (int i = il; i < (lane_piece ? N : 0); i += LP) {
    const R dv = Dval(i, kql);
    Y[(size_t)i * CPW + cpl * 2] = AR::mul(Y[(size_t)i * CPW + cpl * 2], dv);
    Y[(size_t)i * CPW + cpl * 2 + 1] = AR::mul(Y[(size_t)i * CPW + cpl * 2 + 1], dv);
  }
  __syncwarp();
  // ---- back substitution, particular run of this segment (zero x after it) ----
  if (act) {
    R acc[UW];
#pragma unroll
    for (int t = 0; t < UW; ++t) {
      const int r = j1 - 1 - t;
      acc[t] = (r >= j0) ? y[(size_t)r * CPW] : AR::zero();
    }
    R xn = AR::zero();
#pragma unroll UR
    for (int i = j1 - 1; i >= j0; --i) {
      const R xi = AR::nfma(Uup(i, kk, 0), xn, acc[0]);
#pragma unroll
      for (int t = 1; t < UW; ++t)
        if (i - t >= j0) acc[t] = AR::nfma(Uup(i - t, kk, t), xn, acc[t]);
      y[(size_t)i * CPW] = xi;
#pragma unroll
      for (int t = 0; t < UW - 1; ++t) acc[t] = acc[t + 1];
      const int rn = i - UW;
      acc[UW - 1] = (rn >= j0) ? y[(size_t)rn * CPW] : AR::zero();
      xn = xi;
    }
  }
  __syncwarp();
  // ---- back entry values, one component per lane, from the last segment down:
  // SB[s][t] = x of row (start of segment s+1) + t = x^p + PHb . SB[s+1] ----
  for (int ss = SEG - 2; ss >= 0; --ss) {
    int a0, a1;
    seg_range<SEG>(N, ss + 1, a0, a1);
    for (int t = sg; t < UW; t += SEG) {
      if (act) {
        const int r = a0 + t;
        R v = y[(size_t)r * CPW];
        if (ss + 1 < SEG - 1) {
          const R* pb = PBrow(r, kk);
#pragma unroll
          for (int t2 = 0; t2 < UW; ++t2) v = AR::fma(pb[t2], SB[((ss + 1) * 2 * KL + t2) * CPW + c], v);
        }
        SB[(ss * 2 * KL + t) * CPW + c] = v;
      }
    }
    __syncwarp();
  }
  // ---- back corrections ----
  if (act && sg < SEG - 1) {
    R vv[UW];
#pragma unroll
    for (int t = 0; t < UW; ++t) vv[t] = SB[(sg * 2 * KL + t) * CPW + c];
    for (int i = j0; i < j1; ++i) {
      const R* pb = PBrow(i, kk);
      R v = y[(size_t)i * CPW];
#pragma unroll
      for (int t = 0; t < UW; ++t) v = AR::fma(pb[t], vv[t], v);
      y[(size_t)i * CPW] = v;
    }
  }
  __syncwarp();
  // ---- output (and, when sp.bs is set, its three BF16 parts in the split planes of
  // the backward contraction, exactly as k_split_spec would write them) ----
  double2* out2 = reinterpret_cast<double2*>(out);
  const long long prow = sp.bs ? ((long long)m * sp.K2 + 2 * (sgl ? K - kabsl : kabsl)) * sp.Kq : 0;
#pragma unroll UO
  for (int i = il; i < (lane_piece ? N : 0); i += LP) {
    const R yx = Y[(size_t)i * CPW + cpl * 2], yy = Y[(size_t)i * CPW + cpl * 2 + 1];
    double2 v;
    if (step == MLX_STEP_ABCN) {
      const double2 sv = keep_s ? make_double2(Sv[(size_t)i * CPW + cpl * 2], Sv[(size_t)i * CPW + cpl * 2 + 1])
                                : s2[pbase + i];
      v = make_double2(AR::sub_out(yx, sv.x), AR::sub_out(yy, sv.y));
    } else {
      v = make_double2(AR::out(yx), AR::out(yy));
    }
    out2[pbase + i] = v;
    if (Az) reinterpret_cast<double2*>(Az)[pbase + i] = make_double2(0.0, 0.0);
    if (sp.bs) {
      unsigned short h, md, lo;
      split3_f64(v.x, h, md, lo);
      const long long o = prow + i;
      sp.bs[o] = h; sp.bs[sp.part + o] = md; sp.bs[2 * sp.part + o] = lo;
      split3_f64(v.y, h, md, lo);
      sp.bs[o + sp.Kq] = h; sp.bs[sp.part + o + sp.Kq] = md; sp.bs[2 * sp.part + o + sp.Kq] = lo;
    }
  }
}

template <int KL, int SEG, bool NP, bool DF = false>
__global__ void k_band_solve_seg(int M, int nc, int Kz, int K, int groups_per_m, int step, int keep_s,
                                 double dt, const long long* __restrict__ soff,
                                 const long long* __restrict__ band_off, const double* __restrict__ U,
                                 const double* __restrict__ Lm, const int* __restrict__ piv,
                                 const double* __restrict__ invd, const double* __restrict__ PHf,
                                 const double* __restrict__ PHb, const double* __restrict__ PSf,
                                 const double* __restrict__ RNP,
                                 const double* __restrict__ s, const double* __restrict__ A,
                                 const double* __restrict__ Ap, double* __restrict__ out,
                                 SplitPlanes sp, int pair) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5;
  int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  if (pair) {
    // 8 warps per CTA; warps w and w + 4 share an SM sub-partition (and its FP64
    // unit): w < 4 takes a system from the long end of the (m ascending, so
    // N = Nc - m descending) order, w + 4 its mirror from the short end, so that
    // every sub-partition's two chains of rows add up to about the same length
    const int T = M * groups_per_m, H = (T + 1) / 2;
    const int q = blockIdx.x * 4 + (wib & 3);
    gw = (wib < 4) ? (q < H ? q : T) : (T - 1 - q >= H ? T - 1 - q : T);
  }
  unsigned char* base = smem_raw + (size_t)wib * SegSmem<KL, SEG>::per_warp(nc, keep_s, NP);
  band_solve_seg_warp<KL, SEG, NP, DF>(gw, base, M, nc, Kz, K, groups_per_m, step, keep_s, dt, soff, band_off, U,
                                       Lm, piv, invd, PHf, PHb, PSf, RNP, s, A, Ap, out, sp, nullptr, true);
}

// Batched persistent form (batch.cu), as kb_band_solve: warps take (member, warp
// task) items; the member's job also names its influence data and, optionally,
// the split planes its output is written to.
template <int KL, int SEG, bool NP, bool DF = false>
__global__ void kb_band_solve_seg(const BSolveJob* __restrict__ jobs, const int2* __restrict__ items, int nitems,
                                  int slab, int* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* base = smem_raw + (size_t)wib * slab;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(ctr, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= nitems) break;
    const int2 w = items[it];
    const BSolveJob j = jobs[w.x];
    SplitPlanes sp;
    sp.bs = j.bs; sp.part = j.part; sp.Kq = j.kq; sp.K2 = j.k2;
    band_solve_seg_warp<KL, SEG, NP, DF>(w.y, base, j.M, j.nc, j.Kz, j.K, j.gpm, j.step, 0, j.dt, j.soff, j.band_off,
                                     j.U, j.L, j.piv, j.invd, j.PHf, j.PHb, j.PSf, j.RNP, j.s, j.A, j.Ap, j.out, sp,
                                     j.Az);
    __syncwarp();
  }
  if (lane == 0) bq_finish(ctr, gridDim.x * (blockDim.x >> 5));
}

__global__ void k_axpby(long long n, double a, const double2* __restrict__ x, double b,
                        const double2* __restrict__ y, double2* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 u = x[i], v = y[i];
  out[i] = make_double2(a * u.x + b * v.x, a * u.y + b * v.y);
}

}  // namespace

int mlx_band_setup(mlx_ctx* c, cudaStream_t st) {
  const int kl = c->kl;
  const int W = 2 * kl + 1;
  const long long rows = c->band_rows;
  // (re)allocate factor storage
  cudaFree(c->d_Bplus);
  cudaFree(c->lu_half.U); cudaFree(c->lu_half.L); cudaFree(c->lu_half.piv); cudaFree(c->lu_half.invd);
  cudaFree(c->lu_full.U); cudaFree(c->lu_full.L); cudaFree(c->lu_full.piv); cudaFree(c->lu_full.invd);
  for (BandLU* f : {&c->lu_half, &c->lu_full}) {
    cudaFree(f->FS); cudaFree(f->BS);
    cudaFree(f->PHf); cudaFree(f->PHb); cudaFree(f->PSf); cudaFree(f->RNP); cudaFree(f->RDF); cudaFree(f->PSDF);
  }
  c->d_Bplus = nullptr;
  c->lu_half = BandLU();
  c->lu_full = BandLU();
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_Bplus, sizeof(double) * rows * W));
  for (BandLU* f : {&c->lu_half, &c->lu_full}) {
    MLX_CUDA_TRY(c, cudaMalloc(&f->U, sizeof(double) * rows * W));
    MLX_CUDA_TRY(c, cudaMalloc(&f->L, sizeof(double) * rows * kl));
    MLX_CUDA_TRY(c, cudaMalloc(&f->piv, sizeof(int) * rows));
    MLX_CUDA_TRY(c, cudaMalloc(&f->invd, sizeof(double) * rows));
  }
  // scratch: per system 3 band buffers [N][W] + window [N][3kl+1], N <= Nc
  const long long stride = (long long)c->nc * (3 * W + 3 * kl + 1);
  double* scratch = nullptr;
  MLX_CUDA_TRY(c, cudaMalloc(&scratch, sizeof(double) * stride * c->M * c->Kz));
  // Laplacian row offsets
  std::vector<long long> lrows(c->M + 1, 0);
  for (int m = 0; m < c->M; ++m) lrows[m + 1] = lrows[m] + (c->nc - m);
  long long* d_lrows = nullptr;
  MLX_CUDA_TRY(c, cudaMalloc(&d_lrows, sizeof(long long) * (c->M + 1)));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(d_lrows, lrows.data(), sizeof(long long) * (c->M + 1),
                                  cudaMemcpyHostToDevice, st));
  const int nsys = c->M * c->Kz;
  const int tb = 64;
  k_band_setup<<<(nsys + tb - 1) / tb, tb, 0, st>>>(
      c->M, c->nc, c->Kz, c->lz, c->d_band_off, d_lrows, c->d_lap, c->nu, c->nu_h, c->p, c->dt, kl,
      c->d_Bplus, c->lu_half.U, c->lu_half.L, c->lu_half.piv, c->lu_half.invd, c->lu_full.U,
      c->lu_full.L, c->lu_full.piv, c->lu_full.invd, scratch, stride);
  MLX_LAUNCH_CHECK(c);
  // did any system interchange rows?  (the pivot of column i is the local row i
  // when it did not); a family without interchanges runs the pivot-free recurrences
  {
    std::vector<int> hp((size_t)rows);
    for (BandLU* f : {&c->lu_half, &c->lu_full}) {
      MLX_CUDA_TRY(c, cudaMemcpyAsync(hp.data(), f->piv, sizeof(int) * rows, cudaMemcpyDeviceToHost, st));
      MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
      bool none = true;
      for (int m = 0; m < c->M && none; ++m)
        for (int i = 0; i < c->nc - m && none; ++i)
          for (int kz = 0; kz < c->Kz; ++kz)
            if (hp[(size_t)(c->band_off[m] + (long long)i * c->Kz + kz)] != i) { none = false; break; }
      f->nopiv = none && c->solve_nopiv;
    }
  }
  for (BandLU* f : {&c->lu_half, &c->lu_full}) {
    const int rc = mlx_pack_lean(c, *f, kl, c->d_band_off, c->Kz, rows, st);
    if (rc) return rc;
    const int rs = mlx_seg_build(c, *f, c->solve_seg, st);
    if (rs) return rs;
  }
  MLX_LAUNCH_CHECK(c);
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  cudaFree(scratch);
  cudaFree(d_lrows);
  return MLX_OK;
}

// Lean variant: 32 (or 16) real chains per warp, every lane busy in every FP64
// instruction, and few other instructions per row.  On this part an FP64 warp
// instruction occupies the pipe as long with 8 active lanes as with 32, and a
// warp running a recurrence issues one instruction every few cycles, so both the
// lanes per FP64 instruction and the instructions per row decide the time:
//  * the factors are read as per-row records written once by k_pack_lean:
//    forward FS[row] = {L[row][0..KL-1], pivot offset mask (int), pad}, back
//    substitution BS[row] = {U[row - t][t + 1] for t < 2KL, 1/diag[row - 2KL],
//    pad}: the U column the pipelined back substitution touches at that step.  A
//    step stages one contiguous 16-byte-aligned block per |k| with cp.async,
//    LEAN_AHEAD rows ahead of use;
//  * per-lane global addresses are formed once and offset per row, ring slots
//    advance by a running index, the step kind is a template parameter;
//  * the shared-memory operands of the next row are loaded into registers while
//    the current row computes.
// The forward-elimination values go to a per-warp global scratch [row][CPW] (one
// coalesced row per step, read back through the ring, mostly from L2); the
// solution is written straight to the output.  Arithmetic, and its order, is
// that of k_band_solve: the results are bitwise equal.
constexpr int LEAN_AHEAD = 12;
constexpr int LEAN_PLAIN = 0, LEAN_FEBE = 1, LEAN_ABCN = 2;   // right-hand side s, s + h A, AB-CN

template <int KL, int CPW, int NFLD = 1>
struct LeanSmem {
  static constexpr int G = CPW / (4 * NFLD);          // |k| values per warp (4 NFLD real chains each)
  static constexpr int NP = CPW / 2;                  // complex pieces per row
  static constexpr int P = LEAN_AHEAD;
  static constexpr int FW = (KL + 2) & ~1;            // forward record (doubles)
  static constexpr int BW = 2 * KL + 2;               // back-substitution record (doubles)
  static constexpr int R = P + 1;                     // ring slots
  static constexpr size_t f_rhs = (size_t)G * FW * sizeof(double);
  static constexpr size_t fslot = f_rhs + 3 * NP * sizeof(double2);   // + s, A, A_prev pieces
  static constexpr size_t b_y = (size_t)G * BW * sizeof(double);
  static constexpr size_t b_s = b_y + CPW * sizeof(double);
  static constexpr size_t bslot = b_s + NP * sizeof(double2);
  static constexpr size_t per_warp = (R * (fslot > bslot ? fslot : bslot) + 15) / 16 * 16;
};

// NFLD = 2: the two fields of a vortex state (psi, chi; fstride complex values apart)
// in one launch, sharing each staged factor record between 8 real chains per |k|
// (field, sign of k, Re/Im), so that the factors are read once per step.
template <int KL, int CPW, int MODE, int NFLD>
__global__ void __launch_bounds__(64, 1) k_band_solve_lean(
    int M, int nc, int Kz, int K, int groups_per_m, double h, double dt, int hasA, int hasAp,
    const long long* __restrict__ soff, const long long* __restrict__ band_off, int kz_fac, int m0_shift,
    long long fstride,
    const double* __restrict__ FS, const double* __restrict__ BS, const double* __restrict__ invd,
    const double* __restrict__ s, const double* __restrict__ A, const double* __restrict__ Ap,
    double* __restrict__ out, double* __restrict__ scratch) {
  using SM = LeanSmem<KL, CPW, NFLD>;
  constexpr int G = SM::G, NP = SM::NP, P = SM::P, FW = SM::FW, BW = SM::BW, RS = SM::R;
  constexpr int NF = (G * FW / 2 + 31) / 32, NB = (G * BW / 2 + 31) / 32;   // 16-byte chunks per lane, at most
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  if (gw >= M * groups_per_m) return;
  const int m = gw / groups_per_m;
  const int k0 = (gw % groups_per_m) * G;
  const int gcnt = min(G, Kz - k0);
  const int sh = (m == 0) ? m0_shift : 0;
  const int Nm = nc - m;
  const int N = Nm - sh;
  unsigned char* ring = smem_raw + (size_t)wib * SM::per_warp;
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring);
  double* Yg = scratch + (size_t)gw * nc * CPW;       // [row][CPW], this warp's columns
  const long long sm = soff[m];
  const int GS = (kz_fac == 1) ? 1 : gcnt;            // factor records per row
  const long long row0 = band_off[m] + (kz_fac == 1 ? 0 : k0);
  const double2* s2 = reinterpret_cast<const double2*>(s);
  // offset (complex units) of complex piece cp = (kq NFLD + field) 2 + sg at row 0, or -1
  auto piece = [=](int cp) -> long long {
    const int sg = cp & 1, fld = (cp >> 1) % NFLD, kq = (cp >> 1) / NFLD, kabs = k0 + kq;
    if (kq >= gcnt || (sg && kabs == 0)) return -1;
    const int kidx = sg ? K - kabs : kabs;
    return (long long)fld * fstride + sm + (long long)kidx * Nm + sh;
  };
  // ---- this lane's copies ----
  const int nf = GS * FW / 2, nb = GS * BW / 2;
  const double2* fsrc = reinterpret_cast<const double2*>(FS + row0 * FW) + lane;   // chunk `lane` of row 0
  const double2* bsrc = reinterpret_cast<const double2*>(BS + row0 * BW) + lane;
  const long long fstep = (long long)kz_fac * FW / 2, bstep = (long long)kz_fac * BW / 2;   // per row (double2)
  const double2* rsrc0 = nullptr;                     // right-hand-side pieces e = lane, lane + 32 of [3][NP]
  const double2* rsrc1 = nullptr;
  if (MODE != LEAN_PLAIN) {
    auto src_of = [=](int e) -> const double2* {
      if (e >= 3 * NP) return nullptr;
      const int a = e / NP;
      const long long o = piece(e % NP);
      const bool use = a == 0 || (a == 1 && hasA) || (a == 2 && MODE == LEAN_ABCN && hasAp);
      if (o < 0 || !use) return nullptr;
      return reinterpret_cast<const double2*>(a == 0 ? s : (a == 1 ? A : Ap)) + o;
    };
    rsrc0 = src_of(lane);
    rsrc1 = src_of(lane + 32);
  } else if (lane < NP) {
    const long long o = piece(lane);
    if (o >= 0) rsrc0 = s2 + o;
  }
  const long long so = (lane < NP) ? piece(lane) : -1;
  const double2* ssrc = (MODE == LEAN_ABCN && so >= 0) ? s2 + so : nullptr;   // s for the AB-CN "- s"
  const int c = lane;
  const int kk = c / (4 * NFLD), part = c & 1, cpx = c >> 1;
  const bool act = c < CPW && kk < gcnt;
  const bool valid = act && !(((c >> 1) & 1) && k0 + kk == 0);
  const int ks = (kz_fac == 1) ? 0 : (kk < gcnt ? kk : 0);   // lane's record within a row block
  const int cpl = (c < CPW) ? cpx : 0;                       // lane's piece (in range for idle lanes)
  auto rhs = [=](double sv, double q, double qp) -> double {
    if (MODE == LEAN_PLAIN) return sv;
    if (MODE == LEAN_ABCN) return rhs_abcn(sv, q, qp, hasA, hasAp, dt);
    return rhs_febe(sv, q, true, h);
  };
  const long long my0 = (c < CPW) ? piece(cpx) : -1;          // this lane's chain at row 0
  // ---- forward elimination; slot of row r: its records and the pieces of row r + KL ----
  auto stage_f = [=](int r, int slot) {
    const unsigned d = ring_s + (unsigned)(slot * SM::fslot);
    const double2* src = fsrc + r * fstep;
#pragma unroll
    for (int u = 0; u < NF; ++u)
      if (lane + 32 * u < nf) cp_async16_s(d + (lane + 32 * u) * 16, src + 32 * u);
    if (r + KL < N) {
      if (rsrc0) cp_async16_s(d + (unsigned)SM::f_rhs + lane * 16, rsrc0 + r + KL);
      if (rsrc1) cp_async16_s(d + (unsigned)SM::f_rhs + (lane + 32) * 16, rsrc1 + r + KL);
    }
  };
  struct FOps { double l[KL]; int d; double sv, q, qp; };   // d: pivot offset mask
  auto load_f = [=](int slot) -> FOps {
    FOps o;
    const unsigned char* sl = ring + (size_t)slot * SM::fslot;
    const double* rec = reinterpret_cast<const double*>(sl) + ks * FW;
#pragma unroll
    for (int q = 0; q + 1 < KL; q += 2) {
      const double2 v = *reinterpret_cast<const double2*>(rec + q);
      o.l[q] = v.x; o.l[q + 1] = v.y;
    }
    if (KL & 1) {
      const double2 v = *reinterpret_cast<const double2*>(rec + KL - 1);
      o.l[KL - 1] = v.x;
      o.d = __double2loint(v.y);
    } else {
      o.d = reinterpret_cast<const int*>(rec + KL)[0];
    }
    const double* rv = reinterpret_cast<const double*>(sl + SM::f_rhs);
    o.sv = rv[cpl * 2 + part];
    o.q = (MODE != LEAN_PLAIN) ? rv[(NP + cpl) * 2 + part] : 0.0;
    o.qp = (MODE == LEAN_ABCN) ? rv[(2 * NP + cpl) * 2 + part] : 0.0;
    return o;
  };
  for (int r = 0; r < P; ++r) {
    if (r < N) stage_f(r, r);
    cp_async_commit();
  }
  double w[KL + 1];
#pragma unroll
  for (int q = 0; q < KL; ++q) {
    double v = 0.0;
    if (act && my0 >= 0 && q < N) {
      const long long o = 2 * (my0 + q) + part;
      v = rhs(s[o], MODE != LEAN_PLAIN && hasA ? A[o] : 0.0, MODE == LEAN_ABCN && hasAp ? Ap[o] : 0.0);
    }
    w[q + 1] = v;
  }
  cp_async_wait_group<P - 1>();
  __syncwarp();
  FOps cur = load_f(0);
  double* yw = Yg + c;
  int swr = P, srd = 1;                                // slots: next row staged, next row loaded
#pragma unroll 2
  for (int j = 0; j < N; ++j) {
    if (j + P < N) stage_f(j + P, swr);
    cp_async_commit();
    cp_async_wait_group<P - 1>();
    __syncwarp();
    const FOps nxt = load_f(srd);                                  // (a stale slot after the last row: unused)
    swr = (swr == RS - 1) ? 0 : swr + 1;
    srd = (srd == RS - 1) ? 0 : srd + 1;
    if (act) {
      const double nv = (j + KL < N) ? rhs(cur.sv, cur.q, cur.qp) : 0.0;
#pragma unroll
      for (int q = 0; q < KL; ++q) w[q] = w[q + 1];
      w[KL] = nv;
      {   // row interchange with the pivot row (bit q of cur.d: offset q), as selects
        const double w0 = w[0];
        double pv = w0;
#pragma unroll
        for (int q = 1; q <= KL; ++q) {
          const bool sel = (cur.d >> q) & 1;
          pv = sel ? w[q] : pv;
          w[q] = sel ? w0 : w[q];
        }
        w[0] = pv;
      }
      yw[(size_t)j * CPW] = w[0];
#pragma unroll
      for (int q = 1; q <= KL; ++q) w[q] = __fma_rn(-cur.l[q - 1], w[0], w[q]);
    }
    cur = nxt;
  }
  cp_async_wait_all();
  __threadfence_block();
  __syncwarp();
  // ---- back substitution (software-pipelined: acc[t] is the partial sum of row i - t);
  // slot of step i: back record of row i, y_{i - 2KL}, s_i ----
  auto stage_b = [=](int i, int slot) {
    const unsigned d = ring_s + (unsigned)(slot * SM::bslot);
    const double2* src = bsrc + i * bstep;
#pragma unroll
    for (int u = 0; u < NB; ++u)
      if (lane + 32 * u < nb) cp_async16_s(d + (lane + 32 * u) * 16, src + 32 * u);
    if (lane < CPW && i - 2 * KL >= 0)
      cp_async8_s(d + (unsigned)SM::b_y + lane * 8, Yg + (size_t)(i - 2 * KL) * CPW + lane);
    if (MODE == LEAN_ABCN && ssrc) cp_async16_s(d + (unsigned)SM::b_s + lane * 16, ssrc + i);
  };
  struct BOps { double u[2 * KL]; double dinv, y, sv; };
  auto load_b = [=](int slot) -> BOps {
    BOps o;
    const unsigned char* sl = ring + (size_t)slot * SM::bslot;
    const double* rec = reinterpret_cast<const double*>(sl) + ks * BW;
#pragma unroll
    for (int t = 0; t < 2 * KL; t += 2) {
      const double2 v = *reinterpret_cast<const double2*>(rec + t);
      o.u[t] = v.x; o.u[t + 1] = v.y;
    }
    o.dinv = rec[2 * KL];
    o.y = reinterpret_cast<const double*>(sl + SM::b_y)[c < CPW ? c : 0];
    o.sv = (MODE == LEAN_ABCN) ? reinterpret_cast<const double*>(sl + SM::b_s)[cpl * 2 + part] : 0.0;
    return o;
  };
  // steps N-1 .. N-P into slots 0 .. P-1
  for (int t = 0; t < P; ++t) {
    if (N - 1 - t >= 0) stage_b(N - 1 - t, t);
    cp_async_commit();
  }
  double acc[2 * KL];
  const long long drow = row0 + ks;                            // this lane's factor row at r = 0
#pragma unroll
  for (int t = 0; t < 2 * KL; ++t) {
    const int r = N - 1 - t;
    acc[t] = (act && r >= 0) ? __dmul_rn(yw[(size_t)r * CPW], invd[drow + (long long)r * kz_fac]) : 0.0;
  }
  cp_async_wait_group<P - 1>();
  __syncwarp();
  BOps bc = load_b(0);
  double xn = 0.0;   // x_{i+1}
  double* outc = out + 2 * (my0 < 0 ? 0 : my0) + part;
  int bwr = P, brd = 1;
#pragma unroll 2
  for (int i = N - 1; i >= 0; --i) {
    if (i - P >= 0) stage_b(i - P, bwr);
    cp_async_commit();
    cp_async_wait_group<P - 1>();
    __syncwarp();
    const BOps bn = load_b(brd);                                   // (a stale slot after row 0: unused)
    bwr = (bwr == RS - 1) ? 0 : bwr + 1;
    brd = (brd == RS - 1) ? 0 : brd + 1;
    if (act) {
      const double xi = __fma_rn(-bc.u[0], xn, acc[0]);
#pragma unroll
      for (int t = 1; t < 2 * KL; ++t) acc[t] = __fma_rn(-bc.u[t], xn, acc[t]);
      if (valid) {
        outc[2 * (long long)i] = (MODE == LEAN_ABCN) ? xi - bc.sv : xi;
        if (sh) yw[(size_t)i * CPW] = xi;
      }
#pragma unroll
      for (int t = 0; t < 2 * KL - 1; ++t) acc[t] = acc[t + 1];
      acc[2 * KL - 1] = (i - 2 * KL >= 0) ? __dmul_rn(bc.y, bc.dinv) : 0.0;
      xn = xi;
    }
    bc = bn;
  }
  cp_async_wait_all();
  if (sh && valid) {
    double dacc = 0.0;
    for (int i = 0; i < N; ++i) dacc = __fma_rn(sqrt((2.0 * (i + 1) + 1.0) * 0.5), yw[(size_t)i * CPW], dacc);
    out[2 * (my0 - sh) + part] = -dacc / sqrt(0.5);
  }
}

// Lean-solve records of one factor family (see k_band_solve_lean): one thread per
// factor row R = off[m] + r kz_fac + kk.  The pivot is stored as a one-hot mask of
// its offset q from the row (bit q, q = 1 .. KL; 0 when the row is its own pivot),
// an int in the low word of the slot after the multipliers.
__global__ void k_pack_lean(int nc, int kcnt, int kz_fac, int KL, const long long* __restrict__ off,
                            const double* __restrict__ U, const double* __restrict__ L,
                            const int* __restrict__ piv, const double* __restrict__ invd,
                            double* __restrict__ FS, double* __restrict__ BS) {
  const int m = blockIdx.y;
  const int Nm = nc - m;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Nm * kcnt) return;
  const int r = (int)(idx / kcnt), kk = (int)(idx % kcnt);
  const long long R = off[m] + (long long)r * kz_fac + kk;
  const int W = 2 * KL + 1, FW = (KL + 2) & ~1, BW = 2 * KL + 2;
  const int po = piv[R] - r;
  const int mask = (po > 0 && po <= KL) ? (1 << po) : 0;
  for (int q = 0; q < FW; ++q)
    FS[R * FW + q] = (q < KL) ? L[R * KL + q] : (q == KL ? __hiloint2double(0, mask) : 0.0);
  for (int t = 0; t < 2 * KL; ++t)
    BS[R * BW + t] = (r - t >= 0) ? U[(R - (long long)t * kz_fac) * W + t + 1] : 0.0;
  BS[R * BW + 2 * KL] = (r >= 2 * KL) ? invd[R - (long long)2 * KL * kz_fac] : 0.0;
  BS[R * BW + 2 * KL + 1] = 0.0;
}

template <int KL>
static int launch_solve(mlx_ctx* c, int step, const BandLU& f, const long long* fac_off, int kz_fac,
                        int m0_shift, const double2* s, const double2* A, const double2* Ap, double2* out,
                        cudaStream_t st, int nfields = 1, const SplitPlanes* sp = nullptr, bool* wrote = nullptr) {
  if (wrote) *wrote = false;
  int seg_done = 0;
  if (nfields == 2 && c->solve_direct != 2) return MLX_EINVAL;   // two fields per launch: lean only
  if (c->solve_direct == 2) {
    if (!c->d_solve_y || !f.FS || !f.BS) return MLX_ESTATE;
    const int mode = (step == MLX_STEP_ABCN) ? LEAN_ABCN
                     : ((step == MLX_STEP_FEBE_HALF || step == MLX_STEP_FEBE_FULL) && A) ? LEAN_FEBE
                                                                                          : LEAN_PLAIN;
    const double h = (step == MLX_STEP_FEBE_FULL) ? c->dt : 0.5 * c->dt;
    auto go1 = [&](auto cpw_tag, auto mode_tag, auto nf_tag) -> int {
      constexpr int CPWL = decltype(cpw_tag)::value, MODE = decltype(mode_tag)::value;
      constexpr int NFLD = decltype(nf_tag)::value;
      constexpr int G = LeanSmem<KL, CPWL, NFLD>::G;
      const int gpm = (c->Kz + G - 1) / G;
      const int warps = c->M * gpm;
      const int WPB = (warps <= 2 * 148) ? 1 : 2;   // spread few warps over every SM
      const size_t smem = (size_t)WPB * LeanSmem<KL, CPWL, NFLD>::per_warp;
      k_band_solve_lean<KL, CPWL, MODE, NFLD><<<(warps + WPB - 1) / WPB, 32 * WPB, smem, st>>>(
          c->M, c->nc, c->Kz, c->K, gpm, h, c->dt, A != nullptr, Ap != nullptr, c->d_soff, fac_off, kz_fac,
          m0_shift, c->n_spec, f.FS, f.BS, f.invd, (const double*)s, (const double*)A, (const double*)Ap,
          (double*)out, c->d_solve_y);
      return MLX_OK;
    };
    auto go = [&](auto cpw_tag, auto mode_tag) -> int {
      if (nfields == 2) return go1(cpw_tag, mode_tag, std::integral_constant<int, 2>());
      return go1(cpw_tag, mode_tag, std::integral_constant<int, 1>());
    };
    using I16 = std::integral_constant<int, 16>;
    using I32 = std::integral_constant<int, 32>;
    using MP = std::integral_constant<int, LEAN_PLAIN>;
    using MF = std::integral_constant<int, LEAN_FEBE>;
    using MA = std::integral_constant<int, LEAN_ABCN>;
    if (c->solve_lean_cpw == 16) {
      if (mode == LEAN_ABCN) return go(I16(), MA());
      if (mode == LEAN_FEBE) return go(I16(), MF());
      return go(I16(), MP());
    }
    if (mode == LEAN_ABCN) return go(I32(), MA());
    if (mode == LEAN_FEBE) return go(I32(), MF());
    return go(I32(), MP());
  }
  if constexpr (KL == 2) {
    if (c->solve_seg && f.PHf && f.seg && f.seg_m > 0 && kz_fac == c->Kz && m0_shift == 0) {
      const int keep_s = (step == MLX_STEP_ABCN && c->solve_keep_s) ? 1 : 0;
      const bool whole = f.seg_m == c->M;           // else the staged solve takes m >= seg_m
      cudaError_t lerr = cudaSuccess;
      auto go = [&](auto seg_tag) -> bool {
        constexpr int S = decltype(seg_tag)::value;
        const bool np = f.nopiv && f.RNP;
        const bool df = np && c->solve_df && f.RDF && c->precision != MLX_FP64;
        const size_t pw = SegSmem<KL, S>::per_warp(c->nc, keep_s, np);
        int WPB = S;                                // S warps per CTA, halved until the CTA fits 200 KB
        while (WPB > 1 && pw * WPB > 200 * 1024) WPB /= 2;
        if (pw * WPB > 200 * 1024) return false;
        const int G = SegSmem<KL, S>::G;
        const int gpm = (c->Kz + G - 1) / G;
        const int warps = f.seg_m * gpm;
        auto kern = df ? k_band_solve_seg<KL, S, true, true>
                       : (np ? k_band_solve_seg<KL, S, true> : k_band_solve_seg<KL, S, false>);
        const int pair = WPB == 8 ? 1 : 0;
        const int blocks = pair ? ((warps + 1) / 2 + 3) / 4 : (warps + WPB - 1) / WPB;
        lerr = launch_pdl(kern, dim3(blocks), dim3(32 * WPB), pw * WPB, st,
                          f.seg_m, c->nc, c->Kz, c->K, gpm, step, keep_s, c->dt, c->d_soff, fac_off, f.U, f.L,
                          f.piv, f.invd, f.PHf, f.PHb, df ? (const double*)f.PSDF : f.PSf,
                          df ? (const double*)f.RDF : f.RNP, (const double*)s, (const double*)A,
                          (const double*)Ap, (double*)out, (sp && whole) ? *sp : SplitPlanes(), pair);
        if (wrote && sp && sp->bs && whole) *wrote = true;
        return true;
      };
      if (f.seg == 8 ? go(std::integral_constant<int, 8>()) : go(std::integral_constant<int, 4>())) {
        if (lerr != cudaSuccess) { c->last_err = cudaGetErrorString(lerr); return MLX_ECUDA; }
        if (whole) return MLX_OK;
        seg_done = f.seg_m;                         // the staged solve below takes the rest
      }
    }
  }
  // Chains per warp and warps per CTA are launch-shape parameters (measured best
  // at the 128x128x64 workload: 8 chains per warp, 1-4 warps per CTA).
  // seg_done > 0: the orders m < seg_done were solved by the segmented kernel.
  int CPW = c->solve_cpw;
  const int keep_s = (step == MLX_STEP_ABCN && c->solve_keep_s) ? 1 : 0;
  while (CPW > 4 && SolveSmem<KL>::per_warp(c->nc, CPW, keep_s) > 200 * 1024) CPW /= 2;
  const size_t pw = SolveSmem<KL>::per_warp(c->nc, CPW, keep_s);
  int WPB = c->solve_wpb;
  while (WPB > 1 && pw * WPB > 200 * 1024) WPB /= 2;
  if (pw * WPB > 200 * 1024) return MLX_EINVAL;
  const int gpm = (c->Kz + CPW / 4 - 1) / (CPW / 4);
  const int warps = (c->M - seg_done) * gpm;
  const int blocks = (warps + WPB - 1) / WPB;
  k_band_solve<KL><<<blocks, 32 * WPB, pw * WPB, st>>>(
      c->M, c->nc, c->Kz, c->K, CPW, gpm, step, keep_s, c->dt, c->d_soff, fac_off, kz_fac, m0_shift, f.U, f.L,
      f.piv, f.invd, (const double*)s, (const double*)A, (const double*)Ap, (double*)out, seg_done * gpm);
  return MLX_OK;
}

int mlx_band_solve(mlx_ctx* c, int step, const double2* s, const double2* A, const double2* Ap,
                   double2* out, cudaStream_t st, int nfields, const SplitPlanes* sp, bool* wrote) {
  TimedLaunch tl(c, KID_BAND_SOLVE, st);
  const BandLU& f = (step == MLX_STEP_FEBE_FULL) ? c->lu_full : c->lu_half;
  int rc;
  const long long* fo = c->d_band_off;
  if (wrote) *wrote = false;
  switch (c->kl) {
    case 2: rc = launch_solve<2>(c, step, f, fo, c->Kz, 0, s, A, Ap, out, st, nfields, sp, wrote); break;
    case 4: rc = launch_solve<4>(c, step, f, fo, c->Kz, 0, s, A, Ap, out, st, nfields); break;
    case 6: rc = launch_solve<6>(c, step, f, fo, c->Kz, 0, s, A, Ap, out, st, nfields); break;
    case 8: rc = launch_solve<8>(c, step, f, fo, c->Kz, 0, s, A, Ap, out, st, nfields); break;
    default: return MLX_EINVAL;
  }
  if (rc) return rc;
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

// Laplacian-family factors (horizontal Laplacian per m, Helmholtz per (m, |k|)).
int mlx_lap_setup(mlx_ctx* c, cudaStream_t st) {
  if (c->lap_ready) return MLX_OK;
  const long long rows_lap = c->tri, rows_helm = c->band_rows;
  for (BandLU* f : {&c->lu_lap, &c->lu_helm}) {
    const long long rows = (f == &c->lu_lap) ? rows_lap : rows_helm;
    MLX_CUDA_TRY(c, cudaMalloc(&f->U, sizeof(double) * rows * 5));
    MLX_CUDA_TRY(c, cudaMalloc(&f->L, sizeof(double) * rows * 2));
    MLX_CUDA_TRY(c, cudaMalloc(&f->piv, sizeof(int) * rows));
    MLX_CUDA_TRY(c, cudaMalloc(&f->invd, sizeof(double) * rows));
  }
  std::vector<long long> lrows(c->M + 1, 0);
  for (int m = 0; m < c->M; ++m) lrows[m + 1] = lrows[m] + (c->nc - m);
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_lap_off, sizeof(long long) * (c->M + 1)));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(c->d_lap_off, lrows.data(), sizeof(long long) * (c->M + 1),
                                  cudaMemcpyHostToDevice, st));
  const long long stride = (long long)c->nc * (5 + 7);
  double* scratch = nullptr;
  MLX_CUDA_TRY(c, cudaMalloc(&scratch, sizeof(double) * stride * c->M * c->Kz));
  const int tb = 64;
  k_lap_setup<<<(c->M + tb - 1) / tb, tb, 0, st>>>(c->M, c->nc, c->Kz, c->lz, 0, c->d_lap_off, c->d_lap_off,
                                                  c->d_lap, c->lu_lap.U, c->lu_lap.L, c->lu_lap.piv,
                                                  c->lu_lap.invd, scratch, stride);
  MLX_LAUNCH_CHECK(c);
  k_lap_setup<<<(c->M * c->Kz + tb - 1) / tb, tb, 0, st>>>(c->M, c->nc, c->Kz, c->lz, 1, c->d_band_off,
                                                          c->d_lap_off, c->d_lap, c->lu_helm.U, c->lu_helm.L,
                                                          c->lu_helm.piv, c->lu_helm.invd, scratch, stride);
  MLX_LAUNCH_CHECK(c);
  int rc = mlx_pack_lean(c, c->lu_lap, 2, c->d_lap_off, 1, rows_lap, st);
  if (!rc) rc = mlx_pack_lean(c, c->lu_helm, 2, c->d_band_off, c->Kz, rows_helm, st);
  if (rc) { cudaFree(scratch); return rc; }
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  cudaFree(scratch);
  c->lap_ready = true;
  return MLX_OK;
}

// Plain solves with the Laplacian-family factors: family 0 = D_m (decay row at
// m = 0), 1 = D_m - kappa^2.
// Projection factors of the vortex term (families Q, H per m; G per (m, |k|)).
int mlx_proj_setup(mlx_ctx* c, cudaStream_t st) {
  if (c->proj_ready) return MLX_OK;
  const int W = 7, kl = 3;
  BandLU* fams[3] = {&c->lu_Q, &c->lu_H, &c->lu_G};
  for (int f = 0; f < 3; ++f) {
    const long long rows = (f == 2) ? c->band_rows : c->tri;
    MLX_CUDA_TRY(c, cudaMalloc(&fams[f]->U, sizeof(double) * rows * W));
    MLX_CUDA_TRY(c, cudaMalloc(&fams[f]->L, sizeof(double) * rows * kl));
    MLX_CUDA_TRY(c, cudaMalloc(&fams[f]->piv, sizeof(int) * rows));
    MLX_CUDA_TRY(c, cudaMalloc(&fams[f]->invd, sizeof(double) * rows));
  }
  const long long stride = (long long)c->nc * (2 * W + 3 * kl + 1);
  double* scratch = nullptr;
  MLX_CUDA_TRY(c, cudaMalloc(&scratch, sizeof(double) * stride * c->M * c->Kz));
  const int tb = 64;
  for (int f = 0; f < 3; ++f) {
    const int nsys = (f == 2) ? c->M * c->Kz : c->M;
    k_proj_setup<<<(nsys + tb - 1) / tb, tb, 0, st>>>(c->M, c->nc, c->Kz, c->lz, c->ell, f,
                                                      f == 2 ? c->d_band_off : c->d_lap_off, fams[f]->U,
                                                      fams[f]->L, fams[f]->piv, fams[f]->invd, scratch, stride);
    MLX_LAUNCH_CHECK(c);
    const int rc = (f == 2) ? mlx_pack_lean(c, *fams[f], kl, c->d_band_off, c->Kz, c->band_rows, st)
                            : mlx_pack_lean(c, *fams[f], kl, c->d_lap_off, 1, c->tri, st);
    if (rc) { cudaFree(scratch); return rc; }
  }
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  cudaFree(scratch);
  c->proj_ready = true;
  return MLX_OK;
}

// Plain solves with the projection factors: family 0 = Q, 1 = H (decay row at
// m = 0), 2 = G.
int mlx_proj_solve(mlx_ctx* c, int family, const double2* rhs, double2* out, cudaStream_t st) {
  TimedLaunch tl(c, KID_BAND_SOLVE, st);
  int rc;
  if (family == 0) rc = launch_solve<3>(c, MLX_STEP_PLAIN, c->lu_Q, c->d_lap_off, 1, 1, rhs, nullptr, nullptr, out, st);
  else if (family == 1) rc = launch_solve<3>(c, MLX_STEP_PLAIN, c->lu_H, c->d_lap_off, 1, 1, rhs, nullptr, nullptr, out, st);
  else rc = launch_solve<3>(c, MLX_STEP_PLAIN, c->lu_G, c->d_band_off, c->Kz, 0, rhs, nullptr, nullptr, out, st);
  if (rc) return rc;
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

int mlx_lap_solve(mlx_ctx* c, int family, const double2* rhs, double2* out, cudaStream_t st) {
  TimedLaunch tl(c, KID_BAND_SOLVE, st);
  int rc = (family == 0)
               ? launch_solve<2>(c, MLX_STEP_PLAIN, c->lu_lap, c->d_lap_off, 1, 1, rhs, nullptr, nullptr, out, st)
               : launch_solve<2>(c, MLX_STEP_PLAIN, c->lu_helm, c->d_band_off, c->Kz, 0, rhs, nullptr, nullptr,
                                 out, st);
  if (rc) return rc;
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

template <int KL, int NF>
static int set_lean_attrs_nf(mlx_ctx* c, int lim) {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_lean<KL, 16, LEAN_PLAIN, NF>, at, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_lean<KL, 16, LEAN_FEBE, NF>, at, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_lean<KL, 16, LEAN_ABCN, NF>, at, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_lean<KL, 32, LEAN_PLAIN, NF>, at, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_lean<KL, 32, LEAN_FEBE, NF>, at, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_lean<KL, 32, LEAN_ABCN, NF>, at, lim));
  return MLX_OK;
}
template <int KL>
static int set_lean_attrs(mlx_ctx* c, int lim) {
  const int rc = set_lean_attrs_nf<KL, 1>(c, lim);
  return rc ? rc : set_lean_attrs_nf<KL, 2>(c, lim);
}

// Segmented-solve influence data of an implicit-step factor family for S segments
// (S = 0 frees it), half width 2 only.  A system can be cut when every segment has
// at least 2 kl rows, N = Nc - m >= 2 kl S: the data cover the orders m < seg_m
// (the longest systems), and the staged solve takes the rest.  S = 8 falls back to
// 4 when 4 segments reach every order and 8 do not, or when 8 reach none.
__global__ void k_to_df(long long n, const double* __restrict__ src, dfl* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double v = src[i];
    dst[i] = df_from_double(v);
  }
}
void mlx_to_df(const double* src, void* dst, long long n, cudaStream_t st) {
  if (n > 0) k_to_df<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, src, reinterpret_cast<dfl*>(dst));
}

int mlx_seg_build(mlx_ctx* c, BandLU& f, int S, cudaStream_t st) {
  cudaFree(f.PHf); cudaFree(f.PHb); cudaFree(f.PSf); cudaFree(f.RNP); cudaFree(f.RDF); cudaFree(f.PSDF);
  f.PHf = f.PHb = f.PSf = f.RNP = nullptr;
  f.RDF = f.PSDF = nullptr;
  f.seg = 0;
  f.seg_m = 0;
  const int kl = c->kl;
  auto cover = [&](int s_) { return std::max(0, std::min(c->M, c->nc - s_ * 2 * kl + 1)); };
  if (S == 8 && cover(8) < c->M && cover(4) == c->M) S = 4;
  if (S == 8 && cover(8) == 0) S = 4;
  if (S == 0 || kl != 2 || !f.U || cover(S) == 0) return MLX_OK;
  const int segm = cover(S);
  const long long rows = c->band_rows;
  MLX_CUDA_TRY(c, cudaMalloc(&f.PHf, sizeof(double) * rows * kl));
  MLX_CUDA_TRY(c, cudaMalloc(&f.PHb, sizeof(double) * rows * 2 * kl));
  MLX_CUDA_TRY(c, cudaMalloc(&f.PSf, sizeof(double) * (long long)c->M * c->Kz * S * kl * kl));
  const long long nt = (long long)segm * c->Kz * S * 3 * kl;
  if (S == 8)
    k_seg_setup<2, 8><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(segm, c->nc, c->Kz, c->d_band_off, f.U,
                                                                    f.L, f.piv, f.PHf, f.PHb, f.PSf);
  else
    k_seg_setup<2, 4><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(segm, c->nc, c->Kz, c->d_band_off, f.U,
                                                                    f.L, f.piv, f.PHf, f.PHb, f.PSf);
  MLX_LAUNCH_CHECK(c);
  if (f.nopiv) {
    MLX_CUDA_TRY(c, cudaMalloc(&f.RNP, sizeof(double) * rows * SegSmem<2, 8>::RW));
    dim3 grid((unsigned)(((long long)c->Kz * c->nc + 127) / 128), segm);
    k_pack_seg_np<2><<<grid, 128, 0, st>>>(c->nc, c->Kz, c->d_band_off, f.U, f.L, f.invd, f.PHf, f.PHb, f.RNP);
    MLX_LAUNCH_CHECK(c);
    if (c->precision != MLX_FP64) {
      const long long nr = rows * SegSmem<2, 8>::RW, np = (long long)c->M * c->Kz * S * kl * kl;
      MLX_CUDA_TRY(c, cudaMalloc(&f.RDF, sizeof(dfl) * nr));
      MLX_CUDA_TRY(c, cudaMalloc(&f.PSDF, sizeof(dfl) * np));
      mlx_to_df(f.RNP, f.RDF, nr, st);
      mlx_to_df(f.PSf, f.PSDF, np, st);
      MLX_LAUNCH_CHECK(c);
    }
  }
  f.seg = S;
  f.seg_m = segm;
  return MLX_OK;
}

// Lean-solve records (FS, BS) of a factor family just factorised on stream st.
int mlx_pack_lean(mlx_ctx* c, BandLU& f, int kl, const long long* d_off, int kz_fac, long long rows,
                  cudaStream_t st) {
  const int FW = (kl + 2) & ~1, BW = 2 * kl + 2;
  cudaFree(f.FS);
  cudaFree(f.BS);
  f.FS = f.BS = nullptr;
  MLX_CUDA_TRY(c, cudaMalloc(&f.FS, sizeof(double) * rows * FW));
  MLX_CUDA_TRY(c, cudaMalloc(&f.BS, sizeof(double) * rows * BW));
  const int kcnt = (kz_fac == 1) ? 1 : c->Kz;
  const dim3 grid((unsigned)(((long long)c->nc * kcnt + 127) / 128), (unsigned)c->M);
  k_pack_lean<<<grid, 128, 0, st>>>(c->nc, kcnt, kz_fac, kl, d_off, f.U, f.L, f.piv, f.invd, f.FS, f.BS);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

// Scratch of the lean solve: [warp][Nc][CPW] doubles, one warp per (m, CPW / 4 |k|),
// sized for either chain count (16 or 32).
int mlx_solve_scratch(mlx_ctx* c) {
  if (c->d_solve_y) return MLX_OK;
  // [warp][Nc][CPW]: the largest warp count of the variants (32 or 16 chains per warp,
  // one or two fields per launch: 4 NF chains per |k|)
  long long w = 0;
  for (int cpw : {16, 32})
    for (int nf : {1, 2}) {
      const int g = cpw / (4 * nf);
      const long long v = (long long)((c->Kz + g - 1) / g) * cpw;
      w = v > w ? v : w;
    }
  const long long elems = (long long)c->M * c->nc * w;
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_solve_y, sizeof(double) * elems));
  return MLX_OK;
}

int mlx_band_prepare(mlx_ctx* c) {
  const int lim = 200 * 1024;
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_seg<2, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_seg<2, 8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_seg<2, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_seg<2, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_seg<2, 4, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve_seg<2, 8, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  {
    int rc = set_lean_attrs<2>(c, lim);
    if (!rc) rc = set_lean_attrs<3>(c, lim);
    if (!rc) rc = set_lean_attrs<4>(c, lim);
    if (!rc) rc = set_lean_attrs<6>(c, lim);
    if (!rc) rc = set_lean_attrs<8>(c, lim);
    if (rc) return rc;
  }
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_band_solve<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return MLX_OK;
}

int mlx_spec_axpby(mlx_ctx* c, double a, const double2* x, double b, const double2* y,
                   double2* out, cudaStream_t st, long long nn) {
  TimedLaunch tl(c, KID_AXPBY, st);
  const long long n = nn < 0 ? c->n_spec : nn;
  const int tb = 256;
  k_axpby<<<(unsigned)((n + tb - 1) / tb), tb, 0, st>>>(n, a, x, b, y, out);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

// ---- batched persistent staged solve (batch.cu) ----
// Job and warp items of member c (index inst) for one AB-CN solve s, A, Ap -> out
// (A, Ap may be NULL), half width c->kl; *slab: the member's shared memory per warp.
// Az (may be NULL): a buffer the solve fills with zeros (the A^j of a member
// without a nonlinear term).  planes: the segmented variant also writes the BF16x3
// split planes of out into the member's backward data operand when it covers every
// order (*wrote_planes tells whether it will).  The member's solve becomes one or
// two parts, as its single-context launch would split it: the segmented variant
// for the orders m < seg_m, the staged one (its chains per warp) for the rest.
void mlx_band_batch_member(mlx_ctx* c, const double2* s, const double2* A, const double2* Ap, double2* out,
                           double2* Az, bool planes, std::vector<BSolvePart>& parts, bool* wrote_planes) {
  auto per_warp = [&](int cpw) -> size_t {
    switch (c->kl) {
      case 2: return SolveSmem<2>::per_warp(c->nc, cpw, 0);
      case 4: return SolveSmem<4>::per_warp(c->nc, cpw, 0);
      case 6: return SolveSmem<6>::per_warp(c->nc, cpw, 0);
      default: return SolveSmem<8>::per_warp(c->nc, cpw, 0);
    }
  };
  const BandLU& f = c->lu_half;
  const bool seg = c->kl == 2 && c->solve_seg && f.PHf && f.seg && f.seg_m > 0;
  const bool np = seg && f.nopiv && f.RNP;
  const bool df = np && c->solve_df && f.RDF && c->precision != MLX_FP64;
  const int mseg = seg ? f.seg_m : 0;
  BSolveJob base;
  memset(&base, 0, sizeof(base));
  base.M = c->M; base.nc = c->nc; base.Kz = c->Kz; base.K = c->K;
  base.step = MLX_STEP_ABCN;
  base.kz_fac = c->Kz;
  base.dt = c->dt;
  base.soff = c->d_soff; base.band_off = c->d_band_off;
  base.U = f.U; base.L = f.L; base.piv = f.piv; base.invd = f.invd;
  base.s = (const double*)s; base.A = (const double*)A; base.Ap = (const double*)Ap; base.out = (double*)out;
  base.Az = (double*)Az;
  *wrote_planes = false;
  if (seg) {
    BSolvePart pt;
    pt.job = base;
    BSolveJob& j = pt.job;
    j.variant = (f.seg == 8 ? 1 : 2) + (df ? 4 : (np ? 2 : 0));
    j.M = mseg;                      // the segmented kernel's orders
    j.CPW = 32 / f.seg;
    j.gpm = (c->Kz + j.CPW / 4 - 1) / (j.CPW / 4);
    j.PHf = f.PHf; j.PHb = f.PHb;
    j.PSf = df ? (const double*)f.PSDF : f.PSf;
    j.RNP = df ? (const double*)f.RDF : f.RNP;
    if (planes && mseg == c->M && c->precision == MLX_BF16X3 && c->d_bsb) {
      j.bs = reinterpret_cast<unsigned short*>(c->d_bsb);
      j.kq = (int)c->tc_kq;
      j.k2 = 2 * c->K;
      j.part = (long long)c->M * j.k2 * j.kq;
      *wrote_planes = true;
    }
    pt.slab = (int)(f.seg == 8 ? SegSmem<2, 8>::per_warp(c->nc, 0, np) : SegSmem<2, 4>::per_warp(c->nc, 0, np));
    for (int gw = 0; gw < mseg * j.gpm; ++gw) {
      pt.items.push_back(make_int2(0, gw));
      pt.cost.push_back((double)(c->nc - gw / j.gpm));
    }
    parts.push_back(pt);
  }
  if (mseg < c->M) {
    BSolvePart pt;
    pt.job = base;
    BSolveJob& j = pt.job;
    int CPW = c->solve_cpw;
    while (CPW > 4 && per_warp(CPW) > 200 * 1024) CPW /= 2;
    j.variant = 0;
    j.CPW = CPW;
    j.gpm = (c->Kz + CPW / 4 - 1) / (CPW / 4);
    pt.slab = (int)per_warp(CPW);
    for (int gw = mseg * j.gpm; gw < c->M * j.gpm; ++gw) {
      pt.items.push_back(make_int2(0, gw));
      pt.cost.push_back((double)(c->nc - gw / j.gpm));
    }
    parts.push_back(pt);
  }
}

// the kernel of a batched solve group: variant 0 staged (half width kl), 1 / 2
// segmented with 8 / 4 segments, 3 / 4 the same in the pivot-free form, 5 / 6
// pivot-free in double-float arithmetic
const void* mlx_band_batch_kernel(int kl, int variant) {
  switch (variant) {
    case 1: return (const void*)kb_band_solve_seg<2, 8, false>;
    case 2: return (const void*)kb_band_solve_seg<2, 4, false>;
    case 3: return (const void*)kb_band_solve_seg<2, 8, true>;
    case 4: return (const void*)kb_band_solve_seg<2, 4, true>;
    case 5: return (const void*)kb_band_solve_seg<2, 8, true, true>;
    case 6: return (const void*)kb_band_solve_seg<2, 4, true, true>;
    default: break;
  }
  switch (kl) {
    case 2: return (const void*)kb_band_solve<2>;
    case 4: return (const void*)kb_band_solve<4>;
    case 6: return (const void*)kb_band_solve<6>;
    case 8: return (const void*)kb_band_solve<8>;
    default: return nullptr;
  }
}

int mlx_band_batch_launch(int kl, int variant, const BSolveJob* jobs, const int2* items, int nitems, int slab,
                          int wpb, int* ctr, int grid, cudaStream_t st) {
  const size_t smem = (size_t)slab * wpb;
  switch (variant) {
    case 1: kb_band_solve_seg<2, 8, false><<<grid, 32 * wpb, smem, st>>>(jobs, items, nitems, slab, ctr); break;
    case 2: kb_band_solve_seg<2, 4, false><<<grid, 32 * wpb, smem, st>>>(jobs, items, nitems, slab, ctr); break;
    case 3: kb_band_solve_seg<2, 8, true><<<grid, 32 * wpb, smem, st>>>(jobs, items, nitems, slab, ctr); break;
    case 4: kb_band_solve_seg<2, 4, true><<<grid, 32 * wpb, smem, st>>>(jobs, items, nitems, slab, ctr); break;
    case 5: kb_band_solve_seg<2, 8, true, true><<<grid, 32 * wpb, smem, st>>>(jobs, items, nitems, slab, ctr); break;
    case 6: kb_band_solve_seg<2, 4, true, true><<<grid, 32 * wpb, smem, st>>>(jobs, items, nitems, slab, ctr); break;
    default: break;
  }
  if (variant) return cudaGetLastError() == cudaSuccess ? MLX_OK : MLX_ECUDA;
  switch (kl) {
    case 2: kb_band_solve<2><<<grid, 32 * wpb, smem, st>>>(jobs, items, nitems, slab, ctr); break;
    case 4: kb_band_solve<4><<<grid, 32 * wpb, smem, st>>>(jobs, items, nitems, slab, ctr); break;
    case 6: kb_band_solve<6><<<grid, 32 * wpb, smem, st>>>(jobs, items, nitems, slab, ctr); break;
    case 8: kb_band_solve<8><<<grid, 32 * wpb, smem, st>>>(jobs, items, nitems, slab, ctr); break;
    default: return MLX_EINVAL;
  }
  return cudaGetLastError() == cudaSuccess ? MLX_OK : MLX_ECUDA;
}
