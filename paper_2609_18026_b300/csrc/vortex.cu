// K5 (vortex): the toroidal-poloidal nonlinear term P[(U + v) x omega] of Eq. (19)
// (Sec. 3.2, Sec. 5.3), harmonic by harmonic with the banded r d/dr (R) and
// horizontal Laplacian (D_m) of Sec. 3.1:
//   r v_r = i m psi + i kappa R chi        r w_r = i m Psi + i kappa R psi
//   r v_phi = -R psi - m kappa chi         r w_phi = -R Psi - m kappa psi
//   v_z = -D_m chi                         w_z = -D_m psi,   Psi = -(D_m - kappa^2) chi
// Six backward transforms; at the nodes N = (v + U) x omega with U = U0 e_y:
//   A = r N_phi, B = r N_r, C = r^2 N_z (no division by r anywhere: near the axis
//   a division by r^2 would amplify transform round-off by 1/r_min^2).
// Three forward transforms; in coefficient space X1 = R A - i m B (= r^2 (curl N)_z),
// X2 = R B + i m A (= r^2 div_h N), and with J = multiplication by x,
// Q = (I - J^2) diag(-n(n+1)) = r^2 lap_h and (1 - x) r^2 = ell^2 (1 + x):
//   Q psi_N = -X1
//   [(I - J) Q - kappa^2 ell^2 (I + J)] g = (I - J)(X2 + i kappa C)     (k != 0)
//   (I - J) Q chi_N = i kappa ell^2 (I + J) g - (I - J) C               (g = 0 at k = 0)
// with the far-field decay condition replacing the singular first row at m = 0.
//
// Log proxies (Sec. 3.1, Eq. (6)): a flow with net circulation or net axial flux
// carries psi = c_psi Lambda + ..., chi = c_chi Lambda + ... with
// Lambda = ln(r^2 + ell^2).  The proxies' r-weighted velocity and vorticity are
// polynomials of degree <= 3 in x at (m, k) = (0, 0) and are added to those blocks
// of the fields; the background is U = U0 e_y + Uz e_z.
#include "mlx_internal.cuh"
#include "bf16_split.cuh"
#include "df.cuh"

#include <cmath>

namespace {

__device__ __forceinline__ double kappa_of(int kidx, int Kz, int K, double lz) {
  const int k = kidx < Kz ? kidx : kidx - K;
  return 2.0 * M_PI * k / lz;
}

// locate the order m of a flat spectral index by the offset table (M <= 1024)
__device__ __forceinline__ int m_of(long long idx, const long long* soff, int M) {
  int lo = 0, hi = M;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (soff[mid] <= idx) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double2 cmulr(double a, double2 v) { return make_double2(a * v.x, a * v.y); }
__device__ __forceinline__ double2 cimul(double a, double2 v) { return make_double2(-a * v.y, a * v.x); } // i a v
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// Band applications at row n (local index a = n - m) of one (m, k) vector v of length Nm.
__device__ __forceinline__ double2 apply_R(const double* rb, const double2* v, int a, int Nm) {
  double2 r = make_double2(0.0, 0.0);
  if (a - 1 >= 0) r = cadd(r, cmulr(rb[a * 2 + 0], v[a - 1]));
  if (a + 1 < Nm) r = cadd(r, cmulr(rb[a * 2 + 1], v[a + 1]));
  return r;
}
__device__ __forceinline__ double2 apply_D(const double* db, const double2* v, int a, int Nm) {
  double2 r = make_double2(0.0, 0.0);
#pragma unroll
  for (int o = -2; o <= 2; ++o)
    if (a + o >= 0 && a + o < Nm) r = cadd(r, cmulr(db[a * 5 + o + 2], v[a + o]));
  return r;
}

// One CTA per (m, k) vector: psi and chi are staged in shared memory once, D_m chi
// and Psi = -(D_m - kappa^2) chi are formed once per entry, and the six fields are
// read off the staged vectors (no band product is evaluated twice).
__global__ void k_vortex_fields(int nc, int Kz, int K, double lz, const long long* __restrict__ soff,
                                const long long* __restrict__ rows, const double* __restrict__ rdr,
                                const double* __restrict__ lap, const double2* __restrict__ psi,
                                const double2* __restrict__ chi, double2* __restrict__ rvr,
                                double2* __restrict__ rvp, double2* __restrict__ vz, double2* __restrict__ rwr,
                                double2* __restrict__ rwp, double2* __restrict__ wz,
                                const double* __restrict__ lpf, SplitPlanes vp) {
  extern __shared__ double2 vsh[];   // [4][nc]: psi, chi, D chi, Psi
  const int kidx = blockIdx.x, m = blockIdx.y;
  const int Nm = nc - m;
  const long long base = soff[m] + (long long)kidx * Nm;
  double2* P = vsh;
  double2* Ch = vsh + nc;
  double2* Dc = vsh + 2 * nc;
  double2* Ps = vsh + 3 * nc;
  for (int a = threadIdx.x; a < Nm; a += blockDim.x) { P[a] = psi[base + a]; Ch[a] = chi[base + a]; }
  __syncthreads();
  const double kap = kappa_of(kidx, Kz, K, lz);
  const double* rb = rdr + rows[m] * 2;
  const double* db = lap + rows[m] * 5;
  for (int a = threadIdx.x; a < Nm; a += blockDim.x) {
    const double2 d = apply_D(db, Ch, a, Nm);
    Dc[a] = d;
    Ps[a] = csub(cmulr(kap * kap, Ch[a]), d);
  }
  __syncthreads();
  const double mm = (double)m;
  for (int a = threadIdx.x; a < Nm; a += blockDim.x) {
    const long long idx = base + a;
    const double2 Rpsi = apply_R(rb, P, a, Nm);
    const double2 Rchi = apply_R(rb, Ch, a, Nm);
    const double2 RPsi = apply_R(rb, Ps, a, Nm);
    double2 fvp = csub(cmulr(-1.0, Rpsi), cmulr(mm * kap, Ch[a]));
    double2 fvz = cmulr(-1.0, Dc[a]);
    double2 fwp = csub(cmulr(-1.0, RPsi), cmulr(mm * kap, P[a]));
    double2 fwz = cmulr(-1.0, apply_D(db, P, a, Nm));
    if (lpf && m == 0 && kidx == 0 && a < 4) {   // log proxies: real coefficients, n <= 3
      fvp.x += lpf[a];
      fvz.x += lpf[4 + a];
      fwp.x += lpf[8 + a];
      fwz.x += lpf[12 + a];
    }
    const double2 fvr = cadd(cimul(mm, P[a]), cimul(kap, Rchi));
    const double2 fwr = cadd(cimul(mm, Ps[a]), cimul(kap, Rpsi));
    if (vp.bs) {
      // BF16X3: the six fields straight into their split planes (the backward
      // contraction's data operands), as k_split_spec would write them
      const double2 fv[6] = {fvr, fvp, fvz, fwr, fwp, fwz};
      const long long o = ((long long)m * vp.K2 + 2 * kidx) * vp.Kq + a;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        unsigned short* b = vp.bs + (long long)f * 3 * vp.part;
        unsigned short h, md, lo;
        split3_f64(fv[f].x, h, md, lo);
        b[o] = h; b[vp.part + o] = md; b[2 * vp.part + o] = lo;
        split3_f64(fv[f].y, h, md, lo);
        b[o + vp.Kq] = h; b[vp.part + o + vp.Kq] = md; b[2 * vp.part + o + vp.Kq] = lo;
      }
    } else {
      rvr[idx] = fvr;
      rvp[idx] = fvp;
      vz[idx] = fvz;
      rwr[idx] = fwr;
      rwp[idx] = fwp;
      wz[idx] = fwz;
    }
  }
}

// The mixed-precision forms' fields kernel: the same operations in double-float
// arithmetic (about 48 bits; the fields are rounded to FP32 for the transforms
// afterwards), so that the band products run on the FP32 pipe.  The state and the
// proxy terms arrive in FP64 and are split into hi + lo by integer operations; the
// bands were converted once at setup.  Outputs as k_vortex_fields: the FP32 rounding
// of each field into the split planes (vp.bs), or hi + lo as FP64 fields.
__device__ __forceinline__ dfl2 apply_R_df(const dfl* rb, const dfl2* v, int a, int Nm) {
  dfl2 r = dfc_make(df_make(0.f, 0.f), df_make(0.f, 0.f));
  if (a - 1 >= 0) r = dfc_fma(rb[a * 2 + 0], v[a - 1], r);
  if (a + 1 < Nm) r = dfc_fma(rb[a * 2 + 1], v[a + 1], r);
  return r;
}
__device__ __forceinline__ dfl2 apply_D_df(const dfl* db, const dfl2* v, int a, int Nm) {
  dfl2 r = dfc_make(df_make(0.f, 0.f), df_make(0.f, 0.f));
#pragma unroll
  for (int o = -2; o <= 2; ++o)
    if (a + o >= 0 && a + o < Nm) r = dfc_fma(db[a * 5 + o + 2], v[a + o], r);
  return r;
}

__global__ void k_vortex_fields_df(int nc, int Kz, int K, double lz, const long long* __restrict__ soff,
                                   const long long* __restrict__ rows, const dfl* __restrict__ rdr,
                                   const dfl* __restrict__ lap, const double2* __restrict__ psi,
                                   const double2* __restrict__ chi, double2* __restrict__ rvr,
                                   double2* __restrict__ rvp, double2* __restrict__ vz, double2* __restrict__ rwr,
                                   double2* __restrict__ rwp, double2* __restrict__ wz,
                                   const double* __restrict__ lpf, SplitPlanes vp) {
  extern __shared__ dfl2 vdf[];   // [4][nc]: psi, chi, D chi, Psi
  const int kidx = blockIdx.x, m = blockIdx.y;
  const int Nm = nc - m;
  const long long base = soff[m] + (long long)kidx * Nm;
  dfl2* P = vdf;
  dfl2* Ch = vdf + nc;
  dfl2* Dc = vdf + 2 * nc;
  dfl2* Ps = vdf + 3 * nc;
  for (int a = threadIdx.x; a < Nm; a += blockDim.x) {
    P[a] = dfc_from(psi[base + a]);
    Ch[a] = dfc_from(chi[base + a]);
  }
  __syncthreads();
  const dfl kap = df_from_double(kappa_of(kidx, Kz, K, lz));
  const dfl kap2 = df_mul(kap, kap);
  const dfl mm = df_make((float)m, 0.f);
  const dfl mk = df_mul(mm, kap);
  const dfl* rb = rdr + rows[m] * 2;
  const dfl* db = lap + rows[m] * 5;
  for (int a = threadIdx.x; a < Nm; a += blockDim.x) {
    const dfl2 d = apply_D_df(db, Ch, a, Nm);
    Dc[a] = d;
    Ps[a] = dfc_sub(dfc_scale(kap2, Ch[a]), d);
  }
  __syncthreads();
  for (int a = threadIdx.x; a < Nm; a += blockDim.x) {
    const long long idx = base + a;
    const dfl2 Rpsi = apply_R_df(rb, P, a, Nm);
    const dfl2 Rchi = apply_R_df(rb, Ch, a, Nm);
    const dfl2 RPsi = apply_R_df(rb, Ps, a, Nm);
    const dfl2 D_psi = apply_D_df(db, P, a, Nm);
    dfl2 fv[6];
    fv[0] = dfc_add(dfc_iscale(mm, P[a]), dfc_iscale(kap, Rchi));                       // r v_r
    fv[1] = dfc_sub(dfc_make(df_neg(Rpsi.re), df_neg(Rpsi.im)), dfc_scale(mk, Ch[a]));  // r v_phi
    fv[2] = dfc_make(df_neg(Dc[a].re), df_neg(Dc[a].im));                               // v_z
    fv[3] = dfc_add(dfc_iscale(mm, Ps[a]), dfc_iscale(kap, Rpsi));                      // r w_r
    fv[4] = dfc_sub(dfc_make(df_neg(RPsi.re), df_neg(RPsi.im)), dfc_scale(mk, P[a]));   // r w_phi
    fv[5] = dfc_make(df_neg(D_psi.re), df_neg(D_psi.im));                               // w_z
    if (lpf && m == 0 && kidx == 0 && a < 4) {   // log proxies: real coefficients, n <= 3
      fv[1].re = df_add(fv[1].re, df_from_double(lpf[a]));
      fv[2].re = df_add(fv[2].re, df_from_double(lpf[4 + a]));
      fv[4].re = df_add(fv[4].re, df_from_double(lpf[8 + a]));
      fv[5].re = df_add(fv[5].re, df_from_double(lpf[12 + a]));
    }
    if (vp.bs) {
      const long long o = ((long long)m * vp.K2 + 2 * kidx) * vp.Kq + a;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        unsigned short* b = vp.bs + (long long)f * 3 * vp.part;
        __nv_bfloat16 h, md, lo;
        split3<float>(df_round_f32(fv[f].re), h, md, lo);
        b[o] = __bfloat16_as_ushort(h); b[vp.part + o] = __bfloat16_as_ushort(md);
        b[2 * vp.part + o] = __bfloat16_as_ushort(lo);
        split3<float>(df_round_f32(fv[f].im), h, md, lo);
        b[o + vp.Kq] = __bfloat16_as_ushort(h); b[vp.part + o + vp.Kq] = __bfloat16_as_ushort(md);
        b[2 * vp.part + o + vp.Kq] = __bfloat16_as_ushort(lo);
      }
    } else {
      double2* outs[6] = {rvr, rvp, vz, rwr, rwp, wz};
#pragma unroll
      for (int f = 0; f < 6; ++f) outs[f][idx] = make_double2(df_to_double(fv[f].re), df_to_double(fv[f].im));
    }
  }
}

// ---- log-proxy tables -----------------------------------------------------------
// d_lp layout: [16] field additions (r v_phi, v_z, r w_phi, w_z; n = 0..3), [nc] lam =
// lap_h Lambda, [nc] L Lambda, [2 nc] matvec scratch, [1] c of the last solve, then
// [7 nc + 2 nc] scratch of the solve-for-c elimination.
constexpr int kLpFields = 0, kLpLam = 16;
__host__ __device__ inline long long lp_ll(int nc) { return 16 + (long long)nc; }
__host__ __device__ inline long long lp_scr(int nc) { return 16 + 2LL * nc; }
__host__ __device__ inline long long lp_c(int nc) { return 16 + 4LL * nc; }
__host__ __device__ inline long long lp_elim(int nc) { return 17 + 4LL * nc; }
__host__ __device__ inline long long lp_size(int nc) { return 17 + 13LL * nc; }

// (D_0 v)_i with the m = 0 Laplacian band (row i, column i + o - 2)
__device__ double lap0_row(const double* lap0, const double* v, int i, int nc) {
  double acc = 0.0;
  for (int o = 0; o < 5; ++o) {
    const int j = i + o - 2;
    if (j >= 0 && j < nc) acc = fma(lap0[i * 5 + o], v[j], acc);
  }
  return acc;
}

// One thread.  With N_n = sqrt((2n + 1) / 2) (a Legendre sum a_n P_n has the basis
// coefficients a_n / N_n) and the expansions
//   1 + x = P_0 + P_1,  (1 - x)^2 = 4/3 P_0 - 2 P_1 + 2/3 P_2 (Eq. (6)),
//   (1 - x)(1 - x^2) = 2/3 P_0 - 2/5 P_1 - 2/3 P_2 + 2/5 P_3,
// the proxies add  r v_phi = -c_psi (1 + x),  w_z = -c_psi (1 - x)^2 / ell^2,
// v_z = -c_chi (1 - x)^2 / ell^2,  r w_phi = -2 c_chi (1 - x)(1 - x^2) / ell^2, and
// L Lambda = nu lam - nu_h (-1)^{p/2} D_0^{p/2 - 1} lam  (Eq. (11) at (m, k) = (0, 0)).
__global__ void k_lp_setup(int nc, double ell, double cpsi, double cchi, double nu, double nu_h, int p,
                           const double* __restrict__ lap0, double* __restrict__ lp) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double e2 = ell * ell;
  const double sq[4] = {sqrt(0.5), sqrt(1.5), sqrt(2.5), sqrt(3.5)};
  const double onepx[4] = {1.0, 1.0, 0.0, 0.0};
  const double omx2[4] = {4.0 / 3.0, -2.0, 2.0 / 3.0, 0.0};
  const double cub[4] = {2.0 / 3.0, -0.4, -2.0 / 3.0, 0.4};
  for (int n = 0; n < 4; ++n) {
    const bool in = n < nc;
    lp[kLpFields + n] = in ? -cpsi * onepx[n] / sq[n] : 0.0;
    lp[kLpFields + 4 + n] = in ? -cchi * omx2[n] / sq[n] / e2 : 0.0;
    lp[kLpFields + 8 + n] = in ? -2.0 * cchi * cub[n] / sq[n] / e2 : 0.0;
    lp[kLpFields + 12 + n] = in ? -cpsi * omx2[n] / sq[n] / e2 : 0.0;
  }
  double* lam = lp + kLpLam;
  double* LL = lp + lp_ll(nc);
  double* v = lp + lp_scr(nc);
  double* w = v + nc;
  for (int i = 0; i < nc; ++i) {
    lam[i] = i < 3 ? omx2[i] / sq[i] / e2 : 0.0;
    v[i] = lam[i];
    LL[i] = nu * lam[i];
  }
  if (nu_h > 0.0) {
    for (int it = 0; it < p / 2 - 1; ++it) {
      for (int i = 0; i < nc; ++i) w[i] = lap0_row(lap0, v, i, nc);
      for (int i = 0; i < nc; ++i) v[i] = w[i];
    }
    const double sgn = ((p / 2) % 2 == 0) ? 1.0 : -1.0;
    for (int i = 0; i < nc; ++i) LL[i] -= nu_h * sgn * v[i];
  }
}

// the proxies' constant forcing c L Lambda of the (0, 0) blocks of a two-field tendency
__global__ void k_lp_source(int nc, double cpsi, double cchi, const double* __restrict__ LL,
                            double2* __restrict__ Apsi, double2* __restrict__ Achi) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nc) return;
  Apsi[a].x += cpsi * LL[a];
  Achi[a].x += cchi * LL[a];
}

// prescribed-c inversion: the (0, 0) block of the right-hand side minus c lam
__global__ void k_lp_shift(int nc, double cval, const double* __restrict__ lam, double2* __restrict__ f) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < nc) f[a].x -= cval * lam[a];
}

// solve-for-c inversion of the (0, 0) block, one thread: D_0 with its (zero) column 0
// replaced by lam, half width 2 below and (with the fill of partial pivoting) 4
// above, eliminated for the real and imaginary right-hand sides together.  The
// unknown in column 0 is c (from the real part; a real field's (0, 0) block has a
// zero imaginary part, whose column-0 unknown is dropped), and the block's Pbar_0^0
// coefficient is 0.
__global__ void k_lp_solve_c(int nc, const double* __restrict__ lap0, double* __restrict__ lp,
                             const double2* __restrict__ f, double2* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  constexpr int KLO = 2, KUP = 4, WB = KLO + KUP + 1;   // band columns j - i in [-2, 4]
  const double* lam = lp + kLpLam;
  double* ab = lp + lp_elim(nc);                          // [nc][WB]
  double* br = ab + (long long)nc * WB;                   // [nc]
  double* bi = br + nc;                                   // [nc]
  auto at = [&](int i, int j) -> double& { return ab[(long long)i * WB + (j - i + KLO)]; };
  for (int i = 0; i < nc; ++i) {
    for (int o = 0; o < WB; ++o) ab[(long long)i * WB + o] = 0.0;
    for (int o = 0; o < 5; ++o) {
      const int j = i + o - 2;
      if (j >= 1 && j < nc) at(i, j) = lap0[i * 5 + o];
    }
    if (i < 3) at(i, 0) = lam[i];
    br[i] = f[i].x;
    bi[i] = f[i].y;
  }
  for (int k = 0; k < nc; ++k) {
    int piv = k;
    double best = fabs(at(k, k));
    for (int i = k + 1; i <= min(nc - 1, k + KLO); ++i)
      if (fabs(at(i, k)) > best) { best = fabs(at(i, k)); piv = i; }
    if (piv != k) {
      for (int j = k; j <= min(nc - 1, k + KUP); ++j) {
        const double t = at(k, j); at(k, j) = at(piv, j); at(piv, j) = t;
      }
      double t = br[k]; br[k] = br[piv]; br[piv] = t;
      t = bi[k]; bi[k] = bi[piv]; bi[piv] = t;
    }
    const double d = at(k, k);
    for (int i = k + 1; i <= min(nc - 1, k + KLO); ++i) {
      const double l = at(i, k) / d;
      if (l == 0.0) continue;
      for (int j = k + 1; j <= min(nc - 1, k + KUP); ++j) at(i, j) -= l * at(k, j);
      br[i] -= l * br[k];
      bi[i] -= l * bi[k];
    }
  }
  for (int k = nc - 1; k >= 0; --k) {
    double sr = br[k], si = bi[k];
    for (int j = k + 1; j <= min(nc - 1, k + KUP); ++j) {
      sr -= at(k, j) * br[j];
      si -= at(k, j) * bi[j];
    }
    br[k] = sr / at(k, k);
    bi[k] = si / at(k, k);
  }
  lp[lp_c(nc)] = br[0];
  out[0] = make_double2(0.0, 0.0);
  for (int i = 1; i < nc; ++i) out[i] = make_double2(br[i], bi[i]);
}

template <typename T>
__device__ __forceinline__ bool vortex_product_at(long long idx, int nphi, int nr, T U0, T Uz,
                                                  const double* __restrict__ rnode, T* __restrict__ f0,
                                                  T* __restrict__ f1, T* __restrict__ f2,
                                                  const T* __restrict__ f3, const T* __restrict__ f4,
                                                  const T* __restrict__ f5) {
  const int i = (int)(idx % nr);
  const int j = (int)((idx / nr) % nphi);
  const T r = (T)rnode[i];
  T sn, cs;
  if (sizeof(T) == 8) {
    double sd, cd;
    sincospi(2.0 * j / nphi, &sd, &cd);
    sn = (T)sd; cs = (T)cd;
  } else {
    float sf, cf;
    sincospif(2.0f * (float)j / (float)nphi, &sf, &cf);
    sn = (T)sf; cs = (T)cf;
  }
  const T rvr = f0[idx], rvp = f1[idx], rwr = f3[idx], rwp = f4[idx], wz = f5[idx];
  const T vz = f2[idx] + Uz;        // v_z + U_z
  const T ar = rvr + r * U0 * sn;   // r (v_r + U_r)
  const T ap = rvp + r * U0 * cs;   // r (v_phi + U_phi)
  const T A = vz * rwr - ar * wz;                // A = r N_phi
  const T Bv = ap * wz - vz * rwp;               // B = r N_r
  const T C = ar * rwp - ap * rwr;               // C = r^2 N_z
  f0[idx] = A;
  f1[idx] = Bv;
  f2[idx] = C;
  return isfinite(A) && isfinite(Bv) && isfinite(C);
}

template <typename T>
__global__ void k_vortex_product(long long n_phys, int nphi, int nr, T U0, T Uz, const double* __restrict__ rnode,
                                 T* __restrict__ f0, T* __restrict__ f1, T* __restrict__ f2,
                                 const T* __restrict__ f3, const T* __restrict__ f4, const T* __restrict__ f5,
                                 int* __restrict__ err) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool finite = true;
  if (idx < n_phys) finite = vortex_product_at(idx, nphi, nr, U0, Uz, rnode, f0, f1, f2, f3, f4, f5);
  // a non-finite product (blow-up or NaN in the state) sets the status bit that
  // mlx_device_status reports as MLX_ENUMERIC
  if (__any_sync(0xffffffffu, !finite) && (threadIdx.x & 31) == 0) atomicOr(err, 16);
}


// Jacobi matrix entries e_{m,i} = sqrt((n^2 - m^2) / (4 n^2 - 1)), n = m + i + 1, coupling
// local rows i and i + 1 (multiplication by x, from x Pbar_n = a_{n+1} Pbar_{n+1} + a_n Pbar_{n-1});
// tabulated once per context (the square root and division are costly in FP64)
__device__ __forceinline__ double jac_e(int m, int i, int Nm) {
  if (i < 0 || i + 1 >= Nm) return 0.0;
  const double n = (double)(m + i + 1), mm = (double)m;
  return sqrt((n * n - mm * mm) / (4.0 * n * n - 1.0));
}
__global__ void k_jac_table(int M, int nc, const long long* __restrict__ rows, double* __restrict__ jac) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows[M]) return;
  int lo = 0, hi = M;
  while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (rows[mid] <= idx) lo = mid; else hi = mid; }
  jac[idx] = jac_e(lo, (int)(idx - rows[lo]), nc - lo);
}
// (J v)_a = e_{a-1} v_{a-1} + e_a v_{a+1}, e from the table row of m (je = jac + rows[m])
__device__ __forceinline__ double2 apply_J(const double2* v, const double* je, int a, int Nm) {
  double2 r = make_double2(0.0, 0.0);
  if (a - 1 >= 0) r = cadd(r, cmulr(je[a - 1], v[a - 1]));
  if (a + 1 < Nm) r = cadd(r, cmulr(je[a], v[a + 1]));
  return r;
}

// rhs_psi = -(R A - i m B);  T = R B + i m A + i kappa C  (X2 + i kappa C)
__global__ void k_proj_rhs1(long long n_spec, int M, int nc, int Kz, int K, double lz,
                            const long long* __restrict__ soff, const long long* __restrict__ rows,
                            const double* __restrict__ rdr, const double2* __restrict__ A,
                            const double2* __restrict__ Bf, const double2* __restrict__ C,
                            double2* __restrict__ rhs_psi, double2* __restrict__ T) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_spec) return;
  const int m = m_of(idx, soff, M);
  const int Nm = nc - m;
  const long long loc = idx - soff[m];
  const int kidx = (int)(loc / Nm), a = (int)(loc - (long long)kidx * Nm);
  const long long base = soff[m] + (long long)kidx * Nm;
  const double* rb = rdr + rows[m] * 2;
  const double mm = (double)m;
  const double kap = kappa_of(kidx, Kz, K, lz);
  rhs_psi[idx] = cmulr(-1.0, csub(apply_R(rb, A + base, a, Nm), cimul(mm, Bf[idx])));
  T[idx] = cadd(cadd(apply_R(rb, Bf + base, a, Nm), cimul(mm, A[idx])), cimul(kap, C[idx]));
}

// rhs_g = (I - J) T
__global__ void k_proj_rhs2(long long n_spec, int M, int nc, const long long* __restrict__ soff,
                            const long long* __restrict__ rows, const double* __restrict__ jac,
                            const double2* __restrict__ T, double2* __restrict__ rhs_g) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_spec) return;
  const int m = m_of(idx, soff, M);
  const int Nm = nc - m;
  const long long loc = idx - soff[m];
  const int kidx = (int)(loc / Nm), a = (int)(loc - (long long)kidx * Nm);
  const long long base = soff[m] + (long long)kidx * Nm;
  rhs_g[idx] = csub(T[idx], apply_J(T + base, jac + rows[m], a, Nm));
}

// rhs_chi = i kappa ell^2 (I + J) g - (I - J) C  (first term absent at k = 0)
__global__ void k_proj_rhs3(long long n_spec, int M, int nc, int Kz, int K, double lz, double ell,
                            const long long* __restrict__ soff, const long long* __restrict__ rows,
                            const double* __restrict__ jac, const double2* __restrict__ gg,
                            const double2* __restrict__ C, double2* __restrict__ rhs_chi) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_spec) return;
  const int m = m_of(idx, soff, M);
  const int Nm = nc - m;
  const long long loc = idx - soff[m];
  const int kidx = (int)(loc / Nm), a = (int)(loc - (long long)kidx * Nm);
  const long long base = soff[m] + (long long)kidx * Nm;
  const double kap = kappa_of(kidx, Kz, K, lz);
  const double* je = jac + rows[m];
  double2 r = cmulr(-1.0, csub(C[idx], apply_J(C + base, je, a, Nm)));
  if (kidx != 0) r = cadd(r, cimul(kap * ell * ell, cadd(gg[idx], apply_J(gg + base, je, a, Nm))));
  rhs_chi[idx] = r;
}

// r d/dr band: row j has (j, j-1) and (j, j+1) entries on the normalised basis,
//   R[j][j-1] = -(j-1)(j-m)/(2j-1) N_{j-1}/N_j,   R[j][j+1] = (j+2)(j+1+m)/(2j+3) N_{j+1}/N_j
__device__ __forceinline__ double nr_up(int n, int m) {
  return sqrt((2.0 * n + 3.0) * (n + 1.0 - m) / ((2.0 * n + 1.0) * (n + 1.0 + m)));
}
__global__ void k_rdr_band(int M, int nc, const long long* __restrict__ rows, double* __restrict__ rdr) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows[M]) return;
  int lo = 0, hi = M;
  while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (rows[mid] <= idx) lo = mid; else hi = mid; }
  const int m = lo;
  const int j = m + (int)(idx - rows[m]);
  double lower = 0.0, upper = 0.0;
  if (j - 1 >= m) lower = -(j - 1.0) * (j - (double)m) / (2.0 * j - 1.0) / nr_up(j - 1, m);
  if (j + 1 < nc) upper = (j + 2.0) * (j + 1.0 + m) / (2.0 * j + 3.0) * nr_up(j, m);
  rdr[idx * 2 + 0] = lower;
  rdr[idx * 2 + 1] = upper;
}

inline unsigned nblk(long long n, int tb) { return (unsigned)((n + tb - 1) / tb); }

// Kinetic-energy density of one (m, k) harmonic of the velocity, on the Gauss nodes:
// part[m K + k] = mult_m sum_i w_i / (1 - x_i)^2 (|r v_r|^2 / r_i^2 + |r v_phi|^2 / r_i^2 + |v_z|^2)
// with each component evaluated from its coefficients by the FP64 basis table.
// The sum is the grid's energy (that of the backward transform): the blocks m = 0
// and m = Nphi/2 (Nyquist chop), whose grid functions are real parts, contribute
// their Hermitian part in k, (f_k + conj f_{-k}) / 2, with mult 1 and 4; the other
// orders f_k with mult 2; and with the axial Nyquist kept (K = Nz + 1) the rows
// k = +-Nz/2 share one grid bin, which takes their sum (row k = -Nz/2 adds nothing).
constexpr int kEnThreads = 128;
__global__ void __launch_bounds__(kEnThreads) k_energy_blocks(int nc, int nr, int K, int Kz, int nz, int nphi,
                                                              const long long* __restrict__ soff,
                                                              const long long* __restrict__ boff,
                                                              const double* __restrict__ x, const double* __restrict__ w,
                                                              const double* __restrict__ rn, const double* __restrict__ P64,
                                                              const double2* __restrict__ rvr,
                                                              const double2* __restrict__ rvp,
                                                              const double2* __restrict__ vz, double* __restrict__ part) {
  extern __shared__ double2 ev[];      // [3][Nc - m]
  __shared__ double red[kEnThreads];
  const int kidx = blockIdx.x, m = blockIdx.y;
  const int Nm = nc - m;
  const bool nyz = K == nz + 1;
  if (nyz && kidx == Kz) {             // folded into the row k = +Nz/2
    if (threadIdx.x == 0) part[(long long)m * K + kidx] = 0.0;
    return;
  }
  const bool herm = m == 0 || 2 * m == nphi;
  const int prow = (kidx == 0 || (nyz && kidx == Kz - 1)) ? kidx : K - kidx;
  const double2* src[3] = {rvr, rvp, vz};
  auto row = [&](const double2* f, int kk, int a) {
    double2 v = f[soff[m] + (long long)kk * Nm + a];
    if (nyz && kk == Kz - 1) {
      const double2 u = f[soff[m] + (long long)Kz * Nm + a];
      v.x += u.x;
      v.y += u.y;
    }
    return v;
  };
  for (int a = threadIdx.x; a < Nm; a += blockDim.x)
    for (int c = 0; c < 3; ++c) {
      double2 v = row(src[c], kidx, a);
      if (herm) {
        const double2 u = row(src[c], prow, a);
        v = make_double2(0.5 * (v.x + u.x), 0.5 * (v.y - u.y));
      }
      ev[c * Nm + a] = v;
    }
  __syncthreads();
  const double* Pm = P64 + boff[m];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    double f[6] = {0, 0, 0, 0, 0, 0};
    for (int a = 0; a < Nm; ++a) {
      const double pv = Pm[(long long)a * nr + i];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        f[2 * c] = fma(pv, ev[c * Nm + a].x, f[2 * c]);
        f[2 * c + 1] = fma(pv, ev[c * Nm + a].y, f[2 * c + 1]);
      }
    }
    const double om = 1.0 - x[i];
    const double r2 = rn[i] * rn[i];
    const double e = (fma(f[0], f[0], f[1] * f[1]) + fma(f[2], f[2], f[3] * f[3])) / r2 + fma(f[4], f[4], f[5] * f[5]);
    acc = fma(w[i] / (om * om), e, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kEnThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    part[(long long)m * K + kidx] = (m == 0 ? 1.0 : (2 * m == nphi ? 4.0 : 2.0)) * red[0];
}

// Enstrophy and peak vorticity over the nodes from the physical r w_r, r w_phi, w_z:
// per CTA the partial sum of q_i |w|^2 (q_i = w_i ell^2 / (1 - x_i)^2, the mapped
// area rule) and the largest |w|^2; k_enst_sum folds the partials in a fixed order.
constexpr int kEsThreads = 256, kEnstBlocks = 4 * 148;
template <typename T>
__global__ void __launch_bounds__(kEsThreads) k_enst_blocks(long long n_phys, int nr, double ell,
                                                            const double* __restrict__ x, const double* __restrict__ w,
                                                            const double* __restrict__ rn, const T* __restrict__ rwr,
                                                            const T* __restrict__ rwp, const T* __restrict__ wz,
                                                            double* __restrict__ part) {
  __shared__ double rs[kEsThreads], rm[kEsThreads];
  double s = 0.0, mx = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n_phys;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % nr);
    const double r = rn[i];
    const double a = (double)rwr[idx] / r, b = (double)rwp[idx] / r, c = (double)wz[idx];
    const double q2 = fma(a, a, fma(b, b, c * c));
    const double om = 1.0 - x[i];
    s = fma(w[i] * ell * ell / (om * om), q2, s);
    mx = fmax(mx, q2);
  }
  rs[threadIdx.x] = s;
  rm[threadIdx.x] = mx;
  __syncthreads();
  for (int h = kEsThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      rs[threadIdx.x] += rs[threadIdx.x + h];
      rm[threadIdx.x] = fmax(rm[threadIdx.x], rm[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = rs[0];
    part[2 * blockIdx.x + 1] = rm[0];
  }
}

__global__ void k_enst_sum(int nb, const double* __restrict__ part, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double s = 0.0, mx = 0.0;
  for (int b = 0; b < nb; ++b) {
    s += part[2 * b];
    mx = fmax(mx, part[2 * b + 1]);
  }
  out[0] = s;
  out[1] = mx;
}

}  // namespace

int mlx_vortex_prepare(mlx_ctx* c, cudaStream_t st) {
  if (c->vortex_ready) return MLX_OK;
  int rc = mlx_lap_setup(c, st);
  if (rc) return rc;
  if ((rc = mlx_proj_setup(c, st))) return rc;
  const size_t es = elem_size(c->precision);
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_rdr, sizeof(double) * c->tri * 2));
  k_rdr_band<<<nblk(c->tri, 256), 256, 0, st>>>(c->M, c->nc, c->d_lap_off, c->d_rdr);
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_vortex_fields, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double2) * 4 * c->nc)));
  if (c->precision != MLX_FP64) {
    // the double-float fields kernel's band tables (r d/dr, D_m), converted once
    MLX_CUDA_TRY(c, cudaMalloc(&c->d_rdr_df, sizeof(dfl) * c->tri * 2));
    MLX_CUDA_TRY(c, cudaMalloc(&c->d_lap_df, sizeof(dfl) * c->tri * 5));
    mlx_to_df(c->d_rdr, c->d_rdr_df, c->tri * 2, st);
    mlx_to_df(c->d_lap, c->d_lap_df, c->tri * 5, st);
    MLX_LAUNCH_CHECK(c);
    MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_vortex_fields_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(dfl2) * 4 * c->nc)));
  }
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_jac, sizeof(double) * c->tri));
  k_jac_table<<<nblk(c->tri, 256), 256, 0, st>>>(c->M, c->nc, c->d_lap_off, c->d_jac);
  MLX_LAUNCH_CHECK(c);
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_vspec, sizeof(double2) * c->n_spec * 9));
  if (c->precision == MLX_BF16X3 && (rc = mlx_tc_vortex_planes(c, st))) return rc;
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_vphys, es * c->n_phys * 6));
  // two-field state temporaries for the Richardson start and the graph-replayed pair
  for (double2** p : {&c->d_specA, &c->d_spec1, &c->d_spec2, &c->d_spec3}) {
    cudaFree(*p);
    *p = nullptr;
    MLX_CUDA_TRY(c, cudaMalloc(p, sizeof(double2) * c->n_spec * 2));
  }
  mlx_invalidate_graphs(c);
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  c->vortex_ready = true;
  return MLX_OK;
}

template <typename T>
static int vortex_nonlinear_t(mlx_ctx* c, double U0, const double2* state, double2* out, cudaStream_t st) {
  const long long ns = c->n_spec, np = c->n_phys;
  const double2* psi = state;
  const double2* chi = state + ns;
  double2* F[9];
  for (int i = 0; i < 9; ++i) F[i] = c->d_vspec + ns * i;
  T* P[6];
  for (int i = 0; i < 6; ++i) P[i] = reinterpret_cast<T*>(c->d_vphys) + np * i;
  const int tb = 256;
  SplitPlanes planes;   // BF16X3: the fields go straight to the backward contraction's planes
  if (c->precision == MLX_BF16X3 && c->d_bsv && c->vortex_planes) {
    planes.bs = reinterpret_cast<unsigned short*>(c->d_bsv);
    planes.Kq = (int)c->tc_kq;
    planes.K2 = 2 * c->K;
    planes.part = (long long)c->M * planes.K2 * planes.Kq;
  }
  {
    const int vt = c->nc >= 256 ? 256 : ((c->nc + 31) / 32) * 32;
    const double* lpf = c->lp_on ? c->d_lp + kLpFields : nullptr;
    if (c->precision == MLX_FP64)
      k_vortex_fields<<<dim3(c->K, c->M), vt, sizeof(double2) * 4 * c->nc, st>>>(
          c->nc, c->Kz, c->K, c->lz, c->d_soff, c->d_lap_off, c->d_rdr, c->d_lap, psi, chi, F[0], F[1], F[2],
          F[3], F[4], F[5], lpf, planes);
    else
      k_vortex_fields_df<<<dim3(c->K, c->M), vt, sizeof(dfl2) * 4 * c->nc, st>>>(
          c->nc, c->Kz, c->K, c->lz, c->d_soff, c->d_lap_off, (const dfl*)c->d_rdr_df, (const dfl*)c->d_lap_df,
          psi, chi, F[0], F[1], F[2], F[3], F[4], F[5], lpf, planes);
  }
  MLX_LAUNCH_CHECK(c);
  int rc;
  for (int f = 0; f < 6; ++f) {
    if ((rc = planes.bs ? mlx_legendre_tc_backward_field(c, f, st) : mlx_legendre_backward(c, F[f], st))) return rc;
    if ((rc = mlx_fft_backward(c, P[f], st))) return rc;
  }
  k_vortex_product<T><<<nblk(np, tb), tb, 0, st>>>(np, c->nphi, c->nr, (T)U0, (T)c->vortex_uz, c->d_r, P[0], P[1], P[2], P[3],
                                                   P[4], P[5], c->d_err);
  MLX_LAUNCH_CHECK(c);
  // A, B, C -> F[6], F[7], F[8]
  for (int f = 0; f < 3; ++f) {
    if ((rc = mlx_fft_forward(c, P[f], st))) return rc;
    if ((rc = mlx_legendre_forward(c, F[6 + f], st))) return rc;
  }
  // rhs_psi -> F[0], T -> F[1], rhs_g -> F[2], g -> F[3], rhs_chi -> F[4]
  k_proj_rhs1<<<nblk(ns, tb), tb, 0, st>>>(ns, c->M, c->nc, c->Kz, c->K, c->lz, c->d_soff, c->d_lap_off, c->d_rdr,
                                           F[6], F[7], F[8], F[0], F[1]);
  MLX_LAUNCH_CHECK(c);
  k_proj_rhs2<<<nblk(ns, tb), tb, 0, st>>>(ns, c->M, c->nc, c->d_soff, c->d_lap_off, c->d_jac, F[1], F[2]);
  MLX_LAUNCH_CHECK(c);
  if ((rc = mlx_proj_solve(c, 0, F[0], out, st))) return rc;         // psi_N
  if ((rc = mlx_proj_solve(c, 2, F[2], F[3], st))) return rc;        // g
  k_proj_rhs3<<<nblk(ns, tb), tb, 0, st>>>(ns, c->M, c->nc, c->Kz, c->K, c->lz, c->ell, c->d_soff, c->d_lap_off,
                                           c->d_jac, F[3], F[8], F[4]);
  MLX_LAUNCH_CHECK(c);
  return mlx_proj_solve(c, 1, F[4], out + ns, st);                   // chi_N
}

int mlx_vortex_nonlinear(mlx_ctx* c, double U0, const double2* state, double2* out, cudaStream_t st) {
  if (!c->vortex_ready) return MLX_ESTATE;
  if (c->precision == MLX_FP64) return vortex_nonlinear_t<double>(c, U0, state, out, st);
  return vortex_nonlinear_t<float>(c, U0, state, out, st);
}

// Axial energy spectrum of the two-field state: E[|k|] for |k| < Kz (host), see mlx.h.
extern "C" int mlx_axial_energy(mlx_ctx* c, const void* state, double* E, mlx_stream stream) {
  if (!c || !state || !E || (((uintptr_t)state) & 15u)) return MLX_EINVAL;
  if (!c->vortex_ready) return MLX_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  const long long ns = c->n_spec;
  const double2* psi = (const double2*)state;
  const double2* chi = psi + ns;
  double2* F[6];
  for (int i = 0; i < 6; ++i) F[i] = c->d_vspec + ns * i;
  const int vt = c->nc >= 256 ? 256 : ((c->nc + 31) / 32) * 32;
  // the basis part only: the log proxy's swirl has unbounded energy
  k_vortex_fields<<<dim3(c->K, c->M), vt, sizeof(double2) * 4 * c->nc, st>>>(
      c->nc, c->Kz, c->K, c->lz, c->d_soff, c->d_lap_off, c->d_rdr, c->d_lap, psi, chi, F[0], F[1], F[2], F[3],
      F[4], F[5], nullptr, SplitPlanes());
  MLX_LAUNCH_CHECK(c);
  // the partial sums go to the (then unused) seventh spectral temporary
  double* part = reinterpret_cast<double*>(c->d_vspec + ns * 6);
  if ((long long)c->M * c->K > 2 * ns) return MLX_EINVAL;
  k_energy_blocks<<<dim3(c->K, c->M), kEnThreads, sizeof(double2) * 3 * c->nc, st>>>(
      c->nc, c->nr, c->K, c->Kz, c->nz, c->nphi, c->d_soff, c->d_boff, c->d_x, c->d_w, c->d_r, c->d_P64, F[0],
      F[1], F[2], part);
  MLX_LAUNCH_CHECK(c);
  std::vector<double> h((size_t)c->M * c->K);
  MLX_CUDA_TRY(c, cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  const double scale = M_PI * c->lz * c->ell * c->ell;
  for (int k = 0; k < c->Kz; ++k) E[k] = 0.0;
  for (int m = 0; m < c->M; ++m)
    for (int kidx = 0; kidx < c->K; ++kidx) {
      const int k = kidx < c->Kz ? kidx : c->K - kidx;
      E[k] += h[(size_t)m * c->K + kidx];
    }
  for (int k = 0; k < c->Kz; ++k) E[k] *= scale;
  return MLX_OK;
}

// ---- log proxies and the axial background (see mlx.h) ----------------------------

// (Re)build the proxy tables from the context's amplitudes and implicit operator.
int mlx_lp_refresh(mlx_ctx* c, cudaStream_t st) {
  if (!c->d_lp) MLX_CUDA_TRY(c, cudaMalloc(&c->d_lp, sizeof(double) * lp_size(c->nc)));
  k_lp_setup<<<1, 32, 0, st>>>(c->nc, c->ell, c->lp_cpsi, c->lp_cchi, c->implicit_ready ? c->nu : 0.0,
                               c->implicit_ready ? c->nu_h : 0.0, c->p, c->d_lap, c->d_lp);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

// Add the proxies' forcing c L Lambda to a two-field tendency (the time steps).
int mlx_lp_add_source(mlx_ctx* c, double2* A, cudaStream_t st) {
  if (!c->lp_on) return MLX_OK;
  k_lp_source<<<nblk(c->nc, 128), 128, 0, st>>>(c->nc, c->lp_cpsi, c->lp_cchi, c->d_lp + lp_ll(c->nc), A,
                                                A + c->n_spec);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

extern "C" int mlx_vortex_logproxy(mlx_ctx* c, double c_psi, double c_chi, double Uz, mlx_stream stream) {
  if (!c || !std::isfinite(c_psi) || !std::isfinite(c_chi) || !std::isfinite(Uz)) return MLX_EINVAL;
  if (!c->vortex_ready) return MLX_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  c->lp_cpsi = c_psi;
  c->lp_cchi = c_chi;
  c->vortex_uz = Uz;
  c->lp_on = c_psi != 0.0 || c_chi != 0.0;
  int rc = mlx_lp_refresh(c, st);
  if (rc) return rc;
  mlx_invalidate_graphs(c);
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  return MLX_OK;
}

extern "C" int mlx_lap_h_solve_log(mlx_ctx* c, const void* rhs, void* out, int variant, double* cval,
                                   mlx_stream stream) {
  if (!c || !rhs || !out || rhs == out || !cval) return MLX_EINVAL;
  if ((((uintptr_t)rhs) & 15u) || (((uintptr_t)out) & 15u)) return MLX_EINVAL;
  if (variant != MLX_LOGPROXY_PRESCRIBE && variant != MLX_LOGPROXY_SOLVE) return MLX_EINVAL;
  if (variant == MLX_LOGPROXY_PRESCRIBE && !std::isfinite(*cval)) return MLX_EINVAL;
  if (!c->lap_ready || !c->vortex_ready) return MLX_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  if (!c->d_lp) {
    int rc = mlx_lp_refresh(c, st);
    if (rc) return rc;
  }
  const double2* f = (const double2*)rhs;
  if (variant == MLX_LOGPROXY_PRESCRIBE) {
    double2* tmp = c->d_spec3;
    MLX_CUDA_TRY(c, cudaMemcpyAsync(tmp, f, sizeof(double2) * c->n_spec, cudaMemcpyDeviceToDevice, st));
    k_lp_shift<<<nblk(c->nc, 128), 128, 0, st>>>(c->nc, *cval, c->d_lp + kLpLam, tmp);
    MLX_LAUNCH_CHECK(c);
    return mlx_lap_solve(c, 0, tmp, (double2*)out, st);
  }
  int rc = mlx_lap_solve(c, 0, f, (double2*)out, st);   // every other harmonic: the ordinary solve
  if (rc) return rc;
  k_lp_solve_c<<<1, 32, 0, st>>>(c->nc, c->d_lap, c->d_lp, f, (double2*)out);
  MLX_LAUNCH_CHECK(c);
  MLX_CUDA_TRY(c, cudaMemcpyAsync(cval, c->d_lp + lp_c(c->nc), sizeof(double), cudaMemcpyDeviceToHost, st));
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  return MLX_OK;
}

template <typename T>
static int vortex_diag_t(mlx_ctx* c, const double2* state, mlx_vortex_diag_out* out, cudaStream_t st) {
  const long long ns = c->n_spec, np = c->n_phys;
  double2* F[6];
  for (int i = 0; i < 6; ++i) F[i] = c->d_vspec + ns * i;
  T* P[6];
  for (int i = 0; i < 6; ++i) P[i] = reinterpret_cast<T*>(c->d_vphys) + np * i;
  const int vt = c->nc >= 256 ? 256 : ((c->nc + 31) / 32) * 32;
  k_vortex_fields<<<dim3(c->K, c->M), vt, sizeof(double2) * 4 * c->nc, st>>>(
      c->nc, c->Kz, c->K, c->lz, c->d_soff, c->d_lap_off, c->d_rdr, c->d_lap, state, state + ns, F[0], F[1], F[2],
      F[3], F[4], F[5], c->lp_on ? c->d_lp + kLpFields : nullptr, SplitPlanes());
  MLX_LAUNCH_CHECK(c);
  int rc;
  for (int f = 3; f < 6; ++f) {
    if ((rc = mlx_legendre_backward(c, F[f], st))) return rc;
    if ((rc = mlx_fft_backward(c, P[f], st))) return rc;
  }
  const int nb = kEnstBlocks;
  if (!c->d_enst) MLX_CUDA_TRY(c, cudaMalloc(&c->d_enst, sizeof(double) * (2 * nb + 2)));
  double* part = c->d_enst;
  k_enst_blocks<T><<<nb, kEsThreads, 0, st>>>(np, c->nr, c->ell, c->d_x, c->d_w, c->d_r, P[3], P[4], P[5], part);
  MLX_LAUNCH_CHECK(c);
  k_enst_sum<<<1, 32, 0, st>>>(nb, part, part + 2 * nb);
  MLX_LAUNCH_CHECK(c);
  double h[2];
  MLX_CUDA_TRY(c, cudaMemcpyAsync(h, part + 2 * nb, sizeof(h), cudaMemcpyDeviceToHost, st));
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  out->enstrophy = 0.5 * (c->lz / c->nz) * (2.0 * M_PI / c->nphi) * h[0];
  out->peak_vorticity = sqrt(h[1]);
  return MLX_OK;
}

extern "C" int mlx_vortex_diag(mlx_ctx* c, const void* state, mlx_vortex_diag_out* out, mlx_stream stream) {
  if (!c || !state || !out || (((uintptr_t)state) & 15u)) return MLX_EINVAL;
  if (!c->vortex_ready) return MLX_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  if (c->precision == MLX_FP64) return vortex_diag_t<double>(c, (const double2*)state, out, st);
  return vortex_diag_t<float>(c, (const double2*)state, out, st);
}
