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
//   Bplus [N][2kl+1]  band of I + dt/2 L (column i + o at slot o + kl)
//   LU of I - c L, c = dt/2 (half) and dt (full), partial pivoting over the kl
//   rows below the diagonal: U row i holds columns i..i+2kl (slot t = column - i),
//   L multipliers [N][kl], pivot rows, and 1/U[i][i].
// One thread per system factorises; one thread per (m, k) solves (the complex
// right-hand side as two real ones sharing the real factors).
#include "mlx_internal.cuh"

namespace {

// rows of (m, kabs) start at band_off[m] + kabs * (Nc - m)
__device__ __forceinline__ void sys_of(int idx, int M, int nc, int Kz, const long long* band_off,
                                       int& m, int& kabs, long long& row0) {
  // idx enumerates (m, kabs) m-major
  m = idx / Kz;
  kabs = idx % Kz;
  row0 = band_off[m] + (long long)kabs * (nc - m);
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

// Banded LU with partial pivoting of A = I - c L.  work: [N][3kl+1] row windows
// (column j of row i at slot j - i + kl).
__device__ void band_lu(int N, int kl, double c, const double* Lb, double* work, double* U,
                        double* Lm, int* piv, double* invd) {
  const int W = 2 * kl + 1;     // band of L
  const int WW = 3 * kl + 1;    // window: columns i-kl .. i+2kl
  for (long long t = 0; t < (long long)N * WW; ++t) work[t] = 0.0;
  for (int i = 0; i < N; ++i)
    for (int o = -kl; o <= kl; ++o) {
      const int j = i + o;
      if (j < 0 || j >= N) continue;
      double v = -c * Lb[i * W + o + kl];
      if (o == 0) v += 1.0;
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
    piv[j] = pr;
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
      Lm[j * kl + (i - j - 1)] = l;
      work[i * WW + (j - i) + kl] = 0.0;
      for (int cc = j + 1; cc <= cend; ++cc) work[i * WW + (cc - i) + kl] -= l * work[j * WW + (cc - j) + kl];
    }
    for (int i = last + 1; i <= j + kl; ++i) Lm[j * kl + (i - j - 1)] = 0.0;
  }
  for (int i = 0; i < N; ++i) {
    for (int t = 0; t <= 2 * kl; ++t) {
      const int cc = i + t;
      U[i * (2 * kl + 1) + t] = (cc < N) ? work[i * WW + t + kl] : 0.0;
    }
    invd[i] = 1.0 / U[i * (2 * kl + 1)];
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
      Bplus[(row0 + i) * W + o] = v;
    }
  band_lu(N, kl, 0.5 * dt, Lb, work, Uh + row0 * W, Lh + row0 * kl, Ph + row0, Dh + row0);
  band_lu(N, kl, dt, Lb, work, Uf + row0 * W, Lf + row0 * kl, Pf + row0, Df + row0);
}

// One thread per (m, kidx): RHS assembly then forward / back substitution in out.
__global__ void k_band_solve(int M, int nc, int Kz, int K, int kl, int step, double dt,
                             const long long* __restrict__ soff, const long long* __restrict__ band_off,
                             const double* __restrict__ Bplus,
                             const double* __restrict__ U, const double* __restrict__ Lm,
                             const int* __restrict__ piv, const double* __restrict__ invd,
                             const double2* __restrict__ s, const double2* __restrict__ A,
                             const double2* __restrict__ Ap, double2* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * K) return;
  const int m = idx / K, kidx = idx % K;
  const int kabs = kidx < Kz ? kidx : K - kidx;
  const int N = nc - m;
  const long long row0 = band_off[m] + (long long)kabs * N;
  const long long so = soff[m] + (long long)kidx * N;
  const int W = 2 * kl + 1;
  const double2* sv = s + so;
  double2* o = out + so;
  // right-hand side
  for (int i = 0; i < N; ++i) {
    double2 r;
    if (step == MLX_STEP_ABCN) {
      r.x = 0.0; r.y = 0.0;
      const double* bp = Bplus + (row0 + i) * W;
      for (int t = -kl; t <= kl; ++t) {
        const int j = i + t;
        if (j < 0 || j >= N) continue;
        const double b = bp[t + kl];
        const double2 v = sv[j];
        r.x += b * v.x;
        r.y += b * v.y;
      }
      if (A) { const double2 a = A[so + i]; r.x += 1.5 * dt * a.x; r.y += 1.5 * dt * a.y; }
      if (Ap) { const double2 a = Ap[so + i]; r.x -= 0.5 * dt * a.x; r.y -= 0.5 * dt * a.y; }
    } else {
      const double h = (step == MLX_STEP_FEBE_HALF) ? 0.5 * dt : dt;
      r = sv[i];
      if (A) { const double2 a = A[so + i]; r.x += h * a.x; r.y += h * a.y; }
    }
    o[i] = r;
  }
  // forward elimination with the recorded row interchanges
  for (int j = 0; j < N; ++j) {
    const int pr = piv[row0 + j];
    double2 vj = o[j];
    if (pr != j) { const double2 t = o[pr]; o[pr] = vj; vj = t; o[j] = vj; }
    const double* l = Lm + (row0 + j) * kl;
    for (int t = 1; t <= kl && j + t < N; ++t) {
      const double lv = l[t - 1];
      double2 w = o[j + t];
      w.x -= lv * vj.x;
      w.y -= lv * vj.y;
      o[j + t] = w;
    }
  }
  // back substitution
  for (int i = N - 1; i >= 0; --i) {
    const double* u = U + (row0 + i) * W;
    double2 acc = o[i];
    for (int t = 1; t <= 2 * kl && i + t < N; ++t) {
      const double2 x = o[i + t];
      acc.x -= u[t] * x.x;
      acc.y -= u[t] * x.y;
    }
    const double d = invd[row0 + i];
    acc.x *= d;
    acc.y *= d;
    o[i] = acc;
  }
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
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  cudaFree(scratch);
  cudaFree(d_lrows);
  return MLX_OK;
}

int mlx_band_solve(mlx_ctx* c, int step, const double2* s, const double2* A, const double2* Ap,
                   double2* out, cudaStream_t st) {
  TimedLaunch tl(c, KID_BAND_SOLVE, st);
  const BandLU& f = (step == MLX_STEP_FEBE_FULL) ? c->lu_full : c->lu_half;
  const int nsys = c->M * c->K;
  const int tb = 64;
  k_band_solve<<<(nsys + tb - 1) / tb, tb, 0, st>>>(c->M, c->nc, c->Kz, c->K, c->kl, step, c->dt,
                                                    c->d_soff, c->d_band_off, c->d_Bplus, f.U, f.L,
                                                    f.piv, f.invd, s, A, Ap, out);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

int mlx_spec_axpby(mlx_ctx* c, double a, const double2* x, double b, const double2* y,
                   double2* out, cudaStream_t st) {
  TimedLaunch tl(c, KID_AXPBY, st);
  const long long n = c->n_spec;
  const int tb = 256;
  k_axpby<<<(unsigned)((n + tb - 1) / tb), tb, 0, st>>>(n, a, x, b, y, out);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}
