// K1: FP64 generation of nodes, weights, mapped radii, the normalised associated
// Legendre tables, the Laplacian bands and the Fourier twiddles (Sec. 3.1).
#include "mlx_internal.cuh"

#include <math.h>

namespace {

// Gauss-Legendre nodes by Newton iteration on P_N (three-term recurrence), one
// thread per node; weights w = 2 / ((1 - x^2) P_N'(x)^2).  Stored ascending.
__global__ void k_gauss_nodes(int N, double ell, double* __restrict__ x,
                              double* __restrict__ w, double* __restrict__ r) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double xi = cos(M_PI * (j + 0.75) / (N + 0.5));   // descending guesses
  double dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = xi;
    for (int k = 2; k <= N; ++k) {
      double p2 = ((2.0 * k - 1.0) * xi * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double pn = (N == 1) ? xi : p1;
    double pm1 = (N == 1) ? 1.0 : p0;
    dp = -N * (xi * pn - pm1) / ((1.0 - xi) * (1.0 + xi));
    double dx = pn / dp;
    xi -= dx;
    if (fabs(dx) < 1e-16) break;
  }
  {
    double p0 = 1.0, p1 = xi;
    for (int k = 2; k <= N; ++k) {
      double p2 = ((2.0 * k - 1.0) * xi * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double pn = (N == 1) ? xi : p1;
    double pm1 = (N == 1) ? 1.0 : p0;
    dp = -N * (xi * pn - pm1) / ((1.0 - xi) * (1.0 + xi));
  }
  int a = N - 1 - j;
  x[a] = xi;
  w[a] = 2.0 / ((1.0 - xi) * (1.0 + xi) * dp * dp);
  r[a] = ell * sqrt((1.0 + xi) / (1.0 - xi));
}

// Pbar_n^m(x_i) for n = m..Nc-1, one thread per (m, i).  The diagonal climbs
// Pbar_m^m = sqrt((2m+1)/(2m)) sqrt(1-x^2) Pbar_{m-1}^{m-1} from 1/sqrt(2); the
// degree is raised with a_n = sqrt((4n^2-1)/(n^2-m^2)),
// b_n = sqrt(((n-1)^2-m^2)/(4(n-1)^2-1)).  Values are carried as v * 2^e with an
// explicit binary exponent e so that (1-x^2)^{m/2} cannot underflow before the
// recurrence lifts it back; the stored value is ldexp(v, e).
__global__ void k_basis(int M, int nc, int nr, const double* __restrict__ x,
                        const double* __restrict__ w, const long long* __restrict__ boff,
                        double* __restrict__ P64, double* __restrict__ W64,
                        float* __restrict__ P32, float* __restrict__ W32) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * nr) return;
  int m = idx / nr, i = idx % nr;
  double xi = x[i], wi = w[i];
  double s = sqrt((1.0 - xi) * (1.0 + xi));
  double v = 0.70710678118654752440;  // 1/sqrt(2)
  int e = 0;
  for (int mm = 1; mm <= m; ++mm) {
    v *= sqrt((2.0 * mm + 1.0) / (2.0 * mm)) * s;
    if (fabs(v) < 0x1p-200) { v = ldexp(v, 200); e -= 200; }
  }
  long long base = boff[m] + i;
  double pm2 = 0.0, pm1 = v;
  for (int n = m; n < nc; ++n) {
    double cur;
    if (n == m) {
      cur = v;
    } else if (n == m + 1) {
      cur = sqrt(2.0 * m + 3.0) * xi * pm1;
    } else {
      double nn = (double)n, mm = (double)m;
      double a = sqrt((4.0 * nn * nn - 1.0) / (nn * nn - mm * mm));
      double b = sqrt(((nn - 1.0) * (nn - 1.0) - mm * mm) / (4.0 * (nn - 1.0) * (nn - 1.0) - 1.0));
      cur = a * (xi * pm1 - b * pm2);
    }
    if (n > m) { pm2 = pm1; pm1 = cur; }
    if (e < 0 && fabs(cur) > 0x1p+200) {   // rescale the carried pair
      pm1 = ldexp(pm1, -200); pm2 = ldexp(pm2, -200); cur = ldexp(cur, -200); e += 200;
    }
    double val = (e == 0) ? cur : ldexp(cur, e);
    long long o = base + (long long)(n - m) * nr;
    P64[o] = val;
    W64[o] = wi * val;
    P32[o] = (float)val;
    W32[o] = (float)(wi * val);
  }
}

// Normalised pentadiagonal Laplacian (Eq. (5) rescaled by N_j / N_n, Sec. 3.1),
// one thread per (m, n).  N_{n+1}/N_n = sqrt((2n+3)(n+1-m) / ((2n+1)(n+1+m))).
__device__ __forceinline__ double nratio_up(int n, int m) {
  double a = (2.0 * n + 3.0) * (n + 1.0 - m);
  double b = (2.0 * n + 1.0) * (n + 1.0 + m);
  return sqrt(a / b);
}

__global__ void k_lap_band(int M, int nc, double inv_ell2, const long long* __restrict__ soff_rows,
                           double* __restrict__ lap) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  // rows are enumerated m-major: row = sum_{m'<m}(nc-m') + (n-m)
  // find m by a linear scan (M <= 1024, init only)
  long long total = soff_rows[M];
  if (idx >= total) return;
  int m = 0;
  while (soff_rows[m + 1] <= idx) ++m;
  int n = m + (int)(idx - soff_rows[m]);
  double nn = n, mm = m;
  double e[5] = {0, 0, 0, 0, 0};
  if (n - 2 >= m)
    e[0] = -((nn - mm - 1) * (nn - mm) * (nn - 2) * (nn - 1)) / ((2 * nn - 3) * (2 * nn - 1)) /
           (nratio_up(n - 1, m) * nratio_up(n - 2, m));
  if (n - 1 >= m)
    e[1] = 2.0 * nn * (nn - 1) * (nn - mm) / (2 * nn - 1) / nratio_up(n - 1, m);
  e[2] = -2.0 * nn * (nn + 1) * (3 * nn * nn + 3 * nn - mm * mm - 2) / ((2 * nn - 1) * (2 * nn + 3));
  if (n + 1 < nc)
    e[3] = 2.0 * (nn + 1) * (nn + 2) * (nn + mm + 1) / (2 * nn + 3) * nratio_up(n, m);
  if (n + 2 < nc)
    e[4] = -((nn + 2) * (nn + 3) * (nn + mm + 1) * (nn + mm + 2)) / ((2 * nn + 3) * (2 * nn + 5)) *
           (nratio_up(n, m) * nratio_up(n + 1, m));
  for (int o = 0; o < 5; ++o) lap[idx * 5 + o] = e[o] * inv_ell2;
}

// exp(-2 pi i t / N) for t < N/2
__global__ void k_twiddles(int N, double2* __restrict__ t64, float2* __restrict__ t32) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N / 2) return;
  double s, c;
  sincospi(2.0 * t / N, &s, &c);
  t64[t] = make_double2(c, -s);
  t32[t] = make_float2((float)c, (float)-s);
}

}  // namespace

int mlx_basis_build(mlx_ctx* c, cudaStream_t st) {
  const int tb = 128;
  k_gauss_nodes<<<(c->nr + tb - 1) / tb, tb, 0, st>>>(c->nr, c->ell, c->d_x, c->d_w, c->d_r);
  MLX_LAUNCH_CHECK(c);
  k_basis<<<(c->M * c->nr + tb - 1) / tb, tb, 0, st>>>(c->M, c->nc, c->nr, c->d_x, c->d_w,
                                                      c->d_boff, c->d_P64, c->d_W64, c->d_P32,
                                                      c->d_W32);
  MLX_LAUNCH_CHECK(c);
  // row offsets (sum_{m'<m} (Nc - m')) for the band kernel
  std::vector<long long> rows(c->M + 1, 0);
  for (int m = 0; m < c->M; ++m) rows[m + 1] = rows[m] + (c->nc - m);
  long long* d_rows = nullptr;
  MLX_CUDA_TRY(c, cudaMallocAsync((void**)&d_rows, sizeof(long long) * (c->M + 1), st));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(d_rows, rows.data(), sizeof(long long) * (c->M + 1),
                                  cudaMemcpyHostToDevice, st));
  k_lap_band<<<(int)((c->tri + tb - 1) / tb), tb, 0, st>>>(c->M, c->nc, 1.0 / (c->ell * c->ell),
                                                          d_rows, c->d_lap);
  MLX_LAUNCH_CHECK(c);
  k_twiddles<<<(c->nphi / 2 + tb - 1) / tb, tb, 0, st>>>(c->nphi, c->d_twphi64, c->d_twphi32);
  MLX_LAUNCH_CHECK(c);
  if (c->nz > 1) {
    k_twiddles<<<(c->nz / 2 + tb - 1) / tb, tb, 0, st>>>(c->nz, c->d_twz64, c->d_twz32);
    MLX_LAUNCH_CHECK(c);
  }
  MLX_CUDA_TRY(c, cudaFreeAsync(d_rows, st));
  return MLX_OK;
}
