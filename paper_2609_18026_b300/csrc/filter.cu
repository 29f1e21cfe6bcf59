// Adaptive modal filter between time steps (Sec. 3.3, the optional filter).
//
// Every coefficient with normalised mode index
//   zeta = max(n / (Nc - 1), m / (M - 1), |k| / (Kz - 1))      (a term is 0 if its chop keeps one index)
// above the cutoff zeta_c is multiplied by sigma = exp(-eps ((zeta - zeta_c) / (1 - zeta_c))^8).  The
// amplitude eps of each field follows the fraction f of its spectral energy (|shat|^2, multiplicity 2
// for m >= 1) above the cutoff, measured before the filter acts:
//   eps* = eps_max min(1, max(0, (f - tau) / tau)),   eps <- min(eps_max, max(0, eps + relax (eps* - eps))).
// sigma is monotone in zeta, so sigma(max of the three indices) is the smallest of the three
// per-index multipliers: the update kernel tabulates sigma over n, m and |k| (Nc + M + Kz FP64
// exponentials per field and step) and the apply kernel multiplies every coefficient by the smallest
// of its three table entries.  Three launches per field: block partial sums, one-CTA update and
// tables (fixed summation order: deterministic), and the scaling.  eps lives on the device, so the
// filter runs inside the captured time-step graphs.
#include "mlx_internal.cuh"

namespace {

constexpr int kFiltThreads = 128;

__device__ __forceinline__ double zeta_of(int i, int last) { return last > 0 ? (double)i / (double)last : 0.0; }

__global__ void __launch_bounds__(kFiltThreads) k_filt_partials(int nc, int M, int Kz, int K, double zeta_c,
                                                                const long long* __restrict__ soff,
                                                                const double2* __restrict__ spec,
                                                                double* __restrict__ part) {
  __shared__ double red[2][kFiltThreads];
  const int kidx = blockIdx.x, m = blockIdx.y;
  const int Nm = nc - m;
  const double2* blk = spec + soff[m] + (long long)kidx * Nm;
  const int k = kidx < Kz ? kidx : K - kidx;
  const double zmk = fmax(zeta_of(m, M - 1), zeta_of(k, Kz - 1));
  double tot = 0.0, tail = 0.0;
  for (int a = threadIdx.x; a < Nm; a += blockDim.x) {
    const double2 v = blk[a];
    const double e = fma(v.x, v.x, v.y * v.y);
    tot += e;
    if (fmax(zmk, zeta_of(m + a, nc - 1)) > zeta_c) tail += e;
  }
  red[0][threadIdx.x] = tot;
  red[1][threadIdx.x] = tail;
  __syncthreads();
  for (int h = kFiltThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[0][threadIdx.x] += red[0][threadIdx.x + h];
      red[1][threadIdx.x] += red[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double w = m == 0 ? 1.0 : 2.0;
    const long long b = (long long)m * K + kidx;
    part[2 * b] = w * red[0][0];
    part[2 * b + 1] = w * red[1][0];
  }
}

// state: [eps, tail fraction] of this field; tab: sigma over n (nc), m (M), |k| (Kz)
__global__ void k_filt_update(long long nb, int nc, int M, int Kz, double zeta_c, double tau, double eps_max,
                              double relax, const double* __restrict__ part, double* __restrict__ state,
                              double* __restrict__ tab) {
  __shared__ double red[2][256];
  __shared__ double eps_s;
  double tot = 0.0, tail = 0.0;
  for (long long j = threadIdx.x; j < nb; j += blockDim.x) {
    tot += part[2 * j];
    tail += part[2 * j + 1];
  }
  red[0][threadIdx.x] = tot;
  red[1][threadIdx.x] = tail;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[0][threadIdx.x] += red[0][threadIdx.x + h];
      red[1][threadIdx.x] += red[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double f = red[0][0] > 0.0 ? red[1][0] / red[0][0] : 0.0;
    const double target = eps_max * fmin(1.0, fmax(0.0, (f - tau) / tau));
    const double eps = fmin(eps_max, fmax(0.0, state[0] + relax * (target - state[0])));
    state[0] = eps;
    state[1] = f;
    eps_s = eps;
  }
  __syncthreads();
  const double eps = eps_s;
  const int ntab = nc + M + Kz;
  for (int t = threadIdx.x; t < ntab; t += blockDim.x) {
    double z;
    if (t < nc) z = zeta_of(t, nc - 1);
    else if (t < nc + M) z = zeta_of(t - nc, M - 1);
    else z = zeta_of(t - nc - M, Kz - 1);
    double sg = 1.0;
    if (z > zeta_c) {
      const double q = (z - zeta_c) / (1.0 - zeta_c);
      const double q2 = q * q, q4 = q2 * q2;
      sg = exp(-eps * (q4 * q4));
    }
    tab[t] = sg;
  }
}

__global__ void k_filt_apply(int nc, int M, int Kz, int K, const long long* __restrict__ soff,
                             const double* __restrict__ tab, double2* __restrict__ spec) {
  const int m = blockIdx.z, kidx = blockIdx.y;
  const int Nm = nc - m;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Nm) return;
  const int k = kidx < Kz ? kidx : K - kidx;
  const double sg = fmin(tab[m + a], fmin(tab[nc + m], tab[nc + M + k]));
  double2* p = spec + soff[m] + (long long)kidx * Nm + a;
  double2 v = *p;
  v.x *= sg;
  v.y *= sg;
  *p = v;
}

int filt_buffers(mlx_ctx* c) {
  if (c->d_filt) return MLX_OK;
  const long long nb = (long long)c->M * c->K;
  const long long tab = c->nc + c->M + c->Kz;
  const long long n = 4 + 2 * nb + 2 * tab;   // states [2][2], partials, tables [2][tab]
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_filt, sizeof(double) * n));
  MLX_CUDA_TRY(c, cudaMemset(c->d_filt, 0, sizeof(double) * n));
  return MLX_OK;
}

}  // namespace

// Filter every field of a state in place (the advance calls this after every step).
int mlx_filter_fields(mlx_ctx* c, int nfields, double2* state, cudaStream_t st) {
  if (!c->d_filt) return MLX_ESTATE;
  const long long nb = (long long)c->M * c->K;
  const long long tabn = c->nc + c->M + c->Kz;
  double* part = c->d_filt + 4;
  const int tb = c->nc >= 128 ? 128 : 64;
  for (int f = 0; f < nfields; ++f) {
    double2* s = state + (long long)f * c->n_spec;
    double* tab = c->d_filt + 4 + 2 * nb + f * tabn;
    k_filt_partials<<<dim3(c->K, c->M), kFiltThreads, 0, st>>>(c->nc, c->M, c->Kz, c->K, c->filt_zeta_c,
                                                                c->d_soff, s, part);
    k_filt_update<<<1, 256, 0, st>>>(nb, c->nc, c->M, c->Kz, c->filt_zeta_c, c->filt_tau, c->filt_eps_max,
                                     c->filt_relax, part, c->d_filt + 2 * f, tab);
    k_filt_apply<<<dim3((c->nc + tb - 1) / tb, c->K, c->M), tb, 0, st>>>(c->nc, c->M, c->Kz, c->K, c->d_soff,
                                                                         tab, s);
  }
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

extern "C" {

int mlx_filter_setup(mlx_ctx* c, int enable, const mlx_filter_params* p) {
  if (!c) return MLX_EINVAL;
  if (p && !(p->zeta_c >= 0.0 && p->zeta_c < 1.0 && p->tau > 0.0 && p->eps_max >= 0.0 && p->relax > 0.0 &&
             p->relax <= 1.0))
    return MLX_EINVAL;
  if (enable) {
    int rc = filt_buffers(c);
    if (rc) return rc;
    MLX_CUDA_TRY(c, cudaMemset(c->d_filt, 0, sizeof(double) * 4));
    c->filt_zeta_c = p ? p->zeta_c : 2.0 / 3.0;
    c->filt_tau = p ? p->tau : 2e-2;
    c->filt_eps_max = p ? p->eps_max : 36.0;
    c->filt_relax = p ? p->relax : 0.25;
  }
  c->filter_on = enable != 0;
  mlx_invalidate_graphs(c);
  return MLX_OK;
}

int mlx_filter_apply(mlx_ctx* c, void* state, int nfields, mlx_stream stream) {
  if (!c || !state || (((uintptr_t)state) & 15u) || nfields < 1 || nfields > 2) return MLX_EINVAL;
  if (!c->d_filt) return MLX_ESTATE;
  return mlx_filter_fields(c, nfields, (double2*)state, (cudaStream_t)stream);
}

int mlx_filter_state(mlx_ctx* c, double* eps, double* tail) {
  if (!c) return MLX_EINVAL;
  if (!c->d_filt) return MLX_ESTATE;
  double h[4];
  MLX_CUDA_TRY(c, cudaMemcpy(h, c->d_filt, sizeof(h), cudaMemcpyDeviceToHost));
  if (eps) { eps[0] = h[0]; eps[1] = h[2]; }
  if (tail) { tail[0] = h[1]; tail[1] = h[3]; }
  return MLX_OK;
}

}  // extern "C"
