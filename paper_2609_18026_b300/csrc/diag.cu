// Integral diagnostics and checkpoint images of a spectral field (boundary calls
// mlx_diag, mlx_state_bytes, mlx_get_state, mlx_set_state).
//
// mlx_diag evaluates, in FP64 and from the coefficients alone (no transform of the
// context's precision), the plane integrals of Eq. (16) and the area-weighted L2
// norm under the mapped measure r dr = ell^2 dx / (1 - x)^2 (Eq. (1)):
//   integral = (1/Lz) int f dA dz      = 2 pi ell^2 sum_i w_i/(1-x_i)^2 f_00(x_i)
//   moment2  = (1/Lz) int r^2 f dA dz  = 2 pi ell^2 sum_i w_i r_i^2/(1-x_i)^2 f_00(x_i)
//   l2w^2    = (1/Lz) int f^2 dA dz    = 2 pi ell^2 sum_i w_i/(1-x_i)^2 sum_{m,k} mult_m |f_mk(x_i)|^2
// with f_mk(x_i) = sum_n shat_nmk Pbar_n^m(x_i) (the FP64 table of the context), mult_m
// = 1 for m = 0 and 2 otherwise (Parseval over phi and z for the real field of Eq. (2)),
// and spec_l2^2 = sum mult_m |shat|^2.  For a vorticity field, integral and moment2 are
// the circulation Gamma and the second moment M2 of Eq. (16).  One CTA per (m, k)
// block writes its partial sums; one CTA adds them in a fixed order (deterministic).
#include "mlx_internal.cuh"

#include <string.h>

namespace {

constexpr int kDiagThreads = 128;

__global__ void __launch_bounds__(kDiagThreads) k_diag_blocks(int nc, int nr, int K, double ell,
                                                              const long long* __restrict__ soff,
                                                              const long long* __restrict__ boff,
                                                              const double* __restrict__ x,
                                                              const double* __restrict__ w,
                                                              const double* __restrict__ r,
                                                              const double* __restrict__ P64,
                                                              const double2* __restrict__ spec,
                                                              double* __restrict__ part) {
  extern __shared__ double2 sv[];                 // the block's Nc - m coefficients
  __shared__ double red[4][kDiagThreads];
  const int kidx = blockIdx.x, m = blockIdx.y;
  const int Nm = nc - m;
  const double2* blk = spec + soff[m] + (long long)kidx * Nm;
  double sp = 0.0;
  for (int a = threadIdx.x; a < Nm; a += blockDim.x) {
    const double2 v = blk[a];
    sv[a] = v;
    sp = fma(v.x, v.x, fma(v.y, v.y, sp));
  }
  __syncthreads();
  const double mult = m == 0 ? 1.0 : 2.0;
  const double* Pm = P64 + boff[m];               // [n - m][i]
  double l2 = 0.0, f1 = 0.0, f2 = 0.0;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    double fr = 0.0, fi = 0.0;
    for (int a = 0; a < Nm; ++a) {
      const double p = Pm[(long long)a * nr + i];
      fr = fma(p, sv[a].x, fr);
      fi = fma(p, sv[a].y, fi);
    }
    const double om = 1.0 - x[i];
    const double aw = w[i] / (om * om);
    l2 = fma(aw, fma(fr, fr, fi * fi), l2);
    f1 = fma(aw, fr, f1);
    f2 = fma(aw * r[i] * r[i], fr, f2);
  }
  red[0][threadIdx.x] = mult * sp;
  red[1][threadIdx.x] = mult * l2;
  red[2][threadIdx.x] = f1;
  red[3][threadIdx.x] = f2;
  __syncthreads();
  for (int h = kDiagThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long b = (long long)m * K + kidx;
    part[b * 4 + 0] = red[0][0];
    part[b * 4 + 1] = red[1][0];
    part[b * 4 + 2] = (m == 0 && kidx == 0) ? red[2][0] : 0.0;
    part[b * 4 + 3] = (m == 0 && kidx == 0) ? red[3][0] : 0.0;
  }
}

__global__ void k_diag_sum(long long nblocks, double ell, const double* __restrict__ part,
                           double* __restrict__ out) {
  __shared__ double red[2][256];
  double a = 0.0, b = 0.0;
  for (long long j = threadIdx.x; j < nblocks; j += blockDim.x) {
    a += part[j * 4 + 0];
    b += part[j * 4 + 1];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[0][threadIdx.x] += red[0][threadIdx.x + h];
      red[1][threadIdx.x] += red[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double c = 2.0 * M_PI * ell * ell;
    out[0] = c * part[2];                       // the (m, k) = (0, 0) block holds f_00
    out[1] = c * part[3];
    out[2] = sqrt(c * red[1][0]);
    out[3] = sqrt(red[0][0]);
  }
}

// checkpoint image header (host side only)
struct StateHeader {
  char magic[8];                 // "MLXSTAT2"
  int nr, nphi, nz, nc, M, Kz, nfields, p;
  double ell, lz, nu, nu_h, dt;
  long long step;
  long long n_spec;
  int implicit_ready, pad;
  double lp_cpsi, lp_cchi, vortex_uz;   // log-proxy amplitudes and axial background (vortex)
};

int nfields_of(int kind) { return kind == MLX_NONLIN_VORTEX ? 2 : 1; }

}  // namespace

extern "C" {

int mlx_diag(mlx_ctx* c, const void* spec, mlx_diag_out* out, mlx_stream stream) {
  if (!c || !spec || !out || (((uintptr_t)spec) & 15u)) return MLX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const long long nb = (long long)c->M * c->K;
  if (!c->d_diag) MLX_CUDA_TRY(c, cudaMalloc(&c->d_diag, sizeof(double) * (nb * 4 + 4)));
  k_diag_blocks<<<dim3(c->K, c->M), kDiagThreads, sizeof(double2) * c->nc, st>>>(
      c->nc, c->nr, c->K, c->ell, c->d_soff, c->d_boff, c->d_x, c->d_w, c->d_r, c->d_P64,
      (const double2*)spec, c->d_diag);
  MLX_LAUNCH_CHECK(c);
  k_diag_sum<<<1, 256, 0, st>>>(nb, c->ell, c->d_diag, c->d_diag + nb * 4);
  MLX_LAUNCH_CHECK(c);
  double h[4];
  MLX_CUDA_TRY(c, cudaMemcpyAsync(h, c->d_diag + nb * 4, sizeof(h), cudaMemcpyDeviceToHost, st));
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  out->integral = h[0];
  out->moment2 = h[1];
  out->l2w = h[2];
  out->spec_l2 = h[3];
  return MLX_OK;
}

long long mlx_state_bytes(const mlx_ctx* c, int kind) {
  if (!c || (kind != MLX_NONLIN_NONE && kind != MLX_NONLIN_FKPP && kind != MLX_NONLIN_VORTEX)) return -1;
  return (long long)sizeof(StateHeader) + 2LL * nfields_of(kind) * c->n_spec * (long long)sizeof(double2);
}

int mlx_get_state(mlx_ctx* c, int kind, const void* state, const void* prev_A, long long step, void* host,
                  long long bytes, mlx_stream stream) {
  const long long need = mlx_state_bytes(c, kind);
  if (need < 0 || !state || !prev_A || !host || bytes < need) return MLX_EINVAL;
  StateHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, "MLXSTAT2", 8);
  hd.nr = c->nr; hd.nphi = c->nphi; hd.nz = c->nz; hd.nc = c->nc; hd.M = c->M; hd.Kz = c->Kz;
  hd.nfields = nfields_of(kind);
  hd.p = c->p;
  hd.ell = c->ell; hd.lz = c->lz; hd.nu = c->nu; hd.nu_h = c->nu_h; hd.dt = c->dt;
  hd.step = step;
  hd.n_spec = c->n_spec;
  hd.implicit_ready = c->implicit_ready ? 1 : 0;
  if (kind == MLX_NONLIN_VORTEX) {
    hd.lp_cpsi = c->lp_cpsi; hd.lp_cchi = c->lp_cchi; hd.vortex_uz = c->vortex_uz;
  }
  memcpy(host, &hd, sizeof(hd));
  const size_t fb = sizeof(double2) * (size_t)hd.nfields * (size_t)c->n_spec;
  unsigned char* dst = static_cast<unsigned char*>(host) + sizeof(hd);
  cudaStream_t st = (cudaStream_t)stream;
  MLX_CUDA_TRY(c, cudaMemcpyAsync(dst, state, fb, cudaMemcpyDeviceToHost, st));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(dst + fb, prev_A, fb, cudaMemcpyDeviceToHost, st));
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  return MLX_OK;
}

int mlx_set_state(mlx_ctx* c, int kind, const void* host, long long bytes, void* state, void* prev_A,
                  long long* step, mlx_stream stream) {
  const long long need = mlx_state_bytes(c, kind);
  if (need < 0 || !state || !prev_A || !host || bytes < need) return MLX_EINVAL;
  StateHeader hd;
  memcpy(&hd, host, sizeof(hd));
  auto reject = [&](const char* why) {
    c->last_err = std::string("mlx_set_state: ") + why;
    return MLX_EINVAL;
  };
  if (memcmp(hd.magic, "MLXSTAT2", 8) != 0) return reject("not a checkpoint image");
  if (hd.nr != c->nr || hd.nphi != c->nphi || hd.nz != c->nz || hd.nc != c->nc || hd.M != c->M ||
      hd.Kz != c->Kz || hd.n_spec != c->n_spec || hd.ell != c->ell || hd.lz != c->lz)
    return reject("grid, chops, ell or Lz differ from this context");
  if (hd.nfields != nfields_of(kind)) return reject("the image holds another number of fields");
  // A^{j-1} continues the AB-CN recurrence only with the same operator and step
  if (hd.implicit_ready && c->implicit_ready &&
      (hd.dt != c->dt || hd.nu != c->nu || hd.nu_h != c->nu_h || (hd.nu_h > 0.0 && hd.p != c->p)))
    return reject("dt, nu, nu_h or p differ from this context's implicit setup");
  // the proxy amplitudes are part of a vortex state: set them (mlx_vortex_logproxy)
  // before restoring it
  if (kind == MLX_NONLIN_VORTEX &&
      (hd.lp_cpsi != c->lp_cpsi || hd.lp_cchi != c->lp_cchi || hd.vortex_uz != c->vortex_uz))
    return reject("the log-proxy amplitudes or the axial background differ from this context's");
  const size_t fb = sizeof(double2) * (size_t)hd.nfields * (size_t)c->n_spec;
  const unsigned char* src = static_cast<const unsigned char*>(host) + sizeof(hd);
  cudaStream_t st = (cudaStream_t)stream;
  MLX_CUDA_TRY(c, cudaMemcpyAsync(state, src, fb, cudaMemcpyHostToDevice, st));
  MLX_CUDA_TRY(c, cudaMemcpyAsync(prev_A, src + fb, fb, cudaMemcpyHostToDevice, st));
  MLX_CUDA_TRY(c, cudaStreamSynchronize(st));
  if (step) *step = hd.step;
  return MLX_OK;
}

}  // extern "C"
