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
#include "mlx_internal.cuh"

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
                                double2* __restrict__ rwp, double2* __restrict__ wz) {
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
    rvr[idx] = cadd(cimul(mm, P[a]), cimul(kap, Rchi));
    rvp[idx] = csub(cmulr(-1.0, Rpsi), cmulr(mm * kap, Ch[a]));
    vz[idx] = cmulr(-1.0, Dc[a]);
    rwr[idx] = cadd(cimul(mm, Ps[a]), cimul(kap, Rpsi));
    rwp[idx] = csub(cmulr(-1.0, RPsi), cmulr(mm * kap, P[a]));
    wz[idx] = cmulr(-1.0, apply_D(db, P, a, Nm));
  }
}

template <typename T>
__device__ __forceinline__ bool vortex_product_at(long long idx, int nphi, int nr, T U0,
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
  const T rvr = f0[idx], rvp = f1[idx], vz = f2[idx], rwr = f3[idx], rwp = f4[idx], wz = f5[idx];
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
__global__ void k_vortex_product(long long n_phys, int nphi, int nr, T U0, const double* __restrict__ rnode,
                                 T* __restrict__ f0, T* __restrict__ f1, T* __restrict__ f2,
                                 const T* __restrict__ f3, const T* __restrict__ f4, const T* __restrict__ f5,
                                 int* __restrict__ err) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool finite = true;
  if (idx < n_phys) finite = vortex_product_at(idx, nphi, nr, U0, rnode, f0, f1, f2, f3, f4, f5);
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
constexpr int kEnThreads = 128;
__global__ void __launch_bounds__(kEnThreads) k_energy_blocks(int nc, int nr, int K, const long long* __restrict__ soff,
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
  const long long base = soff[m] + (long long)kidx * Nm;
  for (int a = threadIdx.x; a < Nm; a += blockDim.x) {
    ev[a] = rvr[base + a];
    ev[Nm + a] = rvp[base + a];
    ev[2 * Nm + a] = vz[base + a];
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
  if (threadIdx.x == 0) part[(long long)m * K + kidx] = (m == 0 ? 1.0 : 2.0) * red[0];
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
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_jac, sizeof(double) * c->tri));
  k_jac_table<<<nblk(c->tri, 256), 256, 0, st>>>(c->M, c->nc, c->d_lap_off, c->d_jac);
  MLX_LAUNCH_CHECK(c);
  MLX_CUDA_TRY(c, cudaMalloc(&c->d_vspec, sizeof(double2) * c->n_spec * 9));
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
  {
    const int vt = c->nc >= 256 ? 256 : ((c->nc + 31) / 32) * 32;
    k_vortex_fields<<<dim3(c->K, c->M), vt, sizeof(double2) * 4 * c->nc, st>>>(
        c->nc, c->Kz, c->K, c->lz, c->d_soff, c->d_lap_off, c->d_rdr, c->d_lap, psi, chi, F[0], F[1], F[2], F[3],
        F[4], F[5]);
  }
  MLX_LAUNCH_CHECK(c);
  int rc;
  for (int f = 0; f < 6; ++f) {
    if ((rc = mlx_legendre_backward(c, F[f], st))) return rc;
    if ((rc = mlx_fft_backward(c, P[f], st))) return rc;
  }
  k_vortex_product<T><<<nblk(np, tb), tb, 0, st>>>(np, c->nphi, c->nr, (T)U0, c->d_r, P[0], P[1], P[2], P[3],
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
  k_vortex_fields<<<dim3(c->K, c->M), vt, sizeof(double2) * 4 * c->nc, st>>>(
      c->nc, c->Kz, c->K, c->lz, c->d_soff, c->d_lap_off, c->d_rdr, c->d_lap, psi, chi, F[0], F[1], F[2], F[3],
      F[4], F[5]);
  MLX_LAUNCH_CHECK(c);
  // the partial sums go to the (then unused) seventh spectral temporary
  double* part = reinterpret_cast<double*>(c->d_vspec + ns * 6);
  if ((long long)c->M * c->K > 2 * ns) return MLX_EINVAL;
  k_energy_blocks<<<dim3(c->K, c->M), kEnThreads, sizeof(double2) * 3 * c->nc, st>>>(
      c->nc, c->nr, c->K, c->d_soff, c->d_boff, c->d_x, c->d_w, c->d_r, c->d_P64, F[0], F[1], F[2], part);
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
