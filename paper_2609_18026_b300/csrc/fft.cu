// K2/K3: azimuthal (real) and axial (complex) Fourier transforms of the
// transform pair (Eq. (2)), as batched shared-memory FFTs.
//
// Layouts (planar complex, r fastest so that a warp reads consecutive radii):
//   physical  [Nz][Nphi][Nr] real
//   zm        [2][Nz][M][Nr]      after the phi transform (Re plane, Im plane)
//   mixed     [2][K][M][Nr]       after the z transform; for Nz == 1 zm == mixed
// A CTA of the phi kernel owns one z-plane and a tile of R radii; two real radial
// lines (r and r + R/2) are packed into one complex line of length Nphi.  A CTA of
// the z kernel owns one m and a tile of radii.  Transforms are radix-2 Stockham
// passes over smem buffers laid out [point][line] (line fastest).
#include "mlx_internal.cuh"

namespace {

template <typename T> struct C2T;
template <> struct C2T<float> { typedef float2 type; };
template <> struct C2T<double> { typedef double2 type; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}

// Radix-2 Stockham FFT of B lines of length N held at x[pos * B + line].
// tw[t] = exp(-2 pi i t / N) for t < N/2; inverse uses the conjugate (no 1/N).
// Returns the buffer (x or y) that holds the result in natural order.
template <typename C>
__device__ C* fft_lines(C* x, C* y, int N, int B, const C* __restrict__ tw, bool inverse) {
  int n = N, s = 1;
  const int half = (N >> 1) * B;
  while (n > 1) {
    const int m = n >> 1;
    for (int t = threadIdx.x; t < half; t += blockDim.x) {
      const int b = t % B;
      const int pq = t / B;
      const int q = pq % s;
      const int p = pq / s;
      C w = tw[p * s];
      if (inverse) w.y = -w.y;
      const C a0 = x[(q + s * p) * B + b];
      const C a1 = x[(q + s * (p + m)) * B + b];
      y[(q + s * (2 * p)) * B + b] = cadd(a0, a1);
      y[(q + s * (2 * p + 1)) * B + b] = cmul(csub(a0, a1), w);
    }
    __syncthreads();
    C* tmp = x; x = y; y = tmp;
    n = m;
    s <<= 1;
  }
  return x;
}

enum PhiMode { PHI_FWD = 0, PHI_BWD = 1, PHI_FKPP = 2 };

// Forward real analysis of the packed lines in buf (result of fft_lines with
// sign -1), scaled by 1/N, written to zm for this (z, r-tile).
template <typename T, typename C>
__device__ void phi_unpack_store(const C* buf, int N, int B, int M, int Nr, int r0, int z,
                                 T* __restrict__ zre, T* __restrict__ zim) {
  const T inv = (T)1 / (T)N;
  const int R = 2 * B;
  for (int t = threadIdx.x; t < M * R; t += blockDim.x) {
    const int m = t / R, rr = t % R;
    const int b = rr % B;
    const C zm = buf[m * B + b];
    const C zc = buf[((N - m) % N) * B + b];
    T re, im;
    if (rr < B) {  // X_m = (Z_m + conj(Z_{N-m})) / 2
      re = (zm.x + zc.x) * (T)0.5;
      im = (zm.y - zc.y) * (T)0.5;
    } else {       // Y_m = (Z_m - conj(Z_{N-m})) / (2i)
      re = (zm.y + zc.y) * (T)0.5;
      im = (zc.x - zm.x) * (T)0.5;
    }
    const int r = r0 + rr;
    if (r < Nr) {
      const long long o = ((long long)z * M + m) * Nr + r;
      zre[o] = re * inv;
      zim[o] = im * inv;
    }
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_phi(int N, int M, int Nr, int R, T* __restrict__ phys,
                                             T* __restrict__ zre, T* __restrict__ zim,
                                             const typename C2T<T>::type* __restrict__ tw, T gamma) {
  typedef typename C2T<T>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* bufA = reinterpret_cast<C*>(smem_raw);
  const int B = R / 2;
  C* bufB = bufA + N * B;
  const int r0 = blockIdx.x * R;
  const int z = blockIdx.y;
  const long long plane = (long long)z * N * Nr;

  if constexpr (MODE == PHI_FWD) {
    for (int t = threadIdx.x; t < N * R; t += blockDim.x) {
      const int j = t / R, rr = t % R;
      const int r = r0 + rr;
      const T v = (r < Nr) ? phys[plane + (long long)j * Nr + r] : (T)0;
      T* slot = reinterpret_cast<T*>(&bufA[j * B + (rr % B)]);
      slot[rr < B ? 0 : 1] = v;
    }
    __syncthreads();
    C* res = fft_lines<C>(bufA, bufB, N, B, tw, false);
    phi_unpack_store<T, C>(res, N, B, M, Nr, r0, z, zre, zim);
  } else {
  // synthesis: build the packed Hermitian spectrum of line pairs
  for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
    C zero; zero.x = 0; zero.y = 0;
    bufA[t] = zero;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < M * B; t += blockDim.x) {
    const int m = t / B, b = t % B;
    const int ra = r0 + b, rb = r0 + b + B;
    T ar = 0, ai = 0, br = 0, bi = 0;
    const long long oa = ((long long)z * M + m) * Nr;
    if (ra < Nr) { ar = zre[oa + ra]; ai = zim[oa + ra]; }
    if (rb < Nr) { br = zre[oa + rb]; bi = zim[oa + rb]; }
    if (m == 0) {
      C v; v.x = ar; v.y = br;       // real parts of the mean modes
      bufA[b] = v;
    } else {
      C v1; v1.x = ar - bi; v1.y = ai + br;   // A_m + i B_m
      C v2; v2.x = ar + bi; v2.y = br - ai;   // conj(A_m) + i conj(B_m)
      bufA[m * B + b] = v1;
      bufA[(N - m) * B + b] = v2;
    }
  }
  __syncthreads();
  C* res = fft_lines<C>(bufA, bufB, N, B, tw, true);
  if constexpr (MODE == PHI_BWD) {
    for (int t = threadIdx.x; t < N * R; t += blockDim.x) {
      const int j = t / R, rr = t % R;
      const int r = r0 + rr;
      const C v = res[j * B + (rr % B)];
      if (r < Nr) phys[plane + (long long)j * Nr + r] = (rr < B) ? v.x : v.y;
    }
  } else {
  // PHI_FKPP: pointwise gamma u (1 - u) at the nodes, then analysis again
  for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
    C v = res[t];
    v.x = gamma * v.x * ((T)1 - v.x);
    v.y = gamma * v.y * ((T)1 - v.y);
    res[t] = v;
  }
  __syncthreads();
  C* other = (res == bufA) ? bufB : bufA;
  C* res2 = fft_lines<C>(res, other, N, B, tw, false);
  phi_unpack_store<T, C>(res2, N, B, M, Nr, r0, z, zre, zim);
  }
  }
}

// Axial transform for one m and a tile of R radii: lines are radii.
template <typename T, bool INVERSE>
__global__ void __launch_bounds__(256) k_z(int Nz, int Kz, int K, int M, int Nr, int R,
                                           T* __restrict__ zre, T* __restrict__ zim,
                                           T* __restrict__ mre, T* __restrict__ mim,
                                           const typename C2T<T>::type* __restrict__ tw) {
  typedef typename C2T<T>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + Nz * R;
  const int r0 = blockIdx.x * R;
  const int m = blockIdx.y;
  if (!INVERSE) {
    for (int t = threadIdx.x; t < Nz * R; t += blockDim.x) {
      const int l = t / R, b = t % R;
      const int r = r0 + b;
      C v; v.x = 0; v.y = 0;
      if (r < Nr) {
        const long long o = ((long long)l * M + m) * Nr + r;
        v.x = zre[o]; v.y = zim[o];
      }
      bufA[t] = v;
    }
    __syncthreads();
    C* res = fft_lines<C>(bufA, bufB, Nz, R, tw, false);
    const T inv = (T)1 / (T)Nz;
    for (int t = threadIdx.x; t < K * R; t += blockDim.x) {
      const int kk = t / R, b = t % R;
      const int r = r0 + b;
      const int pos = (kk < Kz) ? kk : Nz - (K - kk);
      if (r < Nr) {
        const C v = res[pos * R + b];
        const long long o = ((long long)kk * M + m) * Nr + r;
        mre[o] = v.x * inv;
        mim[o] = v.y * inv;
      }
    }
  } else {
    for (int t = threadIdx.x; t < Nz * R; t += blockDim.x) {
      C zero; zero.x = 0; zero.y = 0;
      bufA[t] = zero;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < K * R; t += blockDim.x) {
      const int kk = t / R, b = t % R;
      const int r = r0 + b;
      const int pos = (kk < Kz) ? kk : Nz - (K - kk);
      if (r < Nr) {
        const long long o = ((long long)kk * M + m) * Nr + r;
        C v; v.x = mre[o]; v.y = mim[o];
        bufA[pos * R + b] = v;
      }
    }
    __syncthreads();
    C* res = fft_lines<C>(bufA, bufB, Nz, R, tw, true);
    for (int t = threadIdx.x; t < Nz * R; t += blockDim.x) {
      const int l = t / R, b = t % R;
      const int r = r0 + b;
      if (r < Nr) {
        const C v = res[t];
        const long long o = ((long long)l * M + m) * Nr + r;
        zre[o] = v.x;
        zim[o] = v.y;
      }
    }
  }
}

template <typename T>
int phi_launch(mlx_ctx* c, int mode, T* phys, T* zbase, const void* tw, double gamma,
               cudaStream_t st) {
  typedef typename C2T<T>::type C;
  int R = 32;
  size_t smem = (size_t)2 * c->nphi * (R / 2) * sizeof(C);
  while (smem > 200 * 1024 && R > 2) { R /= 2; smem = (size_t)2 * c->nphi * (R / 2) * sizeof(C); }
  dim3 grid((c->nr + R - 1) / R, c->nz);
  const long long pl = (long long)c->nz * c->M * c->nr;
  T* zre = zbase;
  T* zim = zbase + pl;
  const C* twp = reinterpret_cast<const C*>(tw);
  TimedLaunch tl(c, mode == PHI_FWD ? KID_PHI_FWD : (mode == PHI_BWD ? KID_PHI_BWD : KID_PHI_FKPP), st);
  if (mode == PHI_FWD) {
    k_phi<T, PHI_FWD><<<grid, 256, smem, st>>>(c->nphi, c->M, c->nr, R, phys, zre, zim, twp, (T)gamma);
  } else if (mode == PHI_BWD) {
    k_phi<T, PHI_BWD><<<grid, 256, smem, st>>>(c->nphi, c->M, c->nr, R, phys, zre, zim, twp, (T)gamma);
  } else {
    k_phi<T, PHI_FKPP><<<grid, 256, smem, st>>>(c->nphi, c->M, c->nr, R, phys, zre, zim, twp, (T)gamma);
  }
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

template <typename T>
int z_launch(mlx_ctx* c, bool inverse, T* zbase, T* mbase, const void* tw, cudaStream_t st) {
  typedef typename C2T<T>::type C;
  int R = 32;
  size_t smem = (size_t)2 * c->nz * R * sizeof(C);
  while (smem > 200 * 1024 && R > 1) { R /= 2; smem = (size_t)2 * c->nz * R * sizeof(C); }
  dim3 grid((c->nr + R - 1) / R, c->M);
  const long long plz = (long long)c->nz * c->M * c->nr;
  const long long plm = (long long)c->K * c->M * c->nr;
  const C* twp = reinterpret_cast<const C*>(tw);
  TimedLaunch tl(c, inverse ? KID_Z_BWD : KID_Z_FWD, st);
  if (!inverse) {
    k_z<T, false><<<grid, 256, smem, st>>>(c->nz, c->Kz, c->K, c->M, c->nr, R, zbase, zbase + plz,
                                           mbase, mbase + plm, twp);
  } else {
    k_z<T, true><<<grid, 256, smem, st>>>(c->nz, c->Kz, c->K, c->M, c->nr, R, zbase, zbase + plz,
                                          mbase, mbase + plm, twp);
  }
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

template <typename T>
int fft_forward_t(mlx_ctx* c, const void* phys, cudaStream_t st, const void* twphi, const void* twz) {
  T* mixed = reinterpret_cast<T*>(c->d_mixed);
  if (c->nz == 1) return phi_launch<T>(c, PHI_FWD, (T*)phys, mixed, twphi, 0.0, st);
  T* zm = reinterpret_cast<T*>(c->d_zm);
  int rc = phi_launch<T>(c, PHI_FWD, (T*)phys, zm, twphi, 0.0, st);
  if (rc) return rc;
  return z_launch<T>(c, false, zm, mixed, twz, st);
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
  if (c->nz == 1) return phi_launch<T>(c, PHI_FKPP, nullptr, mixed, twphi, gamma, st);
  T* zm = reinterpret_cast<T*>(c->d_zm);
  int rc = z_launch<T>(c, true, zm, mixed, twz, st);
  if (rc) return rc;
  rc = phi_launch<T>(c, PHI_FKPP, nullptr, zm, twphi, gamma, st);
  if (rc) return rc;
  return z_launch<T>(c, false, zm, mixed, twz, st);
}

}  // namespace

// Opt every FFT kernel into the largest dynamic shared memory any size needs
// (the launch helpers keep each launch below 200 KB).
int mlx_fft_prepare(mlx_ctx* c) {
  const int lim = 200 * 1024;
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_phi<float, PHI_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_phi<float, PHI_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_phi<float, PHI_FKPP>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_phi<double, PHI_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_phi<double, PHI_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_phi<double, PHI_FKPP>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_z<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_z<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_z<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  MLX_CUDA_TRY(c, cudaFuncSetAttribute(k_z<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return MLX_OK;
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
