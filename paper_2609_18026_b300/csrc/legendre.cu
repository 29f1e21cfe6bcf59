// K4 (SIMT form): the ragged per-m Gauss-quadrature contraction of the transform
// pair (Eq. (2) and its quadrature inverse, Sec. 3.1).
//
// Forward, per m:  spec[m][k][n] = sum_i W_m[n][i] X[k][m][i]   (W = w_i Pbar_n^m(x_i))
// Backward, per m: X[k][m][i]    = sum_n P_m[n][i] spec[m][k][n]
// The real basis times complex data is one real GEMM with 2K columns
// (column c < K: Re of wavenumber slot c; c >= K: Im of slot c - K).
// Work is a host-built list of 64 x 64 output tiles over (m, row tile, col tile),
// so the triangle's shrinking row count (Nc - m) wastes no whole tiles.
// T is the storage and accumulation type (double: FP64 parity form; float: FP32).
#include "mlx_internal.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// One 64 x 64 output tile.
template <typename T, bool FWD>
__device__ __forceinline__ void leg_tile(const LegTile tile, int nc, int nr, int M, int K,
                                         const long long* __restrict__ boff, const long long* __restrict__ soff,
                                         const T* __restrict__ table,  // W (fwd) or P (bwd)
                                         T* __restrict__ mixed,        // planar [2][K][M][Nr]
                                         double2* __restrict__ spec,
                                         const double2* __restrict__ addsrc, double alpha,
                                         T (&As)[BK][BM + 1], T (&Bs)[BK][BN + 1]) {
  const int m = tile.m;
  const int Nm = nc - m;
  const int rows = FWD ? Nm : nr;         // output rows
  const int kdim = FWD ? nr : Nm;         // contraction length
  const int row0 = tile.row0, col0 = tile.col0;
  const int ncol = 2 * K;
  const long long plane = (long long)K * M * nr;
  const T* tab = table + boff[m];
  const long long so = soff[m];
  const int tid = threadIdx.x;
  const int tr = tid & 15, tc = tid >> 4;

  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;

  for (int k0 = 0; k0 < kdim; k0 += BK) {
    // A tile: A(row, kk)
    for (int t = tid; t < BM * BK; t += NT) {
      int row, kk;
      if (FWD) { kk = t % BK; row = t / BK; }   // W_m[row][kk] contiguous in kk
      else     { row = t % BM; kk = t / BM; }   // P_m[kk][row] contiguous in row (= i)
      const int gr = row0 + row, gk = k0 + kk;
      T v = (T)0;
      if (gr < rows && gk < kdim)
        v = FWD ? tab[(long long)gr * nr + gk] : tab[(long long)gk * nr + gr];
      As[kk][row] = v;
    }
    // B tile: B(kk, col)
    for (int t = tid; t < BK * BN; t += NT) {
      const int kk = t % BK, col = t / BK;
      const int gk = k0 + kk, gc = col0 + col;
      T v = (T)0;
      if (gk < kdim && gc < ncol) {
        const int p = gc >= K;
        const int kidx = gc - p * K;
        if (FWD) {
          v = mixed[p * plane + ((long long)kidx * M + m) * nr + gk];
        } else {
          const double2 s = spec[so + (long long)kidx * Nm + gk];
          v = (T)(p ? s.y : s.x);
        }
      }
      Bs[kk][col] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[kk][tr + 16 * q]; b[q] = Bs[kk][tc + 16 * q]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int gr = row0 + tr + 16 * x;
    if (gr >= rows) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int gc = col0 + tc + 16 * y;
      if (gc >= ncol) continue;
      const int p = gc >= K;
      const int kidx = gc - p * K;
      if (FWD) {
        const long long o = so + (long long)kidx * Nm + gr;
        double val = (double)acc[x][y];
        if (addsrc) val += alpha * (p ? addsrc[o].y : addsrc[o].x);   // FP64 epilogue term
        reinterpret_cast<double*>(&spec[o])[p] = val;
      } else {
        mixed[p * plane + ((long long)kidx * M + m) * nr + gr] = acc[x][y];
      }
    }
  }
}

template <typename T, bool FWD>
__global__ void __launch_bounds__(NT) k_legendre(const LegTile* __restrict__ tiles, int nc, int nr,
                                                 int M, int K, const long long* __restrict__ boff,
                                                 const long long* __restrict__ soff,
                                                 const T* __restrict__ table, T* __restrict__ mixed,
                                                 double2* __restrict__ spec,
                                                 const double2* __restrict__ addsrc, double alpha) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  leg_tile<T, FWD>(tiles[blockIdx.x], nc, nr, M, K, boff, soff, table, mixed, spec, addsrc, alpha, As, Bs);
}

// Batched persistent form (batch.cu): CTAs take (member, tile) items from the
// queue; item = {m, row0, col0, member}.
template <typename T, bool FWD>
__global__ void __launch_bounds__(NT) kb_legendre(const BLegJob* __restrict__ jobs, const LegTile* __restrict__ items,
                                                  int nitems, int* __restrict__ ctr) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  __shared__ int s_it;
  for (;;) {
    if (threadIdx.x == 0) s_it = atomicAdd(ctr, 1);
    __syncthreads();
    const int it = s_it;
    if (it >= nitems) break;
    const LegTile t = items[it];
    const BLegJob j = jobs[t.pad];
    leg_tile<T, FWD>(t, j.nc, j.nr, j.M, j.K, j.boff, j.soff, (const T*)j.table, (T*)j.mixed, j.spec, nullptr,
                     0.0, As, Bs);
    __syncthreads();
  }
  if (threadIdx.x == 0) bq_finish(ctr, gridDim.x);
}

}  // namespace

int mlx_legendre_tiles(mlx_ctx* c, std::vector<LegTile>& fwd, std::vector<LegTile>& bwd);

// ---- batched persistent SIMT contraction (FP32 / FP64 members) ----
// Job and items of member c (index inst): forward (mixed -> spec) or backward
// (spec -> mixed), the member's own 64 x 64 tiles.
void mlx_legendre_batch_member(mlx_ctx* c, bool fwd, int inst, double2* spec, BLegJob* job,
                               std::vector<LegTile>& items, std::vector<double>& cost) {
  BLegJob j;
  j.nc = c->nc; j.nr = c->nr; j.M = c->M; j.K = c->K;
  j.boff = c->d_boff; j.soff = c->d_soff;
  const bool dbl = c->precision == MLX_FP64;
  j.table = fwd ? (dbl ? (const void*)c->d_W64 : (const void*)c->d_W32)
                : (dbl ? (const void*)c->d_P64 : (const void*)c->d_P32);
  j.mixed = c->d_mixed;
  j.spec = spec;
  *job = j;
  std::vector<LegTile> tf, tb;
  mlx_legendre_tiles(c, tf, tb);
  for (const LegTile& t : (fwd ? tf : tb)) {
    const int kdim = fwd ? c->nr : c->nc - t.m;
    items.push_back(LegTile{t.m, t.row0, t.col0, inst});
    cost.push_back((double)((kdim + BK - 1) / BK));
  }
}

int mlx_legendre_batch_launch(bool fwd, bool dbl, const BLegJob* jobs, const LegTile* items, int nitems,
                              int* ctr, int grid, cudaStream_t st) {
  if (dbl) {
    if (fwd) kb_legendre<double, true><<<grid, NT, 0, st>>>(jobs, items, nitems, ctr);
    else kb_legendre<double, false><<<grid, NT, 0, st>>>(jobs, items, nitems, ctr);
  } else {
    if (fwd) kb_legendre<float, true><<<grid, NT, 0, st>>>(jobs, items, nitems, ctr);
    else kb_legendre<float, false><<<grid, NT, 0, st>>>(jobs, items, nitems, ctr);
  }
  return cudaGetLastError() == cudaSuccess ? MLX_OK : MLX_ECUDA;
}

const void* mlx_legendre_batch_kernel(bool fwd, bool dbl) {
  if (dbl) return fwd ? (const void*)kb_legendre<double, true> : (const void*)kb_legendre<double, false>;
  return fwd ? (const void*)kb_legendre<float, true> : (const void*)kb_legendre<float, false>;
}

int mlx_legendre_forward(mlx_ctx* c, double2* spec, cudaStream_t st, const double2* addsrc,
                         double alpha) {
  // the BF16X3 forward FFT writes the split planes of the tensor-core form only
  if (c->precision == MLX_BF16X3) return addsrc ? MLX_EINVAL : mlx_legendre_tc_forward(c, spec, st);
  TimedLaunch tl(c, KID_LEG_FWD, st);
  if (c->precision == MLX_FP64)
    k_legendre<double, true><<<c->ntiles_fwd, NT, 0, st>>>(c->d_tiles_fwd, c->nc, c->nr, c->M, c->K,
                                                          c->d_boff, c->d_soff, c->d_W64,
                                                          (double*)c->d_mixed, spec, addsrc, alpha);
  else
    k_legendre<float, true><<<c->ntiles_fwd, NT, 0, st>>>(c->d_tiles_fwd, c->nc, c->nr, c->M, c->K,
                                                         c->d_boff, c->d_soff, c->d_W32,
                                                         (float*)c->d_mixed, spec, addsrc, alpha);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

int mlx_legendre_backward(mlx_ctx* c, const double2* spec, cudaStream_t st, bool planes_ready) {
  if (c->precision == MLX_BF16X3) return mlx_legendre_tc_backward(c, spec, st, planes_ready);
  TimedLaunch tl(c, KID_LEG_BWD, st);
  if (c->precision == MLX_FP64)
    k_legendre<double, false><<<c->ntiles_bwd, NT, 0, st>>>(c->d_tiles_bwd, c->nc, c->nr, c->M, c->K,
                                                           c->d_boff, c->d_soff, c->d_P64,
                                                           (double*)c->d_mixed, (double2*)spec, nullptr, 0.0);
  else
    k_legendre<float, false><<<c->ntiles_bwd, NT, 0, st>>>(c->d_tiles_bwd, c->nc, c->nr, c->M, c->K,
                                                          c->d_boff, c->d_soff, c->d_P32,
                                                          (float*)c->d_mixed, (double2*)spec, nullptr, 0.0);
  MLX_LAUNCH_CHECK(c);
  return MLX_OK;
}

// Host: tile lists for both directions.
int mlx_legendre_tiles(mlx_ctx* c, std::vector<LegTile>& fwd, std::vector<LegTile>& bwd) {
  fwd.clear();
  bwd.clear();
  const int ncol = 2 * c->K;
  for (int m = 0; m < c->M; ++m) {
    const int Nm = c->nc - m;
    for (int r0 = 0; r0 < Nm; r0 += BM)
      for (int c0 = 0; c0 < ncol; c0 += BN) fwd.push_back(LegTile{m, r0, c0, 0});
    for (int r0 = 0; r0 < c->nr; r0 += BM)
      for (int c0 = 0; c0 < ncol; c0 += BN) bwd.push_back(LegTile{m, r0, c0, 0});
  }
  return MLX_OK;
}
