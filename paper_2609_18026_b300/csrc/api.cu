// C-ABI entry points of libmlx (declared in include/mlx.h).
#include "mlx_internal.cuh"

#include <stdlib.h>
#include <string.h>

int mlx_legendre_tiles(mlx_ctx* c, std::vector<LegTile>& fwd, std::vector<LegTile>& bwd);
int mlx_fft_prepare(mlx_ctx* c);
int mlx_band_prepare(mlx_ctx* c);

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
bool aligned16(const void* p) { return (((uintptr_t)p) & 15u) == 0; }

void free_ctx(mlx_ctx* c) {
  if (!c) return;
  mlx_invalidate_graphs(c);
  void* ptrs[] = {c->d_soff, c->d_boff, c->d_x, c->d_w, c->d_r, c->d_P64, c->d_W64, c->d_P32,
                  c->d_W32, c->d_lap, c->d_twphi64, c->d_twz64, c->d_twphi32, c->d_twz32,
                  c->d_tiles_fwd, c->d_tiles_bwd, c->d_mixed, c->d_zm, c->d_phys, c->d_specA,
                  c->d_spec1, c->d_spec2, c->d_spec3, c->d_band_off, c->d_Bplus,
                  c->lu_half.U, c->lu_half.L, c->lu_half.piv, c->lu_half.invd,
                  c->lu_full.U, c->lu_full.L, c->lu_full.piv, c->lu_full.invd,
                  c->d_Wb, c->d_Pb, c->d_arowW, c->d_arowP, c->d_tc_fwd, c->d_tc_bwd, c->d_err,
                  c->lu_lap.U, c->lu_lap.L, c->lu_lap.piv, c->lu_lap.invd,
                  c->lu_helm.U, c->lu_helm.L, c->lu_helm.piv, c->lu_helm.invd, c->d_lap_off,
                  c->d_rdr, c->d_jac, c->d_vspec, c->d_vphys,
                  c->lu_Q.U, c->lu_Q.L, c->lu_Q.piv, c->lu_Q.invd, c->lu_H.U, c->lu_H.L, c->lu_H.piv,
                  c->lu_H.invd, c->lu_G.U, c->lu_G.L, c->lu_G.piv, c->lu_G.invd, c->d_solve_y,
                  c->lu_half.FS, c->lu_half.BS, c->lu_full.FS, c->lu_full.BS, c->lu_lap.FS, c->lu_lap.BS,
                  c->lu_helm.FS, c->lu_helm.BS, c->lu_Q.FS, c->lu_Q.BS, c->lu_H.FS, c->lu_H.BS,
                  c->lu_G.FS, c->lu_G.BS, c->lu_half.PHf, c->lu_half.PHb, c->lu_half.PSf,
                  c->lu_full.PHf, c->lu_full.PHb, c->lu_full.PSf, c->lu_half.RNP, c->lu_full.RNP,
                  c->lu_half.RDF, c->lu_full.RDF, c->lu_half.PSDF, c->lu_full.PSDF, c->d_diag,
                  c->d_bsf, c->d_bsb, c->d_filt, c->d_lp, c->d_enst, c->d_bsv, c->d_rdr_df, c->d_lap_df};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (auto& p : c->timing.pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto& p : c->timing.captured) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : c->timing.pool) cudaEventDestroy(e);
  delete c;
}

template <typename P>
int dalloc(mlx_ctx* c, P** p, size_t bytes) {
  cudaError_t e = cudaMalloc((void**)p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    c->last_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MLX_ENOMEM : MLX_ECUDA;
  }
  return MLX_OK;
}

// Nonlinear term A(s) into A.  Fisher-KPP: A = P[gamma u (1 - u)] with u = B s
// (B backward, P forward transform), the product formed at the nodes (Sec. 3.3).
// In the time steps (src) the vortex tendency also carries the log proxies' constant
// forcing c L Lambda in its (0, 0) blocks.
int nonlinear_into(mlx_ctx* c, int kind, double c0, const double2* s, double2* A, cudaStream_t st,
                   bool src = true, bool planes_ready = false) {
  if (kind == MLX_NONLIN_NONE) {
    MLX_CUDA_TRY(c, cudaMemsetAsync(A, 0, sizeof(double2) * c->n_spec, st));
    return MLX_OK;
  }
  if (kind == MLX_NONLIN_VORTEX) {
    int rc = mlx_vortex_nonlinear(c, c0, s, A, st);
    if (rc || !src) return rc;
    return mlx_lp_add_source(c, A, st);
  }
  int rc = mlx_legendre_backward(c, s, st, planes_ready);
  if (rc) return rc;
  rc = mlx_fft_fkpp(c, c0, st);
  if (rc) return rc;
  return mlx_legendre_forward(c, A, st);
}

// One AB-CN step: A^j = A(s) into Anew, then (I - dt/2 L) out = (I + dt/2 L) s
// + dt/2 (3 A^j - A^{j-1}).

int nfields(int kind) { return kind == MLX_NONLIN_VORTEX ? 2 : 1; }

// implicit step applied to every field of the state (fields share the factors; the
// lean solve takes both fields of a vortex state in one launch, reading the factors once).
// sp / wrote: the split planes of a one-field output (see mlx_band_solve).
int solve_fields(mlx_ctx* c, int kind, int step, const double2* s, const double2* A, const double2* Ap,
                 double2* out, cudaStream_t st, const SplitPlanes* sp = nullptr, bool* wrote = nullptr) {
  if (wrote) *wrote = false;
  if (nfields(kind) == 2 && c->solve_direct == 2 && c->solve_fields2)
    return mlx_band_solve(c, step, s, A, Ap, out, st, 2);
  if (nfields(kind) == 1) return mlx_band_solve(c, step, s, A, Ap, out, st, 1, sp, wrote);
  for (int f = 0; f < nfields(kind); ++f) {
    const long long o = (long long)f * c->n_spec;
    int rc = mlx_band_solve(c, step, s + o, A ? A + o : nullptr, Ap ? Ap + o : nullptr, out + o, st);
    if (rc) return rc;
  }
  return MLX_OK;
}

// Split-plane reuse between the graph-replayed steps of one mlx_advance call: in the
// BF16X3 Fisher-KPP step (no filter) the segmented solve also writes the split
// planes of its output, the state the next step's backward contraction transforms,
// so that step skips k_split_spec.  Only the steps of one call chain this way (the
// caller may change the state between calls).
bool plane_reuse_ok(const mlx_ctx* c, int kind) {
  return c->plane_reuse && c->precision == MLX_BF16X3 && kind == MLX_NONLIN_FKPP && !c->filter_on && c->d_bsb;
}

// planes_in: d_bsb holds the split planes of s; planes_out (may be NULL): set when
// the solve wrote the split planes of out
int abcn_step(mlx_ctx* c, int kind, double c0, const double2* s, double2* Anew,
              const double2* Aprev, double2* out, cudaStream_t st, bool planes_in = false,
              bool* planes_out = nullptr) {
  if (planes_out) *planes_out = false;
  int rc = nonlinear_into(c, kind, c0, s, Anew, st, true, planes_in);
  if (rc) return rc;
  if (planes_out && plane_reuse_ok(c, kind)) {
    SplitPlanes sp;
    sp.bs = reinterpret_cast<unsigned short*>(c->d_bsb);
    sp.Kq = (int)c->tc_kq;
    sp.K2 = 2 * c->K;
    sp.part = (long long)c->M * sp.K2 * sp.Kq;
    rc = solve_fields(c, kind, MLX_STEP_ABCN, s, Anew, Aprev, out, st, &sp, planes_out);
  } else {
    rc = solve_fields(c, kind, MLX_STEP_ABCN, s, Anew, Aprev, out, st);
  }
  if (rc || !c->filter_on) return rc;
  return mlx_filter_fields(c, nfields(kind), out, st);   // the modal filter acts between steps
}

// the two AB-CN steps of one replayed pair; planes_in: d_bsb holds the split planes
// of s (the previous pair wrote them); *planes_out: the pair left those of its output s
int pair_steps(mlx_ctx* c, int kind, double c0, double2* s, double2* Ap, cudaStream_t st, bool planes_in,
               bool* planes_out) {
  bool mid = false;
  int rc = abcn_step(c, kind, c0, s, c->d_specA, Ap, c->d_spec1, st, planes_in, &mid);
  if (rc) return rc;
  return abcn_step(c, kind, c0, c->d_spec1, Ap, c->d_specA, s, st, mid, planes_out);
}

}  // namespace

// Two AB-CN steps (s, A_prev) -> (s, A_prev) through the context's temporaries,
// enqueued on st (the unit that graphs replay).
int mlx_enqueue_step_pair(mlx_ctx* c, int kind, double c0, double2* s, double2* Ap, cudaStream_t st) {
  // each pair starts from the caller's state (split afresh); its second step takes
  // the split planes its first step's solve left
  bool left = false;
  return pair_steps(c, kind, c0, s, Ap, st, false, &left);
}

extern "C" {

const char* mlx_strerror(int code) {
  switch (code) {
    case MLX_OK: return "ok";
    case MLX_EINVAL: return "invalid argument";
    case MLX_ECUDA: return "CUDA error";
    case MLX_ENUMERIC: return "non-finite value detected";
    case MLX_ETIMEOUT: return "bounded device wait expired";
    case MLX_ESTATE: return "call out of order";
    case MLX_ENOMEM: return "device allocation failed";
    default: return "unknown error";
  }
}

const char* mlx_last_cuda_error(const mlx_ctx* ctx) { return ctx ? ctx->last_err.c_str() : ""; }

int mlx_create(const mlx_params* p, mlx_stream stream, mlx_ctx** out) {
  if (!out) return MLX_EINVAL;
  *out = nullptr;
  if (!p) return MLX_EINVAL;
  if (p->nr < 2 || p->nr > 1024) return MLX_EINVAL;
  if (!is_pow2(p->nphi) || p->nphi < 4 || p->nphi > 512) return MLX_EINVAL;
  if (!(p->nz == 1 || (is_pow2(p->nz) && p->nz <= 512))) return MLX_EINVAL;
  if (!(p->ell > 0.0) || !(p->lz > 0.0)) return MLX_EINVAL;
  if (p->precision != MLX_FP64 && p->precision != MLX_FP32 && p->precision != MLX_BF16X3) return MLX_EINVAL;
  if (p->chop_policy != MLX_CHOP_LINEAR && p->chop_policy != MLX_CHOP_TWOTHIRDS &&
      p->chop_policy != MLX_CHOP_NYQUIST) return MLX_EINVAL;
  if (p->nr_c < 0 || p->nphi_c < 0 || p->nz_c < 0) return MLX_EINVAL;
  int nc = p->nr_c ? p->nr_c : p->nr;
  int M, Kz;
  if (p->chop_policy == MLX_CHOP_LINEAR) {
    M = p->nphi / 2;
    Kz = p->nz > 1 ? p->nz / 2 : 1;
  } else if (p->chop_policy == MLX_CHOP_NYQUIST) {
    M = p->nphi / 2 + 1;
    Kz = p->nz > 1 ? p->nz / 2 + 1 : 1;
  } else {
    M = (p->nphi - 1) / 3 + 1;
    Kz = (p->nz - 1) / 3 + 1;
  }
  if (p->nphi_c) M = p->nphi_c;
  if (p->nz_c) Kz = p->nz_c;
  if (nc > p->nr || M > p->nphi / 2 + 1 || M > nc || M < 1) return MLX_EINVAL;
  if (Kz < 1 || (p->nz == 1 && Kz != 1) || (p->nz > 1 && Kz > p->nz / 2 + 1)) return MLX_EINVAL;

  mlx_ctx* c = new mlx_ctx();
  c->nr = p->nr; c->nphi = p->nphi; c->nz = p->nz;
  c->nc = nc; c->M = M; c->Kz = Kz; c->K = 2 * Kz - 1;
  c->precision = p->precision;
  c->ell = p->ell; c->lz = p->lz;
  c->n_phys = (long long)c->nz * c->nphi * c->nr;
  c->soff.assign(M + 1, 0);
  c->boff.assign(M + 1, 0);
  c->band_off.assign(M + 1, 0);
  long long tri = 0;
  for (int m = 0; m < M; ++m) {
    c->soff[m] = (long long)c->K * tri;
    c->boff[m] = tri * c->nr;
    c->band_off[m] = (long long)Kz * tri;
    tri += nc - m;
  }
  c->soff[M] = (long long)c->K * tri;
  c->boff[M] = tri * c->nr;
  c->band_off[M] = (long long)Kz * tri;
  c->tri = tri;
  c->n_spec = (long long)c->K * tri;
  c->band_rows = (long long)Kz * tri;

  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = elem_size(c->precision);
  int rc = MLX_OK;
#define ALLOC(ptr, bytes) do { rc = dalloc(c, &(ptr), (bytes)); if (rc) { free_ctx(c); return rc; } } while (0)
  ALLOC(c->d_soff, sizeof(long long) * (M + 1));
  ALLOC(c->d_boff, sizeof(long long) * (M + 1));
  ALLOC(c->d_band_off, sizeof(long long) * (M + 1));
  ALLOC(c->d_x, sizeof(double) * c->nr);
  ALLOC(c->d_w, sizeof(double) * c->nr);
  ALLOC(c->d_r, sizeof(double) * c->nr);
  ALLOC(c->d_P64, sizeof(double) * tri * c->nr);
  ALLOC(c->d_W64, sizeof(double) * tri * c->nr);
  ALLOC(c->d_P32, sizeof(float) * tri * c->nr);
  ALLOC(c->d_W32, sizeof(float) * tri * c->nr);
  ALLOC(c->d_lap, sizeof(double) * tri * 5);
  ALLOC(c->d_twphi64, sizeof(double2) * (c->nphi / 2));
  ALLOC(c->d_twphi32, sizeof(float2) * (c->nphi / 2));
  ALLOC(c->d_twz64, sizeof(double2) * (c->nz / 2 + 1));
  ALLOC(c->d_twz32, sizeof(float2) * (c->nz / 2 + 1));
  ALLOC(c->d_mixed, es * 2 * c->K * c->M * c->nr);
  if (c->nz > 1) ALLOC(c->d_zm, es * 2 * c->nz * c->M * c->nr);
  ALLOC(c->d_phys, es * c->n_phys);
  ALLOC(c->d_specA, sizeof(double2) * c->n_spec);
  ALLOC(c->d_spec1, sizeof(double2) * c->n_spec);
  ALLOC(c->d_spec2, sizeof(double2) * c->n_spec);
  ALLOC(c->d_spec3, sizeof(double2) * c->n_spec);
  std::vector<LegTile> tf, tb;
  mlx_legendre_tiles(c, tf, tb);
  c->ntiles_fwd = (int)tf.size();
  c->ntiles_bwd = (int)tb.size();
  ALLOC(c->d_tiles_fwd, sizeof(LegTile) * tf.size());
  ALLOC(c->d_tiles_bwd, sizeof(LegTile) * tb.size());
  ALLOC(c->d_err, sizeof(int));
#undef ALLOC
#define TRY(call) do { cudaError_t _e = (call); if (_e != cudaSuccess) { c->last_err = cudaGetErrorString(_e); free_ctx(c); return MLX_ECUDA; } } while (0)
  TRY(cudaMemcpyAsync(c->d_soff, c->soff.data(), sizeof(long long) * (M + 1), cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(c->d_boff, c->boff.data(), sizeof(long long) * (M + 1), cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(c->d_band_off, c->band_off.data(), sizeof(long long) * (M + 1), cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(c->d_tiles_fwd, tf.data(), sizeof(LegTile) * tf.size(), cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(c->d_tiles_bwd, tb.data(), sizeof(LegTile) * tb.size(), cudaMemcpyHostToDevice, st));
  TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
  TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
#undef TRY
  rc = mlx_fft_prepare(c);
  if (!rc) rc = mlx_band_prepare(c);
  if (!rc) rc = mlx_basis_build(c, st);
  if (!rc && c->precision == MLX_BF16X3) rc = mlx_tc_prepare(c, st);
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { c->last_err = cudaGetErrorString(e); rc = MLX_ECUDA; }
  }
  if (rc) { free_ctx(c); return rc; }
  *out = c;
  return MLX_OK;
}

int mlx_destroy(mlx_ctx* ctx) {
  if (!ctx) return MLX_EINVAL;
  free_ctx(ctx);
  return MLX_OK;
}

int mlx_query(const mlx_ctx* c, mlx_info* info) {
  if (!c || !info) return MLX_EINVAL;
  info->nr = c->nr; info->nphi = c->nphi; info->nz = c->nz;
  info->nc = c->nc; info->M = c->M; info->Kz = c->Kz; info->K = c->K;
  info->n_phys = c->n_phys; info->n_spec = c->n_spec;
  info->precision = c->precision;
  info->ell = c->ell; info->lz = c->lz;
  return MLX_OK;
}

int mlx_get_nodes(const mlx_ctx* cc, double* x, double* w, double* r) {
  mlx_ctx* c = const_cast<mlx_ctx*>(cc);
  if (!c) return MLX_EINVAL;
  if (x) MLX_CUDA_TRY(c, cudaMemcpy(x, c->d_x, sizeof(double) * c->nr, cudaMemcpyDeviceToHost));
  if (w) MLX_CUDA_TRY(c, cudaMemcpy(w, c->d_w, sizeof(double) * c->nr, cudaMemcpyDeviceToHost));
  if (r) MLX_CUDA_TRY(c, cudaMemcpy(r, c->d_r, sizeof(double) * c->nr, cudaMemcpyDeviceToHost));
  return MLX_OK;
}

int mlx_forward(mlx_ctx* c, const void* phys, void* spec, mlx_stream stream) {
  if (!c || !phys || !spec || !aligned16(phys) || !aligned16(spec)) return MLX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlx_fft_forward(c, phys, st);
  if (rc) return rc;
  return mlx_legendre_forward(c, (double2*)spec, st);
}

int mlx_backward(mlx_ctx* c, const void* spec, void* phys, mlx_stream stream) {
  if (!c || !phys || !spec || !aligned16(phys) || !aligned16(spec)) return MLX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlx_legendre_backward(c, (const double2*)spec, st);
  if (rc) return rc;
  return mlx_fft_backward(c, phys, st);
}

int mlx_nonlinear(mlx_ctx* c, int kind, const double* coeffs, int ncoeffs, const void* spec_in,
                  void* spec_out, mlx_stream stream) {
  if (!c || !spec_in || !spec_out || spec_in == spec_out) return MLX_EINVAL;
  if (!aligned16(spec_in) || !aligned16(spec_out)) return MLX_EINVAL;
  if ((kind == MLX_NONLIN_FKPP || kind == MLX_NONLIN_VORTEX) && (!coeffs || ncoeffs < 1)) return MLX_EINVAL;
  if (kind != MLX_NONLIN_FKPP && kind != MLX_NONLIN_NONE && kind != MLX_NONLIN_VORTEX) return MLX_EINVAL;
  if (kind == MLX_NONLIN_VORTEX && !c->vortex_ready) return MLX_ESTATE;
  return nonlinear_into(c, kind, coeffs ? coeffs[0] : 0.0, (const double2*)spec_in,
                        (double2*)spec_out, (cudaStream_t)stream, false);
}

int mlx_implicit_setup(mlx_ctx* c, double nu, double nu_h, int p, double dt, mlx_stream stream) {
  if (!c || !(dt > 0.0) || nu < 0.0 || nu_h < 0.0) return MLX_EINVAL;
  if (nu_h > 0.0 && p != 4 && p != 6 && p != 8) return MLX_EINVAL;
  mlx_invalidate_graphs(c);
  c->nu = nu; c->nu_h = nu_h; c->p = p; c->dt = dt;
  c->kl = (nu_h > 0.0) ? p : 2;
  // wide hyperviscous bands: the lean solve (32 chains per warp, packed records)
  c->solve_direct = 0;
  if (c->kl >= 4) {
    const int rc = mlx_solve_scratch(c);
    if (rc) return rc;
    c->solve_direct = 2;
  }
  c->implicit_ready = false;
  int rc = mlx_band_setup(c, (cudaStream_t)stream);
  if (rc) return rc;
  c->implicit_ready = true;
  // the log proxies' forcing c L Lambda depends on the operator
  if (c->d_lp && (rc = mlx_lp_refresh(c, (cudaStream_t)stream))) return rc;
  return MLX_OK;
}

int mlx_implicit_solve(mlx_ctx* c, int step, const void* s, const void* A, const void* A_prev,
                       void* out, mlx_stream stream) {
  if (!c || !s || !out) return MLX_EINVAL;
  if (!c->implicit_ready) return MLX_ESTATE;
  if (step != MLX_STEP_FEBE_HALF && step != MLX_STEP_FEBE_FULL && step != MLX_STEP_ABCN) return MLX_EINVAL;
  if (out == s || out == A || out == A_prev) return MLX_EINVAL;
  return mlx_band_solve(c, step, (const double2*)s, (const double2*)A, (const double2*)A_prev,
                        (double2*)out, (cudaStream_t)stream);
}

int mlx_advance(mlx_ctx* c, int kind, const double* coeffs, int ncoeffs, void* state, void* prev_A,
                int nsteps, int start, mlx_stream stream) {
  if (!c || !state || !prev_A || nsteps < 0 || state == prev_A) return MLX_EINVAL;
  if (!aligned16(state) || !aligned16(prev_A)) return MLX_EINVAL;
  if (kind != MLX_NONLIN_NONE && kind != MLX_NONLIN_FKPP && kind != MLX_NONLIN_VORTEX) return MLX_EINVAL;
  if ((kind == MLX_NONLIN_FKPP || kind == MLX_NONLIN_VORTEX) && (!coeffs || ncoeffs < 1)) return MLX_EINVAL;
  if (!c->implicit_ready) return MLX_ESTATE;
  if (kind == MLX_NONLIN_VORTEX && !c->vortex_ready) return MLX_ESTATE;
  const long long nst = (long long)nfields(kind) * c->n_spec;
  if (nsteps == 0) return MLX_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const double c0 = coeffs ? coeffs[0] : 0.0;
  double2* s = (double2*)state;
  double2* Ap = (double2*)prev_A;
  int rc;
  if (start) {
    // Richardson start: s1 = 2 FEBE_{dt/2}(FEBE_{dt/2}(s0)) - FEBE_dt(s0); A^0 kept.
    if ((rc = nonlinear_into(c, kind, c0, s, Ap, st))) return rc;
    if ((rc = solve_fields(c, kind, MLX_STEP_FEBE_HALF, s, Ap, nullptr, c->d_spec1, st))) return rc;
    if ((rc = nonlinear_into(c, kind, c0, c->d_spec1, c->d_specA, st))) return rc;
    if ((rc = solve_fields(c, kind, MLX_STEP_FEBE_HALF, c->d_spec1, c->d_specA, nullptr, c->d_spec2, st))) return rc;
    if ((rc = solve_fields(c, kind, MLX_STEP_FEBE_FULL, s, Ap, nullptr, c->d_spec3, st))) return rc;
    if ((rc = mlx_spec_axpby(c, 2.0, c->d_spec2, -1.0, c->d_spec3, s, st, nst))) return rc;
    if (c->filter_on && (rc = mlx_filter_fields(c, nfields(kind), s, st))) return rc;
    --nsteps;
  }
  const int pairs = nsteps / 2;
  // capture one pair (planes_in: reuse the split planes the previous pair left) into
  // an executable graph; *left: the pair leaves the split planes of its output s
  // (npairs > 1: that many pairs in one graph, each taking the planes the one
  // before it left)
  auto capture_pair = [&](bool planes_in, cudaGraphExec_t* exec, bool* left, int npairs = 1) -> int {
    cudaGraph_t g = nullptr;
    MLX_CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int r = MLX_OK;
    bool in = planes_in;
    for (int q = 0; q < npairs && !r; ++q) {
      r = pair_steps(c, kind, c0, s, Ap, c->cap_stream, in, left);
      in = *left;
    }
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (r) { if (g) cudaGraphDestroy(g); return r; }
    if (e != cudaSuccess) { c->last_err = cudaGetErrorString(e); return MLX_ECUDA; }
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { c->last_err = cudaGetErrorString(e); return MLX_ECUDA; }
    return MLX_OK;
  };
  if (pairs > 0 && c->timing.on && c->timing.mode == 1) {
    // instrumented mode 1: the same two-step sequence launched directly so that
    // every kernel is bracketed by CUDA events
    bool planes = false;
    for (int i = 0; i < pairs; ++i)
      if ((rc = pair_steps(c, kind, c0, s, Ap, st, planes, &planes))) return rc;
  } else if (pairs > 0 && c->timing.on) {
    // instrumented mode 2: the two-step graphs (the call's first pair, then the pair
    // that reuses the previous pair's split planes) with an event-record node before
    // and after every kernel node, replayed pair by pair; after each replay the node
    // timings of that graph are read (the replays are separated by a host
    // synchronisation, the kernels inside one replay run back to back as in the
    // cached graphs)
    auto release = [&](std::vector<TimingState::Pending>& v) {
      for (auto& p : v) { c->timing.pool.push_back(p.a); c->timing.pool.push_back(p.b); }
      v.clear();
    };
    release(c->timing.captured);
    cudaGraphExec_t ex[2] = {nullptr, nullptr};
    std::vector<TimingState::Pending> cap[2];
    bool left = false, left2 = false;
    rc = capture_pair(false, &ex[0], &left);
    cap[0].swap(c->timing.captured);
    if (!rc && left && pairs > 1) {
      rc = capture_pair(true, &ex[1], &left2);
      cap[1].swap(c->timing.captured);
    }
    for (int i = 0; i < pairs && !rc; ++i) {
      const int v = (i > 0 && ex[1]) ? 1 : 0;
      cudaError_t e = cudaGraphLaunch(ex[v], st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      for (auto& p : cap[v]) {
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
        c->timing.launches[p.kid] += 1;
        c->timing.ms[p.kid] += ms;
      }
      if (e != cudaSuccess) { c->last_err = cudaGetErrorString(e); rc = MLX_ECUDA; }
    }
    for (auto* x : ex) if (x) cudaGraphExecDestroy(x);
    release(cap[0]);
    release(cap[1]);
    release(c->timing.captured);
    if (rc) return rc;
  } else if (pairs > 0) {
    // two steps per graph: (s, A_prev) -> (spec1, specA) -> (s, A_prev), no copies;
    // variant 0 starts from the caller's state, variant 1 (the later pairs of the
    // call) reuses the split planes the previous pair left, variant 2 is kChunk
    // later pairs in one graph (fewer graph launches, each pair as in variant 1,
    // or as in variant 0 when the steps leave no planes)
    constexpr int kChunk = 8;
    cudaGraphExec_t ex[3] = {nullptr, nullptr, nullptr};
    bool left = false;
    for (int v = 0; v < 3; ++v) {
      if (v == 1 && !(left && pairs > 1)) continue;
      if (v == 2 && pairs - 1 < kChunk) break;
      mlx_ctx::GraphKey key{state, prev_A, kind, c0, v};
      auto it = c->graphs.find(key);
      if (it == c->graphs.end()) {
        bool l = false;
        if ((rc = capture_pair(v >= 1 && left, &ex[v], &l, v == 2 ? kChunk : 1))) return rc;
        c->graphs[key] = ex[v];
        c->graph_left[key] = l;
        if (v == 0) left = l;
      } else {
        ex[v] = it->second;
        if (v == 0) left = c->graph_left[key];
      }
    }
    int i = 0;
    MLX_CUDA_TRY(c, cudaGraphLaunch(ex[0], st));
    for (i = 1; ex[2] && i + kChunk <= pairs; i += kChunk) MLX_CUDA_TRY(c, cudaGraphLaunch(ex[2], st));
    for (; i < pairs; ++i) MLX_CUDA_TRY(c, cudaGraphLaunch(ex[1] ? ex[1] : ex[0], st));
  }
  if (nsteps % 2) {
    if ((rc = abcn_step(c, kind, c0, s, c->d_specA, Ap, c->d_spec1, st))) return rc;
    MLX_CUDA_TRY(c, cudaMemcpyAsync(s, c->d_spec1, sizeof(double2) * nst, cudaMemcpyDeviceToDevice, st));
    MLX_CUDA_TRY(c, cudaMemcpyAsync(Ap, c->d_specA, sizeof(double2) * nst, cudaMemcpyDeviceToDevice, st));
  }
  return MLX_OK;
}

int mlx_vortex_setup(mlx_ctx* c, mlx_stream stream) {
  if (!c) return MLX_EINVAL;
  return mlx_vortex_prepare(c, (cudaStream_t)stream);
}

int mlx_lap_h_solve(mlx_ctx* c, const void* rhs, void* out, mlx_stream stream) {
  if (!c || !rhs || !out || rhs == out) return MLX_EINVAL;
  if (!aligned16(rhs) || !aligned16(out)) return MLX_EINVAL;
  if (!c->lap_ready) return MLX_ESTATE;
  return mlx_lap_solve(c, 0, (const double2*)rhs, (double2*)out, (cudaStream_t)stream);
}

int mlx_set_tuning(mlx_ctx* c, const char* key, int value) {
  if (!c || !key) return MLX_EINVAL;
  if (strcmp(key, "solve_cpw") == 0) {
    if (value != 4 && value != 8 && value != 16 && value != 32) return MLX_EINVAL;
    c->solve_cpw = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "solve_keep_s") == 0) {
    if (value != 0 && value != 1) return MLX_EINVAL;
    c->solve_keep_s = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "phi_tile") == 0 || strcmp(key, "z_tile") == 0) {
    if (value != 0 && value != 2 && value != 4 && value != 8 && value != 16 && value != 32) return MLX_EINVAL;
    (key[0] == 'p' ? c->phi_tile : c->z_tile) = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "solve_seg") == 0) {
    if (value != 0 && value != 4 && value != 8) return MLX_EINVAL;
    c->solve_seg = value;
    if (c->implicit_ready) {
      for (BandLU* f : {&c->lu_half, &c->lu_full}) {
        const int rc = mlx_seg_build(c, *f, value, nullptr);
        if (rc) return rc;
      }
      MLX_CUDA_TRY(c, cudaStreamSynchronize(nullptr));
    }
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "solve_df") == 0) {
    if (value != 0 && value != 1) return MLX_EINVAL;
    c->solve_df = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "solve_lean_cpw") == 0) {
    if (value != 16 && value != 32) return MLX_EINVAL;
    c->solve_lean_cpw = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "vortex_planes") == 0) {
    if (value != 0 && value != 1) return MLX_EINVAL;
    c->vortex_planes = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "plane_reuse") == 0) {
    if (value != 0 && value != 1) return MLX_EINVAL;
    c->plane_reuse = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "solve_fields2") == 0) {
    if (value != 0 && value != 1) return MLX_EINVAL;
    c->solve_fields2 = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "solve_direct") == 0) {
    if (value != 0 && value != 2) return MLX_EINVAL;
    if (value == 2) {
      const int rc = mlx_solve_scratch(c);
      if (rc) return rc;
    }
    c->solve_direct = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "tc_expire") == 0) {
    if (value != 0 && value != 1) return MLX_EINVAL;
    c->tc_expire = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "tc_products") == 0) {
    if (value != 6 && value != 8) return MLX_EINVAL;
    c->tc_products = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "tc_bn") == 0) {
    if (c->precision != MLX_BF16X3) return MLX_EINVAL;
    int rc = mlx_tc_retile(c, value, nullptr);
    if (rc) return rc;
    MLX_CUDA_TRY(c, cudaDeviceSynchronize());
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  if (strcmp(key, "solve_wpb") == 0) {
    if (value != 1 && value != 2 && value != 4) return MLX_EINVAL;
    c->solve_wpb = value;
    mlx_invalidate_graphs(c);
    return MLX_OK;
  }
  return MLX_EINVAL;
}

static const char* kKernelNames[KID_COUNT] = {
    "phi_analysis", "phi_synthesis", "phi_fkpp_fused", "z_forward", "z_inverse",
    "legendre_forward", "legendre_backward", "band_solve", "spec_axpby", "legendre_split"};

int mlx_kernel_count(void) { return KID_COUNT; }

int mlx_device_status(mlx_ctx* c) {
  if (!c) return MLX_EINVAL;
  int v = 0;
  MLX_CUDA_TRY(c, cudaMemcpy(&v, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) {
    MLX_CUDA_TRY(c, cudaMemset(c->d_err, 0, sizeof(int)));
    return (v & 7) ? MLX_ETIMEOUT : MLX_ENUMERIC;
  }
  return MLX_OK;
}

const char* mlx_kernel_name(int kernel) {
  return (kernel >= 0 && kernel < KID_COUNT) ? kKernelNames[kernel] : "";
}

int mlx_timing(mlx_ctx* c, int enable) {
  if (!c) return MLX_EINVAL;
  for (auto& p : c->timing.pending) { c->timing.pool.push_back(p.a); c->timing.pool.push_back(p.b); }
  c->timing.pending.clear();
  for (int k = 0; k < KID_COUNT; ++k) { c->timing.launches[k] = 0; c->timing.ms[k] = 0.0; }
  if (enable < 0 || enable > 2) return MLX_EINVAL;
  c->timing.on = enable != 0;
  c->timing.mode = enable;
  return MLX_OK;
}

int mlx_timing_read(mlx_ctx* c, int kernel, long long* launches, double* total_ms) {
  if (!c || kernel < 0 || kernel >= KID_COUNT) return MLX_EINVAL;
  for (auto& p : c->timing.pending) {
    MLX_CUDA_TRY(c, cudaEventSynchronize(p.b));
    float ms = 0.f;
    MLX_CUDA_TRY(c, cudaEventElapsedTime(&ms, p.a, p.b));
    c->timing.launches[p.kid] += 1;
    c->timing.ms[p.kid] += ms;
    c->timing.pool.push_back(p.a);
    c->timing.pool.push_back(p.b);
  }
  c->timing.pending.clear();
  if (launches) *launches = c->timing.launches[kernel];
  if (total_ms) *total_ms = c->timing.ms[kernel];
  return MLX_OK;
}

}  // extern "C"
