/*
 * mlx.h -- C-ABI of the B300 (sm_103a) mapped Legendre / Fourier spectral hot path.
 *
 * The method (Lee & Wang, "MLegS: a modern mapped Legendre spectral method solver
 * for unbounded domains"):
 *   - algebraic map r = ell sqrt((1+x)/(1-x)) onto Gauss-Legendre nodes x_i   (Eq. (1))
 *   - truncated expansion in normalised associated Legendre functions times
 *     Fourier modes in phi and z, triangular n >= m, only m >= 0 stored       (Eq. (2), Eq. (7))
 *   - pentadiagonal horizontal Laplacian D_m, full Laplacian D_m - kappa^2 I   (Eqs. (4)-(5))
 *   - split form ds/dt = A(s) + L s, L = nu lap - nu_h (-lap)^{p/2}           (Eqs. (10)-(11))
 *   - FE-BE and AB-CN with a Richardson start from FE-BE substeps              (Eq. (12), Sec. 3.3)
 *   - Fisher-KPP reaction gamma u (1 - u)                                      (Eq. (17))
 *
 * Conventions shared by every entry point
 *   - Every function returns int: MLX_OK (0) or a negative MLX_E* code; no C++
 *     exception crosses this boundary.  mlx_strerror() names a code.
 *   - The library owns its context (basis tables, operator factors, workspace,
 *     CUDA graphs).  The caller owns every field buffer: device pointers that it
 *     allocated, 16-byte aligned, passed with the CUDA stream to run on.
 *     Nothing is freed or retained by the library after a call returns, except
 *     cached CUDA graphs keyed on the caller's pointers (released by mlx_destroy).
 *   - Physical fields: real, layout [Nz][Nphi][Nr] (r fastest), node (i, j, l) at
 *     r_i, phi_j = 2 pi j / Nphi, z_l = Lz l / Nz.  Element type double for
 *     MLX_FP64 and float for MLX_FP32 / MLX_BF16X3.
 *   - Spectral fields: complex128 (interleaved re, im doubles) in the flat ragged
 *     layout  index(m, k, n) = K * sum_{m' < m} (Nc - m') + k * (Nc - m) + (n - m),
 *     m = 0..M-1, k = 0..K-1 in FFT order (wavenumber k for k < Kz, k - K above),
 *     n = m..Nc-1.  K = 2 Kz - 1.  Basis functions carry no Condon-Shortley phase.
 *     The m = 0 block of a real field is Hermitian in k.
 *   - Calls on one context are not thread-safe; use one context per host thread.
 *   - Errors: MLX_EINVAL for bad sizes, chops, ell <= 0, Lz <= 0, NULL or
 *     misaligned pointers; MLX_ECUDA for a failed CUDA call (the message is kept
 *     per context, see mlx_last_cuda_error); MLX_ESTATE for a call out of order
 *     (solve before setup); MLX_ENOMEM when device allocation fails.
 */
#ifndef MLX_H
#define MLX_H

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;                       /* cudaStream_t without the CUDA headers */
typedef struct CUstream_st* mlx_stream;   /* NULL = the legacy default stream      */

typedef struct mlx_ctx mlx_ctx;

enum {
  MLX_OK = 0,
  MLX_EINVAL = -1,
  MLX_ECUDA = -2,
  MLX_ENUMERIC = -3,
  MLX_ETIMEOUT = -4,
  MLX_ESTATE = -5,
  MLX_ENOMEM = -6
};

/* Arithmetic of the transforms.  The implicit solve and the spectral state are
 * always FP64; basis values, nodes and weights are generated in FP64.
 *   MLX_FP64   : FFTs and Legendre contraction in FP64 (parity form).
 *   MLX_FP32   : FFTs and contraction in FP32 on the CUDA cores.
 *   MLX_BF16X3 : FFTs in FP32; contraction on the tensor cores with every operand
 *                split into three BF16 parts (six products, FP32 accumulation). */
enum { MLX_FP64 = 0, MLX_FP32 = 1, MLX_BF16X3 = 2 };

/* Chop policy used when the corresponding chop in mlx_params is 0.
 * LINEAR: M = Nphi/2, Kz = max(1, Nz/2) (Nyquist dropped).
 * TWOTHIRDS: M = (Nphi-1)/3 + 1, Kz = (Nz-1)/3 + 1 -- the two-thirds mask of
 * Sec. 3.3 realised as storage truncation.
 * NYQUIST: M = Nphi/2 + 1, Kz = Nz/2 + 1 (1 if Nz = 1): |m| <= Nphi/2 and
 * |k| <= Nz/2, the layout of the 256^3 production run of Sec. 4.2 (|m| <= 128,
 * |k| <= 128).  The members of each Nyquist pair (m = +-Nphi/2; the stored rows
 * k = +Nz/2 and k = -Nz/2) multiply the same grid function, so the forward
 * transform gives each half of the grid's bin and the backward transform sums
 * them.  The m = Nphi/2 block is Hermitian in k after a forward transform.
 * Nc = Nr unless nr_c is given. */
enum { MLX_CHOP_LINEAR = 0, MLX_CHOP_TWOTHIRDS = 1, MLX_CHOP_NYQUIST = 2 };

/* Nonlinear term kinds for mlx_nonlinear / mlx_advance.
 *   MLX_NONLIN_FKPP:   one scalar, A = gamma u (1 - u) (Eq. (17)); coeffs[0] = gamma.
 *   MLX_NONLIN_VORTEX: the toroidal-poloidal pair (psi, chi) of Eq. (8), stored as
 *                      two consecutive spectral fields (2 n_spec complex128),
 *                      A = P[(U + v) x omega] (Eq. (19)) with the uniform
 *                      background U = coeffs[0] e_y (moving frame, Sec. 5.3).
 *                      Needs mlx_vortex_setup. */
enum { MLX_NONLIN_NONE = 0, MLX_NONLIN_FKPP = 1, MLX_NONLIN_VORTEX = 2 };

/* Implicit step kinds for mlx_implicit_solve. */
enum { MLX_STEP_FEBE_HALF = 0, MLX_STEP_FEBE_FULL = 1, MLX_STEP_ABCN = 2 };

typedef struct {
  int nr, nphi, nz;          /* collocation counts: 2 <= Nr <= 1024; Nphi a power of
                                two in [4, 512]; Nz 1 or a power of two <= 512       */
  int nr_c, nphi_c, nz_c;    /* chops Nc, M, Kz (0 = from chop_policy); bounds of
                                Sec. 3.1: Nc <= Nr, M <= Nphi/2 + 1, Kz <= Nz/2 + 1
                                (1 if Nz=1), and M <= Nc                              */
  double ell;                /* map scale ell > 0, Eq. (1)                            */
  double lz;                 /* axial period Lz > 0 (kappa_k = 2 pi k / Lz)           */
  int precision;             /* MLX_FP64 | MLX_FP32 | MLX_BF16X3                      */
  int chop_policy;           /* MLX_CHOP_LINEAR | MLX_CHOP_TWOTHIRDS | MLX_CHOP_NYQUIST */
} mlx_params;

typedef struct {
  int nr, nphi, nz;
  int nc, M, Kz, K;          /* chops in effect and K = 2 Kz - 1                      */
  long long n_phys;          /* Nz * Nphi * Nr real values                            */
  long long n_spec;          /* K * sum_m (Nc - m) complex values                     */
  int precision;
  double ell, lz;
} mlx_info;

const char* mlx_strerror(int code);

/* Text of the last CUDA error seen by this context ("" if none). */
const char* mlx_last_cuda_error(const mlx_ctx* ctx);

/* Build a context: Gauss-Legendre nodes and weights by Newton iteration in FP64
 * on the GPU, the mapped radii (Eq. (1)), the normalised associated Legendre
 * tables Pbar_n^m(x_i) by the normalised three-term recurrence (Eq. (7), no
 * factorial is formed), the quadrature table w_i Pbar_n^m(x_i), the pentadiagonal
 * Laplacian bands (Eq. (5), rescaled to the orthonormal basis), Fourier twiddles,
 * and the workspace.  Runs on `stream` and synchronises it before returning.
 * On error *out is set to NULL and nothing stays allocated. */
int mlx_create(const mlx_params* params, mlx_stream stream, mlx_ctx** out);
int mlx_destroy(mlx_ctx* ctx);
int mlx_query(const mlx_ctx* ctx, mlx_info* info);

/* Copy the FP64 nodes x_i (ascending), weights w_i and radii r_i, each Nr
 * doubles, to host buffers (any may be NULL).  Synchronous. */
int mlx_get_nodes(const mlx_ctx* ctx, double* x, double* w, double* r);

/* Forward transform (physical -> spectral), Eq. (2) inverted by the phi and z
 * DFTs (scaled 1/Nphi, 1/Nz) and the Gauss quadrature
 * shat_nmk = sum_i w_i Pbar_n^m(x_i) f_mk(r_i).  Modes beyond the chops are
 * dropped.  phys: device, n_phys reals (double or float, see above); spec:
 * device, n_spec complex128.  Asynchronous on `stream`. */
int mlx_forward(mlx_ctx* ctx, const void* phys, void* spec, mlx_stream stream);

/* Allocation-free forward transform.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc when they transform (code
 * running inside another framework's CUDA-graph capture, or hosts that freeze
 * their device-memory budget after start-up).  Same arguments, layouts and result
 * as mlx_forward, but the intermediate Fourier planes live in a fixed 16 MiB
 * device array built into the library (present on every GPU that loads it, until
 * exit) instead of the context's workspace; no device memory is allocated or
 * freed.  Grids whose intermediates exceed 16 MiB
 * (element size x 2 x (K M Nr + Nz M Nr when Nz > 1)) are rejected with
 * MLX_EINVAL and a message in mlx_last_cuda_error, and so are device ordinals of
 * 64 and above.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, once per device under a lock;
 * make it before any stream capture.  That address, like every context, does not
 * survive cudaDeviceReset.  All calls on a device share the array: calls whose
 * GPU work overlaps (other streams, other contexts) race, so serialise them. */
int mlx_forward_noalloc(mlx_ctx* ctx, const void* phys, void* spec, mlx_stream stream);

/* Backward transform (spectral -> physical): Eq. (2) summed at the nodes,
 * s = Re sum_k f_0k e^{i kappa z} + 2 Re sum_{m>=1,k} f_mk e^{i(m phi + kappa z)}. */
int mlx_backward(mlx_ctx* ctx, const void* spec, void* phys, mlx_stream stream);

/* Nonlinear term A(s) of Eq. (10) in spectral space (transforms with the
 * pointwise products between them, Sec. 3.3):
 *   MLX_NONLIN_FKPP: A = gamma u (1 - u), Eq. (17); coeffs[0] = gamma.
 *   MLX_NONLIN_VORTEX: (psi_N, chi_N) = P[(U + v) x omega], Eq. (19), evaluated
 *     harmonic by harmonic in coefficient space (no division by r at the nodes):
 *     the r-weighted velocity and vorticity r v_r, r v_phi, v_z, r w_r, r w_phi,
 *     w_z from (psi, chi) with the banded r d/dr (R) and D_m (six backward
 *     transforms), at the nodes A = r N_phi, B = r N_r, C = r^2 N_z of
 *     N = (v + U) x omega (three forward transforms), X1 = R A - i m B
 *     (= r^2 (curl N)_z), X2 = R B + i m A (= r^2 div_h N), then with
 *     J = multiplication by x and Q = (I - J^2) diag(-n(n+1)) = r^2 lap_h:
 *     Q psi_N = -X1; for k != 0 [(I - J) Q - kappa^2 ell^2 (I + J)] g =
 *     (I - J)(X2 + i kappa C) (g = (lap - kappa^2)^{-1} div N) and
 *     (I - J) Q chi_N = i kappa ell^2 (I + J) g - (I - J) C; for k = 0
 *     (I - J) Q chi_N = -(I - J) C (all banded, half width 3; 9 transforms).
 *     This equals psi_N = -lap_h^{-1} (curl N)_z, chi_N = -lap_h^{-1} (N_z -
 *     i kappa g) of Eq. (9) up to the truncation of the products.  At m = 0 the
 *     singular first row of Q and (I - J) Q is the far-field decay condition
 *     sum_n Pbar_n^0(1) s_n = 0 (for the basis part of the state;
 *     the log proxies of mlx_vortex_logproxy carry the net circulation and
 *     flux, Sec. 3.1).  coeffs[0] = U0; the axial background Uz and the proxies'
 *     velocity and vorticity come from mlx_vortex_logproxy.
 * spec_in, spec_out: device complex128 ragged (may not alias); two fields each
 * for the vortex kind. */
int mlx_nonlinear(mlx_ctx* ctx, int kind, const double* coeffs, int ncoeffs,
                  const void* spec_in, void* spec_out, mlx_stream stream);

/* Build the horizontal-Laplacian (D_m, decay row at m = 0) and Helmholtz
 * (D_m - kappa^2) band factors, the r d/dr band and the workspace of the vortex
 * term (Sec. 3.2).  Required before MLX_NONLIN_VORTEX and mlx_lap_h_solve.
 * Synchronises `stream`. */
int mlx_vortex_setup(mlx_ctx* ctx, mlx_stream stream);

/* Axial kinetic-energy spectrum of a two-field vortex state (psi, chi) (Eq. (8); the
 * modal energy E_k of Sec. 5.3 from which the Crow growth rate is measured):
 * E[|k|] = (1/2) int over one axial period of |v_{+k}|^2 + |v_{-k}|^2 dV (for k = 0 the
 * k = 0 part alone), |k| < Kz, so that sum_k E[k] is the kinetic energy per period.
 * The velocity comes from the banded r d/dr and D_m as in the vortex term; each
 * harmonic is evaluated on the Gauss nodes with the FP64 basis table (whatever the
 * context's transform precision) under the area element r dr = ell^2 dx / (1 - x)^2.
 * The sum is the energy of the backward-transformed field on the grid: with the
 * Nyquist chop the pairs m = +-Nphi/2 and k = +-Nz/2 enter as the grid sees them
 * (the m = 0 and m = Nphi/2 blocks through their Hermitian part in k; the two rows
 * k = +-Nz/2 summed into E[Nz/2]).  Only the basis part of the state counts: the
 * log proxies' swirl (mlx_vortex_logproxy) has unbounded energy.
 * state: device, 2 n_spec complex128; E: host, Kz doubles.  Needs mlx_vortex_setup
 * (MLX_ESTATE); overwrites the vortex term's temporaries; synchronises `stream`. */
int mlx_axial_energy(mlx_ctx* ctx, const void* state, double* E, mlx_stream stream);

/* Solve grad_h^2 x = rhs harmonic by harmonic (Eq. (9)'s inverse Laplacian):
 * D_m x = rhs with the far-field decay condition in place of the singular first
 * equation at m = 0 (rhs's m = 0, n = 0 entries are not used).  FP64, device
 * complex128 ragged buffers (may not alias).  MLX_ESTATE before mlx_vortex_setup. */
int mlx_lap_h_solve(mlx_ctx* ctx, const void* rhs, void* out, mlx_stream stream);

/* Log proxy of a scalar with a nonzero planar integral (Sec. 3.1, Eq. (6)).  The
 * decaying basis cannot represent the logarithmic far field of a Poisson solution
 * whose source integrates to a nonzero value, so a scalar carries one extra real
 * amplitude c of Lambda = ln(r^2 + ell^2), whose horizontal Laplacian
 * (4/3 P_0 - 2 P_1 + 2/3 P_2) / ell^2 lies in the basis.  mlx_lap_h_solve_log
 * inverts grad_h^2 (c Lambda + x) = rhs; only the (m, k) = (0, 0) block differs
 * from mlx_lap_h_solve:
 *   MLX_LOGPROXY_PRESCRIBE: *c given: D_0 x = rhs - c lam with the far-field decay
 *     condition in place of the singular first equation (x -> 0 at infinity);
 *   MLX_LOGPROXY_SOLVE: c unknown: D_0's first column (zero: a constant has zero
 *     Laplacian) replaced by lam; the unknown in its place is returned in *c (from
 *     the real part: the (0, 0) block of a real field is real), and x's Pbar_0^0
 *     coefficient is 0.
 * The two results differ only in that constant coefficient.  The solved c is the
 * source's planar integral over 4 pi, in which the mapped area weight
 * 1 / (1 - x)^2 magnifies errors of rhs at the outermost nodes: form rhs with FP64
 * transforms (at 256^3, FP32 transforms shift c by 1 %).  FP64, device
 * complex128 ragged buffers (may not alias); *c is a host double.  The solve
 * variant synchronises `stream`.  MLX_ESTATE before mlx_vortex_setup. */
enum { MLX_LOGPROXY_PRESCRIBE = 0, MLX_LOGPROXY_SOLVE = 1 };
int mlx_lap_h_solve_log(mlx_ctx* ctx, const void* rhs, void* out, int variant, double* c, mlx_stream stream);

/* Log-proxy amplitudes of the vortex state and its axial background: psi carries
 * c_psi Lambda, chi carries c_chi Lambda (net circulation -4 pi c_psi, net axial
 * flux -4 pi c_chi), and the background becomes U = U0 e_y + Uz e_z (U0 = the
 * vortex kind's coeffs[0]).  The amplitudes are constants of the motion: the
 * vortex term (mlx_nonlinear) adds the proxies' velocity and vorticity to the
 * (0, 0) blocks of its fields, and the time steps (mlx_advance, the batch) add the
 * proxies' dissipation c L Lambda (Eq. (11) at (m, k) = (0, 0)) to the (0, 0)
 * blocks of each field's tendency.  Zero amplitudes and Uz = 0 give the default
 * vortex term.  Needs mlx_vortex_setup (MLX_ESTATE); drops the cached step graphs;
 * synchronises `stream`. */
int mlx_vortex_logproxy(mlx_ctx* ctx, double c_psi, double c_chi, double Uz, mlx_stream stream);

/* Enstrophy Z = (1/2) int |omega|^2 dV over one axial period and the largest |omega|
 * over the nodes, of a two-field vortex state with its log proxies: the vorticity
 * fields of the vortex term, backward transforms in the context's precision, the
 * mapped area rule r dr = ell^2 dx / (1 - x)^2 and the uniform phi and z rules.
 * state: device, 2 n_spec complex128; out: host.  Needs mlx_vortex_setup
 * (MLX_ESTATE); overwrites the vortex term's temporaries; synchronises `stream`. */
typedef struct {
  double enstrophy;
  double peak_vorticity;
} mlx_vortex_diag_out;
int mlx_vortex_diag(mlx_ctx* ctx, const void* state, mlx_vortex_diag_out* out, mlx_stream stream);

/* Set up the implicit operators for time step dt: per harmonic (m, |k|) the
 * band matrix of L = nu (D_m - kappa^2) - nu_h (-(D_m - kappa^2))^{p/2}
 * (Eq. (11); the power composes truncated band matrices), the band of
 * I + dt/2 L, and banded LU factors with partial pivoting of I - dt/2 L and
 * I - dt L, all in FP64 on the GPU.  p in {4, 6, 8} when nu_h > 0.
 * Synchronises `stream`. */
int mlx_implicit_setup(mlx_ctx* ctx, double nu, double nu_h, int p, double dt,
                       mlx_stream stream);

/* One implicit step per harmonic, FP64 (Eq. (12) and the FE-BE scheme):
 *   MLX_STEP_FEBE_HALF: (I - dt/2 L) out = s + dt/2 A
 *   MLX_STEP_FEBE_FULL: (I - dt   L) out = s + dt   A
 *   MLX_STEP_ABCN:      (I - dt/2 L) out = (I + dt/2 L) s + dt/2 (3 A - A_prev)
 * A may be NULL (A = 0); A_prev is read only by MLX_STEP_ABCN (NULL = 0).
 * out must not alias s, A or A_prev.  MLX_ESTATE before mlx_implicit_setup. */
int mlx_implicit_solve(mlx_ctx* ctx, int step, const void* s, const void* A,
                       const void* A_prev, void* out, mlx_stream stream);

/* Advance `nsteps` time steps of AB-CN (Eq. (12)) with the nonlinear term
 * `kind`, in place on `state` (device complex128 ragged; two fields for the
 * vortex kind, each advanced with the same implicit operator since the
 * projection commutes with the Laplacian, Sec. 3.2).  prev_A (device, same size
 * as state) holds A^{j-1} between calls.  If start != 0 the first step
 * is the Richardson start s^1 = 2 FEBE_{dt/2}(FEBE_{dt/2}(s^0)) - FEBE_dt(s^0)
 * and prev_A is overwritten with A(s^0); otherwise prev_A must hold A^{j-1}.
 * One step is captured once per (state, prev_A) pair into a CUDA graph and
 * replayed; the graph is launched on `stream`. */
int mlx_advance(mlx_ctx* ctx, int kind, const double* coeffs, int ncoeffs,
                void* state, void* prev_A, int nsteps, int start, mlx_stream stream);

/* Adaptive modal filter applied between time steps (Sec. 3.3).  Every
 * coefficient whose normalised mode index zeta = max(n/(Nc-1), m/(M-1), |k|/(Kz-1))
 * (a term is 0 when its chop keeps a single index) lies above zeta_c is multiplied by
 * exp(-eps ((zeta - zeta_c)/(1 - zeta_c))^8).  Each field's amplitude eps follows the
 * fraction f of its spectral energy (|shat|^2, multiplicity 2 for m >= 1) above the
 * cutoff, measured before the filter acts: target eps* = eps_max min(1, max(0,
 * (f - tau)/tau)) (inactive below tau, saturated at 2 tau), relaxed as
 * eps <- eps + relax (eps* - eps) and kept in [0, eps_max].  The paper fixes the form,
 * the tail-fraction rule and tau = 2e-2; the other defaults are this library's
 * readings: zeta_c = 2/3, eps_max = 36, relax = 1/4.
 * mlx_filter_setup: enable != 0 turns the filter on in mlx_advance (after the
 * Richardson start and after every AB-CN step; every field of the state has its own
 * eps) and resets eps to 0, params NULL = the defaults (MLX_EINVAL unless
 * 0 <= zeta_c < 1, tau > 0, eps_max >= 0, 0 < relax <= 1); enable = 0 turns it off.
 * The first enable allocates a small state (partial sums and multiplier tables).
 * Invalidates cached graphs.
 * mlx_filter_apply: one filter step on a device state of nfields (1 or 2)
 * complex128 ragged fields, in place, updating the amplitudes (MLX_ESTATE before
 * the first enable).  mlx_filter_state: host copies of eps and of the last tail
 * fraction f per field (2 values each, may be NULL); synchronous. */
typedef struct {
  double zeta_c, tau, eps_max, relax;
} mlx_filter_params;
int mlx_filter_setup(mlx_ctx* ctx, int enable, const mlx_filter_params* params);
int mlx_filter_apply(mlx_ctx* ctx, void* state, int nfields, mlx_stream stream);
int mlx_filter_state(mlx_ctx* ctx, double* eps, double* tail);

/* Integral diagnostics of one spectral scalar field (Eq. (16) and the weighted
 * norm of the examples, Sec. 5.1), evaluated in FP64 from the coefficients with the
 * context's FP64 basis table, whatever its transform precision; the area element
 * is r dr = ell^2 dx / (1 - x)^2 (Eq. (1)) on the Gauss nodes:
 *   integral = (1/Lz) int f dA dz  (the circulation Gamma when f is omega_z),
 *   moment2  = (1/Lz) int r^2 f dA dz  (the second moment M2),
 *   l2w      = sqrt((1/Lz) int f^2 dA dz)  (the relative weighted L2 error of two
 *              fields is l2w(a - b) / l2w(b)),
 *   spec_l2  = the spectral l2 norm, multiplicity 2 for m >= 1.
 * spec: device complex128 ragged (n_spec values), 16-byte aligned.  The first call
 * allocates a small buffer of partial sums (M K x 4 doubles) kept by the context.
 * Synchronises `stream`.  MLX_EINVAL for NULL or misaligned pointers. */
typedef struct {
  double integral, moment2, l2w, spec_l2;
} mlx_diag_out;
int mlx_diag(mlx_ctx* ctx, const void* spec, mlx_diag_out* out, mlx_stream stream);

/* Checkpoint images of a time-stepping state (no counterpart in the paper's
 * equations; its runs restart from saved fields).  An image is a host buffer of
 * mlx_state_bytes(ctx, kind) bytes: a header (grid, chops, ell, Lz, the implicit
 * setup nu, nu_h, p, dt, the caller's step counter; for the vortex kind the
 * log-proxy amplitudes and axial background of mlx_vortex_logproxy) followed by the state and
 * A^{j-1} (complex128 ragged, one or two fields by kind).  mlx_get_state copies the
 * device buffers state and prev_A into `host` (caller-owned, at least that many
 * bytes); mlx_set_state checks the header against this context and copies back into
 * the device buffers, returning the step counter in *step (may be NULL).  A
 * mismatched grid, chop, ell, Lz or field count, or (when both the image and the
 * context have an implicit setup) another dt, nu, nu_h or p, or (vortex kind) other
 * log-proxy amplitudes or axial background, is MLX_EINVAL with the
 * reason in mlx_last_cuda_error: A^{j-1} continues the AB-CN recurrence (Eq. (12))
 * only under the same operator and step.  Both synchronise `stream`.  Resuming
 * with mlx_advance(..., start = 0) reproduces the uninterrupted run bitwise.
 * mlx_state_bytes returns -1 for a NULL context or an unknown kind. */
long long mlx_state_bytes(const mlx_ctx* ctx, int kind);
int mlx_get_state(mlx_ctx* ctx, int kind, const void* state, const void* prev_A, long long step, void* host,
                  long long bytes, mlx_stream stream);
int mlx_set_state(mlx_ctx* ctx, int kind, const void* host, long long bytes, void* state, void* prev_A,
                  long long* step, mlx_stream stream);

/* Launch-shape tuning (not part of the method).  Keys:
 *   "solve_cpw": real chains per warp of the banded solve, 4, 8, 16 or 32
 *                (default 8);
 *   "solve_wpb": warps per CTA of the banded solve, 1, 2 or 4 (default 4).
 *   "solve_keep_s": 1 (default) = the staged solve keeps a shared-memory copy
 *                of s for the AB-CN "- s" (no global re-read); 0 = re-read s (a
 *                smaller CTA; mlx_batch_create sets 0 on its members).
 *   "solve_direct": 2 = lean banded-solve variant: 32 (or 16, "solve_lean_cpw")
 *                chains per warp, the factors read as per-row records packed at
 *                setup (one contiguous 16-byte-aligned block per row and |k|,
 *                cp.async 12 rows ahead), the eliminated values in a global scratch
 *                of about M * Kz * 4 * Nc doubles (allocated when 2 is first set;
 *                MLX_ENOMEM if that fails); 0 = the staged (or, at half width 2,
 *                segmented) solve.  Default 2 for hyperviscous bands (half width
 *                >= 4, set by mlx_implicit_setup), else 0.  The staged and lean
 *                variants give bitwise-equal results.
 *   "phi_tile", "z_tile": radii per CTA of the phi and z transform kernels,
 *                2, 4, 8, 16 or 32; 0 (default) = the largest tile whose grid
 *                still has 2 (phi) or 4 (z) CTAs per SM.
 *   "solve_seg": 8 (default) or 4 = half-width-2 implicit solves (diffusion,
 *                Fisher-KPP) cut every chain into that many row segments solved
 *                side by side: each segment's particular solution plus a linear
 *                function of its entry state, from influence data computed at
 *                mlx_implicit_setup or when this key changes (needs
 *                Nc - M + 1 >= 4 x segments; 8 falls back to 4, else the staged
 *                solve runs);
 *                results agree with the other variants to rounding, not
 *                bitwise; 0 = off.
 *   "solve_df": 1 (default) = in the MLX_FP32 and MLX_BF16X3 forms the pivot-free
 *                segmented solve computes in double-float arithmetic (pairs of
 *                FP32 numbers, about 47 significant bits per multiply-add) on the
 *                FP32 pipe, from factor records converted at setup; the right-hand
 *                side is formed in FP64 and the output rounded to FP64; 0 = FP64
 *                arithmetic.  Results agree to the FP64 form's error bound with
 *                2^-47 in place of 2^-53; the MLX_FP64 form always uses FP64.
 *   "solve_lean_cpw": real chains per warp of the lean variant, 16 or 32
 *                (default 32).
 *   "vortex_planes": 1 (default) = an MLX_BF16X3 vortex term writes its six
 *                velocity and vorticity fields straight into the backward
 *                contraction's split planes (one set per field, allocated by
 *                mlx_vortex_setup) instead of as FP64 fields split afterwards;
 *                0 = the FP64 fields.  Bitwise-equal results.
 *   "plane_reuse": 1 (default) = in the graph-replayed MLX_BF16X3 Fisher-KPP steps
 *                (no filter) the segmented solve also writes the BF16x3 split
 *                planes of its output, and every step of the call after its first
 *                takes them instead of splitting the state again; 0 = split every
 *                step.  Bitwise-equal results.
 *   "solve_fields2": 1 (default) = the lean variant solves both fields of a
 *                vortex state in one launch (each staged factor record serves
 *                the 8 real chains of both fields at one |k|, so a step reads the
 *                factors once); 0 = one launch per field.  Bitwise-equal results.
 *   "tc_bn":     column-tile width of the MLX_BF16X3 contraction (16..256, used
 *                up to 128; the width actually used is rounded to a multiple of 16
 *                that splits the 2K columns evenly);
 *   "tc_expire": test hook of the bounded waits: 1 makes the MLX_BF16X3
 *                contraction's first shared-memory stage-reuse wait report expiry
 *                at once (the kernel then drains the copies and MMAs it issued, frees
 *                its tensor memory and returns; mlx_device_status reports
 *                MLX_ETIMEOUT; results of that call are undefined); 0 (default) off.
 *                Only launches whose CTAs walk more than four 32-wide K chunks reach
 *                a stage reuse.
 *   "tc_products": BF16 split products per term in the MLX_BF16X3 contraction,
 *                6 (hi*hi, hi*mid, mid*hi, hi*lo, lo*hi, mid*mid) or 8 (adds
 *                mid*lo, lo*mid); default 6.
 *   The substitution is a sequential FP64 recurrence per real chain; the best
 *   shape trades per-warp staging latency against FP64 pipe sharing.
 * Invalidates cached graphs.  MLX_EINVAL for an unknown key or value. */
int mlx_set_tuning(mlx_ctx* ctx, const char* key, int value);

/* ---- batched uneven solves and launch-shape autotuning (no counterpart in the
 * paper, whose runs are single problems) ----
 * A batch groups n independent contexts (any sizes, precisions and kinds; each
 * created and set up by the caller, which keeps owning them).  The batch owns
 * only streams, events, cached CUDA graphs and the work lists of its persistent
 * launches.  Creating a batch sets the tuning key "solve_keep_s" of every member
 * to 0 (smaller shared-memory footprint per solve warp, so that more warps and
 * the instances' kernels co-reside) and "solve_df" to 0 (FP64 recurrences: the
 * persistent solve launch over many small systems runs faster with them). */
typedef struct mlx_batch mlx_batch;
int mlx_batch_create(mlx_ctx* const* ctxs, int n, mlx_batch** out);
int mlx_batch_destroy(mlx_batch* batch);

/* Advance every instance i of the batch by nsteps AB-CN steps, exactly as
 * mlx_advance(ctxs[i], kinds[i], &coeffs[i], 1, states[i], prev_As[i], nsteps,
 * start) would (same arithmetic, bitwise), with the two-step pairs of all
 * instances captured into ONE CUDA graph; one graph launch per pair advances the
 * whole batch.  The Richardson start (start != 0) and an odd last step run per
 * instance.  The graph takes one of two forms (mlx_batch_set_persistent):
 *  - persistent (default, used when every instance is MLX_NONLIN_NONE or
 *    MLX_NONLIN_FKPP, has no filter, Nphi <= 256 and Nz <= 256, and, for
 *    MLX_BF16X3, six split products): each phase of a time step is one persistent
 *    kernel launch whose CTAs (warps for the solve) take (instance, tile) work
 *    items of all instances from a queue, largest first -- the BF16x3 split of the
 *    states with the backward contraction (tensor-core launches serve up to 64
 *    instances each), the inverse z transform, the fused phi synthesis / product /
 *    analysis, the forward z transform, the forward contraction and the banded
 *    solve (one launch per half width and shared-memory size class).  Instances
 *    without a nonlinear term only solve, on a graph branch beside the transform
 *    phases.  Each instance keeps its own launch shapes (transform tiles,
 *    column-tile width, chains per warp), and no kernel waits on another CTA;
 *  - branches: every instance's own kernel sequence on its own graph branch,
 *    the branches running concurrently.
 * The graph is cached per set of (state, prev_A, kind, coefficient) and
 * recaptured when a member's tuning or setup changes.  MLX_ESTATE if an instance
 * lacks mlx_implicit_setup (or mlx_vortex_setup for the vortex kind). */
int mlx_batch_advance(mlx_batch* batch, const int* kinds, const double* coeffs, void* const* states,
                      void* const* prev_As, int nsteps, int start, mlx_stream stream);

/* Select the batch's graph form: 1 (default) persistent per-phase launches
 * whenever the instances qualify (see mlx_batch_advance), 0 one graph branch per
 * instance.  Both give bitwise-equal results.  MLX_EINVAL for another value. */
int mlx_batch_set_persistent(mlx_batch* batch, int on);

/* Choose the launch shapes of ctx for its nonlinear `kind` by timing candidates
 * with CUDA events on the context's temporaries: the tensor-core column-tile
 * width (MLX_BF16X3 only) and the banded-solve variant and shape.  Results are
 * cached in the text file cache_path (may be NULL), one line
 * "sizes precision kind band|bn cpw wpb"; a cached entry is applied without
 * timing.  chosen (may be NULL) receives {bn, cpw, wpb, from_cache}; cpw = 0
 * (wpb = 0) denotes the segmented solve ("solve_seg" 8, half width 2 only),
 * cpw = 2 (wpb = 0) the lean variant ("solve_direct" 2), otherwise the staged
 * solve with cpw chains per warp and wpb warps per CTA.  The context's
 * temporaries are overwritten; call it before advancing.  Synchronises `stream`. */
int mlx_autotune(mlx_ctx* ctx, int kind, const double* coeffs, int ncoeffs, const char* cache_path,
                 int* chosen, mlx_stream stream);

/* ---- learned spectral surrogate of the vortex solver (no counterpart in the
 * paper; its reference is the plain method itself) ----
 * A surrogate advances the two-field vortex state s = (psi, chi) (complex128,
 * 2 n_spec values, D = 4 n_spec reals) by nsub time steps in one call:
 *     s_next = E^nsub s + sigma_out * f(s / sigma_in)
 * where E = (I - dt/2 L)^-1 (I + dt/2 L) is the AB-CN step of Eq. (12) with the
 * nonlinear term removed (dissipation of Eq. (11) only, the context's cached
 * banded factors), and f is a 4-layer perceptron on the real view of the
 * coefficients: f(x) = W4 h3 + b4, h_l = GELU(W_l h_{l-1} + b_l), h_0 = x, with
 * GELU(z) = z Phi(z) (Phi the standard normal CDF).  Weights and activations
 * enter the GEMMs as BF16 (round to nearest even), accumulation and the
 * pre-activations are FP32, master weights and Adam moments FP32.
 * Parameter layout, flat FP32 of mlx_sur_param_count() values:
 *     W1 [w][D], b1 [w], W2 [w][w], b2 [w], W3 [w][w], b3 [w], W4 [D][w], b4 [D]
 * (W_l row-major, one row per output neuron).  Training data (X, T) are device
 * arrays [n][D]: X BF16 inputs s / sigma_in, T FP32 targets
 * (s_next - E^nsub s) / sigma_out, filled by mlx_sur_make_pair.
 * The surrogate owns its parameters, moments, activations and a solver-side
 * workspace allocated on first use with a vortex context (4 two-field states).
 * Calls on one surrogate are not thread-safe. */
typedef struct mlx_sur mlx_sur;

/* Create a surrogate for states of D reals with hidden width `width` (1..1024)
 * and at most bmax (1..4096) samples per training or inference batch.
 * Parameters are drawn uniformly from a counter-based hash of `seed`: hidden
 * layers U(-sqrt(6/fan_in), +), the output layer 1e-3 times that, biases zero.
 * Scales start at 1.  MLX_ENOMEM if device memory runs out. */
int mlx_sur_create(int D, int width, int bmax, unsigned long long seed, mlx_sur** out);
int mlx_sur_destroy(mlx_sur* sur);
/* Number of FP32 parameters (w D + 2 w^2 + D w + 3 w + D), -1 for NULL. */
long long mlx_sur_param_count(const mlx_sur* sur);
/* Device status of the surrogate's tensor-core kernels: MLX_ETIMEOUT (and the word
 * is cleared) if a bounded wait expired since the last call, else MLX_OK.
 * Synchronises the device. */
int mlx_sur_status(mlx_sur* sur);
/* Host copies of the FP32 parameters and of the gradient of the last training
 * step (both in the parameter layout); set_params also refreshes the BF16 copies.
 * These synchronise the device. */
int mlx_sur_get_params(const mlx_sur* sur, float* host);
int mlx_sur_set_params(mlx_sur* sur, const float* host);
int mlx_sur_get_grads(const mlx_sur* sur, float* host);
/* Host copies of sigma_in and sigma_out (D floats each).  set_scales wants
 * sigma_in > 0, sigma_out >= 0 and not all zero (MLX_EINVAL otherwise); it also
 * sets the loss weights w_i above.  A new surrogate has all scales 1 (w_i = 1). */
int mlx_sur_get_scales(const mlx_sur* sur, float* in_scale, float* out_scale);
int mlx_sur_set_scales(mlx_sur* sur, const float* in_scale, const float* out_scale);

/* out = E^nsub state (device two-field states, out != state).  The context must
 * have mlx_vortex_setup and mlx_implicit_setup done (MLX_ESTATE otherwise) and
 * D = 4 n_spec (MLX_EINVAL otherwise). */
int mlx_sur_propagate(mlx_ctx* ctx, mlx_sur* sur, const void* state, void* out, int nsub, mlx_stream stream);
/* Scale fitting: observe accumulates, for one solver pair (s0, s1 = S^nsub(s0)),
 * the squares of s0 and of the remainder r = s1 - E^nsub s0 per coefficient.
 * finalize sets  sigma_in_i = max(rms_i(s0), in_floor rms(s0))  (1 where that is
 * 0) and  sigma_out_i = max(rms_i(r), out_floor rms(r))  (out_floor >= 1: the
 * uniform rms(r)), with rms_i over the observed pairs and rms over pairs and
 * coefficients, then clears the statistics and synchronises `stream`.  A zero
 * sigma_out_i (a coefficient the solver never changes beyond E, e.g. by symmetry)
 * gives that coefficient no correction.  MLX_EINVAL with no observation or a
 * negative floor.  The training loss weights coefficient i by
 * w_i = sigma_out_i^2 / mean_j(sigma_out_j^2), so that it measures the squared
 * coefficient-space error of the correction sigma_out * f, the judge's norm. */
int mlx_sur_observe(mlx_ctx* ctx, mlx_sur* sur, const void* s0, const void* s1, int nsub, mlx_stream stream);
int mlx_sur_finalize_scales(mlx_sur* sur, double in_floor, double out_floor, mlx_stream stream);
/* One training sample from a solver pair: x (device BF16, D) = s0 / sigma_in,
 * t (device FP32, D) = (s1 - E^nsub s0) / sigma_out. */
int mlx_sur_make_pair(mlx_ctx* ctx, mlx_sur* sur, const void* s0, const void* s1, int nsub, void* x, float* t,
                      mlx_stream stream);
/* y (device FP32 [B][D]) = f(X[idx[b]]) for b < B (idx: device int32 [B]). */
int mlx_sur_infer(mlx_sur* sur, const void* X, const int* idx, int B, float* y, mlx_stream stream);
/* One training step on the rows idx[0..B-1] of (X, T): forward, the loss
 * mean_{b,i} w_i (f(x_b)_i - t_{b,i})^2 (written to the device float `loss` when not
 * NULL), its gradient by the hand-written backward pass (kept for
 * mlx_sur_get_grads), and with lr > 0 one Adam step (beta1 0.9, beta2 0.999,
 * eps 1e-8, bias-corrected); lr = 0 computes the gradient only. */
int mlx_sur_train_step(mlx_sur* sur, const void* X, const float* T, const int* idx, int B, float lr, float* loss,
                       mlx_stream stream);
/* One surrogate call on the device two-field state (in place): the prediction
 * E^nsub s + sigma_out f(s / sigma_in), whose m = 0 block (of each field) is then
 * projected onto the structure of every solver state: Hermitian in k (the
 * average of k and -k conjugated; imaginary part 0 at k = 0), and the far-field
 * decay condition sum_n Pbar_n^0(1) s_{k,n} = 0, Pbar_n^0(1) = sqrt((2n+1)/2),
 * solved for s_{k,0} at every k.  With judge != 0 the plain method also
 * advances s by nsub steps (Richardson start, then AB-CN; background U0 e_y as
 * in mlx_advance) and the relative residual ||pred - solver|| / ||solver|| (real
 * Euclidean norm over all coefficients) decides: <= tol keeps the prediction
 * (*accepted = 1), otherwise the solver's state is kept (*accepted = 0).
 * Without the judge the prediction is kept (*accepted = 1, *residual = -1) and
 * the call is asynchronous on `stream`; with the judge it synchronises `stream`.
 * accepted / residual may be NULL. */
int mlx_sur_advance(mlx_ctx* ctx, mlx_sur* sur, void* state, int nsub, double U0, int judge, double tol,
                    int* accepted, double* residual, mlx_stream stream);

/* ---- measurement support (not part of the method) ----
 * Opt-in per-launch timing.  enable = 1: every kernel launch of this context is
 * bracketed by CUDA events recorded on its stream, and mlx_advance launches its
 * steps directly instead of replaying a CUDA graph.  enable = 2: mlx_advance
 * captures its two-step graph with an event-record node before and after every
 * kernel node and replays it pair by pair, reading the node timings after each
 * replay (host synchronisation between replays; inside a replay the kernels run
 * back to back as in the cached graph).  enable = 0 turns timing off; other values
 * are MLX_EINVAL.  Changing the mode resets the counters.  mlx_timing_read
 * synchronises on the recorded events and returns, for kernel id
 * 0 <= kernel < mlx_kernel_count(), the number of timed launches and their summed
 * device time in milliseconds.  mlx_kernel_name gives a stable short name per id
 * ("" when out of range). */
int mlx_timing(mlx_ctx* ctx, int enable);
int mlx_timing_read(mlx_ctx* ctx, int kernel, long long* launches, double* total_ms);
int mlx_kernel_count(void);
const char* mlx_kernel_name(int kernel);

/* Device status: synchronises the device, returns MLX_ETIMEOUT if a kernel of this
 * context gave up a bounded wait since the last call, else MLX_ENUMERIC if a
 * nonlinear-product kernel (the Fisher-KPP reaction or the vortex cross product)
 * met a non-finite value (a blown-up or NaN state), else MLX_OK; the word is
 * cleared by the read.  Kernels that give up a wait skip their remaining work and
 * release their resources; their outputs are then undefined. */
int mlx_device_status(mlx_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MLX_H */
