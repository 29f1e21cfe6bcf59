// Internal definitions shared by the CUDA translation units of libmlx.
#pragma once

#include <cuda.h>            // CUtensorMap (header only; the driver entry point is fetched at run time)
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>
#include <map>
#include <utility>

#include "../../include/mlx.h"

#define MLX_CUDA_TRY(ctx, call)                                              \
  do {                                                                       \
    cudaError_t _e = (call);                                                 \
    if (_e != cudaSuccess) {                                                 \
      if (ctx) (ctx)->last_err = std::string(#call) + ": " + cudaGetErrorString(_e); \
      return MLX_ECUDA;                                                      \
    }                                                                        \
  } while (0)

#define MLX_LAUNCH_CHECK(ctx) MLX_CUDA_TRY(ctx, cudaGetLastError())

// Programmatic dependent launch of the time step's kernels (phi and z transforms,
// the single-context tensor-core contraction, the segmented solve): the kernel may
// be launched while its predecessor in the stream is still finishing, and every
// such kernel calls pdl_wait() -- which returns once the predecessor grid has
// completed and its memory is visible -- before it touches global memory, so the
// order of all memory accesses is that of plain launches.  pdl_trigger() lets the
// successor launch: at the start of single-wave kernels (whose CTAs are all resident
// from the start, so a waiting successor only takes what their exits free), at the
// end of each CTA of the multi-wave transform kernels.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Kernel identifiers for the opt-in per-launch CUDA-event timing.
enum KernelId {
  KID_PHI_FWD = 0, KID_PHI_BWD, KID_PHI_FKPP, KID_Z_FWD, KID_Z_BWD,
  KID_LEG_FWD, KID_LEG_BWD, KID_BAND_SOLVE, KID_AXPBY, KID_LEG_SPLIT, KID_COUNT
};

struct TimingState {
  bool on = false;
  int mode = 0;                  // 1: direct launches bracketed by events; 2: graph replay with
                                 // event-record nodes around every kernel node
  long long launches[KID_COUNT] = {0};
  double ms[KID_COUNT] = {0};
  std::vector<cudaEvent_t> pool;
  struct Pending { int kid; cudaEvent_t a, b; };
  std::vector<Pending> pending;  // recorded by direct launches, resolved by mlx_timing_read
  std::vector<Pending> captured; // recorded as graph nodes, resolved after every replay
};

// One GEMM work tile of the ragged per-m Legendre contraction.
struct LegTile {
  int m;     // azimuthal order
  int row0;  // first output row of the tile (n - m for forward, i for backward)
  int col0;  // first output column (0..2K-1; column c < K is Re of k = c, else Im)
  int pad;
};

// Banded implicit operator storage for one matrix family, per (m, |k|):
// rows i = 0..N_m-1 (N_m = Nc - m).  U row i holds columns i..i+kl+ku
// (ku_f = kl + ku entries after the diagonal), L holds kl multipliers per
// column, piv the pivot row of each column, invd 1/U[i][i].
// Destination of the BF16x3 split planes of a spectral field, the backward
// contraction's data operand: bs[part][(m 2K + 2 kidx + (0 Re, 1 Im)) Kq + (n - m)]
struct SplitPlanes {
  unsigned short* bs = nullptr;
  long long part = 0;
  int Kq = 0, K2 = 0;
};

// ---- batched persistent launches (batch.cu) ----
// A batched launch runs one phase of the time step (a transform stage, the
// contraction, the solve) for many contexts at once: its CTAs (or warps) take
// work items from a queue, ctr[0] handing out item indices in order (items sorted
// by decreasing cost), until the queue is empty.  ctr[1] counts the workers that
// found it empty; the last one resets both words, so that the next launch of the
// same queue (a graph replay) starts from zero without a memset.  No worker waits
// on another.
__device__ __forceinline__ void bq_finish(int* ctr, int workers) {
  __threadfence();
  if (atomicAdd(ctr + 1, 1) == workers - 1) {
    atomicExch(ctr, 0);
    atomicExch(ctr + 1, 0);
  }
}

// One member's transform stage in a batched FFT launch.  phi: a = physical field
// (unused by the fused Fisher-KPP stage), b / c = Re / Im planes of its Fourier
// planes; z: a / b = Re / Im of the zm planes, c / d = Re / Im of the mixed planes.
// bs != NULL: the stage writes the BF16x3 split planes of the contraction's data
// operand (part elements per part plane, row length kp, 2K columns per m).
struct BFftJob {
  int N, logN, M, Nr, R, E;   // N: transform length (Nphi or Nz), E = max(N / 32, 1)
  int Kz, K;
  void* a; void* b; void* c; void* d;
  const void* tw;
  double gamma;
  int* err;
  unsigned short* bs; long long part; int kp, k2;
};

// One member's SIMT contraction (FP32 / FP64) in a batched launch.
struct BLegJob {
  int nc, nr, M, K;
  const long long* boff;
  const long long* soff;
  const void* table;   // W (forward) or P (backward), the member's element type
  void* mixed;
  double2* spec;
};

// One member's AB-CN banded solve (staged form) in a batched launch.
struct BSolveJob {
  int variant;          // 0 staged; 1 / 2 segmented, 8 / 4 segments; 3 / 4 the same, pivot-free;
                        // 5 / 6 pivot-free in double-float arithmetic (RNP, PSf then hold
                        // the double-float records)
  int M, nc, Kz, K, CPW, gpm, step, kz_fac;
  double dt;
  const long long* soff;
  const long long* band_off;
  const double* U;
  const double* L;
  const int* piv;
  const double* invd;
  const double* s;
  const double* A;
  const double* Ap;
  double* out;
  double* Az;           // NULL, or A^j of a member without a nonlinear term (written as zeros)
  const double* PHf;    // segmented variants: influence data and pivot-free records
  const double* PHb;
  const double* PSf;
  const double* RNP;
  unsigned short* bs;   // segmented variants: split planes of out (NULL: none)
  long long part;
  int kq, k2;
};

// One member's BF16x3 split of its spectral state (backward data operand) in a
// batched launch: bs[part][(m 2K + 2 kidx + p) Kq + (n - m)].
struct SplitJob {
  int nc, K, Kq, pad_;
  long long part;
  const long long* soff;
  const double2* spec;
  unsigned short* bs;
};

// members of one batched tensor-core contraction launch (the launch parameters
// hold two 128-byte tensor maps and the sizes of each)
constexpr int kTcBatchMax = 64;
struct TcBatchPlan;
int mlx_tc_batch_plan(mlx_ctx* const* members, int n, bool fwd, double2* const* specs, const char* need_split,
                      TcBatchPlan** out);
int mlx_tc_batch_launch(TcBatchPlan* plan, cudaStream_t st);
void mlx_tc_batch_free(TcBatchPlan* plan);

// One part of a member's solve in a batched launch (host side): its job, its warp
// items (member index 0, warp task) with their costs, and its shared memory per warp.
struct BSolvePart {
  BSolveJob job;
  std::vector<int2> items;
  std::vector<double> cost;
  int slab = 0;
};

struct BandLU {
  double* U = nullptr;     // [rows][W_u] with W_u = 1 + kl + ku
  double* L = nullptr;     // [rows][kl]
  int* piv = nullptr;      // [rows]
  double* invd = nullptr;  // [rows]
  // per-row records of the lean solve: forward {L row, pivot offset mask, pad}, back
  // substitution {U[row - t][t + 1] (t < 2 kl), 1/diag[row - 2 kl], pad}
  double* FS = nullptr;
  double* BS = nullptr;
  // segmented solve (half width 2): forward influence of the entry window per row
  // [rows][kl] and per segment [system][seg][kl][kl], back influence [rows][2 kl]
  double* PHf = nullptr;
  double* PHb = nullptr;
  double* PSf = nullptr;
  int seg = 0;             // segments the influence data were built for (0 = none)
  int seg_m = 0;           // the data cover the orders m < seg_m (the staged solve takes the rest)
  bool nopiv = false;      // no system of the family interchanged rows (segmented solve skips pivoting)
  // pivot-free segmented solve: one contiguous record per system row, the system's
  // rows back to back ([m][|k|][row], record = {L[kl], 1/diag, U upper[kl], PHf[kl],
  // PHb[kl], pad}), so that a warp stages its systems as one block
  double* RNP = nullptr;
  // the same records and the per-segment entry-window data (PSf) as double-float
  // pairs (hi, lo) for the FP32 and BF16x3 forms' double-float solve
  void* RDF = nullptr;
  void* PSDF = nullptr;
};

struct mlx_ctx {
  // sizes
  int nr, nphi, nz, nc, M, Kz, K;
  int precision;
  double ell, lz;
  long long n_phys, n_spec;
  long long tri;                       // T = sum_m (Nc - m)
  std::vector<long long> soff;         // spectral offset of m (complex units), size M+1
  std::vector<long long> boff;         // basis-table offset of m (elements), size M+1
  long long* d_soff = nullptr;
  long long* d_boff = nullptr;

  // nodes and basis (FP64 generated on the GPU)
  double* d_x = nullptr;
  double* d_w = nullptr;
  double* d_r = nullptr;
  double* d_P64 = nullptr;             // Pbar_n^m(x_i), [m][n-m][i]
  double* d_W64 = nullptr;             // w_i Pbar_n^m(x_i), same layout
  float* d_P32 = nullptr;
  float* d_W32 = nullptr;
  double* d_lap = nullptr;             // Laplacian band, [tri][5] (offsets -2..+2)

  // Fourier twiddles exp(-2 pi i t / N), t < N/2, as (cos, sin) pairs
  double2* d_twphi64 = nullptr;
  double2* d_twz64 = nullptr;
  float2* d_twphi32 = nullptr;
  float2* d_twz32 = nullptr;

  // Legendre GEMM tiles
  LegTile* d_tiles_fwd = nullptr;
  LegTile* d_tiles_bwd = nullptr;
  int ntiles_fwd = 0, ntiles_bwd = 0;

  // tensor-core (BF16x3) form of the Legendre contraction
  void* d_Wb = nullptr;                // BF16 splits of W: [3][T][Kp]
  void* d_Pb = nullptr;                // BF16 splits of P^T: [3][M*Nr][Kq]
  CUtensorMap tmapW, tmapP;
  void* d_bsf = nullptr;               // BF16 splits of the forward data operand: [3][M*2K][Kp]
  void* d_bsb = nullptr;               // ... of the backward data operand: [3][M*2K][Kq]
  CUtensorMap tmapBf, tmapBb;
  // the six vortex fields' backward data operands, written by the fields kernel:
  // [6][3][M*2K][Kq] with one tensor map per field (BF16X3 vortex contexts)
  void* d_bsv = nullptr;
  CUtensorMap tmapBv[6];
  long long tc_kp = 0, tc_kq = 0;      // padded contraction lengths (multiples of 32)
  long long* d_arowW = nullptr;
  long long* d_arowP = nullptr;
  LegTile* d_tc_fwd = nullptr;
  LegTile* d_tc_bwd = nullptr;
  int ntc_fwd = 0, ntc_bwd = 0, tc_bn = 0, tc_tmem_cols = 0;
  int tc_products = 6;                 // BF16 split products per term: 6 or 8
  int tc_expire = 0;                   // test hook: the contraction's first stage-reuse wait reports expiry
  int* d_err = nullptr;                // device status word: bits 1, 2, 4 bounded waits that
                                       // expired; bit 16 a non-finite nonlinear product

  // workspace (element type follows precision)
  void* d_mixed = nullptr;             // planar complex [2][K][M][Nr]
  void* d_zm = nullptr;                // planar complex [2][Nz][M][Nr]
  void* d_phys = nullptr;              // physical scratch [Nz][Nphi][Nr]
  double2* d_specA = nullptr;          // A^j
  double2* d_spec1 = nullptr;          // Richardson temporaries
  double2* d_spec2 = nullptr;
  double2* d_spec3 = nullptr;

  // implicit operators
  bool implicit_ready = false;
  double nu = 0, nu_h = 0, dt = 0;
  int p = 8;
  int kl = 2;                          // half bandwidth of L (2, or p with nu_h > 0)
  long long band_rows = 0;             // sum_m (Nc - m) * Kz
  std::vector<long long> band_off;     // row offset of (m, kabs=0), size M+1 (rows of m = Kz * N_m)
  long long* d_band_off = nullptr;
  double* d_Bplus = nullptr;           // band of I + dt/2 L, [rows][2kl+1]
  BandLU lu_half, lu_full;
  // Laplacian-family factors (vortex projection): D_m per m, D_m - kappa^2 per (m, |k|)
  bool lap_ready = false;
  BandLU lu_lap, lu_helm;
  long long* d_lap_off = nullptr;      // row offset of m in the D_m factors (sum_{m'<m} (Nc - m'))
  // vortex projection factors (Q, H per m; G per (m, |k|)), half bandwidth 3
  bool proj_ready = false;
  BandLU lu_Q, lu_H, lu_G;
  // vortex term workspace
  bool vortex_ready = false;
  double* d_rdr = nullptr;             // r d/dr band, [tri][2] (offsets -1, +1)
  void* d_rdr_df = nullptr;            // the same and the D_m band as double-float pairs (hi, lo),
  void* d_lap_df = nullptr;            // for the mixed-precision forms' vortex term
  double* d_jac = nullptr;             // Jacobi matrix off-diagonal e_{m,i} (x Pbar_{m+i} couples i, i+1), [tri]
  double2* d_vspec = nullptr;          // 9 spectral temporaries
  void* d_vphys = nullptr;             // 6 physical temporaries
  double* d_setup_scratch = nullptr;
  double* d_diag = nullptr;            // mlx_diag partial sums [M K][4] and result [4]
  double* d_enst = nullptr;            // mlx_vortex_diag partials [blocks][2] and result [2]
  // log proxies of the vortex state (Sec. 3.1, Eq. (6)) and the axial background
  bool lp_on = false;                  // c_psi or c_chi nonzero
  double lp_cpsi = 0, lp_cchi = 0, vortex_uz = 0;
  double* d_lp = nullptr;              // proxy tables (field additions, lap_h Lambda, L Lambda, scratch)
  // adaptive modal filter (between steps): per-field [eps, tail] x 2, partials [M K][2],
  // multiplier tables [2][Nc + M + Kz]
  bool filter_on = false;
  double* d_filt = nullptr;
  double filt_zeta_c = 2.0 / 3.0, filt_tau = 2e-2, filt_eps_max = 36.0, filt_relax = 0.25;
  int solve_cpw = 8;                   // real chains per warp in the banded solve (4..32)
  int solve_wpb = 4;                   // warps per CTA in the banded solve (1..4)
  int solve_direct = 0;                // 2: lean variant (16 or 32 chains per warp, packed
                                       // factor records, global scratch); 0: staged or segmented
  int solve_lean_cpw = 32;             // chains per warp of the lean variant: 16 or 32
  double* d_solve_y = nullptr;         // scratch of the lean variant, [warp][Nc][CPW]
  int solve_keep_s = 1;                // staged variant: copy of s in shared memory for the AB-CN "- s"
  int phi_tile = 0;                    // radii per CTA of the phi kernels (2..32; 0 = automatic)
  int z_tile = 0;                      // radii per CTA of the z kernels (1..32; 0 = automatic)
  int solve_seg = 8;                   // segments of the half-width-2 segmented solve (8, 4; 0 = off)
  int solve_df = 1;                    // 1: FP32 / BF16X3 forms run the pivot-free segmented solve in double-float
  int solve_nopiv = 1;                 // 1: the segmented solve skips pivoting for families without interchanges
  int solve_fields2 = 1;               // 1: the lean solve takes both vortex fields in one launch
  int plane_reuse = 1;                 // 1: the graph-replayed FKPP steps reuse the solve's split planes
  int vortex_planes = 1;               // 1: the BF16X3 vortex fields are written as split planes directly

  // graphs cached per (state, prev_A, kind, gamma, variant); variant 1 is the pair
  // that reuses the split planes the previous pair left (graph_left: the pair leaves them)
  struct GraphKey {
    void* s; void* a; int kind; double c0; int variant;
    bool operator<(const GraphKey& o) const {
      if (s != o.s) return s < o.s;
      if (a != o.a) return a < o.a;
      if (kind != o.kind) return kind < o.kind;
      if (c0 != o.c0) return c0 < o.c0;
      return variant < o.variant;
    }
  };
  std::map<GraphKey, cudaGraphExec_t> graphs;
  std::map<GraphKey, bool> graph_left;
  unsigned long long graph_gen = 0;    // bumped whenever the cached graphs are invalidated: a
                                       // batch holding graphs of this context recaptures them
  cudaStream_t cap_stream = nullptr;

  TimingState timing;
  std::string last_err;
};

// RAII bracket: with timing on, records CUDA events around one kernel launch on
// its stream (the events are resolved by mlx_timing_read).  Inside a stream
// capture the events become event-record nodes of the graph (timing mode 2), so
// that every replay measures the kernel nodes where they run.
struct TimedLaunch {
  mlx_ctx* c; int kid; cudaStream_t st; cudaEvent_t a = nullptr, b = nullptr; bool cap = false;
  static cudaEvent_t get(mlx_ctx* c) {
    if (!c->timing.pool.empty()) { cudaEvent_t e = c->timing.pool.back(); c->timing.pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  TimedLaunch(mlx_ctx* c_, int kid_, cudaStream_t st_) : c(c_), kid(kid_), st(st_) {
    if (!c->timing.on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    cap = cs == cudaStreamCaptureStatusActive;
    if (cap && c->timing.mode != 2) return;
    a = get(c); b = get(c);
    if (cap) cudaEventRecordWithFlags(a, st, cudaEventRecordExternal);
    else cudaEventRecord(a, st);
  }
  ~TimedLaunch() {
    if (!a) return;
    if (cap) {
      cudaEventRecordWithFlags(b, st, cudaEventRecordExternal);
      c->timing.captured.push_back({kid, a, b});
    } else {
      cudaEventRecord(b, st);
      c->timing.pending.push_back({kid, a, b});
    }
  }
};

// Drop the context's cached CUDA graphs (their kernel nodes hold launch shapes and
// internal pointers that a tuning change or a new setup replaces) and bump the
// generation, so that batches holding graphs of this context recapture theirs.
inline void mlx_invalidate_graphs(mlx_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  c->graph_left.clear();
  ++c->graph_gen;
}

// internal solve mode: right-hand side is the input itself
#define MLX_STEP_PLAIN 3

static inline size_t elem_size(int precision) { return precision == MLX_FP64 ? 8 : 4; }

// ---- kernel-launch entry points (one per translation unit) ----
int mlx_basis_build(mlx_ctx* c, cudaStream_t st);
int mlx_fft_forward(mlx_ctx* c, const void* phys, cudaStream_t st);    // phys -> d_mixed
int mlx_fft_backward(mlx_ctx* c, void* phys, cudaStream_t st);         // d_mixed -> phys
int mlx_fft_fkpp(mlx_ctx* c, double gamma, cudaStream_t st);           // d_mixed -> gamma u (1 - u) (mixed)
// d_mixed -> spec; with addsrc != NULL adds alpha * addsrc in FP64 to every coefficient
int mlx_legendre_forward(mlx_ctx* c, double2* spec, cudaStream_t st,
                         const double2* addsrc = nullptr, double alpha = 0.0);
// spec -> d_mixed; planes_ready (BF16X3): d_bsb already holds spec's split planes
int mlx_legendre_backward(mlx_ctx* c, const double2* spec, cudaStream_t st, bool planes_ready = false);
int mlx_band_setup(mlx_ctx* c, cudaStream_t st);
int mlx_solve_scratch(mlx_ctx* c);                 // scratch of the lean solve variant
int mlx_seg_build(mlx_ctx* c, BandLU& f, int S, cudaStream_t st);   // segmented-solve data (S = 0: none)
int mlx_pack_lean(mlx_ctx* c, BandLU& f, int kl, const long long* d_off, int kz_fac, long long rows,
                  cudaStream_t st);                 // lean-solve records of a factor family
int mlx_lap_setup(mlx_ctx* c, cudaStream_t st);
int mlx_lap_solve(mlx_ctx* c, int family, const double2* rhs, double2* out, cudaStream_t st);
int mlx_proj_setup(mlx_ctx* c, cudaStream_t st);
int mlx_proj_solve(mlx_ctx* c, int family, const double2* rhs, double2* out, cudaStream_t st);
int mlx_vortex_prepare(mlx_ctx* c, cudaStream_t st);
int mlx_vortex_nonlinear(mlx_ctx* c, double U0, const double2* state, double2* out, cudaStream_t st);
int mlx_lp_refresh(mlx_ctx* c, cudaStream_t st);
int mlx_lp_add_source(mlx_ctx* c, double2* A, cudaStream_t st);
int mlx_tc_prepare(mlx_ctx* c, cudaStream_t st);
int mlx_tc_retile(mlx_ctx* c, int bn, cudaStream_t st);
int mlx_enqueue_step_pair(mlx_ctx* c, int kind, double c0, double2* s, double2* Ap, cudaStream_t st);
int mlx_legendre_tc_forward(mlx_ctx* c, double2* spec, cudaStream_t st);
int mlx_legendre_tc_backward(mlx_ctx* c, const double2* spec, cudaStream_t st, bool planes_ready = false);
// the backward contraction of vortex field f from its split planes in d_bsv
int mlx_legendre_tc_backward_field(mlx_ctx* c, int f, cudaStream_t st);
// allocate d_bsv (zero tails) and encode its maps (BF16X3 vortex contexts)
int mlx_tc_vortex_planes(mlx_ctx* c, cudaStream_t st);
// n FP64 values as double-float pairs (df.cuh), elementwise; dst may equal src
void mlx_to_df(const double* src, void* dst, long long n, cudaStream_t st);
// nfields = 2: both fields of a vortex state (n_spec apart) in one launch (lean
// variant only; MLX_EINVAL otherwise).  sp: where the segmented solve also writes
// the BF16x3 split planes of its output for the backward contraction; *wrote says
// whether it did (only the segmented variant does).
int mlx_band_solve(mlx_ctx* c, int step, const double2* s, const double2* A,
                   const double2* Ap, double2* out, cudaStream_t st, int nfields = 1,
                   const SplitPlanes* sp = nullptr, bool* wrote = nullptr);
// Dense BF16 GEMM on the tensor cores (gemm_tc.cu): C (+)= A * B^T, A with P in {1, 3}
// BF16 parts [P][Ma][Kp], B [Nb][Kp], both K-major; see the file for the contract.
int mlx_gemm_tc(int P, const void* A, long long Ma, const void* B, long long Nb, long long Kp, int M, int N, int K,
                float* C, int split, int* err, cudaStream_t st, const float* bias = nullptr);
int mlx_filter_fields(mlx_ctx* c, int nfields, double2* state, cudaStream_t st);   // filter.cu
int mlx_spec_axpby(mlx_ctx* c, double a, const double2* x, double b, const double2* y,
                   double2* out, cudaStream_t st, long long n = -1);
