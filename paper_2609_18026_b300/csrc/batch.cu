// Batched uneven solves and the launch-shape autotuner (no counterpart in the
// paper: its runs are single problems).
//
// A batch groups independent contexts (uneven Nr, Nphi, Nz, ell, kinds).  One
// CUDA graph holds, for every instance, the two-AB-CN-step sequence on its own
// branch (fork/join through events), so a single graph launch advances the whole
// batch and the instances' kernels run concurrently on the GPU.
//
// The autotuner times candidate launch shapes of one context with CUDA events
// (tensor-core column-tile width for the MLX_BF16X3 contraction; chains per warp
// and warps per CTA of the banded solve), keeps the fastest, and records it in a
// text cache keyed by the context's sizes, precision and nonlinear kind.
#include "mlx_internal.cuh"

#include <stdio.h>
#include <string.h>

struct mlx_batch {
  std::vector<mlx_ctx*> ctxs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;
  std::map<std::vector<uintptr_t>, cudaGraphExec_t> graphs;
  std::vector<unsigned long long> gens;   // members' graph generations the cached graphs were made at
};

namespace {

void batch_free(mlx_batch* b) {
  if (!b) return;
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

bool valid_kind(int k) { return k == MLX_NONLIN_NONE || k == MLX_NONLIN_FKPP || k == MLX_NONLIN_VORTEX; }

std::string tune_key(const mlx_ctx* c, int kind) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%d %d %d %d %d %d %d %d %d", c->nr, c->nphi, c->nz, c->nc, c->M, c->Kz,
           c->precision, kind, c->kl);
  return std::string(buf);
}

}  // namespace

extern "C" {

int mlx_batch_create(mlx_ctx* const* ctxs, int n, mlx_batch** out) {
  if (!out) return MLX_EINVAL;
  *out = nullptr;
  if (!ctxs || n <= 0) return MLX_EINVAL;
  mlx_batch* b = new mlx_batch();
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) { batch_free(b); return MLX_EINVAL; }
    b->ctxs.push_back(ctxs[i]);
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      batch_free(b);
      return MLX_ECUDA;
    }
    b->streams.push_back(s);
    b->joins.push_back(e);
  }
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    batch_free(b);
    return MLX_ECUDA;
  }
  // instances run side by side: the staged solve drops its shared-memory copy of s
  // (smaller CTAs co-reside with other instances' kernels; measured 2.1x -> 2.9x
  // over sequential on the 64-instance workload)
  for (mlx_ctx* c : b->ctxs) {
    if (mlx_set_tuning(c, "solve_keep_s", 0) != MLX_OK) { batch_free(b); return MLX_ECUDA; }
    // the segmented solve's CTAs (up to ~200 KB of shared memory) leave no room
    // for the other members' kernels: 32.9k against 38.3k instance-steps/s
    if (mlx_set_tuning(c, "solve_seg", 0) != MLX_OK) { batch_free(b); return MLX_ECUDA; }
  }
  *out = b;
  return MLX_OK;
}

int mlx_batch_destroy(mlx_batch* b) {
  if (!b) return MLX_EINVAL;
  batch_free(b);
  return MLX_OK;
}

int mlx_batch_advance(mlx_batch* b, const int* kinds, const double* coeffs, void* const* states,
                      void* const* prevs, int nsteps, int start, mlx_stream stream) {
  if (!b || !kinds || !coeffs || !states || !prevs || nsteps < 0) return MLX_EINVAL;
  const int n = (int)b->ctxs.size();
  for (int i = 0; i < n; ++i) {
    mlx_ctx* c = b->ctxs[i];
    if (!valid_kind(kinds[i]) || !states[i] || !prevs[i] || states[i] == prevs[i]) return MLX_EINVAL;
    if (!c->implicit_ready) return MLX_ESTATE;
    if (kinds[i] == MLX_NONLIN_VORTEX && !c->vortex_ready) return MLX_ESTATE;
  }
  if (nsteps == 0) return MLX_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if (start) {
    // Richardson start of every instance (one step each), then the rest
    for (int i = 0; i < n; ++i)
      if ((rc = mlx_advance(b->ctxs[i], kinds[i], &coeffs[i], 1, states[i], prevs[i], 1, 1, stream))) return rc;
    --nsteps;
  }
  const int pairs = nsteps / 2;
  if (pairs > 0) {
    // a member whose launch shapes or setup changed since the graphs were
    // captured (its generation moved) invalidates them: their kernel nodes may
    // hold buffers that member has since replaced
    std::vector<unsigned long long> gens(n);
    for (int i = 0; i < n; ++i) gens[i] = b->ctxs[i]->graph_gen;
    if (gens != b->gens) {
      for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
      b->graphs.clear();
      b->gens = gens;
    }
    std::vector<uintptr_t> key;
    for (int i = 0; i < n; ++i) {
      key.push_back((uintptr_t)states[i]);
      key.push_back((uintptr_t)prevs[i]);
      key.push_back((uintptr_t)kinds[i]);
      uint64_t bits;
      memcpy(&bits, &coeffs[i], sizeof(bits));
      key.push_back((uintptr_t)bits);
    }
    auto it = b->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it == b->graphs.end()) {
      cudaGraph_t g = nullptr;
      mlx_ctx* c0 = b->ctxs[0];
      MLX_CUDA_TRY(c0, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
      rc = MLX_OK;
      if (cudaEventRecord(b->fork, b->cap) != cudaSuccess) rc = MLX_ECUDA;
      for (int i = 0; i < n && !rc; ++i) {
        if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) { rc = MLX_ECUDA; break; }
        rc = mlx_enqueue_step_pair(b->ctxs[i], kinds[i], coeffs[i], (double2*)states[i], (double2*)prevs[i],
                                   b->streams[i]);
        if (rc) break;
        if (cudaEventRecord(b->joins[i], b->streams[i]) != cudaSuccess ||
            cudaStreamWaitEvent(b->cap, b->joins[i], 0) != cudaSuccess)
          rc = MLX_ECUDA;
      }
      cudaError_t e = cudaStreamEndCapture(b->cap, &g);
      if (rc) { if (g) cudaGraphDestroy(g); return rc; }
      if (e != cudaSuccess) { c0->last_err = cudaGetErrorString(e); return MLX_ECUDA; }
      e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { c0->last_err = cudaGetErrorString(e); return MLX_ECUDA; }
      b->graphs[key] = exec;
    } else {
      exec = it->second;
    }
    for (int p = 0; p < pairs; ++p) MLX_CUDA_TRY(b->ctxs[0], cudaGraphLaunch(exec, st));
  }
  if (nsteps % 2)
    for (int i = 0; i < n; ++i)
      if ((rc = mlx_advance(b->ctxs[i], kinds[i], &coeffs[i], 1, states[i], prevs[i], 1, 0, stream))) return rc;
  return MLX_OK;
}

int mlx_autotune(mlx_ctx* c, int kind, const double* coeffs, int ncoeffs, const char* cache_path,
                 int* chosen, mlx_stream stream) {
  if (!c || !valid_kind(kind)) return MLX_EINVAL;
  if ((kind != MLX_NONLIN_NONE) && (!coeffs || ncoeffs < 1)) return MLX_EINVAL;
  if (!c->implicit_ready) return MLX_ESTATE;
  if (kind == MLX_NONLIN_VORTEX && !c->vortex_ready) return MLX_ESTATE;
  const std::string key = tune_key(c, kind);
  // solve variant encoding: cpw = 0 segmented (half width 2), cpw = 2 lean, else
  // staged (cpw chains per warp, wpb warps per CTA)
  int bn = c->tc_bn;
  auto variant = [&](int* cp, int* wp) {
    const bool seg = c->kl == 2 && c->solve_seg && c->lu_half.seg;
    *cp = c->solve_direct == 2 ? 2 : (seg ? 0 : c->solve_cpw);
    *wp = (c->solve_direct == 2 || seg) ? 0 : c->solve_wpb;
  };
  int cpw, wpb;
  variant(&cpw, &wpb);
  bool found = false;
  if (cache_path) {
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char line[512];
      while (fgets(line, sizeof(line), f)) {
        char* bar = strchr(line, '|');
        if (!bar) continue;
        *bar = 0;
        if (key == std::string(line)) {
          int a, b2, d;
          if (sscanf(bar + 1, "%d %d %d", &a, &b2, &d) == 3) { bn = a; cpw = b2; wpb = d; found = true; }
        }
      }
      fclose(f);
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const double c0 = coeffs ? coeffs[0] : 0.0;
  auto apply = [&](int bn_, int cpw_, int wpb_) -> int {
    int rc = MLX_OK;
    if (c->precision == MLX_BF16X3 && bn_ != c->tc_bn) rc = mlx_set_tuning(c, "tc_bn", bn_);
    if (cpw_ == 2) return rc ? rc : mlx_set_tuning(c, "solve_direct", 2);
    if (!rc) rc = mlx_set_tuning(c, "solve_direct", 0);
    if (!rc && c->kl == 2) rc = mlx_set_tuning(c, "solve_seg", cpw_ == 0 ? 8 : 0);
    if (cpw_ == 0) return rc;
    if (!rc) rc = mlx_set_tuning(c, "solve_cpw", cpw_);
    if (!rc) rc = mlx_set_tuning(c, "solve_wpb", wpb_);
    return rc;
  };
  if (!found) {
    // time a candidate on the context's temporaries (state and A_prev stand-ins)
    const int nf = kind == MLX_NONLIN_VORTEX ? 2 : 1;
    double2* s = c->d_spec2;
    double2* ap = c->d_spec3;
    MLX_CUDA_TRY(c, cudaMemsetAsync(s, 0, sizeof(double2) * c->n_spec * nf, st));
    MLX_CUDA_TRY(c, cudaMemsetAsync(ap, 0, sizeof(double2) * c->n_spec * nf, st));
    cudaEvent_t e0, e1;
    MLX_CUDA_TRY(c, cudaEventCreate(&e0));
    MLX_CUDA_TRY(c, cudaEventCreate(&e1));
    auto time_it = [&](float* ms) -> int {
      int rc;
      for (int w = 0; w < 2; ++w)
        if ((rc = mlx_enqueue_step_pair(c, kind, c0, s, ap, st))) return rc;
      cudaEventRecord(e0, st);
      for (int w = 0; w < 5; ++w)
        if ((rc = mlx_enqueue_step_pair(c, kind, c0, s, ap, st))) return rc;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return MLX_ECUDA;
      cudaEventElapsedTime(ms, e0, e1);
      return MLX_OK;
    };
    int rc = MLX_OK;
    float best = 1e30f;
    // 1. column tile of the tensor-core contraction
    if (c->precision == MLX_BF16X3) {
      const int ncol = 2 * c->K;
      const int cands[] = {32, 48, 64, 96, 128, 176, 256};
      int best_bn = c->tc_bn;
      for (int cb : cands) {
        if (cb > ((ncol + 15) / 16) * 16 && cb != 32) continue;
        if ((rc = apply(cb, cpw, wpb))) break;
        float ms = 0.f;
        if ((rc = time_it(&ms))) break;
        if (ms < best) { best = ms; best_bn = c->tc_bn; }
      }
      bn = best_bn;
    }
    // 2. banded-solve variant and launch shape
    if (!rc) {
      const int shapes[][2] = {{4, 1}, {8, 1}, {8, 4}, {16, 1}, {32, 1}, {0, 0}, {2, 0}};
      best = 1e30f;
      int bc = cpw, bw = wpb;
      for (auto& sh : shapes) {
        if (sh[0] == 0 && c->kl != 2) continue;       // the segmented solve serves half width 2 only
        if ((rc = apply(bn, sh[0], sh[1]))) break;
        float ms = 0.f;
        if ((rc = time_it(&ms))) break;
        if (ms < best) { best = ms; bc = sh[0]; bw = sh[1]; }
      }
      cpw = bc;
      wpb = bw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (cache_path) {
      FILE* f = fopen(cache_path, "a");
      if (f) {
        fprintf(f, "%s|%d %d %d\n", key.c_str(), bn, cpw, wpb);
        fclose(f);
      }
    }
  }
  int rc = apply(bn, cpw, wpb);
  if (rc) return rc;
  if (chosen) {
    chosen[0] = c->tc_bn;
    variant(&chosen[1], &chosen[2]);
    chosen[3] = found;
  }
  return MLX_OK;
}

}  // extern "C"
