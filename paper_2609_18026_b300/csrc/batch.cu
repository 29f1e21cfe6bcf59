// Batched uneven solves and the launch-shape autotuner (no counterpart in the
// paper: its runs are single problems).
//
// A batch groups independent contexts (uneven Nr, Nphi, Nz, ell, kinds).  One
// CUDA graph per step pair advances the whole batch, in one of two forms:
//  * persistent (default when every member qualifies: diffusion or Fisher-KPP,
//    no filter, Nphi and Nz at most 256): each phase of the time step is one
//    persistent launch over a work queue of (member, tile) items of all members
//    -- the split of the states and the backward contraction, the inverse z
//    transform, the fused phi synthesis / product / analysis, the forward z
//    transform, the forward contraction, the banded solve -- with items sorted by
//    decreasing cost and each member's own launch shapes (tiles, column width,
//    chains per warp).  The members without a nonlinear term need only the solve:
//    theirs runs on a second graph branch beside the transform phases.
//  * branches: every member's own kernel sequence on its own graph branch (fork /
//    join through events), the branches running concurrently.
// Both give each member bitwise the values of its single-context steps.
//
// The autotuner times candidate launch shapes of one context with CUDA events
// (tensor-core column-tile width for the MLX_BF16X3 contraction; chains per warp
// and warps per CTA of the banded solve), keeps the fastest, and records it in a
// text cache keyed by the context's sizes, precision and nonlinear kind.
#include "mlx_internal.cuh"

#include <stdio.h>
#include <string.h>

#include <algorithm>

// host entry points of the batched kernels (fft.cu, legendre.cu, banded.cu)
bool mlx_fft_batch_member(mlx_ctx* c, int stage, double gamma, int inst, BFftJob* job,
                          std::vector<int4>& items, std::vector<double>& cost, size_t* smem);
const void* mlx_fft_batch_kernel(int stage, bool dbl);
int mlx_fft_batch_launch(int stage, bool dbl, const BFftJob* jobs, const int4* items, int nitems, int* ctr,
                         size_t smem, int grid, cudaStream_t st);
void mlx_legendre_batch_member(mlx_ctx* c, bool fwd, int inst, double2* spec, BLegJob* job,
                               std::vector<LegTile>& items, std::vector<double>& cost);
int mlx_legendre_batch_launch(bool fwd, bool dbl, const BLegJob* jobs, const LegTile* items, int nitems,
                              int* ctr, int grid, cudaStream_t st);
const void* mlx_legendre_batch_kernel(bool fwd, bool dbl);
void mlx_band_batch_member(mlx_ctx* c, const double2* s, const double2* A, const double2* Ap, double2* out,
                           double2* Az, bool planes, std::vector<BSolvePart>& parts, bool* wrote_planes);
const void* mlx_band_batch_kernel(int kl, int variant);
int mlx_band_batch_launch(int kl, int variant, const BSolveJob* jobs, const int2* items, int nitems, int slab,
                          int wpb, int* ctr, int grid, cudaStream_t st);

namespace {

// One persistent launch: its kind, the device job and item arrays, the queue
// counters and the launch shape.
struct QLaunch {
  enum Kind { FFT, LEG, SOLVE, TC } kind;
  int stage = 0;          // FFT stage; LEG: 1 forward, 0 backward
  bool dbl = false;
  int kl = 2, variant = 0, slab = 0, wpb = 1;
  void* jobs = nullptr;
  void* items = nullptr;
  int nitems = 0, grid = 0;
  size_t smem = 0;
  int* ctr = nullptr;
  TcBatchPlan* tc = nullptr;
};

// The persistent form of one step pair: per step, the launches of the transform
// branch (in order) and of the solve branch.
struct PGraph {
  std::vector<QLaunch> xf[2];      // transform phases, then the solves of the members with a nonlinear term
  std::vector<QLaunch> lin[2];     // solves of the members without one
  cudaGraphExec_t exec = nullptr;
};

void free_launch(QLaunch& q) {
  if (q.jobs) cudaFree(q.jobs);
  if (q.items) cudaFree(q.items);
  if (q.ctr) cudaFree(q.ctr);
  if (q.tc) mlx_tc_batch_free(q.tc);
  q = QLaunch();
}

void free_pgraph(PGraph* g) {
  if (!g) return;
  for (int k = 0; k < 2; ++k) {
    for (auto& q : g->xf[k]) free_launch(q);
    for (auto& q : g->lin[k]) free_launch(q);
  }
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
}

}  // namespace

struct mlx_batch {
  std::vector<mlx_ctx*> ctxs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;
  std::map<std::vector<uintptr_t>, cudaGraphExec_t> graphs;
  std::map<std::vector<uintptr_t>, PGraph*> pgraphs;
  std::vector<unsigned long long> gens;   // members' graph generations the cached graphs were made at
  int persistent = 1;                     // 1: per-phase persistent launches when every member qualifies
  // persistent capture: the transform chain on a high-priority stream, each solve
  // group on a stream of its own (high priority for the members with a nonlinear
  // term, whose step waits on them; low for the others, which fill the gaps)
  cudaStream_t pcap = nullptr;
  std::vector<cudaStream_t> hi, lo;
  std::vector<cudaEvent_t> evs;
};

namespace {

void batch_free(mlx_batch* b) {
  if (!b) return;
  for (auto& kv : b->pgraphs) free_pgraph(kv.second);
  for (auto st : b->hi) cudaStreamDestroy(st);
  for (auto st : b->lo) cudaStreamDestroy(st);
  for (auto e : b->evs) cudaEventDestroy(e);
  if (b->pcap) cudaStreamDestroy(b->pcap);
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

int device_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

template <typename V>
int upload(const std::vector<V>& v, void** dst) {
  if (cudaMalloc(dst, sizeof(V) * (v.empty() ? 1 : v.size())) != cudaSuccess) return MLX_ECUDA;
  if (!v.empty() && cudaMemcpy(*dst, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return MLX_ECUDA;
  return MLX_OK;
}

// item indices in decreasing cost (stable: equal costs keep their order)
std::vector<int> by_cost(const std::vector<double>& cost) {
  std::vector<int> ord(cost.size());
  for (size_t t = 0; t < ord.size(); ++t) ord[t] = (int)t;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  return ord;
}
template <typename V>
std::vector<V> permute(const std::vector<V>& v, const std::vector<int>& ord) {
  std::vector<V> o(v.size());
  for (size_t t = 0; t < ord.size(); ++t) o[t] = v[ord[t]];
  return o;
}

// persistent CTAs of a queue launch: as many as fit on the GPU at once, at most
// one per `per_cta` items
int queue_grid(const void* kern, int threads, size_t smem, int nitems, int per_cta) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const long long full = (long long)per_sm * device_sms();
  const long long need = (nitems + per_cta - 1) / per_cta;
  return (int)(need < full ? (need > 0 ? need : 1) : full);
}

int new_ctr(int** ctr) {
  if (cudaMalloc(ctr, 2 * sizeof(int)) != cudaSuccess) return MLX_ECUDA;
  return cudaMemset(*ctr, 0, 2 * sizeof(int)) == cudaSuccess ? MLX_OK : MLX_ECUDA;
}

bool persistent_ok(const mlx_batch* b, const int* kinds) {
  if (!b->persistent) return false;
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    const mlx_ctx* c = b->ctxs[i];
    if (kinds[i] != MLX_NONLIN_NONE && kinds[i] != MLX_NONLIN_FKPP) return false;
    if (c->filter_on || c->nphi > 256 || c->nz > 256) return false;
    // the batched contraction forms six split products and has no expiry hook
    if (c->precision == MLX_BF16X3 && (c->tc_products != 6 || c->tc_expire)) return false;
  }
  return true;
}

// The solve launches of `members` for one step: grouped by variant (staged per
// half width, segmented per segment count and form) and by the size class of the
// per-warp slab (each group's warps are sized for its largest member), warps per
// CTA chosen for the most resident warps.  planes[i]: a segmented solve of member
// i also writes the split planes of its output (wrote[i] reports it).
int solve_launches(const std::vector<int>& members, mlx_ctx* const* ctxs,
                   const std::vector<const double2*>& sin, const std::vector<const double2*>& A,
                   const std::vector<const double2*>& Ap, const std::vector<double2*>& out,
                   const std::vector<double2*>& Az, const std::vector<char>& planes, std::vector<char>& wrote,
                   std::vector<QLaunch>& L) {
  std::map<std::vector<int>, std::vector<int>> groups;
  std::vector<BSolvePart> parts;
  for (size_t q = 0; q < members.size(); ++q) {
    const int i = members[q];
    bool w = false;
    const size_t first = parts.size();
    mlx_band_batch_member(ctxs[i], sin[i], A[i], Ap[i], out[i], Az[i], planes[i] != 0, parts, &w);
    wrote[i] = w;
    for (size_t pi = first; pi < parts.size(); ++pi) {
      int cls = 0;
      while (cls < 3 && parts[pi].slab > (16 << 10) << cls) ++cls;
      groups[{ctxs[i]->kl, parts[pi].job.variant, cls}].push_back((int)pi);
    }
  }
  for (auto& kv : groups) {
    QLaunch ql;
    ql.kind = QLaunch::SOLVE;
    ql.kl = kv.first[0];
    ql.variant = kv.first[1];
    std::vector<BSolveJob> jobs;
    std::vector<int2> items;
    std::vector<double> cost;
    int slab = 16;
    for (int q : kv.second) {
      const int j = (int)jobs.size();
      jobs.push_back(parts[q].job);
      for (size_t t = 0; t < parts[q].items.size(); ++t) {
        items.push_back(make_int2(j, parts[q].items[t].y));
        cost.push_back(parts[q].cost[t]);
      }
      if (parts[q].slab > slab) slab = parts[q].slab;
    }
    const std::vector<int> ord = by_cost(cost);
    items = permute(items, ord);
    ql.slab = slab;
    const void* kern = mlx_band_batch_kernel(ql.kl, ql.variant);
    if (!kern) return MLX_EINVAL;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
      return MLX_ECUDA;
    int best = 0;
    for (int wpb : {1, 2, 4}) {
      if ((size_t)slab * wpb > 200 * 1024) break;
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * wpb, (size_t)slab * wpb) != cudaSuccess)
        per_sm = 0;
      if (per_sm * wpb >= best) { best = per_sm * wpb; ql.wpb = wpb; }
    }
    ql.smem = (size_t)slab * ql.wpb;
    ql.nitems = (int)items.size();
    ql.grid = queue_grid(kern, 32 * ql.wpb, ql.smem, ql.nitems, ql.wpb);
    int rc = upload(jobs, &ql.jobs);
    if (!rc) rc = upload(items, &ql.items);
    if (!rc) rc = new_ctr(&ql.ctr);
    L.push_back(ql);
    if (rc) return rc;
  }
  return MLX_OK;
}

// The persistent launches of one step pair.
int build_pgraph(mlx_batch* b, const int* kinds, const double* coeffs, void* const* states, void* const* prevs,
                 PGraph* g) {
  const int n = (int)b->ctxs.size();
  mlx_ctx* const* cs = b->ctxs.data();
  std::vector<int> nl, lin;
  for (int i = 0; i < n; ++i) (kinds[i] == MLX_NONLIN_FKPP ? nl : lin).push_back(i);
  // the first step's segmented solves write the split planes of their outputs
  // (BF16X3 members with a nonlinear term): the second step's backward
  // contraction takes them instead of splitting its states again
  std::vector<char> planes(n, 0), wrote(n, 0), nowrite(n, 0), need_split(n, 1);
  for (int i : nl) planes[i] = cs[i]->precision == MLX_BF16X3;
  for (int k = 0; k < 2; ++k) {
    // step k of the pair: (s, A_prev) -> (out, A^j) as in the single-context pair
    std::vector<const double2*> sin(n), Ap(n), A(n);
    std::vector<double2*> Anew(n), out(n), Az(n, nullptr);
    for (int i = 0; i < n; ++i) {
      mlx_ctx* c = cs[i];
      sin[i] = k == 0 ? (const double2*)states[i] : c->d_spec1;
      Ap[i] = k == 0 ? (const double2*)prevs[i] : c->d_specA;
      Anew[i] = k == 0 ? c->d_specA : (double2*)prevs[i];
      out[i] = k == 0 ? c->d_spec1 : (double2*)states[i];
      A[i] = Anew[i];
      if (kinds[i] == MLX_NONLIN_NONE) {   // no A terms; A^j written as zeros
        A[i] = nullptr;
        Ap[i] = nullptr;
        Az[i] = Anew[i];
      }
    }
    std::vector<QLaunch>& X = g->xf[k];
    int rc = MLX_OK;
    // contractions of the members with a nonlinear term: BF16X3 members by the
    // tensor-core plan (chunks of kTcBatchMax), the others by the SIMT kernel
    auto contraction = [&](bool fwd) -> int {
      std::vector<mlx_ctx*> tcm;
      std::vector<double2*> tcs;
      std::vector<char> tsplit;
      for (int i : nl)
        if (cs[i]->precision == MLX_BF16X3) {
          tcm.push_back(cs[i]);
          tcs.push_back(fwd ? Anew[i] : const_cast<double2*>(sin[i]));
          tsplit.push_back(need_split[i]);
        }
      for (size_t o = 0; o < tcm.size(); o += kTcBatchMax) {
        const int cnt = (int)std::min<size_t>(kTcBatchMax, tcm.size() - o);
        QLaunch ql;
        ql.kind = QLaunch::TC;
        int r = mlx_tc_batch_plan(tcm.data() + o, cnt, fwd, tcs.data() + o, tsplit.data() + o, &ql.tc);
        if (r) return r;
        X.push_back(ql);
      }
      for (int d = 0; d < 2; ++d) {
        std::vector<BLegJob> jobs;
        std::vector<LegTile> items;
        std::vector<double> cost;
        for (int i : nl) {
          const mlx_ctx* c = cs[i];
          if (c->precision == MLX_BF16X3 || (c->precision == MLX_FP64) != (d == 1)) continue;
          BLegJob j;
          const size_t first = items.size();
          mlx_legendre_batch_member(cs[i], fwd, (int)jobs.size(), fwd ? Anew[i] : const_cast<double2*>(sin[i]), &j,
                                    items, cost);
          (void)first;
          jobs.push_back(j);
        }
        if (items.empty()) continue;
        items = permute(items, by_cost(cost));
        QLaunch ql;
        ql.kind = QLaunch::LEG;
        ql.stage = fwd ? 1 : 0;
        ql.dbl = d == 1;
        ql.nitems = (int)items.size();
        ql.grid = queue_grid(mlx_legendre_batch_kernel(fwd, ql.dbl), 256, 0, ql.nitems, 1);
        int r = upload(jobs, &ql.jobs);
        if (!r) r = upload(items, &ql.items);
        if (!r) r = new_ctr(&ql.ctr);
        X.push_back(ql);
        if (r) return r;
      }
      return MLX_OK;
    };
    if ((rc = contraction(false))) return rc;
    for (int stage = 0; stage < 3 && !rc; ++stage)
      for (int d = 0; d < 2 && !rc; ++d) {
        std::vector<BFftJob> jobs;
        std::vector<int4> items;
        std::vector<double> cost;
        size_t smem = 0;
        for (int i : nl) {
          mlx_ctx* c = cs[i];
          if ((c->precision == MLX_FP64) != (d == 1)) continue;
          BFftJob j;
          size_t sm = 0;
          if (mlx_fft_batch_member(c, stage, coeffs[i], (int)jobs.size(), &j, items, cost, &sm)) {
            jobs.push_back(j);
            if (sm > smem) smem = sm;
          }
        }
        if (items.empty()) continue;
        items = permute(items, by_cost(cost));
        QLaunch ql;
        ql.kind = QLaunch::FFT;
        ql.stage = stage;
        ql.dbl = d == 1;
        ql.smem = smem;
        ql.nitems = (int)items.size();
        ql.grid = queue_grid(mlx_fft_batch_kernel(stage, ql.dbl), 256, smem, ql.nitems, 1);
        rc = upload(jobs, &ql.jobs);
        if (!rc) rc = upload(items, &ql.items);
        if (!rc) rc = new_ctr(&ql.ctr);
        X.push_back(ql);
      }
    if (rc) return rc;
    if ((rc = contraction(true))) return rc;
    if (!nl.empty() && (rc = solve_launches(nl, cs, sin, A, Ap, out, Az, k == 0 ? planes : nowrite, wrote, X)))
      return rc;
    if (!lin.empty() && (rc = solve_launches(lin, cs, sin, A, Ap, out, Az, nowrite, wrote, g->lin[k]))) return rc;
    if (k == 0)
      for (int i : nl) need_split[i] = !wrote[i];
  }
  return MLX_OK;
}

int run_launch(const QLaunch& q, cudaStream_t st) {
  switch (q.kind) {
    case QLaunch::FFT:
      return mlx_fft_batch_launch(q.stage, q.dbl, (const BFftJob*)q.jobs, (const int4*)q.items, q.nitems, q.ctr,
                                  q.smem, q.grid, st);
    case QLaunch::LEG:
      return mlx_legendre_batch_launch(q.stage == 1, q.dbl, (const BLegJob*)q.jobs, (const LegTile*)q.items,
                                       q.nitems, q.ctr, q.grid, st);
    case QLaunch::SOLVE:
      return mlx_band_batch_launch(q.kl, q.variant, (const BSolveJob*)q.jobs, (const int2*)q.items, q.nitems,
                                   q.slab, q.wpb, q.ctr, q.grid, st);
    case QLaunch::TC:
      return mlx_tc_batch_launch(q.tc, st);
  }
  return MLX_EINVAL;
}

// Capture the pair.  Per step: the transform phases in order on the capture
// stream, then the solve groups of the members with a nonlinear term side by
// side; the solve groups of the others side by side from the start of the step.
int capture_pgraph(mlx_batch* b, PGraph* g) {
  int lo_prio = 0, hi_prio = 0;
  if (cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess) return MLX_ECUDA;
  if (!b->pcap && cudaStreamCreateWithPriority(&b->pcap, cudaStreamNonBlocking, hi_prio) != cudaSuccess)
    return MLX_ECUDA;
  size_t nhi = 0, nlo = 0;
  for (int k = 0; k < 2; ++k) {
    size_t ns = 0;
    for (const QLaunch& q : g->xf[k]) ns += q.kind == QLaunch::SOLVE;
    nhi = std::max(nhi, ns);
    nlo = std::max(nlo, g->lin[k].size());
  }
  while (b->hi.size() < nhi) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, hi_prio) != cudaSuccess) return MLX_ECUDA;
    b->hi.push_back(st);
  }
  while (b->lo.size() < nlo) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, lo_prio) != cudaSuccess) return MLX_ECUDA;
    b->lo.push_back(st);
  }
  size_t ev_i = 0;
  auto ev = [&](cudaEvent_t* e) -> int {
    if (ev_i == b->evs.size()) {
      cudaEvent_t x = nullptr;
      if (cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) return MLX_ECUDA;
      b->evs.push_back(x);
    }
    *e = b->evs[ev_i++];
    return MLX_OK;
  };
  // run `ls` side by side on `pool`, each after an event recorded on `from`; the
  // join events go to `joins`
  auto fan = [&](const std::vector<const QLaunch*>& ls, std::vector<cudaStream_t>& pool,
                 std::vector<cudaEvent_t>& joins) -> int {
    if (ls.empty()) return MLX_OK;
    cudaEvent_t f;
    int r = ev(&f);
    if (r) return r;
    if (cudaEventRecord(f, b->pcap) != cudaSuccess) return MLX_ECUDA;
    for (size_t j = 0; j < ls.size(); ++j) {
      if (cudaStreamWaitEvent(pool[j], f, 0) != cudaSuccess) return MLX_ECUDA;
      if ((r = run_launch(*ls[j], pool[j]))) return r;
      cudaEvent_t e;
      if ((r = ev(&e))) return r;
      if (cudaEventRecord(e, pool[j]) != cudaSuccess) return MLX_ECUDA;
      joins.push_back(e);
    }
    return MLX_OK;
  };
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(b->pcap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MLX_ECUDA;
  int rc = MLX_OK;
  for (int k = 0; k < 2 && !rc; ++k) {
    std::vector<cudaEvent_t> joins;
    std::vector<const QLaunch*> lin, sol;
    for (const QLaunch& q : g->lin[k]) lin.push_back(&q);
    rc = fan(lin, b->lo, joins);
    for (const QLaunch& q : g->xf[k]) {
      if (rc) break;
      if (q.kind == QLaunch::SOLVE) sol.push_back(&q);
      else rc = run_launch(q, b->pcap);
    }
    if (!rc) rc = fan(sol, b->hi, joins);
    for (cudaEvent_t e : joins)
      if (!rc && cudaStreamWaitEvent(b->pcap, e, 0) != cudaSuccess) rc = MLX_ECUDA;
  }
  cudaError_t e = cudaStreamEndCapture(b->pcap, &graph);
  if (rc || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (!rc) b->ctxs[0]->last_err = cudaGetErrorString(e);
    return rc ? rc : MLX_ECUDA;
  }
  e = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->ctxs[0]->last_err = cudaGetErrorString(e);
    return MLX_ECUDA;
  }
  return MLX_OK;
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
  // over sequential on the 64-instance workload), and the segmented solve keeps FP64
  // recurrences (the persistent launch over the 64 instances' systems: 69.2k against
  // 65.9k instance-steps/s with double-float ones)
  for (mlx_ctx* c : b->ctxs)
    if (mlx_set_tuning(c, "solve_keep_s", 0) != MLX_OK || mlx_set_tuning(c, "solve_df", 0) != MLX_OK) {
      batch_free(b);
      return MLX_ECUDA;
    }
  *out = b;
  return MLX_OK;
}

int mlx_batch_set_persistent(mlx_batch* b, int on) {
  if (!b || (on != 0 && on != 1)) return MLX_EINVAL;
  b->persistent = on;
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
      for (auto& kv : b->pgraphs) free_pgraph(kv.second);
      b->pgraphs.clear();
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
    cudaGraphExec_t exec = nullptr;
    if (persistent_ok(b, kinds)) {
      auto pit = b->pgraphs.find(key);
      if (pit == b->pgraphs.end()) {
        PGraph* g = new PGraph();
        rc = build_pgraph(b, kinds, coeffs, states, prevs, g);
        if (!rc) rc = capture_pgraph(b, g);
        if (rc) { free_pgraph(g); return rc; }
        pit = b->pgraphs.emplace(key, g).first;
      }
      exec = pit->second->exec;
    }
    auto it = b->graphs.find(key);
    if (exec) {
    } else if (it == b->graphs.end()) {
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
