// batch.cu -- batched replicas (include/hande.h, "batches"): many independent
// FCIQMC runs advanced together on one GPU.
//
// Replicas that share a key width, system kind and annihilation tile form a
// group.  One batched iteration is one CUDA graph: for every group, each phase
// of the iteration (det pass, scans, spawning, scatter, annihilation, new
// diagonals, shift) is ONE launch over all its replicas; replica r's blocks
// read its parameter block from a device array, so every replica computes
// exactly what its single run would (results are independent of how many
// blocks a replica gets).  Groups run on their own graph branches.  A planner
// kernel at the start of each batched iteration divides every
// phase's block budget among the replicas in proportion to their work (list
// length, last attempt count), so replicas of very uneven sizes finish each
// phase together; the budgets are chosen by an autotuner that times whole
// batched iterations.  A replica that needs per-iteration host work (a learned
// proposal or a running time-step search) or that is out of step with the rest
// makes the batch fall back to one captured graph per replica on its own
// stream for that iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "engine.h"

using hande::BatchGroup;
using hande::Engine;

struct hande_batch {
  cudaStream_t caller = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaStream_t> streams;   // one per replica (fallback path, replica-level calls)
  std::vector<cudaEvent_t> done;
  std::vector<hande_ctx*> ctx;
  // batched graphs
  std::vector<BatchGroup> groups;
  std::vector<int> group_of;           // replica -> group
  std::vector<cudaStream_t> gs, gaux;  // per group: main chain and second branch
  std::vector<cudaEvent_t> gfork, gjoin, efork, ejoin;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::vector<int64_t> sig;            // per replica: epoch and deterministic-space state
  double scale = 0.0;                  // block budget = single-run grid x scale (0 = 2)
  int group_cap = 8;                   // replicas per group at most (0 = no limit)
  int last_failed = -1;
};

namespace {

void free_graphs(hande_batch* b) {
  for (int c = 0; c < 2; ++c)
    if (b->graph[c]) {
      cudaGraphExecDestroy(b->graph[c]);
      b->graph[c] = nullptr;
    }
}

// the groups' device arrays, streams and events
void free_groups(hande_batch* b) {
  free_graphs(b);
  if (b->caller) cudaStreamSynchronize(b->caller);
  for (auto& g : b->groups) {
    if (g.d_params) cudaFree(g.d_params);
    if (g.d_off) cudaFree(g.d_off);
  }
  for (auto* v : {&b->gfork, &b->gjoin, &b->efork, &b->ejoin})
    for (cudaEvent_t e : *v)
      if (e) cudaEventDestroy(e);
  for (auto* v : {&b->gs, &b->gaux})
    for (cudaStream_t s : *v)
      if (s) cudaStreamDestroy(s);
  b->groups.clear();
  b->group_of.clear();
  for (auto* v : {&b->gfork, &b->gjoin, &b->efork, &b->ejoin}) v->clear();
  b->gs.clear();
  b->gaux.clear();
}

void release(hande_batch* b) {
  free_groups(b);
  for (hande_ctx* c : b->ctx) hande_destroy(c);  // synchronises each replica stream
  for (cudaEvent_t e : b->done)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

bool ok(cudaError_t e) {
  if (e == cudaSuccess) return true;
  cudaGetLastError();
  return false;
}

// The caller's stream waits for every replica stream.
hande_status join(hande_batch* b) {
  const int n = (int)b->ctx.size();
  for (int r = 0; r < n; ++r) {
    if (!ok(cudaEventRecord(b->done[r], b->streams[r])) || !ok(cudaStreamWaitEvent(b->caller, b->done[r], 0)))
      return HANDE_ERR_CUDA;
  }
  return HANDE_OK;
}
// Every replica stream waits for the caller's stream.
hande_status fork_all(hande_batch* b) {
  if (!ok(cudaEventRecord(b->fork, b->caller))) return HANDE_ERR_CUDA;
  for (cudaStream_t s : b->streams)
    if (!ok(cudaStreamWaitEvent(s, b->fork, 0))) return HANDE_ERR_CUDA;
  return HANDE_OK;
}

// group key: replicas whose iterations are the same kernels with the same
// launch shapes
bool same_group(const Engine& a, const Engine& c) {
  return a.W == c.W && a.kind == c.kind && a.merge_warp == c.merge_warp && a.P.tile_cap == c.P.tile_cap &&
         a.P.seg_max == c.P.seg_max && a.P.warp_cap == c.P.warp_cap && a.merge_smem_bytes == c.merge_smem_bytes &&
         a.attempt_grid == c.attempt_grid && a.merge_grid == c.merge_grid && a.merge_warp_grid == c.merge_warp_grid;
}

// Block budgets of each group's phases: `scale` times the single run's grid
// for that phase (the planner divides them among the replicas by their work);
// a replica never gets more than 4 single-run grids, nor more list-pass blocks
// than its scan partials hold.
void set_grids(hande_batch* b) {
  const double f = b->scale > 0.0 ? b->scale : 2.0;
  for (auto& G : b->groups) {
    const Engine& E = *G.eng[0];
    const int base[hande::kPlanPhases] = {hande::kScanBlocks, E.attempt_grid, E.attempt_grid * 4,
                                          std::max(E.merge_warp_grid, 1), E.merge_grid, E.attempt_grid * 2,
                                          E.attempt_grid};
    const int by_att[hande::kPlanPhases] = {0, 1, 1, 0, 0, 0, 0};
    for (int p = 0; p < hande::kPlanPhases; ++p) {
      G.plan.budget[p] = std::max(1, (int)(base[p] * f + 0.5));
      G.plan.cap[p] = p == 0 ? hande::kScanBlocks : 4 * base[p];
      G.plan.by_attempts[p] = by_att[p];
    }
  }
  free_graphs(b);
  b->sig.clear();
}

// Groups: replicas with the same kernels and launch shapes, at most
// group_cap per group (each group is one chain of launches; several groups run
// on parallel graph branches).
hande_status regroup(hande_batch* b) {
  free_groups(b);
  const int n = (int)b->ctx.size();
  b->group_of.assign((size_t)n, -1);
  for (int r = 0; r < n; ++r) {
    Engine& E = b->ctx[r]->E;
    int g = -1;
    for (size_t k = 0; k < b->groups.size(); ++k)
      if (same_group(*b->groups[k].eng[0], E) && (b->group_cap <= 0 || (int)b->groups[k].eng.size() < b->group_cap))
        g = (int)k;
    if (g < 0) {
      b->groups.emplace_back();
      g = (int)b->groups.size() - 1;
    }
    b->groups[g].eng.push_back(&E);
    b->group_of[r] = g;
  }
  const size_t ng = b->groups.size();
  b->gs.assign(ng, nullptr);
  b->gaux.assign(ng, nullptr);
  b->gfork.assign(ng, nullptr);
  b->gjoin.assign(ng, nullptr);
  b->efork.assign(ng, nullptr);
  b->ejoin.assign(ng, nullptr);
  for (size_t k = 0; k < ng; ++k) {
    BatchGroup& G = b->groups[k];
    G.R = (int)G.eng.size();
    const Engine& E = *G.eng[0];
    bool good = ok(cudaMalloc(&G.d_params, sizeof(hande::Params) * (size_t)G.R)) &&
                ok(cudaMalloc(&G.d_off, sizeof(int) * (size_t)hande::kPlanPhases * (G.R + 1))) &&
                ok(cudaStreamCreateWithFlags(&b->gs[k], cudaStreamNonBlocking)) &&
                ok(cudaStreamCreateWithFlags(&b->gaux[k], cudaStreamNonBlocking));
    for (auto* v : {&b->gfork, &b->gjoin, &b->efork, &b->ejoin})
      good = good && ok(cudaEventCreateWithFlags(&(*v)[k], cudaEventDisableTiming));
    good = good &&
           ok(cudaFuncSetAttribute(E.ops.batch_attempt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)E.ops.attempt_smem)) &&
           ok(cudaFuncSetAttribute(E.ops.batch_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)E.merge_smem_bytes));
    if (E.merge_warp)
      good = good && ok(cudaFuncSetAttribute(E.ops.batch_merge_warp_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)E.ops.merge_warp_smem));
    if (!good) return HANDE_ERR_CUDA;
  }
  set_grids(b);
  return HANDE_OK;
}

// upload the parameter blocks and capture the batched iteration for both
// buffer parities (all replicas are in step: one parity)
bool rebuild(hande_batch* b) {
  free_graphs(b);
  for (auto& G : b->groups) {
    std::vector<hande::Params> host((size_t)G.R);
    G.max_ncore = 0;
    for (int i = 0; i < G.R; ++i) {
      host[(size_t)i] = G.eng[i]->P;
      if (G.eng[i]->core_active) G.max_ncore = std::max(G.max_ncore, G.eng[i]->P.ncore);
      else host[(size_t)i].ncore = 0;
    }
    if (!ok(cudaMemcpyAsync(G.d_params, host.data(), sizeof(hande::Params) * host.size(), cudaMemcpyHostToDevice,
                            b->caller)))
      return false;
  }
  for (int cur = 0; cur < 2; ++cur) {
    cudaGraph_t g = nullptr;
    if (!ok(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal))) return false;
    for (size_t k = 0; k < b->groups.size(); ++k) {
      BatchGroup& G = b->groups[k];
      (void)cudaEventRecord(b->gfork[k], b->cap);
      (void)cudaStreamWaitEvent(b->gs[k], b->gfork[k], 0);
      G.eng[0]->ops.iteration_batch(G, cur, b->gs[k], b->gaux[k], b->efork[k], b->ejoin[k]);
      (void)cudaEventRecord(b->gjoin[k], b->gs[k]);
      (void)cudaStreamWaitEvent(b->cap, b->gjoin[k], 0);
    }
    cudaError_t le = cudaGetLastError();
    cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
    if (le != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return false;
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (!ok(ie)) return false;
    b->graph[cur] = ex;
  }
  return true;
}

std::vector<int64_t> signature(hande_batch* b) {
  std::vector<int64_t> s;
  s.reserve(b->ctx.size() * 2);
  for (hande_ctx* c : b->ctx) {
    s.push_back(c->E.epoch);
    s.push_back(c->E.core_active ? 1 : 0);
  }
  return s;
}

// batched graphs usable for this iteration: every replica batchable and in step
bool batchable(hande_batch* b) {
  const Engine& E0 = b->ctx[0]->E;
  for (hande_ctx* c : b->ctx)
    if (!hande::engine_batchable(c->E) || c->E.cur != E0.cur || c->E.host_iter != E0.host_iter) return false;
  return true;
}

// one batched iteration through the group graphs; per-replica bookkeeping after it
hande_status batched_iteration(hande_batch* b) {
  std::vector<int64_t> s = signature(b);
  if (s != b->sig || !b->graph[0]) {
    if (!rebuild(b)) return HANDE_ERR_CUDA;
    b->sig = s;
  }
  const int cur = b->ctx[0]->E.cur;
  if (!ok(cudaGraphLaunch(b->graph[cur], b->caller))) return HANDE_ERR_CUDA;
  for (size_t r = 0; r < b->ctx.size(); ++r) {
    Engine& E = b->ctx[r]->E;
    if (hande::engine_after_iteration(E)) {
      // the deterministic space is chosen now: the replica's stream waits for
      // the iteration, the caller's stream for the selection
      if (!ok(cudaEventRecord(b->fork, b->caller)) || !ok(cudaStreamWaitEvent(b->streams[r], b->fork, 0)))
        return HANDE_ERR_CUDA;
      hande_status st = hande::engine_select_core(E);
      if (st != HANDE_OK) {
        b->last_failed = (int)r;
        return st;
      }
      if (!ok(cudaEventRecord(b->done[r], b->streams[r])) || !ok(cudaStreamWaitEvent(b->caller, b->done[r], 0)))
        return HANDE_ERR_CUDA;
    }
  }
  return HANDE_OK;
}

// one iteration replica by replica (one captured graph each, on its own stream)
hande_status replica_iteration(hande_batch* b) {
  hande_status st = fork_all(b);
  if (st != HANDE_OK) return st;
  for (size_t r = 0; r < b->ctx.size(); ++r) {
    st = hande_iterate(b->ctx[r], 1);
    if (st != HANDE_OK) {
      b->last_failed = (int)r;
      join(b);
      return st;
    }
  }
  return join(b);
}

}  // namespace

extern "C" {

hande_status hande_batch_init(const hande_system* sys, const hande_qmc* qmc, int n, const hande_allocator* allocator,
                              void* cuda_stream, hande_batch** out, int* err_replica) {
  if (err_replica) *err_replica = -1;
  if (!sys || !qmc || !out || n < 1) return HANDE_ERR_INVALID;
  *out = nullptr;
  hande_batch* b = new (std::nothrow) hande_batch;
  if (!b) return HANDE_ERR_NOMEM;
  b->caller = static_cast<cudaStream_t>(cuda_stream);
  b->streams.assign((size_t)n, nullptr);
  b->done.assign((size_t)n, nullptr);
  if (!ok(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) ||
      !ok(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking))) {
    release(b);
    return HANDE_ERR_CUDA;
  }
  for (int r = 0; r < n; ++r) {
    if (!ok(cudaStreamCreateWithFlags(&b->streams[r], cudaStreamNonBlocking)) ||
        !ok(cudaEventCreateWithFlags(&b->done[r], cudaEventDisableTiming))) {
      release(b);
      return HANDE_ERR_CUDA;
    }
  }
  // Replica set-up reads nothing the caller's stream may still be writing, but
  // keep it ordered after that stream all the same.
  if (fork_all(b) != HANDE_OK) {
    release(b);
    return HANDE_ERR_CUDA;
  }
  for (int r = 0; r < n; ++r) {
    hande_ctx* c = nullptr;
    hande_status st = hande_init_system(&sys[r], &qmc[r], allocator, b->streams[r], &c);
    if (st != HANDE_OK) {
      if (err_replica) *err_replica = r;
      release(b);
      return st;
    }
    b->ctx.push_back(c);
  }
  if (regroup(b) != HANDE_OK) {
    release(b);
    return HANDE_ERR_CUDA;
  }
  hande_status st = join(b);
  if (st != HANDE_OK) {
    release(b);
    return st;
  }
  *out = b;
  return HANDE_OK;
}

hande_status hande_batch_iterate(hande_batch* b, int n_iterations) {
  if (!b || n_iterations < 0) return HANDE_ERR_INVALID;
  b->last_failed = -1;
  // the batched graphs run on the caller's stream: order it after the replica
  // streams (replica-level calls), and the replica streams after it at the end
  hande_status st = join(b);
  if (st != HANDE_OK) return st;
  for (int k = 0; k < n_iterations; ++k) {
    st = batchable(b) ? batched_iteration(b) : replica_iteration(b);
    if (st != HANDE_OK) break;
  }
  hande_status fs = fork_all(b);
  return st != HANDE_OK ? st : fs;
}

int hande_batch_failed_replica(const hande_batch* b) { return b ? b->last_failed : -1; }

hande_status hande_batch_autotune(hande_batch* b, int iterations, double* best_scale, double* best_ms) {
  if (!b || iterations < 1) return HANDE_ERR_INVALID;
  const int n = (int)b->ctx.size();
  (void)n;
  struct Cand {
    int cap;
    double scale;
  };
  std::vector<Cand> cand;
  for (int cap : {4, 8, 16, 0})
    for (double f : {1.0, 2.0, 4.0, 8.0}) cand.push_back({cap, f});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!ok(cudaEventCreate(&e0)) || !ok(cudaEventCreate(&e1))) return HANDE_ERR_CUDA;
  double best = -1.0;
  Cand bestc = cand[0];
  hande_status st = join(b);
  for (size_t i = 0; i < cand.size() && st == HANDE_OK; ++i) {
    b->scale = cand[i].scale;
    if (b->group_cap != cand[i].cap || b->groups.empty()) {
      b->group_cap = cand[i].cap;
      if (regroup(b) != HANDE_OK) {
        st = HANDE_ERR_CUDA;
        break;
      }
    }
    set_grids(b);
    // one untimed iteration captures the graphs for this shape
    st = batchable(b) ? batched_iteration(b) : HANDE_ERR_STATE;
    if (st != HANDE_OK) break;
    (void)cudaEventRecord(e0, b->caller);
    for (int k = 0; k < iterations && st == HANDE_OK; ++k) st = batched_iteration(b);
    (void)cudaEventRecord(e1, b->caller);
    if (st != HANDE_OK || !ok(cudaEventSynchronize(e1))) break;
    float ms = 0.0f;
    (void)cudaEventElapsedTime(&ms, e0, e1);
    const double per = ms / iterations;
    if (best < 0.0 || per < best) {
      best = per;
      bestc = cand[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == HANDE_ERR_STATE) {
    // a replica needs per-iteration host work: keep the default shape
    b->scale = 0.0;
    b->group_cap = 8;
    hande_status rs = regroup(b);
    fork_all(b);
    return rs != HANDE_OK ? rs : HANDE_ERR_STATE;
  }
  b->scale = bestc.scale;
  b->group_cap = bestc.cap;
  hande_status rs = regroup(b);
  hande_status fs = fork_all(b);
  if (best_scale) *best_scale = bestc.scale;
  if (best_ms) *best_ms = best;
  if (rs != HANDE_OK) return rs;
  return st != HANDE_OK ? st : fs;
}

int hande_batch_size(const hande_batch* b) { return b ? (int)b->ctx.size() : 0; }

hande_status hande_batch_layout(const hande_batch* b, int* groups, int* group_cap) {
  if (!b) return HANDE_ERR_INVALID;
  if (groups) *groups = (int)b->groups.size();
  if (group_cap) *group_cap = b->group_cap;
  return HANDE_OK;
}

hande_ctx* hande_batch_replica(hande_batch* b, int r) {
  if (!b || r < 0 || r >= (int)b->ctx.size()) return nullptr;
  return b->ctx[r];
}

hande_status hande_batch_synchronize(hande_batch* b) {
  if (!b) return HANDE_ERR_INVALID;
  if (!ok(cudaStreamSynchronize(b->caller))) return HANDE_ERR_CUDA;
  hande_status first = HANDE_OK;
  b->last_failed = -1;
  for (size_t r = 0; r < b->ctx.size(); ++r) {
    hande_status st = hande_synchronize(b->ctx[r]);
    if (st != HANDE_OK && first == HANDE_OK) {
      first = st;
      b->last_failed = (int)r;
    }
  }
  return first;
}

void hande_batch_destroy(hande_batch* b) {
  if (b) release(b);
}

}  // extern "C"
