// engine.h -- host-side state of one FCIQMC context and the per-key-width
// kernel launchers (implemented in inst_w*.cu, dispatched from host.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/hande.h"
#include "kernels.cuh"

namespace hande {

struct Engine;
struct Learner;   // learned excitation proposal (learn.cu)

// Replicas of one batch that share a key width, system kind and annihilation
// tile: each phase of their iteration is one launch over a grid (CTAs per
// replica, replicas) with the replicas' parameter blocks in device memory.
struct BatchGroup {
  std::vector<Engine*> eng;
  Params* d_params = nullptr;   // [R] parameter blocks (device)
  int* d_off = nullptr;         // [kPlanPhases][R + 1] first block of each replica (device, planner)
  int R = 0;
  int max_ncore = 0;
  // block budgets of the phases (list pass, spawning, scatter, warp merge,
  // block merge, copy, diagonals), divided among the replicas by the planner
  Plan plan{};
};

// launchers for one (key width, system kind) pair
struct Ops {
  void (*iteration)(Engine& E, int cur, bool core, cudaStream_t s, cudaEvent_t* ev);
  void (*iteration_batch)(BatchGroup& G, int cur, cudaStream_t s, cudaStream_t aux, cudaEvent_t fork,
                          cudaEvent_t join);
  // batched kernels (for shared-memory attributes and occupancy)
  const void* batch_attempt_kernel;
  const void* batch_merge_kernel;
  const void* batch_merge_warp_kernel;
  void (*hdiag)(Engine& E, int cur, int64_t n, cudaStream_t s);
  void (*eref)(Engine& E, cudaStream_t s);
  void (*csr_count)(Engine& E, int32_t* rowcnt, cudaStream_t s);
  void (*csr_fill)(Engine& E, cudaStream_t s);
  void (*sel_gather)(Engine& E, int cur, uint64_t* core_key, int64_t ncore, cudaStream_t s);
  void (*core_hash)(Engine& E, uint32_t* table, cudaStream_t s);
  void (*check_keys)(Engine& E, const uint64_t* aos, int64_t n, unsigned* out, cudaStream_t s);
  // array of structures <-> structure of arrays with word stride `stride`
  void (*keys_to_soa)(Engine& E, const uint64_t* aos, uint64_t* soa, int64_t n, int64_t stride, cudaStream_t s);
  void (*keys_to_aos)(Engine& E, const uint64_t* soa, uint64_t* aos, int64_t n, int64_t stride, cudaStream_t s);
  // core flags of the list from the core keys (P.core_key, P.ncore); a core key
  // missing from the list sets bit 0 of *missing
  void (*core_mark)(Engine& E, int cur, unsigned* missing, cudaStream_t s);
  void (*sel_hist)(Engine& E, int cur, int shift, uint64_t mask, uint64_t prefix, unsigned long long* hist,
                   cudaStream_t s);
  void (*sel_flags)(Engine& E, int cur, uint64_t vstar, int64_t need_eq, int stage, cudaStream_t s);
  size_t (*merge_smem)(int tc, int sm);
  const void* merge_kernel;
  const void* merge_warp_kernel;
  size_t merge_warp_smem;
  int merge_warp_main, merge_warp_new;   // warp tile: segment entries, staged new keys
  const void* attempt_kernel;
  size_t attempt_smem;
};

constexpr int kPhases = 10;   // timed phases of one iteration

Ops ops_w1(int kind);
Ops ops_w2(int kind);
Ops ops_w8(int kind);

struct Engine {
  Params P{};            // device pointers and run constants (kernel argument)
  Ops ops{};
  int W = 1, kind = 0, nalpha = 0, nbeta = 0;
  int device = 0;                     // CUDA device the context was created on
  cudaStream_t stream = nullptr;      // caller's stream
  cudaStream_t cap_stream = nullptr;  // private stream used for graph capture
  cudaStream_t aux_stream = nullptr;  // second branch of a captured iteration
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  hande_allocator alloc{};
  bool has_alloc = false;
  std::vector<std::pair<void*, size_t>> blocks;
  int merge_grid = 0;
  bool merge_warp = false;   // annihilation with one warp per bucket
  int merge_warp_grid = 0;
  size_t merge_smem_bytes = 0;
  int attempt_grid = 0;
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int cur = 0;
  int64_t host_iter = 0;
  int64_t epoch = 0;   // incremented whenever the parameter block changes (graphs dropped)
  int64_t fetched = 0;
  bool core_active = false;
  int core_size = 0, core_start = 0;
  // core storage (device)
  uint64_t* core_key = nullptr;
  int64_t* core_rowptr = nullptr;
  int32_t* core_col = nullptr;
  double* core_val = nullptr;
  int64_t nnz_cap = 0, ncore_cap = 0;
  uint32_t* core_table = nullptr;   // core membership hash table
  unsigned* check_word = nullptr;   // result word of the walker-list checks
  int64_t core_table_cap = 0;
  double e_ref = 0.0;
  // UEG proposal table (excit_gen = 1): cumulative weights on the device and
  // the drawable mask (host and device); the learned proposal, if attached
  uint32_t* ptab = nullptr;
  uint8_t* pmask_dev = nullptr;
  std::vector<uint8_t> pmask;
  Learner* learn = nullptr;
  // time-step search: requested, still running (until the population first
  // exceeds the target); host copies of the tau-dependent heat-bath amounts
  bool tau_search_on = false, tau_searching = false;
  double inv_double = 0.0;
  std::vector<double> hb_v, hb_inv;
  std::vector<ulonglong2> hb_ent;
  bool failed = false;
  unsigned err_bits = 0;
  std::string err;
};

// learned proposal (learn.cu)
void proposal_init(Engine& E, const int4* kvec, const int16_t* klookup, int nmax, int side);
void proposal_set(Engine& E, const uint32_t* q);
void proposal_get(Engine& E, uint32_t* q);
void learner_attach(Engine& E, const hande_learning& in);
void learner_release(Engine& E);
int64_t learner_nparam(const Engine& E);
void learner_params(Engine& E, float* get, const float* set);
void learner_gradients(Engine& E, const int32_t* rows, const int32_t* tgt, const float* w, int n, float* grads,
                       double* loss);
void learner_probabilities(Engine& E, const int32_t* rows, int n, float* probs);
void learner_refresh(Engine& E);
void learner_step(Engine& E);
bool learner_due(const Engine& E);
// batches (host.cu)
bool engine_batchable(const Engine& E);
bool engine_after_iteration(Engine& E);
hande_status engine_select_core(Engine& E);

}  // namespace hande

// the opaque context of the C ABI
struct hande_ctx {
  hande::Engine E;
};
