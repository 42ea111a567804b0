// batch.cu -- batched replicas (include/hande.h, "batches"): many independent
// FCIQMC runs advanced together on one GPU.  Host code only: each replica is an
// ordinary context on its own non-blocking stream, so a replica's launches are
// exactly those of a single run and its results are bit-identical to one.  One
// batch iteration forks every replica stream from the caller's stream with an
// event, launches one captured iteration graph per replica, and joins the
// replica streams back with one event each.
#include <cuda_runtime.h>

#include <new>
#include <vector>

#include "hande.h"

struct hande_batch {
  cudaStream_t caller = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  std::vector<hande_ctx*> ctx;
};

namespace {

void release(hande_batch* b) {
  for (hande_ctx* c : b->ctx) hande_destroy(c);  // synchronises each replica stream
  for (cudaEvent_t e : b->done)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

// The caller's stream waits for every replica stream.
hande_status join(hande_batch* b) {
  const int n = (int)b->ctx.size();
  for (int r = 0; r < n; ++r) {
    if (cudaEventRecord(b->done[r], b->streams[r]) != cudaSuccess ||
        cudaStreamWaitEvent(b->caller, b->done[r], 0) != cudaSuccess) {
      cudaGetLastError();
      return HANDE_ERR_CUDA;
    }
  }
  return HANDE_OK;
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
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    release(b);
    return HANDE_ERR_CUDA;
  }
  for (int r = 0; r < n; ++r) {
    if (cudaStreamCreateWithFlags(&b->streams[r], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done[r], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      release(b);
      return HANDE_ERR_CUDA;
    }
  }
  // Replica set-up reads nothing the caller's stream may still be writing, but
  // keep it ordered after that stream all the same.
  if (cudaEventRecord(b->fork, b->caller) != cudaSuccess) {
    cudaGetLastError();
    release(b);
    return HANDE_ERR_CUDA;
  }
  for (int r = 0; r < n; ++r) {
    if (cudaStreamWaitEvent(b->streams[r], b->fork, 0) != cudaSuccess) {
      cudaGetLastError();
      release(b);
      return HANDE_ERR_CUDA;
    }
    hande_ctx* c = nullptr;
    hande_status st = hande_init_system(&sys[r], &qmc[r], allocator, b->streams[r], &c);
    if (st != HANDE_OK) {
      if (err_replica) *err_replica = r;
      release(b);
      return st;
    }
    b->ctx.push_back(c);
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
  const int n = (int)b->ctx.size();
  if (cudaEventRecord(b->fork, b->caller) != cudaSuccess) {
    cudaGetLastError();
    return HANDE_ERR_CUDA;
  }
  for (int r = 0; r < n; ++r) {
    if (cudaStreamWaitEvent(b->streams[r], b->fork, 0) != cudaSuccess) {
      cudaGetLastError();
      return HANDE_ERR_CUDA;
    }
  }
  hande_status first = HANDE_OK;
  for (int k = 0; k < n_iterations && first == HANDE_OK; ++k) {
    for (int r = 0; r < n; ++r) {
      hande_status st = hande_iterate(b->ctx[r], 1);
      if (st != HANDE_OK) {
        first = st;
        break;
      }
    }
  }
  hande_status js = join(b);
  return first != HANDE_OK ? first : js;
}

int hande_batch_size(const hande_batch* b) { return b ? (int)b->ctx.size() : 0; }

hande_ctx* hande_batch_replica(hande_batch* b, int r) {
  if (!b || r < 0 || r >= (int)b->ctx.size()) return nullptr;
  return b->ctx[r];
}

hande_status hande_batch_synchronize(hande_batch* b) {
  if (!b) return HANDE_ERR_INVALID;
  hande_status first = HANDE_OK;
  for (hande_ctx* c : b->ctx) {
    hande_status st = hande_synchronize(c);
    if (st != HANDE_OK && first == HANDE_OK) first = st;
  }
  return first;
}

void hande_batch_destroy(hande_batch* b) {
  if (b) release(b);
}

}  // extern "C"
