// runtime.hpp - host-side state behind the C ABI: the expression object,
// its device workspace, the registry of compiled instantiations, tuning
// state and error reporting.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "fx.h"

namespace fx {

struct Binding {
  void* p = nullptr;
  int64_t rows = 0, cols = 0, ld = 0;
  bool bound = false;
};

// Launch shape: threads per block, vectors per thread per step (flat and
// dim kernels), blocks per SM (0: as many as fit).
struct Tune {
  int block = 256;
  int unroll = 4;
  int bps = 0;
  bool tuned = false;
  // kernel variant: 0 the library's choice per tree, 1 copy pipelines
  // (cp.async tiles, bulk-copy flat chunks and rows), 2 register loads; for
  // the batched kernel, 1 selects 8-byte vectors per thread instead of 16
  int pipe = 0;
};

// Device workspace owned by one fx_expr: reduction partials, tickets,
// unfused intermediates, batch descriptors. Grown on demand with
// stream-ordered allocation; new bytes are zeroed (tickets start at 0).
struct Workspace {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  fx_status ensure(size_t need, cudaStream_t st);
  void release();
};

struct BatchCache;  // batch.cuh

struct Entry;

}  // namespace fx

struct fx_expr {
  const fx::Entry* e = nullptr;
  fx::Binding b[FX_MAX_SLOTS];
  double scal[FX_MAX_SCALARS] = {};
  fx::Workspace ws;
  fx::Workspace ws_tmp;  // unfused intermediates
  fx::Workspace ws_err;  // error word of bounded waits (kErrTimeout)
  fx::Workspace ws_gemm; // matrix products of a tree (fusion boundaries)
  // completion tickets of the cross-block combines, apart from the partial
  // sums: launches with different grids (tuning, the unfused baseline) lay
  // their partials out differently, and a ticket inside that area would be
  // overwritten; every launch's last block resets the tickets it used
  fx::Workspace ws_tick;
  fx::Tune tune;
  int last_launches = 0;
  fx::BatchCache* batch = nullptr;
  // fx_eval_host's copy streams and chunk events (created on first use)
  cudaStream_t copy_st[2] = {nullptr, nullptr};
  cudaEvent_t chunk_ev[2 * 8 + 2] = {};  // per chunk in / out, start, finish
};

namespace fx {

using EvalFn = fx_status (*)(fx_expr*, cudaStream_t);
using HostFn = fx_status (*)(fx_expr*, const void* const*, void* const*, cudaStream_t);
using BatchFn = fx_status (*)(fx_expr*, int64_t, const fx_batch_item*, cudaStream_t, int);
using BwdFn = fx_status (*)(fx_expr*, const void*, void* const*, cudaStream_t);
using TuneFn = fx_status (*)(fx_expr*, int, cudaStream_t);
using FreeFn = void (*)(fx_expr*);

struct Entry {
  const char* name;
  const char* formula;
  fx_dtype storage;
  int n_in, n_out, n_scal;
  fx_kind kind;
  const char* const* slot_names;
  const double* defaults;
  EvalFn eval;
  EvalFn eval_unfused;
  BatchFn eval_batch;     // may be null
  BwdFn eval_backward;    // may be null
  TuneFn tune;
  // access mode of each input slot in the normalised tree (Mode of
  // expr.cuh: 0 plain, 1 transposed, 2 each_col vector, 3 each_row vector);
  // -1 for a slot read in two modes
  const signed char* slot_modes;
  // storage type of each input slot (-1: the entry's storage type)
  const signed char* slot_dtypes;
  // autotuner of the batched entry (null when there is none)
  fx_status (*tune_batch)(fx_expr*, int, cudaStream_t, int64_t, const fx_batch_item*);
};

// Storage type of slot k of an entry (outputs: the entry's storage type;
// reduction outputs are the reduce type, see reduce_bytes).
inline fx_dtype slot_dtype(const Entry& e, int k) {
  return (k < e.n_in && e.slot_dtypes[k] >= 0) ? fx_dtype(e.slot_dtypes[k]) : e.storage;
}

std::vector<Entry>& registry();
struct Registrar {
  explicit Registrar(const Entry& e) { registry().push_back(e); }
};

// errors: thread-local message, returned status
fx_status fail(fx_status s, const char* fmt, ...);
fx_status cuda_fail(cudaError_t err, const char* what);
#define FX_CUDA(call)                                          \
  do {                                                         \
    cudaError_t fx_err_ = (call);                              \
    if (fx_err_ != cudaSuccess) return ::fx::cuda_fail(fx_err_, #call); \
  } while (0)
#define FX_TRY(call)                     \
  do {                                   \
    fx_status fx_st_ = (call);           \
    if (fx_st_ != FX_OK) return fx_st_;  \
  } while (0)

// Number of SMs of the current device (cached per device).
int device_sms();
// Name of the current device (for the tuning cache key).
std::string device_name();

size_t storage_bytes(fx_dtype d);
size_t reduce_bytes(fx_dtype d);

// Tuning cache: key -> "block,unroll,bps,pipeline"
bool launch_shape_ok(int block, int unroll, int bps, int pipe);
bool tune_cache_get(const std::string& key, Tune& t);
void tune_cache_put(const std::string& key, const Tune& t);

// Frees an expression's batch descriptors and CUDA graph (batch.cu).
void free_batch_cache(fx_expr* x);

// Test hook for host-side fault injection: FX_INJECT=launch_fail makes
// every launch helper report a failed launch without launching.
bool inject_launch_failure();

}  // namespace fx
