// runtime.cu - the C ABI (include/fx.h) over the registry of compiled trees.
//
// Host code only: argument checks, bindings, workspace, errors, the tuning
// cache file. The kernels live in the instantiation units (inst_*.cu).
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

#include "fx/runtime.hpp"

namespace fx {

static thread_local std::string g_err;

fx_status fail(fx_status s, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

fx_status cuda_fail(cudaError_t err, const char* what) {
  return fail(FX_E_CUDA, "%s: %s (%s)", what, cudaGetErrorName(err), cudaGetErrorString(err));
}

std::vector<Entry>& registry() {
  static std::vector<Entry> r;
  return r;
}

int device_sms() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cache[dev] = n;
  return n;
}

std::string device_name() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess)
    return "unknown";
  return p.name;
}

size_t storage_bytes(fx_dtype d) {
  switch (d) {
    case FX_F32: return 4;
    case FX_F64: return 8;
    case FX_BF16:
    case FX_F16: return 2;
  }
  return 0;
}
size_t reduce_bytes(fx_dtype d) { return d == FX_F64 ? 8 : 4; }

bool inject_launch_failure() {
  const char* v = getenv("FX_INJECT");
  return v && strcmp(v, "launch_fail") == 0;
}

fx_status Workspace::ensure(size_t need, cudaStream_t st) {
  if (need <= bytes && p) return FX_OK;
  if (const char* v = getenv("FX_INJECT"); v && strcmp(v, "alloc_fail") == 0)
    return fail(FX_E_NOMEM, "workspace allocation failed (injected)");
  size_t want = need < 4096 ? 4096 : need;
  want = (want + 255) & ~size_t(255);
  if (p) {
    cudaError_t e = cudaFreeAsync(p, stream ? stream : st);
    p = nullptr;
    bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync(workspace)");
  }
  cudaError_t e = cudaMallocAsync(&p, want, st);
  if (e != cudaSuccess) {
    p = nullptr;
    return fail(FX_E_NOMEM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(p, 0, want, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(workspace)");
  bytes = want;
  stream = st;
  return FX_OK;
}

void Workspace::release() {
  if (p) {
    // The caller guarantees no launch of this object is in flight.
    cudaFree(p);
  }
  p = nullptr;
  bytes = 0;
}

// ---------------------------------------------------------------- tuning cache

static std::string cache_path() {
  const char* v = getenv("FX_TUNE_CACHE");
  return v && *v ? v : "fx_tune.json";
}

// The file is a flat JSON object {"key": "block,unroll,bps,pipeline", ...}.
static std::map<std::string, std::string> read_cache() {
  std::map<std::string, std::string> m;
  std::ifstream f(cache_path());
  if (!f) return m;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  size_t i = 0;
  auto next_str = [&](std::string& out) -> bool {
    size_t a = s.find('"', i);
    if (a == std::string::npos) return false;
    size_t b = s.find('"', a + 1);
    if (b == std::string::npos) return false;
    out = s.substr(a + 1, b - a - 1);
    i = b + 1;
    return true;
  };
  std::string k, v;
  while (next_str(k) && next_str(v)) m[k] = v;
  return m;
}

static std::mutex g_cache_mu;

bool launch_shape_ok(int block, int unroll, int bps, int pipe) {
  const bool b = block >= 64 && block <= 512 && block % 32 == 0;
  const bool u = unroll == 2 || unroll == 4 || unroll == 8;
  return b && u && bps >= 0 && bps <= 32 && pipe >= 0 && pipe <= 2;
}

bool tune_cache_get(const std::string& key, Tune& t) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  auto m = read_cache();
  auto it = m.find(key);
  if (it == m.end()) return false;
  int b = 0, u = 0, s = 0, p = 0;
  if (sscanf(it->second.c_str(), "%d,%d,%d,%d", &b, &u, &s, &p) < 3) return false;
  if (!launch_shape_ok(b, u, s, p)) return false;
  t = Tune{b, u, s, true, p};
  return true;
}

void tune_cache_put(const std::string& key, const Tune& t) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  auto m = read_cache();
  char v[64];
  snprintf(v, sizeof v, "%d,%d,%d,%d", t.block, t.unroll, t.bps, t.pipe);
  m[key] = v;
  std::ofstream f(cache_path());
  f << "{\n";
  size_t n = 0;
  for (auto& kv : m) f << "  \"" << kv.first << "\": \"" << kv.second << "\"" << (++n < m.size() ? ",\n" : "\n");
  f << "}\n";
}

}  // namespace fx

using namespace fx;

// ---------------------------------------------------------------- C ABI

extern "C" {

int fx_list_count(void) { return int(registry().size()); }

fx_status fx_list_get(int i, const char** name, fx_dtype* storage, const char** formula) {
  if (i < 0 || i >= int(registry().size())) return fail(FX_E_ARG, "index %d out of range", i);
  const Entry& e = registry()[i];
  if (name) *name = e.name;
  if (storage) *storage = e.storage;
  if (formula) *formula = e.formula;
  return FX_OK;
}

fx_status fx_expr_create(const char* name, fx_dtype storage, fx_expr** out) {
  if (!name || !out) return fail(FX_E_ARG, "null argument");
  *out = nullptr;
  if (storage < FX_F32 || storage > FX_F16) return fail(FX_E_ARG, "bad storage type %d", int(storage));
  bool known = false;
  for (const Entry& e : registry()) {
    if (strcmp(e.name, name) != 0) continue;
    known = true;
    if (e.storage != storage) continue;
    fx_expr* x = new (std::nothrow) fx_expr;
    if (!x) return fail(FX_E_NOMEM, "out of host memory");
    x->e = &e;
    for (int k = 0; k < e.n_scal; ++k) x->scal[k] = e.defaults[k];
    *out = x;
    return FX_OK;
  }
  if (known) return fail(FX_E_DTYPE, "'%s' is not compiled for storage type %d", name, int(storage));
  return fail(FX_E_NOTFOUND, "no expression named '%s'", name);
}

fx_status fx_expr_destroy(fx_expr* x) {
  if (!x) return FX_OK;
  free_batch_cache(x);
  for (auto& c : x->copy_st)
    if (c) cudaStreamDestroy(c);
  for (auto& ev : x->chunk_ev)
    if (ev) cudaEventDestroy(ev);
  x->ws.release();
  x->ws_tmp.release();
  x->ws_err.release();
  x->ws_gemm.release();
  x->ws_tick.release();
  delete x;
  return FX_OK;
}

fx_status fx_expr_info(const fx_expr* x, int* n_inputs, int* n_outputs, int* n_scalars,
                       fx_kind* kind) {
  if (!x) return fail(FX_E_ARG, "null expression");
  if (n_inputs) *n_inputs = x->e->n_in;
  if (n_outputs) *n_outputs = x->e->n_out;
  if (n_scalars) *n_scalars = x->e->n_scal;
  if (kind) *kind = x->e->kind;
  return FX_OK;
}

fx_status fx_expr_slot_name(const fx_expr* x, int slot, const char** name) {
  if (!x || !name) return fail(FX_E_ARG, "null argument");
  if (slot < 0 || slot >= x->e->n_in + x->e->n_out) return fail(FX_E_ARG, "slot %d out of range", slot);
  *name = x->e->slot_names[slot];
  return FX_OK;
}

fx_status fx_expr_slot_dtype(const fx_expr* x, int slot, fx_dtype* dtype) {
  if (!x || !dtype) return fail(FX_E_ARG, "null argument");
  const Entry& e = *x->e;
  if (slot < 0 || slot >= e.n_in + e.n_out) return fail(FX_E_ARG, "slot %d out of range", slot);
  const bool reduce_out = slot >= e.n_in && e.kind != FX_KIND_ELEMENTWISE &&
                          !(e.kind == FX_KIND_MULTI && slot == e.n_in);
  *dtype = reduce_out ? (e.storage == FX_F64 ? FX_F64 : FX_F32) : slot_dtype(e, slot);
  return FX_OK;
}

fx_status fx_expr_bind(fx_expr* x, int slot, void* dev_ptr, int64_t rows, int64_t cols, int64_t ld) {
  if (!x) return fail(FX_E_ARG, "null expression");
  const Entry& e = *x->e;
  if (slot < 0 || slot >= e.n_in + e.n_out) return fail(FX_E_ARG, "slot %d out of range", slot);
  if (rows < 0 || cols < 0) return fail(FX_E_SHAPE, "negative shape %lld x %lld", (long long)rows, (long long)cols);
  if (ld < (rows > 1 ? rows : 1)) return fail(FX_E_ARG, "ld %lld < rows %lld", (long long)ld, (long long)rows);
  if (rows * cols > 0 && !dev_ptr) return fail(FX_E_ARG, "null pointer for a non-empty buffer");
  const bool reduce_out = slot >= e.n_in && e.kind != FX_KIND_ELEMENTWISE &&
                          !(e.kind == FX_KIND_MULTI && slot == e.n_in);
  const size_t es = reduce_out ? reduce_bytes(e.storage) : storage_bytes(slot_dtype(e, slot));
  if (reinterpret_cast<uintptr_t>(dev_ptr) % es != 0)
    return fail(FX_E_ALIGN, "slot %d: pointer not aligned to its %zu-byte element", slot, es);
  Binding& b = x->b[slot];
  b.p = dev_ptr;
  b.rows = rows;
  b.cols = cols;
  b.ld = ld;
  b.bound = true;
  return FX_OK;
}

fx_status fx_expr_set_scalar(fx_expr* x, int idx, double v) {
  if (!x) return fail(FX_E_ARG, "null expression");
  if (idx < 0 || idx >= x->e->n_scal) return fail(FX_E_ARG, "scalar %d out of range", idx);
  x->scal[idx] = v;
  return FX_OK;
}

fx_status fx_expr_get_scalar(const fx_expr* x, int idx, double* v) {
  if (!x || !v) return fail(FX_E_ARG, "null argument");
  if (idx < 0 || idx >= x->e->n_scal) return fail(FX_E_ARG, "scalar %d out of range", idx);
  *v = x->scal[idx];
  return FX_OK;
}

static fx_status check_bound(const fx_expr* x, int first, int count) {
  for (int k = first; k < first + count; ++k)
    if (!x->b[k].bound) return fail(FX_E_UNBOUND, "slot %d (%s) is not bound", k, x->e->slot_names[k]);
  return FX_OK;
}

fx_status fx_eval(fx_expr* x, void* stream) {
  if (!x) return fail(FX_E_ARG, "null expression");
  FX_TRY(check_bound(x, 0, x->e->n_in + x->e->n_out));
  x->last_launches = 0;
  return x->e->eval(x, static_cast<cudaStream_t>(stream));
}

fx_status fx_eval_unfused(fx_expr* x, void* stream) {
  if (!x) return fail(FX_E_ARG, "null expression");
  FX_TRY(check_bound(x, 0, x->e->n_in + x->e->n_out));
  x->last_launches = 0;
  return x->e->eval_unfused(x, static_cast<cudaStream_t>(stream));
}

// One host<->device copy of columns [c0, c0 + nc) of slot binding b (a
// matrix of `rows` rows stored with leading dimension ld on the device and
// densely on the host), or, for a transposed slot, of rows [c0, c0 + nc).
static fx_status copy_part(const Binding& b, size_t es, int mode, void* host, int64_t c0, int64_t nc,
                           cudaMemcpyKind kind, cudaStream_t st) {
  char* dev = static_cast<char*>(b.p);
  char* h = static_cast<char*>(host);
  const size_t hpitch = size_t(b.rows) * es, dpitch = size_t(b.ld) * es;
  if (mode == 1) {  // transposed leaf: rows [c0, c0 + nc) of every column
    const size_t w = size_t(nc) * es;
    void* d = dev + size_t(c0) * es;
    void* hh = h + size_t(c0) * es;
    if (kind == cudaMemcpyHostToDevice)
      FX_CUDA(cudaMemcpy2DAsync(d, dpitch, hh, hpitch, w, size_t(b.cols), kind, st));
    else
      FX_CUDA(cudaMemcpy2DAsync(hh, hpitch, d, dpitch, w, size_t(b.cols), kind, st));
    return FX_OK;
  }
  void* d = dev + size_t(c0) * dpitch;
  void* hh = h + size_t(c0) * hpitch;
  if (dpitch == hpitch) {
    if (kind == cudaMemcpyHostToDevice)
      FX_CUDA(cudaMemcpyAsync(d, hh, hpitch * size_t(nc), kind, st));
    else
      FX_CUDA(cudaMemcpyAsync(hh, d, hpitch * size_t(nc), kind, st));
  } else if (kind == cudaMemcpyHostToDevice) {
    FX_CUDA(cudaMemcpy2DAsync(d, dpitch, hh, hpitch, hpitch, size_t(nc), kind, st));
  } else {
    FX_CUDA(cudaMemcpy2DAsync(hh, hpitch, d, dpitch, hpitch, size_t(nc), kind, st));
  }
  return FX_OK;
}

// Element-wise trees whose every input is read in one mode: the columns are
// cut into up to 8 chunks; chunk i's inputs go up on one copy stream, the
// tree runs on chunk i on the caller's stream, and chunk i's output comes
// down on a second copy stream, so the copies of neighbouring chunks
// overlap the evaluation and each other. (More upload streams do not help:
// on GB300 host-to-device copies from pinned memory top out near 211 GB/s
// whether issued on one stream or four; up and down together reach 340.)
static fx_status eval_host_pipelined(fx_expr* x, const void* const* host_in, void* const* host_out,
                                     cudaStream_t st, int64_t C, bool* done) {
  const Entry& e = *x->e;
  *done = false;
  if (e.kind != FX_KIND_ELEMENTWISE || C < 32) return FX_OK;
  for (int k = 0; k < e.n_in; ++k)
    if (e.slot_modes[k] < 0) return FX_OK;
  const size_t es = storage_bytes(e.storage);
  for (int k = 0; k < 2; ++k)
    if (!x->copy_st[k]) FX_CUDA(cudaStreamCreateWithFlags(&x->copy_st[k], cudaStreamNonBlocking));
  for (auto& ev : x->chunk_ev)
    if (!ev) FX_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaStream_t up = x->copy_st[0], down = x->copy_st[1];
  // chunks of a multiple of 16 columns, so TMA-aligned views stay aligned
  int64_t cw = ((C + 7) / 8 + 15) / 16 * 16;
  const int nch = int((C + cw - 1) / cw);
  cudaEvent_t* ev_in = x->chunk_ev;
  cudaEvent_t* ev_out = x->chunk_ev + 8;
  cudaEvent_t start = x->chunk_ev[16];
  FX_CUDA(cudaEventRecord(start, st));  // earlier work on the caller's stream comes first
  FX_CUDA(cudaStreamWaitEvent(up, start, 0));
  FX_CUDA(cudaStreamWaitEvent(down, start, 0));
  Binding saved[FX_MAX_SLOTS];
  for (int k = 0; k < FX_MAX_SLOTS; ++k) saved[k] = x->b[k];
  const int zs = e.n_in;
  fx_status status = FX_OK;
  x->last_launches = 0;
  for (int i = 0; i < nch && status == FX_OK; ++i) {
    const int64_t c0 = i * cw, nc = C - c0 < cw ? C - c0 : cw;
    for (int k = 0; k < e.n_in && status == FX_OK; ++k) {
      const Binding& b = saved[k];
      const int md = e.slot_modes[k];
      if (b.rows * b.cols == 0) continue;
      const size_t ek = storage_bytes(slot_dtype(e, k));
      if (md == 0 || md == 1) {
        status = copy_part(b, ek, md, const_cast<void*>(host_in[k]), c0, nc, cudaMemcpyHostToDevice, up);
      } else if (i == 0) {  // vectors: once, whole
        status = copy_part(b, ek, 0, const_cast<void*>(host_in[k]), 0, b.cols, cudaMemcpyHostToDevice, up);
      }
    }
    if (status != FX_OK) break;
    if (cudaEventRecord(ev_in[i], up) != cudaSuccess || cudaStreamWaitEvent(st, ev_in[i], 0) != cudaSuccess) {
      status = cuda_fail(cudaGetLastError(), "chunk events");
      break;
    }
    // views of the chunk: columns [c0, c0 + nc) of plain leaves and Z, rows
    // of transposed leaves, the matching part of each_row vectors
    for (int k = 0; k < e.n_in; ++k) {
      Binding& v = x->b[k];
      v = saved[k];
      const int md = e.slot_modes[k];
      const size_t ek = storage_bytes(slot_dtype(e, k));
      if (md == 0) {
        v.p = static_cast<char*>(v.p) + size_t(c0) * size_t(v.ld) * ek;
        v.cols = nc;
      } else if (md == 1) {
        v.p = static_cast<char*>(v.p) + size_t(c0) * ek;
        v.rows = nc;
      } else if (md == 3) {
        const int64_t stride = v.rows == 1 ? v.ld : 1;
        v.p = static_cast<char*>(v.p) + size_t(c0 * stride) * ek;
        if (v.rows == 1) v.cols = nc;
        else v.rows = nc;
      }
    }
    Binding& z = x->b[zs];
    z = saved[zs];
    z.p = static_cast<char*>(z.p) + size_t(c0) * size_t(z.ld) * es;
    z.cols = nc;
    status = e.eval(x, st);  // adds its launches to x->last_launches
    if (status != FX_OK) break;
    if (cudaEventRecord(ev_out[i], st) != cudaSuccess || cudaStreamWaitEvent(down, ev_out[i], 0) != cudaSuccess) {
      status = cuda_fail(cudaGetLastError(), "chunk events");
      break;
    }
    status = copy_part(saved[zs], es, 0, host_out[0], c0, nc, cudaMemcpyDeviceToHost, down);
  }
  for (int k = 0; k < FX_MAX_SLOTS; ++k) x->b[k] = saved[k];
  // the caller's stream resumes after the last copy down (or whatever was enqueued)
  cudaEvent_t fin = x->chunk_ev[17];
  if (cudaEventRecord(fin, down) == cudaSuccess) cudaStreamWaitEvent(st, fin, 0);
  if (cudaEventRecord(ev_in[7], up) == cudaSuccess) cudaStreamWaitEvent(st, ev_in[7], 0);
  *done = true;
  return status;
}

fx_status fx_eval_host(fx_expr* x, const void* const* host_in, void* const* host_out, void* stream) {
  if (!x || !host_in || !host_out) return fail(FX_E_ARG, "null argument");
  const Entry& e = *x->e;
  FX_TRY(check_bound(x, 0, e.n_in + e.n_out));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < e.n_in; ++k)
    if (!host_in[k] && x->b[k].rows * x->b[k].cols != 0) return fail(FX_E_ARG, "null host input %d", k);
  for (int k = 0; k < e.n_out; ++k)
    if (!host_out[k] && x->b[e.n_in + k].rows * x->b[e.n_in + k].cols != 0)
      return fail(FX_E_ARG, "null host output %d", k);
  {
    bool done = false;
    const fx_status s = eval_host_pipelined(x, host_in, host_out, st, x->b[e.n_in].cols, &done);
    if (done || s != FX_OK) return s;
  }
  for (int k = 0; k < e.n_in + e.n_out; ++k) {
    const Binding& b = x->b[k];
    const bool reduce_out = k >= e.n_in && e.kind != FX_KIND_ELEMENTWISE &&
                            !(e.kind == FX_KIND_MULTI && k == e.n_in);
    const size_t es = reduce_out ? reduce_bytes(e.storage) : storage_bytes(slot_dtype(e, k));
    const size_t width = size_t(b.rows) * es, pitch = size_t(b.ld) * es;
    if (b.rows * b.cols == 0) continue;
    if (k < e.n_in) {
      if (!host_in[k]) return fail(FX_E_ARG, "null host input %d", k);
      if (pitch == width)
        FX_CUDA(cudaMemcpyAsync(b.p, host_in[k], width * b.cols, cudaMemcpyHostToDevice, st));
      else
        FX_CUDA(cudaMemcpy2DAsync(b.p, pitch, host_in[k], width, width, b.cols, cudaMemcpyHostToDevice, st));
    }
  }
  x->last_launches = 0;
  FX_TRY(e.eval(x, st));
  for (int k = e.n_in; k < e.n_in + e.n_out; ++k) {
    const Binding& b = x->b[k];
    const bool reduce_out = e.kind != FX_KIND_ELEMENTWISE && !(e.kind == FX_KIND_MULTI && k == e.n_in);
    const size_t es = reduce_out ? reduce_bytes(e.storage) : storage_bytes(e.storage);
    const size_t width = size_t(b.rows) * es, pitch = size_t(b.ld) * es;
    if (b.rows * b.cols == 0) continue;
    void* h = host_out[k - e.n_in];
    if (!h) return fail(FX_E_ARG, "null host output %d", k - e.n_in);
    if (pitch == width)
      FX_CUDA(cudaMemcpyAsync(h, b.p, width * b.cols, cudaMemcpyDeviceToHost, st));
    else
      FX_CUDA(cudaMemcpy2DAsync(h, width, b.p, pitch, width, b.cols, cudaMemcpyDeviceToHost, st));
  }
  return FX_OK;
}

fx_status fx_eval_batch(fx_expr* x, int64_t n, const fx_batch_item* items, void* stream, int use_graph) {
  if (!x) return fail(FX_E_ARG, "null expression");
  if (n < 0 || (n > 0 && !items)) return fail(FX_E_ARG, "bad batch");
  if (!x->e->eval_batch) return fail(FX_E_UNSUPPORTED, "'%s' has no batched entry", x->e->name);
  x->last_launches = 0;
  return x->e->eval_batch(x, n, items, static_cast<cudaStream_t>(stream), use_graph);
}

fx_status fx_eval_backward(fx_expr* x, const void* grad_out, void* const* grad_ptrs, void* stream) {
  if (!x || !grad_ptrs) return fail(FX_E_ARG, "null argument");
  if (!x->e->eval_backward) return fail(FX_E_UNSUPPORTED, "'%s' has no fused backward", x->e->name);
  FX_TRY(check_bound(x, 0, x->e->n_in));
  x->last_launches = 0;
  return x->e->eval_backward(x, grad_out, grad_ptrs, static_cast<cudaStream_t>(stream));
}

fx_status fx_tune(fx_expr* x, fx_tune_mode mode, void* stream) {
  if (!x) return fail(FX_E_ARG, "null expression");
  if (mode < FX_TUNE_OFF || mode > FX_TUNE_SEARCH) return fail(FX_E_ARG, "bad tune mode");
  if (mode == FX_TUNE_OFF) {
    x->tune = Tune{};
    return FX_OK;
  }
  FX_TRY(check_bound(x, 0, x->e->n_in + x->e->n_out));
  return x->e->tune(x, int(mode), static_cast<cudaStream_t>(stream));
}

fx_status fx_tune_batch(fx_expr* x, int64_t n, const fx_batch_item* items, fx_tune_mode mode,
                        void* stream) {
  if (!x) return fail(FX_E_ARG, "null expression");
  if (mode < FX_TUNE_OFF || mode > FX_TUNE_SEARCH) return fail(FX_E_ARG, "bad tune mode");
  if (!x->e->tune_batch) return fail(FX_E_UNSUPPORTED, "'%s' has no batched entry", x->e->name);
  if (n < 0 || (n > 0 && !items)) return fail(FX_E_ARG, "bad batch");
  if (mode == FX_TUNE_OFF) {
    x->tune = Tune{};
    return FX_OK;
  }
  return x->e->tune_batch(x, int(mode), static_cast<cudaStream_t>(stream), n, items);
}

fx_status fx_expr_launch_shape(const fx_expr* x, int* block, int* unroll, int* bps,
                               int* pipeline) {
  if (!x) return fail(FX_E_ARG, "null expression");
  if (block) *block = x->tune.block;
  if (unroll) *unroll = x->tune.unroll;
  if (bps) *bps = x->tune.bps;
  if (pipeline) *pipeline = x->tune.pipe;
  return FX_OK;
}

fx_status fx_expr_set_launch_shape(fx_expr* x, int block, int unroll, int bps, int pipeline) {
  if (!x) return fail(FX_E_ARG, "null expression");
  if (!launch_shape_ok(block, unroll, bps, pipeline))
    return fail(FX_E_ARG, "bad launch shape (block %d, unroll %d, blocks/SM %d, pipeline %d)", block,
                unroll, bps, pipeline);
  x->tune = Tune{block, unroll, bps, true, pipeline};
  return FX_OK;
}

int fx_expr_last_launches(const fx_expr* x) { return x ? x->last_launches : 0; }

fx_status fx_expr_sync_status(fx_expr* x, void* stream) {
  if (!x) return fail(FX_E_ARG, "null expression");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FX_CUDA(cudaStreamSynchronize(st));
  FX_CUDA(cudaGetLastError());
  if (!x->ws_err.p) return FX_OK;
  unsigned int word = 0;
  FX_CUDA(cudaMemcpy(&word, x->ws_err.p, sizeof word, cudaMemcpyDeviceToHost));
  if (word == 0) return FX_OK;
  FX_CUDA(cudaMemset(x->ws_err.p, 0, sizeof word));
  // a block that gave up skipped its combine and left its ticket counted:
  // start the next evaluation from cleared tickets
  if (x->ws_tick.p) FX_CUDA(cudaMemset(x->ws_tick.p, 0, x->ws_tick.bytes));
  return fail(FX_E_CUDA, "a kernel of '%s' gave up a bounded wait for its bulk copies (code %u)",
              x->e->name, word);
}

const char* fx_last_error_string(void) { return g_err.c_str(); }

const char* fx_status_string(fx_status s) {
  switch (s) {
    case FX_OK: return "ok";
    case FX_E_ARG: return "bad argument";
    case FX_E_SHAPE: return "shape mismatch";
    case FX_E_DTYPE: return "storage type not compiled";
    case FX_E_ALIGN: return "misaligned pointer";
    case FX_E_UNBOUND: return "unbound slot";
    case FX_E_UNSUPPORTED: return "unsupported for this expression";
    case FX_E_CUDA: return "CUDA error";
    case FX_E_NOMEM: return "out of memory";
    case FX_E_NOTFOUND: return "no such expression";
  }
  return "unknown status";
}

}  // extern "C"
