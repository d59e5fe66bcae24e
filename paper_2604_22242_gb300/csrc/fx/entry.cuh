// entry.cuh - turns an expression definition into registry entries, one per
// storage type: fused eval, unfused eval, backward, batch and tuning.
//
// A definition is a struct with
//   name, formula (S-expression), slots[] (input then output names),
//   n_in, n_out, n_scal, defaults[] (scalar values), kind (fx_kind),
//   dtypes (bit mask over fx_dtype), differentiable, batchable,
//   template <class T> static auto build(const double* s)
// where build returns the tree over leaves in<K, T>() with scalars s[i].
#pragma once

#include <chrono>
#include <cmath>

#include "batch.cuh"
#include "gemm.cuh"
#include "unfused.cuh"

namespace fx {

constexpr unsigned dmask(fx_dtype d) { return 1u << unsigned(d); }
constexpr unsigned ALL_DTYPES = dmask(FX_F32) | dmask(FX_F64) | dmask(FX_BF16) | dmask(FX_F16);

// Autotuner: times candidate launch shapes on the bound buffers with CUDA
// events and keeps the fastest; the choice is cached per (expression,
// storage, shape class, device).
inline std::string tune_key(const fx_expr* x) {
  int64_t R = x->b[0].rows, C = x->b[0].cols;
  auto lg = [](int64_t v) { int k = 0; while ((int64_t(1) << k) < v) ++k; return k; };
  char buf[256];
  snprintf(buf, sizeof buf, "%s|%d|%d|%d|%s", x->e->name, int(x->e->storage), lg(R), lg(C),
           device_name().c_str());
  return buf;
}

inline fx_status run_tune(fx_expr* x, int mode, cudaStream_t st, EvalFn ev, int npipe) {
  const std::string key = tune_key(x);
  if (mode == FX_TUNE_CACHE) {
    Tune t;
    if (tune_cache_get(key, t)) x->tune = t;
    return FX_OK;
  }
  static const int blocks[] = {128, 256, 512};
  static const int unrolls[] = {2, 4, 8};
  static const int bpss[] = {0, 2, 4};
  cudaEvent_t a, b;
  FX_CUDA(cudaEventCreate(&a));
  FX_CUDA(cudaEventCreate(&b));
  Tune best{};
  float best_ms = 1e30f;
  fx_status status = FX_OK;
  // the library default is timed first; a candidate replaces the best so far
  // only when it is at least 1% faster, so timing noise does not move a tree
  // off a shape that is as good as any
  auto trial = [&](const Tune& t) {
    x->tune = t;
    for (int w = 0; w < 2 && status == FX_OK; ++w) status = ev(x, st);
    if (status != FX_OK) return;
    cudaEventRecord(a, st);
    for (int it = 0; it < 5 && status == FX_OK; ++it) status = ev(x, st);
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) status = cuda_fail(cudaGetLastError(), "tune");
    if (status != FX_OK) return;
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best_ms * 0.99f) {
      best_ms = ms;
      best = t;
    }
  };
  trial(Tune{256, 4, 0, true, 0});
  for (int pi = 0; pi < npipe && status == FX_OK; ++pi)
    for (int bl : blocks)
      for (int un : unrolls)
        for (int bp : bpss)
          if (status == FX_OK) trial(Tune{bl, un, bp, true, pi});
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (status != FX_OK) {
    x->tune = Tune{};
    return status;
  }
  x->tune = best;
  tune_cache_put(key, best);
  return FX_OK;
}

// Access mode of every input slot of a leaf list (-1: read in two modes).
// Access mode and storage type of every input slot of a leaf list (mode
// -1: read in two modes; type -1: not a leaf of the list).
template <class LL, bool ALL_MIXED = false> struct SlotModes {
  signed char m[FX_MAX_SLOTS];
  signed char dt[FX_MAX_SLOTS];
  constexpr SlotModes() : m{}, dt{} {
    for (int k = 0; k < FX_MAX_SLOTS; ++k) {
      m[k] = -2;
      dt[k] = -1;
    }
    fill<0>();
    for (int k = 0; k < FX_MAX_SLOTS; ++k)
      if (m[k] == -2 || ALL_MIXED) m[k] = ALL_MIXED ? -1 : 0;
  }
  template <int I> constexpr void fill() {
    if constexpr (I < tl_size<LL>::value) {
      using L = typename tl_at<LL, I>::type;
      const signed char md = static_cast<signed char>(L::mode);
      m[L::slot] = (m[L::slot] == -2 || m[L::slot] == md) ? md : static_cast<signed char>(-1);
      dt[L::slot] = static_cast<signed char>(dtype_of<typename L::elem>::value);
      fill<I + 1>();
    }
  }
};

// Batch autotuner: the same search over the batched kernel's launch shapes
// (threads per block 256 / 512, 2 / 3 / 4 stages, blocks per SM, vector
// width 16 or 8 bytes as pipeline 0 or 1), timed on the given items without
// graph capture; cached under the batch size.
using BatchRunFn = fx_status (*)(fx_expr*, int64_t, const fx_batch_item*, cudaStream_t, int);
inline fx_status run_tune_batch(fx_expr* x, int mode, cudaStream_t st, int64_t n,
                                const fx_batch_item* items, BatchRunFn run) {
  const std::string key = "batch|" + tune_key(x) + "|" + std::to_string(n);
  if (mode == FX_TUNE_CACHE) {
    Tune t;
    if (tune_cache_get(key, t)) x->tune = t;
    return FX_OK;
  }
  static const int blocks[] = {256, 512};
  static const int unrolls[] = {2, 4, 8};
  static const int bpss[] = {0, 1, 2};
  static const int widths[] = {0, 1};
  cudaEvent_t a, b;
  FX_CUDA(cudaEventCreate(&a));
  FX_CUDA(cudaEventCreate(&b));
  Tune best{};
  float best_ms = 1e30f;
  fx_status status = FX_OK;
  for (int vw : widths)
  for (int bl : blocks)
    for (int un : unrolls)
      for (int bp : bpss) {
        x->tune = Tune{bl, un, bp, true, vw};
        for (int w = 0; w < 2 && status == FX_OK; ++w) status = run(x, n, items, st, 0);
        if (status != FX_OK) break;
        cudaEventRecord(a, st);
        for (int it = 0; it < 3 && status == FX_OK; ++it) status = run(x, n, items, st, 0);
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) status = cuda_fail(cudaGetLastError(), "tune");
        if (status != FX_OK) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) {
          best_ms = ms;
          best = x->tune;
        }
      }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (status != FX_OK) {
    x->tune = Tune{};
    return status;
  }
  x->tune = best;
  tune_cache_put(key, best);
  return FX_OK;
}

template <class Def, class T> struct Inst {
  static auto root(const fx_expr* x) { return normalize(Def::template build<T>(x->scal)); }
  using Root = std::decay_t<decltype(normalize(Def::template build<T>(nullptr)))>;
  static constexpr bool prods = has_prod_any<Root>::value;
  static fx_status eval(fx_expr* x, cudaStream_t st) {
    if constexpr (prods) return run_with_prods<T, Def::n_in>(x, root(x), Def::kind, st, false);
    else return run_root<T>(run_of(x, st), root(x), Def::kind);
  }
  static fx_status unfused(fx_expr* x, cudaStream_t st) {
    if constexpr (prods) return run_with_prods<T, Def::n_in>(x, root(x), Def::kind, st, true);
    else return run_unfused<T>(x, root(x), Def::kind, st);
  }
  static fx_status backward(fx_expr* x, const void* g, void* const* gp, cudaStream_t st) {
    if constexpr (Def::differentiable && !prods) return run_backward<T>(x, root(x), g, gp, st);
    else return fail(FX_E_UNSUPPORTED, "no fused backward");
  }
  static fx_status batch(fx_expr* x, int64_t n, const fx_batch_item* it, cudaStream_t st, int g) {
    if constexpr (Def::batchable && !prods) return run_batch<T, Def::n_in, Def::kind>(x, root(x), n, it, st, g);
    else return fail(FX_E_UNSUPPORTED, "no batched entry");
  }
  // The search times every kernel variant (pipeline 0, 1, 2) with every
  // block, unroll and residency choice.
  static fx_status tune(fx_expr* x, int mode, cudaStream_t st) {
    return run_tune(x, mode, st, &eval, 3);
  }
  static fx_status tune_batch(fx_expr* x, int mode, cudaStream_t st, int64_t n,
                              const fx_batch_item* items) {
    if constexpr (Def::batchable && !prods) return run_tune_batch(x, mode, st, n, items, &batch);
    else return fail(FX_E_UNSUPPORTED, "no batched entry");
  }
  // input slots of trees with products are consumed by GEMMs: mode -1
  // (no column-chunked host pipeline)
  static constexpr SlotModes<leaves_t<typename root_of<typename Lift<Root, T, Def::n_in>::type>::inner>,
                             prods> modes{};
  static Entry entry() {
    return Entry{Def::name, Def::formula, dtype_of<T>::value, Def::n_in, Def::n_out, Def::n_scal,
                 fx_kind(Def::kind), Def::slots, Def::defaults, &eval, &unfused,
                 Def::batchable ? &batch : nullptr, Def::differentiable ? &backward : nullptr,
                 &tune, modes.m, modes.dt, Def::batchable && !prods ? &tune_batch : nullptr};
  }
};

template <class Def> struct Register {
  Register() {
    if constexpr ((Def::dtypes & dmask(FX_F32)) != 0) registry().push_back(Inst<Def, float>::entry());
    if constexpr ((Def::dtypes & dmask(FX_F64)) != 0) registry().push_back(Inst<Def, double>::entry());
    if constexpr ((Def::dtypes & dmask(FX_BF16)) != 0) registry().push_back(Inst<Def, bf16>::entry());
    if constexpr ((Def::dtypes & dmask(FX_F16)) != 0) registry().push_back(Inst<Def, f16>::entry());
  }
};

}  // namespace fx

#define FX_REGISTER(Def) static ::fx::Register<Def> fx_register_##Def;
