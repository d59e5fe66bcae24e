// launch.cuh - host-side drivers: shape checks, choice of kernel family and
// vector width, grid sizing, workspace layout, the unfused baseline and the
// autotuner. Everything here is templated on the (normalised) tree type.
#pragma once

#include <cmath>
#include <string>


#include "tmatile.cuh"
#include "runtime.hpp"

namespace fx {

inline bool aligned(const void* p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

// What one evaluation sees: bindings (inputs, then outputs), launch shape,
// the reduction workspace and a launch counter.
struct Run {
  const Binding* b;
  int n_in;
  Tune tune;
  Workspace* ws;
  int* launches;
  cudaStream_t st;
  Workspace* errws;  // error word of the bulk kernels' bounded waits
  Workspace* tick;   // completion tickets (zero between launches)
};

inline Run run_of(fx_expr* x, cudaStream_t st) {
  return Run{x->b, x->e->n_in, x->tune, &x->ws, &x->last_launches, st, &x->ws_err, &x->ws_tick};
}

// n completion tickets, zero on entry (fresh workspace is zeroed; every
// launch's last block resets what it used).
inline fx_status tickets(const Run& r, int64_t n, unsigned int** out) {
  FX_TRY(r.tick->ensure(size_t(n > 0 ? n : 1) * sizeof(unsigned int), r.st));
  *out = static_cast<unsigned int*>(r.tick->p);
  return FX_OK;
}

inline fx_status err_word(const Run& r, unsigned int** out) {
  FX_TRY(r.errws->ensure(256, r.st));
  *out = static_cast<unsigned int*>(r.errws->p);
  return FX_OK;
}

// Bulk copies need every plain leaf 16-byte aligned with 16-byte column
// strides, and whole rows of the last row range in multiples of 16 bytes.
template <class LL, int I = 0> bool leaves_bulk(const Binding* b, int64_t R) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    const size_t es = sizeof(typename L::elem);
    if constexpr (L::mode == MN) {
      const Binding& x = b[L::slot];
      if (!aligned(x.p, 16) || (size_t(x.ld) * es) % 16 != 0 || (size_t(R) * es) % 16 != 0)
        return false;
    } else if constexpr (L::mode == MT) {
      return false;
    }
    return leaves_bulk<LL, I + 1>(b, R);
  }
  return true;
}

// Dynamic shared memory above 48 KB must be allowed once per kernel.
// Sets a kernel's dynamic shared-memory limit before each launch that
// needs more than the default 48 KB. Not cached: a template kernel
// instantiated in several translation units is one host symbol over
// several device functions, so a per-instantiation "already set" flag can
// skip the function that is about to run.
template <class K> fx_status allow_smem(K kern, int bytes) {
  if (bytes <= 48 * 1024) return FX_OK;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
  return FX_OK;
}

// Column splits for row-range kernels: enough blocks for the resident
// capacity, at least 2*minc columns per split.
inline int64_t row_splits(int64_t gx, int64_t C, int occ, int minc, const Tune& t) {
  const int sms = device_sms() > 0 ? device_sms() : 1;
  const int bps = t.bps > 0 ? (t.bps < occ ? t.bps : occ) : occ;
  int64_t S = (int64_t(sms) * (bps > 0 ? bps : 1) + gx - 1) / gx;
  const int64_t smax = C / (2 * minc) > 1 ? C / (2 * minc) : 1;
  if (S > smax) S = smax;
  if (S > 65535) S = 65535;
  return S < 1 ? 1 : S;
}

inline Slots make_slots(const Binding* b, int n) {
  Slots s{};
  for (int k = 0; k < n; ++k) {
    s.s[k].p = b[k].p;
    s.s[k].ld = b[k].ld;
    s.s[k].vs = (b[k].rows == 1 && b[k].cols != 1) ? b[k].ld : 1;
  }
  return s;
}

// ---------------------------------------------------------------- leaf checks

template <class LL, int I = 0> fx_status check_leaves(const Binding* b, int64_t R, int64_t C) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    const Binding& x = b[L::slot];
    bool ok = false;
    const char* want = "";
    if constexpr (L::mode == MN) {
      ok = x.rows == R && x.cols == C;
      want = "R x C";
    } else if constexpr (L::mode == MT) {
      ok = x.rows == C && x.cols == R;
      want = "C x R (transposed)";
    } else if constexpr (L::mode == MBC) {
      ok = (x.rows == R && x.cols == 1) || (x.rows == 1 && x.cols == R);
      want = "a vector of length R (each_col)";
    } else {
      ok = (x.rows == C && x.cols == 1) || (x.rows == 1 && x.cols == C);
      want = "a vector of length C (each_row)";
    }
    if (!ok)
      return fail(FX_E_SHAPE, "slot %d is %lld x %lld; expected %s with R=%lld, C=%lld", L::slot,
                  (long long)x.rows, (long long)x.cols, want, (long long)R, (long long)C);
    return check_leaves<LL, I + 1>(b, R, C);
  }
  return FX_OK;
}

// The tree's shape from its first matrix leaf.
template <class LL, int I = 0> bool infer_shape(const Binding* b, int64_t& R, int64_t& C) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    if constexpr (L::mode == MN) {
      R = b[L::slot].rows;
      C = b[L::slot].cols;
      return true;
    } else if constexpr (L::mode == MT) {
      R = b[L::slot].cols;
      C = b[L::slot].rows;
      return true;
    } else {
      return infer_shape<LL, I + 1>(b, R, C);
    }
  }
  return false;
}

template <class LL, int I = 0> FX_HD constexpr bool all_mn() {
  if constexpr (I < tl_size<LL>::value) {
    return tl_at<LL, I>::type::mode == MN && all_mn<LL, I + 1>();
  } else {
    return true;
  }
}

// Flat stream: every matrix leaf dense (ld == rows); for the vector path
// also every matrix leaf and unit-stride each_col vector aligned to A bytes.
template <class LL, int I = 0> bool leaves_dense(const Binding* b) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    const Binding& x = b[L::slot];
    if (L::mode == MN && !(x.ld == x.rows || x.cols <= 1)) return false;
    return leaves_dense<LL, I + 1>(b);
  }
  return true;
}
template <class LL, int I = 0> bool leaves_flat(const Binding* b, size_t a) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    const Binding& x = b[L::slot];
    if (L::mode == MN && !aligned(x.p, a)) return false;
    if (L::mode == MBC && !(x.rows == 1 && x.cols != 1) && !aligned(x.p, a)) return false;
    return leaves_flat<LL, I + 1>(b, a);
  }
  return true;
}

// Can the flat stream kernel run this tree at R x C? (no transposed leaf,
// dense matrix leaves; with broadcast leaves n < 2^32 and R % V == 0)
template <class LL> bool flat_ok(const Binding* b, int64_t R, int64_t C, int V) {
  if (count_mt<LL>() > 0 || !leaves_dense<LL>(b)) return false;
  if (count_bcast<LL>() == 0) return true;
  return R > 0 && R * C < (int64_t(1) << 32) && R % V == 0;
}

// Column-vector path: every full V-vector of every matrix leaf is aligned.
template <class LL, int V, int I = 0> bool leaves_vec(const Binding* b) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    const Binding& x = b[L::slot];
    const size_t a = sizeof(T) * V;
    if constexpr (L::mode == MN || L::mode == MT) {
      if (!aligned(x.p, a) || x.ld % V != 0) return false;
    } else if constexpr (L::mode == MBC) {
      const bool unit = !(x.rows == 1 && x.cols != 1);
      if (unit && !aligned(x.p, a)) return false;
    }
    return leaves_vec<LL, V, I + 1>(b);
  }
  return true;
}

// ---------------------------------------------------------------- launches

template <class K> int grid_for(K kernel, int block, int64_t work, const Tune& t) {
  const int sms = device_sms() > 0 ? device_sms() : 1;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, 0) != cudaSuccess || occ < 1)
    occ = 1;
  const int bps = t.bps > 0 ? (t.bps < occ ? t.bps : occ) : occ;
  int64_t g = int64_t(sms) * bps;
  if (g > work) g = work;
  if (g < 1) g = 1;
  return int(g);
}

inline fx_status after_launch(const Run& r, const char* what) {
  if (inject_launch_failure()) return fail(FX_E_CUDA, "%s: launch failed (injected)", what);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  ++*r.launches;
  return FX_OK;
}

// Reduction workspace for `grid` partials, and the completion ticket.
inline fx_status red_space(const Run& r, int grid, RedArgs& red) {
  const size_t part = size_t(grid) * sizeof(double2);
  FX_TRY(r.ws->ensure(part + 256, r.st));
  red.part = static_cast<double2*>(r.ws->p);
  return tickets(r, 1, &red.ticket);
}

template <class E, class Epi, int V, int U>
fx_status launch_flat_u(const Run& r, const E& e, const Slots& sl, int64_t n, const Epi& epi,
                        RedArgs red, int64_t flat_rows) {
  auto kern = k_flat<E, Epi, V, U>;
  const int block = (r.tune.block >= 64 && r.tune.block <= 512) ? r.tune.block : 256;
  const int64_t nv = n / V;
  int64_t work = (nv + int64_t(block) * U - 1) / (int64_t(block) * U);
  const int grid = grid_for(kern, block, work > 0 ? work : 1, r.tune);
  if constexpr (Epi::reduces) FX_TRY(red_space(r, grid, red));
  FastDiv fd{};
  if constexpr (count_bcast<leaves_t<E>>() > 0) fd = FastDiv::make(uint32_t(flat_rows));
  kern<<<grid, block, 0, r.st>>>(e, sl, n, epi, red, fd);
  return after_launch(r, "k_flat");
}

// Vectors per leaf in flight per thread: at most 16 vectors in all (the
// register budget of a thread), so 8 for one or two leaves, 4 for up to
// four, 2 for up to eight, 1 beyond.
template <class E> constexpr int max_unroll() {
  constexpr int nl = tl_size<leaves_t<E>>::value;
  return nl <= 2 ? 8 : (nl <= 4 ? 4 : (nl <= 8 ? 2 : 1));
}

// k_flat_bulk for trees whose leaves are all dense matrices of one storage
// type with 16-byte aligned bases: one CTA per SM (two when two stages fit
// in half the shared memory), chunks of 1024 elements per leaf.
template <class E, class Epi, int V>
fx_status launch_flat_bulk(const Run& r, const E& e, const Slots& sl, int64_t n, const Epi& epi,
                           RedArgs red, bool* used) {
  using LL = leaves_t<E>;
  *used = false;
  if constexpr (V == 1 || count_bcast<LL>() > 0) {
    return FX_OK;
  } else {
    using T0 = typename tl_at<LL, 0>::type::elem;
    if constexpr (!tma_uniform<LL, T0>() || V * sizeof(T0) != 16) {
      return FX_OK;
    } else {
      constexpr int NTC = 256, CH = 1024 * 16 / int(sizeof(T0)) / 4;
      constexpr int SB = tl_size<LL>::value * CH * int(sizeof(T0));
      if (!leaves_flat<LL>(r.b, 16)) return FX_OK;
      const int fixed = int(sizeof(Ring<8>)) + 2048;
      auto stages = [&](int per_sm) {
        const int k = ((227 * 1024) / per_sm - fixed) / SB;
        return k > 8 ? 8 : k;
      };
      int ns = r.tune.bps == 1 ? 0 : stages(2);
      if (ns < 2 && r.tune.bps < 2) ns = stages(1);
      if (ns < 2) return FX_OK;
      const int smem = ns * SB + fixed;
      auto kern = k_flat_bulk<E, Epi, V, NTC, CH>;
      FX_TRY(allow_smem(kern, smem));
      unsigned int* err = nullptr;
      FX_TRY(err_word(r, &err));
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NTC + 32, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
      }
      const int64_t n16 = n - n % V;
      const int64_t nch = (n16 + CH - 1) / CH;
      const int sms = device_sms() > 0 ? device_sms() : 1;
      int64_t grid = int64_t(sms) * occ;
      if (grid > nch) grid = nch;
      if (grid < 1) grid = 1;
      if constexpr (Epi::reduces) FX_TRY(red_space(r, int(grid), red));
      *used = true;
      kern<<<unsigned(grid), NTC + 32, smem, r.st>>>(e, sl, n, n16, epi, red, ns, err);
      return after_launch(r, "k_flat_bulk");
    }
  }
}

// Flat trees: the bulk-copy kernel for pipeline 1, and by default (0) for
// five or more leaves, where the register kernel's one vector per leaf in
// flight no longer covers HBM latency (measured on GB300: 10000^2 FP32
// add-N, N = 5..16, 6.8-7.0 TB/s bulk against 6.5-6.7 TB/s, and 4.9 TB/s
// for N = 16); register loads otherwise and for pipeline 2.
template <class E, class Epi, int V>
fx_status launch_flat(const Run& r, const E& e, const Slots& sl, int64_t n, const Epi& epi,
                      RedArgs red, int64_t flat_rows) {
  constexpr bool many = tl_size<leaves_t<E>>::value >= 5;
  if (r.tune.pipe == 1 || (r.tune.pipe == 0 && many)) {
    bool used = false;
    const fx_status s = launch_flat_bulk<E, Epi, V>(r, e, sl, n, epi, red, &used);
    if (s != FX_OK || used) return s;
  }
  constexpr int UM = max_unroll<E>();
  switch (r.tune.unroll) {
    case 2: return launch_flat_u<E, Epi, V, (2 < UM ? 2 : UM)>(r, e, sl, n, epi, red, flat_rows);
    case 8: return launch_flat_u<E, Epi, V, UM>(r, e, sl, n, epi, red, flat_rows);
    default: return launch_flat_u<E, Epi, V, (4 < UM ? 4 : UM)>(r, e, sl, n, epi, red, flat_rows);
  }
}

// Tile shapes: 64 x 64 (32 x 32 for FP64) when a transposed leaf is staged
// through shared memory; 256 x 16 otherwise (long contiguous column runs).
template <class E, int V> struct TileCfg {
  static constexpr bool has_t = count_mt<leaves_t<E>>() > 0;
  static constexpr bool dbl = std::is_same<ct_of<E>, double>::value;
  static constexpr int TR = has_t ? (dbl ? 32 : 64) : 256;
  static constexpr int TC = has_t ? (dbl ? 32 : 64) : 16;
  static constexpr int NT = 256;
};

template <class E, class Epi, int V>
fx_status launch_tile(const Run& r, const E& e, const Slots& sl, int64_t R, int64_t C,
                      const Epi& epi, RedArgs red) {
  using TC_ = TileCfg<E, V>;
  auto kern = k_tile<E, Epi, V, TC_::TR, TC_::TC, TC_::NT>;
  const int64_t ntiles = ((R + TC_::TR - 1) / TC_::TR) * ((C + TC_::TC - 1) / TC_::TC);
  const int grid = grid_for(kern, TC_::NT, ntiles > 0 ? ntiles : 1, r.tune);
  if constexpr (Epi::reduces) FX_TRY(red_space(r, grid, red));
  kern<<<grid, TC_::NT, 0, r.st>>>(e, sl, R, C, epi, red);
  return after_launch(r, "k_tile");
}

// Transposed leaves of 2-byte types are copied in element pairs: 4-byte
// aligned base, even leading dimension.
template <class LL, int I = 0> bool mt_pairs_ok(const Binding* b) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    if constexpr (L::mode == MT && sizeof(typename L::elem) == 2) {
      const Binding& x = b[L::slot];
      if (!aligned(x.p, 4) || x.ld % 2 != 0) return false;
    }
    return mt_pairs_ok<LL, I + 1>(b);
  }
  return true;
}

// k_tile_async shapes: 64 x 64 tiles for 2-byte types, 64 x 32 for 4-byte,
// 32 x 32 for 8-byte; three stages.
template <class E, int V> struct TileAsyncCfg {
  static constexpr int es = tl_max_elem<leaves_t<E>>::value;
  static constexpr int TR = es == 8 ? 32 : 64;
  static constexpr int TC = es == 2 ? 64 : 32;
  static constexpr int NT = 256, NBUF = 3;
  static constexpr int SMEM = NBUF * tbuf_offset<leaves_t<E>, TR, TC, tl_size<leaves_t<E>>::value>();
};

template <class E, class Epi, int V>
fx_status launch_tile_async(const Run& r, const E& e, const Slots& sl, int64_t R, int64_t C,
                            const Epi& epi, RedArgs red) {
  using Cf = TileAsyncCfg<E, V>;
  auto kern = k_tile_async<E, Epi, V, Cf::TR, Cf::TC, Cf::NT, Cf::NBUF>;
  FX_TRY(allow_smem(kern, Cf::SMEM));
  const int64_t ntiles = ((R + Cf::TR - 1) / Cf::TR) * ((C + Cf::TC - 1) / Cf::TC);
  const int sms = device_sms() > 0 ? device_sms() : 1;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, Cf::NT, Cf::SMEM) != cudaSuccess || occ < 1) occ = 1;
  const int bps = r.tune.bps > 0 ? (r.tune.bps < occ ? r.tune.bps : occ) : occ;
  int64_t grid = int64_t(sms) * bps;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  if constexpr (Epi::reduces) FX_TRY(red_space(r, int(grid), red));
  kern<<<unsigned(grid), Cf::NT, Cf::SMEM, r.st>>>(e, sl, R, C, epi, red);
  return after_launch(r, "k_tile_async");
}

// k_tile_tma: one CTA per SM (two with blocks_per_sm >= 2), as many
// stages as fit next to the output tiles (two items' worth). Trees whose
// TMA leaves are closed under transposition take symmetric tile pairs.
// *used is false when the operands are not TMA-addressable or fewer than
// two stages fit.
template <class T, class E, class Epi>
fx_status launch_tile_tma(const Run& r, const E& e, const Slots& sl, int64_t R, int64_t C,
                          const Epi& epi, RedArgs red, bool* used) {
  using LL = leaves_t<E>;
  using G = TmaGeom<T>;
  *used = false;
  if constexpr (!tma_uniform<LL, T>()) {
    return FX_OK;
  } else {
    constexpr int NTC = 256;
    constexpr int SB = count_tma<LL>() * G::LEAF;
    TileMaps tm;
    if (!encode_leaf_maps<LL, T>(tm, r.b)) return FX_OK;
    if constexpr (Epi::stores) {
      if (!encode_tile_map<T>(&tm.m[r.n_in], epi.z, R, C, epi.ldz)) return FX_OK;
    }
    constexpr bool SYM = flip_closed<LL>();
    const int fixed = (Epi::stores ? 2 * (SYM ? 2 : 1) * G::LEAF : 0) +
                      int(sizeof(Ring<kTmaMaxStages>)) + 1024;
    // Two CTAs per SM when two stages fit in half the shared memory (their
    // 16 consumer warps keep up with HBM on BF16 trees, where 8 do not),
    // else one; blocks_per_sm 1 or 2 forces the choice. 227 KB per SM,
    // less 2 KB per CTA for the combine's static shared memory.
    auto stages = [&](int per_sm) {
      const int n = ((227 * 1024) / per_sm - 2048 - fixed) / SB;
      return n > kTmaMaxStages ? kTmaMaxStages : n;
    };
    int ns = r.tune.bps == 1 ? 0 : stages(2);
    if (ns < 2 && r.tune.bps < 2) ns = stages(1);
    if (ns < 2) return FX_OK;
    const int smem = ns * SB + fixed;
    auto kern = k_tile_tma<E, Epi, T, NTC, SYM>;
    FX_TRY(allow_smem(kern, smem));
    unsigned int* err = nullptr;
    FX_TRY(err_word(r, &err));
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NTC + 32, smem) != cudaSuccess || occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    const int sms = device_sms() > 0 ? device_sms() : 1;
    const int64_t tr = (R + G::TT - 1) / G::TT;
    const int64_t ntiles = SYM ? tr * (tr + 1) / 2 : tr * ((C + G::TT - 1) / G::TT);
    int64_t grid = int64_t(sms) * occ;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    if constexpr (Epi::reduces) FX_TRY(red_space(r, int(grid), red));
    *used = true;
    kern<<<unsigned(grid), NTC + 32, smem, r.st>>>(e, sl, R, C, epi, red, tm, r.n_in, ns, err);
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
      cudaFuncAttributes fa{};
      cudaFuncGetAttributes(&fa, kern);
      cudaGetLastError();
      return fail(FX_E_CUDA,
                  "k_tile_tma: %s (grid %lld, %d stages, %d + %d bytes of shared memory, limit %d, "
                  "%d registers)",
                  cudaGetErrorString(le), (long long)grid, ns, smem, int(fa.sharedSizeBytes),
                  fa.maxDynamicSharedSizeBytes, fa.numRegs);
    }
    return after_launch(r, "k_tile_tma");
  }
}

// Tiles of a tree with transposed leaves. Launch-shape pipeline 0: the
// TMA kernel when the operands allow it; 1: the cp.async pipeline when
// every plain leaf and the output are vector-aligned; otherwise, and for
// pipeline 2, the register-staged kernel.
template <class T, class E, class EpiV, class Epi1, int V>
fx_status launch_tiles(const Run& r, const E& e, const Slots& sl, int64_t R, int64_t C, bool vec,
                       const EpiV& ev, const Epi1& e1, RedArgs red) {
  using LL = leaves_t<E>;
  if constexpr (count_mt<LL>() > 0) {
    if (r.tune.pipe == 0) {
      bool used = false;
      const fx_status s = launch_tile_tma<T>(r, e, sl, R, C, ev, red, &used);
      if (s != FX_OK || used) return s;
    }
  }
  if constexpr (count_mt<LL>() > 0 && V > 1 && TileAsyncCfg<E, V>::SMEM <= 200 * 1024) {
    if (r.tune.pipe == 1 && vec && mt_pairs_ok<LL>(r.b))
      return launch_tile_async<E, EpiV, V>(r, e, sl, R, C, ev, red);
  }
  if (vec) return launch_tile<E, EpiV, V>(r, e, sl, R, C, ev, red);
  return launch_tile<E, Epi1, 1>(r, e, sl, R, C, e1, red);
}

// ---------------------------------------------------------------- element-wise

template <class T, class E> fx_status run_elementwise(const Run& r, const E& e) {
  using LL = leaves_t<E>;
  constexpr int V = vec_width<E, 16>();
  const Binding& zb = r.b[r.n_in];
  const int64_t R = zb.rows, C = zb.cols;
  FX_TRY(check_leaves<LL>(r.b, R, C));
  if (R * C == 0) return FX_OK;
  const Slots sl = make_slots(r.b, r.n_in);
  T* z = static_cast<T*>(zb.p);
  const bool zdense = zb.ld == R || C == 1;
  if constexpr (count_mt<LL>() == 0) {
    if (zdense && flat_ok<LL>(r.b, R, C, 1)) {
      if (flat_ok<LL>(r.b, R, C, V) && leaves_flat<LL>(r.b, V * sizeof(T)) &&
          aligned(z, V * sizeof(T)))
        return launch_flat<E, EpiStore<T, V>, V>(r, e, sl, R * C, EpiStore<T, V>{z, R}, {}, R);
      return launch_flat<E, EpiStore<T, 1>, 1>(r, e, sl, R * C, EpiStore<T, 1>{z, R}, {}, R);
    }
  }
  const bool vec = leaves_vec<LL, V>(r.b) && aligned(z, V * sizeof(T)) && zb.ld % V == 0;
  return launch_tiles<T, E, EpiStore<T, V>, EpiStore<T, 1>, V>(
      r, e, sl, R, C, vec, EpiStore<T, V>{z, zb.ld}, EpiStore<T, 1>{z, zb.ld}, {});
}

// Element-wise tree plus its accu (outputs Z and s).
template <class T, class E> fx_status run_multi(const Run& r, const E& e) {
  using LL = leaves_t<E>;
  constexpr int V = vec_width<E, 16>();
  const Binding& zb = r.b[r.n_in];
  const Binding& sb = r.b[r.n_in + 1];
  const int64_t R = zb.rows, C = zb.cols;
  FX_TRY(check_leaves<LL>(r.b, R, C));
  if (sb.rows * sb.cols != 1) return fail(FX_E_SHAPE, "the accu output must be 1 x 1");
  const Slots sl = make_slots(r.b, r.n_in);
  T* z = static_cast<T*>(zb.p);
  RedArgs red{};
  red.out = sb.p;
  const bool zdense = zb.ld == R || C == 1;
  if constexpr (count_mt<LL>() == 0) {
    if (zdense && flat_ok<LL>(r.b, R, C, 1)) {
      if (flat_ok<LL>(r.b, R, C, V) && leaves_flat<LL>(r.b, V * sizeof(T)) &&
          aligned(z, V * sizeof(T)))
        return launch_flat<E, EpiStoreSum<T, V>, V>(r, e, sl, R * C, EpiStoreSum<T, V>{z, R}, red,
                                                    R);
      return launch_flat<E, EpiStoreSum<T, 1>, 1>(r, e, sl, R * C, EpiStoreSum<T, 1>{z, R}, red,
                                                  R);
    }
  }
  const bool vec = leaves_vec<LL, V>(r.b) && aligned(z, V * sizeof(T)) && zb.ld % V == 0;
  return launch_tiles<T, E, EpiStoreSum<T, V>, EpiStoreSum<T, 1>, V>(
      r, e, sl, R, C, vec, EpiStoreSum<T, V>{z, zb.ld}, EpiStoreSum<T, 1>{z, zb.ld}, red);
}

// with_accu(E, S): Z = E stored and s = accu(S), one pass over the union of
// their leaves (the kernel's tree is Bin<OpFirst, E, S>; the epilogue sums S
// from the same registers).
template <class T, class Root> fx_status run_multi_side(const Run& r, const Root& root) {
  using E = typename root_of<Root>::inner;   // Bin<OpFirst, E1, S>
  using S = decltype(E::r);
  using LL = leaves_t<E>;
  constexpr int V = vec_width<E, 16>();
  const E& e = inner_of(root);
  const Binding& zb = r.b[r.n_in];
  const Binding& sb = r.b[r.n_in + 1];
  const int64_t R = zb.rows, C = zb.cols;
  FX_TRY(check_leaves<LL>(r.b, R, C));
  if (sb.rows * sb.cols != 1) return fail(FX_E_SHAPE, "the accu output must be 1 x 1");
  const Slots sl = make_slots(r.b, r.n_in);
  T* z = static_cast<T*>(zb.p);
  RedArgs red{};
  red.out = sb.p;
  using EV = EpiStoreSide<T, V, S>;
  using E1 = EpiStoreSide<T, 1, S>;
  const bool zdense = zb.ld == R || C == 1;
  if constexpr (count_mt<LL>() == 0) {
    if (zdense && flat_ok<LL>(r.b, R, C, 1)) {
      if (flat_ok<LL>(r.b, R, C, V) && leaves_flat<LL>(r.b, V * sizeof(T)) &&
          aligned(z, V * sizeof(T)))
        return launch_flat<E, EV, V>(r, e, sl, R * C, EV{z, R, e.r}, red, R);
      return launch_flat<E, E1, 1>(r, e, sl, R * C, E1{z, R, e.r}, red, R);
    }
  }
  const bool vec = leaves_vec<LL, V>(r.b) && aligned(z, V * sizeof(T)) && zb.ld % V == 0;
  return launch_tiles<T, E, EV, E1, V>(r, e, sl, R, C, vec, EV{z, zb.ld, e.r},
                                       E1{z, zb.ld, e.r}, red);
}

// ---------------------------------------------------------------- A5: accu, norm

template <class T, class Root> fx_status run_full_reduce(const Run& r, const Root& root) {
  using E = typename root_of<Root>::inner;
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  constexpr bool SQ = std::is_same<Root, Norm2<E>>::value;
  constexpr int V = vec_width<E, 16>();
  const E& e = inner_of(root);
  int64_t R = 0, C = 0;
  if (!infer_shape<LL>(r.b, R, C)) return fail(FX_E_SHAPE, "no matrix leaf to take the shape from");
  FX_TRY(check_leaves<LL>(r.b, R, C));
  const Binding& ob = r.b[r.n_in];
  if (ob.rows * ob.cols != 1) return fail(FX_E_SHAPE, "the reduction output must be 1 x 1");
  const Slots sl = make_slots(r.b, r.n_in);
  RedArgs red{};
  red.out = ob.p;
  if constexpr (count_mt<LL>() == 0) {
    if (flat_ok<LL>(r.b, R, C, 1)) {
      if (flat_ok<LL>(r.b, R, C, V) && leaves_flat<LL>(r.b, V * sizeof(T)))
        return launch_flat<E, EpiSum<CT, V, SQ>, V>(r, e, sl, R * C, EpiSum<CT, V, SQ>{R}, red, R);
      return launch_flat<E, EpiSum<CT, 1, SQ>, 1>(r, e, sl, R * C, EpiSum<CT, 1, SQ>{R}, red, R);
    }
  }
  return launch_tiles<T, E, EpiSum<CT, V, SQ>, EpiSum<CT, 1, SQ>, V>(
      r, e, sl, R, C, leaves_vec<LL, V>(r.b), EpiSum<CT, V, SQ>{0}, EpiSum<CT, 1, SQ>{0}, red);
}

// ---------------------------------------------------------------- A6: sum / max along a dim

template <class Root> struct dim_of;
template <class E, int D> struct dim_of<SumDim<E, D>> { static constexpr int d = D; static constexpr bool ismax = false; };
template <class E, int D> struct dim_of<MaxDim<E, D>> { static constexpr int d = D; static constexpr bool ismax = true; };

template <class E, bool ISMAX, int V>
fx_status launch_col(const Run& r, const E& e, const Slots& sl, int64_t R, int64_t C, void* out,
                     int64_t ldo) {
  constexpr int NT = 256, U = tl_size<leaves_t<E>>::value <= 2 ? 8 : 4;
  // a block per column for long FP32 columns; a warp per column otherwise,
  // and for FP64 up to 2^16 rows: its slow FP64 unit leaves a block per
  // column waiting on the block-wide merge after only a few steps
  constexpr bool dbl = std::is_same<ct_of<E>, double>::value;
  if (R >= (dbl ? 65536 : 1024)) {
    auto kern = k_col<E, ISMAX, V, U, NT, NT>;
    const int grid = grid_for(kern, NT, C > 0 ? C : 1, r.tune);
    kern<<<grid, NT, 0, r.st>>>(e, sl, R, C, out, ldo);
  } else {
    auto kern = k_col<E, ISMAX, V, U, 32, NT>;
    const int64_t work = (C + NT / 32 - 1) / (NT / 32);
    const int grid = grid_for(kern, NT, work > 0 ? work : 1, r.tune);
    kern<<<grid, NT, 0, r.st>>>(e, sl, R, C, out, ldo);
  }
  return after_launch(r, "k_col");
}

template <class E, bool ISMAX, int V>
fx_status launch_row(const Run& r, const E& e, const Slots& sl, int64_t R, int64_t C, void* out) {
  using CT = ct_of<E>;
  using LL = leaves_t<E>;
  // ~128 KB in flight per SM: 8 column vectors per thread for 1-2 leaves
  constexpr int NT = 256, U = tl_size<LL>::value <= 2 ? 8 : 4, NS = 4;
  RowRed rr{};
  rr.out = out;
  auto space = [&](int64_t gx, int64_t S) -> fx_status {
    rr.S = int(S);
    if (S > 1) {
      const size_t part = size_t(S) * R * sizeof(double2);
      const size_t partm = size_t(S) * R * sizeof(CT);
      FX_TRY(r.ws->ensure(part + partm + 512, r.st));
      char* w = static_cast<char*>(r.ws->p);
      rr.part = reinterpret_cast<double2*>(w);
      rr.partm = w + part;
      FX_TRY(tickets(r, gx, &rr.tickets));
    }
    return FX_OK;
  };
  if constexpr (V > 1) {
   if (r.tune.pipe == 1 && leaves_bulk<LL>(r.b, R)) {
    constexpr int CPS = 2;
    auto kern = k_row_bulk<E, ISMAX, V, NT, NS, CPS>;
    constexpr int smem = NS * CPS * stage_bytes<LL, NT * V>() + int(sizeof(Ring<NS>));
    FX_TRY(allow_smem(kern, smem));
    unsigned int* err = nullptr;
    FX_TRY(err_word(r, &err));
    const int64_t gx = (R + int64_t(NT) * V - 1) / (int64_t(NT) * V);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT + 32, smem) != cudaSuccess || occ < 1) occ = 1;
    const int64_t S = row_splits(gx, C, occ, 2 * NS * CPS, r.tune);
    FX_TRY(space(gx, S));
    kern<<<dim3(unsigned(gx), unsigned(S)), NT + 32, smem, r.st>>>(e, sl, R, C, rr, err);
    return after_launch(r, "k_row_bulk");
  }
  }
  auto kern = k_row<E, ISMAX, V, U, NT>;
  const int64_t gx = (R + int64_t(NT) * V - 1) / (int64_t(NT) * V);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, 0) != cudaSuccess || occ < 1) occ = 1;
  const int64_t S = row_splits(gx, C, occ, U, r.tune);
  FX_TRY(space(gx, S));
  kern<<<dim3(unsigned(gx > 0 ? gx : 1), unsigned(S)), NT, 0, r.st>>>(e, sl, R, C, rr);
  return after_launch(r, "k_row");
}

template <class T, class Root> fx_status run_dim_reduce(const Run& r, const Root& root) {
  using E = typename root_of<Root>::inner;
  using LL = leaves_t<E>;
  constexpr int D = dim_of<Root>::d;
  constexpr bool ISMAX = dim_of<Root>::ismax;
  constexpr int V = vec_width<E, 16>();
  static_assert(count_mt<LL>() == 0, "dim reductions over transposed leaves are not fused");
  const E& e = inner_of(root);
  int64_t R = 0, C = 0;
  if (!infer_shape<LL>(r.b, R, C)) return fail(FX_E_SHAPE, "no matrix leaf to take the shape from");
  FX_TRY(check_leaves<LL>(r.b, R, C));
  const Binding& ob = r.b[r.n_in];
  const Slots sl = make_slots(r.b, r.n_in);
  if (D == 0) {
    if (!(ob.rows == 1 && ob.cols == C)) return fail(FX_E_SHAPE, "sum/max along dim 0 gives 1 x %lld", (long long)C);
    if (C == 0) return FX_OK;
    if (leaves_vec<LL, V>(r.b)) return launch_col<E, ISMAX, V>(r, e, sl, R, C, ob.p, ob.ld);
    return launch_col<E, ISMAX, 1>(r, e, sl, R, C, ob.p, ob.ld);
  }
  if (!(ob.rows == R && ob.cols == 1)) return fail(FX_E_SHAPE, "sum/max along dim 1 gives %lld x 1", (long long)R);
  if (R == 0) return FX_OK;
  if (leaves_vec<LL, V>(r.b)) return launch_row<E, ISMAX, V>(r, e, sl, R, C, ob.p);
  return launch_row<E, ISMAX, 1>(r, e, sl, R, C, ob.p);
}

// ---------------------------------------------------------------- root dispatch

template <class T, class Root> fx_status run_root(const Run& r, const Root& root, int kind) {
  static_assert(!has_prod_v<Root>, "a matrix product is a fusion boundary");
  if constexpr (is_with_accu<Root>::value) {
    return run_multi_side<T>(r, root);
  }
  if (kind == FX_KIND_MULTI) {
    if constexpr (root_of<Root>::kind == FX_KIND_ELEMENTWISE) return run_multi<T>(r, root);
    return fail(FX_E_UNSUPPORTED, "multi-output needs an element-wise tree");
  }
  if constexpr (root_of<Root>::kind == FX_KIND_ELEMENTWISE) return run_elementwise<T>(r, root);
  else if constexpr (root_of<Root>::kind == FX_KIND_FULL_REDUCE) return run_full_reduce<T>(r, root);
  else if constexpr (root_of<Root>::kind == FX_KIND_DIM_REDUCE) return run_dim_reduce<T>(r, root);
  else return fail(FX_E_UNSUPPORTED, "unknown root");
}

// ---------------------------------------------------------------- A9: backward

template <class T, class Root>
fx_status run_backward(fx_expr* x, const Root& root, const void* gout, void* const* grads,
                       cudaStream_t st) {
  if constexpr (!std::is_same<Root, Accu<typename root_of<Root>::inner>>::value) {
    return fail(FX_E_UNSUPPORTED, "fused backward needs an accu(...) root");
  } else {
    using E = typename root_of<Root>::inner;
    using LL = leaves_t<E>;
    // 8-byte accesses: the reverse pass keeps one adjoint per leaf per lane
    // live, so narrower lanes leave room for more resident threads
    constexpr int V = vec_width<E, 8>() > 0 ? vec_width<E, 8>() : 1;
    constexpr int NT = 256, U = 2;
    constexpr int NBC = count_mode<LL>(MBC);
    const Run r = run_of(x, st);
    const E& e = inner_of(root);
    int64_t R = 0, C = 0;
    if (!infer_shape<LL>(r.b, R, C)) return fail(FX_E_SHAPE, "no matrix leaf to take the shape from");
    FX_TRY(check_leaves<LL>(r.b, R, C));
    GradArgs ga{};
    bool vec = leaves_vec<LL, V>(r.b) && R % V == 0;
    for (int k = 0; k < r.n_in; ++k) {
      ga.g[k] = grads[k];
      if (grads[k] && !aligned(grads[k], sizeof(T))) return fail(FX_E_ALIGN, "gradient %d misaligned", k);
      if (grads[k] && !aligned(grads[k], sizeof(T) * V)) vec = false;
    }
    ga.gscale = gout;
    if (R * C == 0) {
      // gradients of an empty sum are zero
      for (int k = 0; k < r.n_in; ++k)
        if (grads[k]) FX_CUDA(cudaMemsetAsync(grads[k], 0, size_t(r.b[k].rows) * r.b[k].cols * sizeof(T), st));
      return FX_OK;
    }
    const Slots sl = make_slots(r.b, r.n_in);
    auto space = [&](int64_t gx, int64_t S) -> fx_status {
      ga.S = int(S);
      if (NBC > 0) {
        const size_t part = size_t(NBC) * S * R * sizeof(double2);
        FX_TRY(x->ws.ensure(part + 512, st));
        ga.part = static_cast<double2*>(x->ws.p);
        FX_TRY(tickets(r, gx, &ga.tickets));
      }
      return FX_OK;
    };
    // bulk-copy pipeline when every plain leaf and gradient allows 16-byte copies
    // thread lanes of 8 bytes (2 FP32, 4 BF16/FP16, 1 FP64): the reverse pass
    // keeps one adjoint per leaf per lane live
    constexpr int VB = vec_width<E, 8>();
    bool bulk = VB > 1 && leaves_bulk<LL>(r.b, R) && R % VB == 0;
    for (int k = 0; k < r.n_in; ++k)
      if (grads[k] && !aligned(grads[k], 16)) bulk = false;
    if (bulk) {
      constexpr int NS = 4, CPS = 4;
      auto kern = k_bwd_bulk<E, VB, NT, NS, CPS>;
      constexpr int smem = NS * CPS * stage_bytes<LL, NT * VB>() + int(sizeof(Ring<NS>));
      FX_TRY(allow_smem(kern, smem));
      unsigned int* err = nullptr;
      FX_TRY(err_word(r, &err));
      const int64_t gx = (R + int64_t(NT) * VB - 1) / (int64_t(NT) * VB);
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT + 32, smem) != cudaSuccess || occ < 1) occ = 1;
      const int64_t S = row_splits(gx, C, occ, 2 * NS * CPS, r.tune);
      FX_TRY(space(gx, S));
      kern<<<dim3(unsigned(gx), unsigned(S)), NT + 32, smem, st>>>(e, sl, R, C, ga, err);
      return after_launch(r, "k_bwd_bulk");
    }
    auto go = [&](auto kern, int v) -> fx_status {
      const int64_t gx = (R + int64_t(NT) * v - 1) / (int64_t(NT) * v);
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, 0) != cudaSuccess || occ < 1) occ = 1;
      const int64_t S = row_splits(gx, C, occ, U, r.tune);
      FX_TRY(space(gx, S));
      kern<<<dim3(unsigned(gx), unsigned(S)), NT, 0, st>>>(e, sl, R, C, ga);
      return after_launch(r, "k_bwd");
    };
    if (vec) return go(k_bwd<E, V, U, NT>, V);
    return go(k_bwd<E, 1, U, NT>, 1);
  }
}

}  // namespace fx
