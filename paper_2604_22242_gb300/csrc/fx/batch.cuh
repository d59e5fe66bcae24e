// batch.cuh - one tree over many independent matrices of uneven shapes.
//
// The host builds a work-list: every matrix is cut into TR x TC tiles
// (matrices in decreasing size order, so the smallest tiles come last and
// fill the tail); one persistent launch (grid = SMs x resident blocks)
// walks the list with a static stride and runs the same tile body as the
// single-matrix tiled kernel (transposed leaves staged through shared
// memory). A tree with an accu output writes one compensated partial per
// tile; a second launch sums each matrix's partials in tile order in FP64
// (one warp per matrix). The list, the descriptors and both launches are
// cached per item array; with use_graph the launches are captured once in a
// CUDA graph and replayed.
#pragma once

#include <algorithm>
#include <cstring>
#include <vector>

#include "launch.cuh"

namespace fx {

struct BatchMat {
  const void* p[FX_MAX_SLOTS];
  int64_t ld[FX_MAX_SLOTS];
  int64_t rows, cols;
  int64_t first;   // first work item of this matrix
  int32_t ntiles;
  int32_t vec;     // every full vector of this matrix is aligned
};
struct BatchItem {
  int32_t mat;
  int32_t tile;
};

template <class T, int V, int KIND> struct batch_epi;
template <class T, int V> struct batch_epi<T, V, FX_KIND_ELEMENTWISE> {
  using type = EpiStore<T, V>;
  static FX_D type make(const BatchMat& m, int zs) { return {static_cast<T*>(const_cast<void*>(m.p[zs])), m.ld[zs]}; }
};
template <class T, int V> struct batch_epi<T, V, FX_KIND_MULTI> {
  using type = EpiStoreSum<T, V>;
  static FX_D type make(const BatchMat& m, int zs) { return {static_cast<T*>(const_cast<void*>(m.p[zs])), m.ld[zs]}; }
};
template <class T, int V> struct batch_epi<T, V, FX_KIND_FULL_REDUCE> {
  using type = EpiSum<compute_t<T>, V, false>;
  static FX_D type make(const BatchMat&, int) { return {0}; }
};

template <class TS, class T, int KIND, class E>
FX_D void batch_tile(const E& e, const Slots& sl, const BatchMat& m, int32_t tile, int zs,
                     double2* part, int64_t it, typename TS::CT* sm) {
  using Bx = batch_epi<T, TS::V, KIND>;
  typename Bx::type epi = Bx::make(m, zs);
  typename Bx::type::State st;
  st.init();
  const int64_t tiles_r = (m.rows + TS::TR - 1) / TS::TR;
  const int64_t tr = tile % tiles_r, tc = tile / tiles_r;
  tile_body<TS>(e, sl, m.rows, m.cols, tr * TS::TR, tc * TS::TC, epi, st, sm);
  if constexpr (Bx::type::reduces) {
    block_merge(st);
    if (threadIdx.x == 0) part[it] = make_double2(double(st.s), double(st.c));
  }
}

// Matrices whose every full vector is aligned use V-wide tiles, the others
// scalar tiles; both TR rows high and as wide as two vectors per thread
// (few registers per thread, so several blocks stay resident per SM).
template <class E, int V, int TR, int TC, int NT> struct BatchShapes {
  using Vec = TileShape<E, V, TR, 2 * (NT / (TR / V)), NT>;
  using One = TileShape<E, 1, TR, 2 * (NT / TR), NT>;
};

template <class E, class T, int V, int TR, int TC, int NT, int KIND, int NIN>
__global__ void __launch_bounds__(NT, 3) k_batch(const E e, const BatchMat* __restrict__ mats,
                                                 const BatchItem* __restrict__ items,
                                                 const int64_t nitems, double2* part) {
  using TSv = typename BatchShapes<E, V, TR, TC, NT>::Vec;
  using TS1 = typename BatchShapes<E, V, TR, TC, NT>::One;
  using CT = typename TSv::CT;
  __shared__ CT sm[TSv::SMEM > TS1::SMEM ? TSv::SMEM : TS1::SMEM];
  for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem w = items[it];
    const BatchMat& m = mats[w.mat];
    Slots sl;
#pragma unroll
    for (int k = 0; k < NIN; ++k) {
      sl.s[k].p = m.p[k];
      sl.s[k].ld = m.ld[k];
      sl.s[k].vs = 1;
    }
    if (m.vec) batch_tile<TSv, T, KIND>(e, sl, m, w.tile, NIN, part, it, sm);
    else batch_tile<TS1, T, KIND>(e, sl, m, w.tile, NIN, part, it, sm);
  }
}

// One warp per matrix: its tiles' partials, in tile order, summed in FP64.
template <class RT>
__global__ void __launch_bounds__(256) k_batch_combine(const BatchMat* __restrict__ mats,
                                                       const int64_t nmat, const double2* part,
                                                       const int sslot) {
  const int64_t i = int64_t(blockIdx.x) * 8 + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (i >= nmat) return;  // whole warps leave together
  const BatchMat& m = mats[i];
  std::conditional_t<std::is_same<RT, double>::value, CompSum<double>, PlainSum<double>> a;
  a.init();
  for (int64_t k = lane; k < m.ntiles; k += 32) {
    double2 q = __ldcg(part + m.first + k);
    a.add(q.x);
    a.add(q.y);
  }
  warp_merge(a);
  if (lane == 0) *static_cast<RT*>(const_cast<void*>(m.p[sslot])) = RT(a.s + a.c);
}

struct BatchCacheEntry {
  uint64_t key = 0;
  int64_t n = 0, nitems = 0;
  Workspace dev;  // descriptors, items, partials
  BatchMat* mats = nullptr;
  BatchItem* items = nullptr;
  double2* part = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t exec_stream = nullptr;
};

}  // namespace fx

struct fx::BatchCache {
  BatchCacheEntry cur;
};

namespace fx {

inline uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

template <class LL, int V, int I = 0>
bool batch_leaf_check(const fx_batch_item& it, int64_t R, int64_t C, bool& vec, int& bad) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    const int k = L::slot;
    const void* p = it.ptr[k];
    int64_t rows = R, cols = C;
    if constexpr (L::mode == MT) {
      rows = C;
      cols = R;
    } else if constexpr (L::mode == MBC) {
      cols = 1;
    } else if constexpr (L::mode == MBR) {
      rows = C;
      cols = 1;
    }
    const int64_t ld = it.ld[k] ? it.ld[k] : (rows > 0 ? rows : 1);
    if (ld < rows || (rows * cols > 0 && !p) || !aligned(p, sizeof(T))) {
      bad = k;
      return false;
    }
    if constexpr (L::mode == MN || L::mode == MT) {
      if (!aligned(p, sizeof(T) * V) || ld % V != 0) vec = false;
    } else if constexpr (L::mode == MBC) {
      if (!aligned(p, sizeof(T) * V)) vec = false;
    }
    return batch_leaf_check<LL, V, I + 1>(it, R, C, vec, bad);
  }
  return true;
}

// A leaf's ld of 0 in an item means its own row count.
template <class LL, int I = 0> void fill_default_ld(BatchMat& m, int64_t R, int64_t C) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    const int k = L::slot;
    if (m.ld[k] == 0) {
      const int64_t rows = L::mode == MN ? R : (L::mode == MT ? C : 1);
      m.ld[k] = rows > 0 ? rows : 1;
    }
    fill_default_ld<LL, I + 1>(m, R, C);
  }
}

template <class T, int NIN, int KIND, class Root>
fx_status run_batch(fx_expr* x, const Root& root, int64_t n, const fx_batch_item* items,
                    cudaStream_t st, int use_graph) {
  constexpr int kind = KIND;
  static_assert(NIN >= 1 && NIN <= 8, "batched trees take 1 to 8 inputs");
  using E = typename root_of<Root>::inner;
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  constexpr int V = vec_width<E, 16>();
  using TC_ = TileCfg<E, V>;
  constexpr int TR = TC_::TR, TCc = TC_::TC, NT = TC_::NT;
  const int n_in = NIN;
  if constexpr (root_of<Root>::kind == FX_KIND_DIM_REDUCE) {
    return fail(FX_E_UNSUPPORTED, "batched dim reductions are not fused");
  } else {
    constexpr int KIND0 = root_of<Root>::kind;
    if (kind == FX_KIND_MULTI && KIND0 != FX_KIND_ELEMENTWISE)
      return fail(FX_E_UNSUPPORTED, "multi-output needs an element-wise tree");
    if (!x->batch) x->batch = new (std::nothrow) BatchCache;
    if (!x->batch) return fail(FX_E_NOMEM, "out of host memory");
    BatchCacheEntry& c = x->batch->cur;
    uint64_t key = fnv1a(items, size_t(n) * sizeof(fx_batch_item));
    key = fnv1a(x->scal, sizeof x->scal, key);
    key = fnv1a(&n, sizeof n, key);
    const int zs = n_in;
    const bool has_z = kind != FX_KIND_FULL_REDUCE;
    const bool has_s = kind != FX_KIND_ELEMENTWISE;
    const int sslot = has_z ? n_in + 1 : n_in;
    if (key != c.key || !c.mats) {
      // validate and build the descriptors and the work-list
      std::vector<int64_t> order(n);
      for (int64_t i = 0; i < n; ++i) order[i] = i;
      std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return items[a].rows * items[a].cols > items[b].rows * items[b].cols;
      });
      std::vector<BatchMat> mats(n);
      std::vector<BatchItem> work;
      for (int64_t oi = 0; oi < n; ++oi) {
        const int64_t i = order[oi];
        const fx_batch_item& it = items[i];
        const int64_t R = it.rows, C = it.cols;
        if (R < 0 || C < 0) return fail(FX_E_SHAPE, "item %lld: negative shape", (long long)i);
        if (R > (int64_t(1) << 31) || C > (int64_t(1) << 31))
          return fail(FX_E_SHAPE, "item %lld: too large for a batch", (long long)i);
        bool vec = true;
        int bad = -1;
        if (!batch_leaf_check<LL, V>(it, R, C, vec, bad))
          return fail(FX_E_ARG, "item %lld: slot %d has a bad pointer or ld", (long long)i, bad);
        BatchMat& m = mats[i];
        memset(&m, 0, sizeof m);
        for (int k = 0; k < n_in; ++k) {
          m.p[k] = it.ptr[k];
          m.ld[k] = it.ld[k];
        }
        fill_default_ld<LL>(m, R, C);
        if (has_z) {
          const int64_t ldz = it.ld[zs] ? it.ld[zs] : (R > 0 ? R : 1);
          if (ldz < R || (R * C > 0 && !it.ptr[zs]) || !aligned(it.ptr[zs], sizeof(T)))
            return fail(FX_E_ARG, "item %lld: bad output Z", (long long)i);
          m.p[zs] = it.ptr[zs];
          m.ld[zs] = ldz;
          if (!aligned(it.ptr[zs], sizeof(T) * V) || ldz % V != 0) vec = false;
        }
        if (has_s) {
          if (!it.ptr[sslot] || !aligned(it.ptr[sslot], sizeof(CT)))
            return fail(FX_E_ARG, "item %lld: bad accu output", (long long)i);
          m.p[sslot] = it.ptr[sslot];
        }
        m.rows = R;
        m.cols = C;
        m.vec = vec ? 1 : 0;
        const int tcm = vec ? BatchShapes<E, V, TR, TCc, NT>::Vec::TC
                            : BatchShapes<E, V, TR, TCc, NT>::One::TC;
        const int64_t nt = ((R + TR - 1) / TR) * ((C + tcm - 1) / tcm);
        m.first = int64_t(work.size());
        m.ntiles = int32_t(nt);
        for (int64_t t = 0; t < nt; ++t) work.push_back(BatchItem{int32_t(i), int32_t(t)});
      }
      if (c.exec) {
        cudaGraphExecDestroy(c.exec);
        c.exec = nullptr;
      }
      const size_t bm = ((sizeof(BatchMat) * n) + 255) & ~size_t(255);
      const size_t bi = ((sizeof(BatchItem) * work.size()) + 255) & ~size_t(255);
      const size_t bp = sizeof(double2) * (work.size() > 0 ? work.size() : 1);
      FX_TRY(c.dev.ensure(bm + bi + bp, st));
      char* base = static_cast<char*>(c.dev.p);
      c.mats = reinterpret_cast<BatchMat*>(base);
      c.items = reinterpret_cast<BatchItem*>(base + bm);
      c.part = reinterpret_cast<double2*>(base + bm + bi);
      if (n > 0) FX_CUDA(cudaMemcpyAsync(c.mats, mats.data(), sizeof(BatchMat) * n, cudaMemcpyHostToDevice, st));
      if (!work.empty())
        FX_CUDA(cudaMemcpyAsync(c.items, work.data(), sizeof(BatchItem) * work.size(), cudaMemcpyHostToDevice, st));
      FX_CUDA(cudaStreamSynchronize(st));  // host vectors die at scope end
      c.key = key;
      c.n = n;
      c.nitems = int64_t(work.size());
    }
    const E& e = inner_of(root);
    Run r = run_of(x, st);
    auto launch_all = [&]() -> fx_status {
      if (c.nitems > 0) {
        auto go = [&](auto kern) -> fx_status {
          const int grid = grid_for(kern, NT, c.nitems, r.tune);
          kern<<<grid, NT, 0, st>>>(e, c.mats, c.items, c.nitems, c.part);
          return after_launch(r, "k_batch");
        };
        constexpr int KE = kind == FX_KIND_MULTI ? FX_KIND_MULTI : KIND0;
        FX_TRY(go(k_batch<E, T, V, TR, TCc, NT, KE, NIN>));
      }
      if (has_s && c.n > 0) {
        k_batch_combine<CT><<<unsigned((c.n + 7) / 8), 256, 0, st>>>(c.mats, c.n, c.part, sslot);
        FX_TRY(after_launch(r, "k_batch_combine"));
      }
      return FX_OK;
    };
    if (!use_graph || st == nullptr) return launch_all();
    if (!c.exec || c.exec_stream != st) {
      if (c.exec) {
        cudaGraphExecDestroy(c.exec);
        c.exec = nullptr;
      }
      FX_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      const int before = x->last_launches;
      fx_status s = launch_all();
      cudaGraph_t g = nullptr;
      cudaError_t ec = cudaStreamEndCapture(st, &g);
      if (s != FX_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
      cudaError_t ei = cudaGraphInstantiate(&c.exec, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate");
      c.exec_stream = st;
      x->last_launches = before;
    }
    FX_CUDA(cudaGraphLaunch(c.exec, st));
    x->last_launches += (c.nitems > 0 ? 1 : 0) + (has_s && c.n > 0 ? 1 : 0);
    return FX_OK;
  }
}

}  // namespace fx
