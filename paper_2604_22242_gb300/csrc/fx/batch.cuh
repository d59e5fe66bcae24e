// batch.cuh - one tree over many independent matrices of uneven shapes.
//
// The host builds a work-list: every matrix is cut into TR x TC tiles
// (matrices in decreasing size order, so the smallest tiles come last and
// fill the tail); one persistent launch (grid = SMs x resident blocks)
// walks the list with a static stride and runs the same tile body as the
// single-matrix tiled kernel (transposed leaves staged through shared
// memory). A tree with an accu output writes one compensated partial per
// warp of each tile; a second launch sums each matrix's partials in order
// in FP64 (one warp per matrix). The list, the descriptors and both launches are
// cached per item array (kept as a copy and compared whole on the next call);
// with use_graph the launches are captured once in a CUDA graph and replayed.
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
  // skewed tiles: every plain leaf and Z share one leading dimension and one
  // base alignment, so shifting each column's rows by its misalignment
  // (sbase + col * ld) mod W makes all their 16-byte chunks aligned
  int32_t skew;
  int32_t sbase;   // (first plain leaf's address / element size) mod W
};
struct BatchItem {
  int32_t mat;
  int32_t tile;
};

// ---------------------------------------------------------------- async tile pipeline
//
// k_batch_async: each block walks its work items (static stride) with an
// NBUF-deep pipeline. For the item NBUF-1 ahead, every thread issues
// asynchronous global->shared copies (cp.async) of the tile's plain leaves
// (stored column-major, TR rows per column; 16-byte chunks where the source
// allows, single elements elsewhere) and transposed leaves (stored as D's
// columns, TC+1 elements per row, so reads in output order avoid bank
// conflicts); then it waits for the item in front, evaluates the tile from
// shared memory V rows of a column per thread-step, stores Z (16-byte
// stores where aligned) and reduces. Copies cost shared memory instead of
// registers, and the item's descriptor is read one item ahead, so the
// dependent global loads leave the critical path.

// Per-item fields the evaluation needs, kept per buffer in shared memory.
struct TileDesc {
  const void* z;   // output Z (or null)
  int64_t ldz;
  int64_t R, C, r0, c0;
  int64_t item;
  int64_t sld;     // leading dimension the skew follows (0: no skew)
  int32_t mat;
  int32_t valid;
  int32_t sbase;
};

// Shared-memory layout of one buffer: plain leaves TC columns of TR rows,
// transposed leaves TR + W - 1 rows (the rows any column's skew can reach,
// W = 16 / element size) of TC+1 elements.
template <class LL, int TR, int TC, int I = 0> FX_HD constexpr int abuf_offset() {
  if constexpr (I == 0) {
    return 0;
  } else {
    using L = typename tl_at<LL, I - 1>::type;
    constexpr int es = int(sizeof(typename L::elem));
    constexpr int W = 16 / es;
    constexpr int sz = L::mode == MN ? TR * TC * es
                                     : (L::mode == MT ? (TR + W - 1) * (TC + 1) * es : 0);
    return abuf_offset<LL, TR, TC, I - 1>() + ((sz + 15) / 16) * 16;
  }
}
template <class LL, int TR, int TC> FX_HD constexpr int abuf_bytes() {
  return abuf_offset<LL, TR, TC, tl_size<LL>::value>();
}

// What issuing one item needs, read from global memory one item early.
template <int NIN> struct IssueDesc {
  const void* p[NIN];
  int64_t ld[NIN];
  const void* z;
  int64_t ldz, R, C, r0, c0, item, sld;
  int32_t mat, vec, valid, sbase;
};

// Row shift of tile column c: its rows are r0 - shift .. r0 - shift + TR - 1.
// W is a power of two, so the residue needs only the low 32 bits of the
// product and the sum.
template <int W> FX_D int col_skew(int64_t sld, int sbase, int64_t col) {
  static_assert((W & (W - 1)) == 0, "skew width is a power of two");
  return sld > 0 ? int((uint32_t(sbase) + uint32_t(col) * uint32_t(sld)) & uint32_t(W - 1)) : 0;
}

template <int NIN, int TR, int TC, int KIND, int KW>
FX_D IssueDesc<NIN> fetch_item(const BatchMat* mats, const BatchItem* items, int64_t it,
                               bool valid) {
  IssueDesc<NIN> d;
  d.valid = valid ? 1 : 0;
  if (!valid) return d;
  const BatchItem w = items[it];
  const BatchMat& m = mats[w.mat];
#pragma unroll
  for (int k = 0; k < NIN; ++k) {
    d.p[k] = m.p[k];
    d.ld[k] = m.ld[k];
  }
  d.z = KIND != FX_KIND_FULL_REDUCE ? m.p[NIN] : nullptr;
  d.ldz = KIND != FX_KIND_FULL_REDUCE ? m.ld[NIN] : 0;
  d.R = m.rows;
  d.C = m.cols;
  // 32-bit: a batch matrix has fewer than 2^31 tiles (64-bit division is a
  // long instruction sequence, executed here by every thread for every item)
  const uint32_t tiles_r = uint32_t((d.R + KW - 1 + TR - 1) / TR);  // rows plus the largest skew
  const uint32_t tc = uint32_t(w.tile) / tiles_r;
  d.r0 = int64_t(uint32_t(w.tile) - tc * tiles_r) * TR;
  d.c0 = int64_t(tc) * TC;
  d.item = it;
  d.mat = w.mat;
  d.vec = m.vec;
  d.sld = m.skew ? m.ld[m.skew - 1] : 0;
  d.sbase = m.sbase;
  return d;
}

// Copies of one item's tile. Plain leaves: thread t takes the W-element
// chunk (t % (TR/W)) of columns t / (TR/W), + NT/(TR/W), ... (W = 16 bytes
// of elements) and moves it with one 16-byte copy when its source is
// 16-byte aligned and wholly inside the matrix, else element by element
// (matrices of any shape and leading dimension). Transposed leaves: thread
// t takes element t % TC of D's columns t / TC, ...; stored as TR rows of
// TC + 1 elements. Offsets are 32-bit: a batch matrix holds fewer than
// 2^31 elements.
template <class LL, int TR, int TC, int NT, int NIN, int I = 0>
FX_D void issue_tile(char* buf, const IssueDesc<NIN>& d) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    T* dst = reinterpret_cast<T*>(buf + abuf_offset<LL, TR, TC, I>());
    const int ld = int(d.ld[L::slot]);
    const int rr = int(d.R - d.r0), cc = int(d.C - d.c0);  // rows / cols left in the matrix
    if constexpr (L::mode == MN) {
      // column c holds rows r0 - s_c .. r0 - s_c + TR - 1 (s_c its skew);
      // offsets from the tile's first column are 32-bit
      const T* src = static_cast<const T*>(d.p[L::slot]) + d.c0 * int64_t(ld);
      constexpr int W = 16 / int(sizeof(T));
      constexpr int CPC = TR / W;  // chunks per column
      static_assert(NT % CPC == 0 && TC % (NT / CPC) == 0, "chunk copy shape");
      const int q = (threadIdx.x % CPC) * W;
      const int R = int(d.R);
      const int r0 = int(d.r0);
      const uint32_t c0 = uint32_t(d.c0);
#pragma unroll
      for (int c = threadIdx.x / CPC; c < TC; c += NT / CPC) {
        if (c >= cc) break;
        const int row = r0 - col_skew<W>(d.sld, d.sbase, c0 + c) + q;
        const T* s = src + (row + c * ld);
        T* t = dst + c * TR + q;
        if (row >= 0 && row + W <= R && (reinterpret_cast<uintptr_t>(s) & 15) == 0) {
          cpa::copy16(t, s);
        } else {
#pragma unroll
          for (int j = 0; j < W; ++j)
            if (row + j >= 0 && row + j < R) cpa::copy<int(sizeof(T))>(t + j, s + j);
        }
      }
    } else if constexpr (L::mode == MT) {
      // output rows r0 - (W - 1) .. r0 + TR - 1: stored row k is output row
      // r0 - (W - 1) + k, i.e. D's column of that index. The stored rows
      // inside the matrix are kb .. ke - 1; each thread walks its share of
      // them with pointer steps.
      constexpr int W = 16 / int(sizeof(T));
      constexpr int KS = NT / TC;  // stored rows per pass of the block
      static_assert(NT % TC == 0, "transposed copy shape");
      const int rlo = int(d.r0) - (W - 1);
      const int kb = rlo < 0 ? -rlo : 0;
      const int left = int(d.R) - rlo;
      const int ke = left < TR + W - 1 ? left : TR + W - 1;
      const int c = threadIdx.x % TC;  // D element (c0 + c, rlo + k)
      if (c < cc) {
        int k = threadIdx.x / TC;
        if (k < kb) k += ((kb - k + KS - 1) / KS) * KS;
        const T* s = static_cast<const T*>(d.p[L::slot]) + d.c0 + c + int64_t(rlo + k) * ld;
        T* t = dst + k * (TC + 1) + c;
        const int64_t step = int64_t(KS) * ld;
        for (; k < ke; k += KS) {
          cpa::copy<int(sizeof(T))>(t, s);
          s += step;
          t += KS * (TC + 1);
        }
      }
    }
    issue_tile<LL, TR, TC, NT, NIN, I + 1>(buf, d);
  }
}

// Slots i..i+V-1 of tile column c of every leaf (skew sk: output rows
// r0 - sk + i ..; lanes outside the matrix are marked in `ok`).
template <class LL, int V, class CT, int TR, int TC, int I = 0>
FX_D void load_tile_vec(Pack<LL, V, CT>& p, const char* buf, const BatchMat& m, int64_t r0,
                        int64_t c0, int i, int c, int sk, const bool (&ok)[V]) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    constexpr int W = 16 / int(sizeof(T));
    const T* b = reinterpret_cast<const T*>(buf + abuf_offset<LL, TR, TC, I>());
    auto& dst = pget<I>::of(p);
    if constexpr (L::mode == MN) {
      dst = *reinterpret_cast<const Raw<T, V>*>(b + c * TR + i);
    } else if constexpr (L::mode == MT) {
#pragma unroll
      for (int j = 0; j < V; ++j)
        dst.v[j] = to_compute<CT>(b[(i + j - sk + W - 1) * (TC + 1) + c]);
    } else if constexpr (L::mode == MBC) {
      const T* q = static_cast<const T*>(m.p[L::slot]) + (r0 - sk + i);
#pragma unroll
      for (int j = 0; j < V; ++j) dst.v[j] = ok[j] ? sload(q + j) : T(0.0f);
    } else {
      dst.v[0] = sload(static_cast<const T*>(m.p[L::slot]) + (c0 + c));
    }
    load_tile_vec<LL, V, CT, TR, TC, I + 1>(p, buf, m, r0, c0, i, c, sk, ok);
  }
}

// Per-warp tile partials: FP32 pairs for FP32 trees (no FP64 conversion on
// the hot kernel's slow FP64 pipe; the combine widens them), FP64 pairs for
// FP64 trees. The partial buffer holds double2 slots either way.
FX_D void store_partial(double2* part, int64_t i, float s, float c) {
  reinterpret_cast<float2*>(part)[i] = make_float2(s, c);
}
FX_D void store_partial(double2* part, int64_t i, double s, double c) {
  part[i] = make_double2(s, c);
}
template <class RT> FX_D double2 load_partial(const double2* part, int64_t i) {
  if constexpr (std::is_same<RT, double>::value) {
    return __ldcg(part + i);
  } else {
    const float2 f = __ldcg(reinterpret_cast<const float2*>(part) + i);
    return make_double2(double(f.x), double(f.y));
  }
}

// VC: consecutive slots of one column a thread evaluates per step (its
// vector width: 16 bytes of elements, or half that); copies and skews stay
// in 16-byte chunks of W elements.
template <class E, class T, int TR, int TC, int NT, int NBUF, int KIND, int NIN, int VC>
__global__ void __launch_bounds__(NT) k_batch_async(const E e, const BatchMat* __restrict__ mats,
                                                    const BatchItem* __restrict__ items,
                                                    const int64_t nitems, double2* part) {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  constexpr int AB = abuf_bytes<LL, TR, TC>();
  constexpr int W = 16 / int(sizeof(T));  // elements of a 16-byte chunk; the largest row skew + 1
  constexpr int V = VC;
  static_assert(V >= 1 && W % V == 0, "vector width divides the chunk");
  extern __shared__ __align__(128) char smem[];
  TileDesc* desc = reinterpret_cast<TileDesc*>(smem + NBUF * AB);
  const int64_t G = gridDim.x;
  const int64_t mine = nitems > int64_t(blockIdx.x) ? (nitems - blockIdx.x + G - 1) / G : 0;
  auto fetch = [&](int64_t j) {
    return fetch_item<NIN, TR, TC, KIND, W>(mats, items, blockIdx.x + j * G, j < mine);
  };
  // issue a fetched item into buffer b (every thread commits a group, even an empty one)
  auto issue = [&](const IssueDesc<NIN>& d, int b) {
    if (d.valid) {
      issue_tile<LL, TR, TC, NT, NIN>(smem + b * AB, d);
      if (threadIdx.x == 0)
        desc[b] = TileDesc{d.z, d.ldz, d.R, d.C, d.r0, d.c0, d.item, d.sld, d.mat, 1, d.sbase};
    }
    cpa::commit();
  };
#pragma unroll
  for (int j = 0; j < NBUF - 1; ++j) issue(fetch(j), j);
  IssueDesc<NIN> next = fetch(NBUF - 1);
  for (int64_t j = 0; j < mine; ++j) {
    issue(next, int((j + NBUF - 1) % NBUF));
    next = fetch(j + NBUF);  // consumed one iteration later: its loads overlap this tile
    cpa::wait_pending<NBUF - 1>();
    __syncthreads();  // every thread's copies of item j have landed; desc visible
    const int b = int(j % NBUF);
    const TileDesc d = desc[b];
    const BatchMat& m = mats[d.mat];
    // V consecutive slots of one column per step (column c's rows start at
    // r0 - skew); a thread adds at most TR*TC/NT values of a tile: a plain
    // sum, merged compensated per warp
    constexpr int RG = TR / V;  // row groups per column
    static_assert(NT % RG == 0 && TC % (NT / RG) == 0, "consumer shape");
    CT tsum = CT(0);
    const char* buf = smem + b * AB;
    const int i = (threadIdx.x % RG) * V;
    const int cc = int(d.C - d.c0);
    const int R = int(d.R);
    const int r0 = int(d.r0);
    const uint32_t c0 = uint32_t(d.c0);
    const int ldz = int(d.ldz);
    // Z from the tile's first column on; offsets inside a matrix are 32-bit
    T* z = KIND != FX_KIND_FULL_REDUCE
               ? static_cast<T*>(const_cast<void*>(d.z)) + d.c0 * int64_t(ldz)
               : nullptr;
#pragma unroll
    for (int c = threadIdx.x / RG; c < TC; c += NT / RG) {
      if (c < cc) {
        const int sk = col_skew<W>(d.sld, d.sbase, c0 + c);
        const int row = r0 - sk + i;  // output row of slot i
        Pack<LL, V, CT> p;
        CT v[V];
        if (row >= 0 && row + V <= R) {  // all V slots inside the matrix
          bool all[V];
#pragma unroll
          for (int j = 0; j < V; ++j) all[j] = true;
          load_tile_vec<LL, V, CT, TR, TC>(p, buf, m, d.r0, d.c0, i, c, sk, all);
          eval_lanes<V>(e, p, v);
          if constexpr (KIND != FX_KIND_FULL_REDUCE) {
            T* q = z + (row + c * ldz);
            if ((reinterpret_cast<uintptr_t>(q) & uintptr_t(V * sizeof(T) - 1)) == 0) {
              Raw<T, V> o;
#pragma unroll
              for (int j = 0; j < V; ++j) o.v[j] = narrow_to<T>::from(v[j]);
              vstore(q, o);
            } else {
#pragma unroll
              for (int j = 0; j < V; ++j) sstore(q + j, narrow_to<T>::from(v[j]));
            }
          }
          if constexpr (KIND != FX_KIND_ELEMENTWISE) {
#pragma unroll
            for (int j = 0; j < V; ++j) tsum += v[j];
          }
        } else if (row + V > 0 && row < R) {  // some slots inside
          bool ok[V];
#pragma unroll
          for (int j = 0; j < V; ++j) ok[j] = row + j >= 0 && row + j < R;
          load_tile_vec<LL, V, CT, TR, TC>(p, buf, m, d.r0, d.c0, i, c, sk, ok);
          eval_lanes<V>(e, p, v);
          if constexpr (KIND != FX_KIND_FULL_REDUCE) {
            T* q = z + (row + c * ldz);
#pragma unroll
            for (int j = 0; j < V; ++j)
              if (ok[j]) sstore(q + j, narrow_to<T>::from(v[j]));
          }
          if constexpr (KIND != FX_KIND_ELEMENTWISE) {
#pragma unroll
            for (int j = 0; j < V; ++j)
              if (ok[j]) tsum += v[j];
          }
        }
      }
    }
    if constexpr (KIND != FX_KIND_ELEMENTWISE) {
      // one partial per warp of the tile, in warp order: part[item * NW + w]
      std::conditional_t<std::is_same<CT, double>::value, PlainSum<CT>, CompSum<CT>> st;
      st.s = tsum;
      st.c = CT(0);
      warp_merge(st);
      if ((threadIdx.x & 31) == 0)
        store_partial(part, d.item * (NT / 32) + threadIdx.x / 32, st.s, st.c);
    }
    __syncthreads();  // buffer b is free for the item issued next
  }
  cpa::wait_pending<0>();
}

// One warp per matrix: its tiles' per-warp partials (nw per tile), in
// order, summed in FP64.
template <class RT>
__global__ void __launch_bounds__(256) k_batch_combine(const BatchMat* __restrict__ mats,
                                                       const int64_t nmat, const double2* part,
                                                       const int sslot, const int nw) {
  const int64_t i = int64_t(blockIdx.x) * 8 + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (i >= nmat) return;  // whole warps leave together
  const BatchMat& m = mats[i];
  std::conditional_t<std::is_same<RT, double>::value, CompSum<double>, PlainSum<double>> a;
  a.init();
  for (int64_t k = lane; k < int64_t(m.ntiles) * nw; k += 32) {
    const double2 q = load_partial<RT>(part, m.first * nw + k);
    a.add(q.x);
    a.add(q.y);
  }
  warp_merge(a);
  if (lane == 0) *static_cast<RT*>(const_cast<void*>(m.p[sslot])) = RT(a.s + a.c);
}

struct BatchCacheEntry {
  // the item array and scalars the descriptors were built from: a call
  // reuses them (and the captured graph) only when both compare equal
  std::vector<fx_batch_item> items_seen;
  double scal_seen[FX_MAX_SCALARS] = {};
  bool built = false;
  int64_t n = 0, nitems = 0;
  Workspace dev;  // descriptors, items, partials
  BatchMat* mats = nullptr;
  BatchItem* items = nullptr;
  double2* part = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t exec_stream = nullptr;
  int exec_shape[4] = {0, 0, 0, 0};  // launch shape the graph was captured with
};

}  // namespace fx

struct fx::BatchCache {
  BatchCacheEntry cur;
};

namespace fx {

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

// The batched kernel addresses a matrix's elements with 32-bit offsets
// (column * ld + row inside a tile, 32-bit tile indices): every matrix
// operand of an item must span fewer than 2^31 elements.
constexpr int64_t kBatchSpan = int64_t(1) << 31;
inline bool batch_span_ok(int64_t rows, int64_t cols, int64_t ld) {
  return rows * cols == 0 || (ld < kBatchSpan && ld * (cols - 1) + rows < kBatchSpan);
}
template <class LL, int I = 0>
bool batch_extent_check(const fx_batch_item& it, int64_t R, int64_t C, int& bad) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    const int k = L::slot;
    if constexpr (L::mode == MN || L::mode == MT) {
      const int64_t rows = L::mode == MT ? C : R, cols = L::mode == MT ? R : C;
      const int64_t ld = it.ld[k] ? it.ld[k] : (rows > 0 ? rows : 1);
      if (!batch_span_ok(rows, cols, ld)) {
        bad = k;
        return false;
      }
    }
    return batch_extent_check<LL, I + 1>(it, R, C, bad);
  }
  return true;
}

// Plain leaves of a batch matrix: one leading dimension, one base alignment
// modulo `align` bytes? `first` receives the first plain leaf's slot.
template <class LL, int I = 0> bool skew_check(const BatchMat& m, int& first, int align) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    if constexpr (L::mode == MN) {
      const int k = L::slot;
      if (first < 0) {
        first = k;
      } else if (m.ld[k] != m.ld[first] ||
                 reinterpret_cast<uintptr_t>(m.p[k]) % uintptr_t(align) !=
                     reinterpret_cast<uintptr_t>(m.p[first]) % uintptr_t(align)) {
        return false;
      }
    }
    return skew_check<LL, I + 1>(m, first, align);
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
  constexpr bool dbl = std::is_same<CT, double>::value;
  constexpr int TR = dbl ? 32 : 64, TCc = 64;
  constexpr int NTMAX = 512;  // partials are sized for the largest block
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
    const bool same = c.built && c.mats && c.n == n &&
                      memcmp(c.scal_seen, x->scal, sizeof c.scal_seen) == 0 &&
                      (n == 0 || memcmp(c.items_seen.data(), items,
                                        size_t(n) * sizeof(fx_batch_item)) == 0);
    const int zs = n_in;
    const bool has_z = kind != FX_KIND_FULL_REDUCE;
    const bool has_s = kind != FX_KIND_ELEMENTWISE;
    const int sslot = has_z ? n_in + 1 : n_in;
    if (!same) {
      c.built = false;
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
        if (R >= kBatchSpan || C >= kBatchSpan)
          return fail(FX_E_SHAPE, "item %lld: too large for a batch", (long long)i);
        bool vec = true;
        int bad = -1;
        if (!batch_leaf_check<LL, V>(it, R, C, vec, bad))
          return fail(FX_E_ARG, "item %lld: slot %d has a bad pointer or ld", (long long)i, bad);
        if (!batch_extent_check<LL>(it, R, C, bad))
          return fail(FX_E_SHAPE, "item %lld: slot %d spans 2^31 elements or more (batch limit)",
                      (long long)i, bad);
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
          if (!batch_span_ok(R, C, ldz))
            return fail(FX_E_SHAPE, "item %lld: Z spans 2^31 elements or more (batch limit)",
                        (long long)i);
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
        // skewed tiles when every plain leaf and Z share ld and base alignment
        {
          constexpr int W = 16 / int(sizeof(T));
          int first = -1;
          bool ok = skew_check<LL>(m, first, W * int(sizeof(T)));
          if (ok && first >= 0 && has_z) {
            const uintptr_t a0 = reinterpret_cast<uintptr_t>(m.p[first]) % uintptr_t(W * sizeof(T));
            ok = m.ld[zs] == m.ld[first] &&
                 reinterpret_cast<uintptr_t>(m.p[zs]) % uintptr_t(W * sizeof(T)) == a0;
          }
          m.skew = (ok && first >= 0) ? first + 1 : 0;
          m.sbase = m.skew ? int((reinterpret_cast<uintptr_t>(m.p[first]) / sizeof(T)) % W) : 0;
        }
        // row tiles cover R plus the largest skew (W - 1 rows)
        const int64_t nt = (R > 0 && C > 0)
                               ? ((R + 16 / int64_t(sizeof(T)) - 1 + TR - 1) / TR) * ((C + TCc - 1) / TCc)
                               : 0;
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
      const size_t bp = sizeof(double2) * (NTMAX / 32) * (work.size() > 0 ? work.size() : 1);
      FX_TRY(c.dev.ensure(bm + bi + bp, st));
      char* base = static_cast<char*>(c.dev.p);
      c.mats = reinterpret_cast<BatchMat*>(base);
      c.items = reinterpret_cast<BatchItem*>(base + bm);
      c.part = reinterpret_cast<double2*>(base + bm + bi);
      if (n > 0) FX_CUDA(cudaMemcpyAsync(c.mats, mats.data(), sizeof(BatchMat) * n, cudaMemcpyHostToDevice, st));
      if (!work.empty())
        FX_CUDA(cudaMemcpyAsync(c.items, work.data(), sizeof(BatchItem) * work.size(), cudaMemcpyHostToDevice, st));
      FX_CUDA(cudaStreamSynchronize(st));  // host vectors die at scope end
      c.items_seen.assign(items, items + n);
      memcpy(c.scal_seen, x->scal, sizeof c.scal_seen);
      c.built = true;
      c.n = n;
      c.nitems = int64_t(work.size());
    }
    const E& e = inner_of(root);
    Run r = run_of(x, st);
    // Launch shape (tunable, fx_tune_batch): threads per block 256 or 512
    // (512 not for 2-byte types), 2, 3 or 4 pipeline stages (unroll 2, 4,
    // 8), blocks per SM (0: as many as fit), and the vector width a thread
    // evaluates per step (pipeline 1: 8 bytes of elements; otherwise 16).
    const int NTsel = (r.tune.block >= 512 && sizeof(T) != 2) ? 512 : 256;
    const int NBsel = r.tune.unroll <= 2 ? 2 : (r.tune.unroll >= 8 ? 4 : 3);
    const int VHsel = r.tune.pipe == 1 ? 1 : 0;
    constexpr int VW = 16 / int(sizeof(T));
    auto launch_one = [&](auto nt_c, auto nb_c) -> fx_status {
      constexpr int NT = decltype(nt_c)::value, NBUF = decltype(nb_c)::value;
      constexpr int KE = kind == FX_KIND_MULTI ? FX_KIND_MULTI : KIND0;
      auto kern = VHsel ? k_batch_async<E, T, TR, TCc, NT, NBUF, KE, NIN, VW / 2>
                        : k_batch_async<E, T, TR, TCc, NT, NBUF, KE, NIN, VW>;
      constexpr int smem = NBUF * abuf_bytes<LL, TR, TCc>() + NBUF * int(sizeof(TileDesc));
      FX_TRY(allow_smem(kern, smem));
      const int sms = device_sms() > 0 ? device_sms() : 1;
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
      }
      const int bps = r.tune.bps > 0 ? (r.tune.bps < occ ? r.tune.bps : occ) : occ;
      int64_t grid = int64_t(sms) * bps;
      if (grid > c.nitems) grid = c.nitems;
      kern<<<unsigned(grid), NT, smem, st>>>(e, c.mats, c.items, c.nitems, c.part);
      return after_launch(r, "k_batch_async");
    };
    using I256 = std::integral_constant<int, 256>;
    using I512 = std::integral_constant<int, (sizeof(T) == 2 ? 256 : 512)>;
    using B2 = std::integral_constant<int, 2>;
    using B3 = std::integral_constant<int, 3>;
    using B4 = std::integral_constant<int, 4>;
    auto launch_all = [&]() -> fx_status {
      if (c.nitems > 0) {
        if (NTsel == 512) {
          if (NBsel == 2) FX_TRY(launch_one(I512{}, B2{}));
          else if (NBsel == 4) FX_TRY(launch_one(I512{}, B4{}));
          else FX_TRY(launch_one(I512{}, B3{}));
        } else {
          if (NBsel == 2) FX_TRY(launch_one(I256{}, B2{}));
          else if (NBsel == 4) FX_TRY(launch_one(I256{}, B4{}));
          else FX_TRY(launch_one(I256{}, B3{}));
        }
      }
      if (has_s && c.n > 0) {
        k_batch_combine<CT><<<unsigned((c.n + 7) / 8), 256, 0, st>>>(c.mats, c.n, c.part, sslot,
                                                                     NTsel / 32);
        FX_TRY(after_launch(r, "k_batch_combine"));
      }
      return FX_OK;
    };
    if (!use_graph || st == nullptr) return launch_all();
    const int shape[4] = {NTsel, NBsel, r.tune.bps, VHsel};
    if (!c.exec || c.exec_stream != st || memcmp(shape, c.exec_shape, sizeof shape) != 0) {
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
      memcpy(c.exec_shape, shape, sizeof shape);
      x->last_launches = before;
    }
    FX_CUDA(cudaGraphLaunch(c.exec, st));
    x->last_launches += (c.nitems > 0 ? 1 : 0) + (has_s && c.n > 0 ? 1 : 0);
    return FX_OK;
  }
}

}  // namespace fx
