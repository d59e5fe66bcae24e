// tmatile.cuh - tiles of trees with transposed leaves, moved by the tensor
// memory accelerator (TMA).
//
// The tiled path of a tree with trans() leaves (Sec. 3: the transposed
// leaf is read with its indices swapped) needs both the plain leaves and the
// transposed ones read along their own columns. Here every plain leaf, every
// transposed leaf and the output are described by a 2-D tensor map, and a
// TT x TT output tile moves as whole boxes: one producer thread issues
// cp.async.bulk.tensor loads of each leaf's tile into a ring of shared-memory
// stages (an mbarrier per stage counts the bytes in), the consumer threads
// evaluate the tree from shared memory and write the output tile back to
// shared memory, and one consumer thread stores it with a single
// cp.async.bulk.tensor store per box. Boxes are 128 bytes wide in their
// inner dimension and use the 128-byte swizzle, so both the column-vector
// reads of plain leaves and the row-wise reads of transposed leaves are free
// of bank conflicts. Ragged edges come for free: loads outside the matrix
// read zeros, stores outside it are dropped, and reductions mask the lanes
// outside it.
//
// Each consumer thread evaluates V = 16 / sizeof(T) consecutive rows of one
// column at a time; the 32 lanes of a warp take 32 consecutive columns.
// Every wait on an mbarrier is bounded (see bulk.cuh); a consumer that gives
// up records the error and all consumers leave the tile loop together at
// the next block-wide barrier.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "async.cuh"
#include "runtime.hpp"

namespace fx {

// Tensor maps, indexed by slot (inputs, then outputs).
struct TileMaps {
  CUtensorMap m[FX_MAX_SLOTS];
};

namespace tma {
// 2-D tiled load of the box at (x, y) (x the inner, contiguous coordinate)
// into shared memory, completing its bytes on `bar`.
FX_D void load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}
// 2-D tiled store of a shared-memory box to (x, y), tracked by bulk groups.
FX_D void store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   map),
               "r"(x), "r"(y), "r"(saddr(src))
               : "memory");
}
FX_D void store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// At most N committed store groups still reading shared memory.
template <int N> FX_D void store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// At most N committed store groups not yet complete.
template <int N> FX_D void store_wait() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}
}  // namespace tma

// Tile geometry for storage type T: boxes IB x TT (IB elements = 128 bytes
// along the contiguous dimension), tiles TT x TT, NB boxes per leaf tile.
template <class T> struct TmaGeom {
  static constexpr int es = int(sizeof(T));
  static constexpr int IB = 128 / es;
  static constexpr int TT = es == 8 ? 32 : 64;
  static constexpr int NB = TT / IB;
  static constexpr int V = 16 / es;
  static constexpr int BOX = 128 * TT;
  static constexpr int LEAF = NB * BOX;
  static_assert(NB * IB == TT && V * es == 16, "tile geometry");
};

// Byte offset of element (i along the 128-byte rows, o across them) in a
// box written with the 128-byte swizzle (16-byte chunk index XOR row % 8;
// box bases 1024-byte aligned).
template <int ES> FX_HD constexpr int swz(int i, int o) {
  return o * 128 + ((((i * ES) >> 4) ^ (o & 7)) << 4) + ((i * ES) & 15);
}

// Leaves moved by TMA (plain and transposed) and the rank of leaf I among them.
template <class LL, int I = 0> FX_HD constexpr int count_tma() {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    return (L::mode == MN || L::mode == MT ? 1 : 0) + count_tma<LL, I + 1>();
  } else {
    return 0;
  }
}
template <class LL, int I, int J = 0> FX_HD constexpr int tma_rank() {
  if constexpr (J < I) {
    using L = typename tl_at<LL, J>::type;
    return (L::mode == MN || L::mode == MT ? 1 : 0) + tma_rank<LL, I, J + 1>();
  } else {
    return 0;
  }
}
// Every TMA leaf has storage type T.
template <class LL, class T, int I = 0> FX_HD constexpr bool tma_uniform() {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    constexpr bool ok = !(L::mode == MN || L::mode == MT) || std::is_same<typename L::elem, T>::value;
    return ok && tma_uniform<LL, T, I + 1>();
  } else {
    return true;
  }
}

// Every TMA leaf (K, MN) has its transpose (K, MT) in the tree and the
// other way round. Such a tree is square (leaf K is both R x C and C x R),
// and the boxes loaded for output tile (i, j) are exactly those that tile
// (j, i) needs, with the two modes of each leaf trading places.
template <class LL, int I = 0> FX_HD constexpr bool flip_closed() {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    constexpr bool ok = !(L::mode == MN || L::mode == MT) ||
                        tl_index<LL, L::slot, flip_mode(L::mode)>::value >= 0;
    return ok && flip_closed<LL, I + 1>();
  } else {
    return count_tma<LL>() > 0;
  }
}

// Symmetric work items: tile pairs {(i, j), (j, i)} with i <= j, numbered
// column by column (item q = j (j + 1) / 2 + i).
FX_D void sym_pair(int64_t q, int64_t& i, int64_t& j) {
  // FP32 estimate (FP64 is slow on this part), then exact integer fix-up
  int64_t jj = int64_t((sqrtf(8.0f * float(q) + 1.0f) - 1.0f) * 0.5f);
  if (jj < 0) jj = 0;
  while ((jj + 1) * (jj + 2) / 2 <= q) ++jj;
  while (jj * (jj + 1) / 2 > q) --jj;
  j = jj;
  i = q - jj * (jj + 1) / 2;
}

// Producer: the boxes of tile (r0, c0) of every TMA leaf into `stage`;
// boxes that start outside the matrix are skipped. Returns the bytes issued.
template <class LL, class T, int I = 0>
FX_D uint32_t issue_tma_tile(char* stage, const TileMaps& maps, int64_t R, int64_t C, int r0,
                             int c0, uint64_t* bar) {
  using G = TmaGeom<T>;
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    uint32_t bytes = 0;
    if constexpr (L::mode == MN || L::mode == MT) {
      char* dst = stage + tma_rank<LL, I>() * G::LEAF;
      const CUtensorMap* m = &maps.m[L::slot];
#pragma unroll
      for (int b = 0; b < G::NB; ++b) {
        if constexpr (L::mode == MN) {
          if (r0 + b * G::IB < R) {
            tma::load_2d(dst + b * G::BOX, m, r0 + b * G::IB, c0, bar);
            bytes += G::BOX;
          }
        } else {
          if (c0 + b * G::IB < C) {
            tma::load_2d(dst + b * G::BOX, m, c0 + b * G::IB, r0, bar);
            bytes += G::BOX;
          }
        }
      }
    }
    return bytes + issue_tma_tile<LL, T, I + 1>(stage, maps, R, C, r0, c0, bar);
  } else {
    return 0;
  }
}

// Bytes issue_tma_tile will issue for tile (r0, c0) (for expect_tx, which
// must be armed before the first copy can complete).
template <class LL, class T>
FX_D uint32_t tma_tile_bytes(int64_t R, int64_t C, int r0, int c0) {
  using G = TmaGeom<T>;
  int nr = 0, nc = 0;
#pragma unroll
  for (int b = 0; b < G::NB; ++b) {
    nr += (r0 + b * G::IB < R) ? 1 : 0;
    nc += (c0 + b * G::IB < C) ? 1 : 0;
  }
  return uint32_t(count_mode<LL>(MN) * nr + count_mode<LL>(MT) * nc) * uint32_t(G::BOX);
}

// Consumer: rows r..r+V-1 of tile column c of every leaf. SWAP: the stage
// holds the boxes of the transposed tile, so each TMA leaf reads the region
// its flipped twin was loaded into.
template <class LL, class T, class CT, bool SWAP = false, int I = 0>
FX_D void load_tma_pack(Pack<LL, TmaGeom<T>::V, CT>& p, const char* stage, const Slots& sl,
                        int64_t r0, int64_t c0, int r, int c, int nvalid) {
  using G = TmaGeom<T>;
  constexpr int V = G::V;
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using TL_ = typename L::elem;
    auto& dst = pget<I>::of(p);
    constexpr int J = (SWAP && (L::mode == MN || L::mode == MT))
                          ? tl_index<LL, L::slot, flip_mode(L::mode)>::value
                          : I;
    const char* base = stage + tma_rank<LL, J>() * G::LEAF;
    if constexpr (L::mode == MN) {
      const char* q = base + (r / G::IB) * G::BOX + swz<G::es>(r % G::IB, c);
      dst = *reinterpret_cast<const Raw<T, V>*>(q);
    } else if constexpr (L::mode == MT) {
      const char* b = base + (c / G::IB) * G::BOX;
      const int i = c % G::IB;
#pragma unroll
      for (int j = 0; j < V; ++j)
        dst.v[j] = to_compute<CT>(*reinterpret_cast<const T*>(b + swz<G::es>(i, r + j)));
    } else if constexpr (L::mode == MBC) {
      const SlotView& s = sl.s[L::slot];
      const TL_* q = static_cast<const TL_*>(s.p) + (r0 + r) * s.vs;
#pragma unroll
      for (int j = 0; j < V; ++j) dst.v[j] = j < nvalid ? sload(q + j * s.vs) : TL_(0.0f);
    } else {
      const SlotView& s = sl.s[L::slot];
      dst.v[0] = sload(static_cast<const TL_*>(s.p) + (c0 + c) * s.vs);
    }
    load_tma_pack<LL, T, CT, SWAP, I + 1>(p, stage, sl, r0, c0, r, c, nvalid);
  }
}

constexpr int kTmaMaxStages = 8;

// SYM (trees whose TMA leaves are closed under transposition): one work
// item is the tile pair {(i, j), (j, i)}, loaded once and evaluated twice,
// so each input element is read once instead of twice.
template <class E, class Epi, class T, int NTC, bool SYM = false>
__global__ void __launch_bounds__(NTC + 32) k_tile_tma(const E e, const Slots sl, const int64_t R,
                                                        const int64_t C, const Epi epi,
                                                        const RedArgs red,
                                                        const __grid_constant__ TileMaps maps,
                                                        const int zslot, const int ns,
                                                        unsigned int* err) {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  using G = TmaGeom<T>;
  constexpr int V = G::V, TT = G::TT;
  constexpr int SB = count_tma<LL>() * G::LEAF;       // one stage
  constexpr int NPT = (TT / V) * TT / NTC;             // vectors per thread per tile
  static_assert(NPT * NTC == (TT / V) * TT, "tile / thread shape");
  static_assert(!SYM || flip_closed<LL>(), "symmetric items need a transpose-closed tree");
  constexpr bool ST = Epi::stores;
  constexpr int ZT = SYM ? 2 : 1;                      // output tiles per item
  extern __shared__ char smem_raw[];
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  char* zbuf = smem + ns * SB;                         // two items' output tiles when storing
  Ring<kTmaMaxStages>& ring =
      *reinterpret_cast<Ring<kTmaMaxStages>*>(zbuf + (ST ? 2 * ZT * G::LEAF : 0));
  const int64_t tiles_r = (R + TT - 1) / TT, tiles_c = (C + TT - 1) / TT;
  const int64_t nitems = SYM ? tiles_r * (tiles_r + 1) / 2 : tiles_r * tiles_c;
  const int64_t G_ = gridDim.x;
  const int64_t mine = nitems > int64_t(blockIdx.x) ? (nitems - blockIdx.x + G_ - 1) / G_ : 0;
  const int tid = threadIdx.x;
  // output tile of item t: (tr, tc), and for SYM also (tc, tr) when tr != tc
  auto coords = [&](int64_t t, int64_t& tr, int64_t& tc) {
    if constexpr (SYM) sym_pair(t, tr, tc);
    else tile_coords(t, tiles_r, tiles_c, tr, tc);
  };
  if (tid == 0) {
    for (int i = 0; i < ns; ++i) {
      tma::mbar_init(&ring.full[i], 1);
      tma::mbar_init(&ring.empty[i], NTC);
    }
    ring.abort = 0;
    tma::fence_mbar_init();
  }
  __syncthreads();
  typename Epi::State st;
  st.init();
  if (tid >= NTC) {
    // producer: lane 0 of the last warp
    if (tid == NTC) {
      bool ok = true;
      int64_t k = 0;
      for (; k < mine; ++k) {
        const int s = int(k % ns);
        if (k >= ns && !tma::wait(&ring.empty[s], uint32_t(((k - ns) / ns) & 1), err)) {
          ok = false;
          break;
        }
        int64_t tr, tc;
        coords(blockIdx.x + k * G_, tr, tc);
        const int r0 = int(tr * TT), c0 = int(tc * TT);
        tma::arrive_expect_tx(&ring.full[s], tma_tile_bytes<LL, T>(R, C, r0, c0));
        issue_tma_tile<LL, T>(smem + s * SB, maps, R, C, r0, c0, &ring.full[s]);
      }
      if (!ok) {
        for (int64_t j = (k > ns ? k - ns : 0); j < k; ++j)
          tma::wait(&ring.full[j % ns], uint32_t((j / ns) & 1), nullptr);
      }
    }
  } else {
    // one output tile at (r0, c0) from the stage; SWAP reads the transposed tile's boxes
    auto tile = [&](const char* stage, int64_t r0, int64_t c0, char* zt, auto swap) {
      constexpr bool SW = decltype(swap)::value;
#pragma unroll
      for (int q = 0; q < NPT; ++q) {
        const int vi = tid + q * NTC;
        const int c = vi % TT, r = (vi / TT) * V;
        const int nvalid = (c0 + c < C) ? clamp_valid(R - r0 - r, V) : 0;
        Pack<LL, V, CT> p;
        load_tma_pack<LL, T, CT, SW>(p, stage, sl, r0, c0, r, c, nvalid);
        CT v[V];
        eval_lanes<V>(e, p, v);
        if constexpr (ST) {
          Raw<T, V> o;
#pragma unroll
          for (int j = 0; j < V; ++j) o.v[j] = narrow_to<T>::from(v[j]);
          *reinterpret_cast<Raw<T, V>*>(zt + (r / G::IB) * G::BOX + swz<G::es>(r % G::IB, c)) = o;
        }
        if constexpr (Epi::side_tree) {
          epi.put_side(st, p, nvalid);
        } else if constexpr (Epi::reduces) {
          if (nvalid == V) {
            CT w[V];
#pragma unroll
            for (int j = 0; j < V; ++j) w[j] = Epi::sqrt_result ? v[j] * v[j] : v[j];
            st.add(lane_sum(w));
          } else {
#pragma unroll
            for (int j = 0; j < V; ++j)
              if (j < nvalid) st.add(Epi::sqrt_result ? v[j] * v[j] : v[j]);
          }
        }
      }
    };
    auto store_tile = [&](int64_t r0, int64_t c0, const char* zt) {
#pragma unroll
      for (int b = 0; b < G::NB; ++b)
        if (r0 + b * G::IB < R) tma::store_2d(&maps.m[zslot], int(r0) + b * G::IB, int(c0), zt + b * G::BOX);
    };
    for (int64_t k = 0; k < mine; ++k) {
      const int s = int(k % ns);
      if (!tma::wait(&ring.full[s], uint32_t((k / ns) & 1), err)) ring.abort = 1;
      if constexpr (ST) {
        if (tid == 0 && k >= 2) tma::store_wait_read<1>();  // output tiles of item k-2 read out
      }
      block_sync(NTC);
      if (ring.abort) break;  // uniform: set only before this barrier
      int64_t tr, tc;
      coords(blockIdx.x + k * G_, tr, tc);
      const int64_t r0 = tr * TT, c0 = tc * TT;
      const char* stage = smem + s * SB;
      char* zt = zbuf + int(k & 1) * ZT * G::LEAF;
      tile(stage, r0, c0, zt, std::false_type{});
      const bool second = SYM && tr != tc;
      if constexpr (SYM) {
        if (second) tile(stage, c0, r0, zt + G::LEAF, std::true_type{});
      }
      tma::arrive(&ring.empty[s]);
      if constexpr (ST) {
        tma::fence_proxy_async();  // this thread's output writes, visible to the TMA store
        block_sync(NTC);
        if (tid == 0) {
          store_tile(r0, c0, zt);
          if (second) store_tile(c0, r0, zt + G::LEAF);
          tma::store_commit();
        }
      }
    }
    if constexpr (ST) {
      if (tid == 0) tma::store_wait<0>();
    }
  }
  if constexpr (Epi::reduces) finish_full_reduce<CT, Epi::sqrt_result>(st, red);
}

// ---------------------------------------------------------------- host side

// cuTensorMapEncodeTiled from the CUDA driver, found once through the runtime.
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    cudaGetLastError();
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

template <class T> constexpr CUtensorMapDataType tmap_dtype() {
  if constexpr (std::is_same<T, float>::value) return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  else if constexpr (std::is_same<T, double>::value) return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  else if constexpr (std::is_same<T, bf16>::value) return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  else return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
}

// Tensor map of a rows x cols column-major matrix (leading dimension ld)
// with IB x TT boxes; false when TMA cannot address it (base not 16-byte
// aligned, ld * sizeof(T) not a multiple of 16, extents beyond int32).
template <class T>
bool encode_tile_map(CUtensorMap* m, const void* p, int64_t rows, int64_t cols, int64_t ld) {
  using G = TmaGeom<T>;
  auto enc = tensor_map_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(p) & 15) != 0 || rows < 1 || cols < 1 || ld < rows) return false;
  if ((ld * int64_t(sizeof(T))) % 16 != 0 || rows >= (int64_t(1) << 31) || cols >= (int64_t(1) << 31))
    return false;
  const cuuint64_t dims[2] = {cuuint64_t(rows), cuuint64_t(cols)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * sizeof(T)};
  const cuuint32_t box[2] = {cuuint32_t(G::IB), cuuint32_t(G::TT)};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, tmap_dtype<T>(), 2, const_cast<void*>(p), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Maps of every plain and transposed leaf; false if one cannot be encoded.
template <class LL, class T, int I = 0> bool encode_leaf_maps(TileMaps& tm, const Binding* b) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    if constexpr (L::mode == MN || L::mode == MT) {
      const Binding& x = b[L::slot];
      if (!encode_tile_map<T>(&tm.m[L::slot], x.p, x.rows, x.cols, x.ld)) return false;
    }
    return encode_leaf_maps<LL, T, I + 1>(tm, b);
  }
  return true;
}

}  // namespace fx
