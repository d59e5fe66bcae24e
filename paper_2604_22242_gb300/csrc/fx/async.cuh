// async.cuh - asynchronous global->shared copies (cp.async) and the
// pipelined tiled kernel for single matrices with transposed leaves.
#pragma once

#include "bulk.cuh"

namespace fx {

// cp.async wrappers: 4-, 8- and 16-byte copies that complete in groups
// (commit_group / wait_group); 2-byte elements are copied through a register.
namespace cpa {
FX_D void copy4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tma::saddr(dst)), "l"(src) : "memory");
}
FX_D void copy8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tma::saddr(dst)), "l"(src) : "memory");
}
FX_D void copy16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tma::saddr(dst)), "l"(src) : "memory");
}
FX_D void commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> FX_D void wait_pending() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
template <int B> FX_D void copy(void* dst, const void* src) {
  if constexpr (B == 4) copy4(dst, src);
  else if constexpr (B == 8) copy8(dst, src);
  else {  // 2-byte elements: cp.async moves 4, 8 or 16 bytes, so copy through a register
    *static_cast<unsigned short*>(dst) = *static_cast<const unsigned short*>(src);
  }
}
}  // namespace cpa

// ---------------------------------------------------------------- single-matrix tiles
//
// k_tile_async: the tiled kernel for one matrix with transposed leaves,
// fed like k_batch_async by an NBUF-deep cp.async pipeline over the block's
// tiles, but vectorised: plain leaves arrive as 16-byte copies into
// column-major tiles, transposed leaves as 4-byte copies (element pairs for
// 2-byte types) into rows padded to an odd word count, and each thread
// evaluates V consecutive rows of P columns from shared memory and stores
// V-wide vectors. Requires every plain leaf and the output aligned for V
// (the host checks); vectors that reach past the last row use scalar
// copies and stores.

template <class T> FX_HD constexpr int trow_pad() { return sizeof(T) == 2 ? 2 : 1; }

template <class LL, int TR, int TC, int I = 0> FX_HD constexpr int tbuf_offset() {
  if constexpr (I == 0) {
    return 0;
  } else {
    using L = typename tl_at<LL, I - 1>::type;
    using T = typename L::elem;
    constexpr int es = int(sizeof(T));
    constexpr int sz = L::mode == MN ? TR * TC * es
                                     : (L::mode == MT ? TR * (TC + trow_pad<T>()) * es : 0);
    return tbuf_offset<LL, TR, TC, I - 1>() + ((sz + 127) / 128) * 128;
  }
}

template <class LL, int TR, int TC, int NT, int V, int I = 0>
FX_D void issue_vtile(char* buf, const Slots& sl, int64_t R, int64_t C, int64_t r0, int64_t c0) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    T* dst = reinterpret_cast<T*>(buf + tbuf_offset<LL, TR, TC, I>());
    const SlotView& sv = sl.s[L::slot];
    if constexpr (L::mode == MN) {
      constexpr int W = 16 / int(sizeof(T));
      static_assert(NT % (TR / W) == 0, "copy shape");
      const T* src = static_cast<const T*>(sv.p) + r0 + c0 * sv.ld;
      const int r = (threadIdx.x % (TR / W)) * W;
      const int64_t rleft = R - r0;
      for (int c = threadIdx.x / (TR / W); c < TC; c += NT / (TR / W)) {
        if (c0 + c >= C) break;
        if (r + W <= rleft) {
          cpa::copy16(dst + c * TR + r, src + r + c * sv.ld);
        } else {
          for (int j = 0; j < W && r + j < rleft; ++j)
            *(dst + c * TR + r + j) = sload(src + r + j + c * sv.ld);
        }
      }
    } else if constexpr (L::mode == MT) {
      // D element (c0 + c, r0 + r) -> row r, column c; CH elements per 4-byte copy
      constexpr int CH = sizeof(T) >= 4 ? 1 : 4 / int(sizeof(T));
      constexpr int SROW = TC + trow_pad<T>();
      static_assert(NT % (TC / CH) == 0, "copy shape");
      const T* src = static_cast<const T*>(sv.p) + c0 + r0 * sv.ld;
      const int c = (threadIdx.x % (TC / CH)) * CH;
      const int64_t cleft = C - c0;
      for (int r = threadIdx.x / (TC / CH); r < TR; r += NT / (TC / CH)) {
        if (r0 + r >= R) break;
        if (c + CH <= cleft) {
          cpa::copy<int(sizeof(T)) * CH>(dst + r * SROW + c, src + c + r * sv.ld);
        } else {
          for (int j = 0; j < CH && c + j < cleft; ++j)
            *(dst + r * SROW + c + j) = sload(src + c + j + r * sv.ld);
        }
      }
    }
    issue_vtile<LL, TR, TC, NT, V, I + 1>(buf, sl, R, C, r0, c0);
  }
}

// Rows r..r+V-1 of column c (tile-local) of every leaf from the stage.
template <class LL, int V, class CT, int TR, int TC, int I = 0>
FX_D void load_vtile(Pack<LL, V, CT>& p, const char* buf, const Slots& sl, int64_t r0, int64_t c0,
                     int r, int c, int nvalid) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    const T* b = reinterpret_cast<const T*>(buf + tbuf_offset<LL, TR, TC, I>());
    auto& dst = pget<I>::of(p);
    if constexpr (L::mode == MN) {
      dst = *reinterpret_cast<const Raw<T, V>*>(b + c * TR + r);
    } else if constexpr (L::mode == MT) {
      constexpr int SROW = TC + trow_pad<T>();
#pragma unroll
      for (int j = 0; j < V; ++j) dst.v[j] = to_compute<CT>(b[(r + j) * SROW + c]);
    } else if constexpr (L::mode == MBC) {
      const SlotView& s = sl.s[L::slot];
#pragma unroll
      for (int j = 0; j < V; ++j)
        dst.v[j] = j < nvalid ? sload(static_cast<const T*>(s.p) + (r0 + r + j) * s.vs) : T(0.0f);
    } else {
      const SlotView& s = sl.s[L::slot];
      dst.v[0] = sload(static_cast<const T*>(s.p) + (c0 + c) * s.vs);
    }
    load_vtile<LL, V, CT, TR, TC, I + 1>(p, buf, sl, r0, c0, r, c, nvalid);
  }
}

template <class E, class Epi, int V, int TR, int TC, int NT, int NBUF>
__global__ void __launch_bounds__(NT) k_tile_async(const E e, const Slots sl, const int64_t R,
                                                   const int64_t C, const Epi epi,
                                                   const RedArgs red) {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  constexpr int AB = tbuf_offset<LL, TR, TC, tl_size<LL>::value>();
  constexpr int TX = TR / V, TY = NT / TX, P = TC / TY;
  static_assert(TX * V == TR && TX * TY == NT && P * TY == TC, "tile shape");
  extern __shared__ __align__(128) char smem[];
  const int64_t tiles_r = (R + TR - 1) / TR, tiles_c = (C + TC - 1) / TC;
  const int64_t ntiles = tiles_r * tiles_c;
  const int64_t G = gridDim.x;
  const int64_t mine = ntiles > int64_t(blockIdx.x) ? (ntiles - blockIdx.x + G - 1) / G : 0;
  auto issue = [&](int64_t j) {
    if (j < mine) {
      int64_t tr, tc;
      tile_coords(blockIdx.x + j * G, tiles_r, tiles_c, tr, tc);
      issue_vtile<LL, TR, TC, NT, V>(smem + int(j % NBUF) * AB, sl, R, C, tr * TR, tc * TC);
    }
    cpa::commit();
  };
  typename Epi::State st;
  st.init();
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
#pragma unroll
  for (int j = 0; j < NBUF - 1; ++j) issue(j);
  for (int64_t j = 0; j < mine; ++j) {
    issue(j + NBUF - 1);
    cpa::wait_pending<NBUF - 1>();
    __syncthreads();
    int64_t tr, tc;
    tile_coords(blockIdx.x + j * G, tiles_r, tiles_c, tr, tc);
    const int64_t r0 = tr * TR, c0 = tc * TC;
    const char* buf = smem + int(j % NBUF) * AB;
    const int r = tx * V;
    const int nvalid = clamp_valid(R - r0 - r, V);
    if (nvalid > 0) {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int c = ty + q * TY;
        if (c0 + c < C) {
          Pack<LL, V, CT> p;
          load_vtile<LL, V, CT, TR, TC>(p, buf, sl, r0, c0, r, c, nvalid);
          CT v[V];
          eval_lanes<V>(e, p, v);
          epi_put(epi, st, (r0 + r) + (c0 + c) * epi.ldz, v, p, nvalid);
        }
      }
    }
    __syncthreads();
  }
  cpa::wait_pending<0>();
  if constexpr (Epi::reduces) finish_full_reduce<CT, Epi::sqrt_result>(st, red);
}

}  // namespace fx
