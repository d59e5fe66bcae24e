// umma.cuh - a matrix product on the fifth-generation tensor cores with the
// tree's element-wise remainder evaluated in its epilogue (BF16 / FP16).
//
// A tree with one matrix product P = op(X) op(Y) (Fig. 1's Z = 2 X Y^T, or
// Z = sigmoid(0.5 X Y + W)) is a fusion boundary for the element-wise
// kernels: P(i, j) needs a whole row and column. Through a library GEMM the
// product is written to memory and read back by the fused pass. Here the
// product stays on chip: each CTA computes a 128 x 256 tile of P with
// tcgen05.mma into tensor memory (TMEM, FP32 accumulation), and its epilogue
// reads the tile back from TMEM and evaluates the rest of the tree - the
// lifted tree, in which P is a leaf - element by element, reading the other
// leaves (W) from global memory and writing Z once.
//
// Persistent: one CTA of 192 threads per SM walks the output tiles (in
// groups of 16 tile rows, for L2 reuse of the operands):
//   warp 0      lane 0 loads the operand tiles with TMA (cp.async.bulk.tensor,
//               128-byte swizzle) into a ring of NS shared-memory stages,
//               one mbarrier per stage counting the bytes in ("full");
//   warp 1      allocates the TMEM (512 columns: two accumulators); lane 0
//               issues, per 64-deep K step, four tcgen05.mma (M 128, N 256,
//               K 16) into the tile's accumulator and commits them to the
//               stage's "empty" mbarrier (the stage is free again when they
//               have read it); after the tile's last step it commits to the
//               accumulator's "full" barrier, and before reusing an
//               accumulator it waits until the epilogue has read it out;
//   warps 2..5  wait for a tile's accumulator, load their 32 TMEM lanes
//               (rows) 16 columns at a time (tcgen05.ld 32x32b), release the
//               accumulator after the last load, evaluate the remainder and
//               store - while the next tile is multiplied into the other
//               accumulator. The other leaves' values for the next 16
//               columns are loaded before the current ones are computed.
//
// Operand layouts: column-major storage makes an operand K-major (K
// contiguous) when it is read transposed or is the right factor, and
// MN-major otherwise; the shared-memory matrix descriptors describe both
// canonical 128-byte-swizzled layouts:
//   K-major:  rows of 128 bytes along K, 8-row groups 1024 bytes apart
//             (stride byte offset 1024); a K step of 16 elements moves the
//             start address by 32 bytes inside the swizzle row;
//   MN-major: 64-element (128-byte) rows along M or N, one row per K index,
//             8-row groups 1024 bytes apart (stride byte offset), 64-element
//             blocks of M or N 8192 bytes apart (leading byte offset); a K
//             step of 16 moves the start address by 16 rows (2048 bytes).
// Every wait is bounded (bulk.cuh); a thread that gives up records the
// error, the MMA thread still commits "acc" (after whatever it issued), the
// producer waits for its copies in flight, and the TMEM is always freed.
#pragma once

#include "tmatile.cuh"

namespace fx {
namespace umma {

constexpr int BM = 128, BN = 256, BK = 64, UK = 16;
constexpr int SA = BM * BK * 2;       // A tile of one stage (16 KB)
constexpr int SB = BN * BK * 2;       // B tile of one stage (32 KB)
constexpr int STAGE = SA + SB;
constexpr int NS = 4;                 // stages
constexpr uint32_t TMEM_COLS = 512;   // two FP32 accumulators of 128 lanes x 256 columns

// Shared-memory matrix descriptor (sm_100 family): start address, leading
// and stride byte offsets (all >> 4), the fixed version bits 46-48 = 0b001,
// and the 128-byte swizzle mode (2) in bits 61-63.
FX_D uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B formats (bits 7-9, 10-12: 0 FP16, 1 BF16, the same for both),
// A and B major-ness (bits 15, 16: 1 = MN-major), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28).
template <class T, bool AMN, bool BMN>
FX_HD constexpr uint32_t idesc() {
  constexpr uint32_t fmt = std::is_same<T, bf16>::value ? 1u : 0u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(AMN) << 15) | (uint32_t(BMN) << 16) |
         (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
}

FX_D void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   tma::saddr(slot)),
               "r"(ncols)
               : "memory");
}
FX_D void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
FX_D void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// D (TMEM) = A * B (+ D when acc != 0)
FX_D void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
// Arrive on `bar` once every tcgen05.mma this thread issued has completed.
FX_D void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   tma::saddr(bar))
               : "memory");
}
FX_D void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
FX_D void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 16 consecutive FP32 columns of this thread's TMEM lane (warp-wide).
FX_D void ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
FX_D void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Element context of the epilogue: the product leaf (slot PS) is the FP32
// accumulator; every other leaf is a plain matrix leaf whose values for the
// thread's CW columns were loaded into w[leaf index][column].
template <class LL, int PS, class T, int CW> struct ECtx {
  using CT = float;
  const T (*w)[CW];
  float acc;
  int j;
  template <int K, int M> FX_D float leaf() const {
    if constexpr (K == PS) {
      return acc;
    } else {
      static_assert(M == MN, "the remainder's other leaves are plain matrices");
      return to_compute<float>(w[tl_index<LL, K, M>::value][j]);
    }
  }
};

// An ordered 2-byte load (volatile, memory clobber): the epilogue's loads
// of the next chunk are issued before the current chunk is computed and
// stored, and the compiler may not sink them next to their use.
template <class TL> FX_D TL ld_ordered(const TL* p) {
  static_assert(sizeof(TL) == 2, "16-bit leaves");
  unsigned short v;
  asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  TL r;
  *reinterpret_cast<unsigned short*>(&r) = v;
  return r;
}

// w[I][j] = leaf I at (m, n0 + j), j < nn (plain leaves other than PS).
template <class LL, int PS, class T, int CW, int I = 0>
FX_D void load_others(T (*w)[CW], const Slots& sl, int64_t m, int64_t n0, int nn) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    if constexpr (L::slot != PS) {
      const SlotView& s = sl.s[L::slot];
      const T* p = static_cast<const T*>(s.p) + m + n0 * s.ld;
#pragma unroll
      for (int j = 0; j < CW; ++j)
        if (j < nn) w[I][j] = ld_ordered(p + int64_t(j) * s.ld);
    }
    load_others<LL, PS, T, CW, I + 1>(w, sl, m, n0, nn);
  }
}

struct Bars {
  uint64_t full[NS];
  uint64_t empty[NS];
  uint64_t accf[2];   // accumulator buffer b complete (MMA commit)
  uint64_t acce[2];   // accumulator buffer b read out (one arrival per epilogue warp)
  uint64_t drain;     // every MMA of the CTA complete (before the TMEM is freed)
  uint32_t taddr;
  volatile int abort;
};

// Tile t of a tiles_m x tiles_n grid, in groups of GM tile rows: inside a
// group the tile rows run fastest, so the tiles in flight at once (one per
// SM) cover GM rows of A and a few column blocks of B, which stay in L2.
constexpr int GM = 16;
FX_D void tile_of(int t, int tiles_m, int tiles_n, int& tm, int& tn) {
  const int group = t / (GM * tiles_n);
  const int first = group * GM;
  const int gsize = tiles_m - first < GM ? tiles_m - first : GM;
  const int within = t - group * GM * tiles_n;
  tm = first + within % gsize;
  tn = within / gsize;
}

constexpr int CW = 16;   // epilogue columns per TMEM load

// Z (M x N, column-major, ldz) = E(P) with P = op(A) op(B) of K terms, on a
// persistent grid: CTA b takes tiles b, b + gridDim.x, ... The MMA warp
// alternates between two TMEM accumulators (columns 0..255 and 256..511),
// so the epilogue of one tile runs while the next tile is multiplied.
// AMN / BMN: the A / B tiles are MN-major (else K-major). PS: the slot of
// the product leaf in E.
template <class T, bool AMN, bool BMN, class E, int PS>
__global__ void __launch_bounds__(192, 1)
    k_gemm_umma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const E e, const Slots sl, T* z, const int64_t ldz, const int M, const int N,
                const int K, unsigned int* err) {
  using LL = leaves_t<E>;
  constexpr int NL = tl_size<LL>::value;
  extern __shared__ char smem_raw[];
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                       ~uintptr_t(1023));
  Bars& bars = *reinterpret_cast<Bars*>(smem + NS * STAGE);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  const int ntiles = tiles_m * tiles_n;
  const int nk = (K + BK - 1) / BK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      tma::mbar_init(&bars.full[s], 1);
      tma::mbar_init(&bars.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tma::mbar_init(&bars.accf[b], 1);
      tma::mbar_init(&bars.acce[b], 4);
    }
    tma::mbar_init(&bars.drain, 1);
    bars.abort = 0;
    tma::fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&bars.taddr, TMEM_COLS);
    tmem_relinquish();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = bars.taddr;

  if (warp == 0) {
    if (lane == 0) {  // producer: every tile's K steps through one ring
      uint32_t g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int tm, tn;
        tile_of(t, tiles_m, tiles_n, tm, tn);
        const int m0 = tm * BM, n0 = tn * BN;
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int s = int(g % NS);
          if (g >= uint32_t(NS) && !tma::wait(&bars.empty[s], ((g - NS) / NS) & 1u, err)) {
            ok = false;
            break;
          }
          char* sa = smem + s * STAGE;
          char* sb = sa + SA;
          const int k0 = kt * BK;
          // boxes that start outside the matrix are skipped (their rows or
          // columns of the product are never stored); partly outside boxes
          // read zeros there
          uint32_t bytes = 0;
          if (AMN) {
            bytes += uint32_t(m0 < M) * (SA / 2) + uint32_t(m0 + 64 < M) * (SA / 2);
          } else {
            bytes += SA;
          }
          if (BMN) {
#pragma unroll
            for (int j = 0; j < 4; ++j) bytes += uint32_t(n0 + 64 * j < N) * (SB / 4);
          } else {
            bytes += SB;
          }
          tma::arrive_expect_tx(&bars.full[s], bytes);
          if (AMN) {
            if (m0 < M) tma::load_2d(sa, &mapA, m0, k0, &bars.full[s]);
            if (m0 + 64 < M) tma::load_2d(sa + SA / 2, &mapA, m0 + 64, k0, &bars.full[s]);
          } else {
            tma::load_2d(sa, &mapA, k0, m0, &bars.full[s]);
          }
          if (BMN) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (n0 + 64 * j < N)
                tma::load_2d(sb + j * (SB / 4), &mapB, n0 + 64 * j, k0, &bars.full[s]);
          } else {
            tma::load_2d(sb, &mapB, k0, n0, &bars.full[s]);
          }
        }
      }
      if (!ok) {  // wait (bounded) for the copies still in flight
        bars.abort = 1;
        for (uint32_t j = (g > uint32_t(NS) ? g - NS : 0); j < g; ++j)
          tma::wait(&bars.full[j % NS], (j / NS) & 1u, nullptr);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t ID = idesc<T, AMN, BMN>();
      uint32_t g = 0;
      int i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const int b = i & 1;
        // the epilogue has read out what this buffer held two tiles ago
        if (i >= 2 && !tma::wait(&bars.acce[b], uint32_t((i - 2) / 2) & 1u, err)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t tacc = tbase + uint32_t(b * BN);
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int s = int(g % NS);
          if (!tma::wait(&bars.full[s], (g / NS) & 1u, err)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sa = tma::saddr(smem + s * STAGE);
          const uint32_t sb = sa + SA;
#pragma unroll
          for (int k = 0; k < BK / UK; ++k) {
            const uint64_t ad = AMN ? desc(sa + k * UK * 128, SA / 2, 1024)
                                    : desc(sa + k * UK * 2, 16, 1024);
            const uint64_t bd = BMN ? desc(sb + k * UK * 128, SB / 4, 1024)
                                    : desc(sb + k * UK * 2, 16, 1024);
            mma(tacc, ad, bd, ID, (kt > 0 || k > 0) ? 1u : 0u);
          }
          commit(&bars.empty[s]);
        }
        if (ok) commit(&bars.accf[b]);
      }
      if (!ok) {  // wake the epilogue (it sees the abort) after what was issued
        bars.abort = 1;
        commit(&bars.accf[0]);
        commit(&bars.accf[1]);
      }
      commit(&bars.drain);
      tma::wait(&bars.drain, 0u, err);
    }
    __syncwarp();
  } else {  // epilogue: warps 2..5 take TMEM lane quarters 2, 3, 0, 1
    const int q = warp & 3;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int b = i & 1;
      const bool ready = tma::wait(&bars.accf[b], uint32_t(i / 2) & 1u, err);
      fence_after();
      // the TMEM loads below are warp-wide: the warp decides together
      if (!__all_sync(0xffffffffu, ready && !bars.abort)) break;
      int tm, tn;
      tile_of(t, tiles_m, tiles_n, tm, tn);
      const int64_t m = int64_t(tm) * BM + q * 32 + lane;
      const int n0 = tn * BN;
      const bool row = m < M;
      T wn[NL][CW], wc[NL][CW];
      if (row) load_others<LL, PS, T, CW>(wn, sl, m, n0, N - n0 < CW ? N - n0 : CW);
#pragma unroll 1
      for (int c = 0; c < BN / CW; ++c) {
        const int nc = n0 + c * CW;
        uint32_t r[CW];
        ld16(tbase + uint32_t(b * BN) + (uint32_t(q * 32) << 16) + uint32_t(c * CW), r);
        wait_ld();
        if (c == BN / CW - 1) {  // the accumulator buffer is free for the MMA warp
          fence_before();
          __syncwarp();
          if (lane == 0) tma::arrive(&bars.acce[b]);
        }
        if (nc >= N) continue;  // warp-uniform
        const int nn = N - nc < CW ? N - nc : CW;
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
          for (int j = 0; j < CW; ++j) wc[l][j] = wn[l][j];
        const int nx = nc + CW;
        if (row && c + 1 < BN / CW && nx < N)
          load_others<LL, PS, T, CW>(wn, sl, m, nx, N - nx < CW ? N - nx : CW);
        if (row) {
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            if (j < nn) {
              ECtx<LL, PS, T, CW> cx{wc, __uint_as_float(r[j]), j};
              sstore(z + m + int64_t(nc + j) * ldz, narrow_to<T>::from(e.ev(cx)));
            }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tbase, TMEM_COLS);
  }
}

}  // namespace umma

// ---------------------------------------------------------------- host side

// 2-D tensor map of a column-major matrix (dims {d0 contiguous, d1}, stride
// ld elements) with a (b0 x b1) box and the 128-byte swizzle; false when
// TMA cannot address it (16-byte aligned base and stride, extents < 2^31).
template <class T>
bool encode_map(CUtensorMap* m, const void* p, int64_t d0, int64_t d1, int64_t ld, int b0, int b1) {
  auto enc = tensor_map_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(p) & 15) != 0 || d0 < 1 || d1 < 1 || ld < d0) return false;
  if ((ld * int64_t(sizeof(T))) % 16 != 0 || d0 >= (int64_t(1) << 31) || d1 >= (int64_t(1) << 31))
    return false;
  const cuuint64_t dims[2] = {cuuint64_t(d0), cuuint64_t(d1)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * sizeof(T)};
  const cuuint32_t box[2] = {cuuint32_t(b0), cuuint32_t(b1)};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, tmap_dtype<T>(), 2, const_cast<void*>(p), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Leaves of the remainder other than the product: plain matrices of type T.
template <class LL, int PS, class T, int I = 0> constexpr bool others_plain() {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    constexpr bool ok = L::slot == PS || (L::mode == MN && std::is_same<typename L::elem, T>::value);
    return ok && others_plain<LL, PS, T, I + 1>();
  } else {
    return true;
  }
}

// The product node of a tree with exactly one (a type search).
template <class E> struct the_prod;
template <class L, class R> struct the_prod<Prod<L, R>> {
  using type = Prod<L, R>;
  static FX_HD const type& get(const Prod<L, R>& p) { return p; }
};
template <class Op, class L, class R> struct the_prod<Bin<Op, L, R>> {
  using S = std::conditional_t<has_prod<L>::value, L, R>;
  using type = typename the_prod<S>::type;
  static FX_HD const type& get(const Bin<Op, L, R>& e) {
    if constexpr (has_prod<L>::value) return the_prod<L>::get(e.l);
    else return the_prod<R>::get(e.r);
  }
};
template <class Op, class E> struct the_prod<Un<Op, E>> {
  using type = typename the_prod<E>::type;
  static FX_HD const type& get(const Un<Op, E>& e) { return the_prod<E>::get(e.e); }
};
template <class Op, class E> struct the_prod<SL<Op, E>> {
  using type = typename the_prod<E>::type;
  static FX_HD const type& get(const SL<Op, E>& e) { return the_prod<E>::get(e.e); }
};
template <class Op, class E> struct the_prod<SR<Op, E>> {
  using type = typename the_prod<E>::type;
  static FX_HD const type& get(const SR<Op, E>& e) { return the_prod<E>::get(e.e); }
};

template <class E> struct prod_of_leaves { static constexpr bool value = false; };
template <int K1, int M1, int K2, int M2, class T1, class T2>
struct prod_of_leaves<Prod<Leaf<K1, T1, M1>, Leaf<K2, T2, M2>>> {
  static constexpr bool value = (M1 == MN || M1 == MT) && (M2 == MN || M2 == MT) &&
                                std::is_same<T1, T2>::value;
};

}  // namespace fx
