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
// Per CTA (192 threads, one CTA per SM):
//   warp 0      lane 0 loads the operand tiles with TMA (cp.async.bulk.tensor,
//               128-byte swizzle) into a ring of NS shared-memory stages,
//               one mbarrier per stage counting the bytes in ("full");
//   warp 1      allocates the TMEM accumulator (256 columns); lane 0 issues,
//               per 64-deep K step, four tcgen05.mma (M 128, N 256, K 16)
//               and commits them to the stage's "empty" mbarrier (the stage
//               is free again when they have read it), and after the last
//               step commits to "acc" (the accumulator is complete);
//   warps 2..5  wait for "acc", load their 32 TMEM lanes (rows) 32 columns at
//               a time (tcgen05.ld 32x32b), evaluate the remainder and store.
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
constexpr uint32_t TMEM_COLS = 256;   // FP32 accumulator: 128 lanes x 256 columns

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
// 32 consecutive FP32 columns of this thread's TMEM lane (warp-wide).
FX_D void ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
FX_D void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Element context of the epilogue: the product leaf (slot PS) is the FP32
// accumulator; every other leaf is a plain matrix leaf whose values for the
// thread's 32 columns were loaded into vals[leaf index][column].
template <class LL, int PS> struct ECtx {
  using CT = float;
  const float (*vals)[32];
  float acc;
  int j;
  template <int K, int M> FX_D float leaf() const {
    if constexpr (K == PS) {
      return acc;
    } else {
      static_assert(M == MN, "the remainder's other leaves are plain matrices");
      return vals[tl_index<LL, K, M>::value][j];
    }
  }
};

// vals[I][j] = leaf I at (m, n0 + j), j < nn (plain leaves other than PS).
template <class LL, int PS, int I = 0>
FX_D void load_others(float (*vals)[32], const Slots& sl, int64_t m, int64_t n0, int nn) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    if constexpr (L::slot != PS) {
      using TL_ = typename L::elem;
      const SlotView& s = sl.s[L::slot];
      const TL_* p = static_cast<const TL_*>(s.p) + m + n0 * s.ld;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        vals[I][j] = j < nn ? to_compute<float>(sload(p + int64_t(j) * s.ld)) : 0.0f;
    }
    load_others<LL, PS, I + 1>(vals, sl, m, n0, nn);
  }
}

struct Bars {
  uint64_t full[NS];
  uint64_t empty[NS];
  uint64_t acc;
  uint32_t taddr;
  volatile int abort;
};

// Z (M x N, column-major, ldz) = E(P) with P = op(A) op(B) of K terms.
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
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int nk = (K + BK - 1) / BK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      tma::mbar_init(&bars.full[s], 1);
      tma::mbar_init(&bars.empty[s], 1);
    }
    tma::mbar_init(&bars.acc, 1);
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
    if (lane == 0) {  // producer
      int kt = 0;
      bool ok = true;
      for (; kt < nk; ++kt) {
        const int s = kt % NS;
        if (kt >= NS && !tma::wait(&bars.empty[s], uint32_t(((kt - NS) / NS) & 1), err)) {
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
            if (n0 + 64 * j < N) tma::load_2d(sb + j * (SB / 4), &mapB, n0 + 64 * j, k0, &bars.full[s]);
        } else {
          tma::load_2d(sb, &mapB, k0, n0, &bars.full[s]);
        }
      }
      if (!ok) {
        bars.abort = 1;
        for (int j = (kt > NS ? kt - NS : 0); j < kt; ++j)
          tma::wait(&bars.full[j % NS], uint32_t((j / NS) & 1), nullptr);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t ID = idesc<T, AMN, BMN>();
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % NS;
        if (!tma::wait(&bars.full[s], uint32_t((kt / NS) & 1), err)) {
          bars.abort = 1;
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
          mma(tbase, ad, bd, ID, (kt > 0 || k > 0) ? 1u : 0u);
        }
        commit(&bars.empty[s]);
      }
      commit(&bars.acc);
    }
    __syncwarp();
  } else {  // epilogue: warps 2..5 take TMEM lane quarters 2, 3, 0, 1
    const int q = warp & 3;
    const bool ready = tma::wait(&bars.acc, 0u, err);
    fence_after();
    const int64_t m = int64_t(m0) + q * 32 + lane;
    // the TMEM loads below are warp-wide: the warp decides together
    const bool go = __all_sync(0xffffffffu, ready && !bars.abort);
    if (go) {
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        const int nc = n0 + c * 32;
        uint32_t r[32];
        ld32(tbase + (uint32_t(q * 32) << 16) + uint32_t(c * 32), r);
        wait_ld();
        if (nc >= N) continue;  // warp-uniform
        const int nn = N - nc < 32 ? N - nc : 32;
        if (m < M) {
          float vals[NL][32];
          load_others<LL, PS>(vals, sl, m, nc, nn);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < nn) {
              ECtx<LL, PS> cx{vals, __uint_as_float(r[j]), j};
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
