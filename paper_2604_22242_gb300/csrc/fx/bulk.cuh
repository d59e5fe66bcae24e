// bulk.cuh - row-range kernels fed by bulk asynchronous copies (TMA).
//
// The row-decomposed kernels (sum/max along dim 1, the fused backward)
// give each thread V consecutive rows and walk the columns. Fed by
// per-thread vector loads, their bytes in flight are bounded by registers.
// Here one producer warp copies, for every column of the block's range, the
// block's row segment of every plain leaf (TRB contiguous elements) into a
// ring of NS shared-memory stages with cp.async.bulk, and signals each
// stage on an mbarrier ("full"); the NT consumer threads read their rows
// from shared memory, and release the stage on a second mbarrier
// ("empty") that the producer waits on before refilling it. Bytes in flight
// then cost shared memory, not registers.
//
// Every wait is bounded: after kSpinLimit polls a thread records
// kErrTimeout in the error word and stops; consumers still reach the
// epilogue (which then skips the cross-block combine), and the producer
// waits (bounded again) for the copies it has issued before it exits.
#pragma once

#include "kernels.cuh"

namespace fx {

constexpr unsigned int kErrTimeout = 1u;
constexpr uint32_t kSpinLimit = 1u << 20;   // polls of try_wait (each may suspend <= 4 us)

namespace tma {

FX_D uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

FX_D void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
FX_D void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
FX_D void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
FX_D void arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
               : "memory");
}
FX_D void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
// Global -> shared bulk copy completing `bytes` transactions on `bar`.
// dst and src 16-byte aligned, bytes a multiple of 16.
FX_D void copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar))
      : "memory");
}
FX_D bool try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 4096; "
      "selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of `bar`; false (and the error recorded) on timeout.
FX_D bool wait(uint64_t* bar, uint32_t parity, unsigned int* err, uint32_t limit = kSpinLimit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (try_wait(bar, parity)) return true;
  if (err) atomicOr(err, kErrTimeout);
  return false;
}

}  // namespace tma

// Plain (MN) leaves: their count and the byte offset of leaf I in a stage.
template <class LL, int I = 0> FX_HD constexpr int count_mn() {
  if constexpr (I < tl_size<LL>::value) {
    return (tl_at<LL, I>::type::mode == MN ? 1 : 0) + count_mn<LL, I + 1>();
  } else {
    return 0;
  }
}
template <class LL, int TRB, int I, int J = 0> FX_HD constexpr int stage_offset() {
  if constexpr (J < I) {
    using L = typename tl_at<LL, J>::type;
    constexpr int sz = L::mode == MN ? ((TRB * int(sizeof(typename L::elem)) + 127) / 128) * 128 : 0;
    return sz + stage_offset<LL, TRB, I, J + 1>();
  } else {
    return 0;
  }
}
template <class LL, int TRB> FX_HD constexpr int stage_bytes() {
  return stage_offset<LL, TRB, tl_size<LL>::value>();
}

// Producer: issue column `col` of every plain leaf into stage `st`.
template <class LL, int TRB, int I = 0>
FX_D void issue_column(char* stage, const Slots& sl, int64_t r0, int64_t col, int rows,
                       uint64_t* bar) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    if constexpr (L::mode == MN) {
      using T = typename L::elem;
      const SlotView& s = sl.s[L::slot];
      const T* src = static_cast<const T*>(s.p) + r0 + col * s.ld;
      tma::copy_g2s(stage + stage_offset<LL, TRB, I>(), src, uint32_t(rows * sizeof(T)), bar);
    }
    issue_column<LL, TRB, I + 1>(stage, sl, r0, col, rows, bar);
  }
}
template <class LL, int I = 0> FX_HD constexpr int column_tx_bytes_per_row() {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    return (L::mode == MN ? int(sizeof(typename L::elem)) : 0) + column_tx_bytes_per_row<LL, I + 1>();
  } else {
    return 0;
  }
}

// Consumer: the thread's V rows of column c, plain leaves from the stage,
// vectors from `hold` (loaded once per block), each_row scalars from global.
// FULL: the caller knows that all V rows are inside the matrix.
template <class LL, int V, class CT, int TRB, bool FULL = false, int I = 0>
FX_D void load_stage(Pack<LL, V, CT>& p, const Pack<LL, V, CT>& hold, const char* stage,
                     const Slots& sl, int t, int64_t c, int nvalid) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    auto& dst = pget<I>::of(p);
    if constexpr (L::mode == MN) {
      const T* q = reinterpret_cast<const T*>(stage + stage_offset<LL, TRB, I>()) + t * V;
      if (FULL || nvalid == V) {
        dst = *reinterpret_cast<const Raw<T, V>*>(q);
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j) dst.v[j] = j < nvalid ? q[j] : T(0.0f);
      }
    } else if constexpr (L::mode == MBC) {
      dst = pget<I>::of(hold);
    } else if constexpr (L::mode == MBR) {
      const SlotView& s = sl.s[L::slot];
      dst.v[0] = sload(static_cast<const T*>(s.p) + c * s.vs);
    }
    load_stage<LL, V, CT, TRB, FULL, I + 1>(p, hold, stage, sl, t, c, nvalid);
  }
}

// The per-thread rows of each_col leaves, once per block.
template <class LL, int V, class CT, int I = 0>
FX_D void load_hold(Pack<LL, V, CT>& p, const Slots& sl, int64_t r, int nvalid) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    if constexpr (L::mode == MBC) {
      const SlotView& s = sl.s[L::slot];
      const T* q = static_cast<const T*>(s.p) + r * s.vs;
#pragma unroll
      for (int j = 0; j < V; ++j) pget<I>::of(p).v[j] = j < nvalid ? sload(q + j * s.vs) : T(0.0f);
    }
    load_hold<LL, V, CT, I + 1>(p, sl, r, nvalid);
  }
}

// Shared state of one block: the stage ring and its barriers.
template <int NS> struct Ring {
  uint64_t full[NS];
  uint64_t empty[NS];
  volatile int abort;  // set by a consumer whose bounded wait gave up
};

// The producer warp's loop (lane 0 issues): columns cb..ce-1 of rows
// r0..r0+rows-1 into the ring, CPS columns per stage. On a timeout it
// stops issuing and waits (bounded) for the copies already in flight.
template <class LL, int TRB, int NS, int CPS>
FX_D void produce(char* stages, Ring<NS>& ring, const Slots& sl, int64_t r0, int rows, int64_t cb,
                  int64_t ce, unsigned int* err) {
  if ((threadIdx.x & 31) != 0) return;
  constexpr int SBC = stage_bytes<LL, TRB>();  // one column
  const uint32_t tx_col = uint32_t(rows) * column_tx_bytes_per_row<LL>();
  const int64_t nst = (ce - cb + CPS - 1) / CPS;
  int64_t k = 0;
  bool ok = true;
  for (; k < nst; ++k) {
    const int s = int(k % NS);
    if (k >= NS && !tma::wait(&ring.empty[s], uint32_t(((k - NS) / NS) & 1), err)) {
      ok = false;
      break;
    }
    const int64_t c0 = cb + k * CPS;
    const int nc = int(ce - c0 < CPS ? ce - c0 : CPS);
    tma::fence_proxy_async();
    tma::arrive_expect_tx(&ring.full[s], tx_col * uint32_t(nc));
    for (int j = 0; j < nc; ++j)
      issue_column<LL, TRB>(stages + (s * CPS + j) * SBC, sl, r0, c0 + j, rows, &ring.full[s]);
  }
  if (!ok) {
    for (int64_t j = (k > NS ? k - NS : 0); j < k; ++j)
      tma::wait(&ring.full[j % NS], uint32_t((j / NS) & 1), nullptr);
  }
}

// ---------------------------------------------------------------- flat stream

// k_flat_bulk: the flat element-wise/reduction kernel for trees whose
// leaves are all dense matrices, fed by bulk copies instead of registers
// (trees with many leaves cannot keep enough vectors per thread in flight
// in registers). The flat range is cut into chunks of CH elements; for each
// of the block's chunks the producer thread copies the chunk of every leaf
// (one cp.async.bulk per leaf) into a ring stage, and the NTC consumers
// evaluate it from shared memory, V elements per step, storing or reducing
// through the epilogue. Chunks cover the first n16 elements (a whole number
// of 16-byte vectors); block 0 evaluates the few elements after them from
// global memory.
template <class LL, int CH, int I = 0>
FX_D void issue_flat_chunk(char* stage, const Slots& sl, int64_t i0, uint32_t bytes_per_es,
                           uint64_t* bar) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    const T* src = static_cast<const T*>(sl.s[L::slot].p) + i0;
    tma::copy_g2s(stage + I * CH * int(sizeof(T)), src, bytes_per_es * uint32_t(sizeof(T)), bar);
    issue_flat_chunk<LL, CH, I + 1>(stage, sl, i0, bytes_per_es, bar);
  }
}
template <class LL, int V, class CT, int CH, int I = 0>
FX_D void load_flat_chunk(Pack<LL, V, CT>& p, const char* stage, int k) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    pget<I>::of(p) = *reinterpret_cast<const Raw<T, V>*>(stage + (I * CH + k) * int(sizeof(T)));
    load_flat_chunk<LL, V, CT, CH, I + 1>(p, stage, k);
  }
}

template <class E, class Epi, int V, int NTC, int CH>
__global__ void __launch_bounds__(NTC + 32) k_flat_bulk(const E e, const Slots sl, const int64_t n,
                                                         const int64_t n16, const Epi epi,
                                                         const RedArgs red, const int ns,
                                                         unsigned int* err) {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  using T0 = typename tl_at<LL, 0>::type::elem;
  constexpr int SB = tl_size<LL>::value * CH * int(sizeof(T0));
  static_assert(CH % (V * NTC) == 0, "chunk shape");
  extern __shared__ __align__(128) char smem[];
  Ring<8>& ring = *reinterpret_cast<Ring<8>*>(smem + ns * SB);
  const int64_t nch = (n16 + CH - 1) / CH;
  const int64_t G = gridDim.x;
  const int64_t mine = nch > int64_t(blockIdx.x) ? (nch - blockIdx.x + G - 1) / G : 0;
  const int tid = threadIdx.x;
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
    if (tid == NTC) {  // producer
      bool ok = true;
      int64_t k = 0;
      for (; k < mine; ++k) {
        const int s = int(k % ns);
        if (k >= ns && !tma::wait(&ring.empty[s], uint32_t(((k - ns) / ns) & 1), err)) {
          ok = false;
          break;
        }
        const int64_t i0 = (blockIdx.x + k * G) * int64_t(CH);
        const uint32_t cnt = uint32_t(n16 - i0 < CH ? n16 - i0 : CH);
        tma::arrive_expect_tx(&ring.full[s], cnt * uint32_t(tl_size<LL>::value) * uint32_t(sizeof(T0)));
        issue_flat_chunk<LL, CH>(smem + s * SB, sl, i0, cnt, &ring.full[s]);
      }
      if (!ok) {
        for (int64_t j = (k > ns ? k - ns : 0); j < k; ++j)
          tma::wait(&ring.full[j % ns], uint32_t((j / ns) & 1), nullptr);
      }
    }
  } else {
    for (int64_t k = 0; k < mine; ++k) {
      const int s = int(k % ns);
      if (!tma::wait(&ring.full[s], uint32_t((k / ns) & 1), err)) {
        ring.abort = 1;
        break;
      }
      const int64_t i0 = (blockIdx.x + k * G) * int64_t(CH);
      const int cnt = int(n16 - i0 < CH ? n16 - i0 : CH);
      const char* stage = smem + s * SB;
#pragma unroll
      for (int q = 0; q < CH / (V * NTC); ++q) {
        const int kk = (tid + q * NTC) * V;
        if (kk < cnt) {
          Pack<LL, V, CT> p;
          load_flat_chunk<LL, V, CT, CH>(p, stage, kk);
          CT v[V];
          eval_lanes<V>(e, p, v);
          epi_put(epi, st, i0 + kk, v, p, V);
        }
      }
      tma::arrive(&ring.empty[s]);
    }
    if (blockIdx.x == 0) {  // elements after the last whole 16-byte vector
      for (int64_t i = n16 + tid; i < n; i += NTC) {
        Pack<LL, 1, CT> q;
        load_flat(q, sl, i, 0, 0);
        CT v1[1];
        eval_lanes<1>(e, q, v1);
        CT v[V];
#pragma unroll
        for (int j = 0; j < V; ++j) v[j] = v1[0];
        epi_put(epi, st, i, v, q, 1);
      }
    }
  }
  if constexpr (Epi::reduces) finish_full_reduce<CT, Epi::sqrt_result>(st, red);
}

// ---------------------------------------------------------------- sum/max along dim 1

template <class E, bool ISMAX, int V, int NTC, int NS, int CPS>
__global__ void __launch_bounds__(NTC + 32) k_row_bulk(const E e, const Slots sl, const int64_t R,
                                                        const int64_t C, const RowRed rr,
                                                        unsigned int* err) {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  constexpr int TRB = NTC * V;
  constexpr int SBC = stage_bytes<LL, TRB>();
  extern __shared__ __align__(128) char smem[];
  Ring<NS>& ring = *reinterpret_cast<Ring<NS>*>(smem + NS * CPS * SBC);
  const int64_t r0 = int64_t(blockIdx.x) * TRB;
  const int rows = int(R - r0 < TRB ? R - r0 : TRB);
  const int s = blockIdx.y;
  const int64_t cb = C * s / rr.S, ce = C * (s + 1) / rr.S;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      tma::mbar_init(&ring.full[i], 1);
      tma::mbar_init(&ring.empty[i], NTC);
    }
    ring.abort = 0;
    tma::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x >= NTC) {  // producer warp
    produce<LL, TRB, NS, CPS>(smem, ring, sl, r0, rows, cb, ce, err);
    return;
  }
  const int t = threadIdx.x;
  const int64_t r = r0 + int64_t(t) * V;
  const int nvalid = clamp_valid(R - r, V);
  ThreadSum<CT> acc[V];
  max_acc_t<E, CT> mx[V];
#pragma unroll
  for (int j = 0; j < V; ++j) {
    acc[j].init();
    mx[j].init();
  }
  Pack<LL, V, CT> hold;
  load_hold(hold, sl, r, nvalid);
  // A consumer that gives up waiting stops consuming but never leaves
  // early: the epilogue's barrier counts every consumer.
  const int64_t nst = (ce - cb + CPS - 1) / CPS;
  for (int64_t k = 0; k < nst; ++k) {
    const int st = int(k % NS);
    if (!tma::wait(&ring.full[st], uint32_t((k / NS) & 1), err)) {
      ring.abort = 1;
      break;
    }
    const int64_t c0 = cb + k * CPS;
    const int nc = int(ce - c0 < CPS ? ce - c0 : CPS);
    if (nvalid > 0) {
      for (int j = 0; j < nc; ++j) {
        Pack<LL, V, CT> p;
        load_stage<LL, V, CT, TRB>(p, hold, smem + (st * CPS + j) * SBC, sl, t, c0 + j, nvalid);
        CT v[V];
        eval_lanes<V>(max_tree<ISMAX, CT>(e), p, v);
#pragma unroll
        for (int q = 0; q < V; ++q) {
          if (ISMAX) mx[q].add(v[q]);
          else acc[q].add(v[q]);
        }
      }
    }
    tma::arrive(&ring.empty[st]);
  }
  CT m[V];
#pragma unroll
  for (int j = 0; j < V; ++j) m[j] = mx[j].get();
  row_finish<ISMAX, V, CT>(rr, acc, m, R, r, nvalid, s, NTC, &ring.abort);
}

// ---------------------------------------------------------------- fused backward

template <class E, int V, int NTC, int NS, int CPS>
__global__ void __launch_bounds__(NTC + 32) k_bwd_bulk(const E e, const Slots sl, const int64_t R,
                                                        const int64_t C, const GradArgs ga,
                                                        unsigned int* err) {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  constexpr int NBC = count_mode<LL>(MBC);
  constexpr int NB = NBC > 0 ? NBC : 1;
  static_assert(count_mode<LL>(MT) == 0 && count_mode<LL>(MBR) == 0,
                "fused backward: plain and each_col leaves only");
  constexpr int TRB = NTC * V;
  constexpr int SBC = stage_bytes<LL, TRB>();
  extern __shared__ __align__(128) char smem[];
  Ring<NS>& ring = *reinterpret_cast<Ring<NS>*>(smem + NS * CPS * SBC);
  const int64_t r0 = int64_t(blockIdx.x) * TRB;
  const int rows = int(R - r0 < TRB ? R - r0 : TRB);
  const int s = blockIdx.y;
  const int64_t cb = C * s / ga.S, ce = C * (s + 1) / ga.S;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      tma::mbar_init(&ring.full[i], 1);
      tma::mbar_init(&ring.empty[i], NTC);
    }
    ring.abort = 0;
    tma::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x >= NTC) {
    produce<LL, TRB, NS, CPS>(smem, ring, sl, r0, rows, cb, ce, err);
    return;
  }
  const int t = threadIdx.x;
  const int64_t r = r0 + int64_t(t) * V;
  const int nvalid = clamp_valid(R - r, V);
  const CT gL = ga.gscale ? __ldg(static_cast<const CT*>(ga.gscale)) : CT(1);
  ThreadSum<CT> bacc[NB][V];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int j = 0; j < V; ++j) bacc[b][j].init();
  Pack<LL, V, CT> hold;
  load_hold(hold, sl, r, nvalid);
  const int64_t nst = (ce - cb + CPS - 1) / CPS;
  for (int64_t k = 0; k < nst; ++k) {
    const int st = int(k % NS);
    if (!tma::wait(&ring.full[st], uint32_t((k / NS) & 1), err)) {
      ring.abort = 1;
      break;
    }
    const int64_t c0 = cb + k * CPS;
    const int nc = int(ce - c0 < CPS ? ce - c0 : CPS);
    if (nvalid > 0) {
      CT bpart[NB][V] = {};  // this stage's columns, summed plainly
      // the host launches this kernel only for row counts that are a
      // multiple of V, so every active thread takes the whole-vector body
      auto columns = [&](auto full) {
        constexpr bool F = decltype(full)::value;
        for (int jc = 0; jc < nc; ++jc) {
          Pack<LL, V, CT> p;
          load_stage<LL, V, CT, TRB, F>(p, hold, smem + (st * CPS + jc) * SBC, sl, t, c0 + jc,
                                        nvalid);
          GradAcc<LL, CT, E> g[V];
          grad_lanes<V>(e, p, gL, g);
          bwd_store<LL, V, CT, NB, F>(g, bpart, ga, r, c0 + jc, R, nvalid);
        }
      };
      if (nvalid == V) columns(std::true_type{});
      else columns(std::false_type{});
      if constexpr (NBC > 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int j = 0; j < V; ++j) bacc[b][j].add(bpart[b][j]);
      }
    }
    tma::arrive(&ring.empty[st]);
  }
  bwd_finish<LL, V, CT, NBC>(ga, bacc, R, r, nvalid, s, NTC, &ring.abort);
}

}  // namespace fx
