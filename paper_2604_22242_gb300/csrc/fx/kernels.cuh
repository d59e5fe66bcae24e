// kernels.cuh - the fused sm_103a kernels (one kernel per expression tree).
//
// Every kernel works in two phases per step: first it issues the loads of
// every distinct leaf for all of its vectors (register packs, so many
// independent 16/32-byte loads are in flight per thread), then it evaluates
// the tree lane by lane from registers and hands the results to an
// epilogue (store, fused reduction, or both). Intermediate values of the
// tree never leave registers: each input element is read once and each
// output element written once (Sec. 5: one pass over the input matrices).
//
// Reductions are deterministic: each thread accumulates a compensated
// (s, c) pair over a fixed set of elements; warps and blocks combine pairs
// in a fixed butterfly order; each block writes one partial; the last block
// to finish (an atomic ticket, no waiting) sums the partials in a fixed
// order in FP64 and writes the result. No block ever waits on another.
#pragma once

#include "plan.cuh"

namespace fx {

// ---------------------------------------------------------------- launch data

struct SlotView {
  const void* p;
  int64_t ld;  // leading dimension (matrix leaves)
  int64_t vs;  // element stride of a vector leaf: 1 (rows x 1) or ld (1 x cols)
};
struct Slots {
  SlotView s[FX_MAX_SLOTS];
};

// Reduction workspace: per-block partials and the completion ticket.
struct RedArgs {
  double2* part;
  unsigned int* ticket;
  void* out;  // float* or double* (the reduction type)
};

// ---------------------------------------------------------------- register packs

template <class L, int V, class CT> struct pack_elem {
  using T = typename L::elem;
  using type = std::conditional_t<L::mode == MT, Raw<CT, V>, Raw<T, (L::mode == MBR ? 1 : V)>>;
};

template <class LL, int V, class CT> struct Pack;
template <int V, class CT> struct Pack<TL<>, V, CT> {};
template <class H, class... Ts, int V, class CT> struct Pack<TL<H, Ts...>, V, CT> {
  typename pack_elem<H, V, CT>::type h;
  Pack<TL<Ts...>, V, CT> t;
};

template <int I> struct pget {
  template <class P> static FX_D auto& of(P& p) { return pget<I - 1>::of(p.t); }
};
template <> struct pget<0> {
  template <class P> static FX_D auto& of(P& p) { return p.h; }
};

// Element context: lane j of a pack.
template <class LL, int V, class CTy> struct Ctx {
  using CT = CTy;
  const Pack<LL, V, CT>& p;
  int j;
  template <int K, int M> FX_D CT leaf() const {
    constexpr int I = tl_index<LL, K, M>::value;
    static_assert(I >= 0, "leaf not in the pack");
    const auto& r = pget<I>::of(p);
    if constexpr (M == MT) {
      return r.v[j];
    } else if constexpr (M == MBR) {
      return to_compute<CT>(r.v[0]);
    } else {
      return to_compute<CT>(r.v[j]);
    }
  }
};

// Pair context: lanes 2j and 2j + 1 of a pack as one F2.
template <class LL, int V> struct Ctx2 {
  using CT = F2;
  const Pack<LL, V, float>& p;
  int j;
  template <int K, int M> FX_D F2 leaf() const {
    constexpr int I = tl_index<LL, K, M>::value;
    static_assert(I >= 0, "leaf not in the pack");
    const auto& r = pget<I>::of(p);
    if constexpr (M == MT) {
      return F2(r.v[2 * j], r.v[2 * j + 1]);
    } else if constexpr (M == MBR) {
      const float x = to_compute<float>(r.v[0]);
      return F2(x, x);
    } else {
      return F2(to_compute<float>(r.v[2 * j]), to_compute<float>(r.v[2 * j + 1]));
    }
  }
};

// The tree at V lanes of a pack; FP32 trees on lane pairs.
template <int V, class E, class LL, class CT>
FX_D void eval_lanes(const E& e, const Pack<LL, V, CT>& p, CT (&v)[V]) {
  if constexpr (std::is_same<CT, float>::value && V % 2 == 0) {
#pragma unroll
    for (int j = 0; j < V / 2; ++j) {
      Ctx2<LL, V> c{p, j};
      const F2 w = e.ev(c);
      v[2 * j] = w.x;
      v[2 * j + 1] = w.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) {
      Ctx<LL, V, CT> c{p, j};
      v[j] = e.ev(c);
    }
  }
}

FX_D int clamp_valid(int64_t left, int V) {
  return left >= V ? V : (left > 0 ? int(left) : 0);
}

// ---------------------------------------------------------------- leaf loads

// Flat layout: element i = r + c*R of every leaf. Matrix leaves are dense
// (ld == R) and read at i; an each_col vector at r (i and R are multiples
// of V, so the V elements share one column); an each_row vector at c.
template <class LL, int V, class CT, int I = 0>
FX_D void load_flat(Pack<LL, V, CT>& p, const Slots& sl, int64_t i, int64_t r, int64_t c) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    static_assert(L::mode != MT, "flat kernels take no transposed leaf");
    auto& dst = pget<I>::of(p);
    const SlotView& s = sl.s[L::slot];
    const T* base = static_cast<const T*>(s.p);
    if constexpr (L::mode == MN) {
      vload(dst, base + i);
    } else if constexpr (L::mode == MBC) {
      if (s.vs == 1) {
        vload(dst, base + r);
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j) dst.v[j] = sload(base + (r + j) * s.vs);
      }
    } else {
      dst.v[0] = sload(base + c * s.vs);
    }
    load_flat<LL, V, CT, I + 1>(p, sl, i, r, c);
  }
}

template <class LL, int I = 0> FX_HD constexpr int count_bcast() {
  if constexpr (I < tl_size<LL>::value) {
    return (tl_at<LL, I>::type::mode >= MBC ? 1 : 0) + count_bcast<LL, I + 1>();
  } else {
    return 0;
  }
}

// Column-vector layout: rows r .. r+V-1 (nvalid of them inside the
// matrix) of column c. V > 1 means the host checked that every such full
// vector is aligned for one access. MT leaves are filled from shared memory
// by the tiled kernel, not here.
template <class LL, int V, class CT, int I = 0>
FX_D void load_rc(Pack<LL, V, CT>& p, const Slots& sl, int64_t r, int64_t c, int nvalid) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    auto& dst = pget<I>::of(p);
    const SlotView& s = sl.s[L::slot];
    const T* base = static_cast<const T*>(s.p);
    if constexpr (L::mode == MN) {
      const T* q = base + r + c * s.ld;
      if (nvalid == V) {
        vload(dst, q);
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j) dst.v[j] = j < nvalid ? sload(q + j) : T(0.0f);
      }
    } else if constexpr (L::mode == MBC) {
      const T* q = base + r * s.vs;
      if (nvalid == V && s.vs == 1) {
        vload(dst, q);
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j) dst.v[j] = j < nvalid ? sload(q + j * s.vs) : T(0.0f);
      }
    } else if constexpr (L::mode == MBR) {
      dst.v[0] = sload(base + c * s.vs);
    }
    load_rc<LL, V, CT, I + 1>(p, sl, r, c, nvalid);
  }
}

// ---------------------------------------------------------------- epilogues
//
// put(state, off, v, nvalid): lanes 0..nvalid-1 of v are the tree's values
// at output offset off .. off+nvalid-1 (off = r + c*ldz).

// Pairwise sum of a vector's V lanes (V a power of two): one compensated
// add per vector instead of one per lane; the tree adds log2(V) roundings
// per element to a sum that is then accumulated compensated.
template <class CT, int V> FX_D CT lane_sum(const CT (&v)[V]) {
  if constexpr (V == 1) {
    return v[0];
  } else {
    CT h[V / 2];
#pragma unroll
    for (int j = 0; j < V / 2; ++j) h[j] = v[2 * j] + v[2 * j + 1];
    return lane_sum<CT, V / 2>(h);
  }
}

template <class T, int V> struct EpiStore {
  T* z;
  int64_t ldz;
  static constexpr bool side_tree = false;
  static constexpr bool stores = true;
  static constexpr bool reduces = false;
  static constexpr bool pure_sum = false;
  static constexpr bool sqrt_result = false;
  struct State {
    FX_D void init() {}
  };
  template <class CT> FX_D void put(State&, int64_t off, const CT (&v)[V], int nvalid) const {
    if (nvalid == V) {
      Raw<T, V> o;
#pragma unroll
      for (int j = 0; j < V; ++j) o.v[j] = narrow_to<T>::from(v[j]);
      vstore(z + off, o);
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (j < nvalid) sstore(z + off + j, narrow_to<T>::from(v[j]));
    }
  }
};

// Fused sum of the elements (SQ: of their squares, for the 2-norm).
template <class CTy, int V, bool SQ> struct EpiSum {
  int64_t ldz;
  static constexpr bool side_tree = false;
  static constexpr bool stores = false;
  static constexpr bool reduces = true;
  static constexpr bool pure_sum = true;  // k_flat may combine several vectors per add
  // the (squared) lanes of one full vector, summed pairwise
  template <class CT> FX_D CT vsum(const CT (&v)[V]) const {
    CT w[V];
#pragma unroll
    for (int j = 0; j < V; ++j) w[j] = SQ ? v[j] * v[j] : v[j];
    return lane_sum(w);
  }
  static constexpr bool sqrt_result = SQ;
  using State = ThreadSum<CTy>;
  template <class CT> FX_D void put(State& st, int64_t, const CT (&v)[V], int nvalid) const {
    if (nvalid == V) {
      CT w[V];
#pragma unroll
      for (int j = 0; j < V; ++j) w[j] = SQ ? v[j] * v[j] : v[j];
      st.add(lane_sum(w));
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (j < nvalid) st.add(SQ ? v[j] * v[j] : v[j]);
    }
  }
};

// Store and sum (a tree with an accu side output: Z and accu(Z)).
template <class T, int V> struct EpiStoreSum {
  T* z;
  int64_t ldz;
  static constexpr bool side_tree = false;
  static constexpr bool stores = true;
  static constexpr bool reduces = true;
  static constexpr bool pure_sum = false;
  static constexpr bool sqrt_result = false;
  using State = ThreadSum<compute_t<T>>;
  template <class CT> FX_D void put(State& st, int64_t off, const CT (&v)[V], int nvalid) const {
    EpiStore<T, V> s{z, ldz};
    typename EpiStore<T, V>::State d;
    s.put(d, off, v, nvalid);
    if (nvalid == V) {
      st.add(lane_sum(v));
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (j < nvalid) st.add(v[j]);
    }
  }
};

// Store one tree and sum a second tree over the same leaves (the root
// with_accu(E, S): Z = E, s = accu(S)). put() stores E's values; put_side()
// evaluates S lane by lane from the same register pack and adds it.
template <class T, int V, class S> struct EpiStoreSide {
  T* z;
  int64_t ldz;
  S side;
  static constexpr bool side_tree = true;
  static constexpr bool stores = true;
  static constexpr bool reduces = true;
  static constexpr bool pure_sum = false;
  static constexpr bool sqrt_result = false;
  using State = ThreadSum<compute_t<T>>;
  template <class CT> FX_D void put(State&, int64_t off, const CT (&v)[V], int nvalid) const {
    EpiStore<T, V> s{z, ldz};
    typename EpiStore<T, V>::State d;
    s.put(d, off, v, nvalid);
  }
  template <class LL, int VP, class CT>
  FX_D void put_side(State& st, const Pack<LL, VP, CT>& p, int nvalid) const {
    CT w[VP];
#pragma unroll
    for (int j = 0; j < VP; ++j) {
      Ctx<LL, VP, CT> c{p, j};
      w[j] = side.ev(c);
    }
    if (nvalid == VP) {
      st.add(lane_sum(w));
    } else {
#pragma unroll
      for (int j = 0; j < VP; ++j)
        if (j < nvalid) st.add(w[j]);
    }
  }
};

// Hands lanes 0..nvalid-1 of v (and, for a side tree, the pack they came
// from) to the epilogue.
template <class Epi, class St, class CT, int V, class P>
FX_D void epi_put(const Epi& epi, St& st, int64_t off, const CT (&v)[V], const P& p, int nvalid) {
  epi.put(st, off, v, nvalid);
  if constexpr (Epi::side_tree) epi.put_side(st, p, nvalid);
}

// ---------------------------------------------------------------- FP64 reduction helpers
//
// FP64 arithmetic is scarce on this part (about 1/64 of the FP32 rate), so
// FP64 reductions spend as few FP64 instructions per element as they can:
//  - a sum whose terms are products (a % b, square(a), the squares of a
//    2-norm) folds the multiply into the accumulation, acc = fma(a, b, acc):
//    one FP64 instruction per term instead of a multiply and an add, each
//    term rounded once. Every lane of every unrolled vector keeps its own
//    accumulator, so the chains are independent;
//  - a maximum of absolute values compares IEEE bit patterns as signed
//    64-bit integers (monotone for values with a clear sign bit; a NaN's
//    pattern is above infinity's, so NaN still wins) on the integer units.

template <class E> struct prod_root { static constexpr bool value = false; };
template <class L, class R> struct prod_root<Bin<OpMul, L, R>> {
  static constexpr bool value = true;
  template <class Ctx, class CT>
  static FX_D void parts(const Bin<OpMul, L, R>& e, const Ctx& c, CT& a, CT& b) {
    a = e.l.ev(c);
    b = e.r.ev(c);
  }
};
template <class X> struct prod_root<Un<OpSquare, X>> {
  static constexpr bool value = true;
  template <class Ctx, class CT>
  static FX_D void parts(const Un<OpSquare, X>& e, const Ctx& c, CT& a, CT& b) {
    a = e.e.ev(c);
    b = a;
  }
};

// The two factors of term j of pack p: the root's operands, or for a sum of
// squares (SQ) the value twice.
template <bool SQ, class E, class LL, int V, class CT>
FX_D void term_parts(const E& e, const Pack<LL, V, CT>& p, int j, CT& a, CT& b) {
  Ctx<LL, V, CT> c{p, j};
  if constexpr (SQ) {
    a = e.ev(c);
    b = a;
  } else {
    prod_root<E>::parts(e, c, a, b);
  }
}

template <class E> struct abs_root { static constexpr bool value = false; };
template <class X> struct abs_root<Un<OpAbs, X>> { static constexpr bool value = true; };

// Running maximum: NaN-propagating compare, or (INT) signed 64-bit compares
// of bit patterns of values known to have a clear sign bit.
template <class CT, bool INT> struct MaxAcc {
  CT m;
  FX_D void init() { m = neg_inf<CT>(); }
  FX_D void add(CT v) { m = max_nan(m, v); }
  FX_D CT get() const { return m; }
};
template <> struct MaxAcc<double, true> {
  long long m;
  FX_D void init() { m = -1; }
  // v is the abs node's operand: its magnitude is the pattern with the sign
  // bit cleared (an integer and, not an FP64 instruction)
  FX_D void add(double v) {
    const long long b = __double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFll;
    m = b > m ? b : m;
  }
  FX_D double get() const { return m < 0 ? neg_inf<double>() : __longlong_as_double(m); }
};
template <class E, class CT>
using max_acc_t = MaxAcc<CT, std::is_same<CT, double>::value && abs_root<E>::value>;

// The tree whose values a maximum takes: for an FP64 maximum of magnitudes
// the abs node's operand (MaxAcc clears the sign bit itself), else the tree.
template <bool ISMAX, class CT, class E> FX_D const auto& max_tree(const E& e) {
  if constexpr (ISMAX && std::is_same<CT, double>::value && abs_root<E>::value) return e.e;
  else return e;
}

// ---------------------------------------------------------------- combines

// Barrier over the first `n` threads of the block (n a multiple of 32):
// a named barrier, so blocks whose producer warp has left can still sync.
FX_D void block_sync(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }

template <class S> FX_D void warp_merge(S& a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    auto s2 = __shfl_xor_sync(0xffffffffu, a.s, o);
    auto c2 = __shfl_xor_sync(0xffffffffu, a.c, o);
    a.merge(s2, c2);
  }
}

// Block-wide merge of per-thread pairs; the total is valid in thread 0.
// Fixed order: butterfly in each warp, then warp 0 over the warp totals.
template <class S> FX_D void block_merge(S& a) {
  using CT = decltype(a.s);
  __shared__ CT bs[32], bc[32];
  warp_merge(a);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();  // bs/bc may still be read by a previous call
  if (lane == 0) {
    bs[w] = a.s;
    bc[w] = a.c;
  }
  __syncthreads();
  if (w == 0) {
    a.s = lane < nw ? bs[lane] : CT(0);
    a.c = lane < nw ? bc[lane] : CT(0);
    warp_merge(a);
  }
}

template <class CT> FX_D CT warp_max(CT m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_nan(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}
template <class CT> FX_D CT block_max(CT m) {
  __shared__ CT bm[32];
  m = warp_max(m);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) bm[w] = m;
  __syncthreads();
  if (w == 0) m = warp_max(lane < nw ? bm[lane] : neg_inf<CT>());
  return m;
}

// Fixed-order FP64 sum of n partial pairs part[i*stride]; the result is
// valid in thread 0. Every thread of the block must call it. COMP selects
// a compensated sum (FP64 trees, whose 1e-13 bound needs it); for FP32
// trees a plain FP64 sum of the partials is already about 2^-40 relative,
// and FP64 operations are scarce on this part.
template <bool COMP> FX_D double block_sum_partials(const double2* part, int64_t n, int64_t stride) {
  using S = std::conditional_t<COMP, CompSum<double>, PlainSum<double>>;
  S a;
  a.init();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double2 q = __ldcg(part + i * stride);
    a.add(q.x);
    a.add(q.y);
  }
  block_merge(a);
  return a.s + a.c;
}

// Every block publishes its partial; the last one combines all of them.
template <class CT, bool SQRT, class S> FX_D void finish_full_reduce(S& a, const RedArgs& red) {
  block_merge(a);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    red.part[blockIdx.x] = make_double2(double(a.s), double(a.c));
    __threadfence();
    unsigned int t = atomicAdd(red.ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tot = block_sum_partials<std::is_same<CT, double>::value>(red.part, gridDim.x, 1);
  if (threadIdx.x == 0) {
    if (SQRT) tot = ::sqrt(tot);
    *static_cast<CT*>(red.out) = static_cast<CT>(tot);
    *red.ticket = 0u;  // ready for the next launch on this stream
  }
}

// ---------------------------------------------------------------- A3: flat stream

// With broadcast leaves, (r, c) of element i comes from one division by R
// per vector (FastDiv; the host guarantees n < 2^32 and R % V == 0).
template <class E, class Epi, int V, int U>
__global__ void __launch_bounds__(512) k_flat(const E e, const Slots sl, const int64_t n,
                                              const Epi epi, const RedArgs red, const FastDiv fd) {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  constexpr bool BC = count_bcast<LL>() > 0;
  const int64_t nv = n / V;
  const int64_t bdim = blockDim.x;
  const int64_t step = int64_t(gridDim.x) * bdim * U;
  // FP64 sums of products: one fma per term into U x V accumulators
  constexpr bool FMA64 = Epi::pure_sum && std::is_same<CT, double>::value &&
                         (Epi::sqrt_result || prod_root<E>::value);
  typename Epi::State st;
  st.init();
  CT facc[FMA64 ? U : 1][FMA64 ? V : 1];
#pragma unroll
  for (int u = 0; u < (FMA64 ? U : 1); ++u)
#pragma unroll
    for (int j = 0; j < (FMA64 ? V : 1); ++j) facc[u][j] = CT(0);
  for (int64_t b = int64_t(blockIdx.x) * bdim * U + threadIdx.x; b < nv; b += step) {
    Pack<LL, V, CT> p[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t vi = b + u * bdim;
      if (vi < nv) {
        int64_t r = 0, c = 0;
        if constexpr (BC) {
          c = fd.div(uint32_t(vi * V));
          r = vi * V - c * fd.d;
        }
        load_flat(p[u], sl, vi * V, r, c);
      }
    }
    if constexpr (FMA64) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (b + u * bdim < nv) {
#pragma unroll
          for (int j = 0; j < V; ++j) {
            CT x, y;
            term_parts<Epi::sqrt_result>(e, p[u], j, x, y);
            facc[u][j] = __fma_rn(x, y, facc[u][j]);
          }
        }
      }
    } else if constexpr (Epi::pure_sum) {
      // one compensated add per step: the U vectors' sums added pairwise
      CT vs[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t vi = b + u * bdim;
        vs[u] = CT(0);
        if (vi < nv) {
          CT v[V];
          eval_lanes<V>(e, p[u], v);
          vs[u] = epi.vsum(v);
        }
      }
      st.add(lane_sum(vs));
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t vi = b + u * bdim;
        if (vi < nv) {
          CT v[V];
          eval_lanes<V>(e, p[u], v);
          epi_put(epi, st, vi * V, v, p[u], V);
        }
      }
    }
  }
  if (V > 1 && !BC && blockIdx.x == 0) {  // the n % V trailing elements, one lane each
    for (int64_t i = nv * V + threadIdx.x; i < n; i += bdim) {
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
  if constexpr (FMA64) {
    CT w[U * V];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < V; ++j) w[u * V + j] = facc[u][j];
    st.add(lane_sum(w));
  }
  if constexpr (Epi::reduces) finish_full_reduce<CT, Epi::sqrt_result>(st, red);
}

// ---------------------------------------------------------------- A4: tiles
//
// A block owns TR x TC output tiles. Thread (tx, ty) handles rows
// r0 + V*tx .. +V-1 of columns c0 + ty + TY*q, q < P. A transposed leaf D
// (C x R) is read along its own columns - rows c0 .. c0+TC-1 of D, which
// are contiguous - with vector loads, staged in shared memory as S[r][c]
// (row stride TC + 1: odd, so column reads are free of bank conflicts),
// and read back in output order, so both the load of D and the store of Z
// stay coalesced (the swapped index of the Sec. 3 transpose rule, used
// directly, would read D with stride ld).

template <class LL, int I = 0> FX_HD constexpr int count_mt() {
  if constexpr (I < tl_size<LL>::value) {
    return (tl_at<LL, I>::type::mode == MT ? 1 : 0) + count_mt<LL, I + 1>();
  } else {
    return 0;
  }
}
template <class LL, int I, int J = 0> FX_HD constexpr int mt_rank() {  // index among MT leaves
  if constexpr (J < I) {
    return (tl_at<LL, J>::type::mode == MT ? 1 : 0) + mt_rank<LL, I, J + 1>();
  } else {
    return 0;
  }
}

template <class E, int V_, int TR_, int TC_, int NT_> struct TileShape {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  static constexpr int V = V_, TR = TR_, TC = TC_, NT = NT_;
  static constexpr int TX = TR / V, TY = NT / TX, P = TC / TY;
  static_assert(TX * V == TR && TX * TY == NT && P * TY == TC, "bad tile shape");
  // transposed-leaf staging: vectors along D's rows (the output's columns)
  static constexpr int DX = TC / V, DY = NT / DX, DP = TR / DY;
  static_assert(DX * V == TC && DX * DY == NT && DP * DY == TR, "bad staging shape");
  static constexpr int NMT = count_mt<LL>();
  static constexpr int SROW = TC + 1;
  static constexpr int SMEM = (NMT > 0 ? NMT : 1) * TR * SROW;  // elements of CT
};

// Global loads of the transposed leaves' tiles into registers.
template <class TS, int I = 0>
FX_D void mt_fetch(typename TS::CT (&regs)[TS::NMT > 0 ? TS::NMT : 1][TS::DP][TS::V],
                   const Slots& sl, int64_t R, int64_t C, int64_t r0, int64_t c0) {
  using LL = typename TS::LL;
  using CT = typename TS::CT;
  constexpr int V = TS::V;
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    if constexpr (L::mode == MT) {
      using T = typename L::elem;
      constexpr int m = mt_rank<LL, I>();
      const SlotView& s = sl.s[L::slot];
      const T* base = static_cast<const T*>(s.p);
      const int dx = threadIdx.x % TS::DX, dy = threadIdx.x / TS::DX;
      const int64_t c = c0 + int64_t(dx) * V;  // row of D
      const int nvalid = clamp_valid(C - c, V);
#pragma unroll
      for (int q = 0; q < TS::DP; ++q) {
        const int64_t r = r0 + dy + int64_t(q) * TS::DY;  // column of D
        Raw<T, V> w;
        if (r < R && nvalid > 0) {
          const T* src = base + c + r * s.ld;
          if (nvalid == V) {
            vload(w, src);
          } else {
#pragma unroll
            for (int j = 0; j < V; ++j) w.v[j] = j < nvalid ? sload(src + j) : T(0.0f);
          }
        } else {
#pragma unroll
          for (int j = 0; j < V; ++j) w.v[j] = T(0.0f);
        }
#pragma unroll
        for (int j = 0; j < V; ++j) regs[m][q][j] = to_compute<CT>(w.v[j]);
      }
    }
    mt_fetch<TS, I + 1>(regs, sl, R, C, r0, c0);
  }
}

// Shared-memory values of the transposed leaves for the thread's vectors.
template <class TS, int I = 0>
FX_D void mt_fill(Pack<typename TS::LL, TS::V, typename TS::CT> (&p)[TS::P],
                  const typename TS::CT* sm) {
  using LL = typename TS::LL;
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    if constexpr (L::mode == MT) {
      constexpr int m = mt_rank<LL, I>();
      const int tx = threadIdx.x % TS::TX, ty = threadIdx.x / TS::TX;
#pragma unroll
      for (int q = 0; q < TS::P; ++q)
#pragma unroll
        for (int j = 0; j < TS::V; ++j)
          pget<I>::of(p[q]).v[j] =
              sm[(m * TS::TR + tx * TS::V + j) * TS::SROW + ty + q * TS::TY];
    }
    mt_fill<TS, I + 1>(p, sm);
  }
}

// Tile t of a tiles_r x tiles_c grid, tile rows fastest: the tiles in
// flight at once cover whole tile columns, so plain leaves (the majority in
// the trees here) stream down contiguous column blocks. Bands of 32 tile
// rows, which shorten the transposed leaves' scattered runs, measured
// slower on GB300 for every transposed tree tried.
FX_D void tile_coords(int64_t t, int64_t tiles_r, int64_t, int64_t& tr, int64_t& tc) {
  tc = t / tiles_r;
  tr = t - tc * tiles_r;
}

// One TR x TC tile at (r0, c0) of an R x C tree.
template <class TS, class E, class Epi>
FX_D void tile_body(const E& e, const Slots& sl, int64_t R, int64_t C, int64_t r0, int64_t c0,
                    const Epi& epi, typename Epi::State& st, typename TS::CT* sm) {
  using LL = typename TS::LL;
  using CT = typename TS::CT;
  constexpr int V = TS::V;
  const int tx = threadIdx.x % TS::TX, ty = threadIdx.x / TS::TX;
  const int64_t r = r0 + int64_t(tx) * V;
  const int nvalid = clamp_valid(R - r, V);
  Pack<LL, V, CT> p[TS::P];
#pragma unroll
  for (int q = 0; q < TS::P; ++q) {
    const int64_t c = c0 + ty + int64_t(q) * TS::TY;
    if (c < C && nvalid > 0) load_rc(p[q], sl, r, c, nvalid);
  }
  if constexpr (TS::NMT > 0) {
    CT regs[TS::NMT][TS::DP][V];
    mt_fetch<TS>(regs, sl, R, C, r0, c0);
    __syncthreads();  // the previous tile's readers are done with sm
    const int dx = threadIdx.x % TS::DX, dy = threadIdx.x / TS::DX;
#pragma unroll
    for (int m = 0; m < TS::NMT; ++m)
#pragma unroll
      for (int q = 0; q < TS::DP; ++q)
#pragma unroll
        for (int j = 0; j < V; ++j)
          sm[(m * TS::TR + dy + q * TS::DY) * TS::SROW + dx * V + j] = regs[m][q][j];
    __syncthreads();
    mt_fill<TS>(p, sm);
  }
#pragma unroll
  for (int q = 0; q < TS::P; ++q) {
    const int64_t c = c0 + ty + int64_t(q) * TS::TY;
    if (c < C && nvalid > 0) {
      CT v[V];
      eval_lanes<V>(e, p[q], v);
      epi_put(epi, st, r + c * epi.ldz, v, p[q], nvalid);
    }
  }
}

template <class E, class Epi, int V, int TR, int TC, int NT>
__global__ void __launch_bounds__(NT) k_tile(const E e, const Slots sl, const int64_t R,
                                             const int64_t C, const Epi epi, const RedArgs red) {
  using TS = TileShape<E, V, TR, TC, NT>;
  using CT = typename TS::CT;
  __shared__ CT sm[TS::SMEM];
  typename Epi::State st;
  st.init();
  const int64_t tiles_r = (R + TR - 1) / TR, tiles_c = (C + TC - 1) / TC;
  const int64_t ntiles = tiles_r * tiles_c;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int64_t tr, tc;
    tile_coords(t, tiles_r, tiles_c, tr, tc);
    tile_body<TS>(e, sl, R, C, tr * TR, tc * TC, epi, st, sm);
  }
  if constexpr (Epi::reduces) finish_full_reduce<CT, Epi::sqrt_result>(st, red);
}

// ---------------------------------------------------------------- A6: dim reductions
//
// sum/max along dim 0 (one value per column): columns are contiguous, so
// a group of G threads (a warp, or the whole block) walks one column with
// vector loads and reduces in a fixed order. Output (0, c) at out[c*ldo].

template <class E, bool ISMAX, int V, int U, int G, int NT>
__global__ void __launch_bounds__(NT) k_col(const E e, const Slots sl, const int64_t R,
                                            const int64_t C, void* out, const int64_t ldo) {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  static_assert(G == 32 || G == NT, "a column is reduced by a warp or a block");
  // FP64 sums of products: one fma per term into U x V accumulators
  constexpr bool FMA64 = !ISMAX && std::is_same<CT, double>::value && prod_root<E>::value;
  constexpr int GPB = NT / G;
  const int g = threadIdx.x / G, lane = threadIdx.x % G;
  for (int64_t cb = int64_t(blockIdx.x) * GPB; cb < C; cb += int64_t(gridDim.x) * GPB) {
    const int64_t c = cb + g;
    ThreadSum<CT> acc;
    acc.init();
    max_acc_t<E, CT> mx;
    mx.init();
    // one accumulator per lane, the U vectors of a step folded in order: an
    // FP64 fma holds the FP64 unit for many cycles per warp anyway, and
    // fewer live registers keep two blocks resident per SM
    CT facc[FMA64 ? V : 1];
#pragma unroll
    for (int j = 0; j < (FMA64 ? V : 1); ++j) facc[j] = CT(0);
    if (c < C) {
      for (int64_t rb = int64_t(lane) * V; rb < R; rb += int64_t(G) * V * U) {
        Pack<LL, V, CT> p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t r = rb + int64_t(u) * G * V;
          const int nv = clamp_valid(R - r, V);
          if (nv > 0) load_rc(p[u], sl, r, c, nv);
        }
        if constexpr (FMA64) {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int nv = clamp_valid(R - (rb + int64_t(u) * G * V), V);
#pragma unroll
            for (int j = 0; j < V; ++j) {
              if (j < nv) {
                CT x, y;
                term_parts<false>(e, p[u], j, x, y);
                facc[j] = __fma_rn(x, y, facc[j]);
              }
            }
          }
          continue;
        }
        // sums: the U vectors' lanes are added pairwise into one value per
        // step, then one compensated add (short dependency chains, which
        // matter for FP64 adds)
        CT vs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t r = rb + int64_t(u) * G * V;
          const int nv = clamp_valid(R - r, V);
          vs[u] = CT(0);
          if (nv > 0) {
            CT v[V];
            eval_lanes<V>(max_tree<ISMAX, CT>(e), p[u], v);
            if (ISMAX) {
#pragma unroll
              for (int j = 0; j < V; ++j)
                if (j < nv) mx.add(v[j]);
            } else if (nv == V) {
              vs[u] = lane_sum(v);
            } else {
#pragma unroll
              for (int j = 0; j < V; ++j)
                if (j < nv) vs[u] += v[j];
            }
          }
        }
        if (!ISMAX) acc.add(lane_sum(vs));
      }
    }
    if constexpr (FMA64) acc.add(lane_sum(facc));
    const CT m = mx.get();
    CT res;
    if constexpr (G == 32) {
      if (ISMAX) {
        res = warp_max(m);
      } else {
        warp_merge(acc);
        res = CT(double(acc.s) + double(acc.c));
      }
    } else {
      if (ISMAX) {
        res = block_max(m);
      } else {
        block_merge(acc);
        res = CT(double(acc.s) + double(acc.c));
      }
    }
    if (lane == 0 && c < C) static_cast<CT*>(out)[c * ldo] = res;
  }
}

// sum/max along dim 1 (one value per row): rows are strided, so a thread
// owns V consecutive rows and walks the columns of its split; a warp reads
// 32*V contiguous elements per column. With S > 1 column splits, each
// block writes per-row partials and the last of the S blocks of its row
// range (an atomic ticket per range) combines them in split order (FP64
// for sums). Output r at out[r].
struct RowRed {
  double2* part;           // [S][R] compensated pairs (sums)
  void* partm;             // [S][R] compute-type maxima
  unsigned int* tickets;   // one per row range (gridDim.x)
  void* out;
  int S;
};

// End of a row-range block: write the thread's rows (one split), or
// publish per-row partials and let the last of the S splits of this row
// range (an atomic ticket) combine them in split order. Called by the
// `nthreads` computing threads only (a named barrier, not __syncthreads).
template <bool ISMAX, int V, class CT>
FX_D void row_finish(const RowRed& rr, ThreadSum<CT> (&acc)[V], CT (&m)[V], int64_t R, int64_t r,
                     int nvalid, int s, int nthreads, const volatile int* abort = nullptr) {
  CT* out = static_cast<CT*>(rr.out);
  if (rr.S == 1) {
#pragma unroll
    for (int j = 0; j < V; ++j)
      if (j < nvalid) out[r + j] = ISMAX ? m[j] : CT(double(acc[j].s) + double(acc[j].c));
    return;
  }
#pragma unroll
  for (int j = 0; j < V; ++j) {
    if (j < nvalid) {
      if (ISMAX) static_cast<CT*>(rr.partm)[int64_t(s) * R + r + j] = m[j];
      else rr.part[int64_t(s) * R + r + j] = make_double2(double(acc[j].s), double(acc[j].c));
    }
  }
  __threadfence();
  block_sync(nthreads);
  if (abort && *abort) return;  // a bounded wait gave up (recorded); no combine
  __shared__ bool last;
  if (threadIdx.x == 0) last = atomicAdd(rr.tickets + blockIdx.x, 1u) == unsigned(rr.S - 1);
  block_sync(nthreads);
  if (!last) return;
  __threadfence();
  // the S partials of each of the thread's rows, in split order; for a
  // fixed split a warp reads 32*V contiguous values; 8 splits in flight
  constexpr int KU = 8;
  if (ISMAX) {
    const CT* pm = static_cast<const CT*>(rr.partm);
    CT mm[V];
#pragma unroll
    for (int j = 0; j < V; ++j) mm[j] = neg_inf<CT>();
    int k = 0;
    for (; k + KU <= rr.S; k += KU) {
      CT q[KU][V];
#pragma unroll
      for (int t = 0; t < KU; ++t)
#pragma unroll
        for (int j = 0; j < V; ++j)
          q[t][j] = j < nvalid ? __ldcg(pm + int64_t(k + t) * R + r + j) : neg_inf<CT>();
#pragma unroll
      for (int t = 0; t < KU; ++t)
#pragma unroll
        for (int j = 0; j < V; ++j) mm[j] = max_nan(mm[j], q[t][j]);
    }
    for (; k < rr.S; ++k)
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (j < nvalid) mm[j] = max_nan(mm[j], __ldcg(pm + int64_t(k) * R + r + j));
#pragma unroll
    for (int j = 0; j < V; ++j)
      if (j < nvalid) out[r + j] = mm[j];
  } else {
    using S = std::conditional_t<std::is_same<CT, double>::value, CompSum<double>, PlainSum<double>>;
    S a[V];
#pragma unroll
    for (int j = 0; j < V; ++j) a[j].init();
    int k = 0;
    for (; k + KU <= rr.S; k += KU) {
      double2 q[KU][V];
#pragma unroll
      for (int t = 0; t < KU; ++t)
#pragma unroll
        for (int j = 0; j < V; ++j)
          q[t][j] = j < nvalid ? __ldcg(rr.part + int64_t(k + t) * R + r + j) : make_double2(0, 0);
#pragma unroll
      for (int t = 0; t < KU; ++t)
#pragma unroll
        for (int j = 0; j < V; ++j) {
          a[j].add(q[t][j].x);
          a[j].add(q[t][j].y);
        }
    }
    for (; k < rr.S; ++k)
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (j < nvalid) {
          double2 q = __ldcg(rr.part + int64_t(k) * R + r + j);
          a[j].add(q.x);
          a[j].add(q.y);
        }
#pragma unroll
    for (int j = 0; j < V; ++j)
      if (j < nvalid) out[r + j] = CT(a[j].s + a[j].c);
  }
  if (threadIdx.x == 0) rr.tickets[blockIdx.x] = 0u;
}

template <class E, bool ISMAX, int V, int U, int NT>
__global__ void __launch_bounds__(NT) k_row(const E e, const Slots sl, const int64_t R,
                                            const int64_t C, const RowRed rr) {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  const int64_t r = (int64_t(blockIdx.x) * NT + threadIdx.x) * V;
  const int nvalid = clamp_valid(R - r, V);
  const int s = blockIdx.y;
  const int64_t cb = C * s / rr.S, ce = C * (s + 1) / rr.S;
  ThreadSum<CT> acc[V];
  max_acc_t<E, CT> mx[V];
#pragma unroll
  for (int j = 0; j < V; ++j) {
    acc[j].init();
    mx[j].init();
  }
  if (nvalid > 0) {
    for (int64_t c = cb; c < ce; c += U) {
      Pack<LL, V, CT> p[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (c + u < ce) load_rc(p[u], sl, r, c + u, nvalid);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c + u < ce) {
          CT v[V];
          eval_lanes<V>(max_tree<ISMAX, CT>(e), p[u], v);
#pragma unroll
          for (int j = 0; j < V; ++j) {
            if (ISMAX) mx[j].add(v[j]);
            else acc[j].add(v[j]);
          }
        }
      }
    }
  }
  CT m[V];
#pragma unroll
  for (int j = 0; j < V; ++j) m[j] = mx[j].get();
  row_finish<ISMAX, V, CT>(rr, acc, m, R, r, nvalid, s, NT);
}

// ---------------------------------------------------------------- A9: fused backward
//
// L = gL * accu(f(leaves)). Per element the tree is re-evaluated and its
// reverse pass (Leaf/Bin/Un/SL/SR ::bwd) hands each distinct leaf its
// local partial derivative. Plain leaves get dL/dleaf written element by
// element; each_col leaves (vectors indexed by row) get their row sums,
// accumulated per thread and combined across column splits like k_row.

// The adjoints start at -0: -0 + a == a exactly for every a (+0 + a is not,
// for a = -0), so the compiler may drop the first add into each adjoint.
template <class CT> FX_D CT grad_zero() { return -CT(0); }

// Per-leaf adjoints of one element (or lane pair). A leaf that occurs once
// in the tree E takes its adjoint by assignment (the add into -0 would be
// exact too, but costs an instruction on lane pairs).
template <class LL, class CT, class E> struct GradAcc {
  CT g[tl_size<LL>::value];
  template <int K, int M> FX_D void add(CT a) {
    constexpr int i = tl_index<LL, K, M>::value;
    if constexpr (leaf_count<E, K, M>::value == 1) g[i] = a;
    else g[i] += a;
  }
};

// Reverse pass of V lanes: every leaf's adjoint per lane. FP32 trees run
// on lane pairs.
template <int V, class E, class LL, class CT>
FX_D void grad_lanes(const E& e, const Pack<LL, V, CT>& p, CT gL, GradAcc<LL, CT, E> (&g)[V]) {
  constexpr int NL = tl_size<LL>::value;
  if constexpr (std::is_same<CT, float>::value && V % 2 == 0) {
#pragma unroll
    for (int j = 0; j < V / 2; ++j) {
      GradAcc<LL, F2, E> h;
#pragma unroll
      for (int q = 0; q < NL; ++q) h.g[q] = F2(-0.0f, -0.0f);
      Ctx2<LL, V> cx{p, j};
      e.bwd(cx, F2(gL, gL), h);
#pragma unroll
      for (int q = 0; q < NL; ++q) {
        g[2 * j].g[q] = h.g[q].x;
        g[2 * j + 1].g[q] = h.g[q].y;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) {
#pragma unroll
      for (int q = 0; q < NL; ++q) g[j].g[q] = grad_zero<CT>();
      Ctx<LL, V, CT> cx{p, j};
      e.bwd(cx, gL, g[j]);
    }
  }
}

struct GradArgs {
  void* g[FX_MAX_SLOTS];    // per input slot: dense column-major gradient, or null
  const void* gscale;       // device scalar (reduction type) or null for 1
  double2* part;            // [NBC][S][R]
  unsigned int* tickets;    // one per row range
  int S;
};

template <class LL, int I = 0> FX_HD constexpr int count_mode(int mode) {
  if constexpr (I < tl_size<LL>::value) {
    return (tl_at<LL, I>::type::mode == mode ? 1 : 0) + count_mode<LL, I + 1>(mode);
  } else {
    return 0;
  }
}
template <class LL, int I, int J = 0> FX_HD constexpr int bc_rank() {
  if constexpr (J < I) {
    return (tl_at<LL, J>::type::mode == MBC ? 1 : 0) + bc_rank<LL, I, J + 1>();
  } else {
    return 0;
  }
}

// Writes the plain leaves' gradients at (r.., c) and adds the each_col
// leaves' partial derivatives to per-row plain partial sums (the caller
// folds those into the compensated running sums once per group of
// columns: one compensated add per group instead of per element).
// FULL: the caller knows that all V rows are inside the matrix.
template <class LL, int V, class CT, int NB, bool FULL = false, int I = 0, class E>
FX_D void bwd_store(const GradAcc<LL, CT, E> (&g)[V], CT (&bpart)[NB][V],
                    const GradArgs& ga, int64_t r, int64_t c, int64_t R, int nvalid) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    if constexpr (L::mode == MN) {
      T* dst = static_cast<T*>(ga.g[L::slot]);
      if (dst) {
        T* q = dst + r + c * R;  // dense, ld = R
        if (FULL || nvalid == V) {
          Raw<T, V> o;
#pragma unroll
          for (int j = 0; j < V; ++j) o.v[j] = narrow_to<T>::from(g[j].g[I]);
          vstore(q, o);
        } else {
#pragma unroll
          for (int j = 0; j < V; ++j)
            if (j < nvalid) sstore(q + j, narrow_to<T>::from(g[j].g[I]));
        }
      }
    } else if constexpr (L::mode == MBC) {
      constexpr int b = bc_rank<LL, I>();
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (FULL || j < nvalid) bpart[b][j] += g[j].g[I];
    }
    bwd_store<LL, V, CT, NB, FULL, I + 1>(g, bpart, ga, r, c, R, nvalid);
  }
}

// Last block of a row range: sum the column splits' row partials in split
// order (FP64, compensated) and write each_col leaves' gradients (dense).
template <class LL, int V, class CT, int I = 0>
FX_D void bwd_bc_finish(const GradArgs& ga, int64_t r, int64_t R, int nvalid) {
  if constexpr (I < tl_size<LL>::value) {
    using L = typename tl_at<LL, I>::type;
    using T = typename L::elem;
    if constexpr (L::mode == MBC) {
      constexpr int b = bc_rank<LL, I>();
      T* dst = static_cast<T*>(ga.g[L::slot]);
      if (dst) {
#pragma unroll
        for (int j = 0; j < V; ++j) {
          if (j < nvalid) {
            std::conditional_t<std::is_same<CT, double>::value, CompSum<double>, PlainSum<double>> a;
            a.init();
            for (int k = 0; k < ga.S; ++k) {
              double2 q = __ldcg(ga.part + (int64_t(b) * ga.S + k) * R + r + j);
              a.add(q.x);
              a.add(q.y);
            }
            sstore(dst + r + j, narrow_to<T>::from(CT(a.s + a.c)));
          }
        }
      }
    }
    bwd_bc_finish<LL, V, CT, I + 1>(ga, r, R, nvalid);
  }
}

// End of a backward row-range block: publish the each_col leaves' row
// partials; the last of the S splits of the row range combines them.
// Called by the `nthreads` computing threads only.
template <class LL, int V, class CT, int NBC, int NB>
FX_D void bwd_finish(const GradArgs& ga, ThreadSum<CT> (&bacc)[NB][V], int64_t R, int64_t r,
                     int nvalid, int s, int nthreads, const volatile int* abort = nullptr) {
  if constexpr (NBC > 0) {
#pragma unroll
    for (int b = 0; b < NBC; ++b)
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (j < nvalid)
          ga.part[(int64_t(b) * ga.S + s) * R + r + j] =
              make_double2(double(bacc[b][j].s), double(bacc[b][j].c));
    __threadfence();
    block_sync(nthreads);
    if (abort && *abort) return;  // a bounded wait gave up (recorded); no combine
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(ga.tickets + blockIdx.x, 1u) == unsigned(ga.S - 1);
    block_sync(nthreads);
    if (!last) return;
    __threadfence();
    bwd_bc_finish<LL, V, CT>(ga, r, R, nvalid);
    if (threadIdx.x == 0) ga.tickets[blockIdx.x] = 0u;
  }
}

template <class E, int V, int U, int NT>
__global__ void __launch_bounds__(NT) k_bwd(const E e, const Slots sl, const int64_t R,
                                            const int64_t C, const GradArgs ga) {
  using LL = leaves_t<E>;
  using CT = ct_of<E>;
  constexpr int NBC = count_mode<LL>(MBC);
  static_assert(count_mode<LL>(MT) == 0 && count_mode<LL>(MBR) == 0,
                "fused backward: plain and each_col leaves only");
  const int64_t r = (int64_t(blockIdx.x) * NT + threadIdx.x) * V;
  const int nvalid = clamp_valid(R - r, V);
  const int s = blockIdx.y;
  const int64_t cb = C * s / ga.S, ce = C * (s + 1) / ga.S;
  const CT gL = ga.gscale ? __ldg(static_cast<const CT*>(ga.gscale)) : CT(1);
  ThreadSum<CT> bacc[NBC > 0 ? NBC : 1][V];
#pragma unroll
  for (int b = 0; b < (NBC > 0 ? NBC : 1); ++b)
#pragma unroll
    for (int j = 0; j < V; ++j) bacc[b][j].init();
  if (nvalid > 0) {
    for (int64_t c = cb; c < ce; c += U) {
      Pack<LL, V, CT> p[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (c + u < ce) load_rc(p[u], sl, r, c + u, nvalid);
      CT bpart[NBC > 0 ? NBC : 1][V] = {};
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c + u < ce) {
          GradAcc<LL, CT, E> g[V];
          grad_lanes<V>(e, p[u], gL, g);
          bwd_store<LL, V, CT, (NBC > 0 ? NBC : 1)>(g, bpart, ga, r, c + u, R, nvalid);
        }
      }
      if constexpr (NBC > 0) {
#pragma unroll
        for (int b = 0; b < NBC; ++b)
#pragma unroll
          for (int j = 0; j < V; ++j) bacc[b][j].add(bpart[b][j]);
      }
    }
  }
  bwd_finish<LL, V, CT, NBC>(ga, bacc, R, r, nvalid, s, NT);
}

}  // namespace fx
