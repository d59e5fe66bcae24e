// plan.cuh - the compile-time fusion planner.
//
// 1. normalize(): pushes every transpose and broadcast down to the leaves
//    (trans(A op B) = trans(A) op trans(B); trans(trans(A)) = A; a transposed
//    each_col is an each_row), so the fused kernels see leaves with one of
//    four access modes (expr.cuh) and no structural nodes.
// 2. leaves_t<E>: the distinct (slot, mode) leaves in first-occurrence
//    order. The fused kernels load each of them once per element, however
//    often it appears in the tree (relu reads X twice, expr1 reads X and
//    X.t()).
// 3. Family selection (the kernel a tree runs on):
//      only MN leaves, contiguous, no reduction        -> flat stream (A3)
//      any MT leaf, broadcast, or strided layout       -> tiled (A4)
//      accu / norm root                                -> same, with a fused
//                                                         reduction epilogue (A5)
//      sum / max along a dimension                     -> dim reduction (A6)
//      with_accu(E, S): Z = E and s = accu(S)           -> E's family, S summed
//                                                         from the same registers
//    A matrix product node is a fusion boundary (has_prod_v): gemm.cuh
//    computes it first into a temporary, bound as a plain leaf of the rest.
#pragma once

#include "expr.cuh"

namespace fx {

// ---------------------------------------------------------------- type lists

template <class... Ts> struct TL {};

template <class L, class X> struct tl_push;
template <class... Ts, class X> struct tl_push<TL<Ts...>, X> { using type = TL<Ts..., X>; };

template <class L, int K, int M> struct tl_index;
template <int K, int M> struct tl_index<TL<>, K, M> { static constexpr int value = -1; };
template <class H, class... Ts, int K, int M> struct tl_index<TL<H, Ts...>, K, M> {
  static constexpr int rest = tl_index<TL<Ts...>, K, M>::value;
  static constexpr int value = (H::slot == K && H::mode == M) ? 0 : (rest < 0 ? -1 : rest + 1);
};

template <class L, class X> struct tl_add_unique {
  using type = std::conditional_t<(tl_index<L, X::slot, X::mode>::value >= 0), L,
                                  typename tl_push<L, X>::type>;
};

template <class L> struct tl_size;
template <class... Ts> struct tl_size<TL<Ts...>> { static constexpr int value = sizeof...(Ts); };

template <class L, int I> struct tl_at;
template <class H, class... Ts> struct tl_at<TL<H, Ts...>, 0> { using type = H; };
template <class H, class... Ts, int I> struct tl_at<TL<H, Ts...>, I> {
  using type = typename tl_at<TL<Ts...>, I - 1>::type;
};

// ---------------------------------------------------------------- leaf collection

template <class E, class Acc> struct collect;
template <int K, class T, int M, class Acc> struct collect<Leaf<K, T, M>, Acc> {
  using type = typename tl_add_unique<Acc, Leaf<K, T, M>>::type;
};
template <class Op, class L, class R, class Acc> struct collect<Bin<Op, L, R>, Acc> {
  using type = typename collect<R, typename collect<L, Acc>::type>::type;
};
template <class Op, class E, class Acc> struct collect<Un<Op, E>, Acc> {
  using type = typename collect<E, Acc>::type;
};
template <class Op, class E, class Acc> struct collect<SL<Op, E>, Acc> {
  using type = typename collect<E, Acc>::type;
};
template <class Op, class E, class Acc> struct collect<SR<Op, E>, Acc> {
  using type = typename collect<E, Acc>::type;
};
template <class E> using leaves_t = typename collect<E, TL<>>::type;

// Any leaf of a mode present?
template <class L, int M> struct tl_has_mode;
template <int M> struct tl_has_mode<TL<>, M> { static constexpr bool value = false; };
template <class H, class... Ts, int M> struct tl_has_mode<TL<H, Ts...>, M> {
  static constexpr bool value = H::mode == M || tl_has_mode<TL<Ts...>, M>::value;
};

// Compute type: double if every leaf stores double, else float. A double
// leaf in a float tree is read as its FP32 rounding (round to nearest), the
// conv_to<fmat> of the Sec. 4 expression expr3.
template <class L> struct tl_all_double;
template <> struct tl_all_double<TL<>> { static constexpr bool value = true; };
template <class H, class... Ts> struct tl_all_double<TL<H, Ts...>> {
  static constexpr bool value =
      std::is_same<typename H::elem, double>::value && tl_all_double<TL<Ts...>>::value;
};
template <class E>
using ct_of = std::conditional_t<tl_all_double<leaves_t<E>>::value, double, float>;

// Widest storage element among the leaves (sets the vector width).
template <class L> struct tl_max_elem;
template <> struct tl_max_elem<TL<>> { static constexpr int value = 1; };
template <class H, class... Ts> struct tl_max_elem<TL<H, Ts...>> {
  static constexpr int a = sizeof(typename H::elem), b = tl_max_elem<TL<Ts...>>::value;
  static constexpr int value = a > b ? a : b;
};

// ---------------------------------------------------------------- normalisation

template <class E, bool F> struct Norm;  // F: an odd number of transposes above

template <int K, class T, int M, bool F> struct Norm<Leaf<K, T, M>, F> {
  using type = Leaf<K, T, F ? flip_mode(M) : M>;
  static FX_HD type make(const Leaf<K, T, M>&) { return {}; }
};
template <class E, bool F> struct Norm<Tr<E>, F> {
  using type = typename Norm<E, !F>::type;
  static FX_HD type make(const Tr<E>& x) { return Norm<E, !F>::make(x.e); }
};
template <int K, class T, bool F> struct Norm<BCol<Leaf<K, T, MN>>, F> {
  using type = Leaf<K, T, F ? MBR : MBC>;
  static FX_HD type make(const BCol<Leaf<K, T, MN>>&) { return {}; }
};
template <int K, class T, bool F> struct Norm<BRow<Leaf<K, T, MN>>, F> {
  using type = Leaf<K, T, F ? MBC : MBR>;
  static FX_HD type make(const BRow<Leaf<K, T, MN>>&) { return {}; }
};
template <class Op, class L, class R, bool F> struct Norm<Bin<Op, L, R>, F> {
  using type = Bin<Op, typename Norm<L, F>::type, typename Norm<R, F>::type>;
  static FX_HD type make(const Bin<Op, L, R>& x) {
    return {{}, Norm<L, F>::make(x.l), Norm<R, F>::make(x.r)};
  }
};
template <class Op, class E, bool F> struct Norm<Un<Op, E>, F> {
  using type = Un<Op, typename Norm<E, F>::type>;
  static FX_HD type make(const Un<Op, E>& x) { return {{}, Norm<E, F>::make(x.e)}; }
};
template <class Op, class E, bool F> struct Norm<SL<Op, E>, F> {
  using type = SL<Op, typename Norm<E, F>::type>;
  static FX_HD type make(const SL<Op, E>& x) { return {{}, x.s, Norm<E, F>::make(x.e)}; }
};
template <class Op, class E, bool F> struct Norm<SR<Op, E>, F> {
  using type = SR<Op, typename Norm<E, F>::type>;
  static FX_HD type make(const SR<Op, E>& x) { return {{}, Norm<E, F>::make(x.e), x.s}; }
};
// Products: normalise the operands; a transposed product swaps and
// transposes them ((L R)^T = R^T L^T).
template <class L, class R> struct Norm<Prod<L, R>, false> {
  using type = Prod<typename Norm<L, false>::type, typename Norm<R, false>::type>;
  static FX_HD type make(const Prod<L, R>& x) {
    return {{}, Norm<L, false>::make(x.l), Norm<R, false>::make(x.r)};
  }
};
template <class L, class R> struct Norm<Prod<L, R>, true> {
  using type = Prod<typename Norm<R, true>::type, typename Norm<L, true>::type>;
  static FX_HD type make(const Prod<L, R>& x) {
    return {{}, Norm<R, true>::make(x.r), Norm<L, true>::make(x.l)};
  }
};
// Reductions: normalise the operand (a reduction is never transposed here).
template <class E> struct Norm<Accu<E>, false> {
  using type = Accu<typename Norm<E, false>::type>;
  static FX_HD type make(const Accu<E>& x) { return {{}, Norm<E, false>::make(x.e)}; }
};
template <class E> struct Norm<Norm2<E>, false> {
  using type = Norm2<typename Norm<E, false>::type>;
  static FX_HD type make(const Norm2<E>& x) { return {{}, Norm<E, false>::make(x.e)}; }
};
template <class E, int D> struct Norm<SumDim<E, D>, false> {
  using type = SumDim<typename Norm<E, false>::type, D>;
  static FX_HD type make(const SumDim<E, D>& x) { return {{}, Norm<E, false>::make(x.e)}; }
};
template <class E, int D> struct Norm<MaxDim<E, D>, false> {
  using type = MaxDim<typename Norm<E, false>::type, D>;
  static FX_HD type make(const MaxDim<E, D>& x) { return {{}, Norm<E, false>::make(x.e)}; }
};

template <class E, class S> struct Norm<WithAccu<E, S>, false> {
  using type = WithAccu<typename Norm<E, false>::type, typename Norm<S, false>::type>;
  static FX_HD type make(const WithAccu<E, S>& x) {
    return {{}, {{}, Norm<E, false>::make(x.both.l), Norm<S, false>::make(x.both.r)}};
  }
};

template <class E> FX_HD typename Norm<E, false>::type normalize(const E& e) {
  return Norm<E, false>::make(e);
}

// ---------------------------------------------------------------- root kinds

template <class E> struct root_of { static constexpr int kind = FX_KIND_ELEMENTWISE; using inner = E; };
template <class E> struct root_of<Accu<E>> { static constexpr int kind = FX_KIND_FULL_REDUCE; using inner = E; };
template <class E> struct root_of<Norm2<E>> { static constexpr int kind = FX_KIND_FULL_REDUCE; using inner = E; };
template <class E, int D> struct root_of<SumDim<E, D>> { static constexpr int kind = FX_KIND_DIM_REDUCE; using inner = E; };
template <class E, int D> struct root_of<MaxDim<E, D>> { static constexpr int kind = FX_KIND_DIM_REDUCE; using inner = E; };

template <class E, class S> struct root_of<WithAccu<E, S>> { static constexpr int kind = FX_KIND_MULTI; using inner = Bin<OpFirst, E, S>; };

template <class E> struct is_with_accu { static constexpr bool value = false; };
template <class E, class S> struct is_with_accu<WithAccu<E, S>> { static constexpr bool value = true; };

template <class E> FX_HD const E& inner_of(const E& e) { return e; }
template <class E, class S> FX_HD const Bin<OpFirst, E, S>& inner_of(const WithAccu<E, S>& e) { return e.both; }
template <class E> FX_HD const E& inner_of(const Accu<E>& e) { return e.e; }
template <class E> FX_HD const E& inner_of(const Norm2<E>& e) { return e.e; }
template <class E, int D> FX_HD const E& inner_of(const SumDim<E, D>& e) { return e.e; }
template <class E, int D> FX_HD const E& inner_of(const MaxDim<E, D>& e) { return e.e; }

// Matrix products inside a tree (fusion boundaries).
template <class E> struct has_prod { static constexpr bool value = false; };
template <class L, class R> struct has_prod<Prod<L, R>> { static constexpr bool value = true; };
template <class Op, class L, class R> struct has_prod<Bin<Op, L, R>> {
  static constexpr bool value = has_prod<L>::value || has_prod<R>::value;
};
template <class Op, class E> struct has_prod<Un<Op, E>> { static constexpr bool value = has_prod<E>::value; };
template <class Op, class E> struct has_prod<SL<Op, E>> { static constexpr bool value = has_prod<E>::value; };
template <class Op, class E> struct has_prod<SR<Op, E>> { static constexpr bool value = has_prod<E>::value; };
template <class E> struct has_prod<Tr<E>> { static constexpr bool value = has_prod<E>::value; };
template <class E> constexpr bool has_prod_v = has_prod<E>::value;

// Number of operator nodes (unfused launches needed for the element-wise part).
template <class E> struct op_count { static constexpr int value = 0; };
template <class Op, class L, class R> struct op_count<Bin<Op, L, R>> {
  static constexpr int value = 1 + op_count<L>::value + op_count<R>::value;
};
template <class Op, class E> struct op_count<Un<Op, E>> { static constexpr int value = 1 + op_count<E>::value; };
template <class Op, class E> struct op_count<SL<Op, E>> { static constexpr int value = 1 + op_count<E>::value; };
template <class Op, class E> struct op_count<SR<Op, E>> { static constexpr int value = 1 + op_count<E>::value; };

// Vector width in elements for a 16-byte (or 32-byte) access of the widest leaf.
template <class E, int BYTES> FX_HD constexpr int vec_width() {
  return BYTES / tl_max_elem<leaves_t<E>>::value;
}

}  // namespace fx
