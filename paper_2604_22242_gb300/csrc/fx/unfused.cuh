// unfused.cuh - the one-kernel-per-operator baseline.
//
// The same tree is evaluated node by node, the way an eager array library
// runs it: every operator node is its own launch that reads its operands
// from memory and writes its result, in the storage type, to a temporary
// in library workspace; a transposed leaf is materialised by a transpose
// launch; a broadcast leaf is read by the operator that uses it; the
// terminal reduction is one more launch over the materialised operand.
// Each single-operator launch uses the same kernels (and vector widths) as
// the fused path, so the comparison measures fusion alone.
#pragma once

#include "launch.cuh"

namespace fx {

// Mode and element type under which a node's value is read by its parent.
template <class E, class T> struct uview { static constexpr int mode = MN; using elem = T; };
template <int K, class T2, int M, class T> struct uview<Leaf<K, T2, M>, T> {
  static constexpr int mode = (M == MT ? MN : M);
  using elem = T2;
};

template <class E> struct mt_occ { static constexpr int value = 0; };
template <int K, class T, int M> struct mt_occ<Leaf<K, T, M>> { static constexpr int value = M == MT ? 1 : 0; };
template <class Op, class L, class R> struct mt_occ<Bin<Op, L, R>> {
  static constexpr int value = mt_occ<L>::value + mt_occ<R>::value;
};
template <class Op, class E> struct mt_occ<Un<Op, E>> { static constexpr int value = mt_occ<E>::value; };
template <class Op, class E> struct mt_occ<SL<Op, E>> { static constexpr int value = mt_occ<E>::value; };
template <class Op, class E> struct mt_occ<SR<Op, E>> { static constexpr int value = mt_occ<E>::value; };

template <class E> constexpr int unfused_temps() { return op_count<E>::value + mt_occ<E>::value; }

struct UState {
  Run r;
  int64_t R, C;
  size_t es;
  char* base;
  size_t cap, used;
};

// The node's result goes to *dst when given (the root writes the output
// directly, as an eager library's last operator does), else to a temporary.
inline fx_status utemp(UState& u, Binding& b, const Binding* dst = nullptr) {
  if (dst) {
    b = *dst;
    return FX_OK;
  }
  const size_t bytes = ((size_t(u.R) * u.C * u.es) + 255) & ~size_t(255);
  if (u.used + bytes > u.cap) return fail(FX_E_NOMEM, "unfused temporaries exceed their workspace");
  b.p = u.base + u.used;
  b.rows = u.R;
  b.cols = u.C;
  b.ld = u.R > 0 ? u.R : 1;
  b.bound = true;
  u.used += bytes;
  return FX_OK;
}

template <class T, class E> struct Unf;

template <class T, int K, class T2, int M> struct Unf<T, Leaf<K, T2, M>> {
  static fx_status run(UState& u, const Leaf<K, T2, M>&, Binding& out, const Binding* dst) {
    if (M == MT || dst) {  // a transpose (or, for a bare-leaf tree, a copy) launch
      Binding b2[2] = {u.r.b[K], Binding{}};
      FX_TRY(utemp(u, b2[1], dst));
      Run r2 = u.r;
      r2.b = b2;
      r2.n_in = 1;
      FX_TRY(run_elementwise<T>(r2, Leaf<0, T2, (M == MT ? MT : M)>{}));
      out = b2[1];
    } else {
      out = u.r.b[K];
    }
    return FX_OK;
  }
};

template <class T, class Op, class A> struct Unf<T, Un<Op, A>> {
  static fx_status run(UState& u, const Un<Op, A>& e, Binding& out, const Binding* dst) {
    Binding b2[2];
    FX_TRY((Unf<T, A>::run(u, e.e, b2[0], nullptr)));
    FX_TRY(utemp(u, b2[1], dst));
    Run r2 = u.r;
    r2.b = b2;
    r2.n_in = 1;
    using LA = Leaf<0, typename uview<A, T>::elem, uview<A, T>::mode>;
    FX_TRY(run_elementwise<T>(r2, Un<Op, LA>{}));
    out = b2[1];
    return FX_OK;
  }
};

template <class T, class Op, class A> struct Unf<T, SL<Op, A>> {
  static fx_status run(UState& u, const SL<Op, A>& e, Binding& out, const Binding* dst) {
    Binding b2[2];
    FX_TRY((Unf<T, A>::run(u, e.e, b2[0], nullptr)));
    FX_TRY(utemp(u, b2[1], dst));
    Run r2 = u.r;
    r2.b = b2;
    r2.n_in = 1;
    using LA = Leaf<0, typename uview<A, T>::elem, uview<A, T>::mode>;
    FX_TRY(run_elementwise<T>(r2, SL<Op, LA>{{}, e.s, LA{}}));
    out = b2[1];
    return FX_OK;
  }
};

template <class T, class Op, class A> struct Unf<T, SR<Op, A>> {
  static fx_status run(UState& u, const SR<Op, A>& e, Binding& out, const Binding* dst) {
    Binding b2[2];
    FX_TRY((Unf<T, A>::run(u, e.e, b2[0], nullptr)));
    FX_TRY(utemp(u, b2[1], dst));
    Run r2 = u.r;
    r2.b = b2;
    r2.n_in = 1;
    using LA = Leaf<0, typename uview<A, T>::elem, uview<A, T>::mode>;
    FX_TRY(run_elementwise<T>(r2, SR<Op, LA>{{}, LA{}, e.s}));
    out = b2[1];
    return FX_OK;
  }
};

template <class T, class Op, class A, class B> struct Unf<T, Bin<Op, A, B>> {
  static fx_status run(UState& u, const Bin<Op, A, B>& e, Binding& out, const Binding* dst) {
    Binding b3[3];
    FX_TRY((Unf<T, A>::run(u, e.l, b3[0], nullptr)));
    FX_TRY((Unf<T, B>::run(u, e.r, b3[1], nullptr)));
    FX_TRY(utemp(u, b3[2], dst));
    Run r2 = u.r;
    r2.b = b3;
    r2.n_in = 2;
    using LA = Leaf<0, typename uview<A, T>::elem, uview<A, T>::mode>;
    using LB = Leaf<1, typename uview<B, T>::elem, uview<B, T>::mode>;
    FX_TRY(run_elementwise<T>(r2, Bin<Op, LA, LB>{{}, LA{}, LB{}}));
    out = b3[2];
    return FX_OK;
  }
};

template <class Root> struct reroot;  // the root node over a materialised operand
template <class E> struct reroot<Accu<E>> { template <class L> using type = Accu<L>; };
template <class E> struct reroot<Norm2<E>> { template <class L> using type = Norm2<L>; };
template <class E, int D> struct reroot<SumDim<E, D>> { template <class L> using type = SumDim<L, D>; };
template <class E, int D> struct reroot<MaxDim<E, D>> { template <class L> using type = MaxDim<L, D>; };

// `over`: the binding table and input count to use instead of the object's
// (trees whose matrix products were computed into temporaries first).
template <class T, class Root>
fx_status run_unfused(fx_expr* x, const Root& root, int kind, cudaStream_t st,
                      const Run* over = nullptr) {
  using E = typename root_of<Root>::inner;
  using LL = leaves_t<E>;
  Run r = over ? *over : run_of(x, st);
  r.tune = Tune{};  // one-operator kernels at the library's default shapes, whatever the tree's tuning
  const E& e = inner_of(root);
  int64_t R = 0, C = 0;
  if (!infer_shape<LL>(r.b, R, C)) return fail(FX_E_SHAPE, "no matrix leaf to take the shape from");
  FX_TRY(check_leaves<LL>(r.b, R, C));
  constexpr int ntmp = unfused_temps<E>();
  const size_t per = ((size_t(R) * C * sizeof(T)) + 255) & ~size_t(255);
  FX_TRY(x->ws_tmp.ensure(per * (ntmp > 0 ? ntmp : 1), st));
  UState u{r, R, C, sizeof(T), static_cast<char*>(x->ws_tmp.p), x->ws_tmp.bytes, 0};
  constexpr int rk = root_of<Root>::kind;
  if constexpr (is_with_accu<Root>::value) {
    // Z = E as its own chain of launches into Z, then S's chain into a
    // temporary and accu over it (an eager library evaluates the two
    // expressions one after the other)
    const Binding& zb = r.b[r.n_in];
    if (zb.rows != R || zb.cols != C) return fail(FX_E_SHAPE, "output shape differs from the tree's");
    Binding z, v;
    FX_TRY((Unf<T, decltype(e.l)>::run(u, e.l, z, &zb)));
    FX_TRY((Unf<T, decltype(e.r)>::run(u, e.r, v, nullptr)));
    Binding b3[2] = {v, r.b[r.n_in + 1]};
    Run r3 = r;
    r3.b = b3;
    r3.n_in = 1;
    using S = decltype(e.r);
    using LV = Leaf<0, typename uview<S, T>::elem, uview<S, T>::mode>;
    return run_full_reduce<T>(r3, Accu<LV>{});
  } else if constexpr (rk == FX_KIND_ELEMENTWISE) {
    const Binding& zb = r.b[r.n_in];
    if (zb.rows != R || zb.cols != C) return fail(FX_E_SHAPE, "output shape differs from the tree's");
    Binding z;
    FX_TRY((Unf<T, E>::run(u, e, z, &zb)));
    if (kind == FX_KIND_MULTI) {  // accu(Z) as its own launch over the stored Z
      Binding b3[2] = {zb, r.b[r.n_in + 1]};
      Run r3 = r;
      r3.b = b3;
      r3.n_in = 1;
      FX_TRY(run_full_reduce<T>(r3, Accu<Leaf<0, T, MN>>{}));
    }
    return FX_OK;
  } else {
    Binding v;
    FX_TRY((Unf<T, E>::run(u, e, v, nullptr)));
    Binding b2[2] = {v, r.b[r.n_in]};
    Run r2 = r;
    r2.b = b2;
    r2.n_in = 1;
    using LV = Leaf<0, typename uview<E, T>::elem, uview<E, T>::mode>;
    using Root2 = typename reroot<Root>::template type<LV>;
    return run_root<T>(r2, Root2{}, FX_KIND_ELEMENTWISE);
  }
}

}  // namespace fx
