// expr.cuh - the expression-template front end.
//
// As in the paper (Sec. 3), an expression's C++ type is its abstract syntax
// tree: A % B + 3.5 * exp(C) - trans(D) has the type
//   Bin<OpSub, Bin<OpAdd, Bin<OpMul, A, B>, SL<OpMul, Un<OpExp, C>>>, Tr<D>>
// and nothing is evaluated when it is built. Node objects carry only what
// must be known at run time: the scalar operands (the paper's `aux`).
// Leaves name an argument slot (K) and a storage element type; the buffers
// behind the slots are bound at evaluation (fx_expr_bind), so one compiled
// tree serves any shapes and leading dimensions.
//
// Element access follows Sec. 3: a leaf yields its element (row, col); a
// transpose swaps row and col for its operand; a scalar node wraps its
// operand's value. The planner (plan.cuh) pushes every transpose and
// broadcast down onto the leaves, so that the kernels see only four leaf
// access modes:
//   MN  element (r, c)           of an R x C matrix
//   MT  element (c, r)           of a C x R matrix   (a transposed leaf)
//   MBC element r of a vector    (each_col: repeated over the columns)
//   MBR element c of a vector    (each_row: repeated over the rows)
#pragma once

#include <cmath>

#include "core.cuh"

namespace fx {

enum Mode : int { MN = 0, MT = 1, MBC = 2, MBR = 3 };

FX_HD constexpr int flip_mode(int m) {
  return m == MN ? MT : m == MT ? MN : m == MBC ? MBR : MBC;
}

// ---------------------------------------------------------------- operators
//
// Each operator tag has the element function f and the partial derivatives
// used by the fused backward pass (k_bwd, k_bwd_bulk).

FX_D float m_exp(float x) { return ::expf(x); }
FX_D double m_exp(double x) { return ::exp(x); }
FX_D float m_log(float x) { return ::logf(x); }
FX_D double m_log(double x) { return ::log(x); }
FX_D float m_sqrt(float x) { return ::sqrtf(x); }
FX_D double m_sqrt(double x) { return ::sqrt(x); }
FX_D float m_abs(float x) { return ::fabsf(x); }
FX_D double m_abs(double x) { return ::fabs(x); }
FX_D float m_tanh(float x) { return ::tanhf(x); }
FX_D double m_tanh(double x) { return ::tanh(x); }
// 1 / x correctly rounded (the same value as the IEEE division 1 / x,
// without the general division's numerator handling)
FX_D float m_rcp(float x) { return __frcp_rn(x); }
FX_D double m_rcp(double x) { return __drcp_rn(x); }
FX_D float m_pow(float x, float k) { return ::powf(x, k); }
FX_D double m_pow(double x, double k) { return ::pow(x, k); }
template <class C> FX_D C m_sign(C x) { return x > C(0) ? C(1) : (x < C(0) ? C(-1) : C(0)); }
template <class C> FX_D C m_gt(C a, C b) { return a > b ? C(1) : C(0); }

// exp inside sigmoid: CUDA's fast __expf for FP32 (its error, a few ulp
// plus |x| * 2^-23 relative from scaling x by log2(e), is further damped by
// the factor 1 - sigmoid in the result), exp for FP64.
FX_D float m_exp_sig(float x) { return __expf(x); }
FX_D double m_exp_sig(double x) { return ::exp(x); }
// The reciprocal inside sigmoid: the hardware's approximate reciprocal for
// FP32 (one instruction, within about one ulp; its argument 1 + exp(-x) is
// at least 1, so flushing subnormals changes nothing), the correctly
// rounded one for FP64.
FX_D float m_rcp_sig(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
FX_D double m_rcp_sig(double x) { return __drcp_rn(x); }

// ---------------------------------------------------------------- lane pairs
//
// F2: two FP32 lanes carried as one value. Blackwell issues FP32 add,
// subtract, multiply and fma on a register pair as one instruction
// (add/sub/mul/fma.rn.f32x2), so a tree evaluated on pairs of rows issues
// about half as many arithmetic instructions. Each lane is rounded exactly
// as the scalar FP32 operation rounds it; transcendentals, division and
// comparisons run lane by lane.
struct F2 {
  float x, y;
  F2() = default;
  FX_HD constexpr F2(float a, float b) : x(a), y(b) {}
  template <class S, std::enable_if_t<std::is_arithmetic<S>::value, int> = 0>
  FX_HD constexpr explicit F2(S s) : x(float(s)), y(float(s)) {}
};
FX_D uint64_t f2_bits(F2 a) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
FX_D F2 f2_of(uint64_t r) {
  F2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
FX_D F2 operator+(F2 a, F2 b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_of(r);
}
FX_D F2 operator-(F2 a, F2 b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_of(r);
}
FX_D F2 operator*(F2 a, F2 b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_of(r);
}
FX_D F2 m_fma(F2 a, F2 b, F2 c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
  return f2_of(r);
}
FX_D F2 operator/(F2 a, F2 b) { return F2(a.x / b.x, a.y / b.y); }
FX_D F2 operator-(F2 a) { return F2(-a.x, -a.y); }
FX_D F2& operator+=(F2& a, F2 b) { return a = a + b; }
// equal in both lanes (used on broadcast scalars)
FX_D bool operator==(F2 a, F2 b) { return a.x == b.x && a.y == b.y; }
FX_D F2 m_exp(F2 a) { return F2(m_exp(a.x), m_exp(a.y)); }
FX_D F2 m_log(F2 a) { return F2(m_log(a.x), m_log(a.y)); }
FX_D F2 m_sqrt(F2 a) { return F2(m_sqrt(a.x), m_sqrt(a.y)); }
FX_D F2 m_abs(F2 a) { return F2(m_abs(a.x), m_abs(a.y)); }
FX_D F2 m_tanh(F2 a) { return F2(m_tanh(a.x), m_tanh(a.y)); }
FX_D F2 m_rcp(F2 a) { return F2(m_rcp(a.x), m_rcp(a.y)); }
FX_D F2 m_pow(F2 a, F2 k) { return F2(m_pow(a.x, k.x), m_pow(a.y, k.y)); }
FX_D F2 m_sign(F2 a) { return F2(m_sign(a.x), m_sign(a.y)); }
FX_D F2 m_gt(F2 a, F2 b) { return F2(m_gt(a.x, b.x), m_gt(a.y, b.y)); }
FX_D F2 m_exp_sig(F2 a) { return F2(m_exp_sig(a.x), m_exp_sig(a.y)); }
FX_D F2 m_rcp_sig(F2 a) { return F2(m_rcp_sig(a.x), m_rcp_sig(a.y)); }

struct OpAdd {
  template <class C> static FX_D C f(C a, C b) { return a + b; }
  template <class C> static FX_D void d(C, C, C& da, C& db) { da = C(1); db = C(1); }
};
struct OpSub {
  template <class C> static FX_D C f(C a, C b) { return a - b; }
  template <class C> static FX_D void d(C, C, C& da, C& db) { da = C(1); db = C(-1); }
};
struct OpMul {
  template <class C> static FX_D C f(C a, C b) { return a * b; }
  template <class C> static FX_D void d(C a, C b, C& da, C& db) { da = b; db = a; }
};
struct OpDiv {
  template <class C> static FX_D C f(C a, C b) { return a / b; }
  template <class C> static FX_D void d(C a, C b, C& da, C& db) {
    da = m_rcp(b);
    db = -a / (b * b);
  }
};
struct OpPow {  // a ^ b (b is a scalar in the trees built here; 2 and 3 by multiplication)
  template <class C> static FX_D C f(C a, C b) {
    if (b == C(2)) return a * a;
    if (b == C(3)) return a * a * a;
    return m_pow(a, b);
  }
  template <class C> static FX_D void d(C a, C b, C& da, C& db) {
    da = b == C(2) ? C(2) * a : (b == C(3) ? C(3) * a * a : b * m_pow(a, b - C(1)));
    db = C(0);
  }
};
struct OpGt {  // 1 where a > b, else 0 (the mask X > 0 of the relu expression)
  template <class C> static FX_D C f(C a, C b) { return m_gt(a, b); }
  template <class C> static FX_D void d(C, C, C& da, C& db) { da = C(0); db = C(0); }
};

// The first of two values. Joins a stored tree and a second tree over the
// same leaves into one node, so that one load of the leaves serves both
// (the multi-output root WithAccu); the second value is read by the
// epilogue from the same registers, not through this node.
struct OpFirst {
  template <class C> static FX_D C f(C a, C) { return a; }
  template <class C> static FX_D void d(C, C, C& da, C& db) { da = C(1); db = C(0); }
};

// Operators whose partial derivatives are the constants 1, -1 or 0: the
// reverse pass hands on the adjoint itself, its negation, or nothing,
// instead of multiplying by the constant (exact either way; the product
// would cost an instruction on lane pairs, where the compiler does not
// fold it).
template <class Op> struct lin_d { static constexpr bool value = false; };
template <> struct lin_d<OpAdd> { static constexpr bool value = true; static constexpr int a = 1, b = 1; };
template <> struct lin_d<OpSub> { static constexpr bool value = true; static constexpr int a = 1, b = -1; };
template <> struct lin_d<OpFirst> { static constexpr bool value = true; static constexpr int a = 1, b = 0; };
template <int S, class CT> FX_D CT lin_adj(CT adj) {
  if constexpr (S == 1) return adj;
  else if constexpr (S == -1) return -adj;
  else return CT(0);
}

struct OpNeg {
  template <class C> static FX_D C f(C a) { return -a; }
  template <class C> static FX_D C d(C, C) { return C(-1); }
};
struct OpExp {
  template <class C> static FX_D C f(C a) { return m_exp(a); }
  template <class C> static FX_D C d(C, C z) { return z; }
};
struct OpLog {
  template <class C> static FX_D C f(C a) { return m_log(a); }
  template <class C> static FX_D C d(C a, C) { return C(1) / a; }
};
struct OpSqrt {
  template <class C> static FX_D C f(C a) { return m_sqrt(a); }
  template <class C> static FX_D C d(C, C z) { return C(0.5) / z; }
};
struct OpAbs {
  template <class C> static FX_D C f(C a) { return m_abs(a); }
  template <class C> static FX_D C d(C a, C) { return m_sign(a); }
};
struct OpSquare {
  template <class C> static FX_D C f(C a) { return a * a; }
  template <class C> static FX_D C d(C a, C) { return C(2) * a; }
};
struct OpSigmoid {  // Sec. 4: sigmoid = 1 / (1 + exp(-X))
  template <class C> static FX_D C f(C a) { return m_rcp_sig(C(1) + m_exp_sig(-a)); }
  template <class C> static FX_D C d(C, C z) { return z * (C(1) - z); }
};
struct OpTanh {
  template <class C> static FX_D C f(C a) { return m_tanh(a); }
  template <class C> static FX_D C d(C, C z) { return C(1) - z * z; }
};

// ---------------------------------------------------------------- nodes

struct ExprBase {};

// Reverse mode over one element: fwd(c) evaluates every node of the tree
// once and keeps each node's value with its children's (a tape held in
// registers); rev(tape, adj, g) walks the same values back down, giving
// each leaf its adjoint. bwd(c, adj, g) is the two passes in a row.
template <class CT, class... Ch> struct Tape;
template <class CT> struct Tape<CT> { CT v; };
template <class CT, class A> struct Tape<CT, A> { CT v; A a; };
template <class CT, class A, class B> struct Tape<CT, A, B> { CT v; A a; B b; };

template <int K, class T, int M = MN> struct Leaf : ExprBase {
  static_assert(K >= 0 && K < FX_MAX_SLOTS, "slot out of range");
  using elem = T;
  static constexpr int slot = K;
  static constexpr int mode = M;
  template <class Ctx> FX_D typename Ctx::CT ev(const Ctx& c) const {
    return c.template leaf<K, M>();
  }
  template <class Ctx> FX_D Tape<typename Ctx::CT> fwd(const Ctx& c) const { return {ev(c)}; }
  template <class CT, class Tp, class G> FX_D void rev(const Tp&, CT adj, G& g) const {
    g.template add<K, M>(adj);
  }
  template <class Ctx, class G>
  FX_D void bwd(const Ctx&, typename Ctx::CT adj, G& g) const {
    g.template add<K, M>(adj);
  }
};

template <class Op, class L, class R> struct Bin;
template <class E> struct is_mul_bin : std::false_type {};
template <class L, class R> struct is_mul_bin<Bin<OpMul, L, R>> : std::true_type {};

template <class Op, class L, class R> struct Bin : ExprBase {
  L l;
  R r;
  // On lane pairs a product added to something is one fma (the scalar path
  // leaves that contraction to the compiler).
  static constexpr bool fma_l = std::is_same<Op, OpAdd>::value && is_mul_bin<L>::value;
  static constexpr bool fma_r = std::is_same<Op, OpAdd>::value && !fma_l && is_mul_bin<R>::value;
  template <class Ctx> FX_D typename Ctx::CT ev(const Ctx& c) const {
    if constexpr (std::is_same<typename Ctx::CT, F2>::value && fma_l) {
      return m_fma(l.l.ev(c), l.r.ev(c), r.ev(c));
    } else if constexpr (std::is_same<typename Ctx::CT, F2>::value && fma_r) {
      return m_fma(r.l.ev(c), r.r.ev(c), l.ev(c));
    } else {
      return Op::f(l.ev(c), r.ev(c));
    }
  }
  template <class Ctx> FX_D auto fwd(const Ctx& c) const {
    using CT = typename Ctx::CT;
    const auto a = l.fwd(c);
    const auto b = r.fwd(c);
    if constexpr (std::is_same<CT, F2>::value && fma_l) {
      return Tape<CT, decltype(a), decltype(b)>{m_fma(a.a.v, a.b.v, b.v), a, b};
    } else if constexpr (std::is_same<CT, F2>::value && fma_r) {
      return Tape<CT, decltype(a), decltype(b)>{m_fma(b.a.v, b.b.v, a.v), a, b};
    } else {
      return Tape<CT, decltype(a), decltype(b)>{Op::f(a.v, b.v), a, b};
    }
  }
  template <class CT, class Tp, class G> FX_D void rev(const Tp& t, CT adj, G& g) const {
    if constexpr (lin_d<Op>::value) {
      l.rev(t.a, lin_adj<lin_d<Op>::a>(adj), g);
      if constexpr (lin_d<Op>::b != 0) r.rev(t.b, lin_adj<lin_d<Op>::b>(adj), g);
    } else {
      CT da, db;
      Op::d(t.a.v, t.b.v, da, db);
      l.rev(t.a, CT(adj * da), g);
      r.rev(t.b, CT(adj * db), g);
    }
  }
  template <class Ctx, class G>
  FX_D void bwd(const Ctx& c, typename Ctx::CT adj, G& g) const {
    rev(fwd(c), adj, g);
  }
};

template <class Op, class E> struct Un : ExprBase {
  E e;
  template <class Ctx> FX_D typename Ctx::CT ev(const Ctx& c) const { return Op::f(e.ev(c)); }
  template <class Ctx> FX_D auto fwd(const Ctx& c) const {
    const auto a = e.fwd(c);
    return Tape<typename Ctx::CT, decltype(a)>{Op::f(a.v), a};
  }
  // the derivative may use the node's own value z = f(a) (exp, sigmoid, tanh)
  template <class CT, class Tp, class G> FX_D void rev(const Tp& t, CT adj, G& g) const {
    if constexpr (std::is_same<Op, OpNeg>::value) {
      e.rev(t.a, CT(-adj), g);
    } else {
      e.rev(t.a, CT(adj * Op::d(t.a.v, t.v)), g);
    }
  }
  template <class Ctx, class G>
  FX_D void bwd(const Ctx& c, typename Ctx::CT adj, G& g) const {
    rev(fwd(c), adj, g);
  }
};

// scalar on the left: s op e; scalar on the right: e op s
template <class Op, class E> struct SL : ExprBase {
  double s;
  E e;
  template <class Ctx> FX_D typename Ctx::CT ev(const Ctx& c) const {
    using CT = typename Ctx::CT;
    return Op::f(CT(s), e.ev(c));
  }
  template <class Ctx> FX_D auto fwd(const Ctx& c) const {
    using CT = typename Ctx::CT;
    const auto b = e.fwd(c);
    return Tape<CT, decltype(b)>{Op::f(CT(s), b.v), b};
  }
  template <class CT, class Tp, class G> FX_D void rev(const Tp& t, CT adj, G& g) const {
    if constexpr (lin_d<Op>::value) {
      if constexpr (lin_d<Op>::b != 0) e.rev(t.a, lin_adj<lin_d<Op>::b>(adj), g);
    } else {
      CT da, db;
      Op::d(CT(s), t.a.v, da, db);
      e.rev(t.a, CT(adj * db), g);
    }
  }
  template <class Ctx, class G>
  FX_D void bwd(const Ctx& c, typename Ctx::CT adj, G& g) const {
    rev(fwd(c), adj, g);
  }
};
template <class Op, class E> struct SR : ExprBase {
  E e;
  double s;
  template <class Ctx> FX_D typename Ctx::CT ev(const Ctx& c) const {
    using CT = typename Ctx::CT;
    return Op::f(e.ev(c), CT(s));
  }
  template <class Ctx> FX_D auto fwd(const Ctx& c) const {
    using CT = typename Ctx::CT;
    const auto a = e.fwd(c);
    return Tape<CT, decltype(a)>{Op::f(a.v, CT(s)), a};
  }
  template <class CT, class Tp, class G> FX_D void rev(const Tp& t, CT adj, G& g) const {
    if constexpr (lin_d<Op>::value) {
      e.rev(t.a, lin_adj<lin_d<Op>::a>(adj), g);
    } else {
      CT da, db;
      Op::d(t.a.v, CT(s), da, db);
      e.rev(t.a, CT(adj * da), g);
    }
  }
  template <class Ctx, class G>
  FX_D void bwd(const Ctx& c, typename Ctx::CT adj, G& g) const {
    rev(fwd(c), adj, g);
  }
};

// Transposes and broadcasts exist only before planning (plan.cuh removes them).
template <class E> struct Tr : ExprBase { E e; };
template <class E> struct BCol : ExprBase { E e; };
template <class E> struct BRow : ExprBase { E e; };

// Matrix product: a fusion boundary. Kept in the type so that a tree can
// name it; the fused kernels reject it (it must be materialised first).
template <class L, class R> struct Prod : ExprBase { L l; R r; };

// Two results over shared leaves (only at the root): Z = e, stored, and
// s = accu(side), both from one pass over the union of their leaves.
template <class E, class S> struct WithAccu : ExprBase { Bin<OpFirst, E, S> both; };

// Terminal reductions (only at the root).
template <class E> struct Accu : ExprBase { E e; };
template <class E> struct Norm2 : ExprBase { E e; };
template <class E, int D> struct SumDim : ExprBase { E e; };
template <class E, int D> struct MaxDim : ExprBase { E e; };

// How often leaf (K, M) occurs in a planned tree (the reverse pass visits
// each occurrence once).
template <class E, int K, int M> struct leaf_count : std::integral_constant<int, 0> {};
template <int K2, class T, int M2, int K, int M>
struct leaf_count<Leaf<K2, T, M2>, K, M> : std::integral_constant<int, (K2 == K && M2 == M) ? 1 : 0> {};
template <class Op, class L, class R, int K, int M>
struct leaf_count<Bin<Op, L, R>, K, M>
    : std::integral_constant<int, leaf_count<L, K, M>::value + leaf_count<R, K, M>::value> {};
template <class Op, class E, int K, int M>
struct leaf_count<Un<Op, E>, K, M> : leaf_count<E, K, M> {};
template <class Op, class E, int K, int M>
struct leaf_count<SL<Op, E>, K, M> : leaf_count<E, K, M> {};
template <class Op, class E, int K, int M>
struct leaf_count<SR<Op, E>, K, M> : leaf_count<E, K, M> {};

template <class E>
constexpr bool is_expr_v = std::is_base_of<ExprBase, std::decay_t<E>>::value;

template <class A, class B>
using both_expr = std::enable_if_t<is_expr_v<A> && is_expr_v<B>, int>;
template <class A> using one_expr = std::enable_if_t<is_expr_v<A>, int>;

// ---------------------------------------------------------------- user syntax
// Armadillo-style, as in the paper: % is the Schur product, * with two
// matrices is the matrix product, trans(X) / X.t() is the transpose.

template <int K, class T> FX_HD Leaf<K, T> in() { return {}; }

template <class A, class B, both_expr<A, B> = 0> FX_HD Bin<OpAdd, A, B> operator+(A a, B b) {
  return {{}, a, b};
}
template <class A, class B, both_expr<A, B> = 0> FX_HD Bin<OpSub, A, B> operator-(A a, B b) {
  return {{}, a, b};
}
template <class A, class B, both_expr<A, B> = 0> FX_HD Bin<OpMul, A, B> operator%(A a, B b) {
  return {{}, a, b};
}
template <class A, class B, both_expr<A, B> = 0> FX_HD Bin<OpDiv, A, B> operator/(A a, B b) {
  return {{}, a, b};
}
template <class A, class B, both_expr<A, B> = 0> FX_HD Prod<A, B> operator*(A a, B b) {
  return {{}, a, b};
}
template <class A, one_expr<A> = 0> FX_HD SL<OpAdd, A> operator+(double s, A a) { return {{}, s, a}; }
template <class A, one_expr<A> = 0> FX_HD SR<OpAdd, A> operator+(A a, double s) { return {{}, a, s}; }
template <class A, one_expr<A> = 0> FX_HD SL<OpSub, A> operator-(double s, A a) { return {{}, s, a}; }
template <class A, one_expr<A> = 0> FX_HD SR<OpSub, A> operator-(A a, double s) { return {{}, a, s}; }
template <class A, one_expr<A> = 0> FX_HD SL<OpMul, A> operator*(double s, A a) { return {{}, s, a}; }
template <class A, one_expr<A> = 0> FX_HD SR<OpMul, A> operator*(A a, double s) { return {{}, a, s}; }
template <class A, one_expr<A> = 0> FX_HD SL<OpDiv, A> operator/(double s, A a) { return {{}, s, a}; }
template <class A, one_expr<A> = 0> FX_HD SR<OpDiv, A> operator/(A a, double s) { return {{}, a, s}; }
template <class A, one_expr<A> = 0> FX_HD SR<OpGt, A> operator>(A a, double s) { return {{}, a, s}; }
template <class A, one_expr<A> = 0> FX_HD Un<OpNeg, A> operator-(A a) { return {{}, a}; }

template <class A, one_expr<A> = 0> FX_HD Un<OpExp, A> exp(A a) { return {{}, a}; }
template <class A, one_expr<A> = 0> FX_HD Un<OpLog, A> log(A a) { return {{}, a}; }
template <class A, one_expr<A> = 0> FX_HD Un<OpSqrt, A> sqrt(A a) { return {{}, a}; }
template <class A, one_expr<A> = 0> FX_HD Un<OpAbs, A> abs(A a) { return {{}, a}; }
template <class A, one_expr<A> = 0> FX_HD Un<OpSquare, A> square(A a) { return {{}, a}; }
template <class A, one_expr<A> = 0> FX_HD Un<OpSigmoid, A> sigmoid(A a) { return {{}, a}; }
template <class A, one_expr<A> = 0> FX_HD Un<OpTanh, A> tanh(A a) { return {{}, a}; }
template <class A, one_expr<A> = 0> FX_HD SR<OpPow, A> pow(A a, double k) { return {{}, a, k}; }
template <class A, one_expr<A> = 0> FX_HD Tr<A> trans(A a) { return {{}, a}; }
template <class A, one_expr<A> = 0> FX_HD BCol<A> each_col(A a) { return {{}, a}; }
template <class A, one_expr<A> = 0> FX_HD BRow<A> each_row(A a) { return {{}, a}; }

template <class A, class B, both_expr<A, B> = 0> FX_HD WithAccu<A, B> with_accu(A a, B b) {
  return {{}, {{}, a, b}};
}
template <class A, one_expr<A> = 0> FX_HD Accu<A> accu(A a) { return {{}, a}; }
template <class A, one_expr<A> = 0> FX_HD Norm2<A> norm2(A a) { return {{}, a}; }
template <int D, class A, one_expr<A> = 0> FX_HD SumDim<A, D> sum(A a) { return {{}, a}; }
template <int D, class A, one_expr<A> = 0> FX_HD MaxDim<A, D> max(A a) { return {{}, a}; }

}  // namespace fx
