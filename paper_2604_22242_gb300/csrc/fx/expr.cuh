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
  template <class C> static FX_D C f(C a, C b) { return a > b ? C(1) : C(0); }
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

template <class Op, class L, class R> struct Bin : ExprBase {
  L l;
  R r;
  template <class Ctx> FX_D typename Ctx::CT ev(const Ctx& c) const {
    return Op::f(l.ev(c), r.ev(c));
  }
  template <class Ctx> FX_D auto fwd(const Ctx& c) const {
    const auto a = l.fwd(c);
    const auto b = r.fwd(c);
    return Tape<typename Ctx::CT, decltype(a), decltype(b)>{Op::f(a.v, b.v), a, b};
  }
  template <class CT, class Tp, class G> FX_D void rev(const Tp& t, CT adj, G& g) const {
    CT da, db;
    Op::d(t.a.v, t.b.v, da, db);
    l.rev(t.a, CT(adj * da), g);
    r.rev(t.b, CT(adj * db), g);
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
    e.rev(t.a, CT(adj * Op::d(t.a.v, t.v)), g);
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
    CT da, db;
    Op::d(CT(s), t.a.v, da, db);
    e.rev(t.a, CT(adj * db), g);
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
    CT da, db;
    Op::d(t.a.v, CT(s), da, db);
    e.rev(t.a, CT(adj * da), g);
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
