// defs.cuh - the expression trees compiled into the library.
//
// Each definition writes its tree with the Armadillo-style syntax of the
// paper (Sec. 2 and Sec. 4): % is the Schur product, trans() the transpose,
// accu() the sum of all elements. Scalars come from the expression object
// (fx_expr_set_scalar), s[0], s[1], ..., with the defaults listed.
#pragma once

#include <utility>

#include "entry.cuh"

namespace fx {
namespace defs {

#define FX_DEF_COMMON(NAME, FORMULA, NIN, NOUT, NSCAL, KIND, DT, DIFF, BATCH) \
  static constexpr const char* name = NAME;                                   \
  static constexpr const char* formula = FORMULA;                             \
  static constexpr int n_in = NIN, n_out = NOUT, n_scal = NSCAL;               \
  static constexpr int kind = KIND;                                           \
  static constexpr unsigned dtypes = DT;                                      \
  static constexpr bool differentiable = DIFF, batchable = BATCH;

// Z = A % B + 3.5 * exp(C) - trans(D); D is cols x rows.
struct SchurExpTrans {
  FX_DEF_COMMON("schur_exp_trans", "(- (+ (% A B) (* s0 (exp C))) (t D))", 4, 1, 1,
                FX_KIND_ELEMENTWISE, ALL_DTYPES, false, true)
  static constexpr const char* slots[] = {"A", "B", "C", "D", "Z"};
  static constexpr double defaults[] = {3.5};
  template <class T> static FX_HD auto build(const double* s) {
    auto A = in<0, T>(); auto B = in<1, T>(); auto C = in<2, T>(); auto D = in<3, T>();
    return A % B + s[0] * exp(C) - trans(D);
  }
};

// s = accu(square(A - B))
struct SqdiffAccu {
  FX_DEF_COMMON("sqdiff_accu", "(accu (square (- A B)))", 2, 1, 0, FX_KIND_FULL_REDUCE,
                ALL_DTYPES, true, true)
  static constexpr const char* slots[] = {"A", "B", "s"};
  static constexpr double defaults[] = {0.0};
  template <class T> static FX_HD auto build(const double*) {
    auto A = in<0, T>(); auto B = in<1, T>();
    return accu(square(A - B));
  }
};

// The 1024^2 workload's two results in one pass over A, B, C, D:
// Z = A % B + 3.5 * exp(C) - trans(D) and s = accu(square(A - B))
struct SchurExpTransSqdiff {
  FX_DEF_COMMON("schur_exp_trans_sqdiff",
                "(- (+ (% A B) (* s0 (exp C))) (t D)) ; (accu (square (- A B)))", 4, 2, 1,
                FX_KIND_MULTI, ALL_DTYPES, false, false)
  static constexpr const char* slots[] = {"A", "B", "C", "D", "Z", "s"};
  static constexpr double defaults[] = {3.5};
  template <class T> static FX_HD auto build(const double* s) {
    auto A = in<0, T>(); auto B = in<1, T>(); auto C = in<2, T>(); auto D = in<3, T>();
    return with_accu(A % B + s[0] * exp(C) - trans(D), square(A - B));
  }
};

// Z = X % Y + sqrt(abs(W)) / (1 + exp(-V))
struct SchurSqrtSigmoid {
  FX_DEF_COMMON("schur_sqrt_sigmoid", "(+ (% X Y) (/ (sqrt (abs W)) (+ s0 (exp (neg V)))))", 4,
                1, 1, FX_KIND_ELEMENTWISE, ALL_DTYPES, false, false)
  static constexpr const char* slots[] = {"X", "Y", "W", "V", "Z"};
  static constexpr double defaults[] = {1.0};
  template <class T> static FX_HD auto build(const double* s) {
    auto X = in<0, T>(); auto Y = in<1, T>(); auto W = in<2, T>(); auto V = in<3, T>();
    return X % Y + sqrt(abs(W)) / (s[0] + exp(-V));
  }
};

// colsum = sum(X % Y, 0): one sum per column (1 x cols)
struct SchurColsum {
  FX_DEF_COMMON("schur_colsum", "(sum (% X Y) 0)", 2, 1, 0, FX_KIND_DIM_REDUCE, ALL_DTYPES,
                false, false)
  static constexpr const char* slots[] = {"X", "Y", "colsum"};
  static constexpr double defaults[] = {0.0};
  template <class T> static FX_HD auto build(const double*) {
    auto X = in<0, T>(); auto Y = in<1, T>();
    return sum<0>(X % Y);
  }
};

// rowmax = max(abs(X - Y), 1): one maximum per row (rows x 1)
struct AbsdiffRowmax {
  FX_DEF_COMMON("absdiff_rowmax", "(max (abs (- X Y)) 1)", 2, 1, 0, FX_KIND_DIM_REDUCE,
                ALL_DTYPES, false, false)
  static constexpr const char* slots[] = {"X", "Y", "rowmax"};
  static constexpr double defaults[] = {0.0};
  template <class T> static FX_HD auto build(const double*) {
    auto X = in<0, T>(); auto Y = in<1, T>();
    return max<1>(abs(X - Y));
  }
};

// nrm = norm(X - Y, 2), read as the vectorised 2-norm sqrt(sum (X-Y)^2)
struct DiffNorm {
  FX_DEF_COMMON("diff_norm", "(norm (- X Y))", 2, 1, 0, FX_KIND_FULL_REDUCE, ALL_DTYPES, false,
                true)
  static constexpr const char* slots[] = {"X", "Y", "nrm"};
  static constexpr double defaults[] = {0.0};
  template <class T> static FX_HD auto build(const double*) {
    auto X = in<0, T>(); auto Y = in<1, T>();
    return norm2(X - Y);
  }
};

// Z = A % B + 0.5 * trans(C) and s = accu(Z), C is cols x rows
struct SchurTransAccu {
  FX_DEF_COMMON("schur_trans_accu", "(+ (% A B) (* s0 (t C)))", 3, 2, 1, FX_KIND_MULTI,
                ALL_DTYPES, false, true)
  static constexpr const char* slots[] = {"A", "B", "C", "Z", "s"};
  static constexpr double defaults[] = {0.5};
  template <class T> static FX_HD auto build(const double* s) {
    auto A = in<0, T>(); auto B = in<1, T>(); auto C = in<2, T>();
    return A % B + s[0] * trans(C);
  }
};

// L = accu(square(sigmoid(X % W + b.each_col) - Y)), b is rows x 1
struct SigmoidSqloss {
  FX_DEF_COMMON("sigmoid_sqloss", "(accu (square (- (sigmoid (+ (% X W) (each_col b))) Y)))", 4,
                1, 0, FX_KIND_FULL_REDUCE, ALL_DTYPES, true, false)
  static constexpr const char* slots[] = {"X", "W", "Y", "b", "L"};
  static constexpr double defaults[] = {0.0};
  template <class T> static FX_HD auto build(const double*) {
    auto X = in<0, T>(); auto W = in<1, T>(); auto Y = in<2, T>(); auto b = in<3, T>();
    return accu(square(sigmoid(X % W + each_col(b)) - Y));
  }
};

// ---------------------------------------------------------------- Sec. 4 suite (FP32)
//
// The expressions of the paper's speed comparison. addN: Z = A1 + ... + AN
// (the add-N bandwidth sweep, N = 2..16; addsub2/addsub4 are add2/add4 on
// submatrix views, i.e. bindings with the parent's leading dimension).

template <int N, class T, std::size_t... I> FX_HD auto add_fold(std::index_sequence<I...>) {
  return (... + in<int(I), T>());
}
#define FX_ADDN(N, ...)                                                                    \
  struct Add##N {                                                                          \
    FX_DEF_COMMON("add" #N, "(+ A1 ... A" #N ")", N, 1, 0, FX_KIND_ELEMENTWISE,            \
                  dmask(FX_F32), false, false)                                             \
    static constexpr const char* slots[] = {__VA_ARGS__, "Z"};                             \
    static constexpr double defaults[] = {0.0};                                            \
    template <class T> static FX_HD auto build(const double*) {                            \
      return add_fold<N, T>(std::make_index_sequence<N>{});                                 \
    }                                                                                      \
  };
FX_ADDN(2, "A1", "A2")
FX_ADDN(3, "A1", "A2", "A3")
FX_ADDN(4, "A1", "A2", "A3", "A4")
FX_ADDN(5, "A1", "A2", "A3", "A4", "A5")
FX_ADDN(6, "A1", "A2", "A3", "A4", "A5", "A6")
FX_ADDN(7, "A1", "A2", "A3", "A4", "A5", "A6", "A7")
FX_ADDN(8, "A1", "A2", "A3", "A4", "A5", "A6", "A7", "A8")
FX_ADDN(9, "A1", "A2", "A3", "A4", "A5", "A6", "A7", "A8", "A9")
FX_ADDN(10, "A1", "A2", "A3", "A4", "A5", "A6", "A7", "A8", "A9", "A10")
FX_ADDN(11, "A1", "A2", "A3", "A4", "A5", "A6", "A7", "A8", "A9", "A10", "A11")
FX_ADDN(12, "A1", "A2", "A3", "A4", "A5", "A6", "A7", "A8", "A9", "A10", "A11", "A12")
FX_ADDN(13, "A1", "A2", "A3", "A4", "A5", "A6", "A7", "A8", "A9", "A10", "A11", "A12", "A13")
FX_ADDN(14, "A1", "A2", "A3", "A4", "A5", "A6", "A7", "A8", "A9", "A10", "A11", "A12", "A13",
        "A14")
FX_ADDN(15, "A1", "A2", "A3", "A4", "A5", "A6", "A7", "A8", "A9", "A10", "A11", "A12", "A13",
        "A14", "A15")
FX_ADDN(16, "A1", "A2", "A3", "A4", "A5", "A6", "A7", "A8", "A9", "A10", "A11", "A12", "A13",
        "A14", "A15", "A16")
#undef FX_ADDN

// expr1: Z = 2*(X.t() + Y) + 2*(X + Y.t()), X and Y square
struct Expr1 {
  FX_DEF_COMMON("expr1", "(+ (* s0 (+ (t X) Y)) (* s0 (+ X (t Y))))", 2, 1, 1,
                FX_KIND_ELEMENTWISE, ALL_DTYPES, false, false)
  static constexpr const char* slots[] = {"X", "Y", "Z"};
  static constexpr double defaults[] = {2.0};
  template <class T> static FX_HD auto build(const double* s) {
    auto X = in<0, T>(); auto Y = in<1, T>();
    return s[0] * (trans(X) + Y) + s[0] * (X + trans(Y));
  }
};

// expr2: Z = a*A + (B + C).t() + log(pow(D, 2)); B and C are cols x rows
struct Expr2 {
  FX_DEF_COMMON("expr2", "(+ (+ (* s0 A) (t (+ B C))) (log (pow D s1)))", 4, 1, 2,
                FX_KIND_ELEMENTWISE, dmask(FX_F32), false, false)
  static constexpr const char* slots[] = {"A", "B", "C", "D", "Z"};
  static constexpr double defaults[] = {0.75, 2.0};
  template <class T> static FX_HD auto build(const double* s) {
    auto A = in<0, T>(); auto B = in<1, T>(); auto C = in<2, T>(); auto D = in<3, T>();
    return s[0] * A + trans(B + C) + log(pow(D, s[1]));
  }
};

// relu: Z = X % (X > 0)
struct Relu {
  FX_DEF_COMMON("relu", "(% X (gt X s0))", 1, 1, 1, FX_KIND_ELEMENTWISE, dmask(FX_F32), false,
                false)
  static constexpr const char* slots[] = {"X", "Z"};
  static constexpr double defaults[] = {0.0};
  template <class T> static FX_HD auto build(const double* s) {
    auto X = in<0, T>();
    return X % (X > s[0]);
  }
};

// sigmoid: Z = 1 / (1 + exp(-X)), written out as in the paper's listing of expressions
struct SigmoidExpr {
  FX_DEF_COMMON("sigmoid", "(/ s0 (+ s0 (exp (neg X))))", 1, 1, 1, FX_KIND_ELEMENTWISE,
                dmask(FX_F32), false, false)
  static constexpr const char* slots[] = {"X", "Z"};
  static constexpr double defaults[] = {1.0};
  template <class T> static FX_HD auto build(const double* s) {
    auto X = in<0, T>();
    return s[0] / (s[0] + exp(-X));
  }
};

// swish: Z = X / (1 + exp(-beta * X))
struct Swish {
  FX_DEF_COMMON("swish", "(/ X (+ 1 (exp (neg (* s0 X)))))", 1, 1, 1, FX_KIND_ELEMENTWISE,
                dmask(FX_F32), false, false)
  static constexpr const char* slots[] = {"X", "Z"};
  static constexpr double defaults[] = {1.0};
  template <class T> static FX_HD auto build(const double* s) {
    auto X = in<0, T>();
    return X / (1.0 + exp(-(s[0] * X)));
  }
};

// gelu: Z = (X / 2) % (1 + tanh(sqrt(2/pi) * (X + alpha * pow(X, 3))))
struct Gelu {
  FX_DEF_COMMON("gelu", "(% (/ X 2) (+ 1 (tanh (* s0 (+ X (* s1 (pow X 3)))))))", 1, 1, 2,
                FX_KIND_ELEMENTWISE, dmask(FX_F32), false, false)
  static constexpr const char* slots[] = {"X", "Z"};
  static constexpr double defaults[] = {0.7978845608028654, 0.044715};
  template <class T> static FX_HD auto build(const double* s) {
    auto X = in<0, T>();
    return (X / 2.0) % (1.0 + tanh(s[0] * (X + s[1] * pow(X, 3.0))));
  }
};

// expr3 (Sec. 4): Z = 1 / (X % conv_to<fmat>(Y) + log(log(X + 2) % W)),
// Y stored in FP64: a float tree reads a double leaf as its FP32 rounding.
struct Expr3 {
  FX_DEF_COMMON("expr3", "(/ 1 (+ (% X (f32 Y)) (log (% (log (+ X 2)) W))))", 3, 1, 0,
                FX_KIND_ELEMENTWISE, dmask(FX_F32), false, false)
  static constexpr const char* slots[] = {"X", "Y", "W", "Z"};
  static constexpr double defaults[] = {0.0};
  template <class T> static FX_HD auto build(const double*) {
    auto X = in<0, T>(); auto Y = in<1, double>(); auto W = in<2, T>();
    return 1.0 / (X % Y + log(log(X + 2.0) % W));
  }
};

// (A + B) % (C + D): diagsum when bound to the diagonal views X.diag(-1),
// X.diag(1), Y.diag(-1), Y.diag(1) (1 x n leaves with ld = parent ld + 1)
struct SumSchur {
  FX_DEF_COMMON("sum_schur", "(% (+ A B) (+ C D))", 4, 1, 0, FX_KIND_ELEMENTWISE,
                dmask(FX_F32), false, false)
  static constexpr const char* slots[] = {"A", "B", "C", "D", "Z"};
  static constexpr double defaults[] = {0.0};
  template <class T> static FX_HD auto build(const double*) {
    auto A = in<0, T>(); auto B = in<1, T>(); auto C = in<2, T>(); auto D = in<3, T>();
    return (A + B) % (C + D);
  }
};

// Fig. 1: Z = 2 X Y^T (a matrix product: a fusion boundary; the scalar
// becomes the GEMM's alpha)
struct GemmScale {
  FX_DEF_COMMON("gemm_scale", "(* s0 (* X (t Y)))", 2, 1, 1, FX_KIND_ELEMENTWISE, ALL_DTYPES,
                false, false)
  static constexpr const char* slots[] = {"X", "Y", "Z"};
  static constexpr double defaults[] = {2.0};
  template <class T> static FX_HD auto build(const double* s) {
    auto X = in<0, T>(); auto Y = in<1, T>();
    return s[0] * (X * trans(Y));
  }
};

// A product with an element-wise remainder, Z = sigmoid(s0 * (X * Y) + W):
// for BF16/FP16 one tensor-core kernel evaluates the remainder from the
// accumulator; otherwise the GEMM, then one fused pass
struct GemmEpilogue {
  FX_DEF_COMMON("gemm_epilogue", "(sigmoid (+ (* s0 (* X Y)) W))", 3, 1, 1, FX_KIND_ELEMENTWISE,
                ALL_DTYPES, false, false)
  static constexpr const char* slots[] = {"X", "Y", "W", "Z"};
  static constexpr double defaults[] = {0.5};
  template <class T> static FX_HD auto build(const double* s) {
    auto X = in<0, T>(); auto Y = in<1, T>(); auto W = in<2, T>();
    return sigmoid(s[0] * (X * Y) + W);
  }
};

// Sec. 4 chain: Z = A * B * C * D (left to right, three products)
struct Chain {
  FX_DEF_COMMON("chain", "(* (* (* A B) C) D)", 4, 1, 0, FX_KIND_ELEMENTWISE, dmask(FX_F32),
                false, false)
  static constexpr const char* slots[] = {"A", "B", "C", "D", "Z"};
  static constexpr double defaults[] = {0.0};
  template <class T> static FX_HD auto build(const double*) {
    auto A = in<0, T>(); auto B = in<1, T>(); auto C = in<2, T>(); auto D = in<3, T>();
    return A * B * C * D;
  }
};

}  // namespace defs
}  // namespace fx
