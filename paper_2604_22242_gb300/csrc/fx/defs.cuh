// defs.cuh - the expression trees compiled into the library.
//
// Each definition writes its tree with the Armadillo-style syntax of the
// paper (Sec. 2 and Sec. 4): % is the Schur product, trans() the transpose,
// accu() the sum of all elements. Scalars come from the expression object
// (fx_expr_set_scalar), s[0], s[1], ..., with the defaults listed.
#pragma once

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

}  // namespace defs
}  // namespace fx
