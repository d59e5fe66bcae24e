// gemm.cuh - matrix products inside a tree: the fusion boundary.
//
// A matrix product cannot be computed one output element at a time from one
// element of each operand, so the planner treats it as a boundary (Sec. 5:
// the fused kernel covers the element-wise part of an expression): every
// product node, innermost first, is computed by a library GEMM (cuBLAS,
// FP32/FP64 arithmetic, BF16/FP16 operands with FP32 accumulation) into a
// temporary matrix of the storage type, the product node is replaced by a
// plain leaf bound to that temporary, and the rest of the tree runs on the
// fused path as usual. Two roots need no second pass: a bare product and a
// scalar times a product (Fig. 1's Z = 2 X Y^T), whose scalar becomes the
// GEMM's alpha and whose output is written straight into Z.
//
// Product operands must be matrix leaves, plain or transposed (a transpose
// becomes the GEMM's operand op), or products themselves (the paper's
// chain Z = A * B * C * D).
#pragma once

#include <cublas_v2.h>

#include "umma.cuh"
#include "unfused.cuh"

namespace fx {

// ---------------------------------------------------------------- lifting

// Lift<E, T, S>: E with its product nodes replaced, in post-order, by plain
// leaves of storage type T at slots S, S+1, ...; count = number replaced.
template <class E, class T, int S> struct Lift {
  using type = E;
  static constexpr int count = 0;
  static FX_HD type make(const E& e) { return e; }
};
template <class Op, class L, class R, class T, int S> struct Lift<Bin<Op, L, R>, T, S> {
  using LA = Lift<L, T, S>;
  using RA = Lift<R, T, S + LA::count>;
  using type = Bin<Op, typename LA::type, typename RA::type>;
  static constexpr int count = LA::count + RA::count;
  static FX_HD type make(const Bin<Op, L, R>& e) { return {{}, LA::make(e.l), RA::make(e.r)}; }
};
template <class Op, class E, class T, int S> struct Lift<Un<Op, E>, T, S> {
  using A = Lift<E, T, S>;
  using type = Un<Op, typename A::type>;
  static constexpr int count = A::count;
  static FX_HD type make(const Un<Op, E>& e) { return {{}, A::make(e.e)}; }
};
template <class Op, class E, class T, int S> struct Lift<SL<Op, E>, T, S> {
  using A = Lift<E, T, S>;
  using type = SL<Op, typename A::type>;
  static constexpr int count = A::count;
  static FX_HD type make(const SL<Op, E>& e) { return {{}, e.s, A::make(e.e)}; }
};
template <class Op, class E, class T, int S> struct Lift<SR<Op, E>, T, S> {
  using A = Lift<E, T, S>;
  using type = SR<Op, typename A::type>;
  static constexpr int count = A::count;
  static FX_HD type make(const SR<Op, E>& e) { return {{}, A::make(e.e), e.s}; }
};
template <class L, class R, class T, int S> struct Lift<Prod<L, R>, T, S> {
  using LA = Lift<L, T, S>;
  using RA = Lift<R, T, S + LA::count>;
  static constexpr int slot = S + LA::count + RA::count;
  using type = Leaf<slot, T, MN>;
  static constexpr int count = LA::count + RA::count + 1;
  static FX_HD type make(const Prod<L, R>&) { return {}; }
};
template <class E, class T, int S> struct Lift<Accu<E>, T, S> {
  using A = Lift<E, T, S>;
  using type = Accu<typename A::type>;
  static constexpr int count = A::count;
  static FX_HD type make(const Accu<E>& e) { return {{}, A::make(e.e)}; }
};
template <class E, class T, int S> struct Lift<Norm2<E>, T, S> {
  using A = Lift<E, T, S>;
  using type = Norm2<typename A::type>;
  static constexpr int count = A::count;
  static FX_HD type make(const Norm2<E>& e) { return {{}, A::make(e.e)}; }
};
template <class E, int D, class T, int S> struct Lift<SumDim<E, D>, T, S> {
  using A = Lift<E, T, S>;
  using type = SumDim<typename A::type, D>;
  static constexpr int count = A::count;
  static FX_HD type make(const SumDim<E, D>& e) { return {{}, A::make(e.e)}; }
};
template <class E, int D, class T, int S> struct Lift<MaxDim<E, D>, T, S> {
  using A = Lift<E, T, S>;
  using type = MaxDim<typename A::type, D>;
  static constexpr int count = A::count;
  static FX_HD type make(const MaxDim<E, D>& e) { return {{}, A::make(e.e)}; }
};

template <class E> struct has_prod_any { static constexpr bool value = has_prod_v<E>; };
template <class E> struct has_prod_any<Accu<E>> { static constexpr bool value = has_prod_v<E>; };
template <class E> struct has_prod_any<Norm2<E>> { static constexpr bool value = has_prod_v<E>; };
template <class E, int D> struct has_prod_any<SumDim<E, D>> { static constexpr bool value = has_prod_v<E>; };
template <class E, int D> struct has_prod_any<MaxDim<E, D>> { static constexpr bool value = has_prod_v<E>; };

// ---------------------------------------------------------------- cuBLAS

inline fx_status blas_fail(cublasStatus_t s, const char* what) {
  return fail(FX_E_CUDA, "%s: cuBLAS status %d", what, int(s));
}

// One handle per thread and device, created on first use.
inline fx_status blas_handle(cublasHandle_t* out) {
  struct Handles {
    cublasHandle_t h[64] = {};
    ~Handles() {
      for (auto& x : h)
        if (x) cublasDestroy(x);
    }
  };
  static thread_local Handles hs;
  int dev = 0;
  FX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(FX_E_UNSUPPORTED, "device %d", dev);
  if (!hs.h[dev]) {
    const cublasStatus_t s = cublasCreate(&hs.h[dev]);
    if (s != CUBLAS_STATUS_SUCCESS) return blas_fail(s, "cublasCreate");
    cublasSetMathMode(hs.h[dev], CUBLAS_DEFAULT_MATH);  // full FP32, no TF32
  }
  *out = hs.h[dev];
  return FX_OK;
}

template <class T> struct BlasType;
template <> struct BlasType<float> {
  static constexpr cudaDataType data = CUDA_R_32F;
  static constexpr cublasComputeType_t compute = CUBLAS_COMPUTE_32F;
  using scale = float;
};
template <> struct BlasType<double> {
  static constexpr cudaDataType data = CUDA_R_64F;
  static constexpr cublasComputeType_t compute = CUBLAS_COMPUTE_64F;
  using scale = double;
};
template <> struct BlasType<bf16> {
  static constexpr cudaDataType data = CUDA_R_16BF;
  static constexpr cublasComputeType_t compute = CUBLAS_COMPUTE_32F;
  using scale = float;
};
template <> struct BlasType<f16> {
  static constexpr cudaDataType data = CUDA_R_16F;
  static constexpr cublasComputeType_t compute = CUBLAS_COMPUTE_32F;
  using scale = float;
};

// A product operand after lifting: a plain or transposed matrix leaf.
template <class O> struct Operand;
template <int K, class T, int M> struct Operand<Leaf<K, T, M>> {
  static_assert(M == MN || M == MT, "a product operand is a matrix, plain or transposed");
  static constexpr int slot = K;
  static constexpr bool trans = M == MT;
};

// C (m x n, leading dimension ldc) = alpha * op(A) * op(B) for lifted
// operand leaves LA, LB bound in b.
template <class T, class LA, class LB>
fx_status gemm_into(const Binding* b, void* c, int64_t ldc, int64_t m_expect, int64_t n_expect,
                    double alpha, cudaStream_t st) {
  using OA = Operand<LA>;
  using OB = Operand<LB>;
  const Binding& a = b[OA::slot];
  const Binding& bb = b[OB::slot];
  const int64_t m = OA::trans ? a.cols : a.rows, ka = OA::trans ? a.rows : a.cols;
  const int64_t kb = OB::trans ? bb.cols : bb.rows, n = OB::trans ? bb.rows : bb.cols;
  if (ka != kb) return fail(FX_E_SHAPE, "matrix product: inner sizes %lld and %lld differ",
                            (long long)ka, (long long)kb);
  if (m != m_expect || n != n_expect)
    return fail(FX_E_SHAPE, "matrix product is %lld x %lld, expected %lld x %lld", (long long)m,
                (long long)n, (long long)m_expect, (long long)n_expect);
  const int64_t lim = int64_t(1) << 31;
  if (m >= lim || n >= lim || ka >= lim || a.ld >= lim || bb.ld >= lim || ldc >= lim)
    return fail(FX_E_SHAPE, "matrix product too large for a 32-bit GEMM");
  if (m == 0 || n == 0) return FX_OK;
  cublasHandle_t h;
  FX_TRY(blas_handle(&h));
  cublasStatus_t s = cublasSetStream(h, st);
  if (s != CUBLAS_STATUS_SUCCESS) return blas_fail(s, "cublasSetStream");
  using BT = BlasType<T>;
  const typename BT::scale al = typename BT::scale(alpha), be = typename BT::scale(0);
  s = cublasGemmEx(h, OA::trans ? CUBLAS_OP_T : CUBLAS_OP_N, OB::trans ? CUBLAS_OP_T : CUBLAS_OP_N,
                   int(m), int(n), int(ka), &al, a.p, BT::data, int(a.ld > 0 ? a.ld : 1), bb.p,
                   BT::data, int(bb.ld > 0 ? bb.ld : 1), &be, c, BT::data, int(ldc > 0 ? ldc : 1),
                   BT::compute, CUBLAS_GEMM_DEFAULT);
  if (s != CUBLAS_STATUS_SUCCESS) return blas_fail(s, "cublasGemmEx");
  return FX_OK;
}

// Rows and columns of a lifted product operand.
template <class L> void operand_shape(const Binding* b, int64_t& r, int64_t& c) {
  using O = Operand<L>;
  const Binding& x = b[O::slot];
  r = O::trans ? x.cols : x.rows;
  c = O::trans ? x.rows : x.cols;
}

// Computes every product of E (normalised, unlifted), innermost first,
// into temporaries bound at slots S, S+1, ... of b (the order Lift uses),
// carved from `base` at running byte offset `off`. With dry set, only the
// bindings' shapes and offsets are set (to size the workspace).
template <class T, int S, class E> struct Prods {
  static fx_status run(Binding*, const E&, char*, size_t&, bool, cudaStream_t) { return FX_OK; }
};
template <class T, int S, class Op, class L, class R> struct Prods<T, S, Bin<Op, L, R>> {
  static fx_status run(Binding* b, const Bin<Op, L, R>& e, char* base, size_t& off, bool dry,
                       cudaStream_t st) {
    FX_TRY((Prods<T, S, L>::run(b, e.l, base, off, dry, st)));
    return Prods<T, S + Lift<L, T, S>::count, R>::run(b, e.r, base, off, dry, st);
  }
};
template <class T, int S, class Op, class E> struct Prods<T, S, Un<Op, E>> {
  static fx_status run(Binding* b, const Un<Op, E>& e, char* base, size_t& off, bool dry,
                       cudaStream_t st) {
    return Prods<T, S, E>::run(b, e.e, base, off, dry, st);
  }
};
template <class T, int S, class Op, class E> struct Prods<T, S, SL<Op, E>> {
  static fx_status run(Binding* b, const SL<Op, E>& e, char* base, size_t& off, bool dry,
                       cudaStream_t st) {
    return Prods<T, S, E>::run(b, e.e, base, off, dry, st);
  }
};
template <class T, int S, class Op, class E> struct Prods<T, S, SR<Op, E>> {
  static fx_status run(Binding* b, const SR<Op, E>& e, char* base, size_t& off, bool dry,
                       cudaStream_t st) {
    return Prods<T, S, E>::run(b, e.e, base, off, dry, st);
  }
};
template <class T, int S, class L, class R> struct Prods<T, S, Prod<L, R>> {
  static fx_status run(Binding* b, const Prod<L, R>& e, char* base, size_t& off, bool dry,
                       cudaStream_t st) {
    using LA = Lift<L, T, S>;
    using RA = Lift<R, T, S + LA::count>;
    FX_TRY((Prods<T, S, L>::run(b, e.l, base, off, dry, st)));
    FX_TRY((Prods<T, S + LA::count, R>::run(b, e.r, base, off, dry, st)));
    int64_t m, k1, k2, n;
    operand_shape<typename LA::type>(b, m, k1);
    operand_shape<typename RA::type>(b, k2, n);
    if (k1 != k2)
      return fail(FX_E_SHAPE, "matrix product: inner sizes %lld and %lld differ", (long long)k1,
                  (long long)k2);
    Binding& out = b[Lift<Prod<L, R>, T, S>::slot];
    out.p = base + off;
    out.rows = m;
    out.cols = n;
    out.ld = m > 0 ? m : 1;
    out.bound = true;
    off += ((size_t(m) * size_t(n) * sizeof(T)) + 255) & ~size_t(255);
    if (dry) return FX_OK;
    return gemm_into<T, typename LA::type, typename RA::type>(b, out.p, out.ld, m, n, 1.0, st);
  }
};

}  // namespace fx

namespace fx {

// Roots whose products need no second pass: a product, or a scalar times a
// product (the scalar becomes the GEMM's alpha).
template <class Root> struct ScaledProd {
  static constexpr bool value = false;
};
template <class L, class R> struct ScaledProd<Prod<L, R>> {
  static constexpr bool value = true;
  using P = Prod<L, R>;
  static double scale(const P&) { return 1.0; }
  static const P& prod(const P& p) { return p; }
};
template <class L, class R> struct ScaledProd<SL<OpMul, Prod<L, R>>> {
  static constexpr bool value = true;
  using P = Prod<L, R>;
  static double scale(const SL<OpMul, P>& e) { return e.s; }
  static const P& prod(const SL<OpMul, P>& e) { return e.e; }
};

// ---------------------------------------------------------------- tcgen05 path

// Trees the tensor-core kernel takes: BF16 or FP16 storage, one matrix
// product of two matrix leaves (plain or transposed), and an element-wise
// remainder whose other leaves are plain matrices of the storage type.
template <class T, int NIN, class Root> struct umma_ok {
  static constexpr bool value = [] {
    if constexpr (!(std::is_same<T, bf16>::value || std::is_same<T, f16>::value)) {
      return false;
    } else if constexpr (root_of<Root>::kind != FX_KIND_ELEMENTWISE || !has_prod_v<Root>) {
      return false;
    } else if constexpr (Lift<Root, T, NIN>::count != 1) {
      return false;
    } else {
      using P = typename the_prod<Root>::type;
      return prod_of_leaves<P>::value &&
             others_plain<leaves_t<typename Lift<Root, T, NIN>::type>, NIN, T>();
    }
  }();
};

// Evaluates the whole tree with umma::k_gemm_umma when the operands allow
// TMA (16-byte aligned bases and leading dimensions) and the shapes agree;
// *used is false otherwise (the caller takes the library-GEMM path, which
// also reports shape errors).
template <class T, int NIN, class Root>
fx_status run_umma(fx_expr* x, const Root& root, cudaStream_t st, bool* used) {
  *used = false;
  using LR = Lift<Root, T, NIN>;
  using Lifted = typename LR::type;
  constexpr int PS = NIN;
  using P = typename the_prod<Root>::type;
  using OA = Operand<std::decay_t<decltype(std::declval<P>().l)>>;
  using OB = Operand<std::decay_t<decltype(std::declval<P>().r)>>;
  constexpr bool AMN = !OA::trans, BMN = OB::trans;
  const Binding& a = x->b[OA::slot];
  const Binding& b = x->b[OB::slot];
  const Binding& zb = x->b[NIN];
  if (!a.bound || !b.bound || !zb.bound) return FX_OK;
  const int64_t M = OA::trans ? a.cols : a.rows, Ka = OA::trans ? a.rows : a.cols;
  const int64_t Kb = OB::trans ? b.cols : b.rows, N = OB::trans ? b.rows : b.cols;
  if (Ka != Kb || zb.rows != M || zb.cols != N || M == 0 || N == 0 || Ka == 0) return FX_OK;
  const int64_t lim = int64_t(1) << 31;
  if (M >= lim || N >= lim || Ka >= lim ||
      ((M + umma::BM - 1) / umma::BM) * ((N + umma::BN - 1) / umma::BN) >= lim)
    return FX_OK;
  Binding bt[FX_MAX_SLOTS];
  for (int k = 0; k < NIN; ++k) bt[k] = x->b[k];
  bt[PS] = Binding{nullptr, M, N, M, true};
  if (check_leaves<leaves_t<Lifted>>(bt, M, N) != FX_OK) {
    cudaGetLastError();
    return FX_OK;  // the library-GEMM path reports the shape error
  }
  CUtensorMap ma, mb;
  const bool oka = AMN ? encode_map<T>(&ma, a.p, M, Ka, a.ld, 64, 64)
                       : encode_map<T>(&ma, a.p, Ka, M, a.ld, 64, umma::BM);
  const bool okb = BMN ? encode_map<T>(&mb, b.p, N, Ka, b.ld, 64, 64)
                       : encode_map<T>(&mb, b.p, Ka, N, b.ld, 64, umma::BN);
  if (!oka || !okb) return FX_OK;
  auto kern = umma::k_gemm_umma<T, AMN, BMN, Lifted, PS>;
  const int smem = umma::NS * umma::STAGE + 1024 + int(sizeof(umma::Bars));
  FX_TRY(allow_smem(kern, smem));
  FX_TRY(x->ws_err.ensure(256, st));
  unsigned int* err = static_cast<unsigned int*>(x->ws_err.p);
  const Slots sl = make_slots(x->b, NIN);
  const int64_t ntiles = ((M + umma::BM - 1) / umma::BM) * ((N + umma::BN - 1) / umma::BN);
  const int sms = device_sms() > 0 ? device_sms() : 1;
  const unsigned grid = unsigned(ntiles < sms ? ntiles : sms);   // persistent: one CTA per SM
  *used = true;
  x->last_launches = 0;
  kern<<<grid, 192, smem, st>>>(ma, mb, LR::make(root), sl, static_cast<T*>(zb.p), zb.ld, int(M),
                                int(N), int(Ka), err);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return cuda_fail(le, "k_gemm_umma");
  x->last_launches = 1;
  return FX_OK;
}

// A tree with matrix products: products into temporaries (slots NIN ..
// NIN+P-1 of a private binding table), then the lifted tree on the fused
// path (or, for the unfused baseline, one launch per operator).
template <class T, int NIN, class Root>
fx_status run_with_prods(fx_expr* x, const Root& root, int kind, cudaStream_t st, bool unfused) {
  using LR = Lift<Root, T, NIN>;
  constexpr int P = LR::count;
  const int n_out = x->e->n_out;
  static_assert(NIN + P + 2 <= FX_MAX_SLOTS, "too many matrix products in one tree");
  using Inner = typename root_of<Root>::inner;
  const Inner& inner = inner_of(root);
  if constexpr (umma_ok<T, NIN, Root>::value) {
    // launch-shape pipeline 0: the tensor-core kernel with the remainder in
    // its epilogue; 1 and 2: the library GEMM and the fused pass
    if (!unfused && kind == FX_KIND_ELEMENTWISE && x->tune.pipe == 0) {
      bool used = false;
      FX_TRY((run_umma<T, NIN>(x, root, st, &used)));
      if (used) return FX_OK;
    }
  }
  Binding bb[FX_MAX_SLOTS];
  for (int k = 0; k < NIN; ++k) bb[k] = x->b[k];
  for (int j = 0; j < n_out; ++j) bb[NIN + P + j] = x->b[NIN + j];
  size_t off = 0;
  if constexpr (ScaledProd<Root>::value) {
    if (!unfused && kind == FX_KIND_ELEMENTWISE) {
      using SP = ScaledProd<Root>;
      using PT = typename SP::P;
      const PT& pr = SP::prod(root);
      using LA = Lift<decltype(pr.l), T, NIN>;
      using RA = Lift<decltype(pr.r), T, NIN + LA::count>;
      FX_TRY((Prods<T, NIN, std::decay_t<decltype(pr.l)>>::run(bb, pr.l, nullptr, off, true, st)));
      FX_TRY((Prods<T, NIN + LA::count, std::decay_t<decltype(pr.r)>>::run(bb, pr.r, nullptr, off,
                                                                            true, st)));
      if (off > 0) FX_TRY(x->ws_gemm.ensure(off + 256, st));
      off = 0;
      char* base = static_cast<char*>(x->ws_gemm.p);
      FX_TRY((Prods<T, NIN, std::decay_t<decltype(pr.l)>>::run(bb, pr.l, base, off, false, st)));
      FX_TRY((Prods<T, NIN + LA::count, std::decay_t<decltype(pr.r)>>::run(bb, pr.r, base, off,
                                                                            false, st)));
      const Binding& z = x->b[NIN];
      x->last_launches = 0;
      return gemm_into<T, typename LA::type, typename RA::type>(bb, z.p, z.ld, z.rows, z.cols,
                                                                 SP::scale(root), st);
    }
  }
  FX_TRY((Prods<T, NIN, Inner>::run(bb, inner, nullptr, off, true, st)));
  if (off > 0) FX_TRY(x->ws_gemm.ensure(off + 256, st));
  off = 0;
  FX_TRY((Prods<T, NIN, Inner>::run(bb, inner, static_cast<char*>(x->ws_gemm.p), off, false, st)));
  Run r = run_of(x, st);
  r.b = bb;
  r.n_in = NIN + P;
  x->last_launches = 0;
  const auto lifted = LR::make(root);
  if (unfused) return run_unfused<T>(x, lifted, kind, st, &r);
  return run_root<T>(r, lifted, kind);
}

}  // namespace fx
