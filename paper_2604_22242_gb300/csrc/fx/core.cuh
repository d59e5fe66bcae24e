// core.cuh - element types, vector memory access and compensated sums.
//
// Storage types: float, double, __nv_bfloat16, __half. Arithmetic happens in
// the compute type: float for float/bf16/f16 storage, double for double
// storage. Conversions to a narrow storage type round to nearest, ties to
// even (the CUDA _rn intrinsics).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "fx.h"

#define FX_HD __host__ __device__ __forceinline__
#define FX_D __device__ __forceinline__

namespace fx {

using bf16 = __nv_bfloat16;
using f16 = __half;

template <class T> struct compute_of { using type = float; };
template <> struct compute_of<double> { using type = double; };
template <class T> using compute_t = typename compute_of<T>::type;

template <class T> struct dtype_of;
template <> struct dtype_of<float> { static constexpr fx_dtype value = FX_F32; };
template <> struct dtype_of<double> { static constexpr fx_dtype value = FX_F64; };
template <> struct dtype_of<bf16> { static constexpr fx_dtype value = FX_BF16; };
template <> struct dtype_of<f16> { static constexpr fx_dtype value = FX_F16; };

// ---------------------------------------------------------------- conversions

FX_D float widen(float x) { return x; }
FX_D double widen(double x) { return x; }
FX_D float widen(bf16 x) { return __bfloat162float(x); }
FX_D float widen(f16 x) { return __half2float(x); }

template <class CT, class T> FX_D CT to_compute(T x) { return static_cast<CT>(widen(x)); }

template <class T> struct narrow_to;
template <> struct narrow_to<float> {
  static FX_D float from(float x) { return x; }
  static FX_D float from(double x) { return __double2float_rn(x); }
};
template <> struct narrow_to<double> {
  static FX_D double from(double x) { return x; }
  static FX_D double from(float x) { return x; }
};
template <> struct narrow_to<bf16> {
  static FX_D bf16 from(float x) { return __float2bfloat16_rn(x); }
  static FX_D bf16 from(double x) { return __double2bfloat16(x); }
};
template <> struct narrow_to<f16> {
  static FX_D f16 from(float x) { return __float2half_rn(x); }
  static FX_D f16 from(double x) { return __double2half(x); }
};

// ---------------------------------------------------------------- vectors
//
// Raw<T, V>: V storage elements, aligned to their total size, moved with one
// global access of V*sizeof(T) bytes (256-bit accesses for 32 bytes).

template <class T, int V> struct alignas(sizeof(T) * V) Raw {
  T v[V];
};

// Read-only streaming loads: non-coherent path, no L1 allocation.
// Vector stores stream (.cs, evict-first): an output element is written
// once, and dirty lines left in L2 are written back during the next
// kernel, slowing its reads (measured on GB300: a reduction that follows a
// 1 GB element-wise tree took 6% longer with plain stores).
template <int B> struct Mem;
template <> struct Mem<32> {
  template <class R> static FX_D void ld(R& r, const void* p) {
    uint32_t* w = reinterpret_cast<uint32_t*>(&r);
    asm("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
          "=r"(w[7])
        : "l"(p));
  }
  template <class R> static FX_D void st(void* p, const R& r) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(&r);
    asm volatile("st.global.cs.v8.u32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(w[0]),
                 "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
  }
};
template <> struct Mem<16> {
  template <class R> static FX_D void ld(R& r, const void* p) {
    uint32_t* w = reinterpret_cast<uint32_t*>(&r);
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
        : "l"(p));
  }
  template <class R> static FX_D void st(void* p, const R& r) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(&r);
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3])
                 : "memory");
  }
};
template <> struct Mem<8> {
  template <class R> static FX_D void ld(R& r, const void* p) {
    uint32_t* w = reinterpret_cast<uint32_t*>(&r);
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "l"(p));
  }
  template <class R> static FX_D void st(void* p, const R& r) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(&r);
    asm volatile("st.global.cs.v2.u32 [%0], {%1,%2};" ::"l"(p), "r"(w[0]), "r"(w[1]) : "memory");
  }
};
template <> struct Mem<4> {
  template <class R> static FX_D void ld(R& r, const void* p) {
    uint32_t* w = reinterpret_cast<uint32_t*>(&r);
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(w[0]) : "l"(p));
  }
  template <class R> static FX_D void st(void* p, const R& r) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(&r);
    asm volatile("st.global.u32 [%0], %1;" ::"l"(p), "r"(w[0]) : "memory");
  }
};
template <> struct Mem<2> {
  template <class R> static FX_D void ld(R& r, const void* p) {
    unsigned short* w = reinterpret_cast<unsigned short*>(&r);
    asm("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(w[0]) : "l"(p));
  }
  template <class R> static FX_D void st(void* p, const R& r) {
    const unsigned short* w = reinterpret_cast<const unsigned short*>(&r);
    asm volatile("st.global.u16 [%0], %1;" ::"l"(p), "h"(w[0]) : "memory");
  }
};

template <class T, int V> FX_D void vload(Raw<T, V>& r, const T* p) {
  Mem<sizeof(T) * V>::ld(r, p);
}
template <class T, int V> FX_D void vstore(T* p, const Raw<T, V>& r) {
  Mem<sizeof(T) * V>::st(p, r);
}
template <class T> FX_D T sload(const T* p) {
  Raw<T, 1> r;
  Mem<sizeof(T)>::ld(r, p);
  return r.v[0];
}
template <class T> FX_D void sstore(T* p, T x) {
  Raw<T, 1> r;
  r.v[0] = x;
  Mem<sizeof(T)>::st(p, r);
}

// ---------------------------------------------------------------- sums
//
// Compensated accumulation. A running pair (s, c) represents s + c. Adding
// x uses the branch-free TwoSum of Knuth (TAOCP vol. 2, 4.2.2): t = s + x is
// the rounded sum and e = (s - (t - z)) + (x - z), z = t - s, is its exact
// rounding error; e goes into c (Neumaier's variant of Kahan summation:
// the error is collected, not fed back). The _rn intrinsics keep the
// compiler from contracting or reassociating these operations.

FX_D float add_rn(float a, float b) { return __fadd_rn(a, b); }
FX_D float sub_rn(float a, float b) { return __fsub_rn(a, b); }
FX_D double add_rn(double a, double b) { return __dadd_rn(a, b); }
FX_D double sub_rn(double a, double b) { return __dsub_rn(a, b); }

template <class CT> struct CompSum {
  CT s, c;
  FX_D void init() { s = CT(0); c = CT(0); }
  FX_D void add(CT x) {
    CT t = add_rn(s, x);
    CT z = sub_rn(t, s);
    CT e = add_rn(sub_rn(s, sub_rn(t, z)), sub_rn(x, z));
    s = t;
    c = add_rn(c, e);
  }
  // (s, c) += (s2, c2): TwoSum of the leading parts, corrections added.
  FX_D void merge(CT s2, CT c2) {
    CT t = add_rn(s, s2);
    CT z = sub_rn(t, s);
    CT e = add_rn(sub_rn(s, sub_rn(t, z)), sub_rn(s2, z));
    s = t;
    c = add_rn(add_rn(c, c2), e);
  }
};

// Plain running sum (FP64 trees: their per-thread error already sits well
// inside the FP64 tolerance, and FP64 adds are scarce on this part).
template <class CT> struct PlainSum {
  CT s, c;
  FX_D void init() { s = CT(0); c = CT(0); }
  FX_D void add(CT x) { s = add_rn(s, x); }
  FX_D void merge(CT s2, CT c2) { s = add_rn(s, add_rn(s2, c2)); }
};

template <class CT>
using ThreadSum = typename std::conditional<std::is_same<CT, double>::value, PlainSum<CT>,
                                            CompSum<CT>>::type;

// ---------------------------------------------------------------- division
//
// n / d for a divisor fixed at launch, by a multiply-high, an add and a
// shift (Granlund and Montgomery, "Division by Invariant Integers using
// Multiplication", PLDI 1994, Sec. 4): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (mulhi(m, n) + n) >> l for
// every 32-bit n, the add done in 64 bits.
struct FastDiv {
  uint32_t d, m, l;
  static FastDiv make(uint32_t d_) {
    uint32_t l_ = 0;
    while ((uint64_t(1) << l_) < d_) ++l_;
    const uint64_t m_ = (((uint64_t(1) << l_) - d_) << 32) / d_ + 1;
    return FastDiv{d_, uint32_t(m_), l_};
  }
  FX_HD uint32_t div(uint32_t n) const {
#ifdef __CUDA_ARCH__
    const uint32_t hi = __umulhi(m, n);
#else
    const uint32_t hi = uint32_t((uint64_t(m) * n) >> 32);
#endif
    return uint32_t((uint64_t(hi) + n) >> l);
  }
};

// NaN-propagating maximum (fmax would drop a NaN operand).
FX_D float max_nan(float a, float b) { return (a > b || a != a) ? a : b; }
FX_D double max_nan(double a, double b) { return (a > b || a != a) ? a : b; }

template <class CT> FX_HD CT neg_inf() {
  return -__builtin_huge_val();
}

}  // namespace fx
