// Host-side checks of index arithmetic the kernels rely on (compiled by
// tests/test_index_math.py with nvcc and run on the CPU; no GPU involved).
//  - FastDiv: the multiply-shift division that maps a flat element index to
//    its column for broadcast leaves equals integer division for every
//    divisor and numerator below 2^32.
//  - swz<ES>: the 128-byte swizzle used to address TMA boxes in shared
//    memory is a permutation of each box that keeps elements inside their
//    16-byte chunk, and 8 consecutive rows at one position fall in 8
//    different chunk slots (the conflict-free column reads of the tiles).
#include <cstdio>
#include <cstdint>
#include <random>
#include <vector>

#include "fx/tmatile.cuh"

using fx::FastDiv;

static long bad = 0;
#define CHECK(c, ...)                 \
  do {                                \
    if (!(c)) {                       \
      if (bad++ < 20) printf(__VA_ARGS__); \
    }                                 \
  } while (0)

static void fastdiv() {
  std::mt19937_64 g(12345);
  auto one = [](uint32_t d, uint32_t n) {
    const uint32_t q = FastDiv::make(d).div(n);
    CHECK(q == n / d, "FastDiv d=%u n=%u: %u != %u\n", d, n, q, n / d);
  };
  for (uint32_t d = 1; d < 20000; ++d) {
    for (int k = 0; k < 64; ++k) one(d, uint32_t(g()));
    for (uint32_t n : {0u, 1u, d - 1, d, d + 1, 2 * d - 1, 2 * d, 0xffffffffu, 0xfffffffeu}) one(d, n);
  }
  for (int k = 0; k < 400000; ++k) {
    uint32_t d = uint32_t(g() >> 32);
    if (d == 0) d = 1;
    one(d, uint32_t(g()));
    one(d, 0xffffffffu);
    one(d, d);
  }
  for (int s = 0; s < 32; ++s) {
    const uint32_t p = 1u << s;
    for (uint32_t d : {p, p + 1, p > 1 ? p - 1 : 1u})
      for (int k = 0; k < 256; ++k) one(d, uint32_t(g()));
  }
  // matrix shapes the flat kernel meets: element index i = r + c*R below 2^32
  for (uint32_t R : {4u, 8u, 12u, 1000u, 8192u, 10000u, 16384u, 65536u}) {
    const FastDiv fd = FastDiv::make(R);
    const uint64_t n = (uint64_t(1) << 32) - 1;
    for (uint64_t i = 0; i < n; i += 7919ull * R + 3) {
      const uint32_t c = fd.div(uint32_t(i));
      CHECK(uint64_t(c) * R <= i && i < uint64_t(c + 1) * R, "column of i=%llu R=%u\n",
            (unsigned long long)i, R);
    }
  }
}

template <class T> static void swizzle() {
  using G = fx::TmaGeom<T>;
  constexpr int ES = G::es;
  std::vector<int> seen(G::BOX, 0);
  for (int o = 0; o < G::TT; ++o)
    for (int i = 0; i < G::IB; ++i) {
      const int off = fx::swz<ES>(i, o);
      CHECK(off >= 0 && off + ES <= G::BOX, "swz<%d>(%d,%d) = %d out of the box\n", ES, i, o, off);
      if (off < 0 || off + ES > G::BOX) continue;
      CHECK(off % ES == 0, "swz<%d>(%d,%d) = %d misaligned\n", ES, i, o, off);
      CHECK(off / 128 == o, "swz<%d>(%d,%d) leaves row %d\n", ES, i, o, o);
      CHECK((off & 15) == ((i * ES) & 15), "swz<%d>(%d,%d) moves within its chunk\n", ES, i, o);
      for (int b = 0; b < ES; ++b) seen[off + b]++;
    }
  for (int b = 0; b < G::BOX; ++b) CHECK(seen[b] == 1, "swz<%d> byte %d covered %d times\n", ES, b, seen[b]);
  // a column read: element i of rows o0..o0+7 lands in 8 distinct 16-byte slots
  for (int o0 = 0; o0 < G::TT; o0 += 8)
    for (int i = 0; i < G::IB; ++i) {
      int slots = 0;
      for (int r = 0; r < 8; ++r) slots |= 1 << ((fx::swz<ES>(i, o0 + r) & 127) >> 4);
      CHECK(slots == 0xff, "swz<%d> column %d rows %d..+7 share chunk slots\n", ES, i, o0);
    }
}

int main() {
  fastdiv();
  swizzle<__nv_bfloat16>();
  swizzle<float>();
  swizzle<double>();
  printf("index math: %ld failures\n", bad);
  return bad != 0;
}
