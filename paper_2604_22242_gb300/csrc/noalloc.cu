// noalloc.cu - a fused reduction that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the moment they evaluate: code
// running inside a pre-planned memory budget (the whole device pool handed
// out up front), code that must not synchronise the device (cudaMalloc and
// cudaFree can), and hosts whose allocator is owned by another framework.
// For them, fx_sqdiff_accu_f32_noalloc computes s = accu(square(A - B)) with
// the same fused kernel and launch plan as fx_eval on "sqdiff_accu", but
// takes its reduction scratch (per-block partial sums and the completion
// ticket) from a fixed array compiled into the library instead of from an
// expression object's workspace. The array is a file-scope __device__
// variable: every GPU that loads the library holds its FX_NOALLOC_SCRATCH
// bytes until the process exits.
#include <mutex>

#include "fx/defs.cuh"

namespace {

constexpr int kMaxPartials = 4096;  // partial sums, one per block of the grid
constexpr size_t kTicketOffset = size_t(kMaxPartials) * sizeof(double2);
constexpr size_t kScratchBytes = kTicketOffset + 256;
static_assert(kScratchBytes == FX_NOALLOC_SCRATCH, "keep fx.h in step");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the array, looked up once per device (the set-up done
// by the first call on that device, with the device current). In host code
// g_noalloc_scratch is only a host-side stand-in for the symbol, never a
// device address, so the kernel is always given the looked-up pointer. The
// cached address belongs to the device's current context: after
// cudaDeviceReset the entry point is not to be used again in the process.
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

fx_status scratch_of_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fx::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return fx::fail(FX_E_UNSUPPORTED, "device %d is beyond the %d devices this entry point serves",
                    dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fx::cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FX_OK;
}

template <bool TILED, class E, class Epi, class K>
fx_status launch_into_scratch(K kern, int block, int64_t work, const E& e, const fx::Slots& sl,
                              int64_t a0, int64_t a1, const Epi& epi, float* s, cudaStream_t st) {
  const int grid = fx::grid_for(kern, block, work > 0 ? work : 1, fx::Tune{});
  if (grid > kMaxPartials)
    return fx::fail(FX_E_UNSUPPORTED,
                    "this launch needs %d partial sums; the static scratch holds %d", grid,
                    kMaxPartials);
  void* base = nullptr;
  FX_TRY(scratch_of_current_device(&base));
  fx::RedArgs red{};
  red.part = static_cast<double2*>(base);
  red.ticket = reinterpret_cast<unsigned int*>(static_cast<char*>(base) + kTicketOffset);
  red.out = s;
  // the ticket must start at zero; the array keeps whatever the last call left
  FX_CUDA(cudaMemsetAsync(red.ticket, 0, sizeof(unsigned int), st));
  if constexpr (TILED) {
    kern<<<grid, block, 0, st>>>(e, sl, a0, a1, epi, red);
  } else {
    kern<<<grid, block, 0, st>>>(e, sl, a0, epi, red, fx::FastDiv{});
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return fx::cuda_fail(err, "no-alloc reduction launch");
  return FX_OK;
}

}  // namespace

extern "C" fx_status fx_sqdiff_accu_f32_noalloc(const float* A, const float* B, int64_t rows,
                                                int64_t cols, int64_t ld, float* s,
                                                void* stream) {
  using namespace fx;
  if (!s) return fail(FX_E_ARG, "null output");
  if (rows < 0 || cols < 0) return fail(FX_E_SHAPE, "negative shape");
  if (ld < (rows > 1 ? rows : 1)) return fail(FX_E_ARG, "ld %lld < rows %lld", (long long)ld, (long long)rows);
  // extents whose products overflow 64-bit indices are refused before any
  // arithmetic on them
  if (cols > 0 && (rows > INT64_MAX / cols || ld > (INT64_MAX - rows) / cols))
    return fail(FX_E_SHAPE, "%lld x %lld (ld %lld) overflows 64-bit element indices",
                (long long)rows, (long long)cols, (long long)ld);
  if (rows * cols > 0 && (!A || !B)) return fail(FX_E_ARG, "null input for a non-empty matrix");
  if (!aligned(A, 4) || !aligned(B, 4) || !aligned(s, 4))
    return fail(FX_E_ALIGN, "pointers must be aligned to 4 bytes");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const auto root = normalize(defs::SqdiffAccu::build<float>(nullptr));
  using Root = std::decay_t<decltype(root)>;
  using E = typename root_of<Root>::inner;
  const E& e = inner_of(root);
  constexpr int V = vec_width<E, 16>();
  Slots sl{};
  sl.s[0] = SlotView{A, ld, 1};
  sl.s[1] = SlotView{B, ld, 1};
  const int64_t R = rows, C = cols;
  const bool dense = ld == R || C <= 1;
  const bool vec16 = aligned(A, 16) && aligned(B, 16);
  // the same family and vector-width choice as fx_eval on "sqdiff_accu"
  if (dense) {
    const int block = 256, U = 4;
    if (vec16) {
      auto kern = k_flat<E, EpiSum<float, V, false>, V, U>;
      const int64_t work = (R * C / V + int64_t(block) * U - 1) / (int64_t(block) * U);
      return launch_into_scratch<false>(kern, block, work, e, sl, R * C, 0,
                                        EpiSum<float, V, false>{R}, s, st);
    }
    auto kern = k_flat<E, EpiSum<float, 1, false>, 1, U>;
    const int64_t work = (R * C + int64_t(block) * U - 1) / (int64_t(block) * U);
    return launch_into_scratch<false>(kern, block, work, e, sl, R * C, 0,
                                      EpiSum<float, 1, false>{R}, s, st);
  }
  if (vec16 && ld % V == 0) {
    using TC_ = TileCfg<E, V>;
    auto kern = k_tile<E, EpiSum<float, V, false>, V, TC_::TR, TC_::TC, TC_::NT>;
    const int64_t work = ((R + TC_::TR - 1) / TC_::TR) * ((C + TC_::TC - 1) / TC_::TC);
    return launch_into_scratch<true>(kern, TC_::NT, work, e, sl, R, C,
                                     EpiSum<float, V, false>{0}, s, st);
  }
  using TC1 = TileCfg<E, 1>;
  auto kern = k_tile<E, EpiSum<float, 1, false>, 1, TC1::TR, TC1::TC, TC1::NT>;
  const int64_t work = ((R + TC1::TR - 1) / TC1::TR) * ((C + TC1::TC - 1) / TC1::TC);
  return launch_into_scratch<true>(kern, TC1::NT, work, e, sl, R, C,
                                   EpiSum<float, 1, false>{0}, s, st);
}
