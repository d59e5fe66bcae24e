// Build-time instantiation of the trees with matrix products (Fig. 1's
// Z = 2 X Y^T, a product with a fused element-wise remainder, Sec. 4's chain).
#include "fx/defs.cuh"

namespace fx {
namespace defs {
FX_REGISTER(GemmScale)
FX_REGISTER(GemmEpilogue)
FX_REGISTER(Chain)
}  // namespace defs
}  // namespace fx
