// Build-time instantiation of the Sec. 4 expression suite.
#include "fx/defs.cuh"

namespace fx {
namespace defs {
FX_REGISTER(Add7)
FX_REGISTER(Add8)
FX_REGISTER(Add9)
FX_REGISTER(Add10)
FX_REGISTER(Add11)
}  // namespace defs
}  // namespace fx
