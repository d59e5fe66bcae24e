// Build-time instantiation of the Sec. 4 expression suite.
#include "fx/defs.cuh"

namespace fx {
namespace defs {
FX_REGISTER(Add2)
FX_REGISTER(Add3)
FX_REGISTER(Add4)
FX_REGISTER(Add5)
FX_REGISTER(Add6)
}  // namespace defs
}  // namespace fx
