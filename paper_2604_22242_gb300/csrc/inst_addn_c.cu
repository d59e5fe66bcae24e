// Build-time instantiation of the Sec. 4 expression suite.
#include "fx/defs.cuh"

namespace fx {
namespace defs {
FX_REGISTER(Add12)
FX_REGISTER(Add13)
FX_REGISTER(Add14)
FX_REGISTER(Add15)
FX_REGISTER(Add16)
}  // namespace defs
}  // namespace fx
