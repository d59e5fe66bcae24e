// Build-time instantiation of one expression tree for its storage types.
#include "fx/defs.cuh"

namespace fx {
namespace defs {
FX_REGISTER(SchurColsum)
}  // namespace defs
}  // namespace fx
