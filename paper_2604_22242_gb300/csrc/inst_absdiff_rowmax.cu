// Build-time instantiation of one expression tree for its storage types.
#include "fx/defs.cuh"

namespace fx {
namespace defs {
FX_REGISTER(AbsdiffRowmax)
}  // namespace defs
}  // namespace fx
