// Build-time instantiation of the two-result tree of the 1024^2 workload
// (Z and accu(square(A - B)) in one pass) for its storage types.
#include "fx/defs.cuh"

namespace fx {
namespace defs {
FX_REGISTER(SchurExpTransSqdiff)
}  // namespace defs
}  // namespace fx
