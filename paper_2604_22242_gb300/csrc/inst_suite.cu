// Build-time instantiation of the Sec. 4 expression suite.
#include "fx/defs.cuh"

namespace fx {
namespace defs {
FX_REGISTER(Expr1)
FX_REGISTER(Expr2)
FX_REGISTER(Expr3)
FX_REGISTER(Relu)
FX_REGISTER(SigmoidExpr)
FX_REGISTER(Swish)
FX_REGISTER(Gelu)
FX_REGISTER(SumSchur)
}  // namespace defs
}  // namespace fx
