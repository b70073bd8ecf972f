// FP32 instantiation of the multi-shift MG-PCG kernels (inner solves of the mixed-precision path).
#include "kernels_impl.cuh"

namespace bura {
template struct Ops<float>;
}  // namespace bura
