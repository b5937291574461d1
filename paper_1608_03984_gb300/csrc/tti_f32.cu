// tti_f32.cu -- instantiations of the 2.5D TTI kernel for float storage
// (FP32 arithmetic); see tti_kernel.cuh.
#include "tti_kernel.cuh"

namespace fdw {
FDW_TTI_DEFINE_STORAGE(f32, float)
}  // namespace fdw
