// tti_f16.cu -- instantiations of the 2.5D TTI kernel for __half storage
// (FP32 arithmetic); see tti_kernel.cuh.
#include "tti_kernel.cuh"

namespace fdw {
FDW_TTI_DEFINE_STORAGE(f16, __half)
}  // namespace fdw
