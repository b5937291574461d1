// tti_bf16.cu -- instantiations of the 2.5D TTI kernel for __nv_bfloat16 storage
// (FP32 arithmetic); see tti_kernel.cuh.
#include "tti_kernel.cuh"

namespace fdw {
FDW_TTI_DEFINE_STORAGE(bf16, __nv_bfloat16)
}  // namespace fdw
