// acoustic_bf16.cu -- instantiations of the 2.5D acoustic kernel for __nv_bfloat16
// storage (FP32 arithmetic); see acoustic_kernel.cuh.
#include "acoustic_kernel.cuh"

namespace fdw {
using StorageT = __nv_bfloat16;
FDW_AC_DEFINE_STORAGE(bf16, StorageT)
}  // namespace fdw
