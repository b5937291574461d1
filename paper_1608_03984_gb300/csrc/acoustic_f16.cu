// acoustic_f16.cu -- instantiations of the 2.5D acoustic kernel for __half
// storage (FP32 arithmetic); see acoustic_kernel.cuh.
#include "acoustic_kernel.cuh"

namespace fdw {
using StorageT = __half;
FDW_AC_DEFINE_STORAGE(f16, StorageT)
}  // namespace fdw
