// acoustic_f32.cu -- instantiations of the 2.5D acoustic kernel for float
// storage (FP32 arithmetic); see acoustic_kernel.cuh.
#include "acoustic_kernel.cuh"

namespace fdw {
using StorageT = float;
FDW_AC_DEFINE_STORAGE(f32, StorageT)
}  // namespace fdw
