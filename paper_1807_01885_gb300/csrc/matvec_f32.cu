// Register-FFT passes of u = K p in float (see matvec_reg.cuh).
#include "matvec_reg.cuh"

namespace bem {
template void reg_pass<float>(const bem_kernel_s*, int, const float*, float*, cudaStream_t, const int*);
template void reg_twiddles<float>(const bem_kernel_s*, cudaStream_t);
template void reg_prepare<float>(const bem_kernel_s*);
}  // namespace bem
