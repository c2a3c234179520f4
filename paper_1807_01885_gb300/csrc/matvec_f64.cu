// Register-FFT passes of u = K p in double (see matvec_reg.cuh).
#include "matvec_reg.cuh"

namespace bem {
template void reg_pass<double>(const bem_kernel_s*, int, const double*, double*, cudaStream_t, const int*);
template void reg_twiddles<double>(const bem_kernel_s*, cudaStream_t);
template void reg_prepare<double>(const bem_kernel_s*);
}  // namespace bem
