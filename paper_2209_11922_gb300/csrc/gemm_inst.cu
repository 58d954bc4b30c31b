// gemm_inst.cu - instantiations of the tensor-core transform pass (tile width BN x operand route).
#include "gemm_pass.cuh"

namespace etd {

const GemmKernelInfo* find_gemm_kernel(int bn, int route) {
  static const GemmKernelInfo tab[] = {
      gemm_kernel_info<32, GR_TF32>(),    gemm_kernel_info<64, GR_TF32>(),    gemm_kernel_info<128, GR_TF32>(),
      gemm_kernel_info<256, GR_TF32>(),   gemm_kernel_info<32, GR_BF16X3>(),  gemm_kernel_info<64, GR_BF16X3>(),
      gemm_kernel_info<128, GR_BF16X3>(), gemm_kernel_info<256, GR_BF16X3>(),
  };
  for (const GemmKernelInfo& k : tab)
    if (k.bn == bn && k.route == route) return &k;
  return nullptr;
}

}  // namespace etd
