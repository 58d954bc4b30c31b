// Instantiations of the split-radix FP32 pass kernels (split_pass.cuh), one per pass kind.
#include "split_pass.cuh"

namespace etd {

template __global__ void split_kernel<OP_ENTRY>(const PassArgs<float>);
template __global__ void split_kernel<OP_EXIT>(const PassArgs<float>);
template __global__ void split_kernel<OP_REACT>(const PassArgs<float>);
template __global__ void split_kernel<OP_TRANSFORM>(const PassArgs<float>);
template __global__ void split_kernel<OP_RK1>(const PassArgs<float>);
template __global__ void split_kernel<OP_S1>(const PassArgs<float>);
template __global__ void split_kernel<OP_S2>(const PassArgs<float>);

const void* find_split_kernel(int op) {
  switch (op) {
    case OP_ENTRY: return reinterpret_cast<const void*>(&split_kernel<OP_ENTRY>);
    case OP_EXIT: return reinterpret_cast<const void*>(&split_kernel<OP_EXIT>);
    case OP_REACT: return reinterpret_cast<const void*>(&split_kernel<OP_REACT>);
    case OP_TRANSFORM: return reinterpret_cast<const void*>(&split_kernel<OP_TRANSFORM>);
    case OP_RK1: return reinterpret_cast<const void*>(&split_kernel<OP_RK1>);
    case OP_S1: return reinterpret_cast<const void*>(&split_kernel<OP_S1>);
    case OP_S2: return reinterpret_cast<const void*>(&split_kernel<OP_S2>);
    default: return nullptr;
  }
}

}  // namespace etd
