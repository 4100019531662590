// Instantiations of the sweep kernel: bfloat16 residual, NR = 1..5.
#include "did_sweep_kernel.cuh"

namespace did {
namespace sweep_impl {

const void* sweep_func_bf16(int NR) {
  switch (NR) {
    case 1: return reinterpret_cast<const void*>(&sweep_kernel<1, true>);
    case 2: return reinterpret_cast<const void*>(&sweep_kernel<2, true>);
    case 3: return reinterpret_cast<const void*>(&sweep_kernel<3, true>);
    case 4: return reinterpret_cast<const void*>(&sweep_kernel<4, true>);
    case 5: return reinterpret_cast<const void*>(&sweep_kernel<5, true>);
  }
  return nullptr;
}

}  // namespace sweep_impl
}  // namespace did
