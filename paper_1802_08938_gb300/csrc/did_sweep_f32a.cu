// Instantiations of the sweep kernel: float32 residual, NR = 1..5.
#include "did_sweep_kernel.cuh"

namespace did {
namespace sweep_impl {

const void* sweep_func_f32a(int NR) {
  switch (NR) {
    case 1: return reinterpret_cast<const void*>(&sweep_kernel<1, false>);
    case 2: return reinterpret_cast<const void*>(&sweep_kernel<2, false>);
    case 3: return reinterpret_cast<const void*>(&sweep_kernel<3, false>);
    case 4: return reinterpret_cast<const void*>(&sweep_kernel<4, false>);
    case 5: return reinterpret_cast<const void*>(&sweep_kernel<5, false>);
  }
  return nullptr;
}

}  // namespace sweep_impl
}  // namespace did
