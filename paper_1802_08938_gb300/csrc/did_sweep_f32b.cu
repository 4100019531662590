// Instantiations of the sweep kernel: float32 residual, NR = 6..10.
#include "did_sweep_kernel.cuh"

namespace did {
namespace sweep_impl {

const void* sweep_func_f32b(int NR) {
  switch (NR) {
    case 6: return reinterpret_cast<const void*>(&sweep_kernel<6, false>);
    case 7: return reinterpret_cast<const void*>(&sweep_kernel<7, false>);
    case 8: return reinterpret_cast<const void*>(&sweep_kernel<8, false>);
    case 9: return reinterpret_cast<const void*>(&sweep_kernel<9, false>);
    case 10: return reinterpret_cast<const void*>(&sweep_kernel<10, false>);
  }
  return nullptr;
}

}  // namespace sweep_impl
}  // namespace did
