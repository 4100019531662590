// Instantiations of the multi-instance sweep kernel used by the serving loop.
#include "did_sweep_kernel.cuh"

namespace did {
namespace sweep_impl {

const void* serve_func(bool bf16) {
  return bf16 ? reinterpret_cast<const void*>(&sweep_multi_kernel<kServeNr, true>)
              : reinterpret_cast<const void*>(&sweep_multi_kernel<kServeNr, false>);
}

}  // namespace sweep_impl
}  // namespace did
