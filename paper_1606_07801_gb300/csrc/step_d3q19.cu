// Step kernels instantiated for one lattice (its own translation unit so
// that the lattices compile in parallel).
#include "step_kernels.cuh"

namespace lbfd {

cudaError_t launch_step_d3q19(int precision, const void *src, void *dst, const StepArgs &a, cudaStream_t stream,
                             int vec_width) {
  return dispatch_storage(precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return step_t<kD3Q19, S>(src, dst, a, stream, vec_width);
  });
}

}  // namespace lbfd
