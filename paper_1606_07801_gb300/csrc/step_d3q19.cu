// Step kernels instantiated for one lattice (its own translation unit so
// that the lattices compile in parallel).
#include "step_kernels.cuh"

namespace lbfd {

cudaError_t launch_step_d3q19(int precision, const void *src, void *dst, const StepArgs &a, cudaStream_t stream) {
  return precision == 1 ? step_t<kD3Q19, double>(src, dst, a, stream) : step_t<kD3Q19, float>(src, dst, a, stream);
}

}  // namespace lbfd
