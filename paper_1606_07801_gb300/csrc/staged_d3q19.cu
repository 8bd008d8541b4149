// Staged step kernels instantiated for one lattice (its own translation unit
// so that the lattices compile in parallel).
#include "staged_kernels.cuh"

namespace lbfd {

cudaError_t launch_step_staged_d3q19(int precision, const void *src, void *dst, const StepArgs &a,
                                  const StagedRows &rows, int *status, uint32_t wait_test_bytes,
                                  cudaStream_t stream) {
  return dispatch_storage(precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return staged_t<kD3Q19, S>(src, dst, a, rows, status, wait_test_bytes, stream);
  });
}

}  // namespace lbfd
