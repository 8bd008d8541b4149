// Fused step-and-sample kernels instantiated for one lattice (its own
// translation unit so that the lattices compile in parallel).
#include "staged_kernels.cuh"

namespace lbfd {

cudaError_t launch_step_sample_d2q9(int precision, const void *src, void *dst, const StepArgs &a, int n_modes,
                                   const void *phase, double *partials, int *nblocks, bool staged_ok,
                                   int *status, cudaStream_t stream) {
  return dispatch_storage(precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return step_sample_t<kD2Q9, S>(src, dst, a, n_modes, phase, partials, nblocks, staged_ok, status, stream);
  });
}

cudaError_t launch_obs_sample_d2q9(int precision, const void *src, const StepArgs &a, int n_modes,
                                   const void *phase, double *partials, int *nblocks, cudaStream_t stream) {
  return dispatch_storage(precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return obs_sample_t<kD2Q9, S>(src, a, n_modes, phase, partials, nblocks, stream);
  });
}

}  // namespace lbfd
