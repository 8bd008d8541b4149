// Batched step kernels instantiated for one lattice (own translation unit so
// that the lattices compile in parallel).
#include "batch_kernels.cuh"

namespace lbfd {

cudaError_t launch_batch_step_d3q19(int precision, void *base, const BatchStep *steps, const int64_t *tile_start,
                                 int nmembers, int64_t ntiles, int passes, int occ, int walk, int vx_max,
                                 int noise_mode, int noise_dist, int grid, cudaStream_t stream) {
  return dispatch_storage(precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return batch_step_t<kD3Q19, S>(base, steps, tile_start, nmembers, ntiles, passes, occ, walk, vx_max, noise_mode,
                                  noise_dist, grid, stream);
  });
}

cudaError_t launch_batch_param_d3q19(int precision, void *base, const BatchParams *groups, int ngroups,
                                 const BatchStep *steps, int passes, int occ, int vx_max, int noise_mode,
                                 int noise_dist, cudaStream_t stream) {
  return dispatch_storage(precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return batch_param_t<kD3Q19, S>(base, groups, ngroups, steps, passes, occ, vx_max, noise_mode, noise_dist, stream);
  });
}

int batch_blocks_per_sm_d3q19(int precision, int occ, int vx_max, int walk, int noise_mode, int noise_dist) {
  int nb = 1;
  dispatch_storage(precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    nb = batch_blocks_per_sm<kD3Q19, S>(occ, vx_max, walk, noise_mode, noise_dist);
    return cudaSuccess;
  });
  return nb;
}

}  // namespace lbfd
