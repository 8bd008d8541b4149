// Ensemble kernels instantiated for one lattice (own translation unit so
// that the lattices compile in parallel).
#include "ensemble_kernels.cuh"

namespace lbfd {

cudaError_t launch_ens_step_d1q3(int precision, int vx, const void *src, void *dst, const EnsMember *members,
                            const EnsTile *tiles, int ntiles, const uint64_t *t_dev, int noise_mode, int noise_dist,
                            int grid, cudaStream_t stream) {
  return dispatch_storage(precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    if (vx == 2)
      return ens_step_t<kD1Q3, S, 2>(src, dst, members, tiles, ntiles, t_dev, noise_mode, noise_dist, grid, stream);
    return ens_step_t<kD1Q3, S, 1>(src, dst, members, tiles, ntiles, t_dev, noise_mode, noise_dist, grid, stream);
  });
}

int ens_blocks_per_sm_d1q3(int precision, int vx, int noise_mode, int noise_dist) {
  int nb = 1;
  dispatch_storage(precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    nb = vx == 2 ? ens_blocks_per_sm<kD1Q3, S, 2>(noise_mode, noise_dist)
                 : ens_blocks_per_sm<kD1Q3, S, 1>(noise_mode, noise_dist);
    return cudaSuccess;
  });
  return nb;
}

}  // namespace lbfd
