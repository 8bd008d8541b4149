// Host helpers of the batched step shared by the ensemble and the server.
#pragma once

#include <vector>

#include "batch_kernels.cuh"
#include "internal.h"

namespace lbfd {

// A member of a batched launch: vx is 2 when vx_max >= 2 and Lx is even,
// else 1; the two population blocks start at value offsets off0 and off1 of
// the batch buffer; t0 is the batch clock value at which its t is 0.
BatchMember make_batch_member(const int64_t dims[3], double tau, double rho_mean, uint64_t seed, uint32_t lattice_id,
                              int64_t off0, int64_t off1, uint64_t t0, int vx_max);

// Groups of at most kParamMembers consecutive members with their
// t-independent arguments, for the parameter-space launches (tile order 3);
// tile0 of every member must be assigned.  Returns the number of groups.
int batch_build_params(const BatchMember *members, int n, int64_t ntiles, int noise_mode, int noise_dist,
                       std::vector<BatchParams> &groups);

// Assigns consecutive tiles of passes x 256 items to members[0..n) in order
// (tile0 and tile_start[m]); returns the number of tiles.
int64_t batch_assign_tiles(BatchMember *members, int n, int passes, int64_t *tile_start);

}  // namespace lbfd
