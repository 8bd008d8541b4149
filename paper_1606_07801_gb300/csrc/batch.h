// Host helpers of the batched step shared by the ensemble and the server.
#pragma once

#include "batch_kernels.cuh"
#include "internal.h"

namespace lbfd {

// A member of a batched launch: vx is 2 when vx_max >= 2 and Lx is even,
// else 1; the two population blocks start at value offsets off0 and off1 of
// the batch buffer; t0 is the batch clock value at which its t is 0.
BatchMember make_batch_member(const int64_t dims[3], double tau, double rho_mean, uint64_t seed, uint32_t lattice_id,
                              int64_t off0, int64_t off1, uint64_t t0, int vx_max);

// Assigns consecutive tiles of passes x 256 items to members[0..n) in order
// (tile0 and tile_start[m]); returns the number of tiles.
int64_t batch_assign_tiles(BatchMember *members, int n, int passes, int64_t *tile_start);

}  // namespace lbfd
