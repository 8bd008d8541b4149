// Slab decomposition of one lattice over several processes (one GPU each):
// the host-side geometry.  No device work here.
//
// The update of eq. LB (paper Sec. II) reads only nearest neighbours, so a
// lattice cut into slabs along its slowest axis (y for D2Q9, z for D3Q19)
// evolves exactly as the whole lattice if, before every step, each slab
// holds one plane beyond each of its faces with the populations that cross
// that face.  In the pull scheme a site of the first owned plane pulls
// g_i(x - v_i); for v_slow = +1 that is the plane below the slab (the lower
// neighbour's last plane), for v_slow = -1 at the last owned plane it is the
// plane above (the upper neighbour's first plane).  So per step and face only
// the Q_cross populations with v_slow pointing into the slab move: 3 for
// D2Q9, 5 for D3Q19, one plane each.  The noise of a site is keyed by its
// global site index, so the split run draws the same variates as the whole
// one and the results agree bit for bit.
//
// A slab handle (lbfd_options.slab_global > 0) stores count + 2 planes: the
// low halo plane, the owned planes 1..count, the high halo plane.
#include <cstdint>

#include "internal.h"
#include "lbfd.h"

using namespace lbfd;

namespace {

// The slowest axis of a lattice (0 x, 1 y, 2 z) and its velocity component.
int slow_axis(int lattice) { return lattice == LBFD_D3Q19 ? 2 : (lattice == LBFD_D2Q9 ? 1 : 0); }

template <int LAT>
int cross_t(int dir, int32_t *pops) {
  using L = Lattice<LAT>;
  const int ax = slow_axis(LAT);
  int n = 0;
  for (int i = 0; i < L::Q; ++i)
    if (L::v(i, ax) == dir) {
      if (pops) pops[n] = i;
      ++n;
    }
  return n;
}

}  // namespace

extern "C" {

int lbfd_slab_bounds(int64_t global_planes, int32_t nranks, int32_t rank, int64_t *first, int64_t *count) {
  if (global_planes < 1 || nranks < 1 || rank < 0 || rank >= nranks || !first || !count)
    return set_last_error(LBFD_EINVAL, "lbfd_slab_bounds: bad argument");
  if (global_planes < nranks)
    return set_last_error(LBFD_EINVAL, "lbfd_slab_bounds: fewer planes than ranks");
  // balanced: the first (global_planes mod nranks) ranks hold one plane more
  const int64_t base = global_planes / nranks, extra = global_planes % nranks;
  *count = base + (rank < extra ? 1 : 0);
  *first = int64_t(rank) * base + (rank < extra ? rank : extra);
  return LBFD_OK;
}

int lbfd_slab_cross(int32_t lattice, int32_t dir, int32_t *pops, int32_t *n_pops) {
  if ((dir != 1 && dir != -1) || !n_pops) return set_last_error(LBFD_EINVAL, "lbfd_slab_cross: bad argument");
  switch (lattice) {
    case LBFD_D2Q9: *n_pops = cross_t<kD2Q9>(dir, pops); return LBFD_OK;
    case LBFD_D3Q19: *n_pops = cross_t<kD3Q19>(dir, pops); return LBFD_OK;
  }
  return set_last_error(LBFD_EINVAL, "lbfd_slab_cross: slabs are cut along y (D2Q9) or z (D3Q19)");
}

int lbfd_slab_halo(int32_t lattice, const int64_t *dims, int32_t face, int64_t *send_off, int64_t *recv_off,
                   int32_t *n_pops, int64_t *plane_values) {
  if (!dims || (face != 0 && face != 1) || !n_pops || !plane_values)
    return set_last_error(LBFD_EINVAL, "lbfd_slab_halo: bad argument");
  if (lattice != LBFD_D2Q9 && lattice != LBFD_D3Q19)
    return set_last_error(LBFD_EINVAL, "lbfd_slab_halo: slabs are cut along y (D2Q9) or z (D3Q19)");
  const int ax = slow_axis(lattice);
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1) return set_last_error(LBFD_EINVAL, "lbfd_slab_halo: every dimension must be >= 1");
  const int64_t count = dims[ax];
  const int64_t plane = ax == 1 ? dims[0] : dims[0] * dims[1];
  const int64_t N = plane * (count + 2);  // sites of the stored slab, halo planes included
  // face 0 (low): send the v_slow = -1 populations of the first owned plane
  // (1) to the lower neighbour; receive its v_slow = +1 populations into the
  // low halo plane (0).  Face 1 (high): send the v_slow = +1 populations of
  // the last owned plane (count); receive into the high halo plane (count+1).
  const int send_dir = face == 0 ? -1 : 1, recv_dir = -send_dir;
  const int64_t send_plane = face == 0 ? 1 : count, recv_plane = face == 0 ? 0 : count + 1;
  int32_t sp[LBFD_MAX_Q], rp[LBFD_MAX_Q], ns = 0, nr = 0;
  lbfd_slab_cross(lattice, send_dir, sp, &ns);
  lbfd_slab_cross(lattice, recv_dir, rp, &nr);
  if (ns != nr) return set_last_error(LBFD_EINVAL, "lbfd_slab_halo: velocity set is not symmetric");
  // the values sent through a face by one side are the ones the other side
  // receives: the lower slab's high face sends v_slow = +1, the upper slab's
  // low face receives v_slow = +1, in the same (velocity) order
  for (int k = 0; k < ns; ++k) {
    if (send_off) send_off[k] = int64_t(sp[k]) * N + send_plane * plane;
    if (recv_off) recv_off[k] = int64_t(rp[k]) * N + recv_plane * plane;
  }
  *n_pops = ns;
  *plane_values = plane;
  return LBFD_OK;
}

}  // extern "C"
