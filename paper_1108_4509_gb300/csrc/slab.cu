// Partition of a stencil problem into z-slabs for several GPUs (host logic,
// no kernels). Every step of the trace minimization is row-parallel over the
// N grid points except the application of H, whose stencil reaches `radius`
// planes (1 for the 7-point rule, 2 for the 13-point rule) into the
// neighbouring slabs, and the N-deep sums (the Grams and the energy), which
// become one all-reduce of their m x m partials (Sec. 2.1: every O(m N) and
// O(m^2 N) step is a loop over grid points; Fig. EGFIG, Fig. ONFIG).
#include <string>

#include "../../include/trm.h"
#include "common.cuh"

extern "C" trm_status trm_slab_plan(int nx, int ny, int nz, int order,
                                    int ranks, int rank, trm_slab* out) {
  if (!out || nx < 1 || ny < 1 || nz < 1 || ranks < 1 || rank < 0 ||
      rank >= ranks || (order != 2 && order != 4)) {
    trm::set_global_error("trm_slab_plan: invalid arguments");
    return TRM_EINVAL;
  }
  const int radius = order == 2 ? 1 : 2;
  const int base = nz / ranks, extra = nz % ranks;
  // the first nz % ranks ranks own one plane more
  auto first = [&](int r) { return r * base + (r < extra ? r : extra); };
  const int z0 = first(rank), z1 = first(rank + 1);
  const int least = base;  // planes of the smallest slab
  if (ranks > 1 && least < radius) {
    trm::set_global_error("trm_slab_plan: every slab needs at least " +
                          std::to_string(radius) +
                          " planes (the stencil's reach)");
    return TRM_EINVAL;
  }
  const int64_t plane = (int64_t)nx * ny;
  out->z0 = z0;
  out->z1 = z1;
  out->halo_lo = rank > 0 ? radius : 0;
  out->halo_hi = rank + 1 < ranks ? radius : 0;
  out->row0 = plane * z0;
  out->rows = plane * (z1 - z0);
  out->ext_z0 = z0 - out->halo_lo;
  out->ext_nz = (z1 - z0) + out->halo_lo + out->halo_hi;
  out->ext_rows = plane * out->ext_nz;
  return TRM_OK;
}
