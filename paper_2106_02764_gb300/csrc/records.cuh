// In-place updates of the skewed octant records (layout in obte_internal.h).
#pragma once

#include "obte_internal.h"

namespace obte {

// Octant records of cell c hold its source (field 0) and the wall
// temperatures through its upwind sides (fields 1..3); write them in place.
template <typename T>
__device__ __forceinline__ void rec_put_src(const GeomDev& g, int c, T v) {
  T* rec = reinterpret_cast<T*>(g.rec4);
  const int nq = g.dim == 3 ? 8 : 4;
  for (int q = 0; q < nq; ++q) rec[(size_t)g.rec_idx[(size_t)c * nq + q] * g.rec_w] = v;
}
// wall side sd (0..5: -x +x -y +y -z +z) is the upwind side of octants with
// bit sd/2 equal to sd&1 (a +x side is upwind for p_x < 0, octant bit 0 set)
template <typename T>
__device__ __forceinline__ void rec_put_wall(const GeomDev& g, int c, int sd, T v) {
  T* rec = reinterpret_cast<T*>(g.rec4);
  const int nq = g.dim == 3 ? 8 : 4;
  const int a = sd >> 1, bit = sd & 1;
  for (int q = 0; q < nq; ++q)
    if (((q >> a) & 1) == bit) rec[(size_t)g.rec_idx[(size_t)c * nq + q] * g.rec_w + 1 + a] = v;
}

}  // namespace obte
