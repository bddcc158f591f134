// cells.cuh - device helpers on cell keys shared by the uniform tree
// (tree.cu) and the adaptive tree (adaptive.cu): ancestor keys, the lattice
// coordinates, centre and stencil class of a cell (Sec. 4-6), and the key of
// the cell at given lattice coordinates.
#pragma once

#include "plan.h"

namespace fmm2d {

__device__ __forceinline__ uint32_t parent_key(int tiling, uint32_t key, int up_levels) {
  if (tiling == FMM2D_SEPT) {
    for (int i = 0; i < up_levels; ++i) key /= 7u;
    return key;
  }
  return key >> (2 * up_levels);
}

// Lattice coordinates, centre (original coordinates) and stencil class of the
// level-l cell `key`.
__device__ __forceinline__ void cell_geometry(const Geo &g, int l, uint32_t key, int4 *crd_out,
                                              double2 *ctr_out, uint8_t *cls_out) {
  int4 crd = make_int4(0, 0, 0, 0);
  double X, Y;    // centre in the tiling frame
  uint8_t cls = 0;
  if (g.tiling == FMM2D_QUAD) {
    int i = (int)compact_bits(key), j = (int)compact_bits(key >> 1);
    crd = make_int4(i, j, 0, 0);
    double h = ldexp(1.0, -l);
    X = (i + 0.5) * h;
    Y = (j + 0.5) * h;
    cls = (uint8_t)(key & 3u);
  } else if (g.tiling == FMM2D_SEPT) {
    int64_t a, b;
    key_to_eis(key, l, &a, &b);
    crd = make_int4((int)a, (int)b, 0, 0);
    // frame centre g_l (a + b w), w = e^{i pi/3}
    double er = (double)a + 0.5 * (double)b, ei = 0.8660254037844386 * (double)b;
    X = g.unit_re[l] * er - g.unit_im[l] * ei;
    Y = g.unit_re[l] * ei + g.unit_im[l] * er;
    cls = (uint8_t)(key % 7u);
  } else {
    int i, j, k;
    tri_key_to_coords(key, l, &i, &j, &k);
    bool up = tri_up(i, j, k, l);
    crd = make_int4(i, j, k, up ? 1 : 0);
    double o = up ? 1.0 : 2.0, rho0 = g.leaf_scale, inv = ldexp(1.0, -l);
    Y = rho0 * (3.0 * i + o) * inv - rho0;
    X = 1.7320508075688772 * rho0 * (double)(k - j) * inv;
    if (l > 0) {
      bool pup = tri_up(i >> 1, j >> 1, k >> 1, l - 1);
      cls = (uint8_t)((key & 3u) + (pup ? 0u : 4u));
    }
  }
  if (g.tiling != FMM2D_QUAD) {
    X += 0.5;
    Y += 0.5;
  }
  *crd_out = crd;
  *ctr_out = make_double2(g.x0 + g.S * X, g.y0 + g.S * Y);
  *cls_out = cls;
}

// Key of the level-l cell at lattice coordinates c, or false if none.
__device__ __forceinline__ bool cell_at(const Geo &g, int l, int4 c, uint32_t *key) {
  if (g.tiling == FMM2D_QUAD) {
    int n = 1 << l;
    if (c.x < 0 || c.y < 0 || c.x >= n || c.y >= n) return false;
    *key = morton((uint32_t)c.x, (uint32_t)c.y);
    return true;
  }
  if (g.tiling == FMM2D_SEPT) return eis_to_key(c.x, c.y, l, key);
  return tri_coords_to_key(c.x, c.y, c.z, l, key);
}

}  // namespace fmm2d
