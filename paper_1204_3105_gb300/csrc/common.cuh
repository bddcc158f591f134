// common.cuh - shared helpers of the fmm2d CUDA library: complex arithmetic,
// and the integer lattice arithmetic of the three tilings (host and device).
//
// Lattice coordinates used for neighbour stencils (all integers):
//  * quadtree (Sec. 4, Fig. 3a): cell (i, j) of level l is the square
//    [i, i+1) x [j, j+1) * 2^-l of the unit frame; key = Morton number with
//    digit xbit + 2*ybit per level.
//  * septree (Sec. 5): a level-l cell is an Eisenstein integer E = a + b w,
//    w = e^{i pi/3}; its GBT index is the base-beta expansion of E with
//    beta = 1 + 2w and digit d <-> unit w^(d-1) (0 <-> 0).  GBT addition is
//    addition of Eisenstein integers (Sec. 5.1), Neighbors(n) = n + units.
//  * triangle quadtree (Sec. 6): a level-l cell is the set of frame points
//    whose barycentric coordinates (vertical, left, right corner of the root)
//    scaled by 2^l have integer parts (I_V, I_L, I_R); I_V + I_L + I_R is
//    2^l - 1 for an upright and 2^l - 2 for an inverted triangle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define FMM_HD __host__ __device__ __forceinline__

namespace fmm2d {

// ---------------------------------------------------------------- complex
template <typename R> struct Cx { R x, y; };
template <typename R> FMM_HD Cx<R> cx(R a, R b) { return Cx<R>{a, b}; }
template <typename R> FMM_HD Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R> FMM_HD Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R> FMM_HD Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R> FMM_HD Cx<R> operator*(R s, Cx<R> a) { return {s * a.x, s * a.y}; }
// a += b * c
template <typename R> FMM_HD void cfma(Cx<R> &a, Cx<R> b, Cx<R> c) {
  a.x += b.x * c.x - b.y * c.y;
  a.y += b.x * c.y + b.y * c.x;
}

// ---------------------------------------------------------------- quadtree
FMM_HD uint32_t spread_bits(uint32_t v) {   // 16-bit -> even bit positions
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
FMM_HD uint32_t compact_bits(uint32_t v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0F0F0F0Fu;
  v = (v | (v >> 4)) & 0x00FF00FFu;
  v = (v | (v >> 8)) & 0x0000FFFFu;
  return v;
}
FMM_HD uint32_t morton(uint32_t i, uint32_t j) { return spread_bits(i) | (spread_bits(j) << 1); }

// ---------------------------------------------------------------- septree
// digit d -> unit w^(d-1) = (A, B) meaning A + B w; index 0 is the zero digit.
// (Tables packed into integer constants, 2 or 3 bits an entry, so that a
// lookup is a shift and a mask rather than an indexed local array.)
//   unit_a: 0, 1, 0, -1, -1, 0, 1      unit_b: 0, 0, 1, 1, 0, -1, -1
FMM_HD int unit_a(int d) { return (int)((9241u >> (2 * d)) & 3u) - 1; }
FMM_HD int unit_b(int d) { return (int)((421u >> (2 * d)) & 3u) - 1; }
// residue (a + 3b) mod 7 -> digit, since w = 3 (mod beta) in Z[w]/(beta) = Z/7:
//   0, 1, 3, 2, 5, 6, 4
FMM_HD int residue_digit(int r) { return (int)((1266888u >> (3 * r)) & 7u); }

FMM_HD int64_t floordiv7(int64_t v) { return v >= 0 ? v / 7 : -((-v + 6) / 7); }
FMM_HD int mod7(int64_t v) { int r = (int)(v % 7); return r < 0 ? r + 7 : r; }
FMM_HD int floordiv7_32(int v) { return v >= 0 ? v / 7 : -((-v + 6) / 7); }
FMM_HD int mod7_32(int v) { int r = v % 7; return r < 0 ? r + 7 : r; }

// Base-beta digits of a + b w; returns false if more than l digits are needed.
FMM_HD bool eis_to_key(int64_t a, int64_t b, int l, uint32_t *key) {
  uint32_t k = 0, pw = 1;
  for (int i = 0; i < l; ++i) {
    int d = residue_digit(mod7(a + 3 * b));
    int64_t a1 = a - unit_a(d), b1 = b - unit_b(d);
    // (a1 + b1 w)(3 - 2w) / 7, exact
    int64_t qa = 3 * a1 + 2 * b1, qb = b1 - 2 * a1;
    a = floordiv7(qa);
    b = floordiv7(qb);
    k += (uint32_t)d * pw;
    pw *= 7u;
  }
  *key = k;
  return a == 0 && b == 0;
}
// The same in 32-bit arithmetic, for |a|, |b| < 2^27 (every lattice
// coordinate of a tree of at most 16 levels).
FMM_HD bool eis_to_key32(int a, int b, int l, uint32_t *key) {
  uint32_t k = 0, pw = 1;
  for (int i = 0; i < l; ++i) {
    int d = residue_digit(mod7_32(a + 3 * b));
    int a1 = a - unit_a(d), b1 = b - unit_b(d);
    int qa = 3 * a1 + 2 * b1, qb = b1 - 2 * a1;
    a = floordiv7_32(qa);
    b = floordiv7_32(qb);
    k += (uint32_t)d * pw;
    pw *= 7u;
  }
  *key = k;
  return a == 0 && b == 0;
}
FMM_HD void key_to_eis(uint32_t key, int l, int64_t *a_out, int64_t *b_out) {
  uint32_t pw = 1;
  for (int i = 1; i < l; ++i) pw *= 7u;
  int64_t a = 0, b = 0;
  for (int i = 0; i < l; ++i) {
    int d = (int)((key / pw) % 7u);
    pw /= 7u;
    int64_t na = a - 2 * b + unit_a(d);   // (a + b w)(1 + 2w) + unit
    int64_t nb = 2 * a + 3 * b + unit_b(d);
    a = na;
    b = nb;
  }
  *a_out = a;
  *b_out = b;
}

// ---------------------------------------------------------------- triangle
// Children of (i, j, k): upright parent  -> type0 (2i,2j,2k) type1 (2i+1,2j,2k)
//                                          type2 (2i,2j+1,2k) type3 (2i,2j,2k+1)
//                        inverted parent -> type0 (2i+1,2j+1,2k+1) type1 (2i,2j+1,2k+1)
//                                          type2 (2i+1,2j+1,2k) type3 (2i+1,2j,2k+1)
FMM_HD void tri_child(int i, int j, int k, bool up, int t, int *ci, int *cj, int *ck) {
  if (up) {
    *ci = 2 * i + (t == 1); *cj = 2 * j + (t == 2); *ck = 2 * k + (t == 3);
  } else {
    *ci = 2 * i + (t != 1); *cj = 2 * j + (t != 3); *ck = 2 * k + (t != 2);
  }
}
FMM_HD bool tri_up(int i, int j, int k, int l) { return i + j + k == (1 << l) - 1; }
FMM_HD void tri_key_to_coords(uint32_t key, int l, int *i, int *j, int *k) {
  int a = 0, b = 0, c = 0;
  for (int m = 1; m <= l; ++m) {
    int t = (int)((key >> (2 * (l - m))) & 3u);
    bool up = tri_up(a, b, c, m - 1);
    int na, nb, nc;
    tri_child(a, b, c, up, t, &na, &nb, &nc);
    a = na; b = nb; c = nc;
  }
  *i = a; *j = b; *k = c;
}
// Inverse of tri_key_to_coords; false if (i, j, k) is not a level-l cell.
FMM_HD bool tri_coords_to_key(int i, int j, int k, int l, uint32_t *key) {
  int n = 1 << l, s = i + j + k;
  if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return false;
  if (s != n - 1 && s != n - 2) return false;
  uint32_t kk = 0;
  for (int m = 1; m <= l; ++m) {
    int sh = l - m + 1;
    int pi = i >> sh, pj = j >> sh, pk = k >> sh;
    int bi = (i >> (l - m)) & 1, bj = (j >> (l - m)) & 1, bk = (k >> (l - m)) & 1;
    bool up = tri_up(pi, pj, pk, m - 1);
    int code = bi * 4 + bj * 2 + bk, t;
    if (up) {
      t = code == 0 ? 0 : code == 4 ? 1 : code == 2 ? 2 : code == 1 ? 3 : -1;
    } else {
      t = code == 7 ? 0 : code == 3 ? 1 : code == 6 ? 2 : code == 5 ? 3 : -1;
    }
    if (t < 0) return false;
    kk = (kk << 2) | (uint32_t)t;
  }
  *key = kk;
  return true;
}

}  // namespace fmm2d
