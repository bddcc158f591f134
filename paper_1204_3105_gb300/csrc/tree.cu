// tree.cu - occupied cells of every level, their lattice coordinates and
// centres, per-leaf point ranges, and the Near / M2L lists (Sec. 4-6).
//
// Cells of all levels live in one array ordered by (level, key): a key ->
// slot map of sum_l b^l entries is filled from an occupancy flag array
// (every occupied leaf marks all its ancestors, Parent(n) = n div b) and one
// exclusive scan.  Lists come from per-class integer stencils of lattice
// offsets (the offsets of Neighbors and of NeighborsE4 = Children[Parent(n)
// u Neighbors(Parent(n))] minus {n} u Neighbors(n), eq. 3), looked up in the
// map; only cells holding sources enter a list.
#include "cells.cuh"
#include "plan.h"

namespace fmm2d {

namespace {

// The first point (in sorted order) of every occupied cell of every level
// marks that cell: the point whose leaf key starts a run marks its leaf and
// then each ancestor up to the first one it shares with the point before it,
// so every flag is written once (no write contention on the top levels).
__global__ void k_mark(Geo g, const uint32_t *__restrict__ key, int64_t n, int *__restrict__ occ,
                       int *__restrict__ hsrc) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t k = key[i];
  const bool first = i == 0;
  uint32_t kp = first ? 0u : key[i - 1];
  if (!first && kp == k) return;
  for (int l = g.L; l >= 0; --l) {
    occ[g.map_off[l] + k] = 1;
    if (hsrc) hsrc[g.map_off[l] + k] = 1;
    if (l == 0) break;
    k = parent_key(g.tiling, k, 1);
    if (!first) {
      kp = parent_key(g.tiling, kp, 1);
      if (kp == k) break;   // this ancestor and all above it are marked by earlier points
    }
  }
}

__device__ __forceinline__ int level_of_map(const Geo &g, int64_t m) {
  int l = 0;
  while (l < g.L && m >= g.map_off[l + 1]) ++l;
  return l;
}

// The triangle tiling's position map: level l holds 2 x 4^l entries, index
// (i 2^l + j) x 2 + up for the cell at lattice position (i, j, k) (k is then
// 2^l - 1 - i - j for an up cell, 2^l - 2 - i - j for a down one, Sec. 6),
// each the cell's slot when it holds sources, else -1.  Levels 0 .. l-1
// take 2 (4^l - 1) / 3 entries.
__device__ __forceinline__ int64_t tri_pmap_index(int l, int i, int j, int up) {
  return 2 * ((((int64_t)1) << (2 * l)) - 1) / 3 + ((((int64_t)i << l) | j) << 1) + up;
}

// The slot of the triangle cell with sources at level-l position q, or -1.
__device__ __forceinline__ int tri_pmap_lookup(const int *__restrict__ pmap, int l, int4 q) {
  const int n = 1 << l, sum = q.x + q.y + q.z;
  if (q.x < 0 || q.y < 0 || q.z < 0 || q.x >= n || q.y >= n || q.z >= n) return -1;
  if (sum != n - 1 && sum != n - 2) return -1;
  return pmap[tri_pmap_index(l, q.x, q.y, sum == n - 1 ? 1 : 0)];
}

__global__ void k_compact(Geo g, const int *__restrict__ occ, const int *__restrict__ scan,
                          const int *__restrict__ hsrc, int64_t map_size, int *__restrict__ map,
                          uint32_t *__restrict__ cell_key, int4 *__restrict__ cell_crd,
                          double2 *__restrict__ cell_ctr, uint8_t *__restrict__ cell_cls,
                          uint8_t *__restrict__ cell_hsrc, int *__restrict__ src_start,
                          int *__restrict__ src_end, int *__restrict__ tgt_start,
                          int *__restrict__ tgt_end, int64_t *__restrict__ lev_first,
                          int *__restrict__ pmap) {
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= map_size) return;
  const int l = level_of_map(g, m);
  if (lev_first) {   // first slot of every level, and the total
    if (m == g.map_off[l]) lev_first[l] = scan[m];
    if (m == map_size - 1) lev_first[g.L + 1] = (int64_t)scan[m] + occ[m];
  }
  const uint32_t key = (uint32_t)(m - g.map_off[l]);
  if (pmap) {   // triangle tiling: every key's position entry (keys and positions correspond one to one)
    int i, j, k;
    tri_key_to_coords(key, l, &i, &j, &k);
    pmap[tri_pmap_index(l, i, j, tri_up(i, j, k, l) ? 1 : 0)] = (occ[m] && hsrc[m]) ? scan[m] : -1;
  }
  if (!occ[m]) {
    map[m] = -1;
    return;
  }
  const int slot = scan[m];
  map[m] = slot;
  cell_key[slot] = key;
  src_start[slot] = src_end[slot] = 0;   // leaf ranges are filled in later
  if (tgt_start) tgt_start[slot] = tgt_end[slot] = 0;
  cell_hsrc[slot] = (uint8_t)(hsrc[m] != 0);
  int4 crd;
  double2 ctr;
  uint8_t cls;
  cell_geometry(g, l, key, &crd, &ctr, &cls);
  cell_crd[slot] = crd;
  cell_ctr[slot] = ctr;
  cell_cls[slot] = cls;
}

// Per sorted point: the leaf's [start, end) at run boundaries, and the point
// relative to its leaf centre.
template <typename TI, typename TO>
__global__ void k_rel(Geo g, const TI *__restrict__ xy, const uint32_t *__restrict__ perm,
                      const uint32_t *__restrict__ key, int64_t n, const int *__restrict__ map,
                      const double2 *__restrict__ ctr, TO *__restrict__ out, int stride,
                      int *__restrict__ start, int *__restrict__ end, float2 *__restrict__ lo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t o = perm[i];
  const uint32_t k = key[i];
  int slot = map[g.map_off[g.L] + k];
  if (i == 0 || key[i - 1] != k) start[slot] = (int)i;
  if (i == n - 1 || key[i + 1] != k) end[slot] = (int)(i + 1);
  double2 c = ctr[slot];
  double x = (double)xy[2 * (int64_t)o], y = (double)xy[2 * (int64_t)o + 1];
  TO *dst = out + i * stride;
  const double dx = x - c.x, dy = y - c.y;
  dst[0] = (TO)dx;
  dst[1] = (TO)dy;
  for (int q = 2; q < stride; ++q) dst[q] = (TO)0;
  if (lo) lo[i] = make_float2((float)(dx - (double)(float)dx), (float)(dy - (double)(float)dy));
}

// One warp per cell: lane e looks up stencil entry e (and e + 32), and a
// ballot compacts the hits in stencil order, so the list is the same as a
// sequential scan of the stencil would give.
__global__ void k_lists(Geo g, const Stencils *__restrict__ st, int lo_level, int l_min,
                        const int *__restrict__ map, const uint8_t *__restrict__ cell_cls,
                        const int4 *__restrict__ cell_crd, const uint8_t *__restrict__ cell_hsrc,
                        int *__restrict__ far_cnt, int *__restrict__ far_src,
                        uint16_t *__restrict__ far_op, int *__restrict__ near_cnt,
                        int *__restrict__ near_src, const int64_t *__restrict__ lev_first,
                        int *__restrict__ far_full, int *__restrict__ cls_cnt,
                        int *__restrict__ cls_cells, int64_t cls_cap, const int *__restrict__ pmap) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t first = lev_first[lo_level];
  const int64_t gslot = first + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (gslot >= lev_first[g.L + 1]) return;   // warp-uniform
  int l = lo_level;
  while (l < g.L && gslot >= lev_first[l + 1]) ++l;
  const int4 c = cell_crd[gslot];
  const int cls = cell_cls[gslot];
  const int64_t fi = gslot - first;
  const int n_far = l >= l_min ? st->far_len[cls] : 0;
  int cnt = 0;
  for (int e0 = 0; e0 < n_far; e0 += 32) {
    const int e = e0 + lane;
    int s = -1;
    if (e < n_far) {
      const int4 q = make_int4(c.x + st->far_d[cls][e][0], c.y + st->far_d[cls][e][1],
                               c.z + st->far_d[cls][e][2], 0);
      if (pmap) {
        s = tri_pmap_lookup(pmap, l, q);
      } else {
        uint32_t k;
        if (cell_at(g, l, q, &k)) {
          s = map[g.map_off[l] + k];
          if (s >= 0 && !cell_hsrc[s]) s = -1;
        }
      }
      if (far_full) far_full[fi * FAR_MAX + e] = s;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, s >= 0);
    if (s >= 0) {
      const int at = cnt + __popc(hit & lt);
      far_src[fi * FAR_MAX + at] = s;
      far_op[fi * FAR_MAX + at] = st->far_op[cls][e];
    }
    cnt += __popc(hit);
  }
  if (lane == 0) {
    far_cnt[fi] = cnt;
    if (cls_cnt && n_far > 0) {
      // group the M2L targets by stencil class for the tensor-core M2L
      const int pos = atomicAdd(&cls_cnt[cls], 1);
      cls_cells[(int64_t)cls * cls_cap + pos] = (int)gslot;
    }
  }
  if (l == g.L) {
    const int o = (g.tiling == FMM2D_TRI && c.w == 0) ? 1 : 0;
    const int64_t ni = gslot - lev_first[g.L];
    int s = -1;
    if (lane < st->near_len[o]) {
      const int4 q = make_int4(c.x + st->near_d[o][lane][0], c.y + st->near_d[o][lane][1],
                               c.z + st->near_d[o][lane][2], 0);
      if (pmap) {
        s = tri_pmap_lookup(pmap, l, q);
      } else {
        uint32_t k;
        if (cell_at(g, l, q, &k)) {
          s = map[g.map_off[l] + k];
          if (s >= 0 && !cell_hsrc[s]) s = -1;
        }
      }
    }
    const unsigned hit = __ballot_sync(0xffffffffu, s >= 0);
    if (s >= 0) near_src[ni * NEAR_MAX + __popc(hit & lt)] = s;
    if (lane == 0) near_cnt[ni] = __popc(hit);
  }
}

inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

}  // namespace

cudaError_t launch_mark(const Geo &g, const uint32_t *key_sorted, int64_t n, int *occ, int *hsrc,
                        cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_mark<<<nblk(n, 256), 256, 0, s>>>(g, key_sorted, n, occ, hsrc);
  return cudaGetLastError();
}

cudaError_t launch_compact(const Geo &g, const int *occ, const int *scan, const int *hsrc,
                           int64_t map_size, int *map, uint32_t *cell_key, int4 *cell_crd,
                           double2 *cell_ctr, uint8_t *cell_cls, uint8_t *cell_hsrc,
                           int *src_start, int *src_end, int *tgt_start, int *tgt_end,
                           int64_t *lev_first, int *pmap, cudaStream_t s) {
  k_compact<<<nblk(map_size, 256), 256, 0, s>>>(g, occ, scan, hsrc, map_size, map, cell_key,
                                                 cell_crd, cell_ctr, cell_cls, cell_hsrc, src_start,
                                                 src_end, tgt_start, tgt_end, lev_first, pmap);
  return cudaGetLastError();
}

cudaError_t launch_rel_coords(const Geo &g, bool f32_in, bool f32_out, const void *xy,
                              const uint32_t *perm, const uint32_t *key_sorted, int64_t n,
                              const int *map, const double2 *ctr, void *out, int out_stride,
                              int *start, int *end, cudaStream_t s, float2 *lo) {
  if (n <= 0) return cudaSuccess;
  unsigned b = nblk(n, 256);
  if (f32_in && f32_out)
    k_rel<float, float><<<b, 256, 0, s>>>(g, (const float *)xy, perm, key_sorted, n, map, ctr, (float *)out, out_stride, start, end, lo);
  else if (f32_in)
    k_rel<float, double><<<b, 256, 0, s>>>(g, (const float *)xy, perm, key_sorted, n, map, ctr, (double *)out, out_stride, start, end, lo);
  else if (f32_out)
    k_rel<double, float><<<b, 256, 0, s>>>(g, (const double *)xy, perm, key_sorted, n, map, ctr, (float *)out, out_stride, start, end, lo);
  else
    k_rel<double, double><<<b, 256, 0, s>>>(g, (const double *)xy, perm, key_sorted, n, map, ctr, (double *)out, out_stride, start, end, lo);
  return cudaGetLastError();
}

cudaError_t launch_lists(const Geo &g, const Stencils *d_sten, int lo_level, int l_min, int64_t cap,
                         const int *map, const uint8_t *cell_cls, const int4 *cell_crd,
                         const uint8_t *cell_hsrc, int *far_cnt, int *far_src, uint16_t *far_op,
                         int *near_cnt, int *near_src, const int64_t *lev_first_dev,
                         int *far_full, int *cls_cnt, int *cls_cells, int64_t cls_cap,
                         const int *pmap, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  k_lists<<<nblk(cap * 32, 256), 256, 0, s>>>(g, d_sten, lo_level, l_min, map, cell_cls, cell_crd,
                                          cell_hsrc, far_cnt, far_src, far_op, near_cnt, near_src,
                                          lev_first_dev, far_full, cls_cnt, cls_cells, cls_cap, pmap);
  return cudaGetLastError();
}

}  // namespace fmm2d
