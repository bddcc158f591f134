// adaptive.cu - the adaptive tree for clustered input: cells split while they
// hold more than `cap` sources or targets, interaction lists by a
// level-synchronous dual traversal, and the two cross-level operators.
//
// Tree.  Points are keyed and sorted on the finest level Lmax, so the points
// of a level-l cell (a key prefix, Parent(n) = n div b, Sec. 4-6) are one
// contiguous range.  Level by level, each cell that must split finds its
// children's ranges by binary search on the sorted keys; occupied children
// are compacted (flag, scan, emit) into the next level.  Cells of all levels
// live in one array ordered by (level, key); children of a cell are
// contiguous.
//
// Lists.  Per level, three kinds of items are expanded (count pass, one scan,
// emit pass, so the output order is deterministic):
//  * a cell a: its Near stencil cells m (Sec. 4-6) that exist - both leaves:
//    P2P pair (U); a leaf and m split: m's children go to the W test; a split
//    and m a leaf: a's children go to the X test; its NeighborsE4 cells (eq. 3)
//    that exist: M2L list, in the uniform tree's format;
//  * a W test (leaf a, finer cell c): c separated from a (no cell of Near(c)
//    lies inside a) -> M2P (W); else c a leaf -> U; else c's children;
//  * an X test (cell a, coarser leaf c): mirrored -> P2L (X), U, or a's
//    children.
// The U, W and X pairs are then grouped by target (stable sort).
//
// Forest.  Many independent instances (same tiling and domain) form one tree
// with one level-0 cell per instance: a level-l key is inst * b^l + the
// instance-local key, so every key arithmetic below works on the local part
// and lookups re-attach the instance.  Instances never interact.
//
// Operators (Greengard-Rokhlin series, scaled like the uniform expansions):
//  * M2P: phi(y) += Q log|y - c| + Re sum_k a^_k (s_c / (y - c))^k
//  * P2L: L_0 += sum u log|x - c|, b^_l += -(1/l) sum u (s_c / (x - c))^l
#include "cells.cuh"
#include "plan.h"

namespace fmm2d {

namespace {

inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

__device__ __forceinline__ uint64_t level_span(int b, int up) {   // b^up
  uint64_t v = 1;
  for (int i = 0; i < up; ++i) v *= (uint64_t)b;
  return v;
}

// split a level-l key into instance and local key
__device__ __forceinline__ uint32_t local_key(int b, int l, uint32_t key, uint32_t *inst) {
  const uint64_t pw = level_span(b, l);
  *inst = (uint32_t)(key / pw);
  return (uint32_t)(key % pw);
}

// first index in [lo, hi) with key >= x
__device__ __forceinline__ int lower_bound_u32(const uint32_t *__restrict__ k, int lo, int hi, uint64_t x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((uint64_t)k[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint64_t ad_hash(uint64_t x) {   // a 64-bit mixer (splitmix64 finaliser)
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// Table key of the level-l lattice position q of instance `inst`, or false
// when q cannot be a cell of level l (so that it never aliases another):
//  * quad and tri: inst * 4^l + x * 2^l + y, below 2^32 as the level's cell
//    keys are; a tri position must also have x + y + z = 2^l - 1 (an up
//    triangle, bit 58) or 2^l - 2, and z in range (Sec. 6);
//  * septree: the Eisenstein coordinates (a, b) of every level-l cell obey
//    |a|, |b| < 7^(l/2) (the cell is a sum of l units times powers of the
//    base, whose modulus is sqrt 7), so each, biased, fits cb = (3l+1)/2 + 2
//    bits, and inst * 2^(2 cb) < 2^40 for the instances a 32-bit key allows.
// Level + 1 sits in bits 59-63, so no key is 0 (the empty slot).
__device__ __forceinline__ bool crd_key(int tiling, int l, uint32_t inst, int4 q, uint64_t *out) {
  uint64_t u;
  if (tiling == FMM2D_SEPT) {
    const int cb = (3 * l + 1) / 2 + 2;
    const int half = 1 << (cb - 1);
    if (q.x < -half || q.x >= half || q.y < -half || q.y >= half) return false;
    u = ((uint64_t)inst << (2 * cb)) | ((uint64_t)(q.x + half) << cb) | (uint64_t)(q.y + half);
  } else {
    const int n = 1 << l;
    if (q.x < 0 || q.y < 0 || q.x >= n || q.y >= n) return false;
    u = ((uint64_t)inst << (2 * l)) | ((uint64_t)q.x << l) | (uint64_t)q.y;
    if (tiling == FMM2D_TRI) {
      const int sum = q.x + q.y + q.z;
      if (q.z < 0 || q.z >= n || (sum != n - 1 && sum != n - 2)) return false;
      if (sum == n - 1) u |= 1ull << 58;
    }
  }
  *out = ((uint64_t)(l + 1) << 59) | u;
  return true;
}

// The cell with sources at level-l lattice position q of instance `inst`, or
// -1 (no such cell, or one without sources): linear probing in the
// (level, instance, position) table.
__device__ __forceinline__ int find_cell(const AdCells &c, int tiling, int l, uint32_t inst, int4 q) {
  uint64_t k;
  if (!crd_key(tiling, l, inst, q, &k)) return -1;
  uint32_t h = (uint32_t)ad_hash(k) & c.hmask;
  for (uint32_t probe = 0; probe <= c.hmask; ++probe) {
    const ulonglong2 e = __ldg(&c.hslot[h]);
    if (e.x == k) return (int)e.y;
    if (e.x == 0) return -1;
    h = (h + 1) & c.hmask;
  }
  return -1;
}

// Does the level-lf lattice position q lie inside the coarser level-lc cell
// (position ccrd, local key ckey)?  Quad and tri: the ancestor d levels up
// of a position is the position shifted right by d (a key's digits are the
// bits of the coordinates, Sec. 6), so no key is formed; septree: through
// the key of q.
__device__ __forceinline__ bool inside_coarse(const Geo &g, int lf, int4 q, int lc, int4 ccrd,
                                              uint32_t ckey) {
  if (g.tiling == FMM2D_SEPT) {
    uint32_t k;
    return cell_at(g, lf, q, &k) && parent_key(g.tiling, k, lf - lc) == ckey;
  }
  const int n = 1 << lf, d = lf - lc;
  if (q.x < 0 || q.y < 0 || q.x >= n || q.y >= n) return false;
  if (g.tiling == FMM2D_TRI) {
    const int sum = q.x + q.y + q.z;
    if (q.z < 0 || q.z >= n || (sum != n - 1 && sum != n - 2)) return false;
    if ((q.z >> d) != ccrd.z) return false;
  }
  return (q.x >> d) == ccrd.x && (q.y >> d) == ccrd.y;
}

// One level-0 cell per instance: instance i owns sources [soff[i], soff[i+1])
// and targets [toff[i], toff[i+1]) (one instance: the whole sets).
__global__ void k_ad_roots(Geo g, int n_inst, const int64_t *__restrict__ soff,
                           const int64_t *__restrict__ toff, int64_t n_s, int64_t n_t, AdCells c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst) return;
  int4 crd;
  double2 ctr;
  uint8_t cls;
  cell_geometry(g, 0, 0u, &crd, &ctr, &cls);
  const int s0 = soff ? (int)soff[i] : 0, s1 = soff ? (int)soff[i + 1] : (int)n_s;
  const int t0 = toff ? (int)toff[i] : 0, t1 = toff ? (int)toff[i + 1] : (int)n_t;
  c.key[i] = (uint32_t)i;
  c.lev[i] = 0;
  c.parent[i] = -1;
  c.child_first[i] = 0;
  c.child_cnt[i] = 0;
  c.split[i] = 0;
  c.ss[i] = s0;
  c.se[i] = s1;
  c.ts[i] = t0;
  c.te[i] = t1;
  c.crd[i] = crd;
  c.ctr[i] = ctr;
  c.cls[i] = cls;
  c.hsrc[i] = s1 > s0;
}

// Instance prefix of the finest-level keys: key += inst * b^L, the instance
// found by binary search in the offsets.
__global__ void k_ad_prefix(int64_t n, uint32_t *__restrict__ key, const int64_t *__restrict__ off,
                            int n_inst, uint64_t span) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = n_inst;   // last instance with off[inst] <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid;
  }
  key[i] = (uint32_t)((uint64_t)key[i] + (uint64_t)lo * span);
}

// Split decision and children's point ranges of the cells of level l.
__global__ void k_ad_split(Geo g, int l, int64_t first, int64_t count, int cap,
                           const uint32_t *__restrict__ skey, const uint32_t *__restrict__ tkey,
                           AdCells c, int *__restrict__ flag, int4 *__restrict__ crange) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t cell = first + i;
  const int ss = c.ss[cell], se = c.se[cell], ts = c.ts[cell], te = c.te[cell];
  const bool split = l < g.L && max(se - ss, te - ts) > cap;
  c.split[cell] = split ? 1 : 0;
  const int b = g.b;
  if (!split) {
    for (int d = 0; d < b; ++d) flag[i * b + d] = 0;
    return;
  }
  const uint64_t span = level_span(b, g.L - l - 1);
  const uint64_t key = c.key[cell];
  int s0 = ss, t0 = ts;
  for (int d = 0; d < b; ++d) {
    const uint64_t hi = (key * b + d + 1) * span;
    const int s1 = lower_bound_u32(skey, s0, se, hi);
    const int t1 = tkey ? lower_bound_u32(tkey, t0, te, hi) : s1;
    crange[i * b + d] = make_int4(s0, s1, tkey ? t0 : s0, t1);
    flag[i * b + d] = (s1 > s0 || t1 > (tkey ? t0 : s0)) ? 1 : 0;
    s0 = s1;
    t0 = t1;
  }
}

// Occupied children of the split cells of level l -> cells of level l + 1.
__global__ void k_ad_emit(Geo g, int l, int64_t first, int64_t count, int64_t next_first,
                          const int *__restrict__ flag, const int *__restrict__ pos,
                          const int4 *__restrict__ crange, AdCells c) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t cell = first + i;
  const int b = g.b;
  int n = 0;
  for (int d = 0; d < b; ++d) {
    if (!flag[i * b + d]) continue;
    const int64_t ch = next_first + pos[i * b + d];
    if (n == 0) c.child_first[cell] = (int)ch;
    ++n;
    const uint32_t key = c.key[cell] * (uint32_t)b + (uint32_t)d;
    int4 crd;
    double2 ctr;
    uint8_t cls;
    uint32_t inst;
    cell_geometry(g, l + 1, local_key(b, l + 1, key, &inst), &crd, &ctr, &cls);
    const int4 r = crange[i * b + d];
    c.key[ch] = key;
    c.lev[ch] = (uint8_t)(l + 1);
    c.parent[ch] = (int)cell;
    c.child_first[ch] = 0;
    c.child_cnt[ch] = 0;
    c.split[ch] = 0;
    c.ss[ch] = r.x;
    c.se[ch] = r.y;
    c.ts[ch] = r.z;
    c.te[ch] = r.w;
    c.crd[ch] = crd;
    c.ctr[ch] = ctr;
    c.cls[ch] = cls;
    c.hsrc[ch] = r.y > r.x;
  }
  c.child_cnt[cell] = (uint8_t)n;
  if (n == 0) c.child_first[cell] = 0;
}

__global__ void k_ad_level_total(int64_t count_b, const int *__restrict__ flag,
                                 const int *__restrict__ pos, int *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    out[0] = count_b > 0 ? pos[count_b - 1] + flag[count_b - 1] : 0;
}

__global__ void k_ad_leaf_flags(int64_t n, const uint8_t *__restrict__ split, int *__restrict__ flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) flag[i] = split[i] ? 0 : 1;
}

__global__ void k_ad_leaf_ids(int64_t n, const int *__restrict__ flag, const int *__restrict__ pos,
                              int *__restrict__ leaf_ids, int *__restrict__ leaf_pos) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (flag[i]) {
    leaf_ids[pos[i]] = (int)i;
    leaf_pos[i] = pos[i];
  } else {
    leaf_pos[i] = -1;
  }
}

// Points of every leaf relative to the leaf centre (one warp per leaf).
template <typename TI, typename TO>
__global__ void k_ad_rel(const TI *__restrict__ xy, const uint32_t *__restrict__ perm,
                         int64_t n_leaves, const int *__restrict__ leaf_ids,
                         const int *__restrict__ start, const int *__restrict__ end,
                         const double2 *__restrict__ ctr, TO *__restrict__ out, int stride,
                         float2 *__restrict__ lo) {
  const int lane = threadIdx.x & 31;
  const int64_t li = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (li >= n_leaves) return;
  const int cell = leaf_ids[li];
  const double2 c = ctr[cell];
  for (int i = start[cell] + lane; i < end[cell]; i += 32) {
    const uint32_t o = perm[i];
    const double x = (double)xy[2 * (int64_t)o], y = (double)xy[2 * (int64_t)o + 1];
    TO *dst = out + (int64_t)i * stride;
    const double dx = x - c.x, dy = y - c.y;
    dst[0] = (TO)dx;
    dst[1] = (TO)dy;
    for (int q = 2; q < stride; ++q) dst[q] = (TO)0;
    if (lo) lo[i] = make_float2((float)(dx - (double)(float)dx), (float)(dy - (double)(float)dy));
  }
}

// ---- list traversal ---------------------------------------------------------
enum { K_U = 0, K_W, K_X, K_T, K_S, K_KINDS };

struct ListOut {
  int *cnt;                           // count pass: [K_KINDS][n_items]
  const int *off;                     // emit pass: exclusive scan of cnt
  int64_t n_items;
  int64_t base[K_KINDS];              // emit pass: global offset of this level's block
  int *u_t, *u_s, *w_t, *w_s, *x_t, *x_s;
  int *t_a, *t_c, *s_a, *s_c;         // next level's W and X tests
};

template <bool EMIT>
struct Emitter {
  const ListOut &o;
  int64_t item;
  int n[K_KINDS];
  __device__ Emitter(const ListOut &out, int64_t it) : o(out), item(it) {
    for (int k = 0; k < K_KINDS; ++k) n[k] = 0;
  }
  __device__ void put(int kind, int a, int c) {
    if (EMIT) {
      const int64_t at = o.base[kind] + (o.off[kind * o.n_items + item] - o.off[kind * o.n_items]) + n[kind];
      int *A, *C;
      switch (kind) {
        case K_U: A = o.u_t; C = o.u_s; break;
        case K_W: A = o.w_t; C = o.w_s; break;
        case K_X: A = o.x_t; C = o.x_s; break;
        case K_T: A = o.t_a; C = o.t_c; break;
        default: A = o.s_a; C = o.s_c; break;
      }
      A[at] = a;
      C[at] = c;
    }
    ++n[kind];
  }
  __device__ void done() {
    if (!EMIT)
      for (int k = 0; k < K_KINDS; ++k) o.cnt[k * o.n_items + item] = n[k];
  }
};

// true when no cell of Near(fine, lf) lies inside the coarser cell
// (level lc, position ccrd, local key ckey)
__device__ bool separated(const Geo &g, const Stencils &st, int lf, int4 fcrd, int lc, int4 ccrd,
                          uint32_t ckey) {
  const int o = (g.tiling == FMM2D_TRI && fcrd.w == 0) ? 1 : 0;
  for (int e = 0; e < st.near_len[o]; ++e) {
    const int4 q = make_int4(fcrd.x + st.near_d[o][e][0], fcrd.y + st.near_d[o][e][1],
                             fcrd.z + st.near_d[o][e][2], 0);
    if (inside_coarse(g, lf, q, lc, ccrd, ckey)) return false;
  }
  return true;
}

// One thread per item it0 .. it1 - 1 (cells of level l, then W tests, then X
// tests): for levels with enough items to fill the GPU, where the cooperative
// forms below would mostly idle lanes.
template <bool EMIT>
__global__ void k_ad_lists_1t(Geo g, const Stencils *__restrict__ stp, int l, int l_min,
                           int64_t first, int64_t count, int64_t n_t, int64_t n_s,
                           const int *__restrict__ t_a, const int *__restrict__ t_c,
                           const int *__restrict__ s_a, const int *__restrict__ s_c, AdCells c,
                           ListOut out, int64_t far_first, int *__restrict__ far_cnt,
                           int *__restrict__ far_src, uint16_t *__restrict__ far_op,
                           int *__restrict__ far_full, int *__restrict__ cls_cnt,
                           int *__restrict__ cls_cells, int64_t cls_cap, int64_t it0, int64_t it1) {
  const int64_t it = it0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (it >= it1) return;
  const Stencils &st = *stp;
  Emitter<EMIT> em(out, it);
  if (it < count) {                                   // a cell of level l
    const int a = (int)(first + it);
    const bool a_tgt = c.te[a] > c.ts[a];
    const int4 ca = c.crd[a];
    uint32_t inst;
    local_key(g.b, l, c.key[a], &inst);
    if (a_tgt) {
      const int o = (g.tiling == FMM2D_TRI && ca.w == 0) ? 1 : 0;
      const bool a_leaf = !c.split[a];
      for (int e = 0; e < st.near_len[o]; ++e) {
        const int4 q = make_int4(ca.x + st.near_d[o][e][0], ca.y + st.near_d[o][e][1],
                                 ca.z + st.near_d[o][e][2], 0);
        const int m = find_cell(c, g.tiling, l, inst, q);
        if (m < 0) continue;
        const bool m_leaf = !c.split[m];
        if (a_leaf && m_leaf) {
          em.put(K_U, a, m);
        } else if (a_leaf) {
          for (int d = 0; d < c.child_cnt[m]; ++d) {
            const int ch = c.child_first[m] + d;
            if (c.hsrc[ch]) em.put(K_T, a, ch);
          }
        } else if (m_leaf) {
          for (int d = 0; d < c.child_cnt[a]; ++d) {
            const int ch = c.child_first[a] + d;
            if (c.te[ch] > c.ts[ch]) em.put(K_S, ch, m);
          }
        }
      }
    }
    if (EMIT && l >= l_min) {                         // M2L list (uniform format)
      const int cls = c.cls[a];
      const int64_t fi = a - far_first;
      int cnt = 0;
      const int n_far = a_tgt ? st.far_len[cls] : 0;
      for (int e = 0; e < st.far_len[cls]; ++e) {
        int sidx = -1;
        if (e < n_far) {
          const int4 q = make_int4(ca.x + st.far_d[cls][e][0], ca.y + st.far_d[cls][e][1],
                                   ca.z + st.far_d[cls][e][2], 0);
          sidx = find_cell(c, g.tiling, l, inst, q);
        }
        if (far_full) far_full[fi * FAR_MAX + e] = sidx;
        if (sidx < 0) continue;
        far_src[fi * FAR_MAX + cnt] = sidx;
        far_op[fi * FAR_MAX + cnt] = st.far_op[cls][e];
        ++cnt;
      }
      far_cnt[fi] = cnt;
      if (cls_cnt && st.far_len[cls] > 0) {
        const int pos = atomicAdd(&cls_cnt[cls], 1);
        cls_cells[(int64_t)cls * cls_cap + pos] = a;
      }
    }
  } else if (it < count + n_t) {                      // W test: leaf a, finer cell cc
    const int64_t j = it - count;
    const int a = t_a[j], cc = t_c[j];
    uint32_t inst;
    if (separated(g, st, l, c.crd[cc], c.lev[a], c.crd[a], local_key(g.b, c.lev[a], c.key[a], &inst)))
      em.put(K_W, a, cc);
    else if (!c.split[cc]) em.put(K_U, a, cc);
    else
      for (int d = 0; d < c.child_cnt[cc]; ++d) {
        const int ch = c.child_first[cc] + d;
        if (c.hsrc[ch]) em.put(K_T, a, ch);
      }
  } else {                                            // X test: cell a, coarser leaf cc
    const int64_t j = it - count - n_t;
    const int a = s_a[j], cc = s_c[j];
    uint32_t inst;
    if (separated(g, st, l, c.crd[a], c.lev[cc], c.crd[cc], local_key(g.b, c.lev[cc], c.key[cc], &inst)))
      em.put(K_X, a, cc);
    else if (!c.split[a]) em.put(K_U, a, cc);
    else
      for (int d = 0; d < c.child_cnt[a]; ++d) {
        const int ch = c.child_first[a] + d;
        if (c.te[ch] > c.ts[ch]) em.put(K_S, ch, cc);
      }
  }
  em.done();
}

// The W and X tests of level l, items it0 = count, count + 1, ...: half a
// warp per test, lane e of the half checking Near stencil entry e of the
// finer cell (does it lie inside the coarser one?); lane 0 of the half then
// writes the outcome as one thread would.
template <bool EMIT>
__global__ void k_ad_lists(Geo g, const Stencils *__restrict__ stp, int l, int64_t count,
                           int64_t n_t, int64_t n_s, const int *__restrict__ t_a,
                           const int *__restrict__ t_c, const int *__restrict__ s_a,
                           const int *__restrict__ s_c, AdCells c, ListOut out, int64_t it0) {
  const int lane = threadIdx.x & 31, sub = lane & 15;
  const unsigned hmask = 0xFFFFu << (lane & 16);
  const int64_t it = it0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 4);
  if (it >= count + n_t + n_s) return;              // uniform within the half warp
  const Stencils &st = *stp;
  const bool w_test = it < count + n_t;
  const int64_t j = w_test ? it - count : it - count - n_t;
  const int a = w_test ? t_a[j] : s_a[j], cc = w_test ? t_c[j] : s_c[j];
  // W: fine cell cc (level l) against the leaf a; X: fine cell a against the leaf cc
  const int fine = w_test ? cc : a, coarse = w_test ? a : cc;
  const int lc = c.lev[coarse];
  uint32_t inst;
  const uint32_t ckey = local_key(g.b, lc, c.key[coarse], &inst);
  const int4 fcrd = c.crd[fine];
  const int o = (g.tiling == FMM2D_TRI && fcrd.w == 0) ? 1 : 0;
  bool inside = false;
  if (sub < st.near_len[o]) {
    const int4 q = make_int4(fcrd.x + st.near_d[o][sub][0], fcrd.y + st.near_d[o][sub][1],
                             fcrd.z + st.near_d[o][sub][2], 0);
    inside = inside_coarse(g, l, q, lc, c.crd[coarse], ckey);
  }
  const bool sep = __ballot_sync(hmask, inside) == 0u;
  if (sub != 0) return;
  Emitter<EMIT> em(out, it);
  if (w_test) {
    if (sep) em.put(K_W, a, cc);
    else if (!c.split[cc]) em.put(K_U, a, cc);
    else
      for (int d = 0; d < c.child_cnt[cc]; ++d) {
        const int ch = c.child_first[cc] + d;
        if (c.hsrc[ch]) em.put(K_T, a, ch);
      }
  } else {
    if (sep) em.put(K_X, a, cc);
    else if (!c.split[a]) em.put(K_U, a, cc);
    else
      for (int d = 0; d < c.child_cnt[a]; ++d) {
        const int ch = c.child_first[a] + d;
        if (c.te[ch] > c.ts[ch]) em.put(K_S, ch, cc);
      }
  }
  em.done();
}

// The cell items of a level's traversal, a warp per cell: lane e takes
// Near stencil entry e (and far stencil entries e, e + 32), so the ~50
// lookups of a cell run side by side; per-kind warp scans (near part) and
// ballots (far part) keep the output in stencil order, as one thread would
// write it.
template <bool EMIT>
__global__ void k_ad_cell_lists(Geo g, const Stencils *__restrict__ stp, int l, int l_min,
                                int64_t first, int64_t count, AdCells c, ListOut out,
                                int64_t far_first, int *__restrict__ far_cnt,
                                int *__restrict__ far_src, uint16_t *__restrict__ far_op,
                                int *__restrict__ far_full, int *__restrict__ cls_cnt,
                                int *__restrict__ cls_cells, int64_t cls_cap) {
  const int lane = threadIdx.x & 31;
  const int64_t it = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (it >= count) return;                          // warp-uniform
  const Stencils &st = *stp;
  const int a = (int)(first + it);
  const bool a_tgt = c.te[a] > c.ts[a];
  const int4 ca = c.crd[a];
  uint32_t inst;
  local_key(g.b, l, c.key[a], &inst);
  // near stencil entry `lane`: U (a, m), T (a, child of m) or S (child of a, m)
  int m = -1, mode = 0, nk = 0;
  if (a_tgt) {
    const int o = (g.tiling == FMM2D_TRI && ca.w == 0) ? 1 : 0;
    if (lane < st.near_len[o]) {
      const int4 q = make_int4(ca.x + st.near_d[o][lane][0], ca.y + st.near_d[o][lane][1],
                               ca.z + st.near_d[o][lane][2], 0);
      m = find_cell(c, g.tiling, l, inst, q);
      if (m >= 0) {
        const bool a_leaf = !c.split[a], m_leaf = !c.split[m];
        if (a_leaf && m_leaf) {
          mode = 1;
          nk = 1;
        } else if (a_leaf) {
          mode = 2;
          for (int d = 0; d < c.child_cnt[m]; ++d) nk += c.hsrc[c.child_first[m] + d] ? 1 : 0;
        } else if (m_leaf) {
          mode = 3;
          for (int d = 0; d < c.child_cnt[a]; ++d) {
            const int ch = c.child_first[a] + d;
            nk += c.te[ch] > c.ts[ch] ? 1 : 0;
          }
        }
      }
    }
  }
  // exclusive scans of the three kinds' counts over the lanes
  const int kind = mode == 1 ? K_U : (mode == 2 ? K_T : K_S);
  int ex[3], tot[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int my = (mode == q + 1) ? nk : 0;
    int v = my;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += y;
    }
    tot[q] = __shfl_sync(0xffffffffu, v, 31);
    ex[q] = v - my;
  }
  if (!EMIT) {
    if (lane < K_KINDS) {
      const int v = lane == K_U ? tot[0] : (lane == K_T ? tot[1] : (lane == K_S ? tot[2] : 0));
      out.cnt[lane * out.n_items + it] = v;
    }
  } else if (mode != 0) {
    const int64_t at0 = out.base[kind] + (out.off[kind * out.n_items + it] - out.off[kind * out.n_items]) +
                        ex[mode - 1];
    int *A = kind == K_U ? out.u_t : (kind == K_T ? out.t_a : out.s_a);
    int *C = kind == K_U ? out.u_s : (kind == K_T ? out.t_c : out.s_c);
    if (mode == 1) {
      A[at0] = a;
      C[at0] = m;
    } else if (mode == 2) {
      int j = 0;
      for (int d = 0; d < c.child_cnt[m]; ++d) {
        const int ch = c.child_first[m] + d;
        if (!c.hsrc[ch]) continue;
        A[at0 + j] = a;
        C[at0 + j] = ch;
        ++j;
      }
    } else {
      int j = 0;
      for (int d = 0; d < c.child_cnt[a]; ++d) {
        const int ch = c.child_first[a] + d;
        if (c.te[ch] <= c.ts[ch]) continue;
        A[at0 + j] = ch;
        C[at0 + j] = m;
        ++j;
      }
    }
  }
  if (EMIT && l >= l_min) {                         // M2L list (uniform format)
    const int cls = c.cls[a];
    const int64_t fi = a - far_first;
    const int fl = st.far_len[cls];
    const int n_far = a_tgt ? fl : 0;
    int cnt = 0;
    for (int e0 = 0; e0 < fl; e0 += 32) {
      const int e = e0 + lane;
      int sidx = -1;
      if (e < n_far) {
        const int4 q = make_int4(ca.x + st.far_d[cls][e][0], ca.y + st.far_d[cls][e][1],
                                 ca.z + st.far_d[cls][e][2], 0);
        sidx = find_cell(c, g.tiling, l, inst, q);
      }
      if (far_full && e < fl) far_full[fi * FAR_MAX + e] = sidx;
      const unsigned bal = __ballot_sync(0xffffffffu, sidx >= 0);
      if (sidx >= 0) {
        const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
        far_src[fi * FAR_MAX + pos] = sidx;
        far_op[fi * FAR_MAX + pos] = st.far_op[cls][e];
      }
      cnt += __popc(bal);
    }
    if (lane == 0) {
      far_cnt[fi] = cnt;
      if (cls_cnt && fl > 0) {
        const int pos = atomicAdd(&cls_cnt[cls], 1);
        cls_cells[(int64_t)cls * cls_cap + pos] = a;
      }
    }
  }
}

__global__ void k_ad_kind_totals(const int *__restrict__ cnt, const int *__restrict__ off,
                                 int64_t n_items, int *__restrict__ out) {
  const int k = threadIdx.x;
  if (k >= K_KINDS || blockIdx.x != 0) return;
  const int64_t last = (int64_t)(k + 1) * n_items - 1;
  out[k] = n_items > 0 ? off[last] + cnt[last] - off[(int64_t)k * n_items] : 0;
}

// ---- grouping by target -----------------------------------------------------
// group of pair i; a target outside [0, n_groups) (never produced by the
// traversal) goes to the spare group n_groups, past the last CSR offset
__global__ void k_ad_keys_of(int64_t n, const int *__restrict__ tgt, const int *__restrict__ map,
                             int n_groups, uint32_t *__restrict__ key, uint32_t *__restrict__ idx) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int v = map ? map[tgt[i]] : tgt[i];
  key[i] = (uint32_t)((v < 0 || v >= n_groups) ? n_groups : v);
  idx[i] = (uint32_t)i;
}

__global__ void k_ad_count(int64_t n, const uint32_t *__restrict__ key, int *__restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[key[i]], 1);
}

__global__ void k_ad_gather(int64_t n, const uint32_t *__restrict__ idx, const int *__restrict__ src,
                            int *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = src[idx[i]];
}

// ---- M2P and P2L --------------------------------------------------------------
constexpr int AWPB = 4;

template <typename R>
__device__ __forceinline__ R warp_sum_ad(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
__device__ __forceinline__ double log_abs(Cx<R> d) {
  if constexpr (sizeof(R) == 4) {   // log|d| = (ln 2 / 2) log2|d|^2 on the MUFU unit
    float y;
    const float r2 = d.x * d.x + d.y * d.y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
    return 0.34657359027997264 * (double)y;
  } else {
    return 0.5 * log(d.x * d.x + d.y * d.y);
  }
}

// Butterfly reduce-scatter of 32 values per lane over the warp: lane l ends
// with the warp's total of value l (31 shuffles, against 32 x 5 for one
// tree reduction per value).
template <typename R>
__device__ __forceinline__ R warp_reduce_scatter32(R (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const R send = up ? v[i] : v[i + o];
      const R keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// One warp per target leaf: phi_near[j] += sum over its W cells of the
// cell's multipole evaluated at target j (Horner in z = s_c / (y - c)).
// The W cells' centres, scales and charges are fetched one per lane, 32 at
// a time; the multipole of the next cell is loaded while the current one is
// evaluated, and held one coefficient per lane (k and k + 32), so Horner's
// rule takes its coefficients by shuffle.
template <typename R>
__global__ void __launch_bounds__(32 * AWPB)
k_ad_m2p(int64_t n_leaves, const int *__restrict__ leaf_ids, const int *__restrict__ w_off,
         const int *__restrict__ w_src, const R *__restrict__ tgt, int tstride,
         const int *__restrict__ ts_, const int *__restrict__ te_, const double2 *__restrict__ ctr,
         const uint8_t *__restrict__ lev, const double2 *__restrict__ scale, int p, int P,
         const double *__restrict__ mQ, const Cx<R> *__restrict__ ma, double *__restrict__ phi) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t li = blockIdx.x * (int64_t)AWPB + w;
  if (li >= n_leaves) return;
  const int a = leaf_ids[li];
  const int e0 = w_off[li], e1 = w_off[li + 1];
  if (e0 == e1) return;
  const int ts = ts_[a], te = te_[a];
  const double2 ca = ctr[a];
  auto coef = [&](const Cx<R> &c0, const Cx<R> &c1, int k) -> Cx<R> {   // k warp-uniform
    const Cx<R> &c = k < 32 ? c0 : c1;
    return Cx<R>{__shfl_sync(FULL, c.x, k & 31), __shfl_sync(FULL, c.y, k & 31)};
  };
  for (int j0 = ts; j0 < te; j0 += 32) {
    const int j = j0 + lane;
    const bool act = j < te;
    const R tx = act ? tgt[(int64_t)j * tstride] : (R)0, ty = act ? tgt[(int64_t)j * tstride + 1] : (R)0;
    double acc = 0.0;
    for (int eb = e0; eb < e1; eb += 32) {
      const int nb = min(32, e1 - eb);
      int cc = 0;
      R dx = (R)0, dy = (R)0, sx = (R)0, sy = (R)0;
      double qc = 0.0;
      if (lane < nb) {
        cc = w_src[eb + lane];
        const double2 c2 = ctr[cc];
        const double2 sc = scale[lev[cc]];
        dx = (R)(ca.x - c2.x);
        dy = (R)(ca.y - c2.y);
        sx = (R)sc.x;
        sy = (R)sc.y;
        qc = mQ[cc];
      }
      Cx<R> cur0 = {(R)0, (R)0}, cur1 = {(R)0, (R)0};
      {
        const int c = __shfl_sync(FULL, cc, 0);
        if (lane < p) cur0 = ma[(int64_t)c * P + lane];
        if (lane + 32 < p) cur1 = ma[(int64_t)c * P + lane + 32];
      }
      for (int m = 0; m < nb; ++m) {
        Cx<R> nxt0 = {(R)0, (R)0}, nxt1 = {(R)0, (R)0};
        if (m + 1 < nb) {
          const int c = __shfl_sync(FULL, cc, m + 1);
          if (lane < p) nxt0 = ma[(int64_t)c * P + lane];
          if (lane + 32 < p) nxt1 = ma[(int64_t)c * P + lane + 32];
        }
        const Cx<R> d = {__shfl_sync(FULL, dx, m) + tx, __shfl_sync(FULL, dy, m) + ty};
        const Cx<R> sm = {__shfl_sync(FULL, sx, m), __shfl_sync(FULL, sy, m)};
        const double qm = __shfl_sync(FULL, qc, m);
        const R den = d.x * d.x + d.y * d.y;
        const Cx<R> id = {d.x / den, -d.y / den};
        const Cx<R> z = sm * id;                      // s_c / (y - c)
        Cx<R> h = coef(cur0, cur1, p - 1);            // a^_p
        for (int k = p - 2; k >= 0; --k) h = h * z + coef(cur0, cur1, k);
        h = h * z;
        acc += qm * log_abs(d) + (double)h.x;
        cur0 = nxt0;
        cur1 = nxt1;
      }
    }
    if (act) phi[j] += acc;
  }
}

// One warp per target cell: adds the local expansion of the sources of its X
// leaves.  The X leaves' ranges and centre offsets are fetched one per lane,
// 32 at a time, and the lanes take the points of those leaves one each, in
// order over the concatenated ranges (a lane finds its leaf by binary search
// over the lanes' range starts), so every lane is busy whatever the leaf
// sizes.  Coefficients come in chunks of KC (one chunk for p <= KC),
// reduced over the warp by reduce-scatter; L_0 is formed in the first chunk.
template <typename R, int KC>
__global__ void __launch_bounds__(32 * AWPB)
k_ad_p2l(int64_t n_cells, const int *__restrict__ x_off, const int *__restrict__ x_src,
         const R *__restrict__ src4, const int *__restrict__ ss_, const int *__restrict__ se_,
         const double2 *__restrict__ ctr, const uint8_t *__restrict__ lev,
         const double2 *__restrict__ inv_scale, int p, int P, double *__restrict__ lL0,
         Cx<R> *__restrict__ lb) {
  static_assert(2 * KC == 32, "one reduce-scatter value per lane");
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t a = blockIdx.x * (int64_t)AWPB + w;
  if (a >= n_cells) return;
  const int e0 = x_off[a], e1 = x_off[a + 1];
  if (e0 == e1) return;
  const double2 ca = ctr[a];
  const double2 is2 = inv_scale[lev[a]];
  const Cx<R> is = {(R)is2.x, (R)is2.y};
  double q = 0.0;   // L_0: sum u log|x - c_a|
  for (int k0 = 1; k0 <= p; k0 += KC) {
    Cx<R> acc[KC];
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) acc[kk] = {(R)0, (R)0};
    for (int eb = e0; eb < e1; eb += 32) {
      const int nb = min(32, e1 - eb);
      int st = 0, n = 0;
      R dcx = (R)0, dcy = (R)0;
      if (lane < nb) {
        const int cc = x_src[eb + lane];
        const double2 c2 = ctr[cc];
        dcx = (R)(c2.x - ca.x);
        dcy = (R)(c2.y - ca.y);
        st = ss_[cc];
        n = se_[cc] - st;
      }
      int incl = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
      }
      const int total = __shfl_sync(FULL, incl, 31);
      const int excl = incl - n;
      for (int i0 = 0; i0 < total; i0 += 32) {
        const int idx = i0 + lane;
        int m = 0;   // the last leaf m < nb whose range starts at or before idx
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int cand = m + step;
          const int ex = __shfl_sync(FULL, excl, cand & 31);
          if (cand < nb && ex <= idx) m = cand;
        }
        const int sm = __shfl_sync(FULL, st, m), xm = __shfl_sync(FULL, excl, m);
        const R ox = __shfl_sync(FULL, dcx, m), oy = __shfl_sync(FULL, dcy, m);
        if (idx < total) {
          const R *pt = src4 + 4 * (int64_t)(sm + idx - xm);
          const Cx<R> d = {pt[0] + ox, pt[1] + oy};
          if (k0 == 1) q += (double)pt[2] * log_abs(d);
          const Cx<R> zeta = d * is;                                  // (x - c_a) / s_a
          const R den = zeta.x * zeta.x + zeta.y * zeta.y;
          const Cx<R> z = {zeta.x / den, -zeta.y / den};              // s_a / (x - c_a)
          Cx<R> v = {pt[2], (R)0};
          for (int t = 0; t < k0; ++t) v = v * z;
#pragma unroll
          for (int kk = 0; kk < KC; ++kk) {
            acc[kk] = acc[kk] + v;
            v = v * z;
          }
        }
      }
    }
    R vals[32];
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      vals[2 * kk] = acc[kk].x;
      vals[2 * kk + 1] = acc[kk].y;
    }
    const R re = warp_reduce_scatter32(vals);     // lane 2kk: Re, lane 2kk+1: Im of chunk entry kk
    const R im = __shfl_down_sync(FULL, re, 1);
    const int k = k0 + (lane >> 1);
    if (!(lane & 1) && k <= p) {
      const R inv = (R)(-1.0) / (R)k;
      const Cx<R> cur = lb[a * P + k - 1];
      lb[a * P + k - 1] = {cur.x + re * inv, cur.y + im * inv};
    }
  }
  q = warp_sum_ad(q);
  if (lane == 0) lL0[a] += q;
}

}  // namespace

cudaError_t ad_launch_roots(const Geo &g, int n_inst, const int64_t *soff, const int64_t *toff,
                            int64_t n_s, int64_t n_t, const AdCells &c, cudaStream_t s) {
  if (n_inst <= 0) return cudaSuccess;
  k_ad_roots<<<nblk(n_inst, 128), 128, 0, s>>>(g, n_inst, soff, toff, n_s, n_t, c);
  return cudaGetLastError();
}

cudaError_t ad_launch_prefix(int64_t n, uint32_t *key, const int64_t *off, int n_inst, uint64_t span,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_ad_prefix<<<nblk(n, 256), 256, 0, s>>>(n, key, off, n_inst, span);
  return cudaGetLastError();
}

cudaError_t ad_launch_split(const Geo &g, int l, int64_t first, int64_t count, int cap,
                            const uint32_t *skey, const uint32_t *tkey, const AdCells &c, int *flag,
                            int4 *crange, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_ad_split<<<nblk(count, 128), 128, 0, s>>>(g, l, first, count, cap, skey, tkey, c, flag, crange);
  return cudaGetLastError();
}

cudaError_t ad_launch_level_total(int64_t count_b, const int *flag, const int *pos, int *total_out,
                                  cudaStream_t s) {
  k_ad_level_total<<<1, 32, 0, s>>>(count_b, flag, pos, total_out);
  return cudaGetLastError();
}

cudaError_t ad_launch_emit(const Geo &g, int l, int64_t first, int64_t count, int64_t next_first,
                           const int *flag, const int *pos, const int4 *crange, const AdCells &c,
                           cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_ad_emit<<<nblk(count, 128), 128, 0, s>>>(g, l, first, count, next_first, flag, pos, crange, c);
  return cudaGetLastError();
}

cudaError_t ad_launch_leaves(int64_t n_cells, const uint8_t *split, int *flag, int *pos,
                             void *scan_scratch, int *leaf_ids, int *leaf_pos, int *n_leaves_out,
                             cudaStream_t s) {
  if (n_cells <= 0) return cudaSuccess;
  k_ad_leaf_flags<<<nblk(n_cells, 256), 256, 0, s>>>(n_cells, split, flag);
  cudaError_t e = exclusive_scan(flag, pos, n_cells, scan_scratch, s);
  if (e != cudaSuccess) return e;
  k_ad_leaf_ids<<<nblk(n_cells, 256), 256, 0, s>>>(n_cells, flag, pos, leaf_ids, leaf_pos);
  k_ad_level_total<<<1, 32, 0, s>>>(n_cells, flag, pos, n_leaves_out);
  return cudaGetLastError();
}

cudaError_t ad_launch_rel(bool f32_in, bool f32_out, const void *xy, const uint32_t *perm,
                          int64_t n_leaves, const int *leaf_ids, const int *start, const int *end,
                          const double2 *ctr, void *out, int stride, cudaStream_t s, float2 *lo) {
  if (n_leaves <= 0) return cudaSuccess;
  const unsigned b = nblk(n_leaves * 32, 256);
  if (f32_in && f32_out)
    k_ad_rel<float, float><<<b, 256, 0, s>>>((const float *)xy, perm, n_leaves, leaf_ids, start, end, ctr, (float *)out, stride, lo);
  else if (f32_in)
    k_ad_rel<float, double><<<b, 256, 0, s>>>((const float *)xy, perm, n_leaves, leaf_ids, start, end, ctr, (double *)out, stride, lo);
  else if (f32_out)
    k_ad_rel<double, float><<<b, 256, 0, s>>>((const double *)xy, perm, n_leaves, leaf_ids, start, end, ctr, (float *)out, stride, lo);
  else
    k_ad_rel<double, double><<<b, 256, 0, s>>>((const double *)xy, perm, n_leaves, leaf_ids, start, end, ctr, (double *)out, stride, lo);
  return cudaGetLastError();
}

// Above these item counts a level fills the GPU with one thread per item
// (~52 dependent lookups per cell, 13 stencil checks per test) and the
// cooperative forms (32 lanes per cell, 16 per test) would mostly idle lanes.
constexpr int64_t COOP_MAX_CELLS = (int64_t)1 << 18;
constexpr int64_t COOP_MAX_TESTS = (int64_t)1 << 19;

namespace {
__global__ void k_ad_hash(Geo g, int64_t n, AdCells c, unsigned long long *__restrict__ slots,
                          uint32_t hmask) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || !c.hsrc[i]) return;
  const int l = c.lev[i];
  uint32_t inst;
  local_key(g.b, l, c.key[i], &inst);
  uint64_t k;
  if (!crd_key(g.tiling, l, inst, c.crd[i], &k)) return;   // never for a cell of the tree
  uint32_t h = (uint32_t)ad_hash(k) & hmask;
  for (uint32_t probe = 0; probe <= hmask; ++probe) {
    const unsigned long long prev = atomicCAS(&slots[2 * (size_t)h], 0ull, (unsigned long long)k);
    if (prev == 0ull || prev == k) {
      slots[2 * (size_t)h + 1] = (unsigned long long)i;
      return;
    }
    h = (h + 1) & hmask;
  }
}
}  // namespace

cudaError_t ad_launch_hash(const Geo &g, int64_t n_cells, const AdCells &c, ulonglong2 *slots,
                           uint32_t hmask, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(slots, 0, ((size_t)hmask + 1) * sizeof(ulonglong2), s);
  if (e != cudaSuccess || n_cells <= 0) return e;
  k_ad_hash<<<nblk(n_cells, 256), 256, 0, s>>>(g, n_cells, c, reinterpret_cast<unsigned long long *>(slots),
                                               hmask);
  return cudaGetLastError();
}

cudaError_t ad_launch_lists(const Geo &g, const Stencils *d_sten, int l, int l_min, int64_t first,
                            int64_t count, int64_t n_t, int64_t n_s, const int *t_a, const int *t_c,
                            const int *s_a, const int *s_c, const AdCells &c, int *cnt,
                            int *off, void *scan_scratch, int *totals, cudaStream_t s) {
  const int64_t n_items = count + n_t + n_s;
  if (n_items <= 0) return cudaSuccess;
  ListOut o{};
  o.cnt = cnt;
  o.n_items = n_items;
  if (count > COOP_MAX_CELLS)
    k_ad_lists_1t<false><<<nblk(count, 128), 128, 0, s>>>(g, d_sten, l, l_min, first, count, n_t, n_s, t_a,
                                                         t_c, s_a, s_c, c, o, 0, nullptr, nullptr, nullptr,
                                                         nullptr, nullptr, nullptr, 0, 0, count);
  else if (count > 0)
    k_ad_cell_lists<false><<<nblk(count * 32, 128), 128, 0, s>>>(g, d_sten, l, l_min, first, count, c, o,
                                                                 0, nullptr, nullptr, nullptr, nullptr,
                                                                 nullptr, nullptr, 0);
  if (n_t + n_s > COOP_MAX_TESTS)
    k_ad_lists_1t<false><<<nblk(n_t + n_s, 128), 128, 0, s>>>(g, d_sten, l, l_min, first, count, n_t, n_s,
                                                             t_a, t_c, s_a, s_c, c, o, 0, nullptr, nullptr,
                                                             nullptr, nullptr, nullptr, nullptr, 0, count,
                                                             n_items);
  else if (n_t + n_s > 0)
    k_ad_lists<false><<<nblk((n_t + n_s) * 16, 128), 128, 0, s>>>(g, d_sten, l, count, n_t, n_s, t_a, t_c,
                                                                 s_a, s_c, c, o, count);
  cudaError_t e = exclusive_scan(cnt, off, n_items * K_KINDS, scan_scratch, s);
  if (e != cudaSuccess) return e;
  k_ad_kind_totals<<<1, 32, 0, s>>>(cnt, off, n_items, totals);
  return cudaGetLastError();
}

cudaError_t ad_launch_lists_emit(const Geo &g, const Stencils *d_sten, int l, int l_min,
                                 int64_t first, int64_t count, int64_t n_t, int64_t n_s,
                                 const int *t_a, const int *t_c, const int *s_a, const int *s_c,
                                 const AdCells &c, const int *off, const int64_t base[5],
                                 int *u_t, int *u_s, int *w_t, int *w_s, int *x_t, int *x_s,
                                 int *nt_a, int *nt_c, int *ns_a, int *ns_c, int64_t far_first,
                                 int *far_cnt, int *far_src, uint16_t *far_op, int *far_full,
                                 int *cls_cnt, int *cls_cells, int64_t cls_cap, cudaStream_t s) {
  const int64_t n_items = count + n_t + n_s;
  if (n_items <= 0) return cudaSuccess;
  ListOut o{};
  o.off = off;
  o.n_items = n_items;
  for (int k = 0; k < K_KINDS; ++k) o.base[k] = base[k];
  o.u_t = u_t; o.u_s = u_s; o.w_t = w_t; o.w_s = w_s; o.x_t = x_t; o.x_s = x_s;
  o.t_a = nt_a; o.t_c = nt_c; o.s_a = ns_a; o.s_c = ns_c;
  if (count > COOP_MAX_CELLS)
    k_ad_lists_1t<true><<<nblk(count, 128), 128, 0, s>>>(g, d_sten, l, l_min, first, count, n_t, n_s, t_a,
                                                        t_c, s_a, s_c, c, o, far_first, far_cnt, far_src,
                                                        far_op, far_full, cls_cnt, cls_cells, cls_cap, 0,
                                                        count);
  else if (count > 0)
    k_ad_cell_lists<true><<<nblk(count * 32, 128), 128, 0, s>>>(g, d_sten, l, l_min, first, count, c, o,
                                                                far_first, far_cnt, far_src, far_op,
                                                                far_full, cls_cnt, cls_cells, cls_cap);
  if (n_t + n_s > COOP_MAX_TESTS)
    k_ad_lists_1t<true><<<nblk(n_t + n_s, 128), 128, 0, s>>>(g, d_sten, l, l_min, first, count, n_t, n_s,
                                                            t_a, t_c, s_a, s_c, c, o, far_first, far_cnt,
                                                            far_src, far_op, far_full, cls_cnt, cls_cells,
                                                            cls_cap, count, n_items);
  else if (n_t + n_s > 0)
    k_ad_lists<true><<<nblk((n_t + n_s) * 16, 128), 128, 0, s>>>(g, d_sten, l, count, n_t, n_s, t_a, t_c,
                                                                s_a, s_c, c, o, count);
  return cudaGetLastError();
}

cudaError_t ad_group(int64_t n, const int *tgt, const int *src, const int *map, int n_groups,
                     uint32_t *key, uint32_t *idx, uint32_t *tmp_k, uint32_t *tmp_v, void *scratch,
                     int *cnt, int *off, int *out_src, cudaStream_t s, int *err) {
  cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)(n_groups + 1) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    k_ad_keys_of<<<nblk(n, 256), 256, 0, s>>>(n, tgt, map, n_groups, key, idx);
    int bits = 1;
    while ((1ll << bits) <= (int64_t)n_groups) ++bits;
    e = radix_sort_pairs(key, idx, tmp_k, tmp_v, n, bits, scratch, s, err);
    if (e != cudaSuccess) return e;
    k_ad_count<<<nblk(n, 256), 256, 0, s>>>(n, key, cnt);
    k_ad_gather<<<nblk(n, 256), 256, 0, s>>>(n, idx, src, out_src);
  }
  return exclusive_scan(cnt, off, (int64_t)n_groups + 1, scratch, s);
}

template <typename R>
cudaError_t ad_launch_m2p(int64_t n_leaves, const int *leaf_ids, const int *w_off, const int *w_src,
                          const R *tgt, int tstride, const int *ts, const int *te,
                          const double2 *ctr, const uint8_t *lev, const double2 *scale, int p,
                          int P, const double *mQ, const Cx<R> *ma, double *phi, cudaStream_t s) {
  if (n_leaves <= 0) return cudaSuccess;
  k_ad_m2p<R><<<nblk(n_leaves, AWPB), 32 * AWPB, 0, s>>>(n_leaves, leaf_ids, w_off, w_src, tgt,
                                                          tstride, ts, te, ctr, lev, scale, p, P,
                                                          mQ, ma, phi);
  return cudaGetLastError();
}

template <typename R>
cudaError_t ad_launch_p2l(int64_t n_cells, const int *x_off, const int *x_src, const R *src4,
                          const int *ss, const int *se, const double2 *ctr, const uint8_t *lev,
                          const double2 *inv_scale, int p, int P, double *lL0, Cx<R> *lb,
                          cudaStream_t s) {
  if (n_cells <= 0) return cudaSuccess;
  k_ad_p2l<R, 16><<<nblk(n_cells, AWPB), 32 * AWPB, 0, s>>>(n_cells, x_off, x_src, src4, ss, se, ctr,
                                                            lev, inv_scale, p, P, lL0, lb);
  return cudaGetLastError();
}

#define AD_INST(R)                                                                                \
  template cudaError_t ad_launch_m2p<R>(int64_t, const int *, const int *, const int *, const R *, \
                                        int, const int *, const int *, const double2 *,           \
                                        const uint8_t *, const double2 *, int, int,               \
                                        const double *, const Cx<R> *, double *, cudaStream_t);   \
  template cudaError_t ad_launch_p2l<R>(int64_t, const int *, const int *, const R *, const int *, \
                                        const int *, const double2 *, const uint8_t *,            \
                                        const double2 *, int, int, double *, Cx<R> *, cudaStream_t);
AD_INST(float)
AD_INST(double)

}  // namespace fmm2d
