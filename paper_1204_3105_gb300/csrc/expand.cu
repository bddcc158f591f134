// expand.cu - expansions and translations of the 2D log-kernel FMM (Sec. 2;
// the Greengard-Rokhlin operators the paper cites), on scaled coefficients.
//
// A level-l multipole is stored as Q (FP64) and a^_k = a_k / s_l^k, a local
// as L_0 (real part, FP64) and b^_l = b_l s_l^l, where s_l is the level's
// complex scale (cell radius; for the septree it also carries the lattice
// rotation of eq. 6).  With that scaling each translation depends only on
// the integer lattice offset (M2L) or the child class (M2M, L2L), so one
// table of (p+1) x (p+1) complex operators serves every level:
//   M2M: A^_l = Q (-w^l / l) + sum_{k<=l} C(l-1,k-1) sigma^k w^(l-k) a^_k
//   M2L: b^_l = Q (-zeta^-l / l) + sum_k C(l+k-1,k-1) (-1)^k zeta^-(l+k) a^_k,
//        L_0 += Q (log|s_l| + log|zeta|) + Re(row 0)
//   L2L: b^'_k = sum_{l>=k} C(l,k) w^(l-k) sigma^k b^_l
// (w = child offset / s_parent, sigma = s_child / s_parent,
//  zeta = (c_src - c_tgt) / s_l).  Column 0 of an operator multiplies Q.
#include "plan.h"

namespace fmm2d {

namespace {

constexpr int WPB = 4;   // warps per block

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Strength of every sorted source into component 2 of its record; with lo,
// the rounding residual u - (R)u goes to component 3 (hybrid P2P).
template <typename R>
__global__ void k_gather_u(const void *__restrict__ u, int f32_in, const uint32_t *__restrict__ perm,
                           int64_t n, R *__restrict__ src4, int lo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t o = perm[i];
  double v = f32_in ? (double)((const float *)u)[o] : ((const double *)u)[o];
  src4[4 * i + 2] = (R)v;
  if (lo) src4[4 * i + 3] = (R)(v - (double)(R)v);
}

template <typename R, int KC>
__global__ void __launch_bounds__(32 * WPB)
k_p2m(ExpandArgs a, const R *__restrict__ src4, const int *__restrict__ start,
      const int *__restrict__ end, double *__restrict__ mQ, Cx<R> *__restrict__ ma) {
  const int lane = threadIdx.x & 31;
  const int64_t li = blockIdx.x * (int64_t)WPB + (threadIdx.x >> 5);
  if (li >= a.n_leaves) return;
  const int64_t g = a.leaf_ids ? (int64_t)a.leaf_ids[li] : a.leaf_first + li;
  const int s = start[g], e = end[g];
  Cx<R> is = {(R)a.inv_s_re, (R)a.inv_s_im};
  if (a.leaf_ids) {
    const double2 v = a.inv_scale[a.cell_lev[g]];
    is = {(R)v.x, (R)v.y};
  }
  double q = 0.0;
  for (int i = s + lane; i < e; i += 32) q += (double)src4[4 * (int64_t)i + 2];
  q = warp_sum(q);
  if (lane == 0) mQ[g] = q;
  for (int k0 = 1; k0 <= a.p; k0 += KC) {
    Cx<R> acc[KC];
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) acc[kk] = {(R)0, (R)0};
    for (int i = s + lane; i < e; i += 32) {
      const R *pt = src4 + 4 * (int64_t)i;
      Cx<R> z = Cx<R>{pt[0], pt[1]} * is;
      Cx<R> w = {pt[2], (R)0};
      for (int t = 0; t < k0; ++t) w = w * z;       // u z^k0
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        acc[kk] = acc[kk] + w;
        w = w * z;
      }
    }
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      R re = warp_sum(acc[kk].x), im = warp_sum(acc[kk].y);
      int k = k0 + kk;
      if (lane == 0 && k <= a.p) {
        R inv = (R)(-1.0) / (R)k;
        ma[g * a.P + (k - 1)] = {re * inv, im * inv};
      }
    }
  }
}

// P2M by powers kept per point: lane i of the warp takes source i of every
// group of 32 and forms u z^k for k = 1, 2, ... by one complex product each;
// 16 powers at a time go through shared memory, where lane (r, h) sums row
// r over the 16 points of half h.  The FP64 work per source is p complex
// products and p / 16 partial sums (the form above repeats the powers below
// each chunk of 8 and reduces every coefficient with shuffles).
template <typename R>
__global__ void __launch_bounds__(32 * WPB)
k_p2m_t(ExpandArgs a, const R *__restrict__ src4, const int *__restrict__ start,
        const int *__restrict__ end, double *__restrict__ mQ, Cx<R> *__restrict__ ma) {
  constexpr int KC = 16, NCH = (MAXP + KC - 1) / KC;
  __shared__ Cx<R> sw[WPB][KC][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t li = blockIdx.x * (int64_t)WPB + w;
  if (li >= a.n_leaves) return;
  const int64_t g = a.leaf_ids ? (int64_t)a.leaf_ids[li] : a.leaf_first + li;
  const int s = start[g], e = end[g];
  Cx<R> is = {(R)a.inv_s_re, (R)a.inv_s_im};
  if (a.leaf_ids) {
    const double2 v = a.inv_scale[a.cell_lev[g]];
    is = {(R)v.x, (R)v.y};
  }
  const int p = a.p, r = lane & (KC - 1), h = lane >> 4;
  double q = 0.0;
  Cx<R> acc[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) acc[c] = {(R)0, (R)0};
  for (int i0 = s; i0 < e; i0 += 32) {
    const int i = i0 + lane;
    Cx<R> z = {(R)0, (R)0}, wk = {(R)0, (R)0};
    if (i < e) {
      const R *pt = src4 + 4 * (int64_t)i;
      z = Cx<R>{pt[0], pt[1]} * is;
      wk = {pt[2], (R)0};
      q += (double)pt[2];
    }
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const int nk = min(KC, p - c * KC);   // warp-uniform
      if (nk <= 0) break;
      for (int kk = 0; kk < nk; ++kk) {
        wk = wk * z;
        sw[w][kk][lane] = wk;
      }
      __syncwarp();
      if (r < nk) {
        Cx<R> t = {(R)0, (R)0};
#pragma unroll
        for (int j = 0; j < 16; ++j) t = t + sw[w][r][16 * h + j];
        acc[c] = acc[c] + t;
      }
      __syncwarp();
    }
  }
  q = warp_sum(q);
  if (lane == 0) mQ[g] = q;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const R re = acc[c].x + __shfl_xor_sync(0xffffffffu, acc[c].x, 16);
    const R im = acc[c].y + __shfl_xor_sync(0xffffffffu, acc[c].y, 16);
    const int k = 1 + c * KC + lane;
    if (lane < KC && k <= p) {
      const R inv = (R)(-1.0) / (R)k;
      ma[g * a.P + (k - 1)] = {re * inv, im * inv};
    }
  }
}

// H lanes per parent cell (the launcher uses a whole warp, H = 32); lane i of
// the group owns output coefficients i+1 and i+1+H.
template <typename R, int H>
__global__ void __launch_bounds__(32 * WPB)
k_m2m(ExpandArgs a, Geo g, int level, int64_t first, int64_t count, const int *__restrict__ map,
      const uint32_t *__restrict__ cell_key, const uint8_t *__restrict__ cell_cls,
      const uint8_t *__restrict__ cell_hsrc, const Cx<R> *__restrict__ ops,
      double *__restrict__ mQ, Cx<R> *__restrict__ ma) {
  constexpr int CPW = 32 / H;
  __shared__ Cx<R> sh[WPB * CPW][MAXP + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int li = lane % H, sub = lane / H, slot = w * CPW + sub;
  const unsigned mask = H == 32 ? 0xffffffffu : (0xffffu << (16 * sub));
  const int64_t ci = (blockIdx.x * (int64_t)WPB + w) * CPW + sub;
  if (ci >= count) return;
  const int64_t gp = first + ci;
  if (a.child_first && a.child_cnt[gp] == 0) return;   // adaptive leaf: keeps its P2M
  const int p = a.p, P1 = p + 1;
  Cx<R> acc0 = {(R)0, (R)0}, acc1 = {(R)0, (R)0};
  double Q = 0.0;
  if (cell_hsrc[gp]) {
    const uint32_t key = cell_key[gp];
    const int nch = a.child_first ? (int)a.child_cnt[gp] : g.b;
    for (int d = 0; d < nch; ++d) {
      int cs = a.child_first ? a.child_first[gp] + d
                             : map[g.map_off[level + 1] + (int64_t)key * g.b + d];
      if (cs < 0 || !cell_hsrc[cs]) continue;
      const double Qc = mQ[cs];
      for (int k = li; k < p; k += H) sh[slot][k + 1] = ma[(int64_t)cs * a.P + k];
      __syncwarp(mask);
      const Cx<R> *op = ops + (int64_t)cell_cls[cs] * P1 * P1;
      const R qc = (R)Qc;
#pragma unroll
      for (int h = 0; h < 64 / H; ++h) {
        const int l = li + 1 + H * h;
        if (l > p) break;
        const Cx<R> *row = op + (int64_t)l * P1;
        Cx<R> s = qc * row[0];
        for (int k = 1; k <= l; ++k) cfma(s, row[k], sh[slot][k]);
        if (h == 0) acc0 = acc0 + s; else acc1 = acc1 + s;
      }
      Q += Qc;
      __syncwarp(mask);
    }
  }
  if (li == 0) mQ[gp] = Q;
  if (li + 1 <= p) ma[gp * a.P + li] = acc0;
  if (li + 1 + H <= p) ma[gp * a.P + li + H] = acc1;
}

// H lanes per target cell (the launcher uses H = 32); lane i of the group owns
// local coefficients i and i+H.
template <typename R, int H>
__global__ void __launch_bounds__(32 * WPB)
k_m2l(ExpandArgs a, int64_t first, int64_t count, const int64_t *__restrict__ lev_first,
      const double *__restrict__ log_abs_scale, const int *__restrict__ far_cnt,
      const int *__restrict__ far_src, const uint16_t *__restrict__ far_op,
      const Cx<R> *__restrict__ ops, const double *__restrict__ logz, const double *__restrict__ mQ,
      const Cx<R> *__restrict__ ma, double *__restrict__ lL0, Cx<R> *__restrict__ lb) {
  constexpr int CPW = 32 / H;
  __shared__ Cx<R> sh[WPB * CPW][MAXP + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int li = lane % H, sub = lane / H, slot = w * CPW + sub;
  const unsigned mask = H == 32 ? 0xffffffffu : (0xffffu << (16 * sub));
  const int64_t fi = (blockIdx.x * (int64_t)WPB + w) * CPW + sub;
  if (fi >= count) return;
  const int64_t gt = first + fi;
  int l = a.l_min;
  while (l < a.L && gt >= lev_first[l + 1]) ++l;
  const double ls = log_abs_scale[l];
  const int p = a.p, P1 = p + 1;
  Cx<R> acc0 = {(R)0, (R)0}, acc1 = {(R)0, (R)0};
  double L0 = 0.0;
  const int n = far_cnt[fi];
  for (int e = 0; e < n; ++e) {
    const int s = far_src[fi * FAR_MAX + e];
    const int op = far_op[fi * FAR_MAX + e];
    const double Qs = mQ[s];
    for (int k = li; k < p; k += H) sh[slot][k + 1] = ma[(int64_t)s * a.P + k];
    __syncwarp(mask);
    const Cx<R> *T = ops + (int64_t)op * P1 * P1;
    const R qs = (R)Qs;
#pragma unroll
    for (int h = 0; h < 64 / H; ++h) {
      const int ll = li + H * h;
      if (ll > p) break;
      const Cx<R> *row = T + (int64_t)ll * P1;
      Cx<R> t = qs * row[0];
      for (int k = 1; k <= p; ++k) cfma(t, row[k], sh[slot][k]);
      if (h == 0) acc0 = acc0 + t; else acc1 = acc1 + t;
    }
    if (li == 0) L0 += Qs * (ls + logz[op]);
    __syncwarp(mask);
  }
  if (li == 0) lL0[gt] = L0 + (double)acc0.x;
  if (li >= 1 && li <= p) lb[gt * a.P + li - 1] = acc0;
  if (li + H <= p) lb[gt * a.P + li + H - 1] = acc1;
}

// H lanes per child cell (the launcher uses H = 32); adds the shifted parent
// local; lane i of the group owns coefficients i and i+H.
template <typename R, int H>
__global__ void __launch_bounds__(32 * WPB)
k_l2l(ExpandArgs a, Geo g, int level, int64_t first, int64_t count, const int *__restrict__ map,
      const uint32_t *__restrict__ cell_key, const uint8_t *__restrict__ cell_cls,
      const Cx<R> *__restrict__ ops, double *__restrict__ lL0, Cx<R> *__restrict__ lb) {
  constexpr int CPW = 32 / H;
  __shared__ Cx<R> sh[WPB * CPW][MAXP + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int li = lane % H, sub = lane / H, slot = w * CPW + sub;
  const unsigned mask = H == 32 ? 0xffffffffu : (0xffffu << (16 * sub));
  const int64_t ci = (blockIdx.x * (int64_t)WPB + w) * CPW + sub;
  if (ci >= count) return;
  const int64_t gc = first + ci;
  int ps;
  if (a.parent) {
    ps = a.parent[gc];
  } else {
    const uint32_t key = cell_key[gc];
    const uint32_t pkey = (g.tiling == FMM2D_SEPT) ? key / 7u : key >> 2;
    ps = map[g.map_off[level - 1] + pkey];
  }
  const int p = a.p, P1 = p + 1;
  for (int k = li; k < p; k += H) sh[slot][k + 1] = lb[(int64_t)ps * a.P + k];
  __syncwarp(mask);
  const Cx<R> *U = ops + (int64_t)cell_cls[gc] * P1 * P1;
#pragma unroll
  for (int h = 0; h < 64 / H; ++h) {
    const int k = li + H * h;
    if (k > p) break;
    const Cx<R> *row = U + (int64_t)k * P1;
    Cx<R> s = {(R)0, (R)0};
    for (int l = (k > 1 ? k : 1); l <= p; ++l) cfma(s, row[l], sh[slot][l]);
    if (k == 0) {
      lL0[gc] += lL0[ps] + (double)s.x;
    } else {
      Cx<R> cur = lb[gc * a.P + k - 1];
      lb[gc * a.P + k - 1] = cur + s;
    }
  }
}

// One warp per leaf; evaluates the local expansion at its targets and writes
// far + near potentials in the caller's target order.
template <typename R>
__global__ void __launch_bounds__(32 * WPB)
k_l2p(ExpandArgs a, const R *__restrict__ tgt, int tstride, const int *__restrict__ start,
      const int *__restrict__ end, const uint32_t *__restrict__ perm, const double *__restrict__ lL0,
      const Cx<R> *__restrict__ lb, const double *__restrict__ phi_near,
      double *__restrict__ phi_far, double *__restrict__ out) {
  __shared__ Cx<R> sh[WPB][MAXP + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t li = blockIdx.x * (int64_t)WPB + w;
  if (li >= a.n_leaves) return;
  const int64_t g = a.leaf_ids ? (int64_t)a.leaf_ids[li] : a.leaf_first + li;
  const int s = start[g], e = end[g];
  if (s >= e) return;
  const int p = a.p;
  for (int k = lane; k < p; k += 32) sh[w][k + 1] = lb[g * a.P + k];
  __syncwarp();
  const double L0 = lL0[g];
  Cx<R> is = {(R)a.inv_s_re, (R)a.inv_s_im};
  if (a.leaf_ids) {
    const double2 v = a.inv_scale[a.cell_lev[g]];
    is = {(R)v.x, (R)v.y};
  }
  for (int j = s + lane; j < e; j += 32) {
    const R *pt = tgt + (int64_t)j * tstride;
    Cx<R> z = Cx<R>{pt[0], pt[1]} * is;
    Cx<R> acc = sh[w][p];
    for (int l = p - 1; l >= 1; --l) acc = acc * z + sh[w][l];
    acc = acc * z;
    double far = L0 + (double)acc.x;
    phi_far[j] = far;
    out[perm[j]] = far + phi_near[j];
  }
}

inline unsigned wblocks(int64_t n) { return (unsigned)((n + WPB - 1) / WPB); }

}  // namespace

template <typename R>
cudaError_t launch_gather_u(const void *u, bool f32_in, const uint32_t *perm, int64_t n, R *src4,
                            cudaStream_t s, bool lo) {
  if (n <= 0) return cudaSuccess;
  k_gather_u<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(u, f32_in ? 1 : 0, perm, n, src4,
                                                            lo ? 1 : 0);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_p2m(const ExpandArgs &a, const R *src4, const int *start, const int *end,
                       double *mQ, Cx<R> *ma, cudaStream_t s) {
  if (a.n_leaves <= 0) return cudaSuccess;
  if constexpr (sizeof(R) == 8) {   // FP64: the powers-per-point form
    k_p2m_t<R><<<wblocks(a.n_leaves), 32 * WPB, 0, s>>>(a, src4, start, end, mQ, ma);
  } else {
    k_p2m<R, 8><<<wblocks(a.n_leaves), 32 * WPB, 0, s>>>(a, src4, start, end, mQ, ma);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_m2m(const ExpandArgs &a, const Geo &g, int level, int64_t first, int64_t count,
                       const int *map, const uint32_t *cell_key, const uint8_t *cell_cls,
                       const uint8_t *cell_hsrc, const Cx<R> *ops, double *mQ, Cx<R> *ma,
                       cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  // a whole warp per cell: measured faster than two cells per warp (H = 16)
  // even when half the lanes idle (p < 16)
  k_m2m<R, 32><<<wblocks(count), 32 * WPB, 0, s>>>(a, g, level, first, count, map, cell_key,
                                                    cell_cls, cell_hsrc, ops, mQ, ma);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_m2l(const ExpandArgs &a, int64_t first, int64_t count, const int64_t *lev_first,
                       const double *log_abs_scale, int64_t, const int *far_cnt, const int *far_src,
                       const uint16_t *far_op, const Cx<R> *ops, const double *logz,
                       const double *mQ, const Cx<R> *ma, double *lL0, Cx<R> *lb, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_m2l<R, 32><<<wblocks(count), 32 * WPB, 0, s>>>(a, first, count, lev_first, log_abs_scale,
                                                    far_cnt, far_src, far_op, ops, logz, mQ, ma,
                                                    lL0, lb);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_l2l(const ExpandArgs &a, const Geo &g, int level, int64_t first, int64_t count,
                       const int *map, const uint32_t *cell_key, const uint8_t *cell_cls,
                       const Cx<R> *ops, double *lL0, Cx<R> *lb, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_l2l<R, 32><<<wblocks(count), 32 * WPB, 0, s>>>(a, g, level, first, count, map, cell_key,
                                                    cell_cls, ops, lL0, lb);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_l2p(const ExpandArgs &a, const R *tgt, int tstride, const int *start,
                       const int *end, const uint32_t *perm, const double *lL0, const Cx<R> *lb,
                       const double *phi_near, double *phi_far, double *out, cudaStream_t s) {
  if (a.n_leaves <= 0) return cudaSuccess;
  k_l2p<R><<<wblocks(a.n_leaves), 32 * WPB, 0, s>>>(a, tgt, tstride, start, end, perm, lL0, lb,
                                                      phi_near, phi_far, out);
  return cudaGetLastError();
}

#define INST(R)                                                                                   \
  template cudaError_t launch_gather_u<R>(const void *, bool, const uint32_t *, int64_t, R *,      \
                                          cudaStream_t, bool);                                    \
  template cudaError_t launch_p2m<R>(const ExpandArgs &, const R *, const int *, const int *,      \
                                     double *, Cx<R> *, cudaStream_t);                            \
  template cudaError_t launch_m2m<R>(const ExpandArgs &, const Geo &, int, int64_t, int64_t,       \
                                     const int *, const uint32_t *, const uint8_t *,              \
                                     const uint8_t *, const Cx<R> *, double *, Cx<R> *,           \
                                     cudaStream_t);                                               \
  template cudaError_t launch_m2l<R>(const ExpandArgs &, int64_t, int64_t, const int64_t *,        \
                                     const double *, int64_t, const int *, const int *,           \
                                     const uint16_t *, const Cx<R> *, const double *,             \
                                     const double *, const Cx<R> *, double *, Cx<R> *,            \
                                     cudaStream_t);                                               \
  template cudaError_t launch_l2l<R>(const ExpandArgs &, const Geo &, int, int64_t, int64_t,       \
                                     const int *, const uint32_t *, const uint8_t *,              \
                                     const Cx<R> *, double *, Cx<R> *, cudaStream_t);             \
  template cudaError_t launch_l2p<R>(const ExpandArgs &, const R *, int, const int *, const int *, \
                                     const uint32_t *, const double *, const Cx<R> *,             \
                                     const double *, double *, double *, cudaStream_t);
INST(float)
INST(double)

}  // namespace fmm2d
