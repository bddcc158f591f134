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
// FP32 P2M for p <= PM: one warp per leaf; each lane sums u z^k for
// k = 1 .. p over its points with the powers formed once per point, then a
// butterfly reduce-scatter over the warp (16 + 8 + 4 + 2 + 1 shuffles of
// halving vectors) leaves lane l with float slot l (PM = 16: Re / Im of
// coefficient l / 2 + 1) or slots 2l, 2l + 1 (PM = 32: coefficient l + 1).
template <int PM>
__global__ void __launch_bounds__(32 * WPB)
k_p2m_bf(ExpandArgs a, const float *__restrict__ src4, const int *__restrict__ start,
         const int *__restrict__ end, double *__restrict__ mQ, Cx<float> *__restrict__ ma) {
  constexpr int NV = 2 * PM;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t li = blockIdx.x * (int64_t)WPB + (threadIdx.x >> 5);
  if (li >= a.n_leaves) return;
  const int64_t g = a.leaf_ids ? (int64_t)a.leaf_ids[li] : a.leaf_first + li;
  const int s = start[g], e = end[g];
  Cx<float> is = {(float)a.inv_s_re, (float)a.inv_s_im};
  if (a.leaf_ids) {
    const double2 v = a.inv_scale[a.cell_lev[g]];
    is = {(float)v.x, (float)v.y};
  }
  const int p = a.p;
  float v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.f;
  double q = 0.0;
  for (int i = s + lane; i < e; i += 32) {
    const float4 pt = reinterpret_cast<const float4 *>(src4)[i];
    const Cx<float> z = Cx<float>{pt.x, pt.y} * is;
    Cx<float> w = {pt.z, 0.f};
    q += (double)pt.z;
#pragma unroll
    for (int k = 0; k < PM; ++k) {
      if (k < p) {
        w = w * z;
        v[2 * k] += w.x;
        v[2 * k + 1] += w.y;
      }
    }
  }
  q = warp_sum(q);
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int o = 16 >> r, m = NV >> r;   // partner distance, current length
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < m / 2; ++i) {
      const float send = up ? v[i] : v[i + m / 2];
      const float keep = up ? v[i + m / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(FULL, send, o);
    }
  }
  if (lane == 0) mQ[g] = q;
  if (PM == 16) {
    const int k = lane >> 1;
    if (k < p) {
      const float inv = -1.f / (float)(k + 1);
      reinterpret_cast<float *>(ma)[(g * a.P + k) * 2 + (lane & 1)] = v[0] * inv;
    }
  } else {
    const int k = lane;
    if (k < p) {
      const float inv = -1.f / (float)(k + 1);
      ma[g * a.P + k] = Cx<float>{v[0] * inv, v[1] * inv};
    }
  }
}

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

// A warp per parent cell, the warps of the grid striding over the level
// (the block stages the operator table once for all its cells); lane i owns
// output coefficients i+1 and i+33.  Every child's slot, charge, class and
// multipole is fetched before any arithmetic, so a cell costs about three
// dependent loads (the parent's fields, the child slots, the child data)
// rather than three per child; the children are then applied in child order.
template <typename R>
__global__ void __launch_bounds__(32 * WPB)
k_m2m(ExpandArgs a, Geo g, int level, int64_t first, int64_t count, const int *__restrict__ map,
      const uint32_t *__restrict__ cell_key, const uint8_t *__restrict__ cell_cls,
      const uint8_t *__restrict__ cell_hsrc, const Cx<R> *__restrict__ ops, int n_staged,
      double *__restrict__ mQ, Cx<R> *__restrict__ ma) {
  constexpr int NB = 7;                        // children of a cell, at most
  constexpr int NLD = (NB * MAXP + 31) / 32;   // multipole loads per lane, at most
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ Cx<R> sh[WPB][NB][MAXP + 1];
  extern __shared__ __align__(16) unsigned char dyn_ops[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = a.p, P1 = p + 1;
  const Cx<R> *op_tab = ops;
  if (n_staged > 0) {   // the operators in shared memory: every child reads them
    Cx<R> *so = reinterpret_cast<Cx<R> *>(dyn_ops);
    for (int i = threadIdx.x; i < n_staged; i += blockDim.x) so[i] = ops[i];
    __syncthreads();
    op_tab = so;
  }
  const int64_t stride = (int64_t)gridDim.x * WPB;
  for (int64_t ci = blockIdx.x * (int64_t)WPB + w; ci < count; ci += stride) {
    const int64_t gp = first + ci;
    const bool hs = cell_hsrc[gp];
    int nch = 0, cs = -1;
    if (a.child_first) {
      nch = a.child_cnt[gp];
      if (nch == 0) continue;                  // adaptive leaf: keeps its P2M (warp-uniform)
      if (!hs) nch = 0;
      if (lane < nch) cs = a.child_first[gp] + lane;
    } else {
      const uint32_t key = cell_key[gp];
      nch = g.b;
      if (lane < nch) cs = map[g.map_off[level + 1] + (int64_t)key * g.b + lane];
      if (!hs) {
        nch = 0;
        cs = -1;
      }
    }
    // lane d < nch: child d's flag, charge and class
    int use = 0, cls = 0;
    double Qc = 0.0;
    if (cs >= 0) {
      use = cell_hsrc[cs];
      Qc = mQ[cs];
      cls = cell_cls[cs];
    }
    // all lanes: the children's multipoles, entry idx = d p + k
    Cx<R> v[NLD];
    const int nv = nch * p;
#pragma unroll
    for (int r = 0; r < NLD; ++r) {
      const int idx = lane + 32 * r;
      const int d = min(idx / max(p, 1), 31);
      const int cd = __shfl_sync(FULL, cs, d);
      v[r] = Cx<R>{(R)0, (R)0};
      if (idx < nv && cd >= 0) v[r] = ma[(int64_t)cd * a.P + (idx - d * p)];
    }
#pragma unroll
    for (int r = 0; r < NLD; ++r) {
      const int idx = lane + 32 * r;
      if (idx < nv) {
        const int d = idx / p;
        sh[w][d][idx - d * p + 1] = v[r];
      }
    }
    __syncwarp();
    Cx<R> acc0 = {(R)0, (R)0}, acc1 = {(R)0, (R)0};
    double Q = 0.0;
    for (int d = 0; d < nch; ++d) {
      const int ud = __shfl_sync(FULL, use, d);
      const double qd = __shfl_sync(FULL, Qc, d);
      const int kd = __shfl_sync(FULL, cls, d);
      if (!ud) continue;                       // warp-uniform
      const Cx<R> *op = op_tab + (int64_t)kd * P1 * P1;
      const R q = (R)qd;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int l = lane + 1 + 32 * h;
        if (l > p) break;
        const Cx<R> *row = op + (int64_t)l * P1;
        Cx<R> s = q * row[0];
        for (int k = 1; k <= l; ++k) cfma(s, row[k], sh[w][d][k]);
        if (h == 0) acc0 = acc0 + s; else acc1 = acc1 + s;
      }
      Q += qd;
    }
    if (lane == 0) mQ[gp] = Q;
    if (lane + 1 <= p) ma[gp * a.P + lane] = acc0;
    if (lane + 33 <= p) ma[gp * a.P + lane + 32] = acc1;
    __syncwarp();   // sh[w] is rewritten by the next cell
  }
}

// Uniform tree, the whole upward pass in one launch.  A warp takes a cell of
// level L-1 (its children are leaves, done by the P2M), forms its multipole,
// and then announces it to the parent: after a device-scope fence it adds
// one to the parent's arrival counter, and the warp that brings the count to
// the parent's number of occupied children goes on with the parent (whose
// children are then all written), up to level l_min.  Each cell is computed
// once, by one warp, with its children in child order, so the result is the
// one of the level-by-level form; no warp waits for another.  Multipoles
// written in this launch are read through L2 (ld.global.cg).
template <typename R, bool STAGED>
__global__ void __launch_bounds__(32 * WPB)
k_m2m_up(ExpandArgs a, Geo g, int l_min, int64_t first, int64_t count,
         const int *__restrict__ map, const uint32_t *__restrict__ cell_key,
         const uint8_t *__restrict__ cell_cls, const uint8_t *__restrict__ cell_hsrc,
         const Cx<R> *__restrict__ ops, int n_staged, double *mQ, Cx<R> *ma,
         int *__restrict__ arrive) {
  constexpr int NB = 7;                        // children of a cell, at most
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ Cx<R> sh[WPB][NB][MAXP + 1];
  extern __shared__ __align__(16) unsigned char dyn_ops[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t ci = blockIdx.x * (int64_t)WPB + w;
  const int p = a.p, P1 = p + 1;
  Cx<R> *so = reinterpret_cast<Cx<R> *>(dyn_ops);
  if (STAGED) {   // the operators in shared memory: every cell reads them
    for (int i = threadIdx.x; i < n_staged; i += blockDim.x) so[i] = ops[i];
    __syncthreads();
  }
  const Cx<R> *op_tab = STAGED ? so : ops;
  if (ci >= count) return;
  int64_t gp = first + ci;
  int level = a.L - 1;
  for (;;) {
    // the cell's fields and its children's slots
    const bool hs = cell_hsrc[gp];
    const uint32_t key = cell_key[gp];
    const int nch = hs ? g.b : 0;
    int cs = -1;
    if (lane < nch) cs = map[g.map_off[level + 1] + (int64_t)key * g.b + lane];
    int use = 0, cls = 0;
    double Qc = 0.0;
    if (cs >= 0) {
      use = cell_hsrc[cs];
      Qc = __ldcg(&mQ[cs]);
      cls = cell_cls[cs];
    }
    // lane k: coefficient k (and k + 32) of every child, loaded together
    Cx<R> v0[NB], v1[NB];
#pragma unroll
    for (int d = 0; d < NB; ++d) {
      const int cd = __shfl_sync(FULL, cs, d);
      v0[d] = v1[d] = Cx<R>{(R)0, (R)0};
      if (d < nch && cd >= 0) {
        const R *src = reinterpret_cast<const R *>(&ma[(int64_t)cd * a.P]);
        if (lane < p) v0[d] = Cx<R>{__ldcg(src + 2 * lane), __ldcg(src + 2 * lane + 1)};
        if (lane + 32 < p) v1[d] = Cx<R>{__ldcg(src + 2 * lane + 64), __ldcg(src + 2 * lane + 65)};
      }
    }
    __syncwarp();
#pragma unroll
    for (int d = 0; d < NB; ++d) {
      if (d < nch) {
        if (lane < p) sh[w][d][lane + 1] = v0[d];
        if (lane + 32 < p) sh[w][d][lane + 33] = v1[d];
      }
    }
    __syncwarp();
    Cx<R> acc0 = {(R)0, (R)0}, acc1 = {(R)0, (R)0};
    double Q = 0.0;
    for (int d = 0; d < nch; ++d) {
      const int ud = __shfl_sync(FULL, use, d);
      const double qd = __shfl_sync(FULL, Qc, d);
      const int kd = __shfl_sync(FULL, cls, d);
      if (!ud) continue;                         // warp-uniform
      const Cx<R> *op = op_tab + (int64_t)kd * P1 * P1;
      const R q = (R)qd;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int l = lane + 1 + 32 * h;
        if (l > p) break;
        const Cx<R> *row = op + (int64_t)l * P1;
        Cx<R> s = q * row[0];
#pragma unroll 4
        for (int k = 1; k <= l; ++k) cfma(s, row[k], sh[w][d][k]);
        if (h == 0) acc0 = acc0 + s; else acc1 = acc1 + s;
      }
      Q += qd;
    }
    if (lane == 0) mQ[gp] = Q;
    if (lane + 1 <= p) ma[gp * a.P + lane] = acc0;
    if (lane + 33 <= p) ma[gp * a.P + lane + 32] = acc1;
    if (level <= l_min) break;
    // announce the cell to its parent; the last of the occupied siblings
    // goes on with the parent
    const uint32_t pkey = (g.tiling == FMM2D_SEPT) ? key / 7u : key >> 2;
    const bool sib = lane < g.b && map[g.map_off[level] + (int64_t)pkey * g.b + lane] >= 0;
    const int nsib = __popc(__ballot_sync(FULL, sib));
    const int ps = map[g.map_off[level - 1] + pkey];
    __threadfence();
    __syncwarp();
    int old = 0;
    if (lane == 0) old = atomicAdd(&arrive[ps], 1);
    old = __shfl_sync(FULL, old, 0);
    if (old != nsib - 1) break;
    __threadfence();   // the siblings' multipoles, announced before their arrivals
    gp = ps;
    --level;
  }
}

// Uniform tree, the downward pass of levels l_min+1 .. L in one launch: a
// persistent grid of warps takes the cells in slot order, i.e. by (level,
// key), from a counter, so a cell's parent was taken earlier by a warp that
// is running; the warp waits for the parent's ready word (bounded: after
// about 2^22 polls it sets bit 2 of *err and goes on), adds the shifted
// parent local to the cell's own (M2L) local, and sets the cell's ready word.
// Each cell is computed once, as in the level-by-level form.  Locals written
// in this launch are read through L2 (ld.global.cg).
template <typename R, bool STAGED>
__global__ void __launch_bounds__(32 * WPB)
k_l2l_down(ExpandArgs a, Geo g, int64_t first, int64_t total, int64_t fixed_end,
           const int64_t *__restrict__ lev_first, const int *__restrict__ map,
           const uint32_t *__restrict__ cell_key, const uint8_t *__restrict__ cell_cls,
           const Cx<R> *__restrict__ ops, int n_staged, double *lL0, Cx<R> *lb, int *ready,
           int *ctr, int *err) {
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ Cx<R> sh[WPB][MAXP + 1];
  extern __shared__ __align__(16) unsigned char dyn_ops[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = a.p, P1 = p + 1;
  const int k0 = lane, k1 = lane + 32;
  Cx<R> *so = reinterpret_cast<Cx<R> *>(dyn_ops);
  if (STAGED) {   // the operators in shared memory: every cell reads them
    for (int i = threadIdx.x; i < n_staged; i += blockDim.x) so[i] = ops[i];
    __syncthreads();
  }
  const Cx<R> *op_tab = STAGED ? so : ops;
  for (;;) {
    int64_t idx = 0;
    if (lane == 0) idx = atomicAdd(reinterpret_cast<unsigned long long *>(ctr), 1ull);
    idx = __shfl_sync(FULL, idx, 0);
    if (idx >= total) break;
    const int64_t gc = first + idx;
    int level = a.l_min + 1;
    while (level < a.L && gc >= lev_first[level + 1]) ++level;
    // the cell's own fields
    const int cls = cell_cls[gc];
    Cx<R> own0 = {(R)0, (R)0}, own1 = {(R)0, (R)0};
    double L0 = 0.0;
    if (k0 == 0) L0 = lL0[gc];
    else if (k0 <= p) own0 = lb[gc * a.P + k0 - 1];
    if (k1 <= p) own1 = lb[gc * a.P + k1 - 1];
    const uint32_t key = cell_key[gc];
    const uint32_t pkey = (g.tiling == FMM2D_SEPT) ? key / 7u : key >> 2;
    const int ps = map[g.map_off[level - 1] + pkey];
    // the parent's final local (level l_min: its M2L local, final already)
    if (ps >= fixed_end) {
      bool ok = true;
      if (lane == 0) {
        const volatile int *rw = ready + ps;
        int polls = 0;
        while (*rw == 0) {
          if (++polls > (1 << 22)) {
            ok = false;
            break;
          }
          if (polls > 16) __nanosleep(64);
        }
        if (!ok) atomicOr(err, 2);
      }
      __syncwarp();
      __threadfence();
    }
    double Lp = 0.0;
    if (k0 == 0) Lp = __ldcg(&lL0[ps]);
    for (int k = lane; k < p; k += 32) {
      const R *src = reinterpret_cast<const R *>(&lb[(int64_t)ps * a.P + k]);
      sh[w][k + 1] = Cx<R>{__ldcg(src), __ldcg(src + 1)};
    }
    __syncwarp();
    const Cx<R> *U = op_tab + (int64_t)cls * P1 * P1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = h == 0 ? k0 : k1;
      if (k > p) break;
      const Cx<R> *row = U + (int64_t)k * P1;
      Cx<R> s = {(R)0, (R)0};
#pragma unroll 4
      for (int l = (k > 1 ? k : 1); l <= p; ++l) cfma(s, row[l], sh[w][l]);
      if (k == 0) lL0[gc] = L0 + (Lp + (double)s.x);
      else lb[gc * a.P + k - 1] = (h == 0 ? own0 : own1) + s;
    }
    // the cell's local is final: publish it
    __threadfence();
    __syncwarp();
    if (lane == 0) *reinterpret_cast<volatile int *>(ready + gc) = 1;
    __syncwarp();   // sh[w] is rewritten by the next cell
  }
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

// A warp per child cell, the warps of the grid striding over the level (the
// block stages the operator table once for all its cells); adds the shifted
// parent local in place; lane i owns coefficients i and i+32.  The cell's
// own local, its class and its parent slot are fetched together, then the
// parent's local.
template <typename R>
__global__ void __launch_bounds__(32 * WPB)
k_l2l(ExpandArgs a, Geo g, int level, int64_t first, int64_t count, const int *__restrict__ map,
      const uint32_t *__restrict__ cell_key, const uint8_t *__restrict__ cell_cls,
      const Cx<R> *__restrict__ ops, int n_staged, double *__restrict__ lL0,
      Cx<R> *__restrict__ lb) {
  __shared__ Cx<R> sh[WPB][MAXP + 1];
  extern __shared__ __align__(16) unsigned char dyn_ops[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = a.p, P1 = p + 1;
  const int k0 = lane, k1 = lane + 32;
  const Cx<R> *op_tab = ops;
  if (n_staged > 0) {   // the operators in shared memory: every cell reads them
    Cx<R> *so = reinterpret_cast<Cx<R> *>(dyn_ops);
    for (int i = threadIdx.x; i < n_staged; i += blockDim.x) so[i] = ops[i];
    __syncthreads();
    op_tab = so;
  }
  const int64_t stride = (int64_t)gridDim.x * WPB;
  for (int64_t ci = blockIdx.x * (int64_t)WPB + w; ci < count; ci += stride) {
    const int64_t gc = first + ci;
    // the cell's own fields
    const int cls = cell_cls[gc];
    Cx<R> own0 = {(R)0, (R)0}, own1 = {(R)0, (R)0};
    double L0 = 0.0;
    if (k0 == 0) L0 = lL0[gc];
    else if (k0 <= p) own0 = lb[gc * a.P + k0 - 1];
    if (k1 <= p) own1 = lb[gc * a.P + k1 - 1];
    int ps;
    if (a.parent) {
      ps = a.parent[gc];
    } else {
      const uint32_t key = cell_key[gc];
      const uint32_t pkey = (g.tiling == FMM2D_SEPT) ? key / 7u : key >> 2;
      ps = map[g.map_off[level - 1] + pkey];
    }
    // the parent's local
    double Lp = 0.0;
    if (k0 == 0) Lp = lL0[ps];
    for (int k = lane; k < p; k += 32) sh[w][k + 1] = lb[(int64_t)ps * a.P + k];
    __syncwarp();
    const Cx<R> *U = op_tab + (int64_t)cls * P1 * P1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = h == 0 ? k0 : k1;
      if (k > p) break;
      const Cx<R> *row = U + (int64_t)k * P1;
      Cx<R> s = {(R)0, (R)0};
      for (int l = (k > 1 ? k : 1); l <= p; ++l) cfma(s, row[l], sh[w][l]);
      if (k == 0) lL0[gc] = L0 + (Lp + (double)s.x);
      else lb[gc * a.P + k - 1] = (h == 0 ? own0 : own1) + s;
    }
    __syncwarp();   // sh[w] is rewritten by the next cell
  }
}

// One warp per leaf; evaluates the local expansion at its targets and writes
// far + near potentials in the caller's target order.
template <typename R>
__global__ void __launch_bounds__(32 * WPB)
k_l2p(ExpandArgs a, const R *__restrict__ tgt, int tstride, const int *__restrict__ start,
      const int *__restrict__ end, const uint32_t *__restrict__ perm, double *__restrict__ lL0,
      Cx<R> *__restrict__ lb, const double *__restrict__ phi_near,
      double *__restrict__ phi_far, double *__restrict__ out) {
  __shared__ Cx<R> sh[WPB][MAXP + 1];
  __shared__ Cx<R> shp[WPB][MAXP + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t li = blockIdx.x * (int64_t)WPB + w;
  if (li >= a.n_leaves) return;
  const int64_t g = a.leaf_ids ? (int64_t)a.leaf_ids[li] : a.leaf_first + li;
  const int s = start[g], e = end[g];
  const int p = a.p;
  double L0;
  if (a.l2l_map) {
    // the leaf's L2L: own (M2L) local + the parent's shifted final local
    const uint32_t key = a.l2l_key[g];
    const int ps = a.l2l_map[a.l2l_map_off + (a.l2l_sept ? key / 7u : key >> 2)];
    const int cls = a.l2l_cls[g];
    const int P1 = p + 1;
    for (int k = lane; k < p; k += 32) shp[w][k + 1] = lb[(int64_t)ps * a.P + k];
    double Lp = 0.0, Lown = 0.0;
    if (lane == 0) {
      Lp = lL0[ps];
      Lown = lL0[g];
    }
    __syncwarp();
    const Cx<R> *U = reinterpret_cast<const Cx<R> *>(a.l2l_ops) + (int64_t)cls * P1 * P1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h;
      if (k > p) break;
      const Cx<R> *row = U + (int64_t)k * P1;
      Cx<R> sv = {(R)0, (R)0};
#pragma unroll 4
      for (int l = (k > 1 ? k : 1); l <= p; ++l) cfma(sv, row[l], shp[w][l]);
      if (k == 0) {
        const double L = Lown + (Lp + (double)sv.x);
        lL0[g] = L;
        Lown = L;
      } else {
        const Cx<R> fin = lb[g * a.P + k - 1] + sv;
        lb[g * a.P + k - 1] = fin;
        sh[w][k] = fin;
      }
    }
    L0 = __shfl_sync(0xffffffffu, Lown, 0);
    __syncwarp();
  } else {
    if (s >= e) return;
    for (int k = lane; k < p; k += 32) sh[w][k + 1] = lb[g * a.P + k];
    __syncwarp();
    L0 = lL0[g];
  }
  if (s >= e) return;
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

// Entries of the M2M / L2L operator table a block stages in shared memory
// (0: the table stays in global memory): all of it when it fits beside the
// kernel's static shared memory within the 48 KB a launch gets by default.
template <typename R>
inline int staged_ops(const ExpandArgs &a, size_t static_bytes) {
  const int64_t n = (int64_t)a.n_cls * (a.p + 1) * (a.p + 1);
  return n > 0 && static_bytes + n * sizeof(Cx<R>) <= 48 * 1024 ? (int)n : 0;
}

}  // namespace

// ready: 2 + n_cells ints (a 64-bit counter, then a word per cell), zeroed here.
template <typename R>
cudaError_t launch_l2l_down(const ExpandArgs &a, const Geo &g, int64_t first, int64_t total,
                            const int64_t *lev_first_dev, const int *map, const uint32_t *cell_key,
                            const uint8_t *cell_cls, const Cx<R> *ops, double *lL0, Cx<R> *lb,
                            int *ready, int64_t n_cells, int sms, int *err, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ready, 0, (size_t)(n_cells + 2) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int n_st = staged_ops<R>(a, sizeof(Cx<R>) * WPB * (MAXP + 1));
  const unsigned blocks = (unsigned)std::min<int64_t>(wblocks(total), (int64_t)sms * 8);
  if (n_st > 0)
    k_l2l_down<R, true><<<blocks, 32 * WPB, n_st * sizeof(Cx<R>), s>>>(
        a, g, first, total, first, lev_first_dev, map, cell_key, cell_cls, ops, n_st, lL0, lb,
        ready + 2, ready, err);
  else
    k_l2l_down<R, false><<<blocks, 32 * WPB, 0, s>>>(
        a, g, first, total, first, lev_first_dev, map, cell_key, cell_cls, ops, 0, lL0, lb,
        ready + 2, ready, err);
  return cudaGetLastError();
}

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
  } else if (a.p <= 16) {
    k_p2m_bf<16><<<wblocks(a.n_leaves), 32 * WPB, 0, s>>>(a, src4, start, end, mQ, ma);
  } else if (a.p <= 32) {
    k_p2m_bf<32><<<wblocks(a.n_leaves), 32 * WPB, 0, s>>>(a, src4, start, end, mQ, ma);
  } else {
    k_p2m<R, 8><<<wblocks(a.n_leaves), 32 * WPB, 0, s>>>(a, src4, start, end, mQ, ma);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_m2m(const ExpandArgs &a, const Geo &g, int level, int64_t first, int64_t count,
                       const int *map, const uint32_t *cell_key, const uint8_t *cell_cls,
                       const uint8_t *cell_hsrc, const Cx<R> *ops, double *mQ, Cx<R> *ma, int sms,
                       cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int n_st = staged_ops<R>(a, sizeof(Cx<R>) * WPB * 7 * (MAXP + 1));
  const unsigned blocks = (unsigned)std::min<int64_t>(wblocks(count), (int64_t)std::max(sms, 1) * 8);
  k_m2m<R><<<blocks, 32 * WPB, n_st * sizeof(Cx<R>), s>>>(
      a, g, level, first, count, map, cell_key, cell_cls, cell_hsrc, ops, n_st, mQ, ma);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_m2m_up(const ExpandArgs &a, const Geo &g, int l_min, int64_t first, int64_t count,
                          const int *map, const uint32_t *cell_key, const uint8_t *cell_cls,
                          const uint8_t *cell_hsrc, const Cx<R> *ops, double *mQ, Cx<R> *ma,
                          int *arrive, int64_t n_cells, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(arrive, 0, (size_t)n_cells * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int n_st = staged_ops<R>(a, sizeof(Cx<R>) * WPB * 7 * (MAXP + 1));
  if (n_st > 0)
    k_m2m_up<R, true><<<wblocks(count), 32 * WPB, n_st * sizeof(Cx<R>), s>>>(
        a, g, l_min, first, count, map, cell_key, cell_cls, cell_hsrc, ops, n_st, mQ, ma, arrive);
  else
    k_m2m_up<R, false><<<wblocks(count), 32 * WPB, 0, s>>>(
        a, g, l_min, first, count, map, cell_key, cell_cls, cell_hsrc, ops, 0, mQ, ma, arrive);
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
                       const Cx<R> *ops, double *lL0, Cx<R> *lb, int sms, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int n_st = staged_ops<R>(a, sizeof(Cx<R>) * WPB * (MAXP + 1));
  const unsigned blocks = (unsigned)std::min<int64_t>(wblocks(count), (int64_t)std::max(sms, 1) * 8);
  k_l2l<R><<<blocks, 32 * WPB, n_st * sizeof(Cx<R>), s>>>(
      a, g, level, first, count, map, cell_key, cell_cls, ops, n_st, lL0, lb);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_l2p(const ExpandArgs &a, const R *tgt, int tstride, const int *start,
                       const int *end, const uint32_t *perm, double *lL0, Cx<R> *lb,
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
                                     const uint8_t *, const Cx<R> *, double *, Cx<R> *, int,      \
                                     cudaStream_t);                                               \
  template cudaError_t launch_l2l_down<R>(const ExpandArgs &, const Geo &, int64_t, int64_t,       \
                                          const int64_t *, const int *, const uint32_t *,         \
                                          const uint8_t *, const Cx<R> *, double *, Cx<R> *,      \
                                          int *, int64_t, int, int *, cudaStream_t);              \
  template cudaError_t launch_m2m_up<R>(const ExpandArgs &, const Geo &, int, int64_t, int64_t,    \
                                        const int *, const uint32_t *, const uint8_t *,           \
                                        const uint8_t *, const Cx<R> *, double *, Cx<R> *, int *, \
                                        int64_t, cudaStream_t);                                   \
  template cudaError_t launch_m2l<R>(const ExpandArgs &, int64_t, int64_t, const int64_t *,        \
                                     const double *, int64_t, const int *, const int *,           \
                                     const uint16_t *, const Cx<R> *, const double *,             \
                                     const double *, const Cx<R> *, double *, Cx<R> *,            \
                                     cudaStream_t);                                               \
  template cudaError_t launch_l2l<R>(const ExpandArgs &, const Geo &, int, int64_t, int64_t,       \
                                     const int *, const uint32_t *, const uint8_t *,              \
                                     const Cx<R> *, double *, Cx<R> *, int, cudaStream_t);        \
  template cudaError_t launch_l2p<R>(const ExpandArgs &, const R *, int, const int *, const int *, \
                                     const uint32_t *, double *, Cx<R> *,                         \
                                     const double *, double *, double *, cudaStream_t);
INST(float)
INST(double)

}  // namespace fmm2d
