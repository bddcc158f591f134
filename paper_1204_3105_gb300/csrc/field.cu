// field.cu - the field F_j = sum_{i : x_i != y_j} u_i / (y_j - x_i): the
// derivative of the complex potential of eq. 1 (Sec. 2).  It is single
// valued (the branch of the logarithm only moves the constant term), and the
// gradient of Re Phi is (Re F, -Im F).  The FMM gives it by differentiating
// the operators a target meets, on the same tree, lists and expansions as the
// potential:
//   P2P'  sum over the Near sources of u_i / (y - x_i)
//   M2P'  (adaptive W lists) Q / (y - c) - sum_k k a_k (y - c)^-(k+1)
//   L2P'  sum_{l>=1} l b_l (y - c)^(l-1)
// With scaled coefficients (a^_k = a_k / s^k, b^_l = b_l s^l) the last two
// are Horner sums in z = s / (y - c) and z = (y - c) / s.
#include "plan.h"

namespace fmm2d {

namespace {

constexpr int FTH = 256;   // threads per block; one warp per target leaf
constexpr int FWPB = 4;    // warps per block of the expansion kernels

template <typename R> struct FieldT;
template <> struct FieldT<float> {
  using V4 = float4;
  // r^2 is floored so that it never reaches 0; a coincident pair has
  // dx = dy = 0 and so contributes nothing (no separate test needed)
  static constexpr float floor_r2 = 1e-30f;
  static __device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
};
template <> struct FieldT<double> {
  using V4 = double4_32a;
  static constexpr double floor_r2 = 1e-300;
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
};

template <typename R>
__device__ __forceinline__ void f_kahan(R &s, R &c, R x) {
  const R y = x - c;
  const R t = s + y;
  c = (t - s) - y;
  s = t;
}

// Sources of one Near leaf against the lane's two targets (a, b), in that
// leaf's frame; partial sums of at most 64 sources go into compensated sums.
template <typename R>
__device__ __forceinline__ void field_leaf(const typename FieldT<R>::V4 *__restrict__ sp, int n,
                                           R ax, R ay, R bx, R by, R (&fa)[4], R (&fb)[4]) {
  using T = FieldT<R>;
  for (int i = 0; i < n; i += 64) {
    const int m = min(n - i, 64);
    R xa = 0, ya = 0, xb = 0, yb = 0;
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
      const typename T::V4 v = sp[i + j];
      const R dxa = ax - v.x, dya = ay - v.y, dxb = bx - v.x, dyb = by - v.y;
      // (u dx) / r^2: a coincident pair gives 0 * (1 / floor) = 0 whatever u
      const R ia = T::rcp(fma(dxa, dxa, fma(dya, dya, T::floor_r2)));
      const R ib = T::rcp(fma(dxb, dxb, fma(dyb, dyb, T::floor_r2)));
      xa = fma(v.z * dxa, ia, xa);
      ya = fma(v.z * dya, ia, ya);
      xb = fma(v.z * dxb, ib, xb);
      yb = fma(v.z * dyb, ib, yb);
    }
    f_kahan(fa[0], fa[1], xa);
    f_kahan(fa[2], fa[3], ya);
    f_kahan(fb[0], fb[1], xb);
    f_kahan(fb[2], fb[3], yb);
  }
}

// FP32 forms with the low parts of the leaf-relative coordinates: the pair
// differences are formed accurately.  A field term u / r has the absolute
// sensitivity u / r^2 to a coordinate error, so an FP32 coordinate rounded
// once (an error of half an ulp of the leaf size) would spoil close pairs.
// The target, shifted into the source leaf's frame by TwoSum (A_hi + A_lo),
// minus the source (s_hi + s_lo) is (A_hi - s_hi) + (A_lo - s_lo): the first
// difference is exact for close points (Sterbenz), so dx is the FP32
// rounding of the true difference and each term has FP32 relative accuracy.
__device__ __forceinline__ void ff_shift(float t_hi, float t_lo, double d, float &a_hi, float &a_lo) {
  const float dh = (float)d, dl = (float)(d - (double)dh);
  const float s = t_hi - dh;
  const float bp = s - t_hi;                    // TwoSum of t_hi and -dh
  const float err = (t_hi - (s - bp)) + (-dh - bp);
  a_hi = s;
  a_lo = err + (t_lo - dl);
}

__device__ __forceinline__ void field_leaf_acc(const float4 *__restrict__ sp,
                                               const float2 *__restrict__ sl, int n, float ax,
                                               float axl, float ay, float ayl, float bx, float bxl,
                                               float by, float byl, float (&fa)[4], float (&fb)[4]) {
  using T = FieldT<float>;
  for (int i = 0; i < n; i += 64) {
    const int m = min(n - i, 64);
    float xa = 0, ya = 0, xb = 0, yb = 0;
#pragma unroll 2
    for (int j = 0; j < m; ++j) {
      const float4 v = sp[i + j];
      const float2 w = sl[i + j];
      const float dxa = (ax - v.x) + (axl - w.x), dya = (ay - v.y) + (ayl - w.y);
      const float dxb = (bx - v.x) + (bxl - w.x), dyb = (by - v.y) + (byl - w.y);
      const float ia = T::rcp(fmaf(dxa, dxa, fmaf(dya, dya, T::floor_r2)));
      const float ib = T::rcp(fmaf(dxb, dxb, fmaf(dyb, dyb, T::floor_r2)));
      xa = fmaf(v.z * dxa, ia, xa);
      ya = fmaf(v.z * dya, ia, ya);
      xb = fmaf(v.z * dxb, ib, xb);
      yb = fmaf(v.z * dyb, ib, yb);
    }
    f_kahan(fa[0], fa[1], xa);
    f_kahan(fa[2], fa[3], ya);
    f_kahan(fb[0], fb[1], xb);
    f_kahan(fb[2], fb[3], yb);
  }
}

// P2P': one warp per target leaf, two targets per lane; the warp streams the
// sources of every Near leaf with broadcast loads.  u / (y - x) =
// u (dx - i dy) / r^2.  Writes fnear[j] (sorted target order).
template <typename R>
__global__ void __launch_bounds__(FTH)
k_p2p_field(int64_t leaf_first, int64_t n_leaves, const int *__restrict__ leaf_ids,
            const R *__restrict__ src4, const R *__restrict__ tgt, int tstride,
            const int *__restrict__ sst, const int *__restrict__ sen, const int *__restrict__ tst,
            const int *__restrict__ ten, const int *__restrict__ near_cnt,
            const int *__restrict__ near_off, const int *__restrict__ near_src,
            const double2 *__restrict__ ctr, double2 *__restrict__ fnear,
            const float2 *__restrict__ src_lo, const float2 *__restrict__ tgt_lo) {
  using T = FieldT<R>;
  const int lane = threadIdx.x & 31;
  const int64_t li = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (li >= n_leaves) return;
  const int64_t g = leaf_ids ? (int64_t)leaf_ids[li] : leaf_first + li;
  const int ts = tst[g], te = ten[g];
  if (ts >= te) return;
  const int nn = near_off ? near_off[li + 1] - near_off[li] : near_cnt[li];
  const int *nsrc = near_off ? near_src + near_off[li] : near_src + li * NEAR_MAX;
  const double2 cg = ctr[g];
  const typename T::V4 *src = reinterpret_cast<const typename T::V4 *>(src4);
  for (int t0 = ts; t0 < te; t0 += 64) {
    const int ia = t0 + lane, ib = t0 + 32 + lane;
    const int ja = ia < te ? ia : ts, jb = ib < te ? ib : ts;   // idle lanes repeat a target
    const R ax0 = tgt[(int64_t)ja * tstride], ay0 = tgt[(int64_t)ja * tstride + 1];
    const R bx0 = tgt[(int64_t)jb * tstride], by0 = tgt[(int64_t)jb * tstride + 1];
    R fa[4] = {0, 0, 0, 0}, fb[4] = {0, 0, 0, 0};   // (x sum, comp, y sum, comp)
    if constexpr (sizeof(R) == 4) {
      if (src_lo) {   // accurate differences from the hi + lo coordinates
        const float2 la = tgt_lo[ja], lb = tgt_lo[jb];
        for (int e = 0; e < nn; ++e) {
          const int s = nsrc[e];
          const int s0 = sst[s], cnt = sen[s] - s0;
          const double2 cs = ctr[s];
          float axh, axl, ayh, ayl, bxh, bxl, byh, byl;
          ff_shift(ax0, la.x, cs.x - cg.x, axh, axl);
          ff_shift(ay0, la.y, cs.y - cg.y, ayh, ayl);
          ff_shift(bx0, lb.x, cs.x - cg.x, bxh, bxl);
          ff_shift(by0, lb.y, cs.y - cg.y, byh, byl);
          field_leaf_acc(src + s0, src_lo + s0, cnt, axh, axl, ayh, ayl, bxh, bxl, byh, byl, fa, fb);
        }
      }
    }
    if (sizeof(R) == 8 || !src_lo) {
      for (int e = 0; e < nn; ++e) {
        const int s = nsrc[e];
        const int s0 = sst[s], cnt = sen[s] - s0;
        const double2 cs = ctr[s];
        const R dcx = (R)(cs.x - cg.x), dcy = (R)(cs.y - cg.y);
        field_leaf<R>(src + s0, cnt, ax0 - dcx, ay0 - dcy, bx0 - dcx, by0 - dcy, fa, fb);
      }
    }
    if (ia < te)
      fnear[ia] = make_double2((double)fa[0] - (double)fa[1], -((double)fa[2] - (double)fa[3]));
    if (ib < te)
      fnear[ib] = make_double2((double)fb[0] - (double)fb[1], -((double)fb[2] - (double)fb[3]));
  }
}

// M2P' (adaptive trees): one warp per target leaf adds, at each of its
// targets, the derivative of every W cell's multipole.
template <typename R>
__global__ void __launch_bounds__(32 * FWPB)
k_m2p_field(int64_t n_leaves, const int *__restrict__ leaf_ids, const int *__restrict__ w_off,
            const int *__restrict__ w_src, const R *__restrict__ tgt, int tstride,
            const int *__restrict__ ts_, const int *__restrict__ te_, const double2 *__restrict__ ctr,
            const uint8_t *__restrict__ lev, const double2 *__restrict__ scale, int p, int P,
            const double *__restrict__ mQ, const Cx<R> *__restrict__ ma, double2 *__restrict__ fnear) {
  __shared__ Cx<R> sh[FWPB][MAXP + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t li = blockIdx.x * (int64_t)FWPB + w;
  if (li >= n_leaves) return;
  const int a = leaf_ids[li];
  const int e0 = w_off[li], e1 = w_off[li + 1];
  if (e0 == e1) return;
  const int ts = ts_[a], te = te_[a];
  const double2 ca = ctr[a];
  for (int j0 = ts; j0 < te; j0 += 32) {
    const int j = j0 + lane;
    const bool act = j < te;
    const R tx = act ? tgt[(int64_t)j * tstride] : (R)0, ty = act ? tgt[(int64_t)j * tstride + 1] : (R)0;
    double fx = 0.0, fy = 0.0;
    for (int e = e0; e < e1; ++e) {
      const int cc = w_src[e];
      __syncwarp();
      for (int k = lane; k < p; k += 32) {
        const Cx<R> v = ma[(int64_t)cc * P + k];
        sh[w][k + 1] = {(R)(k + 1) * v.x, (R)(k + 1) * v.y};   // k a^_k
      }
      __syncwarp();
      const double2 c2 = ctr[cc];
      const double2 sc = scale[lev[cc]];
      const Cx<R> d = {(R)(ca.x - c2.x) + tx, (R)(ca.y - c2.y) + ty};
      const R den = d.x * d.x + d.y * d.y;
      const Cx<R> id = {d.x / den, -d.y / den};           // 1 / (y - c)
      const Cx<R> z = Cx<R>{(R)sc.x, (R)sc.y} * id;       // s_c / (y - c)
      Cx<R> h = sh[w][p];
      for (int k = p - 1; k >= 1; --k) h = h * z + sh[w][k];
      h = h * z;                                          // sum_k k a^_k z^k
      const Cx<R> f = id * Cx<R>{(R)mQ[cc] - h.x, -h.y};
      fx += (double)f.x;
      fy += (double)f.y;
    }
    if (act) {
      double2 v = fnear[j];
      fnear[j] = make_double2(v.x + fx, v.y + fy);
    }
  }
}

// L2P': one warp per leaf; far field from the leaf's local expansion plus the
// near part, written in the caller's target order as (Re F, Im F).
template <typename R>
__global__ void __launch_bounds__(32 * FWPB)
k_l2p_field(ExpandArgs a, const R *__restrict__ tgt, int tstride, const int *__restrict__ start,
            const int *__restrict__ end, const uint32_t *__restrict__ perm,
            const Cx<R> *__restrict__ lb, const double2 *__restrict__ fnear,
            double2 *__restrict__ out) {
  __shared__ Cx<R> sh[FWPB][MAXP + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t li = blockIdx.x * (int64_t)FWPB + w;
  if (li >= a.n_leaves) return;
  const int64_t g = a.leaf_ids ? (int64_t)a.leaf_ids[li] : a.leaf_first + li;
  const int s = start[g], e = end[g];
  if (s >= e) return;
  const int p = a.p;
  for (int k = lane; k < p; k += 32) {
    const Cx<R> v = lb[g * a.P + k];
    sh[w][k + 1] = {(R)(k + 1) * v.x, (R)(k + 1) * v.y};   // l b^_l
  }
  __syncwarp();
  Cx<R> is = {(R)a.inv_s_re, (R)a.inv_s_im};
  if (a.leaf_ids) {
    const double2 v = a.inv_scale[a.cell_lev[g]];
    is = {(R)v.x, (R)v.y};
  }
  for (int j = s + lane; j < e; j += 32) {
    const R *pt = tgt + (int64_t)j * tstride;
    const Cx<R> z = Cx<R>{pt[0], pt[1]} * is;
    Cx<R> acc = sh[w][p];
    for (int l = p - 1; l >= 1; --l) acc = acc * z + sh[w][l];
    acc = acc * is;                                      // d/dy: one factor 1/s
    const double2 nf = fnear[j];
    out[perm[j]] = make_double2(nf.x + (double)acc.x, nf.y + (double)acc.y);
  }
}

}  // namespace

template <typename R>
cudaError_t launch_p2p_field(int64_t leaf_first, int64_t n_leaves, const int *leaf_ids,
                             const R *src4, const R *tgt, int tstride, const int *src_start,
                             const int *src_end, const int *tgt_start, const int *tgt_end,
                             const int *near_cnt, const int *near_off, const int *near_src,
                             const double2 *ctr, double2 *fnear, cudaStream_t s,
                             const float2 *src_lo, const float2 *tgt_lo) {
  if (n_leaves <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n_leaves * 32 + FTH - 1) / FTH);
  k_p2p_field<R><<<blocks, FTH, 0, s>>>(leaf_first, n_leaves, leaf_ids, src4, tgt, tstride,
                                         src_start, src_end, tgt_start, tgt_end, near_cnt,
                                         near_off, near_src, ctr, fnear, src_lo, tgt_lo);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_m2p_field(int64_t n_leaves, const int *leaf_ids, const int *w_off,
                             const int *w_src, const R *tgt, int tstride, const int *ts,
                             const int *te, const double2 *ctr, const uint8_t *lev,
                             const double2 *scale, int p, int P, const double *mQ, const Cx<R> *ma,
                             double2 *fnear, cudaStream_t s) {
  if (n_leaves <= 0) return cudaSuccess;
  k_m2p_field<R><<<(unsigned)((n_leaves + FWPB - 1) / FWPB), 32 * FWPB, 0, s>>>(
      n_leaves, leaf_ids, w_off, w_src, tgt, tstride, ts, te, ctr, lev, scale, p, P, mQ, ma, fnear);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_l2p_field(const ExpandArgs &a, const R *tgt, int tstride, const int *start,
                             const int *end, const uint32_t *perm, const Cx<R> *lb,
                             const double2 *fnear, double2 *out, cudaStream_t s) {
  if (a.n_leaves <= 0) return cudaSuccess;
  k_l2p_field<R><<<(unsigned)((a.n_leaves + FWPB - 1) / FWPB), 32 * FWPB, 0, s>>>(
      a, tgt, tstride, start, end, perm, lb, fnear, out);
  return cudaGetLastError();
}

#define FIELD_INST(R)                                                                              \
  template cudaError_t launch_p2p_field<R>(int64_t, int64_t, const int *, const R *, const R *,    \
                                           int, const int *, const int *, const int *, const int *, \
                                           const int *, const int *, const int *, const double2 *, \
                                           double2 *, cudaStream_t, const float2 *,                \
                                           const float2 *);                                        \
  template cudaError_t launch_m2p_field<R>(int64_t, const int *, const int *, const int *,         \
                                           const R *, int, const int *, const int *,               \
                                           const double2 *, const uint8_t *, const double2 *, int, \
                                           int, const double *, const Cx<R> *, double2 *,          \
                                           cudaStream_t);                                          \
  template cudaError_t launch_l2p_field<R>(const ExpandArgs &, const R *, int, const int *,        \
                                           const int *, const uint32_t *, const Cx<R> *,           \
                                           const double2 *, double2 *, cudaStream_t);
FIELD_INST(float)
FIELD_INST(double)

}  // namespace fmm2d
