// p2p.cu - near-field direct sum (Sec. 2; the M(P2 s) term of App. A-C):
//   phi_near(y_j) = sum over the sources x_i of {leaf(y_j)} u Neighbors(leaf)
//                   of u_i log|y_j - x_i|,  skipping x_i == y_j.
// Two forms: one warp per target leaf (k_p2p) for small leaves, and a
// block-staged form (k_p2p_block) for large ones.  Points are stored relative to
// their leaf centre, so differences keep full precision.  The FP32 form takes
// log2(r^2) on the MUFU unit and scales by ln2/2 once per target; partial
// sums are kept in a compensated (Kahan) running sum.
#include "plan.h"

namespace fmm2d {

namespace {

constexpr int P2P_TH = 256;

template <typename R> struct P2PTraits;
template <> struct P2PTraits<float> {
  using V4 = float4;
  static constexpr double scale = 0.34657359027997264;   // ln2 / 2
  // log2(r^2); r^2 = 0 (a coincident pair) contributes nothing
  static __device__ __forceinline__ float lg(float r2) {
    float y;   // MUFU lg2; r^2 is never subnormal here (zero or >= the floor)
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
    return y;
  }
  static __device__ __forceinline__ float lg_checked(float r2) { return r2 > 0.f ? lg(r2) : 0.f; }
  static constexpr float floor_r2 = 1e-30f;
};
template <> struct P2PTraits<double> {
  using V4 = double4_32a;
  static constexpr double scale = 0.5;
  static __device__ __forceinline__ double lg_checked(double r2) { return r2 > 0.0 ? log(r2) : 0.0; }
  static __device__ __forceinline__ double lg(double r2) { return log(r2); }
  static constexpr double floor_r2 = 1e-300;
};

// Sum over staged sources q0, q0 + K, ... < q1 for two targets at once (each
// staged source is read once for two pairs).  Points of different leaves
// never coincide (equal coordinates give equal keys), so only the target's
// own leaf needs the r^2 > 0 test; elsewhere a tiny floor folded into the FMA
// keeps log2 finite at no extra instruction.  Partial sums of at most 64
// sources are added into a compensated (Kahan) running sum of the same type,
// which keeps the total accurate without the slow FP64 pipe.
template <typename R>
__device__ __forceinline__ void kahan_add(R &sum, R &comp, R x) {
  const R y = x - comp;
  const R t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

template <typename R, bool CHECK>
__device__ __forceinline__ void p2p_pair(const typename P2PTraits<R>::V4 &v, R ax, R ay, R bx, R by,
                                         R &acc_a, R &acc_b) {
  using T = P2PTraits<R>;
  const R dxa = ax - v.x, dya = ay - v.y;
  const R dxb = bx - v.x, dyb = by - v.y;
  if (CHECK) {
    acc_a += v.z * T::lg_checked(dxa * dxa + dya * dya);
    acc_b += v.z * T::lg_checked(dxb * dxb + dyb * dyb);
  } else {
    acc_a += v.z * T::lg(fma(dxa, dxa, fma(dya, dya, (R)T::floor_r2)));
    acc_b += v.z * T::lg(fma(dxb, dxb, fma(dyb, dyb, (R)T::floor_r2)));
  }
}

// One warp per target leaf, no shared memory and no block barriers: each
// lane holds two targets (t0 + lane, t0 + 32 + lane) and the warp streams
// the sources of every Near leaf with broadcast read-only loads.  The
// targets are shifted once per source leaf into that leaf's frame.
template <typename R, bool CHECK>
__device__ __forceinline__ void p2p_leaf(const typename P2PTraits<R>::V4 *__restrict__ sp, int n,
                                         R ax, R ay, R bx, R by, R (&sa)[2], R (&sb)[2]) {
  int i = 0;
  while (i < n) {
    const int m = min(n - i, 64);
    R acc_a = (R)0, acc_b = (R)0;
    int j = 0;
    for (; j + 4 <= m; j += 4) {
      const typename P2PTraits<R>::V4 v0 = sp[i + j], v1 = sp[i + j + 1];
      const typename P2PTraits<R>::V4 v2 = sp[i + j + 2], v3 = sp[i + j + 3];
      p2p_pair<R, CHECK>(v0, ax, ay, bx, by, acc_a, acc_b);
      p2p_pair<R, CHECK>(v1, ax, ay, bx, by, acc_a, acc_b);
      p2p_pair<R, CHECK>(v2, ax, ay, bx, by, acc_a, acc_b);
      p2p_pair<R, CHECK>(v3, ax, ay, bx, by, acc_a, acc_b);
    }
    for (; j < m; ++j) p2p_pair<R, CHECK>(sp[i + j], ax, ay, bx, by, acc_a, acc_b);
    kahan_add(sa[0], sa[1], acc_a);
    kahan_add(sb[0], sb[1], acc_b);
    i += m;
  }
}

template <typename R>
__global__ void __launch_bounds__(P2P_TH)
k_p2p(int64_t leaf_first, int64_t n_leaves, const R *__restrict__ src4, const R *__restrict__ tgt,
      int tstride, const int *__restrict__ sst, const int *__restrict__ sen,
      const int *__restrict__ tst, const int *__restrict__ ten, const int *__restrict__ near_cnt,
      const int *__restrict__ near_src, const double2 *__restrict__ ctr,
      double *__restrict__ phi_near) {
  using T = P2PTraits<R>;
  const int lane = threadIdx.x & 31;
  const int64_t li = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (li >= n_leaves) return;
  const int64_t g = leaf_first + li;
  const int ts = tst[g], te = ten[g];
  if (ts >= te) return;
  const int nn = near_cnt[li];
  const int *nsrc = near_src + li * NEAR_MAX;
  const double2 cg = ctr[g];
  const typename T::V4 *src = reinterpret_cast<const typename T::V4 *>(src4);
  for (int t0 = ts; t0 < te; t0 += 64) {
    const int ia = t0 + lane, ib = t0 + 32 + lane;
    const int ja = ia < te ? ia : ts, jb = ib < te ? ib : ts;   // idle lanes repeat a target
    const R ax0 = tgt[(int64_t)ja * tstride], ay0 = tgt[(int64_t)ja * tstride + 1];
    const R bx0 = tgt[(int64_t)jb * tstride], by0 = tgt[(int64_t)jb * tstride + 1];
    R sa[2] = {(R)0, (R)0}, sb[2] = {(R)0, (R)0};   // Kahan sum and compensation
    for (int e = 0; e < nn; ++e) {
      const int s = nsrc[e];
      const int s0 = sst[s], cnt = sen[s] - s0;
      const double2 cs = ctr[s];
      const R dcx = (R)(cs.x - cg.x), dcy = (R)(cs.y - cg.y);
      const R ax = ax0 - dcx, ay = ay0 - dcy, bx = bx0 - dcx, by = by0 - dcy;
      // points of different leaves never coincide: only the own leaf (listed
      // first by the Near stencils) needs the r^2 > 0 test
      if (s == (int)g) p2p_leaf<R, true>(src + s0, cnt, ax, ay, bx, by, sa, sb);
      else p2p_leaf<R, false>(src + s0, cnt, ax, ay, bx, by, sa, sb);
    }
    if (ia < te) phi_near[ia] = ((double)sa[0] - (double)sa[1]) * T::scale;
    if (ib < te) phi_near[ib] = ((double)sb[0] - (double)sb[1]) * T::scale;
  }
}

// Block-staged form for large leaves: one block per target leaf; the Near
// sources are staged once in shared memory (shifted into the target leaf's
// frame) and the block's threads are split into (target pair, source slice)
// so that every thread works whatever the leaf size; slice partials are
// summed in FP64 at the end.
constexpr int P2P_CAP = 2048;   // staged sources per chunk (FP32 form)

template <typename R, bool CHECK>
__device__ __forceinline__ void p2p_slice(const typename P2PTraits<R>::V4 *sp, int q0, int q1,
                                          int K, R ax, R ay, R bx, R by, R (&sa)[2],
                                          R (&sb)[2]) {
  int n = q1 > q0 ? (q1 - q0 + K - 1) / K : 0;
  const typename P2PTraits<R>::V4 *ptr = sp + q0;
  while (n > 0) {
    const int m = n < 64 ? n : 64;
    n -= m;
    R acc_a = (R)0, acc_b = (R)0;
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
      p2p_pair<R, CHECK>(*ptr, ax, ay, bx, by, acc_a, acc_b);
      ptr += K;
    }
    kahan_add(sa[0], sa[1], acc_a);
    kahan_add(sb[0], sb[1], acc_b);
  }
}

template <typename R>
__global__ void __launch_bounds__(P2P_TH)
k_p2p_block(int64_t leaf_first, const R *__restrict__ src4, const R *__restrict__ tgt, int tstride,
            const int *__restrict__ sst, const int *__restrict__ sen, const int *__restrict__ tst,
            const int *__restrict__ ten, const int *__restrict__ near_cnt,
            const int *__restrict__ near_src, const double2 *__restrict__ ctr,
            double *__restrict__ phi_near) {
  using T = P2PTraits<R>;
  constexpr int CAP = P2P_CAP * 4 / (int)sizeof(R);
  __shared__ typename T::V4 sp[CAP];
  __shared__ double red[P2P_TH], red2[P2P_TH];
  __shared__ int m_s0[NEAR_MAX], m_cnt[NEAR_MAX], m_base[NEAR_MAX + 1];
  __shared__ R m_dx[NEAR_MAX], m_dy[NEAR_MAX];
  const int tid = threadIdx.x;
  const int64_t li = blockIdx.x;
  const int64_t g = leaf_first + li;
  const int ts = tst[g], te = ten[g];
  if (ts >= te) return;
  const int nn = near_cnt[li];
  const int *nsrc = near_src + li * NEAR_MAX;
  if (tid < nn) {
    const int s = nsrc[tid];
    const double2 cg = ctr[g], cs = ctr[s];
    m_s0[tid] = sst[s];
    m_cnt[tid] = sen[s] - sst[s];
    m_dx[tid] = (R)(cs.x - cg.x);
    m_dy[tid] = (R)(cs.y - cg.y);
  }
  __syncthreads();
  if (tid == 0) {
    int b = 0;
    for (int e = 0; e < nn; ++e) {
      m_base[e] = b;
      b += m_cnt[e];
    }
    m_base[nn] = b;
  }
  __syncthreads();
  const int total = m_base[nn];
  // the Near stencils list the leaf itself first
  const int n_self = (nn > 0 && nsrc[0] == (int)g) ? m_cnt[0] : 0;
  for (int t0 = ts; t0 < te; t0 += 2 * P2P_TH) {
    const int ntc = min(2 * P2P_TH, te - t0);
    const int np = (ntc + 1) / 2;
    const int K = P2P_TH / np;                  // source slices per target pair
    const int i = tid % np, k = tid / np;
    const bool act = k < K;
    const bool has_b = i + np < ntc;
    R ax = (R)0, ay = (R)0, bx = (R)0, by = (R)0;
    if (act) {
      ax = tgt[(int64_t)(t0 + i) * tstride];
      ay = tgt[(int64_t)(t0 + i) * tstride + 1];
      const int jb = has_b ? t0 + i + np : t0 + i;
      bx = tgt[(int64_t)jb * tstride];
      by = tgt[(int64_t)jb * tstride + 1];
    }
    R sa[2] = {(R)0, (R)0}, sb[2] = {(R)0, (R)0};
    for (int c0 = 0; c0 < total; c0 += CAP) {
      const int c1 = min(total, c0 + CAP);
      __syncthreads();
      for (int e = 0; e < nn; ++e) {
        const int b = m_base[e];
        const int lo = max(b, c0), hi = min(m_base[e + 1], c1);
        if (lo < hi) {
          const int s0 = m_s0[e];
          const R dcx = m_dx[e], dcy = m_dy[e];
          for (int q = lo + tid; q < hi; q += P2P_TH) {
            const typename T::V4 v = reinterpret_cast<const typename T::V4 *>(src4)[s0 + q - b];
            typename T::V4 w;
            w.x = v.x + dcx;
            w.y = v.y + dcy;
            w.z = v.z;
            w.w = (R)0;
            sp[q - c0] = w;
          }
        }
      }
      __syncthreads();
      if (act) {
        const int m = c1 - c0;
        const int self_end = max(0, min(m, n_self - c0));
        const int first_unchecked = self_end + ((k - self_end) % K + K) % K;
        if (self_end > 0) p2p_slice<R, true>(sp, k, self_end, K, ax, ay, bx, by, sa, sb);
        p2p_slice<R, false>(sp, first_unchecked, m, K, ax, ay, bx, by, sa, sb);
      }
    }
    red[tid] = act ? (double)sa[0] - (double)sa[1] : 0.0;
    red2[tid] = (act && has_b) ? (double)sb[0] - (double)sb[1] : 0.0;
    __syncthreads();
    if (tid < np) {
      double ta = 0.0, tb = 0.0;
      for (int kk = 0; kk < K; ++kk) {
        ta += red[tid + kk * np];
        tb += red2[tid + kk * np];
      }
      phi_near[t0 + tid] = ta * T::scale;
      if (tid + np < ntc) phi_near[t0 + tid + np] = tb * T::scale;
    }
    __syncthreads();
  }
}

}  // namespace

template <typename R>
cudaError_t launch_p2p(int64_t leaf_first, int64_t n_leaves, const R *src4, const R *tgt,
                       int tstride, const int *src_start, const int *src_end,
                       const int *tgt_start, const int *tgt_end, const int *near_cnt,
                       const int *near_src, const double2 *ctr, double *phi_near,
                       double mean_targets, cudaStream_t s) {
  if (n_leaves <= 0) return cudaSuccess;
  if (mean_targets >= 48.0) {   // large leaves: block-staged, sliced sources
    k_p2p_block<R><<<(unsigned)n_leaves, P2P_TH, 0, s>>>(leaf_first, src4, tgt, tstride, src_start,
                                                         src_end, tgt_start, tgt_end, near_cnt,
                                                         near_src, ctr, phi_near);
  } else {                      // small leaves: one warp per leaf
    const unsigned blocks = (unsigned)((n_leaves * 32 + P2P_TH - 1) / P2P_TH);
    k_p2p<R><<<blocks, P2P_TH, 0, s>>>(leaf_first, n_leaves, src4, tgt, tstride, src_start, src_end,
                                        tgt_start, tgt_end, near_cnt, near_src, ctr, phi_near);
  }
  return cudaGetLastError();
}

template cudaError_t launch_p2p<float>(int64_t, int64_t, const float *, const float *, int,
                                       const int *, const int *, const int *, const int *,
                                       const int *, const int *, const double2 *, double *,
                                       double, cudaStream_t);
template cudaError_t launch_p2p<double>(int64_t, int64_t, const double *, const double *, int,
                                        const int *, const int *, const int *, const int *,
                                        const int *, const int *, const double2 *, double *,
                                        double, cudaStream_t);

}  // namespace fmm2d
