// p2p.cu - near-field direct sum (Sec. 2; the M(P2 s) term of App. A-C):
//   phi_near(y_j) = sum over the sources x_i of {leaf(y_j)} u Neighbors(leaf)
//                   of u_i log|y_j - x_i|,  skipping x_i == y_j.
// One block per target leaf.  The sources of its Near list are staged once in
// shared memory (in chunks), already shifted into the target leaf's frame
// (points are stored relative to their leaf centre, so differences keep full
// precision).  The block's threads are split into (target, source slice)
// pairs so that every thread works even when a leaf holds far fewer targets
// than the block has threads; the slices of a target are summed in FP64.
// The FP32 form takes log2(r^2) on the MUFU unit and scales by ln2/2 once
// per target.
#include "plan.h"

namespace fmm2d {

namespace {

constexpr int P2P_TH = 256;

template <typename R> struct P2PTraits;
template <> struct P2PTraits<float> {
  using V4 = float4;
  static constexpr double scale = 0.34657359027997264;   // ln2 / 2
  static constexpr int cap = 2048;                       // staged sources per chunk
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
  static constexpr int cap = 1024;
  static __device__ __forceinline__ double lg_checked(double r2) { return r2 > 0.0 ? log(r2) : 0.0; }
  static __device__ __forceinline__ double lg(double r2) { return log(r2); }
  static constexpr double floor_r2 = 1e-300;
};

// Sum over staged sources [q0, q1) with stride K for one target.  Points of
// different leaves never coincide (equal coordinates give equal keys), so
// only the target's own leaf needs the r^2 > 0 test; elsewhere a tiny floor
// folded into the FMA keeps log2 finite at no extra instruction.
template <typename R, bool CHECK>
__device__ __forceinline__ double p2p_range(const typename P2PTraits<R>::V4 *sp, int q0, int q1,
                                            int K, R tx, R ty) {
  using T = P2PTraits<R>;
  double sum = 0.0;
  for (int a = q0; a < q1; a += 64 * K) {
    const int b = min(q1, a + 64 * K);
    R acc = (R)0;
#pragma unroll 4
    for (int q = a; q < b; q += K) {
      const typename T::V4 v = sp[q];
      const R dx = tx - v.x, dy = ty - v.y;
      if (CHECK) {
        const R r2 = dx * dx + dy * dy;
        acc += v.z * T::lg_checked(r2);
      } else {
        const R r2 = fma(dx, dx, fma(dy, dy, (R)T::floor_r2));
        acc += v.z * T::lg(r2);
      }
    }
    sum += (double)acc;
  }
  return sum;
}

template <typename R>
__global__ void __launch_bounds__(P2P_TH)
k_p2p(int64_t leaf_first, const R *__restrict__ src4, const R *__restrict__ tgt, int tstride,
      const int *__restrict__ sst, const int *__restrict__ sen, const int *__restrict__ tst,
      const int *__restrict__ ten, const int *__restrict__ near_cnt,
      const int *__restrict__ near_src, const double2 *__restrict__ ctr,
      double *__restrict__ phi_near) {
  using T = P2PTraits<R>;
  constexpr int CAP = T::cap;
  __shared__ typename T::V4 sp[CAP];
  __shared__ double red[P2P_TH];
  __shared__ int m_s0[NEAR_MAX], m_cnt[NEAR_MAX], m_base[NEAR_MAX + 1];
  __shared__ R m_dx[NEAR_MAX], m_dy[NEAR_MAX];
  const int tid = threadIdx.x;
  const int64_t li = blockIdx.x;
  const int64_t g = leaf_first + li;
  const int ts = tst[g], te = ten[g];
  if (ts >= te) return;
  const int nn = near_cnt[li];
  const int *nsrc = near_src + li * NEAR_MAX;
  // per near leaf: first source, count, offset in the staged list, shift
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
  for (int t0 = ts; t0 < te; t0 += P2P_TH) {
    const int ntc = min(P2P_TH, te - t0);
    const int K = P2P_TH / ntc;                 // source slices per target
    const int i = tid % ntc, k = tid / ntc;
    const bool act = k < K;
    R tx = (R)0, ty = (R)0;
    if (act) {
      tx = tgt[(int64_t)(t0 + i) * tstride];
      ty = tgt[(int64_t)(t0 + i) * tstride + 1];
    }
    double sum = 0.0;
    for (int c0 = 0; c0 < total; c0 += CAP) {
      const int c1 = min(total, c0 + CAP);
      __syncthreads();
      for (int e = 0; e < nn; ++e) {
        const int b = m_base[e];
        const int s0 = m_s0[e];
        const int lo = max(b, c0), hi = min(m_base[e + 1], c1);
        if (lo < hi) {
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
        // local index range [0, self_end) holds the target's own leaf
        const int self_end = max(0, min(m, n_self - c0));
        const int first_unchecked = self_end + ((k - self_end) % K + K) % K;
        if (self_end > 0) sum += p2p_range<R, true>(sp, k, self_end, K, tx, ty);
        sum += p2p_range<R, false>(sp, first_unchecked, m, K, tx, ty);
      }
    }
    red[tid] = act ? sum : 0.0;
    __syncthreads();
    if (tid < ntc) {
      double t = 0.0;
      for (int kk = 0; kk < K; ++kk) t += red[tid + kk * ntc];
      phi_near[t0 + tid] = t * T::scale;
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
                       cudaStream_t s) {
  if (n_leaves <= 0) return cudaSuccess;
  k_p2p<R><<<(unsigned)n_leaves, P2P_TH, 0, s>>>(leaf_first, src4, tgt, tstride, src_start,
                                                   src_end, tgt_start, tgt_end, near_cnt, near_src,
                                                   ctr, phi_near);
  return cudaGetLastError();
}

template cudaError_t launch_p2p<float>(int64_t, int64_t, const float *, const float *, int,
                                       const int *, const int *, const int *, const int *,
                                       const int *, const int *, const double2 *, double *,
                                       cudaStream_t);
template cudaError_t launch_p2p<double>(int64_t, int64_t, const double *, const double *, int,
                                        const int *, const int *, const int *, const int *,
                                        const int *, const int *, const double2 *, double *,
                                        cudaStream_t);

}  // namespace fmm2d
