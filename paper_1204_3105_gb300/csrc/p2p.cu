// p2p.cu - near-field direct sum (Sec. 2; the M(P2 s) term of App. A-C):
//   phi_near(y_j) = sum over the sources x_i of {leaf(y_j)} u Neighbors(leaf)
//                   of u_i log|y_j - x_i|,  skipping x_i == y_j.
// One block per target leaf.  Each source leaf of the Near list is staged in
// shared memory, already shifted into the target leaf's frame (points are
// stored relative to their leaf centre, so differences keep full precision),
// and every thread sums over it for its target.  The FP32 form takes
// log2(r^2) on the MUFU unit and scales by ln2/2 once per target; partial
// sums per source leaf are accumulated in FP64.
#include "plan.h"

namespace fmm2d {

namespace {

constexpr int P2P_TH = 128;

__device__ __forceinline__ float log_r2(float r2) { return r2 > 0.f ? __log2f(r2) : 0.f; }
__device__ __forceinline__ double log_r2(double r2) { return r2 > 0.0 ? log(r2) : 0.0; }
template <typename R> struct LogScale;
template <> struct LogScale<float> { static constexpr double v = 0.34657359027997264; };  // ln2 / 2
template <> struct LogScale<double> { static constexpr double v = 0.5; };

template <typename R>
__global__ void __launch_bounds__(P2P_TH)
k_p2p(int64_t leaf_first, const R *__restrict__ src4, const R *__restrict__ tgt, int tstride,
      const int *__restrict__ sst, const int *__restrict__ sen, const int *__restrict__ tst,
      const int *__restrict__ ten, const int *__restrict__ near_cnt,
      const int *__restrict__ near_src, const double2 *__restrict__ ctr,
      double *__restrict__ phi_near) {
  __shared__ R sx[P2P_TH], sy[P2P_TH], su[P2P_TH];
  const int64_t li = blockIdx.x;
  const int64_t g = leaf_first + li;
  const int ts = tst[g], te = ten[g];
  if (ts >= te) return;
  const double2 cg = ctr[g];
  const int nn = near_cnt[li];
  for (int j0 = ts; j0 < te; j0 += P2P_TH) {
    const int j = j0 + threadIdx.x;
    const bool act = j < te;
    R tx = (R)0, ty = (R)0;
    if (act) {
      tx = tgt[(int64_t)j * tstride];
      ty = tgt[(int64_t)j * tstride + 1];
    }
    double total = 0.0;
    for (int e = 0; e < nn; ++e) {
      const int s = near_src[li * NEAR_MAX + e];
      const double2 cs = ctr[s];
      const R dcx = (R)(cs.x - cg.x), dcy = (R)(cs.y - cg.y);
      const int ss = sst[s], se = sen[s];
      for (int i0 = ss; i0 < se; i0 += P2P_TH) {
        __syncthreads();
        const int i = i0 + threadIdx.x;
        if (i < se) {
          const R *pt = src4 + 4 * (int64_t)i;
          sx[threadIdx.x] = pt[0] + dcx;
          sy[threadIdx.x] = pt[1] + dcy;
          su[threadIdx.x] = pt[2];
        }
        __syncthreads();
        const int m = min(P2P_TH, se - i0);
        R acc = (R)0;
        for (int q = 0; q < m; ++q) {
          const R dx = tx - sx[q], dy = ty - sy[q];
          const R r2 = dx * dx + dy * dy;
          acc += su[q] * log_r2(r2);
        }
        total += (double)acc;
      }
    }
    if (act) phi_near[j] = total * LogScale<R>::v;
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
