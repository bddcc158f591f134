// m2l_ff.cu - M2L of the hybrid precision form on the FP32 pipes, in
// float-float (hi + lo) arithmetic.
//
// The hybrid form keeps multipoles and locals in FP64 for tolerances below
// the reach of FP32 expansions.  On this GPU the FP64 pipe runs at about
// 1/70 of the FP32 rate, so the M2L sum (Sec. 2: every local coefficient is a
// sum over the NeighborsE4 list of operator x multipole products, eq. 3) is
// done here in float-float: every operator entry and every multipole
// coefficient is an unevaluated sum hi + lo of two floats (48 significant
// bits), each product is formed exactly with an FMA (TwoProd), the two cross
// terms hi*lo are added to a running compensation, and the sum is kept as
// s + c with an error-free TwoSum per term (the compensated dot product of
// Ogita, Rump and Oishi, 2005).  The result is as accurate as an FP64
// evaluation of the same sum to within a few units of 2^-48.
//
// Work is laid out as the dense contraction the operator sharing allows: on
// scaled coefficients the operator depends only on (child class, stencil
// entry), so a CTA takes 64 target cells of one class and, per stencil
// entry, stages that entry's operator once in shared memory together with
// the 64 gathered source multipoles, then applies it to all 64 targets.
#include "plan.h"

namespace fmm2d {

namespace {

constexpr int FF_THREADS = 256;
constexpr int FF_TM = 64;                        // target cells per tile
constexpr int FF_LG = FF_THREADS / FF_TM;        // row groups: row l = lg + FF_LG j
constexpr int FF_NJ = (MAXP + 1 + FF_LG - 1) / FF_LG;

// s + x = t + e exactly (Knuth's TwoSum); s := t, comp += e
__device__ __forceinline__ void two_sum_acc(float &s, float &comp, float x) {
  const float t = s + x;
  const float bp = t - s;
  const float ap = t - bp;
  comp += (s - ap) + (x - bp);
  s = t;
}

// acc += T * a for complex float-float T = (Th, Tl), a = (ah, al), each a
// float4 (hi.re, hi.im, lo.re, lo.im); acc = (s_re, c_re, s_im, c_im)
__device__ __forceinline__ void ff_cmac(float4 &acc, const float4 T, const float4 a) {
  // real part: Th.re ah.re - Th.im ah.im + cross terms
  {
    const float p1 = T.x * a.x;
    const float e1 = fmaf(T.x, a.x, -p1);
    const float p2 = -T.y * a.y;
    const float e2 = fmaf(-T.y, a.y, -p2);
    float cr = fmaf(T.x, a.z, fmaf(T.z, a.x, fmaf(-T.y, a.w, -T.w * a.y)));
    cr += e1 + e2;
    two_sum_acc(acc.x, acc.y, p1);
    two_sum_acc(acc.x, acc.y, p2);
    acc.y += cr;
  }
  // imaginary part: Th.re ah.im + Th.im ah.re + cross terms
  {
    const float p1 = T.x * a.y;
    const float e1 = fmaf(T.x, a.y, -p1);
    const float p2 = T.y * a.x;
    const float e2 = fmaf(T.y, a.x, -p2);
    float ci = fmaf(T.x, a.w, fmaf(T.z, a.y, fmaf(T.y, a.z, T.w * a.x)));
    ci += e1 + e2;
    two_sum_acc(acc.z, acc.w, p1);
    two_sum_acc(acc.z, acc.w, p2);
    acc.w += ci;
  }
}

__device__ __forceinline__ float4 ff_of(double re, double im) {
  const float hr = __double2float_rn(re), hi = __double2float_rn(im);
  return make_float4(hr, hi, __double2float_rn(re - (double)hr), __double2float_rn(im - (double)hi));
}

// Shared memory: the operator of the current entry, [k][l] (k = 0 is the Q
// column), then the gathered multipoles [t][k] (row stride p + 1 made odd),
// then the source indices.
__global__ void __launch_bounds__(FF_THREADS, 2)
k_m2l_ff(FfArgs a) {
  extern __shared__ float4 smem_ff[];
  const int p = a.p, P1 = p + 1;
  float4 *sT = smem_ff;                       // P1 * P1
  const int AS = P1 | 1;                      // odd row stride: no bank conflicts
  float4 *sA = sT + P1 * P1;                  // FF_TM * AS
  int *s_src = reinterpret_cast<int *>(sA + FF_TM * AS);
  __shared__ int s_cnt[MAX_CLASSES];
  const int tid = threadIdx.x;
  const int t = tid % FF_TM, lg = tid / FF_TM;
  if (tid < MAX_CLASSES) s_cnt[tid] = tid < a.n_classes ? a.cls_cnt[tid] : 0;
  __syncthreads();
  int total = 0;
  for (int c = 0; c < a.n_classes; ++c) total += (s_cnt[c] + FF_TM - 1) / FF_TM;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int c = 0, t0 = tile;
    while (t0 >= (s_cnt[c] + FF_TM - 1) / FF_TM) {
      t0 -= (s_cnt[c] + FF_TM - 1) / FF_TM;
      ++c;
    }
    const int row0 = t0 * FF_TM;
    const int nrows = min(FF_TM, s_cnt[c] - row0);
    const int g = t < nrows ? a.cls_cells[(int64_t)c * a.cls_cap + row0 + t] : -1;
    const int64_t fi = g >= 0 ? (int64_t)g - a.far_first : 0;
    double ls = 0.0;
    if (g >= 0 && lg == 0) {
      int l = a.l_min;
      while (l < a.L && (int64_t)g >= a.lev_first[l + 1]) ++l;
      ls = a.log_abs_scale[l];
    }
    double L0 = 0.0;
    float4 acc[FF_NJ];
#pragma unroll
    for (int j = 0; j < FF_NJ; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int E = a.sten_len[c];
    const uint16_t *ops_c = a.sten_ops + c * FAR_MAX;
    for (int e = 0; e < E; ++e) {
      const int op = ops_c[e];
      __syncthreads();   // the previous entry's reads of sT, sA, s_src are done
      if (lg == 0) s_src[t] = g >= 0 ? a.far_full[fi * FAR_MAX + e] : -1;
      const float4 *Tg = a.ops + (int64_t)op * P1 * P1;
      for (int i = tid; i < P1 * P1; i += FF_THREADS) sT[i] = Tg[i];
      __syncthreads();
      for (int i = tid; i < FF_TM * P1; i += FF_THREADS) {
        const int tt = i / P1, k = i - tt * P1;
        const int src = s_src[tt];
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (src >= 0) {
          if (k == 0) {
            v = ff_of(a.mQ[src], 0.0);
          } else {
            const double2 m = a.ma[(int64_t)src * a.P + k - 1];
            v = ff_of(m.x, m.y);
          }
        }
        sA[tt * AS + k] = v;
      }
      __syncthreads();
      const int src = s_src[t];
      if (lg == 0 && src >= 0) L0 += a.mQ[src] * (ls + a.logz[op]);
      const float4 *arow = sA + t * AS;
      for (int k = 0; k <= p; ++k) {
        const float4 av = arow[k];
        const float4 *Tk = sT + k * P1;
#pragma unroll
        for (int j = 0; j < FF_NJ; ++j) {
          const int l = lg + FF_LG * j;
          if (l <= p) ff_cmac(acc[j], Tk[l], av);
        }
      }
    }
    if (g >= 0) {
#pragma unroll
      for (int j = 0; j < FF_NJ; ++j) {
        const int l = lg + FF_LG * j;
        if (l > p) break;
        const double re = (double)acc[j].x + (double)acc[j].y;
        const double im = (double)acc[j].z + (double)acc[j].w;
        if (l == 0) a.lL0[g] = L0 + re;
        else a.lb[(int64_t)g * a.P + l - 1] = make_double2(re, im);
      }
    }
  }
}

}  // namespace

size_t m2l_ff_smem_bytes(int p) {
  const int P1 = p + 1;
  return (size_t)(P1 * P1 + FF_TM * (P1 | 1)) * sizeof(float4) + FF_TM * sizeof(int);
}

void ff_build_table(const std::vector<double> &re, const std::vector<double> &im, int n_ops, int p,
                    std::vector<float> &out) {
  // input [op][l][k] (row l = output coefficient, column k = input, k = 0
  // the Q column); output [op][k][l] as hi.re, hi.im, lo.re, lo.im
  const size_t P1 = (size_t)p + 1;
  out.assign((size_t)n_ops * P1 * P1 * 4, 0.f);
  for (int o = 0; o < n_ops; ++o)
    for (size_t l = 0; l < P1; ++l)
      for (size_t k = 0; k < P1; ++k) {
        const size_t i = ((size_t)o * P1 + l) * P1 + k, j = ((size_t)o * P1 + k) * P1 + l;
        const float hr = (float)re[i], hi = (float)im[i];
        out[4 * j + 0] = hr;
        out[4 * j + 1] = hi;
        out[4 * j + 2] = (float)(re[i] - (double)hr);
        out[4 * j + 3] = (float)(im[i] - (double)hi);
      }
}

cudaError_t launch_m2l_ff(const FfArgs &a, int64_t n_far_cells, cudaStream_t s) {
  if (n_far_cells <= 0) return cudaSuccess;
  if (a.p < 1 || a.p > MAXP) return cudaErrorInvalidValue;
  const size_t smem = m2l_ff_smem_bytes(a.p);
  cudaError_t e = cudaFuncSetAttribute(k_m2l_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // tiles <= cells / 64 + classes; a persistent grid of two CTAs per SM
  const int64_t tiles = n_far_cells / FF_TM + MAX_CLASSES;
  const int grid = (int)std::min<int64_t>(tiles, 2 * (int64_t)std::max(1, a.sms));
  k_m2l_ff<<<grid, FF_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fmm2d
