// m2l_ff.cu - M2L of the hybrid and split precision forms on the FP32 pipes,
// in float-float (hi + lo) arithmetic.
//
// These forms keep multipoles and locals in FP64 for tolerances below the
// reach of FP32 expansions.  On this GPU the FP64 pipe runs at about 1/70 of
// the FP32 rate, so the M2L sum (Sec. 2: every local coefficient is a sum
// over the NeighborsE4 list of operator x multipole products, eq. 3) is done
// here in float-float: every operator value and every multipole coefficient
// is an unevaluated sum hi + lo of two floats (48 significant bits), each
// product is formed exactly with an FMA (TwoProd), the cross terms hi*lo are
// added to a running compensation, and the sum is kept as s + c with an
// error-free TwoSum per term (the compensated dot product of Ogita, Rump and
// Oishi, 2005).  The result is as accurate as an FP64 evaluation of the same
// sum to within a few units of 2^-48.
//
// The scaled operator of an offset zeta = |zeta| u is T_lk = A_lk u^-(l+k)
// with A real, so an entry turns the gathered multipoles by u^-k, applies
// the real A (two real products per entry instead of four) and turns the
// sum by u^-l (k_m2l_ff below).  The multipoles are converted to float-float
// once per cell (k_ma_to_ff) before the gathers.
//
// Work is laid out as the dense contraction the operator sharing allows: on
// scaled coefficients the operator depends only on (child class, stencil
// entry), so a CTA takes 32 target cells of one class and, per stencil
// entry, stages that entry's operator once in shared memory together with
// the 32 gathered source multipoles, then applies it to all 32 targets:
// lane t of every warp owns target t, warp w the output rows w, w + 8, ...
#include <complex>

#include <mutex>

#include "plan.h"

namespace fmm2d {

namespace {

constexpr int FF_THREADS = 256;
constexpr int FF_TM = 32;                        // target cells per tile: lane t of each warp
constexpr int FF_LG = FF_THREADS / FF_TM;        // row groups (warps): row l = lg + FF_LG j
constexpr int FF_NJ = (MAXP + 1 + FF_LG - 1) / FF_LG;

// s + x = t + e exactly (Knuth's TwoSum); s := t, comp += e
__device__ __forceinline__ void two_sum_acc(float &s, float &comp, float x) {
  const float t = s + x;
  const float bp = t - s;
  const float ap = t - bp;
  comp += (s - ap) + (x - bp);
  s = t;
}

// Float-float values are unevaluated sums: a complex one is a float4
// (hi.re, hi.im, lo.re, lo.im); an accumulator float4 (s.re, c.re, s.im,
// c.im) holds the running sum s and its compensation c.

// d += A * c for real A = (Ah, Al) and complex c (float-float): each real
// product exact by TwoProd, the cross terms Ah cl + Al ch into the
// compensation, the sum error-free by TwoSum
__device__ __forceinline__ void ff_rmac(float4 &d, const float2 A, const float4 c) {
  {
    const float p = A.x * c.x;
    const float e = fmaf(A.x, c.x, -p);
    const float cr = fmaf(A.x, c.z, A.y * c.x);
    two_sum_acc(d.x, d.y, p);
    d.y += e + cr;
  }
  {
    const float p = A.x * c.y;
    const float e = fmaf(A.x, c.y, -p);
    const float ci = fmaf(A.x, c.w, A.y * c.y);
    two_sum_acc(d.z, d.w, p);
    d.w += e + ci;
  }
}

// x * y for complex float-float x and y, returned as float-float (hi, lo)
__device__ __forceinline__ float4 ff_cmul(const float4 x, const float4 y) {
  float re, re_lo, im, im_lo;
  {
    const float p1 = x.x * y.x, e1 = fmaf(x.x, y.x, -p1);
    const float p2 = -x.y * y.y, e2 = fmaf(-x.y, y.y, -p2);
    float s = p1, c = 0.f;
    two_sum_acc(s, c, p2);
    c += e1 + e2 + fmaf(x.x, y.z, fmaf(x.z, y.x, fmaf(-x.y, y.w, -x.w * y.y)));
    re = s + c;
    re_lo = c - (re - s);
  }
  {
    const float p1 = x.x * y.y, e1 = fmaf(x.x, y.y, -p1);
    const float p2 = x.y * y.x, e2 = fmaf(x.y, y.x, -p2);
    float s = p1, c = 0.f;
    two_sum_acc(s, c, p2);
    c += e1 + e2 + fmaf(x.x, y.w, fmaf(x.z, y.y, fmaf(x.y, y.z, x.w * y.x)));
    im = s + c;
    im_lo = c - (im - s);
  }
  return make_float4(re, im, re_lo, im_lo);
}

__device__ __forceinline__ float4 ff_of(double re, double im) {
  const float hr = __double2float_rn(re), hi = __double2float_rn(im);
  return make_float4(hr, hi, __double2float_rn(re - (double)hr), __double2float_rn(im - (double)hi));
}

// Every cell's multipole (Q, a^_1 .. a^_p) as float-float, once, so that the
// M2L gathers (each source row is read once per stencil entry that names it)
// need no FP64 arithmetic.
__global__ void k_ma_to_ff(int64_t n_cells, int p, int P, const double *__restrict__ mQ,
                           const double2 *__restrict__ ma, float4 *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int P1 = p + 1;
  if (i >= n_cells * P1) return;
  const int64_t cell = i / P1;
  const int k = (int)(i - cell * P1);
  if (k == 0) {
    out[i] = ff_of(mQ[cell], 0.0);
  } else {
    const double2 m = ma[cell * P + k - 1];
    out[i] = ff_of(m.x, m.y);
  }
}

// The scaled operator of an entry with zeta = |zeta| u is T_lk = A_lk u^-(l+k)
// with A real (the binomial, sign and |zeta| powers), so
//   b^_l = u^-l sum_k A_lk (u^-k a^_k):
// the gathered multipoles are turned by u^-k, the real A applied (two real
// products per entry instead of four), and the sum turned by u^-l.
// Shared memory: A of the current entry [k][l] (float2 hi, lo), its phases
// u^-m (m = 0..p), the turned multipoles [t][k] (row stride p + 1 made odd),
// the source indices.
__global__ void __launch_bounds__(FF_THREADS, 3)
k_m2l_ff(FfArgs a) {
  extern __shared__ float4 smem_ff[];
  const int p = a.p, P1 = p + 1;
  const int AS = P1 | 1;                      // odd row stride: no bank conflicts
  float4 *sC = smem_ff;                       // FF_TM * AS
  float4 *sPh = sC + FF_TM * AS;              // P1
  float2 *sA = reinterpret_cast<float2 *>(sPh + P1);                 // P1 * P1
  float4 *sAcc = reinterpret_cast<float4 *>(sA + ((P1 * P1 + 1) & ~1));   // [FF_NJ][FF_THREADS]
  int *s_src = reinterpret_cast<int *>(sAcc + FF_NJ * FF_THREADS);       // FF_TM
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
    // the running sums of the rows live in shared memory (touched once per
    // entry), the per-entry sums d in registers
#pragma unroll
    for (int j = 0; j < FF_NJ; ++j) sAcc[j * FF_THREADS + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int E = a.sten_len[c];
    const uint16_t *ops_c = a.sten_ops + c * FAR_MAX;
    for (int e = 0; e < E; ++e) {
      const int op = ops_c[e];
      __syncthreads();   // the previous entry's reads of shared memory are done
      if (lg == 0) s_src[t] = g >= 0 ? a.far_full[fi * FAR_MAX + e] : -1;
      const float2 *Ag = a.opA + (int64_t)op * P1 * P1;
      for (int i = tid; i < P1 * P1; i += FF_THREADS) sA[i] = Ag[i];
      for (int i = tid; i < P1; i += FF_THREADS) sPh[i] = a.oph[(int64_t)op * P1 + i];
      __syncthreads();
      for (int i = tid; i < FF_TM * P1; i += FF_THREADS) {
        const int tt = i / P1, k = i - tt * P1;
        const int src = s_src[tt];
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (src >= 0) {
          v = a.ma_ff[(int64_t)src * P1 + k];
          if (k > 0) v = ff_cmul(sPh[k], v);   // u^0 = 1
        }
        sC[tt * AS + k] = v;
      }
      __syncthreads();
      const int src = s_src[t];
      if (lg == 0 && src >= 0) L0 += a.mQ[src] * (ls + a.logz[op]);
      float4 d[FF_NJ];
#pragma unroll
      for (int j = 0; j < FF_NJ; ++j) d[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 *crow = sC + t * AS;
      for (int k = 0; k <= p; ++k) {
        const float4 cv = crow[k];
        const float2 *Ak = sA + k * P1;
#pragma unroll
        for (int j = 0; j < FF_NJ; ++j) {
          const int l = lg + FF_LG * j;
          if (l <= p) ff_rmac(d[j], Ak[l], cv);
        }
      }
      // acc_l += u^-l d_l
#pragma unroll
      for (int j = 0; j < FF_NJ; ++j) {
        const int l = lg + FF_LG * j;
        if (l > p) break;
        const float4 r = ff_cmul(sPh[l], make_float4(d[j].x, d[j].z, d[j].y, d[j].w));
        float4 acc = sAcc[j * FF_THREADS + tid];
        two_sum_acc(acc.x, acc.y, r.x);
        acc.y += r.z;
        two_sum_acc(acc.z, acc.w, r.y);
        acc.w += r.w;
        sAcc[j * FF_THREADS + tid] = acc;
      }
    }
    if (g >= 0) {
#pragma unroll
      for (int j = 0; j < FF_NJ; ++j) {
        const int l = lg + FF_LG * j;
        if (l > p) break;
        const float4 acc = sAcc[j * FF_THREADS + tid];
        const double re = (double)acc.x + (double)acc.y;
        const double im = (double)acc.z + (double)acc.w;
        if (l == 0) a.lL0[g] = L0 + re;
        else a.lb[(int64_t)g * a.P + l - 1] = make_double2(re, im);
      }
    }
  }
}

}  // namespace

size_t m2l_ff_smem_bytes(int p) {
  const int P1 = p + 1;
  return (size_t)(FF_TM * (P1 | 1) + P1 + FF_NJ * FF_THREADS) * sizeof(float4) +
         (size_t)((P1 * P1 + 1) & ~1) * sizeof(float2) + FF_TM * sizeof(int);
}

void ff_build_table(const std::vector<std::complex<double>> &zeta,
                    const std::vector<std::complex<double>> &ops, int p, std::vector<float> &A,
                    std::vector<float> &ph) {
  // ops: per operator [l][k] (k = 0 the Q column); u = zeta / |zeta| and
  // A_lk = T_lk u^(l+k), real by the form of the scaled operator; stored
  // [op][k][l] as (hi, lo), phases u^-m (m = 0..p) as hi.re, hi.im, lo.re, lo.im
  const size_t P1 = (size_t)p + 1, n_ops = zeta.size();
  A.assign(n_ops * P1 * P1 * 2, 0.f);
  ph.assign(n_ops * P1 * 4, 0.f);
  for (size_t o = 0; o < n_ops; ++o) {
    const std::complex<double> u = zeta[o] / std::abs(zeta[o]);
    std::vector<std::complex<double>> up(2 * P1), um(P1);
    up[0] = 1.0;
    for (size_t m = 1; m < 2 * P1; ++m) up[m] = up[m - 1] * u;
    for (size_t m = 0; m < P1; ++m) {
      um[m] = std::conj(up[m]);   // |u| = 1: u^-m
      const float hr = (float)um[m].real(), hi = (float)um[m].imag();
      float *q = &ph[(o * P1 + m) * 4];
      q[0] = hr;
      q[1] = hi;
      q[2] = (float)(um[m].real() - (double)hr);
      q[3] = (float)(um[m].imag() - (double)hi);
    }
    for (size_t l = 0; l < P1; ++l)
      for (size_t k = 0; k < P1; ++k) {
        const double v = (ops[(o * P1 + l) * P1 + k] * up[l + k]).real();
        const float h = (float)v;
        float *q = &A[((o * P1 + k) * P1 + l) * 2];
        q[0] = h;
        q[1] = (float)(v - (double)h);
      }
  }
}

cudaError_t launch_m2l_ff(const FfArgs &a, int64_t n_far_cells, cudaStream_t s) {
  if (n_far_cells <= 0) return cudaSuccess;
  if (a.p < 1 || a.p > MAXP) return cudaErrorInvalidValue;
  const size_t smem = m2l_ff_smem_bytes(a.p);
  {
    // The shared-memory limit is one setting of the kernel for the whole
    // process, and plans of different p launch it from several host threads
    // (server slots): only ever raise it, so that no launch finds it lowered
    // by another thread between its own setting and its launch.
    static std::mutex mu;
    static size_t set_bytes = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (smem > set_bytes) {
      cudaError_t e = cudaFuncSetAttribute(k_m2l_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      set_bytes = smem;
    }
  }
  // tiles <= cells / 32 + classes; a persistent grid of three CTAs per SM
  const int64_t nel = a.n_cells * (a.p + 1);
  k_ma_to_ff<<<(unsigned)((nel + 255) / 256), 256, 0, s>>>(a.n_cells, a.p, a.P, a.mQ, a.ma, a.ma_ff);
  const int64_t tiles = n_far_cells / FF_TM + MAX_CLASSES;
  const int grid = (int)std::min<int64_t>(tiles, 3 * (int64_t)std::max(1, a.sms));
  k_m2l_ff<<<grid, FF_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fmm2d
