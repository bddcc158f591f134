// p2p.cu - near-field direct sum (Sec. 2; the M(P2 s) term of App. A-C):
//   phi_near(y_j) = sum over the sources x_i of {leaf(y_j)} u Neighbors(leaf)
//                   of u_i log|y_j - x_i|,  skipping x_i == y_j.
// FP32 form (k_p2p_x2): packed f32x2 arithmetic, log2(r^2) on the MUFU unit,
// scaled by ln2/2 once per target, partial sums folded without error.  FP64
// form: one warp per target leaf (k_p2p) for small leaves or CSR lists, and a
// block-staged form (k_p2p_block) for large ones, with a table-driven log.
// Points are stored relative to their leaf centre, so differences keep full
// precision.
#include "plan.h"

namespace fmm2d {

namespace {

constexpr int P2P_TH = 256;

template <typename R> struct P2PTraits;
// FP64 natural logarithm, table driven (Tang, "Table-driven implementation of
// the logarithm function in IEEE floating-point arithmetic", ACM TOMS 1990):
// x = 2^k m with m in [1, 2); c = 1 + j/128 with j the top seven fraction bits
// of m; log x = k ln2 + log c + log1p(t), t = (m - c)/c in [0, 1/128), and
// log1p by its Taylor series to t^9 (truncation below 1e-22).  m - c is
// exact; the table holds log c and 1/c, filled per block with the library's
// log.  The result is within a few ulp of log x for every normal x > 0.
__shared__ double2 s_logtab[128];

__device__ __forceinline__ void logtab_init() {
  for (int j = threadIdx.x; j < 128; j += blockDim.x) {
    const double c = 1.0 + j * 0.0078125;
    s_logtab[j] = make_double2(log(c), 1.0 / c);
  }
  __syncthreads();
}

__device__ __forceinline__ double log_tab(double x) {
  // ln 2 split into its leading 32 significant bits (so k * LN2_HI is exact)
  // and the rest, from ln 2 = sum 1/(i 2^i) evaluated to 60 digits
  constexpr double LN2_HI = 0x1.62e42fee00000p-1;
  constexpr double LN2_LO = 0x1.a39ef35793c76p-33;
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int k = (hi >> 20) - 1023;
  const int j = (hi >> 13) & 127;
  const double m = __hiloint2double((hi & 0x000FFFFF) | 0x3FF00000, lo);
  const double c = __hiloint2double(0x3FF00000 | (j << 13), 0);
  const double2 e = s_logtab[j];
  const double t = (m - c) * e.y;
  double s = 1.0 / 9.0;
  s = fma(s, t, -1.0 / 8.0);
  s = fma(s, t, 1.0 / 7.0);
  s = fma(s, t, -1.0 / 6.0);
  s = fma(s, t, 1.0 / 5.0);
  s = fma(s, t, -1.0 / 4.0);
  s = fma(s, t, 1.0 / 3.0);
  s = fma(s, t, -1.0 / 2.0);
  s = fma(s, t, 1.0);
  const double dk = (double)k;
  return fma(dk, LN2_HI, e.x) + fma(dk, LN2_LO, s * t);
}

template <> struct P2PTraits<double> {
  using V4 = double4_32a;
  static constexpr double scale = 0.5;
  static __device__ __forceinline__ double lg_checked(double r2) { return r2 > 0.0 ? log_tab(r2) : 0.0; }
  static __device__ __forceinline__ double lg(double r2) { return log_tab(r2); }
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
k_p2p(int64_t leaf_first, int64_t n_leaves, const int *__restrict__ leaf_ids,
      const R *__restrict__ src4, const R *__restrict__ tgt, int tstride,
      const int *__restrict__ sst, const int *__restrict__ sen, const int *__restrict__ tst,
      const int *__restrict__ ten, const int *__restrict__ near_cnt,
      const int *__restrict__ near_off, const int *__restrict__ near_src,
      const double2 *__restrict__ ctr, double *__restrict__ phi_near) {
  using T = P2PTraits<R>;
  if constexpr (sizeof(R) == 8) logtab_init();   // before any thread leaves
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
  if constexpr (sizeof(R) == 8) logtab_init();   // before any thread leaves
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

// ---- FP32 form on packed f32x2 arithmetic ------------------------------
// Four targets per thread held as two float2 pairs, so that one FADD2/FFMA2
// serves two source-target pairs; sources are staged in the target leaf's
// frame as (-x, -x, -y, -y) and (u, u) so that a staged record feeds the
// packed operations directly.  Per source a thread issues 8 packed FP32
// operations, 4 MUFU lg2 and 2 shared loads for 4 pairs, which leaves the
// kernel bound by the MUFU unit (one lg2 per pair) instead of by issue.
// A group of T threads (a warp, or 2 to 8 warps synchronised by a named
// barrier) owns one target leaf; the block holds 256 / T groups.  Within a
// group, thread (i, k) takes target quadruple i and every K-th staged source
// starting at k; slice partials are combined in FP32 with compensation and
// converted to FP64 once per target.
constexpr int X2_CAP = 1536;        // staged sources per block
constexpr int X2_CAP_COMP = 640;    // hybrid form: hi and lo coordinates, split strengths

template <int T>
__device__ __forceinline__ void x2_sync(int grp) {
  if constexpr (T == 32) __syncwarp();
  else if constexpr (T == P2P_TH) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(T) : "memory");
}

__device__ __forceinline__ float x2_lg(float r2) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
  return y;
}

// One staged source against the thread's four targets: log2 r^2 of the four
// pairs.  CHECK (the target's own leaf): r^2 at the floor means the points
// coincide at FP32 resolution, and the pair contributes nothing.
template <bool CHECK>
__device__ __forceinline__ void x2_logs(const float4 &p, const float2 &xab, const float2 &xcd,
                                        const float2 &yab, const float2 &ycd, float2 &lab,
                                        float2 &lcd) {
  constexpr float FL = 1e-30f;
  const float2 px = make_float2(p.x, p.y), py = make_float2(p.z, p.w);
  const float2 fl = make_float2(FL, FL);
  const float2 dxab = __fadd2_rn(xab, px), dxcd = __fadd2_rn(xcd, px);
  const float2 dyab = __fadd2_rn(yab, py), dycd = __fadd2_rn(ycd, py);
  const float2 rab = __ffma2_rn(dxab, dxab, __ffma2_rn(dyab, dyab, fl));
  const float2 rcd = __ffma2_rn(dxcd, dxcd, __ffma2_rn(dycd, dycd, fl));
  lab.x = x2_lg(rab.x);
  lab.y = x2_lg(rab.y);
  lcd.x = x2_lg(rcd.x);
  lcd.y = x2_lg(rcd.y);
  if (CHECK) {
    lab.x = rab.x == FL ? 0.f : lab.x;
    lab.y = rab.y == FL ? 0.f : lab.y;
    lcd.x = rcd.x == FL ? 0.f : lcd.x;
    lcd.y = rcd.y == FL ? 0.f : lcd.y;
  }
}

// a + b = s + err exactly (Knuth's TwoSum), two lanes at a time
__device__ __forceinline__ void x2_two_sum2(const float2 a, const float2 b, float2 &s, float2 &err) {
  const float2 m1 = make_float2(-1.f, -1.f);
  s = __fadd2_rn(a, b);
  const float2 bp = __ffma2_rn(a, m1, s);    // s - a
  const float2 ap = __ffma2_rn(bp, m1, s);   // s - bp
  err = __fadd2_rn(__ffma2_rn(ap, m1, a), __ffma2_rn(bp, m1, b));   // (a - ap) + (b - bp)
}

// r^2 of two target-source pairs as rh + rl (float-float): the coordinate
// differences by the accurate float-float subtraction (below), squared with
// exact products (FMA), summed by TwoSum and renormalised (about 43 bits of
// r^2 however close the points); rh is floored at FL > 0 (a normal number)
__device__ __forceinline__ void x2_r2_ff(const float2 &xt, const float2 &xs, const float2 &xtl,
                                         const float2 &xsl, const float2 &yt, const float2 &ys,
                                         const float2 &ytl, const float2 &ysl, float2 &rh,
                                         float2 &rl) {
  constexpr float FL = 1e-30f;
  // accurate float-float differences: TwoSum of the hi parts and of the lo
  // parts, the first lo error into the hi error, a TwoSum renormalisation,
  // then the second lo error (|lo| stays near ulp(hi) / 2 however close the
  // two points are)
  float2 dxh, dyh, dxl, dyl;
  {
    float2 sx, ex, lx, lex, sy, ey, ly, ley, rx, ry;
    x2_two_sum2(xt, xs, sx, ex);
    x2_two_sum2(xtl, xsl, lx, lex);
    x2_two_sum2(yt, ys, sy, ey);
    x2_two_sum2(ytl, ysl, ly, ley);
    x2_two_sum2(sx, __fadd2_rn(ex, lx), dxh, rx);
    x2_two_sum2(sy, __fadd2_rn(ey, ly), dyh, ry);
    dxl = __fadd2_rn(rx, lex);
    dyl = __fadd2_rn(ry, ley);
  }
  const float2 qx = __fmul2_rn(dxh, dxh), qy = __fmul2_rn(dyh, dyh);
  const float2 qxe = __ffma2_rn(dxh, dxh, make_float2(-qx.x, -qx.y));
  const float2 qye = __ffma2_rn(dyh, dyh, make_float2(-qy.x, -qy.y));
  float2 h, he;
  x2_two_sum2(qx, qy, h, he);
  const float2 two = make_float2(2.f, 2.f);
  float2 l = __fadd2_rn(__fadd2_rn(qxe, qye), he);
  l = __ffma2_rn(__fmul2_rn(two, dxh), dxl, l);
  l = __ffma2_rn(__fmul2_rn(two, dyh), dyl, l);
  l = __ffma2_rn(dxl, dxl, __ffma2_rn(dyl, dyl, l));
  const float2 t = __fadd2_rn(h, l);                              // renormalise (h >= |l| or h = 0)
  rl = __fadd2_rn(l, __ffma2_rn(t, make_float2(-1.f, -1.f), h)); // l - (t - h)
  rh = make_float2(fmaxf(t.x, FL), fmaxf(t.y, FL));
}

// log2 r^2 = e + lh + ll for r^2 = rh + rl (rh normal): e the exponent of
// rh, lh + ll the log2 of its mantissa m in [1, 2) by Tang's table method
// (m r_j = 1 + f with r_j ~ 1/m from a 128-entry table, |f| <= 2^-8;
// lh + ll = -log2 r_j + log2(1 + f) + rl / (rh ln 2)); table entry j holds
// (r_j, hi and lo of -log2 r_j).  |ll| < 2^-7, accurate to about 2^-31.
__device__ __forceinline__ void x2_log2_ff(float rh, float rl, const float4 *tab, float &e,
                                           float &lh, float &ll) {
  const int b = __float_as_int(rh);
  const float4 tb = tab[(b >> 16) & 127];
  const float m = __int_as_float((b & 0x007FFFFF) | 0x3F800000);
  e = (float)((b >> 23) - 127);
  const float f = fmaf(m, tb.x, -1.f);
  // ln(1 + f) = f - f^2/2 + f^3/3 - f^4/4 (next term below 2^-42)
  float q = fmaf(f, -0.25f, 1.f / 3.f);
  q = fmaf(q, f, -0.5f);
  q = fmaf(q, f, 1.f);
  q *= f;
  lh = tb.y;
  ll = fmaf(q + __fdividef(rl, rh), 1.4426950408889634f, tb.z);
}

// Table of x2_log2_ff, one entry per thread j < 128 of the block.
__device__ __forceinline__ void x2_log2_table(float4 *tab) {
  const int j = threadIdx.x;
  if (j < 128) {
    const float r = __frcp_rn(1.f + (2.f * (float)j + 1.f) * (1.f / 256.f));
    const double lg = -log2((double)r);
    const float hi = (float)lg;
    tab[j] = make_float4(r, hi, (float)(lg - (double)hi), 0.f);
  }
}

template <bool CHECK>
__device__ __forceinline__ void x2_source(const float4 &p, const float2 &u, const float2 &xab,
                                          const float2 &xcd, const float2 &yab, const float2 &ycd,
                                          float2 &acc_ab, float2 &acc_cd) {
  float2 lab, lcd;
  x2_logs<CHECK>(p, xab, xcd, yab, ycd, lab, lcd);
  acc_ab = __ffma2_rn(u, lab, acc_ab);
  acc_cd = __ffma2_rn(u, lcd, acc_cd);
}

// Error-free accumulation (Knuth's TwoSum, exact whatever the magnitudes):
// t = s + x, err = (s - (t - (t - s))) + (x - (t - s)); the errors are summed
// in e.  The sum is s + e.
__device__ __forceinline__ void x2_twosum(float2 &s, float2 &e, const float2 &x) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 t = __fadd2_rn(s, x);
  const float2 bp = __ffma2_rn(s, m1, t);    // t - s
  const float2 ap = __ffma2_rn(bp, m1, t);   // t - bp
  const float2 da = __ffma2_rn(ap, m1, s);   // s - ap
  const float2 db = __ffma2_rn(bp, m1, x);   // x - bp
  e = __fadd2_rn(e, __fadd2_rn(da, db));
  s = t;
}

// Fold x into the running sum s + e without error (TwoSum; e collects the
// rounding errors).  Used once per partial sum, so its cost does not matter.
__device__ __forceinline__ void x2_kahan(float &s, float &e, float x) {
  const float t = s + x;
  const float bp = t - s;
  const float ap = t - bp;
  e += (s - ap) + (x - bp);
  s = t;
}

// Plain form: the staged sources of a group as pair records of 48 bytes,
// rec[3j] = (-x, -x, -y, -y) of source 2j, rec[3j + 1] the same of source
// 2j + 1 and rec[3j + 2] = (u, u) of both; a thread walks a contiguous run of
// records with 32-bit shared addresses and immediate offsets, so a pair of
// sources costs three 16-byte shared loads and no index arithmetic.
constexpr uint32_t X2_REC = 48;

__device__ __forceinline__ float4 x2_lds4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a));
  return v;
}

// Records a, a + st, ... < e (shared byte addresses; st = K records for
// source slice k) against the thread's four targets; partial sums of at most
// 64 sources are folded into the compensated sums.
template <bool CHECK>
__device__ __forceinline__ void x2_pairs(uint32_t a, const uint32_t e, const uint32_t st,
                                         const float2 &xab, const float2 &xcd, const float2 &yab,
                                         const float2 &ycd, float (&s)[4], float (&c)[4]) {
  while (a < e) {
    const uint32_t be = min(e, a + 32 * st);
    // two accumulator sets (even / odd sources) halve the loop-carried FFMA chain
    float2 acc_ab = make_float2(0.f, 0.f), acc_cd = make_float2(0.f, 0.f);
    float2 acc_ab1 = make_float2(0.f, 0.f), acc_cd1 = make_float2(0.f, 0.f);
    for (; a + st < be; a += 2 * st) {
      const uint32_t b = a + st;
      const float4 x0 = x2_lds4(a), x1 = x2_lds4(a + 16), u01 = x2_lds4(a + 32);
      const float4 x2 = x2_lds4(b), x3 = x2_lds4(b + 16), u23 = x2_lds4(b + 32);
      x2_source<CHECK>(x0, make_float2(u01.x, u01.y), xab, xcd, yab, ycd, acc_ab, acc_cd);
      x2_source<CHECK>(x1, make_float2(u01.z, u01.w), xab, xcd, yab, ycd, acc_ab1, acc_cd1);
      x2_source<CHECK>(x2, make_float2(u23.x, u23.y), xab, xcd, yab, ycd, acc_ab, acc_cd);
      x2_source<CHECK>(x3, make_float2(u23.z, u23.w), xab, xcd, yab, ycd, acc_ab1, acc_cd1);
    }
    if (a < be) {
      const float4 x0 = x2_lds4(a), x1 = x2_lds4(a + 16), u01 = x2_lds4(a + 32);
      x2_source<CHECK>(x0, make_float2(u01.x, u01.y), xab, xcd, yab, ycd, acc_ab, acc_cd);
      x2_source<CHECK>(x1, make_float2(u01.z, u01.w), xab, xcd, yab, ycd, acc_ab1, acc_cd1);
      a += st;
    }
    acc_ab = __fadd2_rn(acc_ab, acc_ab1);
    acc_cd = __fadd2_rn(acc_cd, acc_cd1);
    x2_kahan(s[0], c[0], acc_ab.x);
    x2_kahan(s[1], c[1], acc_ab.y);
    x2_kahan(s[2], c[2], acc_cd.x);
    x2_kahan(s[3], c[3], acc_cd.y);
  }
}

// Hybrid precision form (COMP), staged sources q0, q0 + K, ... < q1: r^2 in
// float-float from hi + lo coordinates, log2 r^2 as
// its exact exponent plus a table-driven float-float log2 of the mantissa,
// exact products with the strength and error-free sums (TwoSum): each term
// is accurate to about 2^-31 of |u| instead of ~2^-23.
template <bool CHECK, bool COMP>
__device__ __forceinline__ void x2_slice(const float4 *sxy, const float4 *slo,
                                         const float4 *su4, const float4 *tab, int q0, int q1, int K,
                                         const float2 &xab,
                                         const float2 &xcd, const float2 &yab, const float2 &ycd,
                                         const float2 &xlab, const float2 &xlcd,
                                         const float2 &ylab, const float2 &ylcd, float (&s)[4],
                                         float (&c)[4]) {
  if constexpr (COMP) {
    float2 acc_ab = make_float2(0.f, 0.f), acc_cd = make_float2(0.f, 0.f);
    float2 nc_ab = make_float2(0.f, 0.f), nc_cd = make_float2(0.f, 0.f);
    for (int q = q0; q < q1; q += K) {
      const float4 p = sxy[q], pl = slo[q];
      const float2 px = make_float2(p.x, p.y), py = make_float2(p.z, p.w);
      const float2 pxl = make_float2(pl.x, pl.y), pyl = make_float2(pl.z, pl.w);
      float2 rh_ab, rl_ab, rh_cd, rl_cd;
      x2_r2_ff(xab, px, xlab, pxl, yab, py, ylab, pyl, rh_ab, rl_ab);
      x2_r2_ff(xcd, px, xlcd, pxl, ycd, py, ylcd, pyl, rh_cd, rl_cd);
      float e[4], lh[4], ll[4];
      x2_log2_ff(rh_ab.x, rl_ab.x, tab, e[0], lh[0], ll[0]);
      x2_log2_ff(rh_ab.y, rl_ab.y, tab, e[1], lh[1], ll[1]);
      x2_log2_ff(rh_cd.x, rl_cd.x, tab, e[2], lh[2], ll[2]);
      x2_log2_ff(rh_cd.y, rl_cd.y, tab, e[3], lh[3], ll[3]);
      if (CHECK) {   // a source on the target: no term
        const bool z[4] = {rh_ab.x == 1e-30f && rl_ab.x == 0.f, rh_ab.y == 1e-30f && rl_ab.y == 0.f,
                           rh_cd.x == 1e-30f && rl_cd.x == 0.f, rh_cd.y == 1e-30f && rl_cd.y == 0.f};
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (z[i]) e[i] = lh[i] = ll[i] = 0.f;
      }
      // u (e + lh + ll) with u = uh + ul: uh e and uh lh as exact products
      // (TwoProd), both added error-free (TwoSum); the small rest uh ll +
      // ul (e + lh) goes to the compensation
      const float4 uu = su4[q];
      const float2 uh = make_float2(uu.x, uu.y), ul = make_float2(uu.z, uu.w);
      const float2 eab = make_float2(e[0], e[1]), ecd = make_float2(e[2], e[3]);
      const float2 hab = make_float2(lh[0], lh[1]), hcd = make_float2(lh[2], lh[3]);
      const float2 lab = make_float2(ll[0], ll[1]), lcd = make_float2(ll[2], ll[3]);
      {
        const float2 p1 = __fmul2_rn(uh, eab), p2 = __fmul2_rn(uh, hab);
        const float2 r1 = __ffma2_rn(uh, eab, make_float2(-p1.x, -p1.y));
        const float2 r2 = __ffma2_rn(uh, hab, make_float2(-p2.x, -p2.y));
        x2_twosum(acc_ab, nc_ab, p1);
        x2_twosum(acc_ab, nc_ab, p2);
        const float2 rest = __ffma2_rn(uh, lab, __fmul2_rn(ul, __fadd2_rn(eab, hab)));
        nc_ab = __fadd2_rn(nc_ab, __fadd2_rn(__fadd2_rn(r1, r2), rest));
      }
      {
        const float2 p1 = __fmul2_rn(uh, ecd), p2 = __fmul2_rn(uh, hcd);
        const float2 r1 = __ffma2_rn(uh, ecd, make_float2(-p1.x, -p1.y));
        const float2 r2 = __ffma2_rn(uh, hcd, make_float2(-p2.x, -p2.y));
        x2_twosum(acc_cd, nc_cd, p1);
        x2_twosum(acc_cd, nc_cd, p2);
        const float2 rest = __ffma2_rn(uh, lcd, __fmul2_rn(ul, __fadd2_rn(ecd, hcd)));
        nc_cd = __fadd2_rn(nc_cd, __fadd2_rn(__fadd2_rn(r1, r2), rest));
      }
    }
    x2_kahan(s[0], c[0], acc_ab.x);
    x2_kahan(s[1], c[1], acc_ab.y);
    x2_kahan(s[2], c[2], acc_cd.x);
    x2_kahan(s[3], c[3], acc_cd.y);
    x2_kahan(s[0], c[0], nc_ab.x);
    x2_kahan(s[1], c[1], nc_ab.y);
    x2_kahan(s[2], c[2], nc_cd.x);
    x2_kahan(s[3], c[3], nc_cd.y);
  }
}

template <int T, bool CSR, bool COMP>
__global__ void __launch_bounds__(P2P_TH, COMP ? 2 : (CSR ? 3 : 4))
k_p2p_x2(int64_t leaf_first, int64_t n_leaves, const int *__restrict__ leaf_ids,
         const float *__restrict__ src4, const float *__restrict__ tgt, int tstride,
         const float2 *__restrict__ src_lo, const float2 *__restrict__ tgt_lo,
         const int *__restrict__ sst, const int *__restrict__ sen, const int *__restrict__ tst,
         const int *__restrict__ ten, const int *__restrict__ near_cnt,
         const int *__restrict__ near_off, const int *__restrict__ near_src,
         const double2 *__restrict__ ctr, double *__restrict__ phi_near,
         const int *__restrict__ order) {
  constexpr int CAPB = COMP ? X2_CAP_COMP : X2_CAP;
  constexpr int G = P2P_TH / T, CAP = CAPB / G;
  __shared__ float4 s_xy[COMP ? CAPB : 1];
  __shared__ float4 s_lo[COMP ? CAPB : 1];
  __shared__ float4 s_rec[COMP ? 1 : 3 * CAPB / 2];   // plain form: pair records
  __shared__ float4 s_u4[COMP ? CAPB : 1];   // (uh, uh, ul, ul): strength split in two
  __shared__ float4 s_lg[COMP ? 128 : 1];    // log2 table of the hybrid form
  __shared__ float s_red[2][4][P2P_TH];
  __shared__ int m_s0[G][NEAR_MAX], m_base[G][NEAR_MAX + 1];
  __shared__ float m_dx[G][NEAR_MAX], m_dy[G][NEAR_MAX];
  __shared__ double m_dxd[COMP ? G : 1][NEAR_MAX], m_dyd[COMP ? G : 1][NEAR_MAX];
  const int grp = threadIdx.x / T, tg = threadIdx.x % T;
  if constexpr (COMP) {
    x2_log2_table(s_lg);
    __syncthreads();
  }
  int64_t li = (int64_t)blockIdx.x * G + grp;
  if (li >= n_leaves) return;                 // group-uniform exits only
  if (order) li = order[li];                  // leaves of one size class
  const int64_t g = leaf_ids ? (int64_t)leaf_ids[li] : leaf_first + li;
  const int ts = tst[g], te = ten[g];
  if (ts >= te) return;
  // source leaves: a fixed-stride Near list (uniform tree) or a CSR list of
  // any length (adaptive tree), taken in batches of at most NEAR_MAX leaves;
  // the target's own leaf, when it holds sources, comes first
  const int n_all = CSR ? near_off[li + 1] - near_off[li] : near_cnt[li];
  const int *nall = CSR ? near_src + near_off[li] : near_src + li * NEAR_MAX;
  const bool single = !CSR || n_all <= NEAR_MAX;
  float4 *sxy = COMP ? s_xy + grp * CAP : s_xy;
  float4 *slo = COMP ? s_lo + grp * CAP : s_lo;
  float4 *srec = COMP ? s_rec : s_rec + grp * (3 * CAP / 2);
  float4 *su4 = COMP ? s_u4 + grp * CAP : s_u4;
  const float4 *src = reinterpret_cast<const float4 *>(src4);
  const double2 cg = ctr[g];
  int nn = 0, total = 0;
  auto setup = [&](int b0) {   // shift and prefix table of one batch (group-synchronous)
    nn = min(NEAR_MAX, n_all - b0);
    if (tg < nn) {
      const int sl = nall[b0 + tg];
      const double2 cs = ctr[sl];
      m_s0[grp][tg] = sst[sl];
      m_base[grp][tg + 1] = sen[sl] - sst[sl];   // counts, prefix-summed below
      m_dx[grp][tg] = (float)(cs.x - cg.x);
      m_dy[grp][tg] = (float)(cs.y - cg.y);
      if constexpr (COMP) {
        m_dxd[grp][tg] = cs.x - cg.x;
        m_dyd[grp][tg] = cs.y - cg.y;
      }
    }
    x2_sync<T>(grp);
    if (tg == 0) {
      int b = 0;
      m_base[grp][0] = 0;
      for (int e = 0; e < nn; ++e) {
        b += m_base[grp][e + 1];
        m_base[grp][e + 1] = b;
      }
    }
    x2_sync<T>(grp);
    total = m_base[grp][nn];
  };
  auto stage = [&](int c0, int c1) {
    for (int e = 0; e < nn; ++e) {
      const int b = m_base[grp][e], lo = max(b, c0), hi = min(m_base[grp][e + 1], c1);
      const int s0 = m_s0[grp][e] - b;
      const float dcx = m_dx[grp][e], dcy = m_dy[grp][e];
      for (int q = lo + tg; q < hi; q += T) {
        const float4 v = src[s0 + q];
        if constexpr (COMP) {   // the source in the target leaf's frame, as hi + lo
          const float2 vl = src_lo[s0 + q];
          const double X = ((double)v.x + (double)vl.x) + m_dxd[grp][e];
          const double Y = ((double)v.y + (double)vl.y) + m_dyd[grp][e];
          const float xh = (float)X, yh = (float)Y;
          const float xl = (float)(X - (double)xh), yl = (float)(Y - (double)yh);
          sxy[q - c0] = make_float4(-xh, -xh, -yh, -yh);
          slo[q - c0] = make_float4(-xl, -xl, -yl, -yl);
          // u = uh + ul: the FP32 value and (component 3) its rounding residual
          su4[q - c0] = make_float4(v.z, v.z, v.w, v.w);
        } else {
          const float x = -(v.x + dcx), y = -(v.y + dcy);
          const int j = (q - c0) >> 1, h = (q - c0) & 1;
          srec[3 * j + h] = make_float4(x, x, y, y);
          reinterpret_cast<float2 *>(&srec[3 * j + 2])[h] = make_float2(v.z, v.z);
        }
      }
    }
    if constexpr (!COMP) {   // an odd count: the last record's second source has u = 0
      if (tg == 0 && ((c1 - c0) & 1)) {
        const int j = (c1 - c0) >> 1;
        srec[3 * j + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float2 *>(&srec[3 * j + 2])[1] = make_float2(0.f, 0.f);
      }
    }
  };
  bool once = false;
  if (single) {
    setup(0);
    once = total <= CAP;   // all Near sources fit: stage them once
    if (once) {
      stage(0, total);
      x2_sync<T>(grp);
    }
  }
  for (int t0 = ts; t0 < te; t0 += 4 * T) {
    const int ntc = min(4 * T, te - t0);
    const int ng = (ntc + 3) / 4;          // target quadruples
    const int K = T / ng;                  // source slices per quadruple
    const int i = tg % ng, k = tg / ng;
    const bool act = k < K;
    float2 xab, xcd, yab, ycd;
    float2 xlab = make_float2(0.f, 0.f), xlcd = xlab, ylab = xlab, ylcd = xlab;
    {
      int j[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) j[r] = t0 + (i + r * ng < ntc ? i + r * ng : i);
      xab = make_float2(tgt[(int64_t)j[0] * tstride], tgt[(int64_t)j[1] * tstride]);
      yab = make_float2(tgt[(int64_t)j[0] * tstride + 1], tgt[(int64_t)j[1] * tstride + 1]);
      xcd = make_float2(tgt[(int64_t)j[2] * tstride], tgt[(int64_t)j[3] * tstride]);
      ycd = make_float2(tgt[(int64_t)j[2] * tstride + 1], tgt[(int64_t)j[3] * tstride + 1]);
      if constexpr (COMP) {
        const float2 l0 = tgt_lo[j[0]], l1 = tgt_lo[j[1]], l2 = tgt_lo[j[2]], l3 = tgt_lo[j[3]];
        xlab = make_float2(l0.x, l1.x);
        ylab = make_float2(l0.y, l1.y);
        xlcd = make_float2(l2.x, l3.x);
        ylcd = make_float2(l2.y, l3.y);
      }
    }
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int b0 = 0; b0 < n_all; b0 += NEAR_MAX) {
      if (!single) {
        x2_sync<T>(grp);   // the previous batch's table and staging are no longer read
        setup(b0);
      }
      const int n_self = (b0 == 0 && nn > 0 && nall[0] == (int)g) ? m_base[grp][1] : 0;
      for (int c0 = 0; c0 < total; c0 += CAP) {
        const int c1 = min(total, c0 + CAP);
        if (!once) {
          x2_sync<T>(grp);
          stage(c0, c1);
          x2_sync<T>(grp);
        }
        if (act) {
          const int m = c1 - c0;
          const int self_end = max(0, min(m, n_self - c0));
          if constexpr (COMP) {
            const int first_unchecked = self_end + ((k - self_end) % K + K) % K;
            if (self_end > 0)
              x2_slice<true, COMP>(sxy, slo, su4, s_lg, k, self_end, K, xab, xcd, yab, ycd, xlab,
                                   xlcd, ylab, ylcd, s, c);
            x2_slice<false, COMP>(sxy, slo, su4, s_lg, first_unchecked, m, K, xab, xcd, yab, ycd,
                                  xlab, xlcd, ylab, ylcd, s, c);
          } else {
            // slice k: records k, k + K, ...; records holding a source of
            // the target's own leaf take the coincidence check
            const int nrec = (m + 1) >> 1, rself = (self_end + 1) >> 1;
            const int ru = rself + ((k - rself) % K + K) % K;
            const uint32_t base = (uint32_t)__cvta_generic_to_shared(srec), st = K * X2_REC;
            if (k < rself)
              x2_pairs<true>(base + k * X2_REC, base + rself * X2_REC, st, xab, xcd, yab, ycd, s, c);
            x2_pairs<false>(base + ru * X2_REC, base + nrec * X2_REC, st, xab, xcd, yab, ycd, s, c);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      s_red[0][r][threadIdx.x] = act ? s[r] : 0.f;
      s_red[1][r][threadIdx.x] = act ? c[r] : 0.f;
    }
    x2_sync<T>(grp);
    if (tg < ng) {
      const int base = grp * T;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (i + r * ng >= ntc) continue;
        float S = 0.f, E = 0.f, es = 0.f;
        for (int kk = 0; kk < K; ++kk) {
          x2_kahan(S, E, s_red[0][r][base + kk * ng + i]);
          es += s_red[1][r][base + kk * ng + i];
        }
        phi_near[t0 + i + r * ng] = ((double)S + ((double)E + (double)es)) * 0.34657359027997264;  // ln2/2
      }
    }
    x2_sync<T>(grp);
  }
}

}  // namespace

template <typename R>
cudaError_t launch_p2p(int64_t leaf_first, int64_t n_leaves, const int *leaf_ids, const R *src4,
                       const R *tgt, int tstride, const int *src_start, const int *src_end,
                       const int *tgt_start, const int *tgt_end, const int *near_cnt,
                       const int *near_off, const int *near_src, const double2 *ctr,
                       double *phi_near, double mean_targets, cudaStream_t s, const float2 *src_lo,
                       const float2 *tgt_lo, const int *bin_order, const int64_t *bin_count) {
  if (n_leaves <= 0) return cudaSuccess;
  const bool comp = src_lo != nullptr;
  if constexpr (sizeof(R) == 4) {
#define X2_LAUNCH_3(TT, CS, CP)                                                                   \
  k_p2p_x2<TT, CS, CP><<<blocks, P2P_TH, 0, s>>>(leaf_first, nl, leaf_ids, src4, tgt, tstride,      \
                                                 src_lo, tgt_lo, src_start, src_end, tgt_start,    \
                                                 tgt_end, near_cnt, near_off, near_src, ctr,       \
                                                 phi_near, order)
#define X2_LAUNCH(TT)                                                                             \
  do {                                                                                            \
    if (near_off && comp) X2_LAUNCH_3(TT, true, true);                                            \
    else if (near_off) X2_LAUNCH_3(TT, true, false);                                              \
    else if (comp) X2_LAUNCH_3(TT, false, true);                                                  \
    else X2_LAUNCH_3(TT, false, false);                                                           \
  } while (0)
    auto launch_T = [&](int T, int64_t nl, const int *order) {
      const int G = P2P_TH / T;
      const unsigned blocks = (unsigned)((nl + G - 1) / G);
      if (T == 32) X2_LAUNCH(32);
      else if (T == 64) X2_LAUNCH(64);
      else if (T == 128) X2_LAUNCH(128);
      else X2_LAUNCH(256);
    };
#undef X2_LAUNCH
#undef X2_LAUNCH_3
    if (bin_order && bin_count) {
      // leaves binned by their own target count (p2p_size_class): one launch
      // per class with that class's group size
      int64_t off = 0;
      for (int c = 0; c < 4; ++c) {
        if (bin_count[c] > 0) launch_T(32 << c, bin_count[c], bin_order + off);
        off += bin_count[c];
      }
    } else {
      // group size: the smallest T for which a leaf of mean + 2 sigma (Poisson)
      // targets still gets about three source slices per target quadruple (so
      // that a group's lanes stay busy whatever the leaf's exact size)
      const double want = 0.75 * (mean_targets + 2.0 * sqrt(mean_targets));
      launch_T(want <= 32 ? 32 : want <= 64 ? 64 : want <= 128 ? 128 : 256, n_leaves, nullptr);
    }
  } else if (mean_targets >= 48.0 && !near_off) {   // FP64, large leaves: block-staged
    k_p2p_block<R><<<(unsigned)n_leaves, P2P_TH, 0, s>>>(leaf_first, src4, tgt, tstride, src_start,
                                                         src_end, tgt_start, tgt_end, near_cnt,
                                                         near_src, ctr, phi_near);
  } else {                             // FP64, small leaves or CSR lists: one warp per leaf
    const unsigned blocks = (unsigned)((n_leaves * 32 + P2P_TH - 1) / P2P_TH);
    k_p2p<R><<<blocks, P2P_TH, 0, s>>>(leaf_first, n_leaves, leaf_ids, src4, tgt, tstride,
                                        src_start, src_end, tgt_start, tgt_end, near_cnt, near_off,
                                        near_src, ctr, phi_near);
  }
  return cudaGetLastError();
}

namespace {
// Size class of a leaf with nt targets: the group size T = 32 << class is the
// smallest of 32 ... 256 with T >= 3 nt / 4, so a target quadruple gets about
// three source slices.  It depends on the leaf alone.
__device__ __forceinline__ int p2p_size_class(int nt) {
  return 3 * nt <= 128 ? 0 : (3 * nt <= 256 ? 1 : (3 * nt <= 512 ? 2 : 3));
}

// One atomic per warp and class: the lanes of a class are counted by ballot
// (all lanes of every warp take part; those past the end have no class).
__global__ void k_p2p_bin_count(int64_t n_leaves, const int *__restrict__ leaf_ids,
                                const int *__restrict__ ts, const int *__restrict__ te,
                                int *__restrict__ cnt) {
  const int64_t li = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int c = -1;
  if (li < n_leaves) {
    const int g = leaf_ids[li];
    c = p2p_size_class(te[g] - ts[g]);
  }
  for (int k = 0; k < 4; ++k) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, c == k);
    if (m != 0u && lane == __ffs(m) - 1) atomicAdd(&cnt[k], __popc(m));
  }
}

// order[off_c + j] = leaf position li (the order inside a class does not
// matter: every leaf's sum is computed on its own); a warp reserves the
// slots of its lanes of each class with one atomic
__global__ void k_p2p_bin_scatter(int64_t n_leaves, const int *__restrict__ leaf_ids,
                                  const int *__restrict__ ts, const int *__restrict__ te,
                                  int *__restrict__ cnt, int *__restrict__ order) {
  const int64_t li = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int c = -1;
  if (li < n_leaves) {
    const int g = leaf_ids[li];
    c = p2p_size_class(te[g] - ts[g]);
  }
  int off = 0;
  for (int k = 0; k < 4; ++k) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, c == k);
    if (m != 0u) {   // warp-uniform
      const int leader = __ffs(m) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(&cnt[4 + k], __popc(m));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      if (c == k) order[off + base + __popc(m & ((1u << lane) - 1u))] = (int)li;
    }
    off += cnt[k];
  }
}
}  // namespace

cudaError_t launch_p2p_bins(int64_t n_leaves, const int *leaf_ids, const int *ts, const int *te,
                            int *cnt8, int *order, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cnt8, 0, 8 * sizeof(int), s);
  if (e != cudaSuccess || n_leaves <= 0) return e;
  const unsigned blocks = (unsigned)((n_leaves + 255) / 256);
  k_p2p_bin_count<<<blocks, 256, 0, s>>>(n_leaves, leaf_ids, ts, te, cnt8);
  k_p2p_bin_scatter<<<blocks, 256, 0, s>>>(n_leaves, leaf_ids, ts, te, cnt8, order);
  return cudaGetLastError();
}

template cudaError_t launch_p2p<float>(int64_t, int64_t, const int *, const float *,
                                       const float *, int, const int *, const int *, const int *,
                                       const int *, const int *, const int *, const int *,
                                       const double2 *, double *, double, cudaStream_t,
                                       const float2 *, const float2 *, const int *, const int64_t *);
template cudaError_t launch_p2p<double>(int64_t, int64_t, const int *, const double *,
                                        const double *, int, const int *, const int *, const int *,
                                        const int *, const int *, const int *, const int *,
                                        const double2 *, double *, double, cudaStream_t,
                                        const float2 *, const float2 *, const int *, const int64_t *);

}  // namespace fmm2d
