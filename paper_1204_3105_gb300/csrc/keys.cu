// keys.cu - CellIndex of every point (Sec. 4-6) as an integer leaf key.
//
// The floating-point front end is FP64 with every operation explicitly
// rounded (__dadd_rn & co.: no FMA contraction), so a key is a deterministic
// function of the input point.  After it the work is integer only.
//  * quadtree: Morton key of (floor(tx 2^L), floor(ty 2^L)), t = (x - x0)/S.
//  * septree (Sec. 5, CellIndex steps 1-6): change of basis (eq. 7), the four
//    candidate lattice points (eq. 9) mapped back with eq. (8), nearest one
//    by squared distance (first candidate kept on ties), then the GBT index
//    of the lattice point b + c w as its base-beta digit string.
//  * triangle quadtree (Sec. 6, CellIndex): top-down descent into the child
//    whose corner holds barycentric coordinate > 1/2 (else the centre child),
//    done exactly on 2^-60 fixed-point barycentric coordinates; this is the
//    nearest-of-four lattice search of eq. (13) (the children's centroids
//    are the Voronoi sites of the children inside the parent).
#include <algorithm>
#include <cmath>

#include "plan.h"

namespace fmm2d {

namespace {

constexpr double kSqrt3 = 1.7320508075688772;   // sqrt(3) rounded to double

template <typename T>
__device__ __forceinline__ void load_xy(const T *xy, int64_t i, double &x, double &y) {
  x = (double)xy[2 * i];
  y = (double)xy[2 * i + 1];
}

__device__ __forceinline__ bool frame_t(double x, double y, double x0, double y0, double S,
                                        double &tx, double &ty) {
  tx = __ddiv_rn(__dsub_rn(x, x0), S);
  ty = __ddiv_rn(__dsub_rn(y, y0), S);
  return tx >= 0.0 && tx < 1.0 && ty >= 0.0 && ty < 1.0;
}

// Exact kernels: every point, or (list != null) only the *list_n points of
// list, with a grid-stride loop.
#define EXACT_LOOP_BEGIN                                                                          \
  const int64_t n_work = list ? (int64_t)*list_n : n;                                             \
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n_work;                    \
       w += (int64_t)gridDim.x * blockDim.x) {                                                    \
    const int64_t i = list ? (int64_t)list[w] : w;
#define EXACT_LOOP_END }

template <typename T>
__global__ void k_keys_quad(const T *__restrict__ xy, int64_t n, double x0, double y0, double S,
                            int L, uint32_t *__restrict__ key, uint32_t *__restrict__ iota,
                            int *err, const uint32_t *__restrict__ list, const int *__restrict__ list_n) {
  EXACT_LOOP_BEGIN
  double x, y, tx, ty;
  load_xy(xy, i, x, y);
  uint32_t k = 0;
  if (!frame_t(x, y, x0, y0, S, tx, ty)) {
    atomicOr(err, 1);
  } else {
    double sc = (double)(1u << L);
    uint32_t ci = (uint32_t)floor(__dmul_rn(tx, sc));
    uint32_t cj = (uint32_t)floor(__dmul_rn(ty, sc));
    k = morton(ci, cj);
  }
  key[i] = k;
  if (iota) iota[i] = (uint32_t)i;
  EXACT_LOOP_END
}

template <typename T>
__global__ void k_keys_sept(const T *__restrict__ xy, int64_t n, double x0, double y0, double S,
                            int L, double r, uint32_t *__restrict__ key, uint32_t *__restrict__ iota,
                            int *err, const uint32_t *__restrict__ list, const int *__restrict__ list_n) {
  EXACT_LOOP_BEGIN
  double x, y, tx, ty;
  load_xy(xy, i, x, y);
  uint32_t k = 0;
  if (!frame_t(x, y, x0, y0, S, tx, ty)) {
    atomicOr(err, 1);
  } else {
    const double X = __dsub_rn(tx, 0.5), Y = __dsub_rn(ty, 0.5);
    const double k3r = __dmul_rn(3.0, r), rs3 = __dmul_rn(r, kSqrt3);
    const double b = __ddiv_rn(__dmul_rn(2.0, X), k3r);
    const double c = __ddiv_rn(__dsub_rn(__dmul_rn(Y, kSqrt3), X), k3r);
    const double fb = floor(b), cb = ceil(b), fc = floor(c), cc = ceil(c);
    const double cand_b[4] = {fb, cb, fb, cb};
    const double cand_c[4] = {fc, fc, cc, cc};
    double best = 0.0, bb = 0.0, bc = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double xh = __dmul_rn(__dmul_rn(k3r, cand_b[q]), 0.5);
      double yh = __dmul_rn(__dmul_rn(rs3, __dadd_rn(__dmul_rn(2.0, cand_c[q]), cand_b[q])), 0.5);
      double dx = __dsub_rn(X, xh), dy = __dsub_rn(Y, yh);
      double d = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      if (q == 0 || d < best) {
        best = d;
        bb = cand_b[q];
        bc = cand_c[q];
      }
    }
    if (!eis_to_key((int64_t)bb, (int64_t)bc, L, &k)) {
      atomicOr(err, 2);
      k = 0;
    }
  }
  key[i] = k;
  if (iota) iota[i] = (uint32_t)i;
  EXACT_LOOP_END
}

template <typename T>
__global__ void k_keys_tri(const T *__restrict__ xy, int64_t n, double x0, double y0, double S,
                           int L, double rho0, uint32_t *__restrict__ key,
                           uint32_t *__restrict__ iota, int *err, const uint32_t *__restrict__ list,
                           const int *__restrict__ list_n) {
  EXACT_LOOP_BEGIN
  double x, y, tx, ty;
  load_xy(xy, i, x, y);
  uint32_t k = 0;
  if (!frame_t(x, y, x0, y0, S, tx, ty)) {
    atomicOr(err, 1);
  } else {
    const double X = __dsub_rn(tx, 0.5), Y = __dsub_rn(ty, 0.5);
    const double k3 = __dmul_rn(3.0, rho0);
    const double half3 = __dmul_rn(kSqrt3, 0.5);
    const double av = __ddiv_rn(__dadd_rn(Y, rho0), k3);
    const double al = __ddiv_rn(__dsub_rn(__dsub_rn(rho0, __dmul_rn(half3, X)), __dmul_rn(0.5, Y)), k3);
    const int64_t ONE = (int64_t)1 << 60, HALF = (int64_t)1 << 59;
    int64_t AV = (int64_t)floor(__dmul_rn(av, 1152921504606846976.0));
    int64_t AL = (int64_t)floor(__dmul_rn(al, 1152921504606846976.0));
    int64_t AR = ONE - AV - AL;
    if (AV < 0 || AL < 0 || AR < 0) {
      atomicOr(err, 4);
    } else {
      for (int m = 0; m < L; ++m) {
        uint32_t d;
        int64_t nv, nl, nr;
        if (AV > HALF) {
          d = 1; nv = 2 * AV - ONE; nl = 2 * AL; nr = 2 * AR;
        } else if (AL > HALF) {
          d = 2; nv = 2 * AV; nl = 2 * AL - ONE; nr = 2 * AR;
        } else if (AR > HALF) {
          d = 3; nv = 2 * AV; nl = 2 * AL; nr = 2 * AR - ONE;
        } else {
          d = 0; nv = ONE - 2 * AV; nl = ONE - 2 * AR; nr = ONE - 2 * AL;
        }
        AV = nv; AL = nl; AR = nr;
        k = (k << 2) | d;
      }
    }
  }
  key[i] = k;
  if (iota) iota[i] = (uint32_t)i;
  EXACT_LOOP_END
}

// ---- FP32 filter ----------------------------------------------------------
// Every decision of the exact front end (domain test, floor, nearest of four,
// descent step) is a comparison of a computed value with a threshold.  The
// filter computes the same values in FP32 together with a proven bound on
// their distance from the exact FP64 values (from the input rounding eX and
// the FP32 operation count); when every comparison clears its threshold by
// more than that bound, the FP64 front end takes the same decisions, so the
// key is the same.  Otherwise the point is queued for the exact kernel.
struct KeyFilter {
  float x0, y0, inv_s;     // frame map in FP32
  float eX;                // bound on |X32 - X64| (frame coordinates)
  float c1, c2, c3;        // per tiling (see the kernels)
  float d1, d2;            // decision margins
};

__device__ __forceinline__ void queue_exact(int64_t i, uint32_t *list, int *list_n) {
  const int at = atomicAdd(list_n, 1);
  list[at] = (uint32_t)i;
}

template <typename T>
__global__ void k_keys_fast(const T *__restrict__ xy, int64_t n, int tiling, int L, KeyFilter f,
                            uint32_t *__restrict__ key, uint32_t *__restrict__ iota,
                            uint32_t *__restrict__ list, int *__restrict__ list_n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (iota) iota[i] = (uint32_t)i;
  const float x = (float)xy[2 * i], y = (float)xy[2 * i + 1];
  const float tx = (x - f.x0) * f.inv_s, ty = (y - f.y0) * f.inv_s;
  const float et = f.eX;
  if (!(tx > et && tx < 1.f - et && ty > et && ty < 1.f - et)) {   // near or outside the edge
    queue_exact(i, list, list_n);
    return;
  }
  uint32_t k = 0;
  if (tiling == FMM2D_QUAD) {
    // c1 = 2^L; d1 = margin on the fractional part of t 2^L
    const float u = tx * f.c1, v = ty * f.c1;
    const float fu = floorf(u), fv = floorf(v);
    if (u - fu < f.d1 || fu + 1.f - u < f.d1 || v - fv < f.d1 || fv + 1.f - v < f.d1) {
      queue_exact(i, list, list_n);
      return;
    }
    k = morton((uint32_t)fu, (uint32_t)fv);
  } else if (tiling == FMM2D_SEPT) {
    // c1 = 1/(3r), c2 = 3r, c3 = r sqrt3; d1 = margin on frac(b), frac(c);
    // d2 = margin on squared distances
    const float X = tx - 0.5f, Y = ty - 0.5f;
    const float b = 2.f * X * f.c1, c = (Y * 1.7320508f - X) * f.c1;
    const float fb = floorf(b), fc = floorf(c);
    if (b - fb < f.d1 || fb + 1.f - b < f.d1 || c - fc < f.d1 || fc + 1.f - c < f.d1) {
      queue_exact(i, list, list_n);
      return;
    }
    float best = 0.f, second = 3.4e38f;
    int q_best = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float cb = fb + (float)(q & 1), cc = fc + (float)(q >> 1);
      const float xh = 0.5f * f.c2 * cb, yh = 0.5f * f.c3 * (2.f * cc + cb);
      const float dx = X - xh, dy = Y - yh;
      const float d = dx * dx + dy * dy;
      if (q == 0) {
        best = d;
      } else if (d < best) {
        second = best;
        best = d;
        q_best = q;
      } else if (d < second) {
        second = d;
      }
    }
    if (second - best < f.d2) {
      queue_exact(i, list, list_n);
      return;
    }
    // |fb|, |fc| <= 2.8 / (3 r) + 1, far below 2^27 for any supported depth
    const int bb = (int)fb + (q_best & 1), bc = (int)fc + (q_best >> 1);
    if (!eis_to_key32(bb, bc, L, &k)) {   // outside the root: the exact kernel reports it
      queue_exact(i, list, list_n);
      return;
    }
  } else {
    // c1 = 1/(3 rho0), c2 = rho0; d1 = margin on the descent comparisons at
    // level 0 (doubled every level)
    const float X = tx - 0.5f, Y = ty - 0.5f;
    float av = (Y + f.c2) * f.c1;
    float al = (f.c2 - 0.8660254f * X - 0.5f * Y) * f.c1;
    float ar = 1.f - av - al;
    float m = f.d1;
    if (av < m || al < m || ar < m) {
      queue_exact(i, list, list_n);
      return;
    }
    for (int lv = 0; lv < L; ++lv) {
      if (fabsf(av - 0.5f) < m || fabsf(al - 0.5f) < m || fabsf(ar - 0.5f) < m) {
        queue_exact(i, list, list_n);
        return;
      }
      uint32_t d;
      float nv, nl, nr;
      if (av > 0.5f) {
        d = 1; nv = 2.f * av - 1.f; nl = 2.f * al; nr = 2.f * ar;
      } else if (al > 0.5f) {
        d = 2; nv = 2.f * av; nl = 2.f * al - 1.f; nr = 2.f * ar;
      } else if (ar > 0.5f) {
        d = 3; nv = 2.f * av; nl = 2.f * al; nr = 2.f * ar - 1.f;
      } else {
        d = 0; nv = 1.f - 2.f * av; nl = 1.f - 2.f * ar; nr = 1.f - 2.f * al;
      }
      av = nv; al = nl; ar = nr;
      m *= 2.f;
      k = (k << 2) | d;
    }
  }
  key[i] = k;
}

// FP32 filter parameters with their error bounds; false when the frame map
// is too ill-conditioned in FP32 for the filter to pay (then every point goes
// through the exact kernel).
static bool make_filter(const Geo &g, bool f32_in, KeyFilter *f) {
  const double u = 1.0 / 16777216.0;   // 2^-24
  const double ax = std::max(std::fabs(g.x0), std::fabs(g.y0)) / g.S;
  // |t32 - t64|: input rounding to FP32 (FP64 inputs), x0 and 1/S rounding,
  // subtraction and product rounding, with a factor 2 of slack
  const double et = 2.0 * u * ((f32_in ? 1.0 : 2.0) * ax + 6.0);
  if (!(et < 1e-4)) return false;
  f->x0 = (float)g.x0;
  f->y0 = (float)g.y0;
  f->inv_s = (float)(1.0 / g.S);
  f->eX = (float)(2.0 * et);
  const double eX = et + u;            // X = t - 1/2 adds one rounding
  if (g.tiling == FMM2D_QUAD) {
    const double sc = std::ldexp(1.0, g.L);
    f->c1 = (float)sc;
    f->d1 = (float)(4.0 * (eX * sc + 2.0 * u * sc));
    if (!(f->d1 < 0.25f)) return false;
  } else if (g.tiling == FMM2D_SEPT) {
    const double k3r = 3.0 * g.leaf_scale, inv = 1.0 / k3r;
    f->c1 = (float)inv;
    f->c2 = (float)k3r;
    f->c3 = (float)(g.leaf_scale * 1.7320508075688772);
    const double bmax = 2.8 * inv;     // |b|, |c| <= (1 + sqrt3) max|X| / (3r)
    f->d1 = (float)(4.0 * (2.8 * eX * inv + 6.0 * u * bmax));
    // |d32 - d64| <= 2 |dx| e_dx + 2 |dy| e_dy + 4 u d, |dx|, |dy| <= 2r,
    // e_dx <= eX + 4 u (|xh| <= 0.6)
    const double edx = eX + 4.0 * u * 0.6;
    f->d2 = (float)(4.0 * (2.0 * (8.0 * g.leaf_scale * edx + 4.0 * u * 8.0 * g.leaf_scale * g.leaf_scale)));
    if (!(f->d1 < 0.25f)) return false;
  } else {
    const double rho0 = g.leaf_scale, inv = 1.0 / (3.0 * rho0);
    f->c1 = (float)inv;
    f->c2 = (float)rho0;
    // barycentrics: |a32 - a64| <= 2 eX / (3 rho0) + 8 u; the exact side
    // truncates to 2^-60 (negligible); a descent step doubles the error
    f->d1 = (float)(4.0 * (2.0 * eX * inv + 8.0 * u));
    if (!(std::ldexp((double)f->d1, g.L) < 0.25)) return false;
  }
  return true;
}

template <typename T>
cudaError_t keys_t(const Geo &g, const T *xy, int64_t n, uint32_t *key, uint32_t *iota, int *err,
                   uint32_t *list, int *list_n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int th = 256;
  const unsigned blocks = (unsigned)((n + th - 1) / th);
  KeyFilter f{};
  const bool filt = list && list_n && make_filter(g, sizeof(T) == 4, &f);
  unsigned eblocks = blocks;
  if (filt) {
    cudaError_t e = cudaMemsetAsync(list_n, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_keys_fast<T><<<blocks, th, 0, s>>>(xy, n, g.tiling, g.L, f, key, iota, list, list_n);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    eblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sms * 4));
  } else {
    list = nullptr;
    list_n = nullptr;
  }
  if (g.tiling == FMM2D_QUAD)
    k_keys_quad<T><<<eblocks, th, 0, s>>>(xy, n, g.x0, g.y0, g.S, g.L, key, iota, err, list, list_n);
  else if (g.tiling == FMM2D_SEPT)
    k_keys_sept<T><<<eblocks, th, 0, s>>>(xy, n, g.x0, g.y0, g.S, g.L, g.leaf_scale, key, iota, err,
                                          list, list_n);
  else
    k_keys_tri<T><<<eblocks, th, 0, s>>>(xy, n, g.x0, g.y0, g.S, g.L, g.leaf_scale, key, iota, err,
                                         list, list_n);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_keys(const Geo &g, const void *xy, bool f32, int64_t n, uint32_t *key,
                        uint32_t *perm_iota, int *err, cudaStream_t s, uint32_t *list, int *list_n) {
  if (f32) return keys_t<float>(g, (const float *)xy, n, key, perm_iota, err, list, list_n, s);
  return keys_t<double>(g, (const double *)xy, n, key, perm_iota, err, list, list_n, s);
}

}  // namespace fmm2d
