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

template <typename T>
__global__ void k_keys_quad(const T *__restrict__ xy, int64_t n, double x0, double y0, double S,
                            int L, uint32_t *__restrict__ key, uint32_t *__restrict__ iota,
                            int *err) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
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
}

template <typename T>
__global__ void k_keys_sept(const T *__restrict__ xy, int64_t n, double x0, double y0, double S,
                            int L, double r, uint32_t *__restrict__ key, uint32_t *__restrict__ iota,
                            int *err) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
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
}

template <typename T>
__global__ void k_keys_tri(const T *__restrict__ xy, int64_t n, double x0, double y0, double S,
                           int L, double rho0, uint32_t *__restrict__ key,
                           uint32_t *__restrict__ iota, int *err) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
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
}

template <typename T>
cudaError_t keys_t(const Geo &g, const T *xy, int64_t n, uint32_t *key, uint32_t *iota, int *err,
                   cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int th = 256;
  const unsigned blocks = (unsigned)((n + th - 1) / th);
  if (g.tiling == FMM2D_QUAD)
    k_keys_quad<T><<<blocks, th, 0, s>>>(xy, n, g.x0, g.y0, g.S, g.L, key, iota, err);
  else if (g.tiling == FMM2D_SEPT)
    k_keys_sept<T><<<blocks, th, 0, s>>>(xy, n, g.x0, g.y0, g.S, g.L, g.leaf_scale, key, iota, err);
  else
    k_keys_tri<T><<<blocks, th, 0, s>>>(xy, n, g.x0, g.y0, g.S, g.L, g.leaf_scale, key, iota, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_keys(const Geo &g, const void *xy, bool f32, int64_t n, uint32_t *key,
                        uint32_t *perm_iota, int *err, cudaStream_t s) {
  if (f32) return keys_t<float>(g, (const float *)xy, n, key, perm_iota, err, s);
  return keys_t<double>(g, (const double *)xy, n, key, perm_iota, err, s);
}

}  // namespace fmm2d
