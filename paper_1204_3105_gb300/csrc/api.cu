// api.cu - the C ABI of libfmm2d (include/fmm2d.h): planner rules, per-plan
// stencils and operator tables, and the orchestration of build / evaluate.
// Host code only; every numerical step of the FMM runs in the kernels of
// keys.cu, sort.cu, tree.cu, expand.cu and p2p.cu.
#include <algorithm>
#include <climits>
#include <cmath>
#include <complex>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "plan.h"

struct fmm2d_plan : public fmm2d::Plan {};

namespace fmm2d {

using cd = std::complex<double>;

static thread_local std::string g_create_err;
static const double kSqrt3 = std::sqrt(3.0);

cudaError_t dbuf_reserve(DBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}
void dbuf_free(DBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// Grow a buffer to at least `bytes`, keeping its first `keep` bytes.
static cudaError_t dbuf_grow_keep(DBuf &b, size_t bytes, size_t keep, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return cudaSuccess;
  const size_t nb = std::max(bytes, b.bytes + b.bytes / 2);
  void *np = nullptr;
  cudaError_t e = cudaMalloc(&np, nb);
  if (e != cudaSuccess) return e;
  if (b.p && keep > 0) {
    e = cudaMemcpyAsync(np, b.p, std::min(keep, b.bytes), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaFree(np);
      return e;
    }
  }
  if (b.p) cudaFree(b.p);
  b.p = np;
  b.bytes = nb;
  return cudaSuccess;
}

// ------------------------------------------------------------ planner rules
static int64_t sept_min_outside_norm(int L) {
  static std::mutex mu;
  static std::map<int, int64_t> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(L);
  if (it != cache.end()) return it->second;
  const int R = (int)(0.6 * std::pow(7.0, L / 2.0)) + 4;
  // rows a of the (2R+1)^2 window split over host threads (the window holds
  // ~6e7 points at L = 9); each thread keeps its own minimum
  const int nth = R > 64 ? (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())) : 1;
  std::vector<int64_t> part(nth, INT64_MAX);
  auto scan = [&](int t) {
    int64_t best = INT64_MAX;
    for (int a = -R + t; a <= R; a += nth)
      for (int b = -R; b <= R; ++b) {
        const int64_t n = (int64_t)a * a + (int64_t)a * b + (int64_t)b * b;
        if (n >= best) continue;
        uint32_t k;
        if (!eis_to_key(a, b, L, &k)) best = n;
      }
    part[t] = best;
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nth; ++t) th.emplace_back(scan, t);
  scan(0);
  for (auto &x : th) x.join();
  const int64_t best = *std::min_element(part.begin(), part.end());
  cache[L] = best;
  return best;
}

// Deepest septree level whose minimal outside norm m_L is enumerated (about
// 6e7 lattice points); deeper levels use the lower bound below.
constexpr int SEPT_ENUM_LEVELS = 9;

// sqrt(m_L), or for L > SEPT_ENUM_LEVELS a lower bound of it: a point z
// outside the (L+1)-digit region, z = d (mod beta), has (z - unit_d) / beta
// outside the L-digit region, so |z| >= sqrt7 sqrt(m_L) - 1.  The recursion
// from the enumerated level, less 1e-9 per step for rounding, stays below the
// true value, which only makes the leaf radius larger (still covering).
static double sept_root_norm(int L) {
  if (L <= SEPT_ENUM_LEVELS) return std::sqrt((double)sept_min_outside_norm(L));
  double m = std::sqrt((double)sept_min_outside_norm(SEPT_ENUM_LEVELS));
  for (int l = SEPT_ENUM_LEVELS; l < L; ++l) m = std::sqrt(7.0) * m - 1.0 - 1e-9;
  return m;
}

// Septree leaf circumradius r_L: every point of the frame square (inside the
// disc of radius sqrt(1/2)) has its nearest leaf-lattice point (spacing r
// sqrt3, covering radius r) inside the L-digit GBT region.
double sept_leaf_r(int L) {
  const double m = sept_root_norm(L);
  double raw = std::sqrt(0.5) / (kSqrt3 * m - 1.0);
  return std::ceil(raw * 1099511627776.0) / 1099511627776.0;   // 2^40
}

// The septree leaf radii of every level an adaptive tree may reach (a few
// tenths of a second of host work at the deepest enumerated level, then
// cached).
void planner_precompute() {
  for (int L = 1; L <= SEPT_ENUM_LEVELS; ++L) sept_leaf_r(L);
}

// Triangle root inradius: the upright triangle centred at the origin that
// contains the frame square [-1/2, 1/2)^2, widened by 2^-20.
double tri_rho0() { return (kSqrt3 + 1.0) / 4.0 * (1.0 + std::ldexp(1.0, -20)); }

static double kappa(int tiling) {
  if (tiling == FMM2D_QUAD) return 1.0 / (1.0 + 2.0 * (std::sqrt(2.0) - 1.0));
  if (tiling == FMM2D_SEPT) return 0.525;
  return 1.0 / (1.0 + (std::sqrt(7.0) - 2.0));
}

static int max_levels(int tiling) { return tiling == FMM2D_SEPT ? 9 : 12; }
// adaptive trees: keys of the finest level fit 32 bits (quadtree and triangle
// quadtree: 2 bits a level; septree: 7^11 < 2^32)
static int ad_max_levels(int tiling) { return tiling == FMM2D_SEPT ? 11 : 16; }
static int max_levels_for(int tiling, unsigned flags) {
  return (flags & FMM2D_ADAPTIVE) ? ad_max_levels(tiling) : max_levels(tiling);
}

static double leaf_area(int tiling, int L) {
  if (tiling == FMM2D_QUAD) return std::pow(4.0, -L);
  if (tiling == FMM2D_TRI) {
    double rho0 = tri_rho0();
    return 3.0 * kSqrt3 * rho0 * rho0 / std::pow(4.0, L);
  }
  double r = sept_leaf_r(L);
  return 1.5 * kSqrt3 * r * r;
}

static int auto_levels(int tiling, int64_t n, int leaf_target) {
  int top = tiling == FMM2D_SEPT ? 8 : 12;
  for (int L = 1; L <= top; ++L)
    if ((double)n * leaf_area(tiling, L) <= (double)leaf_target) return L;
  return top;
}

// S_opt of Table 2 (App. A-C): the leaf level whose expected sources per
// leaf s_L = N leaf_area(L) minimise the s-dependent FMM cost
// (N / s) b/(b-1) (P4 + 2) p^2 + M P2 s (M2L work of N / s leaves against
// the direct work of M targets), P4 = 27 / 42 / 39 and P2 = 9 / 7 / 13.
int planner_sopt_levels(int tiling, int64_t n_src, int64_t n_tgt, int p) {
  const double P4 = tiling == FMM2D_QUAD ? 27.0 : tiling == FMM2D_SEPT ? 42.0 : 39.0;
  const double P2 = tiling == FMM2D_QUAD ? 9.0 : tiling == FMM2D_SEPT ? 7.0 : 13.0;
  const double b = tiling == FMM2D_SEPT ? 7.0 : 4.0;
  const double N = (double)std::max<int64_t>(1, n_src), M = (double)std::max<int64_t>(1, n_tgt);
  const double m2l = b / (b - 1.0) * (P4 + 2.0) * (double)p * (double)p;
  const int top = tiling == FMM2D_SEPT ? 8 : 12;
  int best_l = 1;
  double best = 0.0;
  for (int L = 1; L <= top; ++L) {
    const double sl = N * leaf_area(tiling, L);
    const double c = N / sl * m2l + M * P2 * sl;
    if (L == 1 || c < best) {
      best = c;
      best_l = L;
    }
  }
  return best_l;
}

static int p_from_eps(int tiling, double eps) {
  int p = (int)std::ceil(std::log(eps) / std::log(kappa(tiling))) - 1;
  return std::max(1, p);
}

static int key_bits(int tiling, int L) {
  if (tiling != FMM2D_SEPT) return 2 * L;
  uint64_t v = 1;
  for (int i = 0; i < L; ++i) v *= 7;
  int b = 0;
  while ((1ull << b) < v) ++b;
  return b;
}

// ------------------------------------------------------------ stencils
struct I3 { int a, b, c; };
static bool operator==(const I3 &x, const I3 &y) { return x.a == y.a && x.b == y.b && x.c == y.c; }

static std::vector<I3> tri_near(I3 c, int l) {
  bool up = tri_up(c.a, c.b, c.c, l);
  I3 v[3];
  if (up) v[0] = {c.a + 1, c.b, c.c}, v[1] = {c.a, c.b + 1, c.c}, v[2] = {c.a, c.b, c.c + 1};
  else v[0] = {c.a, c.b + 1, c.c + 1}, v[1] = {c.a + 1, c.b, c.c + 1}, v[2] = {c.a + 1, c.b + 1, c.c};
  std::vector<I3> out;
  for (auto &x : v) {
    I3 t[6] = {{x.a - 1, x.b, x.c}, {x.a, x.b - 1, x.c}, {x.a, x.b, x.c - 1},
               {x.a - 1, x.b - 1, x.c}, {x.a - 1, x.b, x.c - 1}, {x.a, x.b - 1, x.c - 1}};
    for (auto &y : t)
      if (std::find(out.begin(), out.end(), y) == out.end()) out.push_back(y);
  }
  return out;
}
static I3 tri_child3(I3 p, int l, int t) {
  I3 c;
  tri_child(p.a, p.b, p.c, tri_up(p.a, p.b, p.c, l), t, &c.a, &c.b, &c.c);
  return c;
}

struct OpKey { int u, v; bool operator<(const OpKey &o) const { return u != o.u ? u < o.u : v < o.v; } };

struct Tables {
  Stencils st;
  std::vector<cd> zeta;          // per M2L operator
  std::vector<cd> cw, csig;      // per child class: w and sigma of M2M / L2L
  int n_classes;
};

static void add_far(Tables &T, int cls, I3 d, OpKey key, cd z, std::map<OpKey, int> &ids) {
  auto it = ids.find(key);
  int id;
  if (it == ids.end()) {
    id = (int)T.zeta.size();
    ids[key] = id;
    T.zeta.push_back(z);
  } else {
    id = it->second;
  }
  int e = T.st.far_len[cls]++;
  T.st.far_d[cls][e][0] = d.a;
  T.st.far_d[cls][e][1] = d.b;
  T.st.far_d[cls][e][2] = d.c;
  T.st.far_op[cls][e] = (uint16_t)id;
}

static Tables make_tables(int tiling) {
  Tables T;
  std::memset(&T.st, 0, sizeof(T.st));
  std::map<OpKey, int> ids;
  const double s2 = std::sqrt(2.0);
  if (tiling == FMM2D_QUAD) {
    T.n_classes = 4;
    for (int d = 0; d < 4; ++d) {
      int bx = d & 1, by = d >> 1, ci = 32 + bx, cj = 32 + by;
      for (int dpj = -1; dpj <= 1; ++dpj)
        for (int dpi = -1; dpi <= 1; ++dpi)
          for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
              int di = 2 * (16 + dpi) + cx - ci, dj = 2 * (16 + dpj) + cy - cj;
              if (std::abs(di) <= 1 && std::abs(dj) <= 1) continue;
              add_far(T, d, {di, dj, 0}, {di, dj}, s2 * cd(di, dj), ids);
            }
      T.cw.push_back(cd(bx - 0.5, by - 0.5) / s2);
      T.csig.push_back(cd(0.5, 0));
    }
    // Near stencil: the leaf itself first (the P2P kernel relies on it)
    T.st.near_len[0] = 1;
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        if (di == 0 && dj == 0) continue;
        int e = T.st.near_len[0]++;
        T.st.near_d[0][e][0] = di;
        T.st.near_d[0][e][1] = dj;
      }
  } else if (tiling == FMM2D_SEPT) {
    T.n_classes = 7;
    const cd w6(0.5, kSqrt3 / 2), beta(2.0, kSqrt3);
    auto unit = [](int d) { return I3{unit_a(d), unit_b(d), 0}; };
    auto is_near = [&](I3 x) {
      for (int d = 0; d < 7; ++d)
        if (x.a == unit_a(d) && x.b == unit_b(d)) return true;
      return false;
    };
    for (int d = 0; d < 7; ++d) {
      I3 E = unit(d);   // a level-l cell whose parent is the origin
      for (int dp = 0; dp < 7; ++dp) {
        I3 P = unit(dp);
        I3 BP = {P.a - 2 * P.b, 2 * P.a + 3 * P.b, 0};   // beta * P
        for (int d2 = 0; d2 < 7; ++d2) {
          I3 ch = {BP.a + unit_a(d2), BP.b + unit_b(d2), 0};
          I3 del = {ch.a - E.a, ch.b - E.b, 0};
          if (is_near(del)) continue;
          add_far(T, d, del, {del.a, del.b}, kSqrt3 * (double(del.a) + double(del.b) * w6), ids);
        }
      }
      cd e = d == 0 ? cd(0, 0) : std::polar(1.0, (d - 1) * M_PI / 3.0);
      T.cw.push_back(kSqrt3 * e / beta);
      T.csig.push_back(1.0 / beta);
    }
    for (int d = 0; d < 7; ++d) {
      T.st.near_d[0][d][0] = unit_a(d);
      T.st.near_d[0][d][1] = unit_b(d);
    }
    T.st.near_len[0] = 7;
  } else {
    T.n_classes = 8;
    const int lp = 7, lc = 8;
    for (int pinv = 0; pinv < 2; ++pinv) {
      I3 par = pinv ? I3{42, 42, 42} : I3{42, 42, 43};
      std::vector<I3> pn = tri_near(par, lp);
      for (int t = 0; t < 4; ++t) {
        int cls = t + 4 * pinv;
        I3 cell = tri_child3(par, lp, t);
        bool cup = tri_up(cell.a, cell.b, cell.c, lc);
        std::vector<I3> ex = tri_near(cell, lc);
        for (auto &q : pn)
          for (int t2 = 0; t2 < 4; ++t2) {
            I3 ch = tri_child3(q, lp, t2);
            if (std::find(ex.begin(), ex.end(), ch) != ex.end()) continue;
            bool sup = tri_up(ch.a, ch.b, ch.c, lc);
            int di = ch.a - cell.a, dj = ch.b - cell.b, dk = ch.c - cell.c;
            int dob = (sup ? 1 : 2) - (cup ? 1 : 2);
            int u = dk - dj, v = 3 * di + dob;
            add_far(T, cls, {di, dj, dk}, {u, v}, cd(kSqrt3 / 2 * u, 0.5 * v), ids);
          }
        double up_p = pinv ? -1.0 : 1.0;
        cd w = t == 0 ? cd(0, 0) : 0.5 * std::polar(1.0, up_p * (M_PI / 2 + 2 * (t - 1) * M_PI / 3));
        T.cw.push_back(w);
        T.csig.push_back(cd(0.5, 0));
      }
    }
    I3 reps[2] = {{84, 85, 86}, {84, 85, 85}};   // upright, inverted (level 8)
    for (int o = 0; o < 2; ++o) {
      std::vector<I3> nb = tri_near(reps[o], 8);
      // the leaf itself first (the P2P kernel relies on it)
      auto self = std::find(nb.begin(), nb.end(), reps[o]);
      std::rotate(nb.begin(), self, self + 1);
      T.st.near_len[o] = (int)nb.size();
      for (size_t e = 0; e < nb.size(); ++e) {
        T.st.near_d[o][e][0] = nb[e].a - reps[o].a;
        T.st.near_d[o][e][1] = nb[e].b - reps[o].b;
        T.st.near_d[o][e][2] = nb[e].c - reps[o].c;
      }
    }
  }
  T.st.n_classes = T.n_classes;
  return T;
}

// ------------------------------------------------------------ operators
static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// M2L operator on scaled coefficients, (p+1) x (p+1), column 0 = Q column.
static void m2l_op(cd z, int p, std::vector<cd> &out) {
  const int P1 = p + 1;
  out.assign((size_t)P1 * P1, cd(0, 0));
  std::vector<cd> ip(2 * p + 2);
  cd inv = 1.0 / z;
  ip[0] = 1.0;
  for (int i = 1; i < 2 * p + 2; ++i) ip[i] = ip[i - 1] * inv;
  for (int l = 0; l <= p; ++l) {
    if (l >= 1) out[(size_t)l * P1] = -ip[l] / double(l);
    for (int k = 1; k <= p; ++k)
      out[(size_t)l * P1 + k] = binom(l + k - 1, k - 1) * ((k & 1) ? -1.0 : 1.0) * ip[l + k];
  }
}
static void m2m_op(cd w, cd sig, int p, std::vector<cd> &out) {
  const int P1 = p + 1;
  out.assign((size_t)P1 * P1, cd(0, 0));
  for (int l = 1; l <= p; ++l) {
    out[(size_t)l * P1] = -std::pow(w, l) / double(l);
    for (int k = 1; k <= l; ++k)
      out[(size_t)l * P1 + k] = binom(l - 1, k - 1) * std::pow(sig, k) * std::pow(w, l - k);
  }
}
static void l2l_op(cd w, cd sig, int p, std::vector<cd> &out) {
  const int P1 = p + 1;
  out.assign((size_t)P1 * P1, cd(0, 0));
  for (int k = 0; k <= p; ++k)
    for (int l = k; l <= p; ++l)
      out[(size_t)k * P1 + l] = binom(l, k) * std::pow(w, l - k) * std::pow(sig, k);
}

}  // namespace fmm2d

using namespace fmm2d;

// ------------------------------------------------------------ plan helpers
namespace {

fmm2d_status fail(fmm2d_plan *pl, fmm2d_status st, const std::string &msg) {
  if (pl) pl->err = msg;
  return st;
}
fmm2d_status cuda_fail(fmm2d_plan *pl, cudaError_t e, const char *where) {
  // a failed device allocation is reported as such (the caller may free
  // memory and retry); any other failed CUDA call as FMM2D_ECUDA
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();   // clear the (non-sticky) allocation error
    return fail(pl, FMM2D_ENOMEM, std::string(where) + ": " + cudaGetErrorString(e));
  }
  return fail(pl, FMM2D_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(expr, where)                                  \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) return cuda_fail(pl, _e, where); \
  } while (0)

// FP64 expansions (the FP64 form and the hybrid form)
bool is_fp64(const fmm2d_plan *pl) {
  const unsigned pr = pl->flags & FMM2D_PREC_MASK;
  return pr == FMM2D_PREC_FP64 || pr == FMM2D_PREC_HYBRID || pr == FMM2D_PREC_SPLIT;
}
bool is_hybrid(const fmm2d_plan *pl) { return (pl->flags & FMM2D_PREC_MASK) == FMM2D_PREC_HYBRID; }
// forms whose M2L runs in float-float on the FP32 pipes (k_m2l_ff)
static bool ff_m2l(const fmm2d_plan *pl) {
  const unsigned pr = pl->flags & FMM2D_PREC_MASK;
  return pr == FMM2D_PREC_HYBRID || pr == FMM2D_PREC_SPLIT;
}

struct StageScope {
  fmm2d_plan *pl;
  int st;
  cudaStream_t s;
  cudaEvent_t b = nullptr, e = nullptr;
  StageScope(fmm2d_plan *p, int stage, cudaStream_t str, int launches) : pl(p), st(stage), s(str) {
    if (!pl->profiling) return;
    pl->stage_launches[st] += launches;
    b = get();
    e = get();
    cudaEventRecord(b, s);
  }
  cudaEvent_t get() {
    if (pl->ev_used >= pl->ev_pool.size()) {
      cudaEvent_t ev;
      cudaEventCreate(&ev);
      pl->ev_pool.push_back(ev);
    }
    return pl->ev_pool[pl->ev_used++];
  }
  ~StageScope() {
    if (!pl->profiling) return;
    cudaEventRecord(e, s);
    pl->ev_pending.push_back({st, {b, e}});
  }
};

void flush_events(fmm2d_plan *pl) {
  for (auto &x : pl->ev_pending) {
    cudaEventSynchronize(x.second.second);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, x.second.first, x.second.second);
    pl->stage_ms[x.first] += ms;
  }
  pl->ev_pending.clear();
  pl->ev_used = 0;
}

// Tensor-core M2L: how many CTAs share a tile's stencil entries, and the
// partial-sum buffers that needs (after the far-cell count is known).
static cudaError_t tc_prepare_split(fmm2d_plan *pl) {
  pl->tc_split_n = 1;
  if ((pl->flags & FMM2D_PREC_MASK) != FMM2D_PREC_MIXED_TC || pl->n_far_cells <= 0) return cudaSuccess;
  const int S = tc_split(pl->n_far_cells, pl->sten.n_classes, pl->n_sms, pl->tc_K, pl->tc_N);
  if (S > 1) {
    cudaError_t e = dbuf_reserve(pl->d_tc_part_lb, (size_t)S * pl->n_far_cells * pl->P * sizeof(float2));
    if (e == cudaSuccess) e = dbuf_reserve(pl->d_tc_part_L0, (size_t)S * pl->n_far_cells * sizeof(double));
    if (e != cudaSuccess) return e;
  }
  pl->tc_split_n = S;
  return cudaSuccess;
}

// The hybrid form's M2L: float-float on the FP32 pipes over the class lists.
static cudaError_t run_m2l_ff(fmm2d_plan *pl, int L, int64_t far_first, const double *mQ,
                              const void *ma, double *lL0, void *lb, cudaStream_t f) {
  FfArgs t;
  t.p = pl->p;
  t.P = pl->P;
  t.n_classes = pl->sten.n_classes;
  t.sms = pl->n_sms;
  t.far_first = far_first;
  t.cls_cap = pl->cls_cap;
  t.cls_cnt = (const int *)pl->d_cls_cnt.p;
  t.cls_cells = (const int *)pl->d_cls_cells.p;
  t.far_full = (const int *)pl->d_far_full.p;
  t.sten_ops = (const uint16_t *)((const char *)pl->d_sten.p + offsetof(Stencils, far_op));
  t.sten_len = (const int *)((const char *)pl->d_sten.p + offsetof(Stencils, far_len));
  t.opA = (const float2 *)pl->d_ff_ops.p;
  t.oph = (const float4 *)pl->d_ff_ph.p;
  t.logz = (const double *)pl->d_m2l_logz.p;
  t.log_abs_scale = (const double *)pl->d_geo_scale.p;
  t.lev_first = (const int64_t *)pl->d_lev_first.p;
  t.l_min = pl->l_min;
  t.L = L;
  t.mQ = mQ;
  t.ma = (const double2 *)ma;
  t.lL0 = lL0;
  t.lb = (double2 *)lb;
  t.ma_ff = (float4 *)pl->d_ma_ff.p;
  t.n_cells = pl->n_cells;
  return launch_m2l_ff(t, pl->n_far_cells, f);
}

// The plan's far-field stream (highest priority) and its fork / join events;
// with serialised profiling, the caller's stream itself.
static cudaError_t far_stream(fmm2d_plan *pl, cudaStream_t *out) {
  if (pl->profiling == 2) {
    *out = pl->last_stream;
    return cudaSuccess;
  }
  if (!pl->far_stream) {
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e != cudaSuccess) return e;
    e = cudaStreamCreateWithPriority(&pl->far_stream, cudaStreamNonBlocking, hi);
    if (e != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  *out = pl->far_stream;
  return cudaSuccess;
}

// Geometry, stencils and operator tables for the current (tiling, L, p).
// Skipped when the plan already holds them for the same parameters.
fmm2d_status setup_geometry(fmm2d_plan *pl) {
  if (pl->geo_valid && pl->geo_key_L == pl->L && pl->geo_key_p == pl->p &&
      pl->geo_key_x0 == pl->x0 && pl->geo_key_y0 == pl->y0 && pl->geo_key_S == pl->S)
    return FMM2D_OK;
  pl->geo_valid = false;
  Geo &g = pl->geo;
  g.tiling = pl->tiling;
  g.L = pl->L;
  g.b = pl->b;
  g.x0 = pl->x0;
  g.y0 = pl->y0;
  g.S = pl->S;
  const int L = pl->L;
  if (pl->tiling == FMM2D_QUAD) g.leaf_scale = std::ldexp(1.0, -L);
  else if (pl->tiling == FMM2D_TRI) g.leaf_scale = tri_rho0();
  else g.leaf_scale = sept_leaf_r(L);
  int64_t off = 0, pw = 1;
  for (int l = 0; l <= L; ++l) {
    g.map_off[l] = off;
    off += pw;
    pw *= pl->b;
  }
  g.map_off[L + 1] = off;
  pl->map_size = off;
  const cd beta(2.0, kSqrt3), e6 = std::polar(1.0, M_PI / 6);
  for (int l = 0; l <= L; ++l) {
    cd s;
    if (pl->tiling == FMM2D_QUAD) {
      s = cd(pl->S * std::ldexp(1.0, -l) * std::sqrt(2.0) / 2, 0);
      g.unit_re[l] = g.unit_im[l] = 0;
    } else if (pl->tiling == FMM2D_TRI) {
      s = cd(pl->S * 2.0 * g.leaf_scale * std::ldexp(1.0, -l), 0);
      g.unit_re[l] = g.unit_im[l] = 0;
    } else {
      cd bl = std::pow(beta, L - l);
      cd unit = g.leaf_scale * kSqrt3 * e6 * bl;   // frame lattice unit g_l
      g.unit_re[l] = unit.real();
      g.unit_im[l] = unit.imag();
      s = pl->S * g.leaf_scale * e6 * bl;
    }
    pl->scale_re[l] = s.real();
    pl->scale_im[l] = s.imag();
    pl->log_abs_scale[l] = std::log(std::abs(s));
  }
  Tables T = make_tables(pl->tiling);
  pl->sten = T.st;
  pl->n_ops = (int)T.zeta.size();
  pl->max_far = 0;
  for (int c = 0; c < T.n_classes; ++c) pl->max_far = std::max(pl->max_far, T.st.far_len[c]);
  pl->max_near = std::max(T.st.near_len[0], T.st.near_len[1]);
  const int p = pl->p, P1 = p + 1;
  std::vector<cd> m2l((size_t)pl->n_ops * P1 * P1), m2m((size_t)T.n_classes * P1 * P1),
      l2l((size_t)T.n_classes * P1 * P1), tmp;
  pl->m2l_logz_host.resize(pl->n_ops);
  for (int o = 0; o < pl->n_ops; ++o) {
    m2l_op(T.zeta[o], p, tmp);
    std::copy(tmp.begin(), tmp.end(), m2l.begin() + (size_t)o * P1 * P1);
    pl->m2l_logz_host[o] = std::log(std::abs(T.zeta[o]));
  }
  for (int c = 0; c < T.n_classes; ++c) {
    m2m_op(T.cw[c], T.csig[c], p, tmp);
    std::copy(tmp.begin(), tmp.end(), m2m.begin() + (size_t)c * P1 * P1);
    l2l_op(T.cw[c], T.csig[c], p, tmp);
    std::copy(tmp.begin(), tmp.end(), l2l.begin() + (size_t)c * P1 * P1);
  }
  const bool f64 = is_fp64(pl);
  auto upload = [&](DBuf &b, const std::vector<cd> &v) -> cudaError_t {
    if (f64) {
      cudaError_t e = dbuf_reserve(b, v.size() * sizeof(double2));
      if (e) return e;
      return cudaMemcpy(b.p, v.data(), v.size() * sizeof(double2), cudaMemcpyHostToDevice);
    }
    std::vector<float2> f(v.size());
    for (size_t i = 0; i < v.size(); ++i) f[i] = make_float2((float)v[i].real(), (float)v[i].imag());
    cudaError_t e = dbuf_reserve(b, f.size() * sizeof(float2));
    if (e) return e;
    return cudaMemcpy(b.p, f.data(), f.size() * sizeof(float2), cudaMemcpyHostToDevice);
  };
  CK(upload(pl->d_m2l_ops, m2l), "upload m2l");
  if ((pl->flags & FMM2D_PREC_MASK) == FMM2D_PREC_MIXED_TC) {
    std::vector<double> re(m2l.size()), im(m2l.size());
    for (size_t i = 0; i < m2l.size(); ++i) {
      re[i] = m2l[i].real();
      im[i] = m2l[i].imag();
    }
    std::vector<uint32_t> tab;
    tc_build_tables(re, im, pl->n_ops, p, pl->tc_K, pl->tc_N, tab);
    CK(dbuf_reserve(pl->d_tc_ops, tab.size() * 4), "alloc tc ops");
    CK(cudaMemcpy(pl->d_tc_ops.p, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice), "upload tc ops");
    int dev = 0;
    cudaGetDevice(&dev);
    CK(cudaDeviceGetAttribute(&pl->n_sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
  }
  if (ff_m2l(pl)) {   // float-float operators for the FP32-pipe M2L
    std::vector<float> A, ph;
    ff_build_table(T.zeta, m2l, p, A, ph);
    CK(dbuf_reserve(pl->d_ff_ops, A.size() * 4), "alloc ff ops");
    CK(cudaMemcpy(pl->d_ff_ops.p, A.data(), A.size() * 4, cudaMemcpyHostToDevice), "upload ff ops");
    CK(dbuf_reserve(pl->d_ff_ph, ph.size() * 4), "alloc ff phases");
    CK(cudaMemcpy(pl->d_ff_ph.p, ph.data(), ph.size() * 4, cudaMemcpyHostToDevice), "upload ff phases");
    int dev = 0;
    cudaGetDevice(&dev);
    CK(cudaDeviceGetAttribute(&pl->n_sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
  }
  CK(upload(pl->d_m2m_ops, m2m), "upload m2m");
  CK(upload(pl->d_l2l_ops, l2l), "upload l2l");
  CK(dbuf_reserve(pl->d_m2l_logz, pl->n_ops * sizeof(double)), "alloc logz");
  CK(cudaMemcpy(pl->d_m2l_logz.p, pl->m2l_logz_host.data(), pl->n_ops * sizeof(double),
                cudaMemcpyHostToDevice), "upload logz");
  CK(dbuf_reserve(pl->d_sten, sizeof(Stencils)), "alloc stencils");
  CK(cudaMemcpy(pl->d_sten.p, &pl->sten, sizeof(Stencils), cudaMemcpyHostToDevice), "upload stencils");
  CK(dbuf_reserve(pl->d_geo_scale, (MAXLEV + 1) * sizeof(double)), "alloc scale");
  CK(cudaMemcpy(pl->d_geo_scale.p, pl->log_abs_scale, (MAXLEV + 1) * sizeof(double),
                cudaMemcpyHostToDevice), "upload scale");
  pl->geo_valid = true;
  pl->geo_key_L = pl->L;
  pl->geo_key_p = pl->p;
  pl->geo_key_x0 = pl->x0;
  pl->geo_key_y0 = pl->y0;
  pl->geo_key_S = pl->S;
  return FMM2D_OK;
}

template <typename R>
fmm2d_status evaluate_t(fmm2d_plan *pl, const void *u, double *out, cudaStream_t s) {
  const bool f32_in = (pl->flags & FMM2D_IN_F32) != 0;
  const int L = pl->L;
  R *src4 = (R *)pl->d_src4.p;
  const R *tgt = pl->same_sets ? src4 : (const R *)pl->d_tgt2.p;
  const int tstride = pl->same_sets ? 4 : 2;
  const uint32_t *tperm = (const uint32_t *)(pl->same_sets ? pl->d_perm_s.p : pl->d_perm_t.p);
  const int *tst = (const int *)(pl->same_sets ? pl->d_src_start.p : pl->d_tgt_start.p);
  const int *ten = (const int *)(pl->same_sets ? pl->d_src_end.p : pl->d_tgt_end.p);
  Cx<R> *ma = (Cx<R> *)pl->d_ma.p, *lb = (Cx<R> *)pl->d_lb.p;
  double *mQ = (double *)pl->d_mQ.p, *lL0 = (double *)pl->d_lL0.p;
  ExpandArgs a;
  a.p = pl->p;
  a.P = pl->P;
  a.L = L;
  a.l_min = pl->l_min;
  a.b = pl->b;
  a.n_cls = pl->sten.n_classes;
  a.leaf_first = pl->lev_first[L];
  a.n_leaves = pl->lev_count[L];
  cd inv_s = 1.0 / cd(pl->scale_re[L], pl->scale_im[L]);
  a.inv_s_re = inv_s.real();
  a.inv_s_im = inv_s.imag();
  {
    StageScope sc(pl, ST_OTHER, s, 1);
    CK(launch_gather_u<R>(u, f32_in, (const uint32_t *)pl->d_perm_s.p, pl->n_src, src4, s), "gather");
    if (is_hybrid(pl))
      CK(launch_gather_u<float>(u, f32_in, (const uint32_t *)pl->d_perm_s.p, pl->n_src,
                                (float *)pl->d_src4f.p, s, true), "gather");
  }
  // fork: the far-field chain on the plan's high-priority stream f, P2P on s
  cudaStream_t f;
  CK(far_stream(pl, &f), "far stream");
  if (f != s) {
    CK(cudaEventRecord(pl->ev_fork, s), "fork");
    CK(cudaStreamWaitEvent(f, pl->ev_fork, 0), "fork");
  }
  // the device error word of this evaluation (bounded waits report there)
  CK(cudaMemsetAsync(pl->d_dev_err.p, 0, 4, f), "memset");
  {
    StageScope sc(pl, ST_P2M, f, 1);
    CK(launch_p2m<R>(a, src4, (const int *)pl->d_src_start.p, (const int *)pl->d_src_end.p, mQ, ma, f), "p2m");
  }
  if (L - 1 >= pl->l_min) {   // levels L-1 .. l_min in one launch
    StageScope sc(pl, ST_M2M, f, 1);
    CK(launch_m2m_up<R>(a, pl->geo, pl->l_min, pl->lev_first[L - 1], pl->lev_count[L - 1],
                        (const int *)pl->d_map.p, (const uint32_t *)pl->d_cell_key.p,
                        (const uint8_t *)pl->d_cell_cls.p, (const uint8_t *)pl->d_cell_hsrc.p,
                        (const Cx<R> *)pl->d_m2m_ops.p, mQ, ma, (int *)pl->d_m2m_arrive.p,
                        pl->n_cells, f),
       "m2m");
  }
  if (L < pl->l_min) {
    CK(cudaMemsetAsync(lL0, 0, pl->n_cells * sizeof(double), f), "zero locals");
    CK(cudaMemsetAsync(lb, 0, pl->n_cells * pl->P * sizeof(Cx<R>), f), "zero locals");
  } else if (ff_m2l(pl)) {
    StageScope sc(pl, ST_M2L, f, 1);
    CK(run_m2l_ff(pl, L, pl->lev_first[pl->l_min], mQ, ma, lL0, lb, f), "m2l_ff");
  } else if ((pl->flags & FMM2D_PREC_MASK) == FMM2D_PREC_MIXED_TC) {
    StageScope sc(pl, ST_M2L, f, pl->tc_split_n > 1 ? 2 : 1);
    TcArgs t;
    t.p = pl->p;
    t.P = pl->P;
    t.n_classes = pl->sten.n_classes;
    t.sms = pl->n_sms;
    t.far_first = pl->lev_first[pl->l_min];
    t.cls_cap = pl->cls_cap;
    t.cls_cnt = (const int *)pl->d_cls_cnt.p;
    t.cls_cells = (const int *)pl->d_cls_cells.p;
    t.far_full = (const int *)pl->d_far_full.p;
    t.sten_ops = (const uint16_t *)((const char *)pl->d_sten.p + offsetof(Stencils, far_op));
    t.sten_len = (const int *)((const char *)pl->d_sten.p + offsetof(Stencils, far_len));
    t.btab = (const unsigned char *)pl->d_tc_ops.p;
    t.logz = (const double *)pl->d_m2l_logz.p;
    t.log_abs_scale = (const double *)pl->d_geo_scale.p;
    t.lev_first = (const int64_t *)pl->d_lev_first.p;
    t.l_min = pl->l_min;
    t.L = L;
    t.mQ = mQ;
    t.ma = (const float2 *)ma;
    t.lL0 = lL0;
    t.lb = (float2 *)lb;
    t.err = (int *)pl->d_dev_err.p;
    t.split = pl->tc_split_n;
    t.part_lb = (float2 *)pl->d_tc_part_lb.p;
    t.part_L0 = (double *)pl->d_tc_part_L0.p;
    t.n_far = pl->n_far_cells;
    t.debug_stall = pl->debug_stall;
    CK(cudaMemsetAsync(pl->d_dev_err.p, 0, 4, f), "memset");
    CK(launch_m2l_tc(t, pl->tc_K, pl->tc_N, pl->n_far_cells, f), "m2l_tc");
  } else {
    StageScope sc(pl, ST_M2L, f, 1);
    CK(launch_m2l<R>(a, pl->lev_first[pl->l_min], pl->n_far_cells, (const int64_t *)pl->d_lev_first.p,
                     (const double *)pl->d_geo_scale.p, 0, (const int *)pl->d_far_cnt.p,
                     (const int *)pl->d_far_src.p, (const uint16_t *)pl->d_far_op.p,
                     (const Cx<R> *)pl->d_m2l_ops.p, (const double *)pl->d_m2l_logz.p, mQ, ma, lL0,
                     lb, f),
       "m2l");
  }
  {
    // levels l_min+1 .. L-1 in one launch; the leaf level's L2L is done by
    // the L2P
    StageScope sc(pl, ST_L2L, f, L - 1 > pl->l_min ? 1 : 0);
    if (L - 1 > pl->l_min) {
      const int64_t first = pl->lev_first[pl->l_min + 1];
      CK(launch_l2l_down<R>(a, pl->geo, first, pl->lev_first[L] - first, (const int64_t *)pl->d_lev_first.p,
                            (const int *)pl->d_map.p, (const uint32_t *)pl->d_cell_key.p,
                            (const uint8_t *)pl->d_cell_cls.p, (const Cx<R> *)pl->d_l2l_ops.p, lL0,
                            lb, (int *)pl->d_l2l_ready.p, pl->n_cells, pl->n_sms,
                            (int *)pl->d_dev_err.p, f),
         "l2l");
    }
  }
  {
    StageScope sc(pl, ST_P2P, s, 1);
    if (is_hybrid(pl)) {   // FP32 P2P on the FP32 copies
      const float *s4 = (const float *)pl->d_src4f.p;
      CK(launch_p2p<float>(a.leaf_first, a.n_leaves, nullptr, s4,
                           pl->same_sets ? s4 : (const float *)pl->d_tgt2f.p, tstride,
                           (const int *)pl->d_src_start.p, (const int *)pl->d_src_end.p, tst, ten,
                           (const int *)pl->d_near_cnt.p, nullptr, (const int *)pl->d_near_src.p,
                           (const double2 *)pl->d_cell_ctr.p, (double *)pl->d_phi_near.p,
                           a.n_leaves > 0 ? (double)pl->n_tgt / (double)a.n_leaves : 0.0, s,
                           (const float2 *)pl->d_srclo.p,
                           (const float2 *)(pl->same_sets ? pl->d_srclo.p : pl->d_tgtlo.p)),
         "p2p");
    } else
    CK(launch_p2p<R>(a.leaf_first, a.n_leaves, nullptr, src4, tgt, tstride,
                     (const int *)pl->d_src_start.p, (const int *)pl->d_src_end.p, tst, ten,
                     (const int *)pl->d_near_cnt.p, nullptr, (const int *)pl->d_near_src.p,
                     (const double2 *)pl->d_cell_ctr.p,
                     (double *)pl->d_phi_near.p,
                     a.n_leaves > 0 ? (double)pl->n_tgt / (double)a.n_leaves : 0.0, s),
       "p2p");
  }
  if (f != s) {   // join: L2P needs the locals
    CK(cudaEventRecord(pl->ev_join, f), "join");
    CK(cudaStreamWaitEvent(s, pl->ev_join, 0), "join");
  }
  {
    StageScope sc(pl, ST_L2P, s, 1);
    if (L > pl->l_min) {   // the leaf level's L2L
      a.l2l_map = (const int *)pl->d_map.p;
      a.l2l_map_off = pl->geo.map_off[L - 1];
      a.l2l_key = (const uint32_t *)pl->d_cell_key.p;
      a.l2l_cls = (const uint8_t *)pl->d_cell_cls.p;
      a.l2l_ops = pl->d_l2l_ops.p;
      a.l2l_sept = pl->tiling == FMM2D_SEPT;
    }
    CK(launch_l2p<R>(a, tgt, tstride, tst, ten, tperm, lL0, lb, (const double *)pl->d_phi_near.p,
                     (double *)pl->d_phi_far.p, out, s),
       "l2p");
  }
  return FMM2D_OK;
}

}  // namespace

// ------------------------------------------------------------ C ABI
// ------------------------------------------------------------ adaptive tree
static AdCells ad_cells(fmm2d_plan *pl) {
  AdCells c;
  c.key = (uint32_t *)pl->d_cell_key.p;
  c.lev = (uint8_t *)pl->d_cell_lev.p;
  c.parent = (int *)pl->d_parent.p;
  c.child_first = (int *)pl->d_child_first.p;
  c.child_cnt = (uint8_t *)pl->d_child_cnt.p;
  c.split = (uint8_t *)pl->d_split.p;
  c.ss = (int *)pl->d_src_start.p;
  c.se = (int *)pl->d_src_end.p;
  c.ts = pl->same_sets ? c.ss : (int *)pl->d_tgt_start.p;
  c.te = pl->same_sets ? c.se : (int *)pl->d_tgt_end.p;
  c.crd = (int4 *)pl->d_cell_crd.p;
  c.ctr = (double2 *)pl->d_cell_ctr.p;
  c.cls = (uint8_t *)pl->d_cell_cls.p;
  c.hsrc = (uint8_t *)pl->d_cell_hsrc.p;
  return c;
}

// Keys and sort on the finest level, the tree level by level (one read-back
// of each level's cell count), the leaves, and the U / W / X / M2L lists by
// the level-synchronous traversal (one read-back of each level's list sizes).
static fmm2d_status build_adaptive(fmm2d_plan *pl, const void *src, int64_t n_src, const void *tgt,
                                   int64_t n_tgt, cudaStream_t s, int n_inst = 1,
                                   const int64_t *inst_off = nullptr) {
  const bool f32 = (pl->flags & FMM2D_IN_F32) != 0;
  const bool f64 = is_fp64(pl);
  // a forest's level-L keys carry the instance: n_inst b^L must fit 32 bits
  auto fits = [&](int Lc) {
    double v = (double)n_inst;
    for (int i = 0; i < Lc; ++i) v *= pl->b;
    return v <= 4294967296.0;   // keys up to n_inst b^L - 1 < 2^32
  };
  int L = pl->levels_req;
  if (L == 0) {
    L = ad_max_levels(pl->tiling);
    while (L > 1 && !fits(L)) --L;
  }
  if (!fits(L)) return fail(pl, FMM2D_EINVAL, "too many instances for this finest level");
  pl->n_inst = n_inst;
  const int p = pl->p_req ? pl->p_req : p_from_eps(pl->tiling, pl->eps);
  const bool tc_form = (pl->flags & FMM2D_PREC_MASK) == FMM2D_PREC_MIXED_TC;
  if (tc_form && !tc_shape(p, &pl->tc_K, &pl->tc_N))
    return fail(pl, FMM2D_EINVAL, "tensor-core M2L supports p <= 31");
  const bool tc = tc_form || ff_m2l(pl);   // class lists: tensor-core and float-float M2L
  pl->L = L;
  pl->p = p;
  pl->P = (p + 1) & ~1;
  fmm2d_status st = setup_geometry(pl);
  if (st != FMM2D_OK) return st;
  const Geo &g = pl->geo;
  const int b = pl->b;
  const int64_t nmax = std::max<int64_t>(1, std::max(n_src, n_tgt));
  CK(dbuf_reserve(pl->d_key_s, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_perm_s, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_key_t, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_perm_t, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_tmp_k, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_tmp_v, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_sort_scratch, radix_sort_scratch_bytes(nmax)), "alloc");
  const size_t rsz = f64 ? sizeof(double) : sizeof(float);
  CK(dbuf_reserve(pl->d_src4, std::max<int64_t>(1, n_src) * 4 * rsz), "alloc");
  CK(dbuf_reserve(pl->d_tgt2, std::max<int64_t>(1, n_tgt) * 2 * rsz), "alloc");
  CK(dbuf_reserve(pl->d_phi_near, std::max<int64_t>(1, n_tgt) * 8), "alloc");
  CK(dbuf_reserve(pl->d_phi_far, std::max<int64_t>(1, n_tgt) * 8), "alloc");
  CK(dbuf_reserve(pl->d_err, 16), "alloc");
  CK(dbuf_reserve(pl->d_dev_err, 16), "alloc");
  CK(dbuf_reserve(pl->d_lev_first, (MAXLEV + 2) * 8), "alloc");
  CK(dbuf_reserve(pl->d_ad_tot, 64), "alloc");
  CK(cudaMemsetAsync(pl->d_err.p, 0, 16, s), "memset");
  CK(cudaMemsetAsync(pl->d_dev_err.p, 0, 16, s), "memset");
  const int bits = key_bits(pl->tiling, L);
  uint32_t *ks = (uint32_t *)pl->d_key_s.p, *ps = (uint32_t *)pl->d_perm_s.p;
  uint32_t *kt = (uint32_t *)pl->d_key_t.p, *pt = (uint32_t *)pl->d_perm_t.p;
  {
    StageScope sc(pl, ST_KEYS, s, pl->same_sets ? 1 : 2);
    CK(launch_keys(g, src, f32, n_src, ks, ps, (int *)pl->d_err.p, s, (uint32_t *)pl->d_tmp_v.p,
                   (int *)pl->d_err.p + 2), "keys");
    if (!pl->same_sets)
      CK(launch_keys(g, tgt, f32, n_tgt, kt, pt, (int *)pl->d_err.p, s, (uint32_t *)pl->d_tmp_v.p,
                     (int *)pl->d_err.p + 2), "keys");
  }
  int sbits = bits;
  if (inst_off) {   // forest: prefix the keys with the instance
    CK(dbuf_reserve(pl->d_inst_off, (n_inst + 1) * 8), "alloc");
    CK(cudaMemcpyAsync(pl->d_inst_off.p, inst_off, (n_inst + 1) * 8, cudaMemcpyHostToDevice, s), "upload");
    uint64_t span = 1;
    for (int i = 0; i < L; ++i) span *= (uint64_t)pl->b;
    CK(ad_launch_prefix(n_src, ks, (const int64_t *)pl->d_inst_off.p, n_inst, span, s), "prefix");
    sbits = 0;
    while (sbits < 32 && ((uint64_t)1 << sbits) < span * (uint64_t)n_inst) ++sbits;
  }
  {
    StageScope sc(pl, ST_SORT, s,
                  radix_sort_launches(n_src, sbits) + (pl->same_sets ? 0 : radix_sort_launches(n_tgt, sbits)));
    CK(radix_sort_pairs(ks, ps, (uint32_t *)pl->d_tmp_k.p, (uint32_t *)pl->d_tmp_v.p, n_src, sbits,
                        pl->d_sort_scratch.p, s, (int *)pl->d_err.p), "sort");
    if (!pl->same_sets)
      CK(radix_sort_pairs(kt, pt, (uint32_t *)pl->d_tmp_k.p, (uint32_t *)pl->d_tmp_v.p, n_tgt, sbits,
                          pl->d_sort_scratch.p, s, (int *)pl->d_err.p), "sort");
  }
  int err_h = 0;
  CK(cudaMemcpyAsync(&err_h, pl->d_err.p, 4, cudaMemcpyDeviceToHost, s), "readback");
  CK(cudaStreamSynchronize(s), "keys sync");
  if (err_h & 8) return fail(pl, FMM2D_ETIMEOUT, "a bounded wait of the radix sort gave up");
  if (err_h) return fail(pl, FMM2D_EDOMAIN, "a point lies outside the domain square or root cell");

  // ---- cell capacity: a split cell holds more than leaf_cap sources or
  // targets, so a level has at most n_src/(cap+1) + n_tgt/(cap+1) of them
  const int cap = pl->leaf_cap;
  const int64_t nsplit = pl->same_sets ? n_src / (cap + 1) : n_src / (cap + 1) + n_tgt / (cap + 1);
  int64_t cap_cells = n_inst, pw = n_inst;   // pw: cells a level can hold
  for (int l = 0; l < L; ++l) {
    const int64_t prev = pw;
    pw = pw > ((int64_t)1 << 40) ? pw : pw * b;
    cap_cells += std::min<int64_t>(pw, (int64_t)b * std::max<int64_t>(1, std::min<int64_t>(nsplit, prev)));
  }
  CK(dbuf_reserve(pl->d_cell_key, cap_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_cell_lev, cap_cells), "alloc");
  CK(dbuf_reserve(pl->d_parent, cap_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_child_first, cap_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_child_cnt, cap_cells), "alloc");
  CK(dbuf_reserve(pl->d_split, cap_cells), "alloc");
  CK(dbuf_reserve(pl->d_src_start, cap_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_src_end, cap_cells * 4), "alloc");
  if (!pl->same_sets) {
    CK(dbuf_reserve(pl->d_tgt_start, cap_cells * 4), "alloc");
    CK(dbuf_reserve(pl->d_tgt_end, cap_cells * 4), "alloc");
  }
  CK(dbuf_reserve(pl->d_cell_crd, cap_cells * sizeof(int4)), "alloc");
  CK(dbuf_reserve(pl->d_cell_ctr, cap_cells * sizeof(double2)), "alloc");
  CK(dbuf_reserve(pl->d_cell_cls, cap_cells), "alloc");
  CK(dbuf_reserve(pl->d_cell_hsrc, cap_cells), "alloc");
  AdCells c = ad_cells(pl);
  int64_t lf[MAXLEV + 2];
  for (int l = 0; l <= MAXLEV + 1; ++l) lf[l] = 0;
  lf[1] = n_inst;
  int depth = 0;
  {
    StageScope sc(pl, ST_TREE, s, 1);
    const int64_t *doff = inst_off ? (const int64_t *)pl->d_inst_off.p : nullptr;
    CK(ad_launch_roots(g, n_inst, doff, doff, n_src, pl->same_sets ? n_src : n_tgt, c, s), "roots");
    for (int l = 0; l <= L; ++l) {
      const int64_t count = lf[l + 1] - lf[l];
      CK(dbuf_reserve(pl->d_ad_flag, std::max<int64_t>(1, count * b) * 4), "alloc");
      CK(dbuf_reserve(pl->d_ad_pos, std::max<int64_t>(1, count * b) * 4), "alloc");
      CK(dbuf_reserve(pl->d_ad_crange, std::max<int64_t>(1, count * b) * sizeof(int4)), "alloc");
      CK(dbuf_reserve(pl->d_sort_scratch, std::max(radix_sort_scratch_bytes(nmax),
                                                   scan_scratch_bytes(count * b + 1))), "alloc");
      CK(ad_launch_split(g, l, lf[l], count, cap, ks, pl->same_sets ? nullptr : kt, c,
                         (int *)pl->d_ad_flag.p, (int4 *)pl->d_ad_crange.p, s), "split");
      depth = l;
      if (l == L) break;
      CK(exclusive_scan((const int *)pl->d_ad_flag.p, (int *)pl->d_ad_pos.p, count * b,
                        pl->d_sort_scratch.p, s), "scan");
      CK(ad_launch_level_total(count * b, (const int *)pl->d_ad_flag.p, (const int *)pl->d_ad_pos.p,
                               (int *)pl->d_ad_tot.p, s), "total");
      int tot = 0;
      CK(cudaMemcpyAsync(&tot, pl->d_ad_tot.p, 4, cudaMemcpyDeviceToHost, s), "readback");
      CK(cudaStreamSynchronize(s), "tree sync");
      if (lf[l + 1] + tot > cap_cells) return fail(pl, FMM2D_ECUDA, "adaptive tree capacity exceeded");
      CK(ad_launch_emit(g, l, lf[l], count, lf[l + 1], (const int *)pl->d_ad_flag.p,
                        (const int *)pl->d_ad_pos.p, (const int4 *)pl->d_ad_crange.p, c, s), "emit");
      lf[l + 2] = lf[l + 1] + tot;
      if (tot == 0) break;
    }
  }
  const int64_t n_cells = lf[depth + 1];
  for (int l = depth + 2; l <= MAXLEV + 1; ++l) lf[l] = n_cells;
  for (int l = 0; l <= MAXLEV + 1; ++l) pl->lev_first[l] = lf[l];
  for (int l = 0; l <= MAXLEV; ++l) pl->lev_count[l] = lf[l + 1] - lf[l];
  pl->n_cells = n_cells;
  CK(cudaMemcpyAsync(pl->d_lev_first.p, lf, (MAXLEV + 2) * 8, cudaMemcpyHostToDevice, s), "upload");
  // ---- leaves, and points relative to their leaf centre
  CK(dbuf_reserve(pl->d_ad_flag, n_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_ad_pos, n_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_leaf_ids, n_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_leaf_pos, n_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_sort_scratch, std::max(radix_sort_scratch_bytes(nmax),
                                               scan_scratch_bytes(n_cells + 1))), "alloc");
  int n_leaves = 0;
  {
    StageScope sc(pl, ST_TREE, s, 4);
    CK(ad_launch_leaves(n_cells, c.split, (int *)pl->d_ad_flag.p, (int *)pl->d_ad_pos.p,
                        pl->d_sort_scratch.p, (int *)pl->d_leaf_ids.p, (int *)pl->d_leaf_pos.p,
                        (int *)pl->d_ad_tot.p, s), "leaves");
    CK(cudaMemcpyAsync(&n_leaves, pl->d_ad_tot.p, 4, cudaMemcpyDeviceToHost, s), "readback");
    CK(cudaStreamSynchronize(s), "leaves sync");
    pl->n_leaves_ad = n_leaves;
    // FP32 forms of a field plan: also the low parts of the leaf-relative
    // coordinates (the accurate pair differences of the field's P2P)
    const bool keep_lo = !f64 && (pl->flags & FMM2D_FIELD);
    if (keep_lo) {
      CK(dbuf_reserve(pl->d_srclo, std::max<int64_t>(1, n_src) * 8), "alloc");
      if (!pl->same_sets) CK(dbuf_reserve(pl->d_tgtlo, std::max<int64_t>(1, n_tgt) * 8), "alloc");
    }
    CK(ad_launch_rel(f32, !f64, src, ps, n_leaves, (const int *)pl->d_leaf_ids.p, c.ss, c.se, c.ctr,
                     pl->d_src4.p, 4, s, keep_lo ? (float2 *)pl->d_srclo.p : nullptr), "rel");
    if (!pl->same_sets)
      CK(ad_launch_rel(f32, !f64, tgt, pt, n_leaves, (const int *)pl->d_leaf_ids.p, c.ts, c.te, c.ctr,
                       pl->d_tgt2.p, 2, s, keep_lo ? (float2 *)pl->d_tgtlo.p : nullptr), "rel");
    if (is_hybrid(pl)) {   // FP32 hi + lo copies for the P2P
      CK(dbuf_reserve(pl->d_src4f, std::max<int64_t>(1, n_src) * 16), "alloc");
      CK(dbuf_reserve(pl->d_srclo, std::max<int64_t>(1, n_src) * 8), "alloc");
      CK(ad_launch_rel(f32, true, src, ps, n_leaves, (const int *)pl->d_leaf_ids.p, c.ss, c.se, c.ctr,
                       pl->d_src4f.p, 4, s, (float2 *)pl->d_srclo.p), "rel");
      if (!pl->same_sets) {
        CK(dbuf_reserve(pl->d_tgt2f, std::max<int64_t>(1, n_tgt) * 8), "alloc");
        CK(dbuf_reserve(pl->d_tgtlo, std::max<int64_t>(1, n_tgt) * 8), "alloc");
        CK(ad_launch_rel(f32, true, tgt, pt, n_leaves, (const int *)pl->d_leaf_ids.p, c.ts, c.te,
                         c.ctr, pl->d_tgt2f.p, 2, s, (float2 *)pl->d_tgtlo.p), "rel");
      }
    }
  }
  // the FP32 P2P's leaf size classes (group size per leaf)
  pl->p2p_binned = !f64 || is_hybrid(pl);
  if (pl->p2p_binned) {
    CK(dbuf_reserve(pl->d_p2p_order, std::max(1, n_leaves) * 4), "alloc");
    CK(dbuf_reserve(pl->d_p2p_cnt, 8 * 4), "alloc");
    CK(launch_p2p_bins(n_leaves, (const int *)pl->d_leaf_ids.p, c.ts, c.te, (int *)pl->d_p2p_cnt.p,
                       (int *)pl->d_p2p_order.p, s), "p2p bins");
  }
  // ---- lists
  const int64_t far_first = depth >= pl->l_min ? lf[pl->l_min] : n_cells;
  pl->n_far_cells = n_cells - far_first;
  const int64_t nfc = std::max<int64_t>(1, pl->n_far_cells);
  CK(dbuf_reserve(pl->d_far_cnt, nfc * 4), "alloc");
  CK(dbuf_reserve(pl->d_far_src, nfc * FAR_MAX * 4), "alloc");
  CK(dbuf_reserve(pl->d_far_op, nfc * FAR_MAX * 2), "alloc");
  if (tc) {
    CK(dbuf_reserve(pl->d_far_full, nfc * FAR_MAX * 4), "alloc");
    CK(dbuf_reserve(pl->d_cls_cnt, MAX_CLASSES * 4), "alloc");
    CK(dbuf_reserve(pl->d_cls_cells, (size_t)MAX_CLASSES * nfc * 4), "alloc");
    CK(cudaMemsetAsync(pl->d_cls_cnt.p, 0, MAX_CLASSES * 4, s), "memset");
  }
  pl->cls_cap = nfc;
  int64_t n_u = 0, n_w = 0, n_x = 0, n_t = 0, n_s = 0;
  {
    StageScope sc(pl, ST_LISTS, s, 4 * (depth + 1) + 1);
    // the stencil lookups of the list kernels go through a (level, instance,
    // lattice position) -> cell table of the cells with sources, at most
    // half full
    uint64_t hcap = 1024;
    while (hcap < 2 * (uint64_t)n_cells) hcap <<= 1;
    CK(dbuf_reserve(pl->d_ad_hash, hcap * sizeof(ulonglong2)), "alloc");
    c.hslot = (const ulonglong2 *)pl->d_ad_hash.p;
    c.hmask = (uint32_t)(hcap - 1);
    CK(ad_launch_hash(g, n_cells, c, (ulonglong2 *)pl->d_ad_hash.p, c.hmask, s), "cell table");
    for (int l = 0; l <= depth; ++l) {
      const int64_t count = lf[l + 1] - lf[l];
      const int64_t items = count + n_t + n_s;
      if (items == 0) continue;
      CK(dbuf_reserve(pl->d_ad_cnt, items * 5 * 4), "alloc");
      CK(dbuf_reserve(pl->d_ad_off, items * 5 * 4), "alloc");
      CK(dbuf_reserve(pl->d_sort_scratch, std::max(radix_sort_scratch_bytes(nmax),
                                                   scan_scratch_bytes(items * 5))), "alloc");
      CK(ad_launch_lists(g, (const Stencils *)pl->d_sten.p, l, pl->l_min, lf[l], count, n_t, n_s,
                         (const int *)pl->d_ad_ta.p, (const int *)pl->d_ad_tc.p,
                         (const int *)pl->d_ad_sa.p, (const int *)pl->d_ad_sc.p, c,
                         (int *)pl->d_ad_cnt.p, (int *)pl->d_ad_off.p, pl->d_sort_scratch.p,
                         (int *)pl->d_ad_tot.p, s), "lists");
      int tot[5];
      CK(cudaMemcpyAsync(tot, pl->d_ad_tot.p, 20, cudaMemcpyDeviceToHost, s), "readback");
      CK(cudaStreamSynchronize(s), "lists sync");
      CK(dbuf_grow_keep(pl->d_ad_ut, (n_u + tot[0]) * 4, n_u * 4, s), "alloc");
      CK(dbuf_grow_keep(pl->d_ad_us, (n_u + tot[0]) * 4, n_u * 4, s), "alloc");
      CK(dbuf_grow_keep(pl->d_ad_wt, (n_w + tot[1]) * 4, n_w * 4, s), "alloc");
      CK(dbuf_grow_keep(pl->d_ad_ws, (n_w + tot[1]) * 4, n_w * 4, s), "alloc");
      CK(dbuf_grow_keep(pl->d_ad_xt, (n_x + tot[2]) * 4, n_x * 4, s), "alloc");
      CK(dbuf_grow_keep(pl->d_ad_xs, (n_x + tot[2]) * 4, n_x * 4, s), "alloc");
      CK(dbuf_reserve(pl->d_ad_ta2, std::max(1, tot[3]) * 4), "alloc");
      CK(dbuf_reserve(pl->d_ad_tc2, std::max(1, tot[3]) * 4), "alloc");
      CK(dbuf_reserve(pl->d_ad_sa2, std::max(1, tot[4]) * 4), "alloc");
      CK(dbuf_reserve(pl->d_ad_sc2, std::max(1, tot[4]) * 4), "alloc");
      const int64_t base[5] = {n_u, n_w, n_x, 0, 0};
      CK(ad_launch_lists_emit(g, (const Stencils *)pl->d_sten.p, l, pl->l_min, lf[l], count, n_t, n_s,
                              (const int *)pl->d_ad_ta.p, (const int *)pl->d_ad_tc.p,
                              (const int *)pl->d_ad_sa.p, (const int *)pl->d_ad_sc.p, c,
                              (const int *)pl->d_ad_off.p, base, (int *)pl->d_ad_ut.p,
                              (int *)pl->d_ad_us.p, (int *)pl->d_ad_wt.p, (int *)pl->d_ad_ws.p,
                              (int *)pl->d_ad_xt.p, (int *)pl->d_ad_xs.p, (int *)pl->d_ad_ta2.p,
                              (int *)pl->d_ad_tc2.p, (int *)pl->d_ad_sa2.p, (int *)pl->d_ad_sc2.p,
                              far_first, (int *)pl->d_far_cnt.p, (int *)pl->d_far_src.p,
                              (uint16_t *)pl->d_far_op.p, tc ? (int *)pl->d_far_full.p : nullptr,
                              tc ? (int *)pl->d_cls_cnt.p : nullptr,
                              tc ? (int *)pl->d_cls_cells.p : nullptr, nfc, s), "lists");
      std::swap(pl->d_ad_ta, pl->d_ad_ta2);
      std::swap(pl->d_ad_tc, pl->d_ad_tc2);
      std::swap(pl->d_ad_sa, pl->d_ad_sa2);
      std::swap(pl->d_ad_sc, pl->d_ad_sc2);
      n_u += tot[0];
      n_w += tot[1];
      n_x += tot[2];
      n_t = tot[3];
      n_s = tot[4];
    }
    if (n_t || n_s) return fail(pl, FMM2D_ECUDA, "adaptive traversal did not terminate");
    pl->n_u = n_u;
    pl->n_w = n_w;
    pl->n_x = n_x;
    // group U and W by target leaf, X by target cell
    const int64_t ng = std::max<int64_t>({n_u, n_w, n_x, 1});
    CK(dbuf_reserve(pl->d_tmp_k, std::max<int64_t>(nmax, ng) * 4), "alloc");
    CK(dbuf_reserve(pl->d_tmp_v, std::max<int64_t>(nmax, ng) * 4), "alloc");
    CK(dbuf_reserve(pl->d_ad_cnt, std::max<int64_t>(ng, n_cells + 1) * 4), "alloc");
    CK(dbuf_reserve(pl->d_ad_off, std::max<int64_t>(ng, n_cells + 1) * 4), "alloc");
    CK(dbuf_reserve(pl->d_ad_flag, ng * 4), "alloc");
    CK(dbuf_reserve(pl->d_ad_pos, ng * 4), "alloc");
    CK(dbuf_reserve(pl->d_sort_scratch, std::max(radix_sort_scratch_bytes(ng),
                                                 scan_scratch_bytes(n_cells + 1))), "alloc");
    CK(dbuf_reserve(pl->d_u_off, (n_leaves + 1) * 4), "alloc");
    CK(dbuf_reserve(pl->d_w_off, (n_leaves + 1) * 4), "alloc");
    CK(dbuf_reserve(pl->d_x_off, (n_cells + 1) * 4), "alloc");
    CK(dbuf_reserve(pl->d_u_src, std::max<int64_t>(1, n_u) * 4), "alloc");
    CK(dbuf_reserve(pl->d_w_src, std::max<int64_t>(1, n_w) * 4), "alloc");
    CK(dbuf_reserve(pl->d_x_src, std::max<int64_t>(1, n_x) * 4), "alloc");
    auto group = [&](int64_t n, DBuf &t, DBuf &sr, const int *map, int ngroups, DBuf &off, DBuf &out) {
      return ad_group(n, (const int *)t.p, (const int *)sr.p, map, ngroups, (uint32_t *)pl->d_ad_flag.p,
                      (uint32_t *)pl->d_ad_pos.p, (uint32_t *)pl->d_tmp_k.p, (uint32_t *)pl->d_tmp_v.p,
                      pl->d_sort_scratch.p, (int *)pl->d_ad_cnt.p, (int *)off.p, (int *)out.p, s,
                      (int *)pl->d_err.p);
    };
    CK(group(n_u, pl->d_ad_ut, pl->d_ad_us, (const int *)pl->d_leaf_pos.p, n_leaves, pl->d_u_off, pl->d_u_src), "group U");
    CK(group(n_w, pl->d_ad_wt, pl->d_ad_ws, (const int *)pl->d_leaf_pos.p, n_leaves, pl->d_w_off, pl->d_w_src), "group W");
    CK(group(n_x, pl->d_ad_xt, pl->d_ad_xs, nullptr, (int)n_cells, pl->d_x_off, pl->d_x_src), "group X");
  }
  // per-level scales for the kernels
  std::vector<double2> sc(MAXLEV + 1), isc(MAXLEV + 1);
  for (int l = 0; l <= MAXLEV; ++l) {
    const cd v = l <= L ? cd(pl->scale_re[l], pl->scale_im[l]) : cd(1.0, 0.0);
    const cd iv = 1.0 / v;
    sc[l] = make_double2(v.real(), v.imag());
    isc[l] = make_double2(iv.real(), iv.imag());
  }
  CK(dbuf_reserve(pl->d_ad_scale, (MAXLEV + 1) * sizeof(double2)), "alloc");
  CK(dbuf_reserve(pl->d_ad_inv_scale, (MAXLEV + 1) * sizeof(double2)), "alloc");
  CK(cudaMemcpyAsync(pl->d_ad_scale.p, sc.data(), (MAXLEV + 1) * sizeof(double2), cudaMemcpyHostToDevice, s), "upload");
  CK(cudaMemcpyAsync(pl->d_ad_inv_scale.p, isc.data(), (MAXLEV + 1) * sizeof(double2), cudaMemcpyHostToDevice, s), "upload");
  const int64_t need_exp = n_cells * pl->P;
  const size_t csz = f64 ? sizeof(double2) : sizeof(float2);
  CK(dbuf_reserve(pl->d_mQ, n_cells * 8), "alloc");
  CK(dbuf_reserve(pl->d_lL0, n_cells * 8), "alloc");
  CK(dbuf_reserve(pl->d_ma, need_exp * csz), "alloc");
  if (ff_m2l(pl)) CK(dbuf_reserve(pl->d_ma_ff, n_cells * (pl->p + 1) * sizeof(float4)), "alloc");
  CK(dbuf_reserve(pl->d_lb, need_exp * csz), "alloc");
  int bin_h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (pl->p2p_binned)
    CK(cudaMemcpyAsync(bin_h, pl->d_p2p_cnt.p, sizeof(bin_h), cudaMemcpyDeviceToHost, s), "readback");
  int err_g = 0;   // the sorts of the list grouping
  CK(cudaMemcpyAsync(&err_g, pl->d_err.p, 4, cudaMemcpyDeviceToHost, s), "readback");
  CK(cudaStreamSynchronize(s), "build sync");
  if (err_g & 8) return fail(pl, FMM2D_ETIMEOUT, "a bounded wait of the radix sort gave up");
  for (int k = 0; k < 4; ++k) pl->p2p_bin_count[k] = bin_h[k];
  CK(tc_prepare_split(pl), "alloc");
  CK(cudaGetLastError(), "build");
  pl->n_m2l = -1;
  pl->n_p2p_pairs = -1;
  ++pl->build_gen;
  pl->built = true;
  return FMM2D_OK;
}

template <typename R>
fmm2d_status evaluate_adaptive_t(fmm2d_plan *pl, const void *u, double *out, cudaStream_t s) {
  const bool f32_in = (pl->flags & FMM2D_IN_F32) != 0;
  const int L = pl->L;
  R *src4 = (R *)pl->d_src4.p;
  const R *tgt = pl->same_sets ? src4 : (const R *)pl->d_tgt2.p;
  const int tstride = pl->same_sets ? 4 : 2;
  const uint32_t *tperm = (const uint32_t *)(pl->same_sets ? pl->d_perm_s.p : pl->d_perm_t.p);
  AdCells c = ad_cells(pl);
  Cx<R> *ma = (Cx<R> *)pl->d_ma.p, *lb = (Cx<R> *)pl->d_lb.p;
  double *mQ = (double *)pl->d_mQ.p, *lL0 = (double *)pl->d_lL0.p;
  int depth = 0;
  while (depth < L && pl->lev_count[depth + 1] > 0) ++depth;
  ExpandArgs a;
  a.p = pl->p;
  a.P = pl->P;
  a.L = L;
  a.l_min = pl->l_min;
  a.b = pl->b;
  a.n_cls = pl->sten.n_classes;
  a.leaf_first = 0;
  a.n_leaves = pl->n_leaves_ad;
  a.inv_s_re = 1.0;
  a.inv_s_im = 0.0;
  a.leaf_ids = (const int *)pl->d_leaf_ids.p;
  a.cell_lev = c.lev;
  a.inv_scale = (const double2 *)pl->d_ad_inv_scale.p;
  a.child_first = c.child_first;
  a.child_cnt = c.child_cnt;
  a.parent = c.parent;
  {
    StageScope sc(pl, ST_OTHER, s, 1);
    CK(launch_gather_u<R>(u, f32_in, (const uint32_t *)pl->d_perm_s.p, pl->n_src, src4, s), "gather");
    if (is_hybrid(pl))
      CK(launch_gather_u<float>(u, f32_in, (const uint32_t *)pl->d_perm_s.p, pl->n_src,
                                (float *)pl->d_src4f.p, s, true), "gather");
  }
  cudaStream_t f;   // far-field chain on the plan's stream, P2P on s
  CK(far_stream(pl, &f), "far stream");
  if (f != s) {
    CK(cudaEventRecord(pl->ev_fork, s), "fork");
    CK(cudaStreamWaitEvent(f, pl->ev_fork, 0), "fork");
  }
  {
    StageScope sc(pl, ST_P2M, f, 1);
    CK(launch_p2m<R>(a, src4, c.ss, c.se, mQ, ma, f), "p2m");
  }
  {
    StageScope sc(pl, ST_M2M, f, std::max(0, depth - 1));
    for (int l = depth - 1; l >= 1; --l)
      CK(launch_m2m<R>(a, pl->geo, l, pl->lev_first[l], pl->lev_count[l], nullptr, c.key, c.cls,
                       c.hsrc, (const Cx<R> *)pl->d_m2m_ops.p, mQ, ma, pl->n_sms, f), "m2m");
  }
  {
    // cells above the first M2L level get no M2L write: their locals (read by
    // L2P when such a cell is a leaf) start at zero
    const int64_t ff = pl->n_cells - pl->n_far_cells;
    if (ff > 0) {
      CK(cudaMemsetAsync(lL0, 0, ff * sizeof(double), f), "zero locals");
      CK(cudaMemsetAsync(lb, 0, ff * pl->P * sizeof(Cx<R>), f), "zero locals");
    }
  }
  if (pl->n_far_cells == 0) {
  } else if constexpr (sizeof(R) == 4) {
    if ((pl->flags & FMM2D_PREC_MASK) == FMM2D_PREC_MIXED_TC) {
      StageScope sc(pl, ST_M2L, f, pl->tc_split_n > 1 ? 2 : 1);
      TcArgs t;
      t.p = pl->p;
      t.P = pl->P;
      t.n_classes = pl->sten.n_classes;
      t.sms = pl->n_sms;
      t.far_first = pl->n_cells - pl->n_far_cells;
      t.cls_cap = pl->cls_cap;
      t.cls_cnt = (const int *)pl->d_cls_cnt.p;
      t.cls_cells = (const int *)pl->d_cls_cells.p;
      t.far_full = (const int *)pl->d_far_full.p;
      t.sten_ops = (const uint16_t *)((const char *)pl->d_sten.p + offsetof(Stencils, far_op));
      t.sten_len = (const int *)((const char *)pl->d_sten.p + offsetof(Stencils, far_len));
      t.btab = (const unsigned char *)pl->d_tc_ops.p;
      t.logz = (const double *)pl->d_m2l_logz.p;
      t.log_abs_scale = (const double *)pl->d_geo_scale.p;
      t.lev_first = (const int64_t *)pl->d_lev_first.p;
      t.l_min = pl->l_min;
      t.L = L;
      t.mQ = mQ;
      t.ma = (const float2 *)ma;
      t.lL0 = lL0;
      t.lb = (float2 *)lb;
      t.err = (int *)pl->d_dev_err.p;
      t.split = pl->tc_split_n;
      t.part_lb = (float2 *)pl->d_tc_part_lb.p;
      t.part_L0 = (double *)pl->d_tc_part_L0.p;
      t.n_far = pl->n_far_cells;
      t.debug_stall = pl->debug_stall;
      CK(cudaMemsetAsync(pl->d_dev_err.p, 0, 4, f), "memset");
      CK(launch_m2l_tc(t, pl->tc_K, pl->tc_N, pl->n_far_cells, f), "m2l_tc");
    } else {
      StageScope sc(pl, ST_M2L, f, 1);
      const int64_t ff = pl->n_cells - pl->n_far_cells;
      CK(launch_m2l<R>(a, ff, pl->n_far_cells, (const int64_t *)pl->d_lev_first.p,
                       (const double *)pl->d_geo_scale.p, 0, (const int *)pl->d_far_cnt.p,
                       (const int *)pl->d_far_src.p, (const uint16_t *)pl->d_far_op.p,
                       (const Cx<R> *)pl->d_m2l_ops.p, (const double *)pl->d_m2l_logz.p, mQ, ma,
                       lL0, lb, f), "m2l");
    }
  } else if (ff_m2l(pl)) {
    StageScope sc(pl, ST_M2L, f, 1);
    CK(run_m2l_ff(pl, L, pl->n_cells - pl->n_far_cells, mQ, ma, lL0, lb, f), "m2l_ff");
  } else {
    StageScope sc(pl, ST_M2L, f, 1);
    const int64_t ff = pl->n_cells - pl->n_far_cells;
    CK(launch_m2l<R>(a, ff, pl->n_far_cells, (const int64_t *)pl->d_lev_first.p,
                     (const double *)pl->d_geo_scale.p, 0, (const int *)pl->d_far_cnt.p,
                     (const int *)pl->d_far_src.p, (const uint16_t *)pl->d_far_op.p,
                     (const Cx<R> *)pl->d_m2l_ops.p, (const double *)pl->d_m2l_logz.p, mQ, ma, lL0,
                     lb, f), "m2l");
  }
  {
    StageScope sc(pl, ST_M2L, f, 1);   // P2L (X lists) completes the locals before L2L
    CK(ad_launch_p2l<R>(pl->n_cells, (const int *)pl->d_x_off.p, (const int *)pl->d_x_src.p, src4,
                        c.ss, c.se, c.ctr, c.lev, (const double2 *)pl->d_ad_inv_scale.p, pl->p,
                        pl->P, lL0, lb, f), "p2l");
  }
  {
    StageScope sc(pl, ST_L2L, f, std::max(0, depth - pl->l_min));
    for (int l = pl->l_min + 1; l <= depth; ++l)
      CK(launch_l2l<R>(a, pl->geo, l, pl->lev_first[l], pl->lev_count[l], nullptr, c.key, c.cls,
                       (const Cx<R> *)pl->d_l2l_ops.p, lL0, lb, pl->n_sms, f), "l2l");
  }
  {
    StageScope sc(pl, ST_P2P, s, 1);
    if (is_hybrid(pl)) {   // FP32 P2P on the FP32 copies
      const float *s4 = (const float *)pl->d_src4f.p;
      CK(launch_p2p<float>(0, pl->n_leaves_ad, (const int *)pl->d_leaf_ids.p, s4,
                           pl->same_sets ? s4 : (const float *)pl->d_tgt2f.p, tstride, c.ss, c.se,
                           c.ts, c.te, nullptr, (const int *)pl->d_u_off.p,
                           (const int *)pl->d_u_src.p, c.ctr, (double *)pl->d_phi_near.p,
                           (double)std::max(1, pl->leaf_cap), s, (const float2 *)pl->d_srclo.p,
                           (const float2 *)(pl->same_sets ? pl->d_srclo.p : pl->d_tgtlo.p),
                           (const int *)pl->d_p2p_order.p, pl->p2p_bin_count),
         "p2p");
    } else
    CK(launch_p2p<R>(0, pl->n_leaves_ad, (const int *)pl->d_leaf_ids.p, src4, tgt, tstride, c.ss,
                     c.se, c.ts, c.te, nullptr, (const int *)pl->d_u_off.p,
                     (const int *)pl->d_u_src.p, c.ctr, (double *)pl->d_phi_near.p,
                     (double)std::max(1, pl->leaf_cap), s, nullptr, nullptr,
                     // FP32: the group size of each leaf follows its own target
                     // count, so that a leaf's sum does not depend on the other
                     // leaves (or instances)
                     pl->p2p_binned ? (const int *)pl->d_p2p_order.p : nullptr,
                     pl->p2p_binned ? pl->p2p_bin_count : nullptr),
       "p2p");
  }
  if (f != s) {   // join: M2P and L2P need the expansions
    CK(cudaEventRecord(pl->ev_join, f), "join");
    CK(cudaStreamWaitEvent(s, pl->ev_join, 0), "join");
  }
  {
    StageScope sc(pl, ST_P2P, s, 1);
    CK(ad_launch_m2p<R>(pl->n_leaves_ad, (const int *)pl->d_leaf_ids.p, (const int *)pl->d_w_off.p,
                        (const int *)pl->d_w_src.p, tgt, tstride, c.ts, c.te, c.ctr, c.lev,
                        (const double2 *)pl->d_ad_scale.p, pl->p, pl->P, mQ, ma,
                        (double *)pl->d_phi_near.p, s), "m2p");
  }
  {
    StageScope sc(pl, ST_L2P, s, 1);
    CK(launch_l2p<R>(a, tgt, tstride, c.ts, c.te, tperm, lL0, lb, (const double *)pl->d_phi_near.p,
                     (double *)pl->d_phi_far.p, out, s), "l2p");
  }
  return FMM2D_OK;
}

// The field F = sum u / (y - x) after an evaluation on s (the strengths are
// gathered and the locals final): P2P' (and M2P' on adaptive trees) into the
// near part, then L2P' adds the far part and writes the caller's order.
template <typename R>
fmm2d_status field_t(fmm2d_plan *pl, double *field, cudaStream_t s) {
  const bool ad = (pl->flags & FMM2D_ADAPTIVE) != 0;
  const int L = pl->L;
  const R *src4 = (const R *)pl->d_src4.p;
  const R *tgt = pl->same_sets ? src4 : (const R *)pl->d_tgt2.p;
  const int tstride = pl->same_sets ? 4 : 2;
  const uint32_t *tperm = (const uint32_t *)(pl->same_sets ? pl->d_perm_s.p : pl->d_perm_t.p);
  const int *ss = (const int *)pl->d_src_start.p, *se = (const int *)pl->d_src_end.p;
  const int *ts = pl->same_sets ? ss : (const int *)pl->d_tgt_start.p;
  const int *te = pl->same_sets ? se : (const int *)pl->d_tgt_end.p;
  const double2 *ctr = (const double2 *)pl->d_cell_ctr.p;
  CK(dbuf_reserve(pl->d_fnear, std::max<int64_t>(1, pl->n_tgt) * sizeof(double2)), "alloc");
  double2 *fnear = (double2 *)pl->d_fnear.p;
  ExpandArgs a;
  a.p = pl->p;
  a.P = pl->P;
  a.L = L;
  a.l_min = pl->l_min;
  a.b = pl->b;
  a.n_cls = pl->sten.n_classes;
  if (ad) {
    a.leaf_first = 0;
    a.n_leaves = pl->n_leaves_ad;
    a.inv_s_re = 1.0;
    a.inv_s_im = 0.0;
    a.leaf_ids = (const int *)pl->d_leaf_ids.p;
    a.cell_lev = (const uint8_t *)pl->d_cell_lev.p;
    a.inv_scale = (const double2 *)pl->d_ad_inv_scale.p;
  } else {
    a.leaf_first = pl->lev_first[L];
    a.n_leaves = pl->lev_count[L];
    const cd inv_s = 1.0 / cd(pl->scale_re[L], pl->scale_im[L]);
    a.inv_s_re = inv_s.real();
    a.inv_s_im = inv_s.imag();
  }
  StageScope sc(pl, ST_FIELD, s, ad ? 3 : 2);
  // FP32 forms: the low parts of the coordinates give accurate differences
  const float2 *slo = sizeof(R) == 4 ? (const float2 *)pl->d_srclo.p : nullptr;
  const float2 *tlo = sizeof(R) == 4 ? (const float2 *)(pl->same_sets ? pl->d_srclo.p : pl->d_tgtlo.p)
                                     : nullptr;
  if (ad) {
    CK(launch_p2p_field<R>(0, pl->n_leaves_ad, a.leaf_ids, src4, tgt, tstride, ss, se, ts, te,
                           nullptr, (const int *)pl->d_u_off.p, (const int *)pl->d_u_src.p, ctr,
                           fnear, s, slo, tlo), "p2p field");
    CK(launch_m2p_field<R>(pl->n_leaves_ad, a.leaf_ids, (const int *)pl->d_w_off.p,
                           (const int *)pl->d_w_src.p, tgt, tstride, ts, te, ctr, a.cell_lev,
                           (const double2 *)pl->d_ad_scale.p, pl->p, pl->P,
                           (const double *)pl->d_mQ.p, (const Cx<R> *)pl->d_ma.p, fnear, s),
       "m2p field");
  } else {
    CK(launch_p2p_field<R>(a.leaf_first, a.n_leaves, nullptr, src4, tgt, tstride, ss, se, ts, te,
                           (const int *)pl->d_near_cnt.p, nullptr, (const int *)pl->d_near_src.p,
                           ctr, fnear, s, slo, tlo), "p2p field");
  }
  CK(launch_l2p_field<R>(a, tgt, tstride, ts, te, tperm, (const Cx<R> *)pl->d_lb.p, fnear,
                         (double2 *)field, s), "l2p field");
  return FMM2D_OK;
}

// Every device buffer a plan owns.
template <typename F>
static void for_each_dbuf(fmm2d_plan *pl, F f) {
  DBuf *const bufs[] = {&pl->d_key_s, &pl->d_perm_s, &pl->d_key_t, &pl->d_perm_t, &pl->d_tmp_k,
                  &pl->d_tmp_v, &pl->d_sort_scratch, &pl->d_err, &pl->d_occ, &pl->d_hsrc,
                  &pl->d_scan, &pl->d_map, &pl->d_cell_key, &pl->d_cell_crd, &pl->d_cell_ctr,
                  &pl->d_cell_cls, &pl->d_cell_hsrc, &pl->d_src_start, &pl->d_src_end,
                  &pl->d_tgt_start, &pl->d_tgt_end, &pl->d_lev_first, &pl->d_far_cnt,
                  &pl->d_far_src, &pl->d_far_op, &pl->d_near_cnt, &pl->d_near_src, &pl->d_src4,
                  &pl->d_tgt2, &pl->d_mQ, &pl->d_ma, &pl->d_ma_ff, &pl->d_lL0, &pl->d_lb, &pl->d_phi_near,
                  &pl->d_fnear, &pl->d_tc_part_lb, &pl->d_tc_part_L0, &pl->d_m2m_arrive, &pl->d_l2l_ready,
                  &pl->d_ad_hash, &pl->d_pmap,
                  &pl->d_phi_far, &pl->d_sten, &pl->d_geo_scale, &pl->d_m2l_ops, &pl->d_m2l_logz,
                  &pl->d_m2m_ops, &pl->d_l2l_ops, &pl->d_counts, &pl->d_far_full,
                  &pl->d_cls_cnt, &pl->d_cls_cells, &pl->d_tc_ops, &pl->d_ff_ops, &pl->d_ff_ph, &pl->d_dev_err,
                  &pl->d_p2p_order, &pl->d_p2p_cnt,
                  &pl->d_cell_lev, &pl->d_parent, &pl->d_child_first, &pl->d_child_cnt,
                  &pl->d_split, &pl->d_leaf_ids, &pl->d_leaf_pos, &pl->d_ad_scale,
                  &pl->d_ad_inv_scale, &pl->d_u_off, &pl->d_u_src, &pl->d_w_off, &pl->d_w_src,
                  &pl->d_x_off, &pl->d_x_src, &pl->d_ad_flag, &pl->d_ad_pos, &pl->d_ad_crange,
                  &pl->d_ad_cnt, &pl->d_ad_off, &pl->d_ad_tot, &pl->d_ad_ta, &pl->d_ad_tc,
                  &pl->d_ad_sa, &pl->d_ad_sc, &pl->d_ad_ta2, &pl->d_ad_tc2, &pl->d_ad_sa2,
                  &pl->d_ad_sc2, &pl->d_ad_ut, &pl->d_ad_us, &pl->d_ad_wt, &pl->d_ad_ws,
                  &pl->d_ad_xt, &pl->d_ad_xs, &pl->d_inst_off, &pl->d_src4f, &pl->d_tgt2f, &pl->d_srclo,
                  &pl->d_tgtlo};
  for (DBuf *b : bufs) f(*b);
}

namespace fmm2d {
size_t plan_device_bytes(const fmm2d_plan *cpl) {
  size_t tot = 0;
  for_each_dbuf(const_cast<fmm2d_plan *>(cpl), [&](DBuf &b) { tot += b.bytes; });
  return tot;
}
}  // namespace fmm2d

extern "C" {

fmm2d_status fmm2d_evaluate_field(fmm2d_plan *pl, const void *u, double *out, double *field,
                                  void *stream) {
  if (!pl) return FMM2D_EINVAL;
  if (pl->built && pl->n_tgt > 0 && !field) return fail(pl, FMM2D_EINVAL, "null field pointer");
  if (!is_fp64(pl) && !(pl->flags & FMM2D_FIELD))
    return fail(pl, FMM2D_EINVAL, "FP32 forms need a plan created with FMM2D_FIELD");
  const fmm2d_status st = fmm2d_evaluate(pl, u, out, stream);
  if (st != FMM2D_OK || pl->n_tgt == 0) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (is_fp64(pl)) return field_t<double>(pl, field, s);
  return field_t<float>(pl, field, s);
}

fmm2d_status fmm2d_default_params(int tiling, int64_t n_points, int leaf_target, double eps,
                                  int *levels_out, int *p_out, double *leaf_scale_out) {
  if (tiling < 0 || tiling > 2 || n_points < 0 || !(eps > 0.0 && eps < 1.0) || leaf_target < 0)
    return FMM2D_EINVAL;
  const int p = p_from_eps(tiling, eps);
  int L = leaf_target > 0 ? auto_levels(tiling, n_points, leaf_target)
                          : planner_sopt_levels(tiling, n_points, n_points, p);
  if (levels_out) *levels_out = L;
  if (p_out) *p_out = p;
  if (leaf_scale_out) {
    if (tiling == FMM2D_QUAD) *leaf_scale_out = std::ldexp(1.0, -L);
    else if (tiling == FMM2D_TRI) *leaf_scale_out = tri_rho0();
    else *leaf_scale_out = sept_leaf_r(L);
  }
  return FMM2D_OK;
}

fmm2d_status fmm2d_plan_create(int tiling, int levels, int p, double eps, unsigned flags,
                               fmm2d_plan **out) {
  if (!out) return FMM2D_EINVAL;
  *out = nullptr;
  if (tiling < 0 || tiling > 2) { g_create_err = "unknown tiling"; return FMM2D_EINVAL; }
  if (levels < 0 || levels > max_levels_for(tiling, flags)) { g_create_err = "levels out of range"; return FMM2D_EINVAL; }
  if (p < 0 || p > MAXP) { g_create_err = "p out of range (0..48)"; return FMM2D_EINVAL; }
  if (p == 0 && !(eps > 0.0 && eps < 1.0)) { g_create_err = "eps must be in (0, 1)"; return FMM2D_EINVAL; }
  if ((flags & ~(FMM2D_PREC_MASK | FMM2D_IN_F32 | FMM2D_ADAPTIVE | FMM2D_FIELD)) != 0 ||
      (flags & FMM2D_PREC_MASK) > FMM2D_PREC_SPLIT) {
    g_create_err = "unknown flags";
    return FMM2D_EINVAL;
  }
  fmm2d_plan *pl = new (std::nothrow) fmm2d_plan();
  if (!pl) { g_create_err = "out of host memory"; return FMM2D_ENOMEM; }
  pl->tiling = tiling;
  pl->levels_req = levels;
  pl->p_req = p;
  pl->eps = eps;
  pl->flags = flags;
  pl->b = tiling == FMM2D_SEPT ? 7 : 4;
  pl->l_min = tiling == FMM2D_SEPT ? 1 : 2;
  *out = pl;
  return FMM2D_OK;
}

fmm2d_status fmm2d_plan_set_params(fmm2d_plan *pl, int levels, int p, double eps) {
  if (!pl) return FMM2D_EINVAL;
  if (levels < 0 || levels > max_levels_for(pl->tiling, pl->flags))
    return fail(pl, FMM2D_EINVAL, "levels out of range");
  if (p < 0 || p > MAXP) return fail(pl, FMM2D_EINVAL, "p out of range (0..48)");
  if (p == 0 && !(eps > 0.0 && eps < 1.0)) return fail(pl, FMM2D_EINVAL, "eps must be in (0, 1)");
  pl->levels_req = levels;
  pl->p_req = p;
  pl->eps = eps;
  pl->built = false;
  return FMM2D_OK;
}

fmm2d_status fmm2d_plan_set_leaf_size(fmm2d_plan *pl, int leaf_size) {
  if (!pl) return FMM2D_EINVAL;
  if (leaf_size < 0) return fail(pl, FMM2D_EINVAL, "leaf size must be >= 0");
  pl->leaf_cap = leaf_size;
  pl->built = false;
  return FMM2D_OK;
}

fmm2d_status fmm2d_plan_set_domain(fmm2d_plan *pl, double x0, double y0, double size) {
  if (!pl) return FMM2D_EINVAL;
  if (!(size > 0.0) || !std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(size))
    return fail(pl, FMM2D_EINVAL, "domain size must be positive and finite");
  pl->x0 = x0;
  pl->y0 = y0;
  pl->S = size;
  pl->built = false;
  return FMM2D_OK;
}

fmm2d_status fmm2d_build(fmm2d_plan *pl, const void *src, int64_t n_src, const void *tgt,
                         int64_t n_tgt, void *stream) {
  if (!pl) return FMM2D_EINVAL;
  pl->built = false;
  if (n_src < 0 || n_tgt < 0) return fail(pl, FMM2D_EINVAL, "negative point count");
  if ((n_src > 0 && !src) || (n_tgt > 0 && !tgt)) return fail(pl, FMM2D_EINVAL, "null point pointer");
  if (n_src >= (int64_t)INT_MAX || n_tgt >= (int64_t)INT_MAX) return fail(pl, FMM2D_EINVAL, "too many points");
  cudaStream_t s = (cudaStream_t)stream;
  pl->last_stream = s;
  const bool f32 = (pl->flags & FMM2D_IN_F32) != 0;
  const bool f64 = is_fp64(pl);
  pl->same_sets = (src == tgt && n_src == n_tgt);
  pl->n_src = n_src;
  pl->n_tgt = n_tgt;
  if (pl->flags & FMM2D_ADAPTIVE) return build_adaptive(pl, src, n_src, tgt, n_tgt, s);
  int L = pl->levels_req, p = pl->p_req;
  if (L == 0) L = auto_levels(pl->tiling, std::max(n_src, n_tgt), 64);
  if (p == 0) p = p_from_eps(pl->tiling, pl->eps);
  if (L < 1 || L > max_levels(pl->tiling)) return fail(pl, FMM2D_EINVAL, "levels out of range");
  const bool tc_form = (pl->flags & FMM2D_PREC_MASK) == FMM2D_PREC_MIXED_TC;
  if (tc_form && !tc_shape(p, &pl->tc_K, &pl->tc_N))
    return fail(pl, FMM2D_EINVAL, "tensor-core M2L supports p <= 31");
  const bool tc = tc_form || ff_m2l(pl);   // class lists: tensor-core and float-float M2L
  pl->L = L;
  pl->p = p;
  pl->P = (p + 1) & ~1;   // even stride: rows of complex values stay 16-byte aligned
  fmm2d_status st = setup_geometry(pl);
  if (st != FMM2D_OK) return st;
  const Geo &g = pl->geo;
  const int64_t nmax = std::max<int64_t>(1, std::max(n_src, n_tgt));
  // ---- buffers sized by points
  CK(dbuf_reserve(pl->d_key_s, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_perm_s, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_key_t, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_perm_t, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_tmp_k, nmax * 4), "alloc");
  CK(dbuf_reserve(pl->d_tmp_v, nmax * 4), "alloc");
  size_t scr = std::max(radix_sort_scratch_bytes(nmax), scan_scratch_bytes(pl->map_size));
  CK(dbuf_reserve(pl->d_sort_scratch, scr), "alloc");
  const size_t rsz = f64 ? sizeof(double) : sizeof(float);
  CK(dbuf_reserve(pl->d_src4, std::max<int64_t>(1, n_src) * 4 * rsz), "alloc");
  CK(dbuf_reserve(pl->d_tgt2, std::max<int64_t>(1, n_tgt) * 2 * rsz), "alloc");
  CK(dbuf_reserve(pl->d_phi_near, std::max<int64_t>(1, n_tgt) * 8), "alloc");
  CK(dbuf_reserve(pl->d_phi_far, std::max<int64_t>(1, n_tgt) * 8), "alloc");
  CK(dbuf_reserve(pl->d_err, 16), "alloc");
  CK(dbuf_reserve(pl->d_lev_first, (MAXLEV + 2) * 8), "alloc");
  // ---- map-sized buffers
  const int64_t ms = pl->map_size;
  CK(dbuf_reserve(pl->d_occ, ms * 4), "alloc");
  CK(dbuf_reserve(pl->d_hsrc, ms * 4), "alloc");
  CK(dbuf_reserve(pl->d_scan, ms * 4), "alloc");
  CK(dbuf_reserve(pl->d_map, ms * 4), "alloc");
  const bool use_pmap = g.tiling == FMM2D_TRI;
  if (use_pmap) CK(dbuf_reserve(pl->d_pmap, 2 * (((int64_t)1 << (2 * (pl->L + 1))) - 1) / 3 * 4), "alloc");
  const int64_t cap = ms;   // upper bound on occupied cells
  CK(dbuf_reserve(pl->d_cell_key, cap * 4), "alloc");
  CK(dbuf_reserve(pl->d_cell_crd, cap * sizeof(int4)), "alloc");
  CK(dbuf_reserve(pl->d_cell_ctr, cap * sizeof(double2)), "alloc");
  CK(dbuf_reserve(pl->d_cell_cls, cap), "alloc");
  CK(dbuf_reserve(pl->d_cell_hsrc, cap), "alloc");

  CK(cudaMemsetAsync(pl->d_err.p, 0, 16, s), "memset");
  const int bits = key_bits(pl->tiling, L);
  uint32_t *ks = (uint32_t *)pl->d_key_s.p, *ps = (uint32_t *)pl->d_perm_s.p;
  uint32_t *kt = (uint32_t *)pl->d_key_t.p, *pt = (uint32_t *)pl->d_perm_t.p;
  {
    StageScope sc(pl, ST_KEYS, s, pl->same_sets ? 1 : 2);
    CK(launch_keys(g, src, f32, n_src, ks, ps, (int *)pl->d_err.p, s, (uint32_t *)pl->d_tmp_v.p,
                   (int *)pl->d_err.p + 2), "keys");
    if (!pl->same_sets)
      CK(launch_keys(g, tgt, f32, n_tgt, kt, pt, (int *)pl->d_err.p, s, (uint32_t *)pl->d_tmp_v.p,
                     (int *)pl->d_err.p + 2), "keys");
  }
  {
    StageScope sc(pl, ST_SORT, s,
                  radix_sort_launches(n_src, bits) + (pl->same_sets ? 0 : radix_sort_launches(n_tgt, bits)));
    CK(radix_sort_pairs(ks, ps, (uint32_t *)pl->d_tmp_k.p, (uint32_t *)pl->d_tmp_v.p, n_src, bits,
                        pl->d_sort_scratch.p, s, (int *)pl->d_err.p), "sort");
    if (!pl->same_sets)
      CK(radix_sort_pairs(kt, pt, (uint32_t *)pl->d_tmp_k.p, (uint32_t *)pl->d_tmp_v.p, n_tgt, bits,
                          pl->d_sort_scratch.p, s, (int *)pl->d_err.p), "sort");
  }
  // ---- capacities: a level holds at most min(b^l, points) occupied cells,
  // so every later buffer and launch can be sized before the counts are known
  // and the build needs no host synchronisation until its end
  const int64_t npts = pl->same_sets ? n_src : n_src + n_tgt;
  int64_t cap_l[MAXLEV + 2], cap_cells = 0, pw = 1;
  for (int l = 0; l <= L; ++l) {
    cap_l[l] = std::max<int64_t>(1, std::min<int64_t>(pw, npts));
    cap_cells += cap_l[l];
    pw = pw > ((int64_t)1 << 40) ? pw : pw * pl->b;
  }
  const int lo_level = L >= pl->l_min ? pl->l_min : L;   // first level with lists
  int64_t cap_list = 0;
  for (int l = lo_level; l <= L; ++l) cap_list += cap_l[l];
  const int64_t cap_leaf = cap_l[L];
  const size_t csz = f64 ? sizeof(double2) : sizeof(float2);
  CK(dbuf_reserve(pl->d_src_start, cap_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_src_end, cap_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_tgt_start, cap_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_tgt_end, cap_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_mQ, cap_cells * 8), "alloc");
  CK(dbuf_reserve(pl->d_m2m_arrive, cap_cells * 4), "alloc");
  CK(dbuf_reserve(pl->d_l2l_ready, (cap_cells + 2) * 4), "alloc");
  CK(dbuf_reserve(pl->d_lL0, cap_cells * 8), "alloc");
  CK(dbuf_reserve(pl->d_ma, cap_cells * pl->P * csz), "alloc");
  if (ff_m2l(pl)) CK(dbuf_reserve(pl->d_ma_ff, cap_cells * (pl->p + 1) * sizeof(float4)), "alloc");
  CK(dbuf_reserve(pl->d_lb, cap_cells * pl->P * csz), "alloc");
  CK(dbuf_reserve(pl->d_far_cnt, cap_list * 4), "alloc");
  CK(dbuf_reserve(pl->d_far_src, cap_list * FAR_MAX * 4), "alloc");
  CK(dbuf_reserve(pl->d_far_op, cap_list * FAR_MAX * 2), "alloc");
  if (tc) {
    CK(dbuf_reserve(pl->d_far_full, cap_list * FAR_MAX * 4), "alloc");
    CK(dbuf_reserve(pl->d_cls_cnt, MAX_CLASSES * 4), "alloc");
    CK(dbuf_reserve(pl->d_cls_cells, (size_t)MAX_CLASSES * cap_list * 4), "alloc");
  }
  CK(dbuf_reserve(pl->d_dev_err, 16), "alloc");
  CK(dbuf_reserve(pl->d_near_cnt, cap_leaf * 4), "alloc");
  CK(dbuf_reserve(pl->d_near_src, cap_leaf * NEAR_MAX * 4), "alloc");
  pl->cls_cap = cap_list;
  {
    StageScope sc(pl, ST_TREE, s, (pl->same_sets ? 1 : 2) + exclusive_scan_launches(ms) + 1);
    CK(cudaMemsetAsync(pl->d_occ.p, 0, ms * 4, s), "memset");
    CK(cudaMemsetAsync(pl->d_hsrc.p, 0, ms * 4, s), "memset");
    CK(launch_mark(g, ks, n_src, (int *)pl->d_occ.p, (int *)pl->d_hsrc.p, s), "mark");
    if (!pl->same_sets) CK(launch_mark(g, kt, n_tgt, (int *)pl->d_occ.p, nullptr, s), "mark");
    CK(exclusive_scan((const int *)pl->d_occ.p, (int *)pl->d_scan.p, ms, pl->d_sort_scratch.p, s), "scan");
    CK(launch_compact(g, (const int *)pl->d_occ.p, (const int *)pl->d_scan.p, (const int *)pl->d_hsrc.p,
                      ms, (int *)pl->d_map.p, (uint32_t *)pl->d_cell_key.p, (int4 *)pl->d_cell_crd.p,
                      (double2 *)pl->d_cell_ctr.p, (uint8_t *)pl->d_cell_cls.p,
                      (uint8_t *)pl->d_cell_hsrc.p, (int *)pl->d_src_start.p, (int *)pl->d_src_end.p,
                      pl->same_sets ? nullptr : (int *)pl->d_tgt_start.p,
                      pl->same_sets ? nullptr : (int *)pl->d_tgt_end.p, (int64_t *)pl->d_lev_first.p,
                      use_pmap ? (int *)pl->d_pmap.p : nullptr, s), "compact");
  }
  {
    StageScope sc(pl, ST_TREE, s, pl->same_sets ? 1 : 2);
    // FP32 forms of a field plan: also the low parts of the leaf-relative
    // coordinates (the accurate pair differences of the field's P2P)
    const bool keep_lo = !f64 && (pl->flags & FMM2D_FIELD);
    if (keep_lo) {
      CK(dbuf_reserve(pl->d_srclo, std::max<int64_t>(1, n_src) * 8), "alloc");
      if (!pl->same_sets) CK(dbuf_reserve(pl->d_tgtlo, std::max<int64_t>(1, n_tgt) * 8), "alloc");
    }
    CK(launch_rel_coords(g, f32, !f64, src, ps, ks, n_src, (const int *)pl->d_map.p,
                         (const double2 *)pl->d_cell_ctr.p, pl->d_src4.p, 4, (int *)pl->d_src_start.p,
                         (int *)pl->d_src_end.p, s, keep_lo ? (float2 *)pl->d_srclo.p : nullptr), "rel");
    if (!pl->same_sets)
      CK(launch_rel_coords(g, f32, !f64, tgt, pt, kt, n_tgt, (const int *)pl->d_map.p,
                           (const double2 *)pl->d_cell_ctr.p, pl->d_tgt2.p, 2,
                           (int *)pl->d_tgt_start.p, (int *)pl->d_tgt_end.p, s,
                           keep_lo ? (float2 *)pl->d_tgtlo.p : nullptr), "rel");
    if (is_hybrid(pl)) {   // FP32 hi + lo copies for the P2P
      CK(dbuf_reserve(pl->d_src4f, std::max<int64_t>(1, n_src) * 16), "alloc");
      CK(dbuf_reserve(pl->d_srclo, std::max<int64_t>(1, n_src) * 8), "alloc");
      CK(launch_rel_coords(g, f32, true, src, ps, ks, n_src, (const int *)pl->d_map.p,
                           (const double2 *)pl->d_cell_ctr.p, pl->d_src4f.p, 4,
                           (int *)pl->d_src_start.p, (int *)pl->d_src_end.p, s,
                           (float2 *)pl->d_srclo.p), "rel");
      if (!pl->same_sets) {
        CK(dbuf_reserve(pl->d_tgt2f, std::max<int64_t>(1, n_tgt) * 8), "alloc");
        CK(dbuf_reserve(pl->d_tgtlo, std::max<int64_t>(1, n_tgt) * 8), "alloc");
        CK(launch_rel_coords(g, f32, true, tgt, pt, kt, n_tgt, (const int *)pl->d_map.p,
                             (const double2 *)pl->d_cell_ctr.p, pl->d_tgt2f.p, 2,
                             (int *)pl->d_tgt_start.p, (int *)pl->d_tgt_end.p, s,
                             (float2 *)pl->d_tgtlo.p), "rel");
      }
    }
  }
  {
    StageScope sc(pl, ST_LISTS, s, 1);
    if (tc) CK(cudaMemsetAsync(pl->d_cls_cnt.p, 0, MAX_CLASSES * 4, s), "memset");
    CK(cudaMemsetAsync(pl->d_dev_err.p, 0, 16, s), "memset");
    CK(launch_lists(g, (const Stencils *)pl->d_sten.p, lo_level, pl->l_min, cap_list,
                    (const int *)pl->d_map.p, (const uint8_t *)pl->d_cell_cls.p,
                    (const int4 *)pl->d_cell_crd.p, (const uint8_t *)pl->d_cell_hsrc.p,
                    (int *)pl->d_far_cnt.p, (int *)pl->d_far_src.p, (uint16_t *)pl->d_far_op.p,
                    (int *)pl->d_near_cnt.p, (int *)pl->d_near_src.p,
                    (const int64_t *)pl->d_lev_first.p, tc ? (int *)pl->d_far_full.p : nullptr,
                    tc ? (int *)pl->d_cls_cnt.p : nullptr, tc ? (int *)pl->d_cls_cells.p : nullptr,
                    cap_list, use_pmap ? (const int *)pl->d_pmap.p : nullptr, s), "lists");
  }
  // ---- the one synchronisation: level counts for the evaluation and the
  // domain check
  int64_t lev_first_h[MAXLEV + 2];
  int err_h = 0;
  CK(cudaMemcpyAsync(lev_first_h, pl->d_lev_first.p, (L + 2) * 8, cudaMemcpyDeviceToHost, s), "readback");
  CK(cudaMemcpyAsync(&err_h, pl->d_err.p, 4, cudaMemcpyDeviceToHost, s), "readback");
  CK(cudaStreamSynchronize(s), "build sync");
  if (err_h & 8) return fail(pl, FMM2D_ETIMEOUT, "a bounded wait of the radix sort gave up");
  if (err_h) return fail(pl, FMM2D_EDOMAIN, "a point lies outside the domain square or root cell");
  for (int l = 0; l <= L + 1; ++l) pl->lev_first[l] = lev_first_h[l];
  pl->n_cells = lev_first_h[L + 1];
  for (int l = 0; l <= L; ++l) pl->lev_count[l] = pl->lev_first[l + 1] - pl->lev_first[l];
  for (int l = L + 1; l <= MAXLEV + 1; ++l) pl->lev_first[l] = pl->n_cells;
  const int64_t lfirst = L >= pl->l_min ? pl->lev_first[pl->l_min] : pl->n_cells;
  pl->n_far_cells = pl->n_cells - lfirst;
  CK(tc_prepare_split(pl), "alloc");
  CK(cudaGetLastError(), "build");
  pl->n_m2l = -1;
  pl->n_p2p_pairs = -1;
  ++pl->build_gen;
  pl->built = true;
  return FMM2D_OK;
}

fmm2d_status fmm2d_build_forest(fmm2d_plan *pl, const void *xy, const int64_t *offsets, int n_inst,
                                void *stream) {
  if (!pl) return FMM2D_EINVAL;
  pl->built = false;
  if (!(pl->flags & FMM2D_ADAPTIVE)) return fail(pl, FMM2D_EINVAL, "forest builds need an FMM2D_ADAPTIVE plan");
  if (n_inst < 1 || !offsets) return fail(pl, FMM2D_EINVAL, "need n_inst >= 1 and offsets");
  if (offsets[0] != 0) return fail(pl, FMM2D_EINVAL, "offsets[0] must be 0");
  for (int i = 0; i < n_inst; ++i)
    if (offsets[i + 1] < offsets[i]) return fail(pl, FMM2D_EINVAL, "offsets must not decrease");
  const int64_t n = offsets[n_inst];
  if (n > 0 && !xy) return fail(pl, FMM2D_EINVAL, "null point pointer");
  if (n >= (int64_t)INT_MAX) return fail(pl, FMM2D_EINVAL, "too many points");
  cudaStream_t s = (cudaStream_t)stream;
  pl->last_stream = s;
  pl->same_sets = true;
  pl->n_src = n;
  pl->n_tgt = n;
  return build_adaptive(pl, xy, n, xy, n, s, n_inst, offsets);
}

static fmm2d_status evaluate_dispatch(fmm2d_plan *pl, const void *u, double *out, cudaStream_t s) {
  if (pl->flags & FMM2D_ADAPTIVE) {
    if (is_fp64(pl)) return evaluate_adaptive_t<double>(pl, u, out, s);
    return evaluate_adaptive_t<float>(pl, u, out, s);
  }
  if (is_fp64(pl)) return evaluate_t<double>(pl, u, out, s);
  return evaluate_t<float>(pl, u, out, s);
}

fmm2d_status fmm2d_evaluate(fmm2d_plan *pl, const void *u, double *out, void *stream) {
  if (!pl) return FMM2D_EINVAL;
  if (!pl->built) return fail(pl, FMM2D_ENOTREADY, "plan is not built");
  if ((pl->n_src > 0 && !u) || (pl->n_tgt > 0 && !out)) return fail(pl, FMM2D_EINVAL, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  pl->last_stream = s;
  if (pl->n_tgt == 0) return FMM2D_OK;
  return evaluate_dispatch(pl, u, out, s);
}

// The evaluation's launches (both streams, memsets included) recorded once
// into a CUDA graph and then replayed with one launch per call, while the
// build and the strength / potential pointers stay the same.  An evaluation
// makes no allocation and no host synchronisation, so it records whole.
fmm2d_status fmm2d_evaluate_graph(fmm2d_plan *pl, const void *u, double *out, void *stream) {
  if (!pl) return FMM2D_EINVAL;
  if (!pl->built) return fail(pl, FMM2D_ENOTREADY, "plan is not built");
  if ((pl->n_src > 0 && !u) || (pl->n_tgt > 0 && !out)) return fail(pl, FMM2D_EINVAL, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  // the legacy default stream cannot be captured, and profiling records
  // events per stage: both evaluate directly
  if (pl->profiling || s == nullptr || s == cudaStreamLegacy) return fmm2d_evaluate(pl, u, out, stream);
  pl->last_stream = s;
  if (pl->n_tgt == 0) return FMM2D_OK;
  const bool valid = pl->graph_exec && pl->graph_gen == pl->build_gen && pl->graph_u == u &&
                     pl->graph_out == out;
  if (!valid) {
    if (pl->graph_exec) {
      cudaGraphExecDestroy(pl->graph_exec);
      pl->graph_exec = nullptr;
    }
    cudaStream_t f;
    CK(far_stream(pl, &f), "far stream");   // created before, not during, the capture
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
    const fmm2d_status st = evaluate_dispatch(pl, u, out, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (st != FMM2D_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(pl, ec, "end capture");
    }
    // node priorities kept: the far-field chain stays ahead of P2P, as on its stream
    const cudaError_t ei = cudaGraphInstantiate(&pl->graph_exec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      pl->graph_exec = nullptr;
      return cuda_fail(pl, ei, "graph instantiate");
    }
    pl->graph_gen = pl->build_gen;
    pl->graph_u = u;
    pl->graph_out = out;
  }
  CK(cudaGraphLaunch(pl->graph_exec, s), "graph launch");
  return FMM2D_OK;
}

fmm2d_status fmm2d_plan_query(const fmm2d_plan *cpl, fmm2d_info *info) {
  if (!cpl || !info) return FMM2D_EINVAL;
  fmm2d_plan *pl = const_cast<fmm2d_plan *>(cpl);
  std::memset(info, 0, sizeof(*info));
  info->tiling = pl->tiling;
  info->levels = pl->built ? pl->L : pl->levels_req;
  info->p = pl->built ? pl->p : pl->p_req;
  info->l_min = pl->l_min;
  info->flags = pl->flags;
  info->built = pl->built ? 1 : 0;
  info->eps = pl->eps;
  info->domain[0] = pl->x0;
  info->domain[1] = pl->y0;
  info->domain[2] = pl->S;
  info->n_src = pl->n_src;
  info->n_tgt = pl->n_tgt;
  if (!pl->built) return FMM2D_OK;
  info->leaf_scale = pl->geo.leaf_scale;
  for (int l = 0; l <= pl->L && l < 24; ++l) info->n_cells[l] = pl->lev_count[l];
  info->n_m2l_ops = pl->n_ops;
  info->max_far = pl->max_far;
  info->max_near = pl->max_near;
  if (pl->n_m2l < 0 && (pl->flags & FMM2D_ADAPTIVE)) {
    cudaStreamSynchronize(pl->last_stream);
    std::vector<int> fc(std::max<int64_t>(1, pl->n_far_cells));
    int64_t tot = 0;
    if (pl->n_far_cells > 0) {
      cudaMemcpy(fc.data(), pl->d_far_cnt.p, pl->n_far_cells * 4, cudaMemcpyDeviceToHost);
      for (int64_t i = 0; i < pl->n_far_cells; ++i) tot += fc[i];
    }
    pl->n_m2l = tot;
    const int64_t nl = pl->n_leaves_ad, nc = pl->n_cells;
    std::vector<int> off(nl + 1), us(std::max<int64_t>(1, pl->n_u)), ids(std::max<int64_t>(1, nl));
    std::vector<int> ss(nc), se(nc), ts(nc), te(nc);
    cudaMemcpy(off.data(), pl->d_u_off.p, (nl + 1) * 4, cudaMemcpyDeviceToHost);
    if (pl->n_u) cudaMemcpy(us.data(), pl->d_u_src.p, pl->n_u * 4, cudaMemcpyDeviceToHost);
    if (nl) cudaMemcpy(ids.data(), pl->d_leaf_ids.p, nl * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(ss.data(), pl->d_src_start.p, nc * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(se.data(), pl->d_src_end.p, nc * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(ts.data(), pl->same_sets ? pl->d_src_start.p : pl->d_tgt_start.p, nc * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(te.data(), pl->same_sets ? pl->d_src_end.p : pl->d_tgt_end.p, nc * 4, cudaMemcpyDeviceToHost);
    int64_t pairs = 0, ml_s = 0, ml_t = 0, occ = 0;
    for (int64_t i = 0; i < nl; ++i) {
      const int a = ids[i];
      for (int e = off[i]; e < off[i + 1]; ++e) pairs += (int64_t)(te[a] - ts[a]) * (se[us[e]] - ss[us[e]]);
      ml_s = std::max<int64_t>(ml_s, se[a] - ss[a]);
      ml_t = std::max<int64_t>(ml_t, te[a] - ts[a]);
      occ += (se[a] > ss[a] || te[a] > ts[a]) ? 1 : 0;
    }
    pl->n_p2p_pairs = pairs;
    pl->n_leaves_q = occ;
    pl->max_leaf_src = ml_s;
    pl->max_leaf_tgt = ml_t;
  }
  if (pl->n_m2l < 0) {
    cudaStreamSynchronize(pl->last_stream);
    std::vector<int> fc(std::max<int64_t>(1, pl->n_far_cells));
    int64_t tot = 0;
    if (pl->n_far_cells > 0) {
      cudaMemcpy(fc.data(), pl->d_far_cnt.p, pl->n_far_cells * 4, cudaMemcpyDeviceToHost);
      for (int64_t i = 0; i < pl->n_far_cells; ++i) tot += fc[i];
    }
    pl->n_m2l = tot;
    const int64_t nl = pl->lev_count[pl->L];
    std::vector<int> nc(std::max<int64_t>(1, nl)), ns(std::max<int64_t>(1, nl * NEAR_MAX));
    std::vector<int> ss(pl->n_cells), se(pl->n_cells), ts(pl->n_cells), te(pl->n_cells);
    int64_t pairs = 0;
    if (nl > 0) {
      cudaMemcpy(nc.data(), pl->d_near_cnt.p, nl * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(ns.data(), pl->d_near_src.p, nl * NEAR_MAX * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(ss.data(), pl->d_src_start.p, pl->n_cells * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(se.data(), pl->d_src_end.p, pl->n_cells * 4, cudaMemcpyDeviceToHost);
      const void *tsp = pl->same_sets ? pl->d_src_start.p : pl->d_tgt_start.p;
      const void *tep = pl->same_sets ? pl->d_src_end.p : pl->d_tgt_end.p;
      cudaMemcpy(ts.data(), tsp, pl->n_cells * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(te.data(), tep, pl->n_cells * 4, cudaMemcpyDeviceToHost);
      int64_t ml_s = 0, ml_t = 0;
      for (int64_t i = 0; i < nl; ++i) {
        int64_t gt = pl->lev_first[pl->L] + i;
        int64_t nt = te[gt] - ts[gt];
        ml_s = std::max<int64_t>(ml_s, se[gt] - ss[gt]);
        ml_t = std::max<int64_t>(ml_t, nt);
        for (int e = 0; e < nc[i]; ++e) {
          int sl = ns[i * NEAR_MAX + e];
          pairs += nt * (int64_t)(se[sl] - ss[sl]);
        }
      }
      pl->max_leaf_src = ml_s;
      pl->max_leaf_tgt = ml_t;
    }
    pl->n_leaves_q = nl;
    pl->n_p2p_pairs = pairs;
  }
  {
    int derr = 0;
    if (pl->d_dev_err.p) {
      cudaStreamSynchronize(pl->last_stream);
      cudaMemcpy(&derr, pl->d_dev_err.p, 4, cudaMemcpyDeviceToHost);
    }
    info->device_error = derr;
  }
  info->n_m2l = pl->n_m2l;
  info->n_p2p_pairs = pl->n_p2p_pairs;
  info->n_leaves = pl->n_leaves_q;
  info->max_leaf_src = pl->max_leaf_src;
  info->max_leaf_tgt = pl->max_leaf_tgt;
  return FMM2D_OK;
}

fmm2d_status fmm2d_debug_export(fmm2d_plan *pl, int what, int level, void *host_buf, size_t cap,
                                size_t *written) {
  if (!pl) return FMM2D_EINVAL;
  if (!pl->built) return fail(pl, FMM2D_ENOTREADY, "plan is not built");
  const int L = pl->L;
  if ((what >= 5 && what <= 9) || what == 12) {
    if (level < 0 || level > L) return fail(pl, FMM2D_EINVAL, "level out of range");
  }
  CK(cudaStreamSynchronize(pl->last_stream), "export sync");
  std::vector<uint8_t> out;
  auto put64 = [&](int64_t v) { out.insert(out.end(), (uint8_t *)&v, (uint8_t *)&v + 8); };
  auto putd = [&](double v) { out.insert(out.end(), (uint8_t *)&v, (uint8_t *)&v + 8); };
  const bool same = pl->same_sets;
  const int64_t lf = (what >= 5) ? pl->lev_first[level < 0 ? 0 : level] : 0;
  const int64_t lc = (what >= 5) ? pl->lev_count[level < 0 ? 0 : level] : 0;
  std::vector<uint32_t> ckey(std::max<int64_t>(1, pl->n_cells));
  if (pl->n_cells > 0)
    CK(cudaMemcpy(ckey.data(), pl->d_cell_key.p, pl->n_cells * 4, cudaMemcpyDeviceToHost), "copy");
  switch (what) {
    case 1: case 2: case 3: case 4: {
      bool tg = what >= 3;
      int64_t n = tg ? pl->n_tgt : pl->n_src;
      const void *kp = (tg && !same) ? pl->d_key_t.p : pl->d_key_s.p;
      const void *pp = (tg && !same) ? pl->d_perm_t.p : pl->d_perm_s.p;
      std::vector<uint32_t> k(std::max<int64_t>(1, n)), pm(std::max<int64_t>(1, n));
      if (n > 0) {
        CK(cudaMemcpy(k.data(), kp, n * 4, cudaMemcpyDeviceToHost), "copy");
        CK(cudaMemcpy(pm.data(), pp, n * 4, cudaMemcpyDeviceToHost), "copy");
      }
      if (what == 1 || what == 3) {
        std::vector<int64_t> ko(n);
        for (int64_t i = 0; i < n; ++i) ko[pm[i]] = k[i];
        for (int64_t i = 0; i < n; ++i) put64(ko[i]);
      } else {
        for (int64_t i = 0; i < n; ++i) put64(pm[i]);
      }
      break;
    }
    case 5:
      for (int64_t i = 0; i < lc; ++i) put64(ckey[lf + i]);
      break;
    case 6: case 7: {
      if (what == 6) level = L;
      const int64_t f = pl->lev_first[level], c = pl->lev_count[level];
      const int64_t lfirst = pl->n_cells - pl->n_far_cells;
      if (what == 7 && (level < pl->l_min || pl->n_far_cells == 0)) break;
      const int stride = what == 6 ? NEAR_MAX : FAR_MAX;
      const int64_t base = what == 6 ? f - pl->lev_first[L] : f - lfirst;
      std::vector<int> cnt(std::max<int64_t>(1, c)), src(std::max<int64_t>(1, c * stride));
      if (c > 0) {
        const char *cp = (const char *)(what == 6 ? pl->d_near_cnt.p : pl->d_far_cnt.p);
        const char *sp = (const char *)(what == 6 ? pl->d_near_src.p : pl->d_far_src.p);
        CK(cudaMemcpy(cnt.data(), cp + base * 4, c * 4, cudaMemcpyDeviceToHost), "copy");
        CK(cudaMemcpy(src.data(), sp + base * stride * 4, c * stride * 4, cudaMemcpyDeviceToHost), "copy");
      }
      for (int64_t i = 0; i < c; ++i)
        for (int e = 0; e < cnt[i]; ++e) {
          put64(ckey[f + i]);
          put64(ckey[src[i * stride + e]]);
        }
      break;
    }
    case 8: case 9: case 12: {
      const bool f64 = is_fp64(pl);
      const int p = pl->p, P = pl->P;
      std::vector<double> q(std::max<int64_t>(1, lc));
      std::vector<double2> c2(std::max<int64_t>(1, lc * P));
      if (what == 12) {
        std::vector<double2> ct(std::max<int64_t>(1, lc));
        if (lc) CK(cudaMemcpy(ct.data(), (double2 *)pl->d_cell_ctr.p + lf, lc * 16, cudaMemcpyDeviceToHost), "copy");
        for (int64_t i = 0; i < lc; ++i) { putd(ct[i].x); putd(ct[i].y); }
        break;
      }
      const void *qs = what == 8 ? pl->d_mQ.p : pl->d_lL0.p;
      const char *cs = (const char *)(what == 8 ? pl->d_ma.p : pl->d_lb.p);
      if (lc) {
        CK(cudaMemcpy(q.data(), (const double *)qs + lf, lc * 8, cudaMemcpyDeviceToHost), "copy");
        if (f64) {
          CK(cudaMemcpy(c2.data(), cs + lf * P * 16, lc * P * 16, cudaMemcpyDeviceToHost), "copy");
        } else {
          std::vector<float2> c1(lc * P);
          CK(cudaMemcpy(c1.data(), cs + lf * P * 8, lc * P * 8, cudaMemcpyDeviceToHost), "copy");
          for (int64_t i = 0; i < lc * P; ++i) c2[i] = make_double2(c1[i].x, c1[i].y);
        }
      }
      const cd sl(pl->scale_re[level], pl->scale_im[level]);
      for (int64_t i = 0; i < lc; ++i) {
        putd(q[i]);
        putd(0.0);
        cd pw = 1.0;
        for (int k = 1; k <= p; ++k) {
          pw *= sl;
          cd v(c2[i * P + k - 1].x, c2[i * P + k - 1].y);
          cd u = what == 8 ? v * pw : v / pw;
          putd(u.real());
          putd(u.imag());
        }
      }
      break;
    }
    case 10: case 11: {
      const int64_t n = pl->n_tgt;
      std::vector<double> v(std::max<int64_t>(1, n));
      std::vector<uint32_t> pm(std::max<int64_t>(1, n));
      if (n) {
        CK(cudaMemcpy(v.data(), what == 10 ? pl->d_phi_near.p : pl->d_phi_far.p, n * 8,
                      cudaMemcpyDeviceToHost), "copy");
        CK(cudaMemcpy(pm.data(), same ? pl->d_perm_s.p : pl->d_perm_t.p, n * 4,
                      cudaMemcpyDeviceToHost), "copy");
      }
      std::vector<double> o(n);
      for (int64_t i = 0; i < n; ++i) o[pm[i]] = v[i];
      for (int64_t i = 0; i < n; ++i) putd(o[i]);
      break;
    }
    case 13: case 14: case 15: case 16: case 17: {
      if (!(pl->flags & FMM2D_ADAPTIVE)) return fail(pl, FMM2D_EINVAL, "not an adaptive plan");
      const int64_t nc = pl->n_cells;
      std::vector<uint8_t> lev(nc), spl(nc);
      CK(cudaMemcpy(lev.data(), pl->d_cell_lev.p, nc, cudaMemcpyDeviceToHost), "copy");
      CK(cudaMemcpy(spl.data(), pl->d_split.p, nc, cudaMemcpyDeviceToHost), "copy");
      if (what == 13) {
        for (int64_t i = 0; i < nc; ++i) { put64(lev[i]); put64(ckey[i]); put64(spl[i]); }
        break;
      }
      if (what == 17) {
        const int64_t ff = nc - pl->n_far_cells;
        std::vector<int> cnt(std::max<int64_t>(1, pl->n_far_cells)), src(std::max<int64_t>(1, pl->n_far_cells * FAR_MAX));
        if (pl->n_far_cells) {
          CK(cudaMemcpy(cnt.data(), pl->d_far_cnt.p, pl->n_far_cells * 4, cudaMemcpyDeviceToHost), "copy");
          CK(cudaMemcpy(src.data(), pl->d_far_src.p, pl->n_far_cells * FAR_MAX * 4, cudaMemcpyDeviceToHost), "copy");
        }
        for (int64_t i = 0; i < pl->n_far_cells; ++i)
          for (int e = 0; e < cnt[i]; ++e) {
            const int sc = src[i * FAR_MAX + e];
            put64(lev[ff + i]); put64(ckey[ff + i]); put64(lev[sc]); put64(ckey[sc]);
          }
        break;
      }
      const bool by_leaf = what != 16;
      const int64_t ng = by_leaf ? pl->n_leaves_ad : nc;
      const int64_t n = what == 14 ? pl->n_u : what == 15 ? pl->n_w : pl->n_x;
      const DBuf &ob = what == 14 ? pl->d_u_off : what == 15 ? pl->d_w_off : pl->d_x_off;
      const DBuf &sb = what == 14 ? pl->d_u_src : what == 15 ? pl->d_w_src : pl->d_x_src;
      std::vector<int> off(ng + 1), src(std::max<int64_t>(1, n)), ids(std::max<int64_t>(1, ng));
      CK(cudaMemcpy(off.data(), ob.p, (ng + 1) * 4, cudaMemcpyDeviceToHost), "copy");
      if (n) CK(cudaMemcpy(src.data(), sb.p, n * 4, cudaMemcpyDeviceToHost), "copy");
      if (by_leaf && ng) CK(cudaMemcpy(ids.data(), pl->d_leaf_ids.p, ng * 4, cudaMemcpyDeviceToHost), "copy");
      for (int64_t i = 0; i < ng; ++i) {
        const int a = by_leaf ? ids[i] : (int)i;
        for (int e = off[i]; e < off[i + 1]; ++e) {
          put64(lev[a]); put64(ckey[a]); put64(lev[src[e]]); put64(ckey[src[e]]);
        }
      }
      break;
    }
    default:
      return fail(pl, FMM2D_EINVAL, "unknown export item");
  }
  if (written) *written = out.size();
  if (!host_buf) return FMM2D_OK;
  if (cap < out.size()) return fail(pl, FMM2D_EINVAL, "export buffer too small");
  std::memcpy(host_buf, out.data(), out.size());
  return FMM2D_OK;
}

fmm2d_status fmm2d_plan_set_debug_stall(fmm2d_plan *pl, int on) {
  if (!pl) return FMM2D_EINVAL;
  pl->debug_stall = on ? 1 : 0;
  return FMM2D_OK;
}

fmm2d_status fmm2d_plan_set_profiling(fmm2d_plan *pl, int on) {
  if (!pl) return FMM2D_EINVAL;
  flush_events(pl);
  pl->profiling = on == 2 ? 2 : (on != 0 ? 1 : 0);
  for (int i = 0; i < ST_COUNT; ++i) {
    pl->stage_ms[i] = 0;
    pl->stage_launches[i] = 0;
  }
  return FMM2D_OK;
}

fmm2d_status fmm2d_stage_times(fmm2d_plan *pl, double *ms, int64_t *launches, int cap, int *n_stages) {
  if (!pl) return FMM2D_EINVAL;
  flush_events(pl);
  if (n_stages) *n_stages = ST_COUNT;
  for (int i = 0; i < ST_COUNT && i < cap; ++i) {
    if (ms) ms[i] = pl->stage_ms[i];
    if (launches) launches[i] = pl->stage_launches[i];
  }
  return FMM2D_OK;
}

void fmm2d_plan_destroy(fmm2d_plan *pl) {
  if (!pl) return;
  flush_events(pl);
  for (auto ev : pl->ev_pool) cudaEventDestroy(ev);
  for_each_dbuf(pl, [](DBuf &b) { dbuf_free(b); });
  if (pl->far_stream) {
    cudaStreamSynchronize(pl->far_stream);
    cudaStreamDestroy(pl->far_stream);
  }
  if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
  if (pl->ev_join) cudaEventDestroy(pl->ev_join);
  if (pl->graph_exec) cudaGraphExecDestroy(pl->graph_exec);
  delete pl;
}

const char *fmm2d_last_error(const fmm2d_plan *pl) {
  if (!pl) return g_create_err.c_str();
  return pl->err.c_str();
}

}  // extern "C"
