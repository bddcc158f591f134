// plan.h - internal plan object of the fmm2d library and the launchers of
// every kernel (defined in keys.cu, sort.cu, tree.cu, expand.cu, p2p.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <complex>
#include <vector>

#include "common.cuh"
#include "fmm2d.h"

namespace fmm2d {

constexpr int MAXLEV = 23;
constexpr int MAXP = 48;
constexpr int MAX_CLASSES = 8;   // tri: 4 child types x 2 parent orientations
constexpr int FAR_MAX = 48;      // longest M2L stencil (septree: 42)
constexpr int NEAR_MAX = 16;     // longest Near stencil (triangle: 13)

enum Stage { ST_KEYS, ST_SORT, ST_TREE, ST_LISTS, ST_P2M, ST_M2M, ST_M2L, ST_L2L, ST_L2P, ST_P2P,
             ST_OTHER, ST_FIELD, ST_COUNT };

// Grow-only device buffer owned by a plan.
struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

// Tiling geometry passed by value to kernels.
struct Geo {
  int tiling, L, b;
  double x0, y0, S;
  double leaf_scale;                 // sept r, tri rho0, quad 2^-L (frame units)
  double unit_re[MAXLEV + 1];        // septree: level-l lattice unit g_l (frame)
  double unit_im[MAXLEV + 1];
  int64_t map_off[MAXLEV + 2];       // offset of level l in the key -> slot map
};

// Stencils of one plan (host copy; device copy in Plan::d_sten).
struct Stencils {
  int n_classes;
  int far_len[MAX_CLASSES];
  int far_d[MAX_CLASSES][FAR_MAX][3];      // lattice offsets
  uint16_t far_op[MAX_CLASSES][FAR_MAX];   // M2L operator id of each entry
  int near_len[2];
  int near_d[2][NEAR_MAX][3];              // [orientation][entry] (quad/sept use [0])
};

struct Plan {
  // parameters
  int tiling = 0, levels_req = 0, p_req = 0;
  double eps = 1e-6;
  unsigned flags = 0;
  double x0 = 0, y0 = 0, S = 1;
  // derived at build
  int L = 0, p = 0, P = 0, l_min = 0, b = 4;
  Geo geo;
  Stencils sten;
  int n_ops = 0;
  bool built = false, same_sets = false;
  int64_t n_src = 0, n_tgt = 0;
  int64_t map_size = 0;
  int64_t lev_first[MAXLEV + 2] = {0}, lev_count[MAXLEV + 2] = {0};
  int64_t n_cells = 0, n_far_cells = 0, n_m2l = 0, n_p2p_pairs = 0;
  int64_t n_leaves_q = 0, max_leaf_src = 0, max_leaf_tgt = 0;   // filled by fmm2d_plan_query
  int max_far = 0, max_near = 0;
  double scale_re[MAXLEV + 1], scale_im[MAXLEV + 1], log_abs_scale[MAXLEV + 1];
  std::string err;
  cudaStream_t last_stream = nullptr;
  // profiling
  int profiling = 0;                  // 0 off, 1 stage events, 2 stage events, stages serialised
  double stage_ms[ST_COUNT] = {0};
  int64_t stage_launches[ST_COUNT] = {0};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  size_t ev_used = 0;

  // device buffers
  DBuf d_key_s, d_perm_s, d_key_t, d_perm_t, d_tmp_k, d_tmp_v, d_sort_scratch;
  DBuf d_err;
  DBuf d_occ, d_hsrc, d_scan, d_map;
  DBuf d_cell_key, d_cell_crd, d_cell_ctr, d_cell_cls, d_cell_hsrc;
  DBuf d_src_start, d_src_end, d_tgt_start, d_tgt_end, d_lev_first;
  DBuf d_far_cnt, d_far_src, d_far_op, d_near_cnt, d_near_src;
  DBuf d_src4, d_tgt2;
  DBuf d_src4f, d_tgt2f;               // FP32 copies (high parts) for the P2P of FMM2D_PREC_HYBRID
  DBuf d_srclo, d_tgtlo;               // their low parts (float2 per point)
  DBuf d_mQ, d_ma, d_lL0, d_lb;
  DBuf d_phi_near, d_phi_far;
  DBuf d_m2m_arrive;                // uniform upward pass: arrivals per cell
  DBuf d_pmap;                      // uniform triangle tree: position -> slot of the lists
  DBuf d_ad_hash;                   // adaptive tree: (level, instance, position) -> cell table
  DBuf d_l2l_ready;                 // uniform downward pass: counter + ready word per cell
  DBuf d_fnear;                        // near part of the field (fmm2d_evaluate_field)
  DBuf d_sten, d_geo_scale;
  DBuf d_m2l_ops, d_m2l_logz, d_m2m_ops, d_l2l_ops;   // element type per precision
  DBuf d_counts;
  DBuf d_far_full, d_cls_cnt, d_cls_cells, d_tc_ops, d_ff_ops, d_ff_ph, d_ma_ff, d_dev_err;
  DBuf d_tc_part_lb, d_tc_part_L0;     // tensor-core M2L: partial locals of split tiles
  int tc_split_n = 1;
  int debug_stall = 0;                // test switch: M2L CTAs time out before their MMAs
  DBuf d_p2p_order, d_p2p_cnt;        // adaptive tree: P2P leaf size classes
  int tc_K = 0, tc_N = 0, n_sms = 148;
  int64_t cls_cap = 1;
  // adaptive tree (FMM2D_ADAPTIVE): cells split while they hold more than
  // leaf_cap sources or targets; U / W / X lists in CSR form by target
  int leaf_cap = 64;
  int64_t n_leaves_ad = 0, n_u = 0, n_w = 0, n_x = 0;
  // adaptive FP32 P2P: leaves by size class (launch_p2p_bins), class counts
  bool p2p_binned = false;
  int64_t p2p_bin_count[4] = {0, 0, 0, 0};
  DBuf d_cell_lev, d_parent, d_child_first, d_child_cnt, d_split;
  DBuf d_leaf_ids, d_leaf_pos, d_ad_scale, d_ad_inv_scale;
  DBuf d_u_off, d_u_src, d_w_off, d_w_src, d_x_off, d_x_src;
  DBuf d_ad_flag, d_ad_pos, d_ad_crange, d_ad_cnt, d_ad_off, d_ad_tot;
  DBuf d_ad_ta, d_ad_tc, d_ad_sa, d_ad_sc, d_ad_ta2, d_ad_tc2, d_ad_sa2, d_ad_sc2;
  DBuf d_ad_ut, d_ad_us, d_ad_wt, d_ad_ws, d_ad_xt, d_ad_xs;
  int n_inst = 1;                     // instances of a forest build
  DBuf d_inst_off;
  // the far-field chain (P2M ... L2L) runs on a high-priority plan stream
  // while P2P runs on the caller's stream; two events fork and join them
  cudaStream_t far_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // fmm2d_evaluate_graph: the recorded evaluation, valid for one build
  // (build_gen counts the builds) and one pair of strength / potential pointers
  uint64_t build_gen = 0, graph_gen = 0;
  cudaGraphExec_t graph_exec = nullptr;
  const void *graph_u = nullptr;
  double *graph_out = nullptr;
  // parameters the cached geometry / operator tables were built for
  bool geo_valid = false;
  int geo_key_L = -1, geo_key_p = -1;
  double geo_key_x0 = 0, geo_key_y0 = 0, geo_key_S = 0;
  std::vector<double> m2l_logz_host;
};

// ---------------------------------------------------------------- helpers
// Host-side planner constants that take a moment to compute (septree leaf
// radii), computed ahead of the first plan that needs them.
void planner_precompute();
// Septree leaf circumradius r_L of an L-level tree (frame units): the
// smallest multiple of 2^-40 for which every point of the frame square has
// its nearest leaf-lattice point inside the L-digit GBT region (Sec. 5).
// Computed once per L by enumeration, then cached; host work only.
double sept_leaf_r(int L);
// Triangle quadtree root inradius rho0 (frame units, Sec. 6).
double tri_rho0();
// Leaf level of the S_opt rule (Table 2, App. A-C) for N sources, M targets
// and expansion order p.
int planner_sopt_levels(int tiling, int64_t n_src, int64_t n_tgt, int p);
}  // namespace fmm2d
// Device memory (bytes) a plan holds in its buffers.
struct fmm2d_plan;
namespace fmm2d {
size_t plan_device_bytes(const fmm2d_plan *pl);

cudaError_t dbuf_reserve(DBuf &b, size_t bytes);
void dbuf_free(DBuf &b);

// ---------------------------------------------------------------- keys.cu
// list / list_n (optional, n entries + one counter): scratch for the FP32
// filter; without them every point takes the exact FP64 front end.
cudaError_t launch_keys(const Geo &g, const void *xy, bool f32, int64_t n, uint32_t *key,
                        uint32_t *perm_iota, int *err, cudaStream_t s, uint32_t *list = nullptr,
                        int *list_n = nullptr);

// ---------------------------------------------------------------- sort.cu
size_t radix_sort_scratch_bytes(int64_t n);
// Stable LSD sort of (key, val) pairs on the low `bits` bits; result in
// keys/vals.  A look-back wait that gives up ORs 8 into *err (when err is
// given; the output is then invalid but every write stays in bounds).
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tmp_k, uint32_t *tmp_v,
                             int64_t n, int bits, void *scratch, cudaStream_t s,
                             int *err = nullptr);
// Kernel launches of one radix_sort_pairs / exclusive_scan call.
int radix_sort_launches(int64_t n, int bits);
int exclusive_scan_launches(int64_t n);
size_t scan_scratch_bytes(int64_t n);
// Exclusive prefix sum of int32 values; out may alias in.
cudaError_t exclusive_scan(const int *in, int *out, int64_t n, void *scratch, cudaStream_t s);

// ---------------------------------------------------------------- tree.cu
cudaError_t launch_mark(const Geo &g, const uint32_t *key_sorted, int64_t n, int *occ, int *hsrc,
                        cudaStream_t s);
// Cells of every level from the occupancy scan; also the first slot of every
// level and the total in lev_first[0 .. L+1].  pmap (triangle tiling, else
// null): the position map of the lists, 2 (4^(L+1) - 1) / 3 ints, every
// entry written.
cudaError_t launch_compact(const Geo &g, const int *occ, const int *scan, const int *hsrc,
                           int64_t map_size, int *map, uint32_t *cell_key, int4 *cell_crd,
                           double2 *cell_ctr, uint8_t *cell_cls, uint8_t *cell_hsrc,
                           int *src_start, int *src_end, int *tgt_start, int *tgt_end,
                           int64_t *lev_first, int *pmap, cudaStream_t s);
// Sorted points relative to their leaf centre, and the leaves' point ranges.
// lo (optional): the low parts (leaf-relative coordinate minus its FP32 value).
cudaError_t launch_rel_coords(const Geo &g, bool f32_in, bool f32_out, const void *xy,
                              const uint32_t *perm, const uint32_t *key_sorted, int64_t n,
                              const int *map, const double2 *ctr, void *out, int out_stride,
                              int *start, int *end, cudaStream_t s, float2 *lo = nullptr);
// Near lists of the leaves and M2L lists of levels >= l_min, for the cells
// of levels lo_level..L (count read on the device; cap = launch bound).
cudaError_t launch_lists(const Geo &g, const Stencils *d_sten, int lo_level, int l_min, int64_t cap,
                         const int *map, const uint8_t *cell_cls, const int4 *cell_crd,
                         const uint8_t *cell_hsrc, int *far_cnt, int *far_src, uint16_t *far_op,
                         int *near_cnt, int *near_src, const int64_t *lev_first_dev,
                         int *far_full, int *cls_cnt, int *cls_cells, int64_t cls_cap,
                         const int *pmap, cudaStream_t s);

// ---------------------------------------------------------------- adaptive.cu
// Cell arrays of the adaptive tree (one array over all levels, ordered by
// (level, key)); ts/te alias ss/se when sources and targets are one set.
struct AdCells {
  uint32_t *key;
  uint8_t *lev;
  int *parent, *child_first;
  uint8_t *child_cnt, *split;
  int *ss, *se, *ts, *te;
  int4 *crd;
  double2 *ctr;
  uint8_t *cls, *hsrc;
  // (level, instance, lattice position) -> cell, for the cells with
  // sources: open addressing with linear probing, built once the cells
  // exist (for the list traversal); slot = {packed position (0 = empty),
  // cell}, one 16-byte read per probe
  const ulonglong2 *hslot = nullptr;
  uint32_t hmask = 0;                  // capacity - 1 (a power of two)
};
// Fill the (level, instance, lattice position) -> cell table with the
// cells that hold sources, of the n_cells cells (slots zeroed here;
// capacity hmask + 1, at least twice n_cells).
cudaError_t ad_launch_hash(const Geo &g, int64_t n_cells, const AdCells &c, ulonglong2 *slots,
                           uint32_t hmask, cudaStream_t s);
// level-0 cells: one per instance (soff / toff: n_inst + 1 device offsets),
// or one cell holding everything (null offsets, n_inst = 1)
cudaError_t ad_launch_roots(const Geo &g, int n_inst, const int64_t *soff, const int64_t *toff,
                            int64_t n_s, int64_t n_t, const AdCells &c, cudaStream_t s);
// add the instance prefix inst * span to sorted-order-independent keys
cudaError_t ad_launch_prefix(int64_t n, uint32_t *key, const int64_t *off, int n_inst, uint64_t span,
                             cudaStream_t s);
cudaError_t ad_launch_split(const Geo &g, int l, int64_t first, int64_t count, int cap,
                            const uint32_t *skey, const uint32_t *tkey, const AdCells &c, int *flag,
                            int4 *crange, cudaStream_t s);
cudaError_t ad_launch_level_total(int64_t count_b, const int *flag, const int *pos, int *total_out,
                                  cudaStream_t s);
cudaError_t ad_launch_emit(const Geo &g, int l, int64_t first, int64_t count, int64_t next_first,
                           const int *flag, const int *pos, const int4 *crange, const AdCells &c,
                           cudaStream_t s);
cudaError_t ad_launch_leaves(int64_t n_cells, const uint8_t *split, int *flag, int *pos,
                             void *scan_scratch, int *leaf_ids, int *leaf_pos, int *n_leaves_out,
                             cudaStream_t s);
cudaError_t ad_launch_rel(bool f32_in, bool f32_out, const void *xy, const uint32_t *perm,
                          int64_t n_leaves, const int *leaf_ids, const int *start, const int *end,
                          const double2 *ctr, void *out, int stride, cudaStream_t s,
                          float2 *lo = nullptr);
// count pass of one level's traversal; totals[5] = U, W, X, next W tests, next X tests
cudaError_t ad_launch_lists(const Geo &g, const Stencils *d_sten, int l, int l_min, int64_t first,
                            int64_t count, int64_t n_t, int64_t n_s, const int *t_a, const int *t_c,
                            const int *s_a, const int *s_c, const AdCells &c, int *cnt,
                            int *off, void *scan_scratch, int *totals, cudaStream_t s);
cudaError_t ad_launch_lists_emit(const Geo &g, const Stencils *d_sten, int l, int l_min,
                                 int64_t first, int64_t count, int64_t n_t, int64_t n_s,
                                 const int *t_a, const int *t_c, const int *s_a, const int *s_c,
                                 const AdCells &c, const int *off, const int64_t base[5],
                                 int *u_t, int *u_s, int *w_t, int *w_s, int *x_t, int *x_s,
                                 int *nt_a, int *nt_c, int *ns_a, int *ns_c, int64_t far_first,
                                 int *far_cnt, int *far_src, uint16_t *far_op, int *far_full,
                                 int *cls_cnt, int *cls_cells, int64_t cls_cap, cudaStream_t s);
// Stable grouping of n (target, source) pairs by target (map[target] when map
// is given): CSR offsets off[0..n_groups] and the sources in group order.
cudaError_t ad_group(int64_t n, const int *tgt, const int *src, const int *map, int n_groups,
                     uint32_t *key, uint32_t *idx, uint32_t *tmp_k, uint32_t *tmp_v, void *scratch,
                     int *cnt, int *off, int *out_src, cudaStream_t s, int *err = nullptr);
template <typename R>
cudaError_t ad_launch_m2p(int64_t n_leaves, const int *leaf_ids, const int *w_off, const int *w_src,
                          const R *tgt, int tstride, const int *ts, const int *te,
                          const double2 *ctr, const uint8_t *lev, const double2 *scale, int p,
                          int P, const double *mQ, const Cx<R> *ma, double *phi, cudaStream_t s);
template <typename R>
cudaError_t ad_launch_p2l(int64_t n_cells, const int *x_off, const int *x_src, const R *src4,
                          const int *ss, const int *se, const double2 *ctr, const uint8_t *lev,
                          const double2 *inv_scale, int p, int P, double *lL0, Cx<R> *lb,
                          cudaStream_t s);

// ---------------------------------------------------------------- expand.cu
struct ExpandArgs {
  int p, P, L, l_min, b;
  int n_cls = 0;                      // M2M / L2L operators in the table (child classes)
  int64_t leaf_first, n_leaves;
  double inv_s_re, inv_s_im;          // 1 / s_L
  // adaptive tree (null for the uniform one): leaf li is cell leaf_ids[li],
  // of level cell_lev[...], whose inverse scale is inv_scale[level]
  const int *leaf_ids = nullptr;
  const uint8_t *cell_lev = nullptr;
  const double2 *inv_scale = nullptr;
  // adaptive tree: children of a split cell are contiguous, parents explicit
  const int *child_first = nullptr;
  const uint8_t *child_cnt = nullptr;
  const int *parent = nullptr;
  // uniform tree: the L2L of the leaf level done by the L2P (the leaf's M2L
  // local plus its parent's shifted final local, written back to lL0 / lb)
  const int *l2l_map = nullptr;          // key -> slot map, level L-1 part at l2l_map_off
  int64_t l2l_map_off = 0;
  const uint32_t *l2l_key = nullptr;     // cell keys
  const uint8_t *l2l_cls = nullptr;      // child classes
  const void *l2l_ops = nullptr;         // L2L operator table (Cx<R>)
  int l2l_sept = 0;                      // parent key = key / 7 (septree), else key >> 2
};
template <typename R>
cudaError_t launch_gather_u(const void *u, bool f32_in, const uint32_t *perm, int64_t n, R *src4,
                            cudaStream_t s, bool lo = false);
template <typename R>
cudaError_t launch_p2m(const ExpandArgs &a, const R *src4, const int *start, const int *end,
                       double *mQ, Cx<R> *ma, cudaStream_t s);
// Uniform tree: the downward pass of levels l_min+1 .. L (cells first ..
// first + total) in one persistent launch; ready: n_cells + 2 ints, zeroed
// here; a bounded wait that gives up ORs 2 into *err.
template <typename R>
cudaError_t launch_l2l_down(const ExpandArgs &a, const Geo &g, int64_t first, int64_t total,
                            const int64_t *lev_first_dev, const int *map, const uint32_t *cell_key,
                            const uint8_t *cell_cls, const Cx<R> *ops, double *lL0, Cx<R> *lb,
                            int *ready, int64_t n_cells, int sms, int *err, cudaStream_t s);
// Uniform tree: the upward pass of levels L-1 .. l_min in one launch (cells
// of level L-1 first at first .. first + count; arrive: n_cells ints, zeroed
// here).
template <typename R>
cudaError_t launch_m2m_up(const ExpandArgs &a, const Geo &g, int l_min, int64_t first, int64_t count,
                          const int *map, const uint32_t *cell_key, const uint8_t *cell_cls,
                          const uint8_t *cell_hsrc, const Cx<R> *ops, double *mQ, Cx<R> *ma,
                          int *arrive, int64_t n_cells, cudaStream_t s);
template <typename R>
cudaError_t launch_m2m(const ExpandArgs &a, const Geo &g, int level, int64_t first, int64_t count,
                       const int *map, const uint32_t *cell_key, const uint8_t *cell_cls,
                       const uint8_t *cell_hsrc, const Cx<R> *ops, double *mQ, Cx<R> *ma, int sms,
                       cudaStream_t s);
template <typename R>
cudaError_t launch_m2l(const ExpandArgs &a, int64_t first, int64_t count, const int64_t *lev_of_cell_first,
                       const double *log_abs_scale_dev, int64_t far_base, const int *far_cnt,
                       const int *far_src, const uint16_t *far_op, const Cx<R> *ops,
                       const double *logz, const double *mQ, const Cx<R> *ma, double *lL0,
                       Cx<R> *lb, cudaStream_t s);
template <typename R>
cudaError_t launch_l2l(const ExpandArgs &a, const Geo &g, int level, int64_t first, int64_t count,
                       const int *map, const uint32_t *cell_key, const uint8_t *cell_cls,
                       const Cx<R> *ops, double *lL0, Cx<R> *lb, int sms, cudaStream_t s);
template <typename R>
cudaError_t launch_l2p(const ExpandArgs &a, const R *tgt, int tstride, const int *start,
                       const int *end, const uint32_t *perm, double *lL0, Cx<R> *lb,
                       const double *phi_near, double *phi_far, double *out, cudaStream_t s);

// ---------------------------------------------------------------- m2l_tc.cu
// Tensor-core M2L (tcgen05, TF32 hi/lo split, FP32 accumulation in TMEM).
struct TcArgs {
  int p, P, n_classes, sms;
  int64_t far_first, cls_cap;
  const int *cls_cnt, *cls_cells, *far_full;
  const uint16_t *sten_ops;           // [MAX_CLASSES][FAR_MAX] operator id per stencil entry
  const int *sten_len;                // [MAX_CLASSES]
  const unsigned char *btab;          // per operator: B hi then B lo, core-matrix layout
  const double *logz, *log_abs_scale;
  const int64_t *lev_first;
  int l_min, L;
  const double *mQ;
  const float2 *ma;
  double *lL0;
  float2 *lb;
  int *err;
  // stencil entries of a tile split over `split` CTAs (split > 1): partial
  // locals [split][far cell][P] and partial L_0 [split][far cell], summed in
  // split order by a second kernel
  int split = 1;
  float2 *part_lb = nullptr;
  double *part_L0 = nullptr;
  int64_t n_far = 0;
  int debug_stall = 0;                // test switch (fmm2d_plan_set_debug_stall)
};
bool tc_shape(int p, int *K, int *N);
// CTAs over which the stencil entries of one tile are split, for a level
// range with n_far_cells M2L targets (chosen for load balance over the SMs).
int tc_split(int64_t n_far_cells, int n_classes, int sms, int K, int N);
// Measured TF32 tensor-core throughput (TFLOP/s) of this device.
cudaError_t tc_measure_tf32(double *tflops);
// B tables (hi/lo TF32 splits of the real-ified operators) for all operators.
void tc_build_tables(const std::vector<double> &m2l_re, const std::vector<double> &m2l_im,
                     int n_ops, int p, int K, int N, std::vector<uint32_t> &out);
cudaError_t launch_m2l_tc(const TcArgs &a, int K, int N, int64_t n_far_cells, cudaStream_t s);

// ---------------------------------------------------------------- m2l_ff.cu
// M2L of the hybrid form: float-float arithmetic on the FP32 pipes, one CTA
// per 64 targets of a class (the class lists of the tensor-core form).
struct FfArgs {
  int p, P, n_classes, sms;
  int64_t far_first, cls_cap;
  const int *cls_cnt, *cls_cells, *far_full;
  const uint16_t *sten_ops;           // [MAX_CLASSES][FAR_MAX] operator id per stencil entry
  const int *sten_len;                // [MAX_CLASSES]
  const float2 *opA;                  // per operator the real factor A [k][l]: hi, lo
  const float4 *oph;                  // per operator the phases u^-m, m = 0..p
  const double *logz, *log_abs_scale;
  const int64_t *lev_first;
  int l_min, L;
  const double *mQ;
  const double2 *ma;
  double *lL0;
  double2 *lb;
  float4 *ma_ff;                      // scratch: every cell's Q, a^_1..a^_p as float-float
  int64_t n_cells;
};
size_t m2l_ff_smem_bytes(int p);
// From the offsets zeta and the FP64 operators ([op][l][k]): the real
// factors A (float-float, [op][k][l]) and the phases u^-m of the kernel.
void ff_build_table(const std::vector<std::complex<double>> &zeta,
                    const std::vector<std::complex<double>> &ops, int p, std::vector<float> &A,
                    std::vector<float> &ph);
cudaError_t launch_m2l_ff(const FfArgs &a, int64_t n_far_cells, cudaStream_t s);

// ---------------------------------------------------------------- p2p.cu
// src_lo / tgt_lo (FP32 form, hybrid precision): low parts of the points'
// leaf-relative coordinates (hi + lo floats); with them every term is also
// accumulated with compensation.
// leaf_ids: null (leaves leaf_first + li) or the cell of leaf li; near lists
// fixed-stride (near_off null: near_cnt[li], near_src[li * NEAR_MAX + e]) or
// CSR (near_src[near_off[li] .. near_off[li + 1])).
template <typename R>
cudaError_t launch_p2p(int64_t leaf_first, int64_t n_leaves, const int *leaf_ids, const R *src4,
                       const R *tgt, int tstride, const int *src_start, const int *src_end,
                       const int *tgt_start, const int *tgt_end, const int *near_cnt,
                       const int *near_off, const int *near_src, const double2 *ctr,
                       double *phi_near, double mean_targets, cudaStream_t s,
                       const float2 *src_lo = nullptr, const float2 *tgt_lo = nullptr,
                       const int *bin_order = nullptr, const int64_t *bin_count = nullptr);
// Adaptive trees: the leaves (positions li of leaf_ids) by size class, for
// launch_p2p's per-class group sizes; cnt8[0..3] the class counts.
cudaError_t launch_p2p_bins(int64_t n_leaves, const int *leaf_ids, const int *ts, const int *te,
                            int *cnt8, int *order, cudaStream_t s);

// ---------------------------------------------------------------- field.cu
// The field F = sum u / (y - x) by the differentiated P2P, M2P and L2P
// (fmm2d_evaluate_field); fnear: per target (sorted order) double2.
template <typename R>
cudaError_t launch_p2p_field(int64_t leaf_first, int64_t n_leaves, const int *leaf_ids,
                             const R *src4, const R *tgt, int tstride, const int *src_start,
                             const int *src_end, const int *tgt_start, const int *tgt_end,
                             const int *near_cnt, const int *near_off, const int *near_src,
                             const double2 *ctr, double2 *fnear, cudaStream_t s,
                             const float2 *src_lo = nullptr, const float2 *tgt_lo = nullptr);
template <typename R>
cudaError_t launch_m2p_field(int64_t n_leaves, const int *leaf_ids, const int *w_off,
                             const int *w_src, const R *tgt, int tstride, const int *ts,
                             const int *te, const double2 *ctr, const uint8_t *lev,
                             const double2 *scale, int p, int P, const double *mQ, const Cx<R> *ma,
                             double2 *fnear, cudaStream_t s);
template <typename R>
cudaError_t launch_l2p_field(const ExpandArgs &a, const R *tgt, int tstride, const int *start,
                             const int *end, const uint32_t *perm, const Cx<R> *lb,
                             const double2 *fnear, double2 *out, cudaStream_t s);

}  // namespace fmm2d
