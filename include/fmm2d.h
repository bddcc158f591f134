/*
 * fmm2d.h - C ABI of the GB300 (sm_103a) 2D fast multipole method over three
 * tilings of the plane: quadtree, septree of hexagons and triangle quadtree
 * (Luo & Duraiswami, "Alternative tilings for the fast multipole method on
 * the plane", arXiv:1204.3105).
 *
 * What is computed (Sec. 2, eqs. 1-2): for sources x_i with real strengths
 * u_i and targets y_j in the plane (points as complex numbers),
 *
 *     Phi_j = sum_{i : x_i != y_j} u_i log|y_j - x_i|
 *
 * i.e. the real part of sum_i u_i log(y_j - x_i) (the complex logarithm of
 * eq. 1 is multivalued; its real part, the 2D Coulomb potential, is not).
 * A source that coincides with the target is skipped.
 *
 * The evaluation is the hierarchical FMM of Sec. 2: every point is keyed with
 * the tiling's CellIndex (Sec. 4-6) and sorted; occupied cells of every level
 * get Near lists (the cell and its Neighbors, Sec. 4) and M2L lists
 * (NeighborsE4, eq. 3, read as Children[Parent(n) u Neighbors(Parent(n))]
 * minus Near(n)); then P2M, M2M, M2L, L2L, L2P and the P2P near-field sum.
 * Every step runs in the library's own CUDA kernels; there is no CPU
 * fallback.
 *
 * Conventions for every call below
 *   - Pointers named *_dev are device pointers (cudaMalloc / PyTorch CUDA
 *     memory) on the current device; pointers named *_host are host memory.
 *     The caller owns every buffer it passes; the library never frees them.
 *   - Points are interleaved (x, y) pairs: 2*n values of float64, or of
 *     float32 when the plan was created with FMM2D_IN_F32.  Strengths are n
 *     values of the same type.  Potentials are always float64.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *     work is ordered on it; a call returns once its work is enqueued, except
 *     fmm2d_build, which waits for its own work (it reads back the cell
 *     counts that size the evaluation).
 *   - Errors are status codes; no C++ exception crosses the ABI.  The text of
 *     the last error of a plan is available from fmm2d_last_error.
 *   - A plan is not thread safe; distinct plans may be used concurrently.
 */
#ifndef FMM2D_H
#define FMM2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { FMM2D_QUAD = 0, FMM2D_SEPT = 1, FMM2D_TRI = 2 } fmm2d_tiling;

typedef enum {
  FMM2D_OK = 0,
  FMM2D_EINVAL = 1,    /* bad argument (tiling, levels, p, sizes, null pointer) */
  FMM2D_ENOMEM = 2,    /* a device or host allocation failed */
  FMM2D_EDOMAIN = 3,   /* a point lies outside the plan's domain square */
  FMM2D_ECUDA = 4,     /* a CUDA runtime call failed (message in fmm2d_last_error) */
  FMM2D_EBUSY = 5,     /* server: no admission possible right now */
  FMM2D_ETIMEOUT = 6,  /* a bounded wait gave up */
  FMM2D_ENOTREADY = 7  /* server: ticket not finished yet / plan not built */
} fmm2d_status;

/* Plan flags (bitwise or). */
#define FMM2D_PREC_FP64     0x0u  /* every expansion, translation and P2P in FP64 */
#define FMM2D_PREC_MIXED    0x1u  /* FP32 expansions, translations and P2P; the
                                     leading Q log term, L_0 and the final sums in FP64 */
#define FMM2D_PREC_MIXED_TC 0x2u  /* as MIXED, with M2L on the tensor cores
                                     (split hi/lo TF32 products, FP32 accumulation) */
#define FMM2D_PREC_HYBRID   0x3u  /* FP64 expansions, P2M, M2M, L2L and L2P, the M2L
                                     of FMM2D_PREC_SPLIT, and a P2P in FP32 pairs
                                     (float-float r^2 and log2, exact products,
                                     error-free sums): for tolerances between about
                                     1e-9 and 1e-6 */
#define FMM2D_PREC_SPLIT    0x4u  /* as FP64, with the M2L sums in float-float
                                     (hi + lo FP32 pairs, exact products,
                                     error-free sums) on the FP32 pipes: the
                                     FP64 leading terms and a split-precision
                                     M2L, for tolerances down to about 1e-12 */
#define FMM2D_PREC_MASK     0x7u
#define FMM2D_IN_F32        0x10u /* points and strengths are float32 (default float64) */
#define FMM2D_ADAPTIVE      0x20u /* adaptive tree for clustered input: a cell is split
                                     while it holds more than the leaf size (default 64,
                                     fmm2d_plan_set_leaf_size) sources or targets, down
                                     to `levels` (0 = 16 for the quadtree and triangle
                                     quadtree, 11 for the septree); cells of different
                                     levels interact by M2P and P2L (W and X lists).
                                     The paper refines uniformly (Sec. 2); this is the
                                     adaptive extension for non-uniform data (Sec. 9). */

#define FMM2D_FIELD         0x80u /* the plan will also be evaluated with
                                     fmm2d_evaluate_field: the FP32 forms then
                                     keep the low parts of the points'
                                     leaf-relative coordinates (needed for the
                                     field's accurate pair differences) */
/* Server requests only: take the FMM2D_PREC_* bits as given, including
 * FMM2D_PREC_FP64 (value 0), instead of letting the server choose. */
#define FMM2D_SERVE_PREC_AS_GIVEN 0x40u

typedef struct fmm2d_plan fmm2d_plan;

/* Plan description returned by fmm2d_plan_query. */
typedef struct {
  int32_t tiling;          /* fmm2d_tiling */
  int32_t levels;          /* leaf level L (root = level 0) */
  int32_t p;               /* highest expansion power (p coefficients + Q) */
  int32_t l_min;           /* first level with M2L translations */
  uint32_t flags;
  int32_t built;           /* 1 after a successful fmm2d_build */
  double eps;              /* requested tolerance */
  double domain[3];        /* x0, y0, S: domain square [x0, x0+S) x [y0, y0+S) */
  double leaf_scale;       /* septree: leaf hexagon circumradius r; triangle:
                              root inradius rho0; quadtree: 2^-L (frame units) */
  int64_t n_src, n_tgt;
  int64_t n_cells[24];     /* occupied cells per level 0..L */
  int64_t n_m2l;           /* M2L translations (list entries) */
  int64_t n_p2p_pairs;     /* source-target pairs summed directly */
  int32_t n_m2l_ops;       /* distinct M2L operators (lattice offsets) */
  int32_t max_far;         /* longest M2L list (P4 of Table 2 for interior cells) */
  int32_t max_near;        /* longest Near list (P2 of Table 2) */
  int32_t device_error;    /* nonzero if a kernel of the last evaluation gave up a
                              bounded wait (results of that evaluation invalid) */
  int64_t n_leaves;        /* leaves holding points (adaptive: of every level) */
  int64_t max_leaf_src;    /* most sources in one leaf */
  int64_t max_leaf_tgt;    /* most targets in one leaf */
} fmm2d_info;

/*
 * fmm2d_default_params - the planner's rules, exposed for callers and tests.
 *   levels_out: with leaf_target >= 1, the smallest leaf level L whose
 *     expected mean points per occupied leaf of a uniform input of n_points
 *     points is <= leaf_target (the tiling's leaf area times n_points); with
 *     leaf_target == 0, the level of S_opt (Table 2, App. A-C): the L whose
 *     expected points per leaf s minimise the s-dependent cost
 *     (N / s) b/(b-1) (P4 + 2) p^2 + M P2 s for N = M = n_points and p_out.
 *   p_out: smallest p with kappa^(p+1) <= eps, kappa = 1/(1 + rho/r) from
 *     Table 2 (Sec. 8; septree rho/r measured on the GBT aggregates, giving
 *     kappa = 0.525).
 *   leaf_scale_out: septree leaf circumradius for that L (frame units; the
 *     smallest 2^-40 multiple for which every point of the domain square has
 *     its nearest hexagon centre inside the L-digit GBT region), triangle root
 *     inradius, or 2^-L for the quadtree.
 * Any output pointer may be NULL.  Returns FMM2D_EINVAL for a bad tiling,
 * eps outside (0, 1), n_points < 0 or leaf_target < 0.
 */
fmm2d_status fmm2d_default_params(int tiling, int64_t n_points, int leaf_target, double eps,
                                  int *levels_out, int *p_out, double *leaf_scale_out);

/*
 * fmm2d_plan_create - make an empty plan.  The expansion order follows the
 * truncation error bounds of Sec. 8 (eqs. 14-15) with the ratios of Table 2:
 * with p == 0 the plan keeps the smallest p with kappa^(p+1) <= eps (as
 * fmm2d_default_params).
 *   tiling: FMM2D_QUAD, FMM2D_SEPT or FMM2D_TRI.
 *   levels: leaf level L (1..12 quadtree/triangle, 1..9 septree; with
 *     FMM2D_ADAPTIVE the finest level, 1..16 and 1..11), or 0 to
 *     choose it at fmm2d_build time with fmm2d_default_params (leaf target 64).
 *   p: highest expansion power 1..48, or 0 to derive it from eps.
 *   eps: requested relative tolerance (used when p == 0), 0 < eps < 1.
 *   flags: FMM2D_PREC_* | FMM2D_IN_F32 | FMM2D_ADAPTIVE | FMM2D_FIELD.
 * The domain defaults to the unit square [0,1)^2.  On success *out owns all
 * plan memory until fmm2d_plan_destroy.  Errors: FMM2D_EINVAL, FMM2D_ENOMEM.
 */
fmm2d_status fmm2d_plan_create(int tiling, int levels, int p, double eps, unsigned flags,
                               fmm2d_plan **out);

/*
 * fmm2d_plan_set_params - change the leaf level, expansion order and
 * tolerance of a plan (same meaning and ranges as fmm2d_plan_create); the
 * plan's device memory is kept and reused.  Invalidates a previous build.
 */
fmm2d_status fmm2d_plan_set_params(fmm2d_plan *plan, int levels, int p, double eps);

/*
 * fmm2d_plan_set_leaf_size - leaf size of an FMM2D_ADAPTIVE plan: a cell is
 * split while it holds more than leaf_size sources or more than leaf_size
 * targets and is above the finest level (leaf_size >= 0; 0 splits every
 * occupied cell down to the finest level, which reproduces the uniform
 * tree).  Ignored by uniform plans.  Invalidates a previous build.
 * Errors: FMM2D_EINVAL (null plan, negative size).
 */
fmm2d_status fmm2d_plan_set_leaf_size(fmm2d_plan *plan, int leaf_size);

/*
 * fmm2d_plan_set_domain - set the domain square [x0, x0+S) x [y0, y0+S)
 * (S > 0).  Every source and target must lie in it (else fmm2d_build returns
 * FMM2D_EDOMAIN).  Invalidates a previous build.
 */
fmm2d_status fmm2d_plan_set_domain(fmm2d_plan *plan, double x0, double y0, double size);

/*
 * fmm2d_build - key, sort and tree the point sets (Sec. 4-6: CellIndex,
 * Parent/Children, Neighbors, NeighborsE4).
 *   src_xy_dev: n_src interleaved points; tgt_xy_dev: n_tgt points.  Passing
 *   the same pointer and count for both marks the sets as identical (the
 *   sort is shared).  n_src, n_tgt >= 0.
 * The points are copied (sorted, relative to their leaf centres) into plan
 * memory; the caller may reuse its buffers after the call returns.  The call
 * synchronises `stream` once to read back the per-level cell counts.
 * Errors: FMM2D_EINVAL, FMM2D_ENOMEM, FMM2D_EDOMAIN (plan left unbuilt),
 * FMM2D_ETIMEOUT (a bounded wait between tiles of the radix sort gave up;
 * plan left unbuilt), FMM2D_ECUDA.
 */
fmm2d_status fmm2d_build(fmm2d_plan *plan, const void *src_xy_dev, int64_t n_src,
                         const void *tgt_xy_dev, int64_t n_tgt, void *stream);

/*
 * fmm2d_build_forest - build many independent instances at once (batched
 * solves): instance i holds the points [offsets[i], offsets[i+1]) of xy_dev
 * (sources = targets); all instances share the plan's tiling, domain, p and
 * leaf size, and never interact.  The instances form one adaptive tree with
 * one level-0 cell per instance, so one fmm2d_evaluate (strengths and
 * potentials concatenated in the same order) runs every instance with the
 * launches of a single solve.  Needs an FMM2D_ADAPTIVE plan; its `levels`
 * (0 = the largest level for which n_inst * b^levels < 2^32) is the finest
 * level.  offsets: HOST array of n_inst + 1 non-decreasing int64, offsets[0]
 * = 0.  The paper has no batched form; each instance is the FMM of Sec. 2.
 * Errors: FMM2D_EINVAL (not adaptive, bad offsets, too many instances for the
 * finest level), FMM2D_ENOMEM, FMM2D_EDOMAIN, FMM2D_ETIMEOUT (as fmm2d_build),
 * FMM2D_ECUDA.
 */
fmm2d_status fmm2d_build_forest(fmm2d_plan *plan, const void *xy_dev, const int64_t *offsets,
                                int n_inst, void *stream);

/*
 * fmm2d_evaluate - one FMM evaluation on the built geometry (Sec. 2):
 * P2M, M2M, M2L, L2L, L2P and P2P, then the potentials are written in the
 * caller's original target order.
 *   strengths_dev: n_src values (float64, or float32 with FMM2D_IN_F32).
 *   potentials_dev: n_tgt float64 outputs, Re Phi_j.
 * May be called any number of times with new strengths.  Asynchronous on
 * `stream`.  Errors: FMM2D_ENOTREADY (not built), FMM2D_EINVAL, FMM2D_ECUDA.
 */
fmm2d_status fmm2d_evaluate(fmm2d_plan *plan, const void *strengths_dev, double *potentials_dev,
                            void *stream);

/*
 * fmm2d_evaluate_graph - fmm2d_evaluate (Sec. 2) through a CUDA graph, for
 * callers that evaluate many strength vectors on one geometry.  The first
 * call after a build, or with other strength / potential pointers, records
 * the evaluation's launches (on both of the plan's streams) into a graph and
 * instantiates it; every call then launches that graph on `stream`, one
 * launch instead of about twenty.  The graph reads the strengths from, and
 * writes the potentials to, the recorded addresses: change the values in
 * those buffers between calls, not the pointers (new pointers re-record).
 * Results are those of fmm2d_evaluate, bit for bit.
 *   strengths_dev, potentials_dev: as fmm2d_evaluate (device, caller-owned,
 *     kept valid while the graph may be replayed).
 *   stream: a created stream; the legacy default stream (NULL), or a plan
 *     with profiling on, gets a plain fmm2d_evaluate instead.
 * Any fmm2d_build / fmm2d_build_forest invalidates the graph (the next call
 * re-records).  The plan owns the graph (freed by fmm2d_plan_destroy).
 * Asynchronous on `stream`.  Must not be called while `stream` is being
 * captured by the caller.  Errors: as fmm2d_evaluate; FMM2D_ECUDA when the
 * recording or the instantiation fails.
 */
fmm2d_status fmm2d_evaluate_graph(fmm2d_plan *plan, const void *strengths_dev,
                                  double *potentials_dev, void *stream);

/*
 * fmm2d_evaluate_field - fmm2d_evaluate, and also the field
 *     F_j = sum_{i : x_i != y_j} u_i / (y_j - x_i),
 * the derivative of the complex potential of eq. 1 (Sec. 2).  Unlike the
 * potential's imaginary part it is single valued; the gradient of Re Phi is
 * (Re F_j, -Im F_j).  It is computed on the same tree, lists and expansions by
 * the differentiated operators: sum u_i / (y - x_i) over the Near sources,
 * sum_{l>=1} l b_l (y - c)^(l-1) of the leaf's local expansion, and on
 * adaptive trees Q / (y - c) - sum_k k a_k (y - c)^-(k+1) of each W cell's
 * multipole.  In the FP32 forms the field's near and far sums run in FP32
 * (compensated partial sums), in the others in FP64.
 *   strengths_dev, potentials_dev: as fmm2d_evaluate.
 *   field_dev: 2 * n_tgt float64 outputs, (Re F_j, Im F_j) interleaved, in
 *     the caller's target order.
 * FP32 forms (FMM2D_PREC_MIXED, FMM2D_PREC_MIXED_TC) need a plan created with
 * FMM2D_FIELD.  Asynchronous on `stream`.  Errors: as fmm2d_evaluate;
 * FMM2D_EINVAL for a null field pointer or an FP32-form plan created without
 * FMM2D_FIELD.
 */
fmm2d_status fmm2d_evaluate_field(fmm2d_plan *plan, const void *strengths_dev,
                                  double *potentials_dev, double *field_dev, void *stream);

/* fmm2d_plan_query - fill *info (host struct) with the plan's parameters and
 * counts.  Errors: FMM2D_EINVAL. */
fmm2d_status fmm2d_plan_query(const fmm2d_plan *plan, fmm2d_info *info);

/*
 * fmm2d_debug_export - copy one intermediate of the last build / evaluate to
 * host memory for verification (synchronises the plan's last stream).
 *   what:
 *     1 source keys (int64, leaf key of every source, input order)
 *     2 source sort permutation (int64, sorted position -> input index)
 *     3 target keys, 4 target sort permutation (as 1, 2)
 *     5 occupied cell keys of `level` (int64, ascending)
 *     6 Near list pairs at the leaf level (int64 pairs: target key, source key)
 *     7 M2L list pairs of `level` (int64 pairs: target key, source key)
 *     8 multipoles of `level`: per cell (in the order of 5) p+1 complex128
 *       values, Q then a_1..a_p, unscaled (Greengard-Rokhlin form about the
 *       cell centre)
 *     9 locals of `level`: per cell p+1 complex128 values b_0..b_p (b_0 real
 *       part only)
 *    10 near-field part of Phi (float64, input target order)
 *    11 far-field part of Phi (float64, input target order)
 *    12 cell centres of `level` (complex128, order of 5, original coordinates)
 *   FMM2D_ADAPTIVE plans (int64 tuples; `level` ignored):
 *    13 cells: (level, key, split) of every cell, ordered by (level, key)
 *    14 U (P2P) pairs, 15 W (M2P) pairs, 16 X (P2L) pairs, 17 M2L pairs:
 *       (target level, target key, source level, source key), grouped by
 *       target in cell order
 *   host_buf / cap: destination and its size in bytes; with host_buf NULL only
 *   *written (required bytes) is set.
 * Errors: FMM2D_EINVAL (unknown what / level, cap too small),
 * FMM2D_ENOTREADY.
 */
fmm2d_status fmm2d_debug_export(fmm2d_plan *plan, int what, int level, void *host_buf,
                                size_t cap, size_t *written);

/*
 * fmm2d_plan_set_profiling - when on (1 or 2), fmm2d_build / fmm2d_evaluate
 * record CUDA events around every stage on the stream that runs it, and
 * fmm2d_stage_times returns the accumulated milliseconds per stage
 * (keys, sort, tree, lists, p2m, m2m, m2l, l2l, l2p, p2p, other, field) and the
 * number of launches of each.  With 1 the evaluation runs as usual: the
 * far-field stages (P2M ... L2L) run on a plan stream concurrently with P2P
 * on the caller's stream, so their times overlap.  With 2 every stage runs
 * on the caller's stream, one after the other, so that each time is the
 * stage's own.  Resets the accumulators.
 */
fmm2d_status fmm2d_plan_set_profiling(fmm2d_plan *plan, int on);
fmm2d_status fmm2d_stage_times(fmm2d_plan *plan, double *ms_host, int64_t *launches_host,
                               int cap, int *n_stages);

/*
 * fmm2d_plan_set_debug_stall - test switch of the bounded device waits (the
 * paper has no counterpart).  When on, every CTA of the tensor-core M2L
 * (FMM2D_PREC_MIXED_TC) makes its first operator wait on an mbarrier that
 * nothing arrives on, before it issues any MMA: the wait gives up after about
 * a second, the CTA lets its operator copies in flight land, frees its tensor
 * memory and returns, and the evaluation's device_error (fmm2d_plan_query)
 * is set; its results are then invalid.  The next evaluation with the switch
 * off is normal (device_error is cleared at the start of each one).  Errors:
 * FMM2D_EINVAL (null plan).
 */
fmm2d_status fmm2d_plan_set_debug_stall(fmm2d_plan *plan, int on);

/* fmm2d_plan_destroy - free all plan memory (device and host).  NULL is a no-op. */
void fmm2d_plan_destroy(fmm2d_plan *plan);

/* fmm2d_last_error - text of the plan's last error ("" if none).  The
 * pointer stays valid until the next call on the plan.  NULL plan: the last
 * error of a failed fmm2d_plan_create on this thread. */
const char *fmm2d_last_error(const fmm2d_plan *plan);

/*
 * fmm2d_measure_alu_peaks - measured peak rates of the units the kernels are
 * bound by, for roofline denominators (the paper has no counterpart).
 *   out[0]: FP32 FMA throughput, TFLOP/s (2 flops per FMA)
 *   out[1]: MUFU log2 throughput, 1e9 results/s
 *   out[2]: FP64 FMA throughput, TFLOP/s
 *   out[3]: number of SMs
 *   out[4]: TF32 tensor-core throughput (tcgen05.mma kind::tf32, FP32
 *     accumulation), TFLOP/s
 * out_host must hold 5 values.  Runs four short kernels on the current
 * device (legacy default stream) and synchronises.  Errors: FMM2D_EINVAL,
 * FMM2D_ENOMEM, FMM2D_ECUDA.
 */
fmm2d_status fmm2d_measure_alu_peaks(double *out_host);

/*
 * fmm2d_autotune - choose the leaf level L and expansion order p for a
 * point set by measurement (the a-priori p of Sec. 8, kappa^(p+1) <= eps, is a
 * worst-case bound and far larger than typical inputs need).
 *   The caller's points are evaluated with seeded probe strengths (uniform in
 *   [-1, 1]); potentials at 1024 evenly spaced targets are compared with an
 *   FP64 direct sum of eq. (2) computed on the GPU.  For L in {L0-1, L0,
 *   L0+1} (L0 the S_opt level of Table 2 for n_src, n_tgt and the a-priori
 *   p, as fmm2d_default_params with leaf_target 0) the smallest p with
 *   eps_rel_inf <= eps/3 is found by bisection and build + evaluate is timed;
 *   the fastest (L, p) is returned.
 *   tiling, eps, flags, domain (NULL = unit square): as for a plan.
 *   src_xy_dev / tgt_xy_dev: the points (device, layout as fmm2d_build).
 *   levels_out, p_out: the choice; err_out: its measured eps_rel_inf on the
 *   probe; ms_out: its build + evaluate time.  If no candidate meets eps/3,
 *   the a-priori (L0, p) is returned with err_out = ms_out = -1.
 * Allocates temporary device memory and synchronises `stream`.  Errors:
 * FMM2D_EINVAL, FMM2D_ENOMEM, FMM2D_ECUDA.
 */
fmm2d_status fmm2d_autotune(int tiling, double eps, unsigned flags, const double *domain,
                            const void *src_xy_dev, int64_t n_src, const void *tgt_xy_dev,
                            int64_t n_tgt, void *stream, int *levels_out, int *p_out,
                            double *err_out, double *ms_out);

/*
 * fmm2d_keys_sort_noalloc - leaf keys of a point set and their stable sort,
 * for callers that cannot allocate GPU memory.  The paper has no
 * counterpart: this is a library convenience, not a step of the method.
 *
 * Who needs it: code that runs where cudaMalloc is not allowed - inside a
 * memory arena owned by someone else, in a stream-ordered region that must
 * not synchronise on the allocator, or under a framework that forbids
 * allocations outside its own pool.  It does the keying (CellIndex, Sec. 4-6)
 * and sorting steps of fmm2d_build without creating a plan and without
 * allocating anything: the sort temporaries live in a static device array of
 * about 8.5 MiB that every GPU loading the library keeps until the process
 * exits.
 *   tiling, levels: as fmm2d_plan_create (levels >= 1).
 *   leaf_scale: septree only - 0, and the library uses the leaf circumradius
 *     of `levels` (the one fmm2d_build uses; the first call for a level
 *     enumerates it on the host, up to a few tenths of a second at level 9,
 *     then it is cached), or exactly that value (as fmm2d_plan_query reports
 *     it); any other value gives FMM2D_EINVAL.  Ignored for the other
 *     tilings.
 *   domain: NULL for the unit square, else {x0, y0, S}.
 *   xy_dev: n interleaved points (float64, or float32 with FMM2D_IN_F32 in
 *     flags), 0 <= n <= 1048576 (larger n: FMM2D_EINVAL, use fmm2d_build).
 *   keys_sorted_dev, perm_dev: n uint32 outputs (caller-owned device memory):
 *     the leaf keys in ascending order and, for each sorted position, the
 *     input index (equal keys keep their input order) - the same values
 *     fmm2d_debug_export reports for a plan built on these points.
 *   err_buf / err_cap: optional caller buffer that receives the error text.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress.  Every call synchronises `stream` (it reads back the
 * domain-error flag into host memory), so it must not be made while a stream
 * is being captured.  All calls share the array, so calls whose GPU work
 * overlaps race and must be serialised by the caller.  Errors: FMM2D_EINVAL, FMM2D_EDOMAIN,
 * FMM2D_ETIMEOUT (a bounded wait of the radix sort gave up), FMM2D_ECUDA.
 */
fmm2d_status fmm2d_keys_sort_noalloc(int tiling, int levels, double leaf_scale,
                                     const double *domain, const void *xy_dev, int64_t n,
                                     unsigned flags, uint32_t *keys_sorted_dev, uint32_t *perm_dev,
                                     void *stream, char *err_buf, size_t err_cap);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching server for FMM solves.  The paper has no
 * serving layer; each request runs the evaluation of fmm2d_build +
 * fmm2d_evaluate.  Requests are admitted, oldest first, as execution slots
 * and the HBM budget allow, and run concurrently on the slots' streams;
 * small adaptive requests (targets = sources, at most 524288 points) that
 * wait together with equal tiling, eps, p, flags and domain are solved as
 * one forest (fmm2d_build_forest), their results equal to the requests
 * solved alone within eps.  If such a merged solve fails, its requests are
 * run one by one, so each gets its own status.
 * ---------------------------------------------------------------------- */
typedef struct fmm2d_server fmm2d_server;

/* One solve.  All pointers are HOST memory owned by the caller and must stay
 * valid until the request completes. */
typedef struct {
  int32_t tiling;          /* fmm2d_tiling */
  int32_t levels;          /* leaf level, 0 = planner */
  int32_t p;               /* expansion order, 0 = from eps */
  uint32_t flags;          /* FMM2D_IN_F32, optionally FMM2D_PREC_* and
                              FMM2D_ADAPTIVE (leaf size 64 for the quadtree,
                              128 for the septree and the triangle tiling;
                              levels = finest level, 0 = the default); with no
                              precision bit the server uses the tensor-core
                              mixed form for eps >= 1e-6, the hybrid form down
                              to 1e-9 and the split form below, unless
                              FMM2D_SERVE_PREC_AS_GIVEN asks for the bits as
                              they are (FMM2D_PREC_FP64: the plain FP64 form) */
  double eps;
  double domain[3];        /* x0, y0, S; S <= 0 means the unit square */
  const void *src_xy;      /* n_src interleaved points */
  int64_t n_src;
  const void *tgt_xy;      /* n_tgt points, or NULL: targets = sources */
  int64_t n_tgt;
  const void *strengths;   /* n_src values */
  double *potentials;      /* output, one per target */
} fmm2d_request;

typedef struct {
  int32_t status;          /* fmm2d_status of the solve */
  int32_t levels, p;       /* parameters used */
  uint32_t flags;          /* precision used */
  int32_t slot;            /* execution slot that ran it */
  int32_t batched;         /* requests solved together with it as one forest
                              (1: alone); small adaptive requests with equal
                              tiling, eps, flags and domain that wait together
                              are merged (fmm2d_build_forest) */
  double queue_ms;         /* submit -> start */
  double run_ms;           /* start -> potentials in host memory */
  double latency_ms;       /* submit -> completion */
  char error[128];         /* text of the error of a failed request ("" if none) */
} fmm2d_result;

typedef struct {
  int64_t queued, running, completed;
  size_t bytes_in_use, budget_bytes;
  int32_t slots;
} fmm2d_serve_info;

/*
 * fmm2d_serve_create - start a server on the current device with `max_slots`
 * execution slots (host threads, each with its own stream and plans; 1..256)
 * and an HBM budget in bytes for the requests running at once.  Each slot
 * keeps the plans of its recent requests (operator tables and buffers); when
 * less than a tenth of the device memory is free, a slot trims them to
 * budget / (2 max_slots) bytes, least recently used first, and a request
 * whose solve runs out of device memory frees its slot's plans and buffers
 * and runs once more before it reports FMM2D_ENOMEM.
 * Errors: FMM2D_EINVAL, FMM2D_ENOMEM, FMM2D_ECUDA (no device).
 */
fmm2d_status fmm2d_serve_create(size_t hbm_budget_bytes, int max_slots, fmm2d_server **out);

/*
 * fmm2d_serve_submit - queue a request (non-blocking) and return its ticket.
 * Requests are admitted oldest first as a slot frees and their memory
 * estimate fits the budget next to the running ones; a request that does not
 * fit lets later, smaller ones go first.  Errors: FMM2D_EINVAL (bad request),
 * FMM2D_EBUSY (its estimate alone exceeds the budget), FMM2D_ENOMEM.
 */
fmm2d_status fmm2d_serve_submit(fmm2d_server *server, const fmm2d_request *request,
                                uint64_t *ticket);

/* fmm2d_serve_poll - FMM2D_ENOTREADY while the request runs; FMM2D_OK once it
 * is complete (the result is copied and the ticket released).  EINVAL for an
 * unknown ticket. */
fmm2d_status fmm2d_serve_poll(fmm2d_server *server, uint64_t ticket, fmm2d_result *result);

/* fmm2d_serve_wait - block until the request completes or `timeout_ms`
 * passes (FMM2D_ETIMEOUT, ticket kept). */
fmm2d_status fmm2d_serve_wait(fmm2d_server *server, uint64_t ticket, double timeout_ms,
                              fmm2d_result *result);

/* fmm2d_serve_stats - queue and memory counters. */
fmm2d_status fmm2d_serve_stats(fmm2d_server *server, fmm2d_serve_info *info);

/* fmm2d_serve_destroy - finish running requests, drop queued ones, free all. */
void fmm2d_serve_destroy(fmm2d_server *server);

#ifdef __cplusplus
}
#endif

#endif /* FMM2D_H */
