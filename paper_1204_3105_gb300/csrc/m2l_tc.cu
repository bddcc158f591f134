// m2l_tc.cu - M2L on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The M2L of a target cell is a sum over its NeighborsE4 list (eq. 3) of
// operator x multipole products.  On scaled coefficients the operator depends
// only on the lattice offset, i.e. on (child class, stencil entry), and not on
// the level, so all M2L targets of one class - whatever their level - share
// one operator per stencil entry.  A CTA takes 128 targets of one class and,
// for every stencil entry e, accumulates
//
//      D[128 x N] += A_e[128 x K] . B_op(e)[K x N]
//
// where row t of A_e is the gathered source multipole of target t for entry e
// as real numbers (Re a^_1, Im a^_1, ..., Re a^_p, Im a^_p, Q, 0...) and B is
// the real form of the complex (p+1) x (p+1) operator (output columns
// Re b^_0, Im b^_0, ..., Re b^_p, Im b^_p, 0...).  Both operands are split
// into TF32 parts: the gathered multipole in two (A = A0 + A1, i.e. rounded
// once to 22 significant bits) and the precomputed operator in three
// (B = B0 + B1 + B2, 33 bits).  Five products A0.B0 + A0.B1 + A0.B2 + A1.B0 +
// A1.B1, accumulated in FP32 in tensor memory (entries spread round-robin over
// eight accumulators added with compensation at the end), leave out only terms of
// relative size 2^-33, so the result has FP32-class accuracy (the one-time
// 22-bit rounding of A, 2^-23, dominates).  The Q log|z0| part of L_0 is
// accumulated separately in FP64 on the CUDA cores.
//
// Data movement: operator tiles (already split and laid out as the MMA reads
// them) arrive by cp.async.bulk (TMA bulk copy) into shared memory; the
// threads gather and split the multipole rows.  Two stages are pipelined with
// mbarriers: tcgen05.commit releases a stage once its MMAs have read it.
// Every wait is bounded: on time-out the kernel sets an error word, lets its
// copies in flight land, frees its tensor memory and returns.
#include <cstring>

#include "plan.h"

namespace fmm2d {

namespace {

constexpr int TC_M = 128;
constexpr int NACC = 8;                  // accumulators, entry e -> e % NACC
constexpr long long WAIT_CYCLES = 2000000000ll;   // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait on one phase of an mbarrier; false on time-out, or at once
// when another thread of the CTA has set *abort.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          const volatile int *abort = nullptr) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) return false;
    if (abort && *abort) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// Shared-memory matrix descriptor: no swizzle, K-major core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// byte step between 8-row groups along M / N.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// x rounded to TF32 (10 fraction bits), to nearest with ties away from zero,
// as integer operations on the bit pattern (finite x): adding half a unit of
// the kept last place to the magnitude and clearing the 13 dropped bits
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Byte offset of element (row, k) in a K-major no-swizzle operand tile.
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K / 4) * 128 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Shape of one kernel instance: accumulator column stride, pipeline depths
// and CTAs per SM.
template <int K, int N> struct TcShape {
  static constexpr uint32_t ACC = N <= 32 ? 32 : 64;
  static constexpr uint32_t COLS = NACC * ACC;            // 256 or 512 TMEM columns
  static constexpr int NA = K <= 32 ? 4 : 2;              // multipole (A) stages
  static constexpr int NB = K <= 32 ? 4 : 2;              // operator (B) stages
  static constexpr uint32_t A_BYTES = 128 * K * 4, B_BYTES = N * K * 4;
  static constexpr uint32_t SMEM = NA * (2 * A_BYTES) + NB * (3 * B_BYTES);
  static constexpr int CTAS = (N <= 32 && SMEM <= 104 * 1024) ? 2 : 1;
};

// Warp roles of a CTA: warps 0-7 gather (two threads per target row, one
// half of K each), split the rows into TF32 hi + lo and write the A stages,
// then read the accumulators in the epilogue; warp 8 (one thread) issues the
// MMAs; warp 9 (one thread) copies the operator tiles.  Hand-offs are
// mbarriers only: a_full / b_full (stage written / landed), a_empty /
// b_empty (stage read by the MMAs: tcgen05.commit), acc_full (a tile's MMAs
// done) and acc_empty (its accumulators read).
constexpr int TC_PROD = 256;                      // gathering threads
constexpr int TC_THREADS = TC_PROD + 64;          // + MMA warp + operator warp
constexpr int TC_MMA_WARP = 8, TC_LOAD_WARP = 9;

template <int K, int N>
__global__ void __launch_bounds__(TC_THREADS, (TcShape<K, N>::CTAS)) k_m2l_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  using SH = TcShape<K, N>;
  constexpr uint32_t A_BYTES = SH::A_BYTES, B_BYTES = SH::B_BYTES;
  constexpr int NA = SH::NA, NB = SH::NB;
  constexpr uint32_t SBO = (K / 4) * 128, LBO = 128;
  constexpr uint32_t IDESC = idesc_tf32(TC_M, N);
  constexpr uint32_t ACC = SH::ACC, COLS = SH::COLS;
  constexpr int QH = K / 8;                 // 16-byte chunks of a row per half
  // layout: A stages [NA] x (A0, A1), operator stages [NB] x (B0, B1, B2),
  // then the barriers and a few words
  unsigned char *const Bbase = smem + NA * (2 * A_BYTES);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SH::SMEM);
  uint64_t *a_full = bars, *a_empty = bars + NA, *b_full = bars + 2 * NA,
           *b_empty = bars + 2 * NA + NB, *acc_full = bars + 2 * NA + 2 * NB,
           *acc_empty = acc_full + 1, *never_bar = acc_full + 2;
  constexpr int NBARS = 2 * NA + 2 * NB + 3;
  static_assert(NBARS * 8 + 8 + (MAX_CLASSES + 2) * 4 <= 1024, "barrier area");
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + NBARS);
  int *s_cnt = reinterpret_cast<int *>(tmem_slot + 2);               // [MAX_CLASSES]
  volatile int *s_abort = s_cnt + MAX_CLASSES;
  volatile uint32_t *s_consumed = reinterpret_cast<volatile uint32_t *>(s_cnt + MAX_CLASSES + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == TC_MMA_WARP) tmem_alloc(tmem_slot, COLS);
  if (tid == 0) {
    for (int i = 0; i < NA; ++i) {
      mbar_init(&a_full[i], TC_PROD / 32);
      mbar_init(&a_empty[i], 1);
    }
    for (int i = 0; i < NB; ++i) {
      mbar_init(&b_full[i], 1);
      mbar_init(&b_empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, TC_PROD / 32);
    mbar_init(never_bar, 1);
    fence_barrier_init();
    *s_abort = 0;
    *s_consumed = 0;
  }
  if (tid < MAX_CLASSES) s_cnt[tid] = tid < a.n_classes ? a.cls_cnt[tid] : 0;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  int total_tiles = 0;
  for (int c = 0; c < a.n_classes; ++c) total_tiles += (s_cnt[c] + TC_M - 1) / TC_M;
  const int S = a.split;                    // work item = (tile, part of its entries)
  const int p = a.p;
  // the work items of this CTA and their entry ranges (the same sequence for
  // every role)
  auto item_info = [&](int item, int &c, int &row0, int &nrows, int &e_lo, int &E) {
    const int tile = item / S, sidx = item - tile * S;
    c = 0;
    int t0 = tile;
    while (t0 >= (s_cnt[c] + TC_M - 1) / TC_M) {
      t0 -= (s_cnt[c] + TC_M - 1) / TC_M;
      ++c;
    }
    row0 = t0 * TC_M;
    nrows = min(TC_M, s_cnt[c] - row0);
    const int E_all = a.sten_len[c];
    const int chunk = (E_all + S - 1) / S;
    e_lo = min(E_all, sidx * chunk);
    E = min(E_all, e_lo + chunk) - e_lo;
  };

  if (warp == TC_LOAD_WARP) {
    // ---- operator copies: entry it into stage it % NB once its previous
    // use (entry it - NB) has been read by the MMAs
    if (lane == 0) {
      uint32_t it = 0;
      for (int item = blockIdx.x; item < total_tiles * S && !*s_abort; item += gridDim.x) {
        int c, row0, nrows, e_lo, E;
        item_info(item, c, row0, nrows, e_lo, E);
        const uint16_t *ops_c = a.sten_ops + c * FAR_MAX + e_lo;
        for (int e = 0; e < E; ++e, ++it) {
          const int st = it % NB;
          if (it >= NB && !mbar_wait(&b_empty[st], ((it / NB) - 1) & 1, s_abort)) {
            *s_abort = 1;
            break;
          }
          mbar_expect_tx(&b_full[st], 3 * B_BYTES);
          bulk_g2s(Bbase + st * (3 * B_BYTES), a.btab + (size_t)ops_c[e] * 3 * B_BYTES, 3 * B_BYTES,
                   &b_full[st]);
        }
      }
      // let the copies in flight land before the CTA exits: those of the
      // entries the MMA thread did not wait for
      __syncwarp(1u);
      const uint32_t issued = it, from = *s_consumed;
      for (uint32_t u = from; u < issued; ++u) mbar_wait(&b_full[u % NB], (u / NB) & 1);
    }
  } else if (warp == TC_MMA_WARP) {
    // ---- MMAs: entry it from A stage it % NA and operator stage it % NB,
    // into accumulator e % NACC of the item
    if (lane == 0) {
      uint32_t it = 0, j = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < total_tiles * S && ok; item += gridDim.x, ++j) {
        int c, row0, nrows, e_lo, E;
        item_info(item, c, row0, nrows, e_lo, E);
        // the previous item's accumulators must have been read
        if (j >= 1 && !mbar_wait(acc_empty, (j - 1) & 1, s_abort)) ok = false;
        for (int e = 0; e < E && ok; ++e, ++it) {
          const int sa = it % NA, sb = it % NB;
          if (!mbar_wait(&a_full[sa], (it / NA) & 1, s_abort)) { ok = false; break; }
          // test switch: the CTA's first operator wait is on a barrier that
          // nothing arrives on, so its bounded wait runs out before any MMA
          const bool stall = a.debug_stall && it == 0;
          if (stall ? !mbar_wait(never_bar, 0) : !mbar_wait(&b_full[sb], (it / NB) & 1, s_abort)) {
            ok = false;
            break;
          }
          *s_consumed = it + 1;
          tc_fence_after();
          // descriptors of the stage's operands; a K step advances the start
          // address field (address / 16) by 2 LBO / 16
          const uint64_t dA0 = sdesc(smem_u32(smem + sa * (2 * A_BYTES)), LBO, SBO);
          const uint64_t dA1 = dA0 + (A_BYTES >> 4);
          const uint64_t dB0 = sdesc(smem_u32(Bbase + sb * (3 * B_BYTES)), LBO, SBO);
          const uint64_t dB1 = dB0 + (B_BYTES >> 4), dB2 = dB1 + (B_BYTES >> 4);
          const uint32_t acc = tmem + (uint32_t)(e % NACC) * ACC;
#pragma unroll
          for (int ks = 0; ks < K / 8; ++ks) {
            const uint64_t o = (uint64_t)(ks * 2 * LBO) >> 4;
            mma_tf32(acc, dA0 + o, dB0 + o, IDESC, (e >= NACC || ks > 0) ? 1u : 0u);
            mma_tf32(acc, dA0 + o, dB1 + o, IDESC, 1u);
            mma_tf32(acc, dA0 + o, dB2 + o, IDESC, 1u);
            mma_tf32(acc, dA1 + o, dB0 + o, IDESC, 1u);
            mma_tf32(acc, dA1 + o, dB1 + o, IDESC, 1u);
          }
          mma_commit(&a_empty[sa]);
          mma_commit(&b_empty[sb]);
        }
        if (ok) mma_commit(acc_full);   // the item's MMAs (none: at once)
      }
      if (!ok) *s_abort = 1;
      // the MMAs committed so far, before their TMEM is freed
      if (*s_consumed > 0) {
        const uint32_t last = *s_consumed - 1;
        mbar_wait(&a_empty[last % NA], (last / NA) & 1);
      }
    }
  } else {
    // ---- producers: warps 0-7, thread (row, half)
    const int row = tid & (TC_M - 1), half = tid >> 7;
    uint32_t it = 0, j = 0;
    for (int item = blockIdx.x; item < total_tiles * S; item += gridDim.x, ++j) {
      int c, row0, nrows, e_lo, E;
      item_info(item, c, row0, nrows, e_lo, E);
      const int sidx = item - (item / S) * S;
      const int g = row < nrows ? a.cls_cells[(int64_t)c * a.cls_cap + row0 + row] : -1;
      const int64_t fi = g >= 0 ? (int64_t)g - a.far_first : 0;
      double ls = 0.0;
      if (g >= 0 && half == 0) {
        int l = a.l_min;
        while (l < a.L && (int64_t)g >= a.lev_first[l + 1]) ++l;
        ls = a.log_abs_scale[l];
      }
      double L0 = 0.0;
      const uint16_t *ops_c = a.sten_ops + c * FAR_MAX + e_lo;
      const int *srcs = a.far_full + fi * FAR_MAX + e_lo;
      auto src_of = [&](int e) { return (g >= 0 && e < E) ? srcs[e] : -1; };
      auto lz_of = [&](int e) { return (half == 0 && e < E) ? a.logz[ops_c[e]] : 0.0; };
      auto load_row = [&](int src_e, float4 (&f)[QH], double &q, int &src) {
        src = src_e;
        const float4 *rowp = reinterpret_cast<const float4 *>(a.ma + (int64_t)(src >= 0 ? src : 0) * a.P);
#pragma unroll
        for (int qq = 0; qq < QH; ++qq) {
          const int qi = half * QH + qq;
          f[qq] = (src >= 0 && 4 * qi < 2 * p) ? rowp[qi] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        q = src >= 0 ? a.mQ[src] : 0.0;
      };
      // Two slots, each holding one entry's row, Q, source slot and log|zeta|
      // of its operator; after an entry is written out its slot is refilled
      // with the entry two ahead, whose source slot was read one entry
      // earlier still.  The loop body handles the two slots in turn, so no
      // register is copied while its load is in flight.
      float4 f0[QH], f1[QH];
      double q0, q1, lz0 = lz_of(0), lz1 = lz_of(1);
      int s0, s1;
      load_row(src_of(0), f0, q0, s0);
      load_row(src_of(1), f1, q1, s1);
      int nx0 = src_of(2), nx1 = src_of(3);   // source slots of the next refills
      auto step = [&](int e, float4 (&f)[QH], double &q, int &sv, double &lz, int &nx) {
        const int sa = it % NA;
        unsigned char *A0 = smem + sa * (2 * A_BYTES), *A1 = A0 + A_BYTES;
        // the stage's previous entry (it - NA) must have been read
        if (it >= NA && !mbar_wait(&a_empty[sa], ((it / NA) - 1) & 1, s_abort)) *s_abort = 1;
        if (*s_abort) return false;
        // split the row into TF32 A0 + A1 (Q sits at index 2p)
        const float qf = (float)q;
#pragma unroll
        for (int qq = 0; qq < QH; ++qq) {
          const int qi = half * QH + qq;
          float v[4] = {f[qq].x, f[qq].y, f[qq].z, f[qq].w};
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int k = 4 * qi + jj;
            v[jj] = k < 2 * p ? v[jj] : (k == 2 * p ? qf : 0.f);
          }
          float4 h, l;
          h.x = tf32_rna(v[0]); l.x = tf32_rna(v[0] - h.x);
          h.y = tf32_rna(v[1]); l.y = tf32_rna(v[1] - h.y);
          h.z = tf32_rna(v[2]); l.z = tf32_rna(v[2] - h.z);
          h.w = tf32_rna(v[3]); l.w = tf32_rna(v[3] - h.w);
          const uint32_t off = core_off(row, 4 * qi, K);
          *reinterpret_cast<float4 *>(A0 + off) = h;
          *reinterpret_cast<float4 *>(A1 + off) = l;
        }
        if (sv >= 0 && half == 0) L0 += q * (ls + lz);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[sa]);
        ++it;
        // refill the slot with entry e + 2
        load_row(nx, f, q, sv);
        lz = lz_of(e + 2);
        nx = src_of(e + 4);
        return true;
      };
      for (int e = 0; e < E; e += 2) {
        if (!step(e, f0, q0, s0, lz0, nx0)) break;
        if (e + 1 < E && !step(e + 1, f1, q1, s1, lz1, nx1)) break;
      }
      if (*s_abort) break;
      // the item's MMAs done: read and sum the accumulators
      if (!mbar_wait(acc_full, j & 1, s_abort)) {
        *s_abort = 1;
        break;
      }
      tc_fence_after();
      // sum the used accumulators in FP32 with Kahan compensation, 16 columns
      // at a time; warps 0-3 take the even column chunks, warps 4-7 the odd
      // ones (same TMEM lanes)
      const int nacc = E < NACC ? E : NACC;
      const uint32_t lane_base = ((uint32_t)((warp & 3) * 32)) << 16;
#pragma unroll
      for (int q = 0; q < N / 16; ++q) {
        if ((q & 1) != half) continue;
        float d[16], cmp[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) d[i] = cmp[i] = 0.f;
        for (int ac = 0; ac < nacc; ++ac) {
          float t16[16];
          tmem_ld16(tmem + lane_base + (uint32_t)ac * ACC + q * 16, t16);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float y = t16[i] - cmp[i];
            const float t = d[i] + y;
            cmp[i] = (t - d[i]) - y;
            d[i] = t;
          }
        }
        if (g >= 0 && S == 1) {
          if (q == 0) a.lL0[g] = L0 + (double)d[0];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int l = 8 * q + i;
            if (l >= 1 && l <= p) a.lb[(int64_t)g * a.P + l - 1] = make_float2(d[2 * i], d[2 * i + 1]);
          }
        } else if (g >= 0) {   // this part's sums, added up by k_m2l_tc_reduce
          const int64_t pr = (int64_t)sidx * a.n_far + fi;
          if (q == 0) a.part_L0[pr] = L0 + (double)d[0];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int l = 8 * q + i;
            if (l >= 1 && l <= p) a.part_lb[pr * a.P + l - 1] = make_float2(d[2 * i], d[2 * i + 1]);
          }
        }
      }
      // the accumulators may be overwritten by the next item's MMAs
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
  }
  __syncwarp();   // the single-thread roles rejoin their warps
  if (*s_abort && tid == 0) atomicOr(a.err, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == TC_MMA_WARP) tmem_dealloc(tmem, COLS);
}

// Sum of the split parts of every far cell, in part order (FP64, rounded once).
__global__ void k_m2l_tc_reduce(int split, int64_t n_far, int64_t far_first, int p, int P,
                                const float2 *__restrict__ part_lb,
                                const double *__restrict__ part_L0, double *__restrict__ lL0,
                                float2 *__restrict__ lb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // (cell, column)
  const int64_t fi = i / (p + 1);
  const int l = (int)(i - fi * (p + 1));
  if (fi >= n_far) return;
  const int64_t g = far_first + fi;
  if (l == 0) {
    double v = 0.0;
    for (int sp = 0; sp < split; ++sp) v += part_L0[(int64_t)sp * n_far + fi];
    lL0[g] = v;
  } else {
    double re = 0.0, im = 0.0;
    for (int sp = 0; sp < split; ++sp) {
      const float2 v = part_lb[((int64_t)sp * n_far + fi) * P + l - 1];
      re += (double)v.x;
      im += (double)v.y;
    }
    lb[g * P + l - 1] = make_float2((float)re, (float)im);
  }
}

template <int K, int N>
cudaError_t launch_tc(const TcArgs &a, int64_t n_far_cells, cudaStream_t s) {
  using SH = TcShape<K, N>;
  const size_t smem = SH::SMEM + 1024;   // + barriers and words (under 1 KB)
  cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<K, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int S = a.split > 1 && a.part_lb && a.part_L0 ? a.split : 1;
  TcArgs b = a;
  b.split = S;
  int64_t items = ((n_far_cells + TC_M - 1) / TC_M + a.n_classes) * S;
  int grid = (int)std::min<int64_t>(items, (int64_t)a.sms * SH::CTAS);
  if (grid < 1) return cudaSuccess;
  k_m2l_tc<K, N><<<grid, TC_THREADS, smem, s>>>(b);
  if (S > 1) {
    const int64_t work = n_far_cells * (a.p + 1);
    k_m2l_tc_reduce<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(
        S, a.n_far, a.far_first, a.p, a.P, a.part_lb, a.part_L0, a.lL0, a.lb);
  }
  return cudaGetLastError();
}

uint32_t tf32_round_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x1000u;
  u &= ~0x1FFFu;
  return u;
}

// TF32 tensor-core throughput probe: one CTA per SM, one thread issuing
// `reps` back-to-back tcgen05.mma of M = 128, N = 256, K = 8 (TF32 in, FP32
// accumulate in TMEM) from fixed shared-memory operands; the commit of the
// last one is waited on (bounded) before TMEM is freed.
constexpr int PK_N = 256;
__global__ void __launch_bounds__(128, 1) k_tf32_peak(int reps, int *err) {
  __shared__ __align__(1024) unsigned char sm[TC_M * 32 + PK_N * 32];
  __shared__ uint64_t bar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x;
  for (int i = tid; i < (TC_M * 32 + PK_N * 32) / 4; i += blockDim.x)
    reinterpret_cast<float *>(sm)[i] = 0.f;
  if (tid < 32) tmem_alloc(&slot, PK_N);
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = slot;
  if (tid == 0) {
    constexpr uint32_t IDESC = idesc_tf32(TC_M, PK_N);
    const uint32_t a = smem_u32(sm), b = a + TC_M * 32;
    const uint64_t da = sdesc(a, 128, 256), db = sdesc(b, 128, 256);
    for (int r = 0; r < reps; ++r) mma_tf32(tmem, da, db, IDESC, r > 0 ? 1u : 0u);
    mma_commit(&bar);
    if (!mbar_wait(&bar, 0)) atomicOr(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32) tmem_dealloc(tmem, PK_N);
}

}  // namespace

cudaError_t tc_measure_tf32(double *tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int *err = nullptr;
  if ((e = cudaMalloc(&err, sizeof(int))) != cudaSuccess) return e;
  cudaMemset(err, 0, sizeof(int));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int reps = 8192;
  // a large dynamic shared-memory request keeps it to one CTA per SM
  const int pad = 150 * 1024;
  e = cudaFuncSetAttribute(k_tf32_peak, cudaFuncAttributeMaxDynamicSharedMemorySize, pad);
  if (e != cudaSuccess) {
    cudaFree(err);
    return e;
  }
  k_tf32_peak<<<sms, 128, pad>>>(64, err);   // warm-up
  cudaEventRecord(e0);
  k_tf32_peak<<<sms, 128, pad>>>(reps, err);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  int err_h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err_h, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(err);
  if (e != cudaSuccess) return e;
  if (err_h) return cudaErrorLaunchTimeout;
  *tflops = 2.0 * TC_M * PK_N * 8 * (double)reps * sms / (ms * 1e-3) * 1e-12;
  return cudaSuccess;
}

static int tc_ctas(int K, int N) {
  if (K == 32 && N == 32) return TcShape<32, 32>::CTAS;
  if (K == 48 && N == 48) return TcShape<48, 48>::CTAS;
  if (K == 56 && N == 64) return TcShape<56, 64>::CTAS;
  return TcShape<64, 64>::CTAS;
}

int tc_split(int64_t n_far_cells, int n_classes, int sms, int K, int N) {
  // Items of a tile's stencil entries split S ways, chosen for load balance:
  // the longest CTA runs ceil(tiles S / slots) items of 1/S of a tile; a
  // split costs about a tenth of a tile more (partial writes and the
  // reduction kernel).
  const int64_t slots = (int64_t)sms * tc_ctas(K, N);
  const int64_t tiles = (n_far_cells + TC_M - 1) / TC_M + n_classes;
  int best = 1;
  double best_cost = 1e30;
  for (int S = 1; S <= 4; ++S) {
    const double waves = (double)((tiles * S + slots - 1) / slots);
    const double cost = waves / S * (S > 1 ? 1.1 : 1.0);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = S;
    }
  }
  return best;
}

bool tc_shape(int p, int *K, int *N) {
  if (p <= 15) { *K = 32; *N = 32; return true; }
  if (p <= 23) { *K = 48; *N = 48; return true; }
  if (p <= 27) { *K = 56; *N = 64; return true; }
  if (p <= 31) { *K = 64; *N = 64; return true; }
  return false;
}

void tc_build_tables(const std::vector<double> &re, const std::vector<double> &im, int n_ops, int p,
                     int K, int N, std::vector<uint32_t> &out) {
  const int P1 = p + 1;
  const size_t words = (size_t)N * K;    // one operand tile in 32-bit words
  out.assign((size_t)n_ops * 3 * words, 0u);
  for (int o = 0; o < n_ops; ++o) {
    uint32_t *w0 = out.data() + (size_t)o * 3 * words, *w1 = w0 + words, *w2 = w1 + words;
    for (int n = 0; n < N; ++n) {
      const int l = n >> 1, part = n & 1;
      for (int kk = 0; kk < K; ++kk) {
        double val = 0.0;
        if (l <= p) {
          if (kk < 2 * p) {
            const int k = kk / 2 + 1, comp = kk & 1;
            const size_t idx = (size_t)o * P1 * P1 + (size_t)l * P1 + k;
            const double tr = re[idx], ti = im[idx];
            val = part == 0 ? (comp == 0 ? tr : -ti) : (comp == 0 ? ti : tr);
          } else if (kk == 2 * p) {
            const size_t idx = (size_t)o * P1 * P1 + (size_t)l * P1;
            val = part == 0 ? re[idx] : im[idx];
          }
        }
        // three TF32 parts of the FP64 value: B0 + B1 + B2 (33 bits)
        const uint32_t off = core_off(n, kk, K) / 4;
        double rest = val;
        uint32_t *dst[3] = {w0, w1, w2};
        for (int part = 0; part < 3; ++part) {
          const uint32_t w = tf32_round_host((float)rest);
          float wf;
          std::memcpy(&wf, &w, 4);
          dst[part][off] = w;
          rest -= (double)wf;
        }
      }
    }
  }
}

cudaError_t launch_m2l_tc(const TcArgs &a, int K, int N, int64_t n_far_cells, cudaStream_t s) {
  if (n_far_cells <= 0) return cudaSuccess;
  if (K == 32 && N == 32) return launch_tc<32, 32>(a, n_far_cells, s);
  if (K == 48 && N == 48) return launch_tc<48, 48>(a, n_far_cells, s);
  if (K == 56 && N == 64) return launch_tc<56, 64>(a, n_far_cells, s);
  if (K == 64 && N == 64) return launch_tc<64, 64>(a, n_far_cells, s);
  return cudaErrorInvalidValue;
}

}  // namespace fmm2d
