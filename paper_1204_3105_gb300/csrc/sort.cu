// sort.cu - device exclusive scan and stable LSD radix sort of (key, value)
// pairs, used to order points by leaf key (Sec. 4: Morton / GBT indexing
// orders cells in memory) and to compact the occupied cells.
//
// Radix sort: 8-bit digits.  One kernel counts every pass's digit totals in
// a single read of the keys; each pass is then one kernel: a tile takes its
// index from a counter (so tiles start in order), ranks its keys stably
// (each warp ranks its 32 keys per round with __match_any_sync and the
// warps are ordered by a scan of their per-digit counts), publishes its
// per-digit counts and finds the counts of all earlier tiles by a decoupled
// look-back over their published words, then scatters.  Input order is kept
// among equal keys.  The look-back's waits are bounded: after a fixed
// number of polls the tile sets an error bit and goes on.
#include "plan.h"

namespace fmm2d {

namespace {

constexpr int SCAN_TH = 256, SCAN_IPT = 16, SCAN_TILE = SCAN_TH * SCAN_IPT;
constexpr int64_t SCAN_SINGLE_MAX = 1 << 14;   // arrays scanned by one block
constexpr int RS_TH = 256, RS_WARPS = RS_TH / 32, RS_IPT = 16, RS_TILE = RS_TH * RS_IPT;

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the total.
__device__ int block_excl_scan(int v, int &excl, int *sm_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) sm_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    int t = lane < nw ? sm_warp[lane] : 0;
    int ti = warp_incl_scan(t);
    if (lane < nw) sm_warp[lane] = ti - t;
    if (lane == nw - 1) sm_warp[32] = ti;
  }
  __syncthreads();
  excl = sm_warp[w] + inc - v;
  int total = sm_warp[32];
  __syncthreads();
  return total;
}

__global__ void k_scan_reduce(const int *__restrict__ in, int64_t n, int *__restrict__ sums) {
  __shared__ int sm[33];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int s = 0;
  for (int i = 0; i < SCAN_IPT; ++i) {
    int64_t idx = base + (int64_t)i * SCAN_TH + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  int ex;
  int tot = block_excl_scan(s, ex, sm);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of nb sums in place.
__global__ void k_scan_sums(int *sums, int nb) {
  __shared__ int sm[33];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < nb ? sums[i] : 0;
    int ex;
    int tot = block_excl_scan(v, ex, sm);
    if (i < nb) sums[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

// Single block: exclusive scan of n values (in place allowed), chunks of
// 1024 threads x 16 items with a running carry.  Used for small arrays.
__global__ void __launch_bounds__(1024) k_scan_single(const int *__restrict__ in,
                                                      int *__restrict__ out, int64_t n) {
  __shared__ int sm[33];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  constexpr int IPT = 16;
  for (int64_t base = 0; base < n; base += 1024 * IPT) {
    int v[IPT], s = 0;
    const int64_t b0 = base + (int64_t)threadIdx.x * IPT;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      v[i] = b0 + i < n ? in[b0 + i] : 0;
      s += v[i];
    }
    int ex;
    const int tot = block_excl_scan(s, ex, sm);
    int run = carry + ex;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      if (b0 + i < n) out[b0 + i] = run;
      run += v[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

__global__ void k_scan_tile(const int *__restrict__ in, int *__restrict__ out, int64_t n,
                            const int *__restrict__ sums) {
  __shared__ int tile[SCAN_TILE];
  __shared__ int sm[33];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  for (int i = 0; i < SCAN_IPT; ++i) {
    int64_t idx = base + (int64_t)i * SCAN_TH + threadIdx.x;
    tile[i * SCAN_TH + threadIdx.x] = idx < n ? in[idx] : 0;
  }
  __syncthreads();
  int loc[SCAN_IPT];
  int s = 0;
  for (int i = 0; i < SCAN_IPT; ++i) {
    loc[i] = s;
    s += tile[threadIdx.x * SCAN_IPT + i];
  }
  int ex;
  block_excl_scan(s, ex, sm);
  const int off = sums[blockIdx.x] + ex;
  for (int i = 0; i < SCAN_IPT; ++i) tile[threadIdx.x * SCAN_IPT + i] = off + loc[i];
  __syncthreads();
  for (int i = 0; i < SCAN_IPT; ++i) {
    int64_t idx = base + (int64_t)i * SCAN_TH + threadIdx.x;
    if (idx < n) out[idx] = tile[i * SCAN_TH + threadIdx.x];
  }
}

// Scratch of one sort (byte offsets): the digit totals of every pass, the
// tile counters, the look-back words (one per pass, tile and digit).
constexpr size_t RS_HIST_OFF = 0;                       // int [4][256]
constexpr size_t RS_CTR_OFF = 4 * 256 * sizeof(int);    // int [4] tile counters, int err
constexpr size_t RS_LB_OFF = RS_CTR_OFF + 256;          // uint64 [4][tiles][256]
// A look-back word: flag in the top two bits, a count below.
constexpr uint64_t LB_LOCAL = 1ull << 62, LB_INCL = 2ull << 62, LB_COUNT = LB_LOCAL - 1;
constexpr int LB_POLLS = 1 << 22;   // polls of one word before the wait gives up
constexpr int LB_WIN = 8;           // look-back words read per round

// Digit totals of every pass (atomics into the zeroed totals) and, for the
// tile of this block, the look-back words of every pass set to "not yet".
__global__ void k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int passes,
                             int *__restrict__ hist, uint64_t *__restrict__ lb, int nblocks) {
  __shared__ int h[4][256];
  for (int ps = 0; ps < 4; ++ps) h[ps][threadIdx.x] = 0;
  for (int ps = 0; ps < passes; ++ps)
    lb[((int64_t)ps * nblocks + blockIdx.x) * 256 + threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = 0; i < RS_IPT; ++i) {
    int64_t idx = base + (int64_t)i * RS_TH + threadIdx.x;
    if (idx < n) {
      const uint32_t k = keys[idx];
      for (int ps = 0; ps < passes; ++ps) atomicAdd(&h[ps][(k >> (8 * ps)) & 255u], 1);
    }
  }
  __syncthreads();
  for (int ps = 0; ps < passes; ++ps) {
    const int c = h[ps][threadIdx.x];
    if (c) atomicAdd(&hist[ps * 256 + threadIdx.x], c);
  }
}

__device__ __forceinline__ uint64_t lb_load(const uint64_t *p) {
  return *reinterpret_cast<const volatile uint64_t *>(p);
}
__device__ __forceinline__ void lb_store(uint64_t *p, uint64_t v) {
  *reinterpret_cast<volatile uint64_t *>(p) = v;
}

// One pass over one tile (the tile index comes from a counter, so every
// earlier tile has started): every element's rank inside the tile in
// (digit, input order) order, the tile's per-digit counts published and the
// counts of all earlier tiles gathered by look-back, the tile reordered in
// shared memory by rank, then written out run by run so that consecutive
// threads store to consecutive addresses of each digit's destination range.
__global__ void __launch_bounds__(RS_TH)
k_radix_onesweep(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                 uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
                 const int *__restrict__ hist, uint64_t *__restrict__ lb, int *__restrict__ ctr,
                 int *__restrict__ err) {
  __shared__ int wcnt[RS_WARPS][257];
  __shared__ int goff[256], dstart[256];
  __shared__ int sm_scan[33];
  __shared__ int s_tile;
  __shared__ uint32_t tk[RS_TILE], tv[RS_TILE];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1);
  for (int i = threadIdx.x; i < RS_WARPS * 257; i += RS_TH) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t tile0 = (int64_t)tile * RS_TILE;
  const int64_t base = tile0 + (int64_t)w * (32 * RS_IPT);
  const unsigned lt = (1u << lane) - 1u;
  uint32_t key[RS_IPT], val[RS_IPT];
  int loc[RS_IPT];
#pragma unroll
  for (int r = 0; r < RS_IPT; ++r) {
    int64_t idx = base + r * 32 + lane;
    bool valid = idx < n;
    key[r] = valid ? kin[idx] : 0u;
    val[r] = valid ? vin[idx] : 0u;
    int d = valid ? (int)((key[r] >> shift) & 255u) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int before = wcnt[w][d];
    loc[r] = before + __popc(peers & lt);
    __syncwarp();
    if (lane == __ffs(peers) - 1) wcnt[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  const int d = threadIdx.x;
  int run = 0;   // this tile's count of digit d
  for (int ww = 0; ww < RS_WARPS; ++ww) {   // exclusive scan over warps
    int t = wcnt[ww][d];
    wcnt[ww][d] = run;
    run += t;
  }
  // publish before waiting on anyone, so that later tiles always progress
  lb_store(&lb[(int64_t)tile * 256 + d], (tile == 0 ? LB_INCL : LB_LOCAL) | (uint64_t)run);
  int ex;
  const int tot = block_excl_scan(run, ex, sm_scan);
  dstart[d] = ex;
  int dbase;
  block_excl_scan(hist[d], dbase, sm_scan);
  // look-back: the counts of digit d in all earlier tiles, LB_WIN words
  // read at once per round (one memory latency per LB_WIN tiles walked)
  int64_t excl = 0;
  if (tile > 0) {
    int j = tile - 1, polls = 0;
    bool done = false;
    while (!done && j >= 0) {
      uint64_t v[LB_WIN];
#pragma unroll
      for (int q = 0; q < LB_WIN; ++q) v[q] = j - q >= 0 ? lb_load(&lb[(int64_t)(j - q) * 256 + d]) : LB_INCL;
      int used = 0;
#pragma unroll
      for (int q = 0; q < LB_WIN; ++q) {
        if (done || used < q) continue;   // stop at the first word not yet published
        if (v[q] & LB_INCL) {
          excl += (int64_t)(v[q] & LB_COUNT);
          done = true;
        } else if (v[q] & LB_LOCAL) {
          excl += (int64_t)(v[q] & LB_COUNT);
          used = q + 1;
        }
      }
      j -= used;
      if (done) break;
      if (used > 0) {
        polls = 0;
      } else {
        if (++polls > LB_POLLS) {   // the earlier tile never published: give up
          atomicOr(err, 8);
          break;
        }
        if (polls > 32) __nanosleep(64);
      }
    }
    lb_store(&lb[(int64_t)tile * 256 + d], LB_INCL | (uint64_t)(excl + run));
  }
  goff[d] = (int)(dbase + excl);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_IPT; ++r) {
    int64_t idx = base + r * 32 + lane;
    if (idx < n) {
      int dd = (int)((key[r] >> shift) & 255u);
      int tp = dstart[dd] + wcnt[w][dd] + loc[r];   // rank inside the tile
      tk[tp] = key[r];
      tv[tp] = val[r];
    }
  }
  __syncthreads();
  for (int tp = threadIdx.x; tp < tot; tp += RS_TH) {
    const uint32_t k = tk[tp];
    const int dd = (int)((k >> shift) & 255u);
    const int64_t pos = (int64_t)goff[dd] + (tp - dstart[dd]);
    if (pos >= 0 && pos < n) {   // always true unless a look-back gave up
      kout[pos] = k;
      vout[pos] = tv[tp];
    }
  }
}

}  // namespace

size_t scan_scratch_bytes(int64_t n) {
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  return (size_t)(nb + 1) * sizeof(int);
}

cudaError_t exclusive_scan(const int *in, int *out, int64_t n, void *scratch, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n <= SCAN_SINGLE_MAX) {   // one launch for small arrays
    k_scan_single<<<1, 1024, 0, s>>>(in, out, n);
    return cudaGetLastError();
  }
  int nb = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
  int *sums = (int *)scratch;
  k_scan_reduce<<<nb, SCAN_TH, 0, s>>>(in, n, sums);
  k_scan_sums<<<1, 1024, 0, s>>>(sums, nb);
  k_scan_tile<<<nb, SCAN_TH, 0, s>>>(in, out, n, sums);
  return cudaGetLastError();
}

int exclusive_scan_launches(int64_t n) {
  return n <= 0 ? 0 : (n <= SCAN_SINGLE_MAX ? 1 : 3);
}

size_t radix_sort_scratch_bytes(int64_t n) {
  const int64_t nb = (std::max<int64_t>(n, 1) + RS_TILE - 1) / RS_TILE;
  return RS_LB_OFF + (size_t)4 * nb * 256 * sizeof(uint64_t) + 256;
}

int radix_sort_launches(int64_t n, int bits) {
  return n <= 1 || bits <= 0 ? 0 : 1 + std::min(4, (bits + 7) / 8);
}

cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tmp_k, uint32_t *tmp_v,
                             int64_t n, int bits, void *scratch, cudaStream_t s, int *err) {
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int nb = (int)((n + RS_TILE - 1) / RS_TILE);
  const int passes = std::min(4, (bits + 7) / 8);
  char *sc = (char *)scratch;
  int *hist = (int *)(sc + RS_HIST_OFF);
  int *ctr = (int *)(sc + RS_CTR_OFF);
  uint64_t *lb = (uint64_t *)(sc + RS_LB_OFF);
  if (!err) err = ctr + 4;   // a word of the scratch: a give-up is then not reported
  // digit totals, tile counters and the scratch's own error word
  cudaError_t e = cudaMemsetAsync(sc, 0, RS_LB_OFF, s);
  if (e != cudaSuccess) return e;
  k_radix_hist<<<nb, RS_TH, 0, s>>>(keys, n, passes, hist, lb, nb);
  uint32_t *ka = keys, *va = vals, *kb = tmp_k, *vb = tmp_v;
  for (int ps = 0; ps < passes; ++ps) {
    k_radix_onesweep<<<nb, RS_TH, 0, s>>>(ka, va, kb, vb, n, 8 * ps, hist + 256 * ps,
                                          lb + (int64_t)ps * nb * 256, ctr + ps, err);
    uint32_t *t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  if (ka != keys) {
    e = cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace fmm2d
