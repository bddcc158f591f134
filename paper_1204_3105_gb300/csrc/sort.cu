// sort.cu - device exclusive scan and stable LSD radix sort of (key, value)
// pairs, used to order points by leaf key (Sec. 4: Morton / GBT indexing
// orders cells in memory) and to compact the occupied cells.
//
// Radix sort: 8-bit digits, three kernels per pass - per-tile digit
// histogram, exclusive scan of the digit-major count table, and a stable
// scatter in which each warp ranks its 32 keys per round with
// __match_any_sync and the warps of a tile are ordered by a scan of their
// per-digit counts.  Input order is kept among equal keys.
#include "plan.h"

namespace fmm2d {

namespace {

constexpr int SCAN_TH = 256, SCAN_IPT = 16, SCAN_TILE = SCAN_TH * SCAN_IPT;
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
// 1024 threads x 8 items with a running carry.  Used for small arrays.
__global__ void __launch_bounds__(1024) k_scan_single(const int *__restrict__ in,
                                                      int *__restrict__ out, int64_t n) {
  __shared__ int sm[33];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  constexpr int IPT = 8;
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

__global__ void k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                             int *__restrict__ counts, int nblocks) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = 0; i < RS_IPT; ++i) {
    int64_t idx = base + (int64_t)i * RS_TH + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: every element's rank inside the tile in
// (digit, input order) order, the tile reordered in shared memory by that
// rank, then written out run by run so that consecutive threads store to
// consecutive addresses of each digit's destination range.
__global__ void __launch_bounds__(RS_TH)
k_radix_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
                const int *__restrict__ offs, int nblocks) {
  __shared__ int wcnt[RS_WARPS][257];
  __shared__ int goff[256], dstart[256];
  __shared__ int sm_scan[33];
  __shared__ uint32_t tk[RS_TILE], tv[RS_TILE];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * 257; i += RS_TH) (&wcnt[0][0])[i] = 0;
  goff[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
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
  int tot;
  {  // exclusive scan over warps, per digit; then over digits
    int d = threadIdx.x, run = 0;
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      int t = wcnt[ww][d];
      wcnt[ww][d] = run;
      run += t;
    }
    int ex;
    tot = block_excl_scan(run, ex, sm_scan);
    dstart[d] = ex;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_IPT; ++r) {
    int64_t idx = base + r * 32 + lane;
    if (idx < n) {
      int d = (int)((key[r] >> shift) & 255u);
      int tp = dstart[d] + wcnt[w][d] + loc[r];   // rank inside the tile
      tk[tp] = key[r];
      tv[tp] = val[r];
    }
  }
  __syncthreads();
  for (int tp = threadIdx.x; tp < tot; tp += RS_TH) {
    const uint32_t k = tk[tp];
    const int d = (int)((k >> shift) & 255u);
    const int64_t pos = (int64_t)goff[d] + (tp - dstart[d]);
    kout[pos] = k;
    vout[pos] = tv[tp];
  }
}

}  // namespace

size_t scan_scratch_bytes(int64_t n) {
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  return (size_t)(nb + 1) * sizeof(int);
}

cudaError_t exclusive_scan(const int *in, int *out, int64_t n, void *scratch, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n <= 8192) {   // one launch for small arrays
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

size_t radix_sort_scratch_bytes(int64_t n) {
  int64_t nb = (n + RS_TILE - 1) / RS_TILE;
  int64_t cnt = 256 * nb;
  return (size_t)cnt * sizeof(int) + scan_scratch_bytes(cnt) + 256;
}

cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tmp_k, uint32_t *tmp_v,
                             int64_t n, int bits, void *scratch, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int nb = (int)((n + RS_TILE - 1) / RS_TILE);
  int *counts = (int *)scratch;
  void *scan_scr = (char *)scratch + (((size_t)256 * nb * sizeof(int) + 255) & ~(size_t)255);
  uint32_t *ka = keys, *va = vals, *kb = tmp_k, *vb = tmp_v;
  const int passes = (bits + 7) / 8;
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 8 * ps;
    k_radix_hist<<<nb, RS_TH, 0, s>>>(ka, n, shift, counts, nb);
    cudaError_t e = exclusive_scan(counts, counts, (int64_t)256 * nb, scan_scr, s);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<nb, RS_TH, 0, s>>>(ka, va, kb, vb, n, shift, counts, nb);
    uint32_t *t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  if (ka != keys) {
    cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  }
  return cudaGetLastError();
}

}  // namespace fmm2d
