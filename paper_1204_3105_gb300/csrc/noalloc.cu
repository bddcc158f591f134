// noalloc.cu - fmm2d_keys_sort_noalloc: leaf keys and their stable sort for
// callers that cannot allocate GPU memory.
//
// Some callers cannot call cudaMalloc at the point where they need the keys:
// code running inside a memory pool they do not own, inside a stream-ordered
// region that must not synchronise on the allocator, or under a framework
// that forbids allocations outside its own arena.  This entry point does the
// same work as the keying and sorting steps of fmm2d_build, but its sort
// temporaries live in the file-scope device array below, whose address is
// taken once per device with cudaGetSymbolAddress.  Every GPU that loads the
// library holds the array (kScratchBytes, about 8.5 MiB) until the process
// exits.  All calls share it: calls whose GPU work overlaps (on different
// streams or threads) race on it and must be serialised by the caller.
#include <mutex>

#include "plan.h"

namespace fmm2d {
namespace {

constexpr int64_t kMaxPoints = 1 << 20;
constexpr size_t kTmpKeyOff = 0;
constexpr size_t kTmpValOff = kTmpKeyOff + 4 * (size_t)kMaxPoints;
constexpr size_t kSortOff = kTmpValOff + 4 * (size_t)kMaxPoints;
constexpr size_t kSortBytes = 2304 * 1024;
constexpr size_t kErrOff = kSortOff + kSortBytes;
constexpr size_t kScratchBytes = kErrOff + 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Clears the domain-error word of the scratch array (device code names the
// array directly).
__global__ void k_noalloc_clear_err() {
  if (threadIdx.x == 0) *reinterpret_cast<int *>(g_noalloc_scratch + kErrOff) = 0;
}

std::mutex g_mu;
void *g_dev_ptr[kMaxDevices] = {nullptr};

void set_msg(char *buf, size_t cap, const char *msg) {
  if (!buf || cap == 0) return;
  size_t i = 0;
  for (; i + 1 < cap && msg[i]; ++i) buf[i] = msg[i];
  buf[i] = 0;
}

}  // namespace
}  // namespace fmm2d

using namespace fmm2d;

extern "C" fmm2d_status fmm2d_keys_sort_noalloc(int tiling, int levels, double leaf_scale,
                                                const double *domain, const void *xy_dev,
                                                int64_t n, unsigned flags,
                                                uint32_t *keys_sorted_dev, uint32_t *perm_dev,
                                                void *stream, char *err_buf, size_t err_cap) {
  set_msg(err_buf, err_cap, "");
  if (tiling < 0 || tiling > 2) {
    set_msg(err_buf, err_cap, "unknown tiling");
    return FMM2D_EINVAL;
  }
  const int max_l = tiling == FMM2D_SEPT ? 9 : 12;
  if (levels < 1 || levels > max_l) {
    set_msg(err_buf, err_cap, "levels out of range (1..12, septree 1..9)");
    return FMM2D_EINVAL;
  }
  if (n < 0 || n > kMaxPoints) {
    set_msg(err_buf, err_cap,
            "n exceeds the no-allocation maximum of 1048576 points (use fmm2d_build instead)");
    return FMM2D_EINVAL;
  }
  if (n > 0 && (!xy_dev || !keys_sorted_dev || !perm_dev)) {
    set_msg(err_buf, err_cap, "null pointer");
    return FMM2D_EINVAL;
  }
  // The septree leaf radius belongs to the level count: it is computed here
  // (host work, cached per level; no device memory), as fmm2d_build does.  A
  // caller-given value must be that one, or the keys would silently differ.
  const double sept_r = tiling == FMM2D_SEPT ? sept_leaf_r(levels) : 0.0;
  if (tiling == FMM2D_SEPT && leaf_scale != 0.0 && leaf_scale != sept_r) {
    set_msg(err_buf, err_cap,
            "leaf_scale is not the septree leaf radius of this level count (pass 0)");
    return FMM2D_EINVAL;
  }
  const double S = domain ? domain[2] : 1.0;
  if (!(S > 0.0)) {
    set_msg(err_buf, err_cap, "domain size must be positive");
    return FMM2D_EINVAL;
  }
  const int bits = tiling == FMM2D_SEPT ? (int)ceil(levels * 2.807354922057604) : 2 * levels;
  if (radix_sort_scratch_bytes(kMaxPoints) > kSortBytes) {
    set_msg(err_buf, err_cap, "internal: sort scratch region too small");
    return FMM2D_EINVAL;
  }
  // Once per device, with that device current: the device address of the
  // scratch array (in host code its name is only a host-side stand-in).
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_msg(err_buf, err_cap, "cudaGetDevice failed or device ordinal too large");
    return FMM2D_ECUDA;
  }
  unsigned char *base;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_msg(err_buf, err_cap, "cudaGetSymbolAddress of the scratch array failed");
        return FMM2D_ECUDA;
      }
      g_dev_ptr[dev] = p;
    }
    base = (unsigned char *)g_dev_ptr[dev];
  }
  if (n == 0) return FMM2D_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Geo g;
  g.tiling = tiling;
  g.L = levels;
  g.b = tiling == FMM2D_SEPT ? 7 : 4;
  g.x0 = domain ? domain[0] : 0.0;
  g.y0 = domain ? domain[1] : 0.0;
  g.S = S;
  if (tiling == FMM2D_QUAD) g.leaf_scale = ldexp(1.0, -levels);
  else if (tiling == FMM2D_TRI) g.leaf_scale = tri_rho0();
  else g.leaf_scale = sept_r;
  int *err = (int *)(base + kErrOff);
  k_noalloc_clear_err<<<1, 32, 0, s>>>();
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = launch_keys(g, xy_dev, (flags & FMM2D_IN_F32) != 0, n, keys_sorted_dev, perm_dev, err, s);
  if (e == cudaSuccess)
    e = radix_sort_pairs(keys_sorted_dev, perm_dev, (uint32_t *)(base + kTmpKeyOff),
                         (uint32_t *)(base + kTmpValOff), n, bits, base + kSortOff, s, err);
  int err_h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err_h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_msg(err_buf, err_cap, cudaGetErrorString(e));
    return FMM2D_ECUDA;
  }
  if (err_h & 8) {
    set_msg(err_buf, err_cap, "a bounded wait of the radix sort gave up");
    return FMM2D_ETIMEOUT;
  }
  if (err_h) {
    set_msg(err_buf, err_cap, "a point lies outside the domain square or root cell");
    return FMM2D_EDOMAIN;
  }
  return FMM2D_OK;
}
