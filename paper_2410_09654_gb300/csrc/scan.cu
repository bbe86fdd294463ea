// Device-wide exclusive prefix sums (tile scan per block, recursive scan of the tile
// totals, then a uniform add).  out[0..n] with out[n] = total.
#include "common.cuh"

namespace ps {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const T* __restrict__ in, uint64_t* __restrict__ out,
                                                            int64_t n, uint64_t* __restrict__ tile_sums) {
  __shared__ uint64_t warp_tot[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint64_t v[kScanItems];
  uint64_t sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    v[k] = (i < n) ? (uint64_t)in[i] : 0;
    sum += v[k];
  }
  // inclusive warp scan of per-thread sums
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint64_t t = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
    uint64_t ti = t;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint64_t u = __shfl_up_sync(0xffffffffu, ti, d);
      if (lane >= d) ti += u;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == kScanThreads / 32 - 1) {
      tile_sums[blockIdx.x] = ti;
      if (gridDim.x == 1) out[n] = ti;  // a single tile: its sum is the total
    }
  }
  __syncthreads();
  uint64_t run = warp_tot[warp] + incl - sum;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

// Adds each tile's offset; the last tile also writes the total, out[n].
__global__ void k_add_offsets(uint64_t* __restrict__ out, int64_t n, const uint64_t* __restrict__ offs,
                              const uint64_t* __restrict__ tile_sums) {
  int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  uint64_t o = offs[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k, i += kScanThreads)
    if (i < n) out[i] += o;
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = o + tile_sums[blockIdx.x];
}

template <class T>
int scan_impl(const T* in, uint64_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    PS_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
    return PS_OK;
  }
  int64_t tiles = ceil_div(n, kScanTile);
  Buf<uint64_t> sums;
  PS_TRY(sums.alloc((size_t)tiles + 1, s));
  PS_LAUNCH("k_tile_scan", s, k_tile_scan<T><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums.p));
  PS_CUDA(cudaGetLastError());
  if (tiles > 1) {
    Buf<uint64_t> offs;
    PS_TRY(offs.alloc((size_t)tiles + 1, s));
    PS_TRY(scan_impl<uint64_t>(sums.p, offs.p, tiles, s));
    PS_LAUNCH("k_add_offsets", s, k_add_offsets<<<(unsigned)tiles, kScanThreads, 0, s>>>(out, n, offs.p, sums.p));
    PS_CUDA(cudaGetLastError());
  }
  return PS_OK;
}

}  // namespace

int scan_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s) { return scan_impl<uint64_t>(in, out, n, s); }
int scan_u32_to_u64(const uint32_t* in, uint64_t* out, int64_t n, cudaStream_t s) {
  return scan_impl<uint32_t>(in, out, n, s);
}

}  // namespace ps
