// Device-wide exclusive scan and stable LSD radix sort of (uint64 key, uint32 value)
// pairs. Used once per mesh by the pattern build (the index part of `sparse`,
// Section 3 of the paper): every element slot gets a 64-bit key row * n + col and
// the sort brings equal keys together, in ascending slot order within a key.
#include <stdio.h>

#include "fe_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

constexpr int SORT_WARPS = 8;
constexpr int SORT_THREADS = SORT_WARPS * 32;
constexpr int SORT_ROUNDS = 16;                      // keys per lane
constexpr int SORT_TILE = SORT_THREADS * SORT_ROUNDS;  // 4096 keys per block
constexpr int RADIX = 256;

// exclusive scan of a block tile; writes the tile total to block_sums[blockIdx.x]
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tile(const uint32_t* in, uint32_t* out,
                                                            int64_t n, uint32_t* block_sums) {
  __shared__ uint32_t warp_tot[SCAN_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    sum += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : 0u;
    uint32_t s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = s - t;  // exclusive warp offsets
    if (lane == 31 && block_sums) block_sums[blockIdx.x] = s;
  }
  __syncthreads();
  uint32_t run = warp_tot[warp] + x - sum;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

__global__ void k_scan_add(uint32_t* out, int64_t n, const uint32_t* block_off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += block_off[i / SCAN_TILE];
}

__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift) {
  return (uint32_t)(k >> shift) & (RADIX - 1);
}

__global__ void __launch_bounds__(SORT_THREADS) k_radix_hist(const uint64_t* keys, int64_t n,
                                                             int shift, uint32_t* hist,
                                                             int64_t ntiles) {
  __shared__ uint32_t cnt[RADIX];
  for (int i = threadIdx.x; i < RADIX; i += SORT_THREADS) cnt[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
  for (int i = threadIdx.x; i < SORT_TILE; i += SORT_THREADS) {
    const int64_t p = base + i;
    if (p < n) atomicAdd(&cnt[digit_of(keys[p], shift)], 1u);
  }
  __syncthreads();
  for (int dgt = threadIdx.x; dgt < RADIX; dgt += SORT_THREADS)
    hist[(int64_t)dgt * ntiles + blockIdx.x] = cnt[dgt];
}

// Stable scatter: within a tile, key order is (warp, round, lane), which is the
// input order; ranks come from per-warp digit counters and __match_any_sync.
__global__ void __launch_bounds__(SORT_THREADS) k_radix_scatter(
    const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ offsets,
    int64_t ntiles) {
  __shared__ uint32_t whist[SORT_WARPS][RADIX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < SORT_WARPS * RADIX; i += SORT_THREADS) (&whist[0][0])[i] = 0;
  const int64_t base = (int64_t)blockIdx.x * SORT_TILE + (int64_t)warp * (SORT_ROUNDS * 32) + lane;
  uint64_t k[SORT_ROUNDS];
  uint32_t v[SORT_ROUNDS];
#pragma unroll
  for (int r = 0; r < SORT_ROUNDS; ++r) {
    const int64_t p = base + r * 32;
    k[r] = (p < n) ? kin[p] : 0ull;
    v[r] = (p < n) ? vin[p] : 0u;
  }
  __syncthreads();
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < SORT_ROUNDS; ++r) {
    const bool valid = base + r * 32 < n;
    const uint32_t dg = valid ? digit_of(k[r], shift) : 0xFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, dg);
    if (valid && (peers & lt_mask) == 0) whist[warp][dg] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int dgt = threadIdx.x; dgt < RADIX; dgt += SORT_THREADS) {
    uint32_t run = offsets[(int64_t)dgt * ntiles + blockIdx.x];
    for (int w = 0; w < SORT_WARPS; ++w) {
      const uint32_t c = whist[w][dgt];
      whist[w][dgt] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < SORT_ROUNDS; ++r) {
    const bool valid = base + r * 32 < n;
    const uint32_t dg = valid ? digit_of(k[r], shift) : 0xFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, dg);
    uint32_t pos = 0;
    if (valid) pos = whist[warp][dg] + __popc(peers & lt_mask);
    __syncwarp();
    if (valid) {
      kout[pos] = k[r];
      vout[pos] = v[r];
      if ((peers & lt_mask) == 0) whist[warp][dg] += __popc(peers);
    }
    __syncwarp();
  }
}

}  // namespace

size_t fe_scan_tmp_size(int64_t n) {
  size_t total = 0;
  while (n > SCAN_TILE) {
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    total += (size_t)nb;
    n = nb;
  }
  return total + 1;
}

int fe_scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s) {
  if (n <= 0) return FE_OK;
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 1) {
    k_scan_tile<<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
  }
  uint32_t* sums = tmp;
  k_scan_tile<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums);
  FE_CUDA_TRY(cudaGetLastError());
  FE_TRY(fe_scan_exclusive(sums, sums, nb, tmp + nb, s));
  k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums);
  FE_CUDA_TRY(cudaGetLastError());
  return FE_OK;
}

size_t fe_sort_hist_size(int64_t n) {
  const int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
  return (size_t)RADIX * (size_t)(ntiles > 0 ? ntiles : 1);
}

int fe_radix_sort(int64_t n, int bits, fe_sort_buffers* b, uint64_t** keys, uint32_t** vals,
                  cudaStream_t s) {
  uint64_t* kin = b->k0;
  uint64_t* kout = b->k1;
  uint32_t* vin = b->v0;
  uint32_t* vout = b->v1;
  const int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
  if (n > 1) {
    for (int shift = 0; shift < bits; shift += 8) {
      k_radix_hist<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(kin, n, shift, b->hist, ntiles);
      FE_CUDA_TRY(cudaGetLastError());
      FE_TRY(fe_scan_exclusive(b->hist, b->hist, (int64_t)RADIX * ntiles, b->scan_tmp, s));
      k_radix_scatter<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(kin, vin, kout, vout, n, shift,
                                                                b->hist, ntiles);
      FE_CUDA_TRY(cudaGetLastError());
      uint64_t* tk = kin; kin = kout; kout = tk;
      uint32_t* tv = vin; vin = vout; vout = tv;
    }
  }
  *keys = kin;
  *vals = vin;
  return FE_OK;
}
