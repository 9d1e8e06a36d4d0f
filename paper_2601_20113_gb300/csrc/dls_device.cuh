// Device helpers shared by the packing kernels (bit packing, block scans).
#pragma once

#include "dls_internal.cuh"

namespace dls {

// Word w of a bit stream whose element l (value val(l), width wdt) sits at bit l*wdt.
template <typename F>
__device__ __forceinline__ uint32_t compose_word(int64_t w, int wdt, int64_t count, F val) {
  const int64_t b0 = w * 32;
  int64_t l = b0 / wdt;
  uint32_t word = 0;
  for (; l < count; ++l) {
    const int64_t pos = l * wdt;
    if (pos >= b0 + 32) break;
    const uint32_t z = val(l);
    const int64_t sh = pos - b0;
    if (sh >= 0) word |= (uint32_t)((uint64_t)z << sh);
    else word |= (uint32_t)(z >> (-sh));
  }
  return word;
}

__device__ __forceinline__ void or_bits(uint32_t* words, uint64_t pos, uint32_t val, int width) {
  if (width == 0) return;
  const uint64_t wi = pos >> 5;
  const int sh = (int)(pos & 31);
  const uint64_t v = (uint64_t)val << sh;
  atomicOr(&words[wi], (uint32_t)v);
  if (sh + width > 32) atomicOr(&words[wi + 1], (uint32_t)(v >> 32));
}

// Block-wide exclusive scan of one int per thread (all threads must call);
// returns the exclusive prefix and writes the tile total to *total.
__device__ __forceinline__ int block_excl_scan(int v, int* sh_warp, int* total) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = lane < (int)(blockDim.x / 32) ? sh_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh_warp[lane] = s;
  }
  __syncthreads();
  const int excl = (warp > 0 ? sh_warp[warp - 1] : 0) + x - v;
  *total = sh_warp[blockDim.x / 32 - 1];
  __syncthreads();
  return excl;
}

}  // namespace dls
