// Ascending sort of the slice's candidate hosts (uint32 keys, unique).
//
// Least-significant-digit radix sort, 8-bit digits, 4 passes.  A tile is 4096 keys handled
// by 16 warps; each warp ranks its 256 keys in 8 rounds of 32 with __match_any_sync, which
// keeps the ranking stable (index order within a round, rounds in order, warps in order).
// Lists of up to one tile are sorted by a single block in shared memory (bitonic); longer
// lists by all blocks of the same cooperative launch.  The list length lives on the device,
// so the kernel reads it and takes the matching path.
#pragma once

#include "device.cuh"

namespace srla {


__device__ __forceinline__ uint32_t sort_len(const Ctl* ctl, uint32_t cmax) {
  return min(ctl->cat_count[ctl->T & 1], cmax);
}

__device__ __forceinline__ uint32_t* sort_list(const Ctl* ctl, uint32_t* l0, uint32_t* l1) {
  return (ctl->T & 1) ? l1 : l0;
}

// Rank the keys of one tile by the digit at `shift`.  On return, wcnt[w][d] holds the
// number of keys of digit d in warp w, and key[r], rank[r] the r-th key of this lane and
// its rank among the warp's keys with the same digit.
__device__ __forceinline__ void rank_tile(const uint32_t* src, uint32_t tile_base, uint32_t n, int shift,
                                          uint32_t (*wcnt)[kRadix], uint32_t key[8], uint32_t rank[8],
                                          bool valid[8]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < 8; r++) {
    const uint32_t idx = tile_base + (uint32_t)w * kKeysPerWarp + (uint32_t)r * 32u + (uint32_t)lane;
    const bool ok = idx < n;
    const uint32_t kk = ok ? src[idx] : 0u;
    const uint32_t d = (kk >> shift) & 0xFFu;
    const unsigned vm = __ballot_sync(kFull, ok);
    uint32_t rk = 0;
    if (ok) {
      const unsigned peers = __match_any_sync(vm, d);
      const uint32_t before = wcnt[w][d];
      __syncwarp(vm);
      rk = before + (uint32_t)__popc(peers & lt);
      if ((peers & lt) == 0) wcnt[w][d] = before + (uint32_t)__popc(peers);
    }
    __syncwarp();
    key[r] = kk;
    rank[r] = rk;
    valid[r] = ok;
  }
}

// Turn wcnt[w][d] into the exclusive prefix over warps; tot[d] receives the tile's count.
__device__ __forceinline__ void warp_prefix(uint32_t (*wcnt)[kRadix], uint32_t* tot) {
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
    uint32_t run = 0;
    for (int w = 0; w < kSortWarps; w++) {
      const uint32_t c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
    tot[d] = run;
  }
}

// A list of at most one tile: a bitonic sort in shared memory by one block.  The list is
// padded to a power of two with 0xFFFFFFFF; the keys are unique, so the first n of the
// sorted array are the sorted list even when a key equals the pad value.
__device__ __forceinline__ void bitonic_block(uint32_t* list, uint32_t n, uint32_t* smem) {
  uint32_t N = 2;
  while (N < n) N <<= 1;
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) smem[x] = x < n ? list[x] : 0xFFFFFFFFu;
  __syncthreads();
  // Pair t of a stage with distance j (a power of two) is (i, i + j), i = 2j*(t/j) + t%j.
  // For j <= 32 the 32 pairs of a warp stay inside one run of 64 elements from stage to
  // stage, so those stages only need the warp to agree (__syncwarp).
  for (uint32_t k = 2; k <= N; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t t = threadIdx.x; t < N / 2; t += blockDim.x) {
        const uint32_t i = ((t & ~(j - 1u)) << 1) | (t & (j - 1u));  // lower index of the pair
        const uint32_t l = i + j;
        const bool up = (i & k) == 0;
        const uint32_t a = smem[i], b = smem[l];
        if ((a > b) == up) {
          smem[i] = b;
          smem[l] = a;
        }
      }
      // the next stage is (k, j/2), or (2k, k) after j = 1
      if (j > 32 || (j == 1 && k > 32))
        __syncthreads();
      else
        __syncwarp();
    }
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) list[x] = smem[x];
}

// Lists longer than one tile: one cooperative kernel runs the four passes, each as three
// phases separated by grid barriers -- digit histogram of every tile (stored digit-major,
// hist[d * ntiles + t], so one exclusive scan yields every scatter offset), the scan by
// block 0, and the stable scatter of every tile.  The launch is cooperative, so all blocks
// are resident; the barrier still gives up after a bounded wait and flags SRLA_E_TIMEOUT.

constexpr unsigned kBarrierSpinLimit = 1u << 24;

// Returns false (in every thread of the block) if the wait gave up.
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, unsigned nblocks, unsigned spin_limit = kBarrierSpinLimit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &ctl->bar_gen;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&ctl->bar_count, 1u) == nblocks - 1u) {
      ctl->bar_count = 0;
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      unsigned it = 0;
      while (*gen == g) {
        if (++it > spin_limit) {
          atomicOr(&ctl->overflow, 4u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ void radix_hist_tiles(const uint32_t* src, uint32_t n, uint32_t ntiles, int shift,
                                                 uint32_t* hist, uint32_t* cnt) {
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    const uint32_t lo = t * kSortTile, hi = min(n, lo + kSortTile);
    for (uint32_t x = lo + threadIdx.x; x < hi; x += blockDim.x) atomicAdd(&cnt[(src[x] >> shift) & 0xFFu], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(size_t)d * ntiles + t] = cnt[d];
    __syncthreads();
  }
}

// Exclusive scan of hist[0 .. N) in place by one block (N a multiple of 8, hist 16-byte
// aligned, at most 31 warps; `part` holds 32 words).  The array goes by in chunks of 8
// consecutive entries per thread (two 16-byte loads, so a warp reads 1 KB contiguous), four
// chunks' loads in flight before any is used; each chunk is then scanned across the block
// and offset by the total of the chunks before it.  (A contiguous run of N / blockDim
// entries per thread made every warp load touch 32 lines, one round trip after another.)
__device__ __forceinline__ void radix_scan_block(uint32_t* hist, uint32_t N, uint32_t* part) {
  constexpr int kChunks = 4;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t nw = blockDim.x >> 5, chunk = blockDim.x * 8u;
  uint4* h4 = reinterpret_cast<uint4*>(hist);
  uint32_t carry = 0;  // total of the chunks already scanned, the same in every thread
  for (uint32_t base = 0; base < N; base += kChunks * chunk) {
    uint4 v[kChunks][2];
#pragma unroll
    for (int c = 0; c < kChunks; c++) {
      const uint32_t x = base + c * chunk + threadIdx.x * 8u;  // this thread's 8 entries
#pragma unroll
      for (int k = 0; k < 2; k++) v[c][k] = x < N ? h4[x / 4 + k] : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int c = 0; c < kChunks; c++) {
      const uint32_t x = base + c * chunk + threadIdx.x * 8u;
      const uint32_t s = v[c][0].x + v[c][0].y + v[c][0].z + v[c][0].w + v[c][1].x + v[c][1].y + v[c][1].z + v[c][1].w;
      uint32_t incl = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
      }
      if (lane == 31) part[w] = incl;
      __syncthreads();
      if (w == 0) {  // exclusive prefix of the warps' sums; lane 31 gets the chunk's total
        const uint32_t p = ((uint32_t)lane < nw) ? part[lane] : 0u;
        uint32_t pi = p;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t = __shfl_up_sync(kFull, pi, o);
          if (lane >= o) pi += t;
        }
        part[lane] = pi - p;
      }
      __syncthreads();
      uint32_t run = carry + part[w] + incl - s;
      if (x < N) {
#pragma unroll
        for (int k = 0; k < 2; k++) {
          uint4 o;
          o.x = run; run += v[c][k].x;
          o.y = run; run += v[c][k].y;
          o.z = run; run += v[c][k].z;
          o.w = run; run += v[c][k].w;
          h4[x / 4 + k] = o;
        }
      }
      carry += part[31];
      __syncthreads();  // part is rewritten by the next chunk
    }
  }
}

__device__ __forceinline__ void radix_scatter_tiles(const uint32_t* src, uint32_t* dst, uint32_t n, uint32_t ntiles,
                                                    int shift, const uint32_t* hist, uint32_t (*wcnt)[kRadix],
                                                    uint32_t* tot) {
  const int w = threadIdx.x >> 5;
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (int x = threadIdx.x; x < kSortWarps * kRadix; x += blockDim.x) (&wcnt[0][0])[x] = 0;
    __syncthreads();
    uint32_t key[8], rank[8];
    bool valid[8];
    rank_tile(src, t * kSortTile, n, shift, wcnt, key, rank, valid);
    __syncthreads();
    warp_prefix(wcnt, tot);
    // the tile's output offset of every digit, read once into shared memory (tot's tile
    // counts are not needed here)
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) tot[d] = hist[(size_t)d * ntiles + t];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; r++) {
      if (valid[r]) {
        const uint32_t d = (key[r] >> shift) & 0xFFu;
        dst[tot[d] + wcnt[w][d] + rank[r]] = key[r];
      }
    }
    __syncthreads();
  }
}

}  // namespace srla
