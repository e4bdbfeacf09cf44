// The candidate sort kernel of one link (device parts in sort_parts.cuh).
#pragma once

#include "sort_parts.cuh"

namespace srla {

// The slice's candidate sort: one cooperative launch whatever the list length.
__global__ void __launch_bounds__(kSortThreads) k_sort(Ctl* __restrict__ ctl, uint32_t* l0, uint32_t* l1,
                                                       uint32_t* tmp, uint32_t cmax, uint32_t* __restrict__ hist) {
  const uint32_t n = sort_len(ctl, cmax);
  if (n <= (uint32_t)kSortTile) {  // one block sorts in shared memory; the grid leaves together
    extern __shared__ uint32_t bsm[];
    if (blockIdx.x == 0 && n > 1) bitonic_block(sort_list(ctl, l0, l1), n, bsm);
    return;
  }
  __shared__ uint32_t wcnt[kSortWarps][kRadix];
  __shared__ uint32_t tot[kRadix];
  __shared__ uint32_t part[32];
  uint32_t* list = sort_list(ctl, l0, l1);
  const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
  for (int pass = 0; pass < 4; pass++) {
    const uint32_t* src = (pass & 1) ? tmp : list;
    uint32_t* dst = (pass & 1) ? list : tmp;
    radix_hist_tiles(src, n, ntiles, pass * 8, hist, tot);
    if (!grid_barrier(ctl, gridDim.x)) return;
    if (blockIdx.x == 0) radix_scan_block(hist, ntiles * kRadix, part);
    if (!grid_barrier(ctl, gridDim.x)) return;
    radix_scatter_tiles(src, dst, n, ntiles, pass * 8, hist, wcnt, tot);
    if (!grid_barrier(ctl, gridDim.x)) return;
  }
}

// Self-test of the bounded wait: two blocks meet at one grid barrier, but the last `absent`
// blocks never arrive, so the others give up after spin_limit polls and flag the timeout.
__global__ void k_wait_selftest(Ctl* ctl, unsigned absent, unsigned spin_limit) {
  if (blockIdx.x >= gridDim.x - absent) return;  // this block never joins
  grid_barrier(ctl, gridDim.x, spin_limit);
}

}  // namespace srla
