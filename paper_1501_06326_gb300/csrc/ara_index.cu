// Event-major index of a resident YET: for each catalogue event, its
// occurrences (trial, event index in the trial), in trial order.  Built once
// per YET (ara_build_yet_index); batched passes then reach a layer's hit
// events through its ELTs' events instead of streaming every trial's events
// (Section 2.1's lookup, taken from the ELT side).
#include <cuda_runtime.h>

#include <cstdint>

#include "ara_batch.h"

namespace ara {

namespace {

// key = event id, value = (trial << 32) | event index: one warp per trial
__global__ void k_yet_pairs(const int64_t* __restrict__ off, const int32_t* __restrict__ ids, int64_t n_trials,
                            unsigned long long* keys, int64_t* vals) {
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5); t < n_trials;
       t += warps) {
    const int64_t a = off[t], b = off[t + 1];
    for (int64_t i = a + lane; i < b; i += 32) {
      keys[i] = static_cast<unsigned long long>(static_cast<uint32_t>(ids[i]));
      vals[i] = (t << 32) | (i - a);
    }
  }
}

__global__ void k_fill_u32(uint32_t* a, int64_t n, uint32_t v) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) a[i] = v;
}

// ev_off[e] = the first sorted position of event e (an event without
// occurrences takes the next event's start; events past the last key keep n)
__global__ void k_event_starts(const unsigned long long* __restrict__ keys, int64_t n, uint32_t* ev_off) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int64_t cur = static_cast<int64_t>(keys[i]);
    const int64_t prev = i > 0 ? static_cast<int64_t>(keys[i - 1]) : -1;
    for (int64_t e = prev + 1; e <= cur; ++e) ev_off[e] = static_cast<uint32_t>(i);
  }
}

// ev_grid[e * (cells + 1) + k] = the first of event e's occurrences with
// trial >= k << grid_shift, by binary search within e's range
__global__ void k_event_grid(const unsigned long long* __restrict__ occ, const uint32_t* __restrict__ ev_off,
                             int64_t n_entries, int64_t cells, int grid_shift, uint32_t* ev_grid) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_entries; i += stride) {
    const int64_t e = i / (cells + 1), k = i - e * (cells + 1);
    const int64_t key = k << grid_shift;
    uint32_t lo = ev_off[e], hi = ev_off[e + 1];
    while (lo < hi) {
      const uint32_t mid = lo + (hi - lo) / 2u;
      if (static_cast<int64_t>(occ[mid] >> 32) < key) lo = mid + 1u;
      else hi = mid;
    }
    ev_grid[i] = lo;
  }
}

// ---- the bucket build: occurrences counted, placed and sorted per (event, grid cell)

// cnt[e * cells1 + (t >> grid_shift)] += 1 for each event e of trial t: a warp per trial
__global__ void k_count_cells(const int64_t* __restrict__ off, const int32_t* __restrict__ ids, int64_t n_trials,
                              int64_t cells1, int grid_shift, uint32_t* cnt) {
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5); t < n_trials;
       t += warps) {
    const int64_t a = off[t], b = off[t + 1], c = t >> grid_shift;
    for (int64_t i = a + lane; i < b; i += 32)
      atomicAdd(cnt + static_cast<int64_t>(ids[i]) * cells1 + c, 1u);
  }
}

__global__ void k_max_u32(const uint32_t* __restrict__ a, int64_t n, uint32_t* out) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  uint32_t m = 0u;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) m = max(m, a[i]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31u) == 0u && m) atomicMax(out, m);
}

// Each occurrence of an event in [e_lo, e_hi) to a slot of its (event, cell)
// bucket, claimed with an atomic add (the order within a bucket is the claims'
// order, then sorted).  The trials go in order, so each event of the range has
// one partly written line at a time; a range of 2^18 events keeps fewer of them
// in L2 at once (paper-1m: 39 ms a build against 42 ms at 2^19 events, 51 ms at
// 2^20, 84 ms in one pass, 49 ms at 2^17 with its 16 reads of the ids).
__global__ void k_scatter_cells(const int64_t* __restrict__ off, const int32_t* __restrict__ ids, int64_t n_trials,
                                int64_t cells1, int grid_shift, int32_t e_lo, int32_t e_hi,
                                const uint32_t* __restrict__ ev_grid, uint32_t* __restrict__ cur,
                                unsigned long long* __restrict__ occ) {
  constexpr int kU = 8;  // a lane's claims in flight before its stores
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5); t < n_trials;
       t += warps) {
    const int64_t a = off[t], b = off[t + 1], c = t >> grid_shift;
    for (int64_t i0 = a + lane; i0 < b; i0 += 32 * kU) {
      int64_t cell[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t i = i0 + 32 * u;
        const int32_t e = i < b ? ids[i] : -1;
        cell[u] = (e >= e_lo && e < e_hi) ? static_cast<int64_t>(e) * cells1 + c : -1;
      }
      uint32_t slot[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (cell[u] >= 0) slot[u] = ev_grid[cell[u]] + atomicAdd(cur + cell[u], 1u);
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (cell[u] >= 0)
          occ[slot[u]] = (static_cast<unsigned long long>(t) << 32) | static_cast<unsigned long long>(i0 + 32 * u - a);
    }
  }
}

// Each bucket in ascending (trial, event index) order: a thread per bucket, an
// insertion sort (the claims come nearly in trial order, as the warps take the
// trials in order, so few elements move)
__global__ void k_sort_cells(const uint32_t* __restrict__ ev_grid, int64_t n_buckets, unsigned long long* occ) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t bk = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; bk < n_buckets; bk += stride) {
    const uint32_t lo = ev_grid[bk], hi = ev_grid[bk + 1];
    if (hi - lo < 2u) continue;
    unsigned long long prev = occ[lo];
    for (uint32_t i = lo + 1u; i < hi; ++i) {
      const unsigned long long v = occ[i];
      if (v >= prev) {
        prev = v;
        continue;
      }
      uint32_t j = i;  // v goes below position i: shift the larger ones up
      do {
        occ[j] = occ[j - 1u];
        --j;
      } while (j > lo && occ[j - 1u] > v);
      occ[j] = v;
    }
  }
}

constexpr int64_t kScatterEvents = int64_t{1} << 18;  // events a scatter pass places

int grid_of(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return static_cast<int>(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

}  // namespace

int64_t yet_grid_cells(int64_t n_trials, int grid_shift) {
  return n_trials > 0 ? ((n_trials - 1) >> grid_shift) + 1 : 0;
}

size_t yet_bucket_scratch_bytes(int32_t catalogue, int64_t cells) {
  const int64_t n = static_cast<int64_t>(catalogue) * (cells + 1);
  return sizeof(uint32_t) * (static_cast<size_t>(n) + scan_tmp_words(n) + 64);
}

cudaError_t yet_index_count(const int64_t* off, const int32_t* ids, int64_t n_trials, int32_t catalogue, int grid_shift,
                            uint32_t* ev_grid, void* scratch, cudaStream_t s, int* n_launch) {
  const int64_t cells1 = yet_grid_cells(n_trials, grid_shift) + 1;
  const int64_t n = static_cast<int64_t>(catalogue) * cells1;
  uint32_t* cnt = static_cast<uint32_t*>(scratch);
  uint32_t* d_max = cnt + n;
  uint32_t* tmp = d_max + 32;
  cudaError_t err = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (static_cast<size_t>(n) + 32), s);
  if (err != cudaSuccess) return err;
  if (n_trials > 0) {
    k_count_cells<<<grid_of(n_trials * 32, 256), 256, 0, s>>>(off, ids, n_trials, cells1, grid_shift, cnt);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (n_launch) ++*n_launch;
  }
  k_max_u32<<<grid_of(n, 256), 256, 0, s>>>(cnt, n, d_max);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (n_launch) ++*n_launch;
  return scan_exclusive_u32(cnt, ev_grid, n, tmp, s, n_launch);
}

const uint32_t* yet_index_max_bucket(const void* scratch, int32_t catalogue, int64_t cells) {
  return static_cast<const uint32_t*>(scratch) + static_cast<int64_t>(catalogue) * (cells + 1);
}

cudaError_t yet_index_fill(const int64_t* off, const int32_t* ids, int64_t n_trials, int32_t catalogue, int grid_shift,
                           const uint32_t* ev_grid, unsigned long long* occ, void* scratch, cudaStream_t s,
                           int* n_launch) {
  const int64_t cells1 = yet_grid_cells(n_trials, grid_shift) + 1;
  const int64_t n = static_cast<int64_t>(catalogue) * cells1;
  uint32_t* cur = static_cast<uint32_t*>(scratch);
  cudaError_t err = cudaMemsetAsync(cur, 0, sizeof(uint32_t) * static_cast<size_t>(n), s);
  if (err != cudaSuccess || n_trials <= 0) return err;
  int launched = 1;
  for (int64_t e_lo = 0; e_lo < catalogue; e_lo += kScatterEvents, ++launched) {
    const int32_t e_hi = static_cast<int32_t>(e_lo + kScatterEvents < catalogue ? e_lo + kScatterEvents : catalogue);
    k_scatter_cells<<<grid_of(n_trials * 32, 256), 256, 0, s>>>(off, ids, n_trials, cells1, grid_shift,
                                                               static_cast<int32_t>(e_lo), e_hi, ev_grid, cur, occ);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  k_sort_cells<<<grid_of(n, 256), 256, 0, s>>>(ev_grid, n, occ);
  if (n_launch) *n_launch += launched;
  return cudaGetLastError();
}

size_t yet_index_scratch_bytes(int64_t n_events, int32_t catalogue) {
  return sizeof(unsigned long long) * static_cast<size_t>(n_events) + sort_pairs_scratch_bytes(n_events) +
         sizeof(uint32_t) * (static_cast<size_t>(catalogue) + 2) + 512;
}

cudaError_t build_yet_index(const int64_t* off, const int32_t* ids, int64_t n_trials, int64_t n_events,
                            int32_t catalogue, int grid_shift, unsigned long long* occ, uint32_t* ev_grid,
                            void* scratch, cudaStream_t s, int* n_launch) {
  unsigned long long* keys = static_cast<unsigned long long*>(scratch);
  uint32_t* ev_off = reinterpret_cast<uint32_t*>(keys + n_events);  // [catalogue + 1]
  void* sort_scratch = reinterpret_cast<char*>(scratch) + sizeof(unsigned long long) * static_cast<size_t>(n_events) +
                       ((sizeof(uint32_t) * (static_cast<size_t>(catalogue) + 2) + 255) & ~size_t{255});
  const int64_t cells = yet_grid_cells(n_trials, grid_shift);
  const int64_t n_entries = static_cast<int64_t>(catalogue) * (cells + 1);
  k_fill_u32<<<grid_of(static_cast<int64_t>(catalogue) + 1, 256), 256, 0, s>>>(ev_off, static_cast<int64_t>(catalogue) + 1,
                                                                              static_cast<uint32_t>(n_events));
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  int launched = 1;
  if (n_events > 0) {
    k_yet_pairs<<<grid_of(n_trials * 32, 256), 256, 0, s>>>(off, ids, n_trials, keys, reinterpret_cast<int64_t*>(occ));
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    int key_bits = 1;
    while (key_bits < 31 && (1ll << key_bits) < static_cast<int64_t>(catalogue)) ++key_bits;
    if ((err = sort_pairs_ascending(keys, reinterpret_cast<int64_t*>(occ), n_events, key_bits, sort_scratch, s,
                                    n_launch)) != cudaSuccess)
      return err;
    k_event_starts<<<grid_of(n_events, 256), 256, 0, s>>>(keys, n_events, ev_off);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    launched += 2;
  }
  if (n_entries > 0) {
    k_event_grid<<<grid_of(n_entries, 256), 256, 0, s>>>(occ, ev_off, n_entries, cells, grid_shift, ev_grid);
    ++launched;
  }
  if (n_launch) *n_launch += launched;
  return cudaGetLastError();
}

}  // namespace ara
