// Internal interface of the event-major YET index and the batched passes that
// read it (ara_index.cu, ara_batch.cu, ara_select.cu, ara_abi.cu).  Not part
// of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ara_internal.h"

namespace ara {

// --------------------------------------------------------------- sort
// Stable ascending sort of n (key, value) pairs by the low key_bits bits of the
// keys (8 bits a pass), in place; `scratch` holds sort_pairs_scratch_bytes(n).
size_t sort_pairs_scratch_bytes(int64_t n);
cudaError_t sort_pairs_ascending(unsigned long long* keys, int64_t* vals, int64_t n, int key_bits, void* scratch,
                                 cudaStream_t s, int* n_launch);

// --------------------------------------------------------------- batched PML/TVaR
// Several YLTs' PML/TVaR in one set of five launches per batch of up to 32
// jobs (a YLT and a group of up to four return periods), each job with its own
// grid and scratch, so that it gives the bits pml_tvar_device gives on its YLT.
// rps: host arrays, read during the call; pml/tvar: device arrays of n_rp.
// pool: the jobs' scratch, at least select_job_bytes(n, n_rp) for each YLT;
// jobs that do not fit together go in later batches that reuse the pool in
// stream order.  n >= 1 and 1 <= n_rp, else cudaErrorInvalidValue.
struct SelectSpec {
  const double* ylt;
  int64_t n;
  const double* rps;
  int32_t n_rp;
  double* pml;
  double* tvar;
};
size_t select_job_bytes(int64_t n, int n_rp);
cudaError_t pml_tvar_batch(const SelectSpec* specs, int n_specs, void* pool, size_t pool_bytes, cudaStream_t s,
                           int* n_launch);

// --------------------------------------------------------------- event-major YET index
// occ[i] = (trial << 32) | event index, grouped by event id and in trial order
// within an event.  ev_grid[e * (cells + 1) + k], k = 0..cells, is the first
// position of event e's occurrences whose trial is at least k << grid_shift
// (the end of e's occurrences where there is none): e's occurrences are
// occ[ev_grid[e * (cells + 1)], ev_grid[e * (cells + 1) + cells]), with
// cells = yet_grid_cells(n_trials, grid_shift).  n_events < 2^32.  `scratch`
// holds yet_index_scratch_bytes(n_events, catalogue).
int64_t yet_grid_cells(int64_t n_trials, int grid_shift);
// The bucket build.  yet_index_count counts each (event, grid cell)'s
// occurrences and scans the counts into ev_grid; the largest count is left in
// device memory at yet_index_max_bucket(scratch, ...).  yet_index_fill then
// places each occurrence in its bucket (an atomic slot claim) and sorts each
// bucket by one thread's insertion sort: fast while buckets are small.
// `scratch` holds yet_bucket_scratch_bytes(catalogue, cells) for both.
size_t yet_bucket_scratch_bytes(int32_t catalogue, int64_t cells);
cudaError_t yet_index_count(const int64_t* off, const int32_t* ids, int64_t n_trials, int32_t catalogue, int grid_shift,
                            uint32_t* ev_grid, void* scratch, cudaStream_t s, int* n_launch);
const uint32_t* yet_index_max_bucket(const void* scratch, int32_t catalogue, int64_t cells);
cudaError_t yet_index_fill(const int64_t* off, const int32_t* ids, int64_t n_trials, int32_t catalogue, int grid_shift,
                           const uint32_t* ev_grid, unsigned long long* occ, void* scratch, cudaStream_t s,
                           int* n_launch);
// The sort build (any bucket sizes): a stable radix sort of the YET's events
// by id, then the grid by a binary search per (event, cell).
size_t yet_index_scratch_bytes(int64_t n_events, int32_t catalogue);
cudaError_t build_yet_index(const int64_t* off, const int32_t* ids, int64_t n_trials, int64_t n_events,
                            int32_t catalogue, int grid_shift, unsigned long long* occ, uint32_t* ev_grid,
                            void* scratch, cudaStream_t s, int* n_launch);

// --------------------------------------------------------------- indexed batched pass
// The fourth work item of the batched losses (after kItemTile, kItemTrial and
// kItemDense): a warp per distinct event of the pass's ELT union, over the
// event's occurrences in [t_begin, t_end) from the index; each (occurrence,
// layer) adds the same fixed-point number as the other work items, into acc
// with a 64-bit atomic add.  No k_gather.
constexpr int kItemIndexed = 3;
struct IndexedParams {
  BatchParams b;                  // the pass
  const unsigned long long* occ;  // the index (build_yet_index)
  const uint32_t* ev_grid;
  int64_t grid_cells;
  int grid_shift;
  int slice_shift;                // the pass runs in slices [j << slice_shift, (j + 1) << slice_shift) of the
                                  // trials (clipped to the pass), every event over one slice before the next;
                                  // slice_shift >= grid_shift, so inner slice bounds are grid bounds
  const int32_t* u_event;         // [n_u] the union's distinct events, in pair order
  const uint32_t* u_first;        // [n_u + 1] each one's first pair; u_first[n_u] = the pair count
  const uint32_t* n_u;            // device: the number of distinct events
  unsigned long long* acc;        // [n_layers][t_end - t_begin] fixed-point sums (zeroed before)
  int64_t yet_trials;             // the YET's trials
  uint32_t* slice_queue;          // [indexed_slices(t_begin, t_end, slice_shift)] each slice's queue (zeroed before)
};
__host__ __device__ inline int64_t indexed_slices(int64_t t_begin, int64_t t_end, int slice_shift) {
  return t_end > t_begin ? ((t_end - 1) >> slice_shift) - (t_begin >> slice_shift) + 1 : 0;
}
// The union's distinct events from the pairs' event ids (pev, in pair order):
// flags and scan hold n_recs + 1 words, scan_tmp scan_tmp_words(n_recs); the
// count is left at scan[n_recs].
cudaError_t launch_union_events(const int32_t* pev, int64_t n_recs, uint32_t* flags, uint32_t* scan,
                                uint32_t* scan_tmp, int32_t* u_event, uint32_t* u_first, cudaStream_t s,
                                int* n_launch);
cudaError_t launch_losses_indexed(const IndexedParams& q, int grid, cudaStream_t s);
// The year losses from acc: each layer's trials [t_begin, layer_t_end).
cudaError_t launch_indexed_years(const IndexedParams& q, cudaStream_t s);
int losses_indexed_blocks_per_sm();

}  // namespace ara
