// Work queue of the uneven batch (one persistent launch over many circuits).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace svk {

// One pass of one circuit.
struct BatchCP {
  uint64_t state_off;  // float2 offset of the circuit's state in the batch buffer
  uint32_t pass;       // index into the batch plan's pass array
  uint32_t prev;       // BatchCP index of the circuit's previous pass (kNoPrev if first)
  uint32_t tiles;      // tiles of this pass
  uint32_t circuit;
};
constexpr uint32_t kNoPrev = 0xFFFFFFFFu;

// One tile of one circuit-pass.  Items are dispensed in array order: all first passes,
// then all second passes, ...; an item waits only for its circuit's previous pass, which
// was dispensed earlier to a CTA that is already running, so the queue cannot deadlock.
struct BatchItem {
  uint32_t cp;
  uint32_t tile;
};

// Device words of one launch: [0] next item, [1] error flag, then one done counter per cp.
constexpr int kBatchHeader = 2;

// wait_ns: limit of one dependency wait (after which the error word is set and the CTA
// leaves); max_grid > 0 caps the number of CTAs.
cudaError_t launch_batch(float2 *states, const DevPlanView &plan, const BatchCP *cps, const BatchItem *items,
                         uint64_t n_items, unsigned int *words, int m, cudaStream_t st,
                         unsigned long long wait_ns = 5000000000ull, int max_grid = 0);
int batch_block_threads(int m);

// Per-circuit fp64 norm and sum |alpha|^4: chunk c covers [start, start + len) of circuit
// circ; partials (2 doubles per chunk) then one thread per circuit adds its chunks in order.
struct BatchChunk {
  uint64_t start;
  uint32_t len;
  uint32_t circuit;
};
cudaError_t launch_batch_stats(const float2 *states, const BatchChunk *chunks, int n_chunks, double *partials,
                               const int *chunk_begin, int n_circuits, double *stats, cudaStream_t st);

}  // namespace svk
