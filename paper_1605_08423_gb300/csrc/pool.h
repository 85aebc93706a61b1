// pool.h -- handles carved from a caller-owned device block (library
// internal: the serving loop admits trajectories without cudaMalloc).
#pragma once
#include <cstddef>

#include <cuda_runtime.h>

#include "../../include/qmcmd.h"

namespace qmc {

// Alignment of every array carved from a block, and an upper bound on the
// arrays of one handle (qmc_footprint_bytes includes kPoolAllocs * kPoolAlign
// of slack, so a block of that size always holds the handle).
constexpr size_t kPoolAlign = 256;
constexpr size_t kPoolAllocs = 96;

// qmc_init with two differences: the handle's device arrays are carved from
// `block` (block_bytes >= qmc_footprint_bytes(p); block = nullptr: cudaMalloc
// as usual), and the handle works on `stream` (nullptr: a stream of its own).
// wait = false returns without waiting for the set-up copies and kernels on
// the stream (their errors surface at the next qmc_sync).  qmc_destroy frees
// nothing carved from a block; the block stays the caller's.
int init_handle(const qmc_params* p, const double* R, void* block, size_t block_bytes, cudaStream_t stream,
                bool wait, qmc_system** out);

}  // namespace qmc
