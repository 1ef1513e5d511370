// gv_launch.h -- host-side launchers of the GraphVine kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "gv_internal.cuh"

namespace gv {

struct LaunchCfg {
    int num_sms;
    cudaStream_t stream;
};

// Group-by-source counting pass over a pair batch (all modes).
cudaError_t launch_count(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                         unsigned long long n, const LaunchCfg &lc);
// Rejected-pair count only (batches that cannot match any stored edge).
cudaError_t launch_count_rejects(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                 unsigned long long n, unsigned long long *rejected,
                                 const LaunchCfg &lc);
// Insert: plan (block demand, pop offsets), link (CBT), scatter (slots), finalize.
cudaError_t launch_insert_tail(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                               unsigned long long n, unsigned long long tcap,
                               unsigned long long *counts, const LaunchCfg &lc);
// Delete / query: plan, arena init, scatter into membership sets, mark,
// (delete) vscan + move, finalize; (query) result gather.
cudaError_t launch_member_tail(int mode, const GraphView &g, const uint32_t *src,
                               const uint32_t *dst, unsigned long long n, unsigned long long tcap,
                               unsigned long long *counts, uint8_t *qout, const LaunchCfg &lc);
// Vertex delete: mark dead, free own blocks, remove incoming edges, finalize.
cudaError_t launch_vertex_delete(const GraphView &g, const uint32_t *ids, uint32_t k,
                                 const LaunchCfg &lc);
// Vertices [from, to): alive, empty sentinel.
cudaError_t launch_init_vertices(const GraphView &g, uint32_t from, uint32_t to,
                                 const LaunchCfg &lc);
// Dictionary doubling copy.
cudaError_t launch_copy_dictionary(uint4 *dst_sent, uint8_t *dst_alive, const uint4 *src_sent,
                                   const uint8_t *src_alive, uint32_t n, const LaunchCfg &lc);
// Edge queue initialisation: queue[i] = i.
cudaError_t launch_init_queue(uint32_t *queue, unsigned long long P, const LaunchCfg &lc);
// Neighbour lists: offsets (exclusive scan of degrees), then copy.
cudaError_t launch_neighbor_offsets(const GraphView &g, const uint32_t *vids, uint32_t n,
                                    unsigned long long *offsets, unsigned long long *partials,
                                    const LaunchCfg &lc);
cudaError_t launch_neighbor_copy(const GraphView &g, const uint32_t *vids, uint32_t n,
                                 const unsigned long long *offsets, uint32_t *nbrs,
                                 const LaunchCfg &lc);
cudaError_t launch_degrees(const GraphView &g, uint32_t *deg, uint8_t *alive,
                           const LaunchCfg &lc);
cudaError_t launch_iota(uint32_t *out, uint32_t first, uint32_t k, const LaunchCfg &lc);
cudaError_t launch_validate(const GraphView &g, uint32_t *owner_bits,
                            unsigned long long *violations, const LaunchCfg &lc);

// Sizes shared with the host code.
constexpr int AGG_THREADS = 256;
constexpr int AGG_EPT = 8;
constexpr int AGG_TILE = AGG_THREADS * AGG_EPT;  // pairs per tile
constexpr int AGG_H = 4096;                      // shared hash slots per tile (>= 2 * tile)
constexpr int MASK_WORDS = 16;                   // survivor bits per item (512 slots)

}  // namespace gv
