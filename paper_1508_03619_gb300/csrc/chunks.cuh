// chunks.cuh — heavy-row chunk lists, shared by the batch path (many graphs)
// and the personalized-PageRank engine (one graph).
//
// A row with more than `heavy` in-arcs is split into ceil(deg / chunk) chunks
// of consecutive arcs (all of `chunk` arcs but the last).  Chunks are listed
// graph after graph, row after row, so the chunks of one row are contiguous
// and `first` (the id of its first chunk) orders them.  The list is a
// run-time decision on the input graph and is rebuilt by every call that
// needs it (§2.3: no per-graph precomputed parameters).
#pragma once

#include "graph.cuh"

namespace gap {

struct ChunkDesc {
  int64_t a0;     // first arc of the chunk (index into the graph's in_idx)
  int64_t first;  // chunk id of the row's first chunk
  int32_t len;    // arcs in the chunk
  int32_t v;      // the row (vertex id within its graph)
  int32_t nch;    // chunks of the row
  int32_t graph;  // graph index (0 for a single graph)
};

// Row offsets of one graph, as the chunk builder needs them.
struct ChunkGraph {
  const int64_t* off;
  int64_t n;
};

// Upper bound of the chunk count of a graph with m arcs.
inline int64_t chunk_capacity(int64_t m, int heavy, int chunk) { return m / chunk + m / (heavy + 1) + 1; }

// Device scratch of the builder for `tiles` row tiles.
struct ChunkBuilder {
  Scratch tile_base;  // int64[ng + 1]: first tile of each graph (host-computed)
  Scratch tile_cnt;   // int64[tiles]: chunks per tile, then their exclusive scan
  int64_t tiles = 0;
};

constexpr int CHUNK_TILE_ROWS = 1024;

// List the chunks of `ng` graphs (device array `graphs`; host copy `hgraphs`
// for the tile layout) into desc[0 .. total) and zero ctr[0 .. total);
// chunk_base[i] (device, ng + 1 entries) receives the first chunk id of graph
// i and chunk_base[ng] the total.  `cap` is the capacity of desc / ctr
// (the sum of chunk_capacity over the graphs).  All work is on stream s.
gap_status build_chunks(ChunkBuilder* b, const ChunkGraph* graphs, const ChunkGraph* hgraphs, int ng, int heavy,
                        int chunk, ChunkDesc* desc, unsigned int* ctr, int64_t* chunk_base, cudaStream_t s);

}  // namespace gap
