// K4, the tile sort, instantiated for 2 lanes per odd-even transposition
// group (tile_sort2.cuh), CTAs of 256 and 512 threads.
#include "tile_sort2.cuh"

namespace bsort {

cudaError_t launch_tile_sort2_g2(int cluster, int threads, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t supertiles,
                                 int max_grid, int max_width, uint64_t* keys, EmitOut eo, Meta* meta,
                                 uint64_t wait_limit, cudaStream_t st) {
  return tile_sort2_lanes<2>(cluster, threads, segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta, wait_limit,
                              st);
}

}  // namespace bsort
