// batched_tile2.cu -- the batched solver kernel for CTA tile 2 (64 x 32
// quaternion entries), compiled in its own translation unit.
#define QP_BATCHED_TILE 2
#define QP_TILE_RM 4
#define QP_TILE_RN 2
#define QP_TILE_MINB 1
#define QP_TILE_LAUNCH batched_launch_t2
#define QP_TILE_OCCUPANCY batched_occupancy_t2
#include "batched_impl.cuh"
