// batched_tile3.cu -- the batched solver kernel for CTA tile 3 (32 x 64
// quaternion entries), compiled in its own translation unit.
#define QP_BATCHED_TILE 3
#define QP_TILE_RM 2
#define QP_TILE_RN 4
#define QP_TILE_MINB 1
#define QP_TILE_LAUNCH batched_launch_t3
#define QP_TILE_OCCUPANCY batched_occupancy_t3
#include "batched_impl.cuh"
