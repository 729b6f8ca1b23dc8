// batched_tile1.cu -- the batched solver kernel for CTA tile 1 (32 x 32
// quaternion entries), compiled in its own translation unit.
#define QP_BATCHED_TILE 1
#define QP_TILE_RM 2
#define QP_TILE_RN 2
#define QP_TILE_MINB 2
#define QP_TILE_LAUNCH batched_launch_t1
#define QP_TILE_OCCUPANCY batched_occupancy_t1
#include "batched_impl.cuh"
