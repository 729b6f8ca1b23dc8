// batched_tile4.cu -- the batched solver kernel for CTA tile 4 (64 x 64
// quaternion entries), compiled in its own translation unit.
#define QP_BATCHED_TILE 4
#define QP_TILE_RM 4
#define QP_TILE_RN 4
#define QP_TILE_MINB 1
#define QP_TILE_LAUNCH batched_launch_t4
#define QP_TILE_OCCUPANCY batched_occupancy_t4
#include "batched_impl.cuh"
