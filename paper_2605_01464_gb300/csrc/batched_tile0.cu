// batched_tile0.cu -- the batched solver kernel for CTA tile 0 (16 x 16
// quaternion entries), compiled in its own translation unit.
#define QP_BATCHED_TILE 0
#define QP_TILE_RM 1
#define QP_TILE_RN 1
#define QP_TILE_MINB 2
#define QP_TILE_LAUNCH batched_launch_t0
#define QP_TILE_OCCUPANCY batched_occupancy_t0
#include "batched_impl.cuh"
