// 2D warp-kernel variants with two-warp groups: list OBTE_SWEEP2D_W2 of sweep2d_variants.h.
#include "sweep2d.cuh"
#include "sweep2d_variants.h"

OBTE_SWEEP2D_W2(OBTE_SWEEP2D_W2_DEFINE)
