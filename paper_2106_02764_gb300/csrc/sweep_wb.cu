// 2D warp-kernel variants: list OBTE_SWEEP2D_WB of sweep2d_variants.h.
#include "sweep2d.cuh"
#include "sweep2d_variants.h"

OBTE_SWEEP2D_WB(OBTE_SWEEP2D_DEFINE)
