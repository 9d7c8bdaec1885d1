// 3D block-kernel variants (sweep3d_variants.h).
#include "sweep3d.cuh"
#include "sweep3d_variants.h"

OBTE_SWEEP3D_VARIANTS(OBTE_SWEEP3D_DEFINE)
