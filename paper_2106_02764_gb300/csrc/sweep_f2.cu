// Sweep kernel variants: list OBTE_SWEEP_F2 of sweep_variants.h.
#include "sweep.cuh"
#include "sweep_variants.h"

OBTE_SWEEP_F2(OBTE_SWEEP_DEFINE)
