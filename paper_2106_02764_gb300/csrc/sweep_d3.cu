// Sweep kernel variants: list OBTE_SWEEP_D3 of sweep_variants.h.
#include "sweep.cuh"
#include "sweep_variants.h"

OBTE_SWEEP_D3(OBTE_SWEEP_DEFINE)
