// Sweep kernel variants: list OBTE_SWEEP_S of sweep_variants.h.
#include "sweep.cuh"
#include "sweep_variants.h"

OBTE_SWEEP_S(OBTE_SWEEP_DEFINE)
