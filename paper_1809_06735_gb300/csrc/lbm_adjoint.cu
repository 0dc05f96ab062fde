// Adjoint of the D2Q9 step (placeholder translation unit, filled below).
#include "lbm_internal.cuh"
