// Apply kernels for degree 1 (k = 2 points per direction).
#include "dg_apply.cuh"
DG_DEFINE_APPLY_LAUNCHER(2)
