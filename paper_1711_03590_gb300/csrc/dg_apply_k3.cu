// Apply kernels for degree 2 (k = 3 points per direction).
#include "dg_apply.cuh"
DG_DEFINE_APPLY_LAUNCHER(3)
