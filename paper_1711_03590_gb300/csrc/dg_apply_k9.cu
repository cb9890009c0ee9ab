// Apply kernels for degree 8 (k = 9 points per direction).
#include "dg_apply.cuh"
DG_DEFINE_APPLY_LAUNCHER(9)
