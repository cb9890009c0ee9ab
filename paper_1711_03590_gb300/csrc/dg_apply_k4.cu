// Apply kernels for degree 3 (k = 4 points per direction).
#include "dg_apply.cuh"
DG_DEFINE_APPLY_LAUNCHER(4)
