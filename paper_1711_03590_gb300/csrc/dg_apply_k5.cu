// Apply kernels for degree 4 (k = 5 points per direction).
#include "dg_apply.cuh"
DG_DEFINE_APPLY_LAUNCHER(5)
