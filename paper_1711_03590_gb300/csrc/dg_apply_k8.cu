// Apply kernels for degree 7 (k = 8 points per direction).
#include "dg_apply.cuh"
DG_DEFINE_APPLY_LAUNCHER(8)
