// Apply kernels for degree 6 (k = 7 points per direction).
#include "dg_apply.cuh"
DG_DEFINE_APPLY_LAUNCHER(7)
