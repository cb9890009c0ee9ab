// Apply kernels for degree 5 (k = 6 points per direction).
#include "dg_apply.cuh"
DG_DEFINE_APPLY_LAUNCHER(6)
