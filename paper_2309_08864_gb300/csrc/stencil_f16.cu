// stencil_f16.cu -- temporal-blocking kernels for f16 storage.
#define STORAGE_T __half
#define STORAGE_HAS_VARCOEF 0
#define STORAGE_HAS_FAST 1
#define LAUNCH_FN launch_stencil_f16
#define OCC_FN occupancy_stencil_f16
#include "stencil_inst.inc"
