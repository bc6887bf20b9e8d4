// stencil_f64.cu -- temporal-blocking kernels for f64 storage.
#define STORAGE_T double
#define STORAGE_HAS_VARCOEF 1
#define STORAGE_HAS_FAST 0
#define LAUNCH_FN launch_stencil_f64
#define OCC_FN occupancy_stencil_f64
#include "stencil_inst.inc"
