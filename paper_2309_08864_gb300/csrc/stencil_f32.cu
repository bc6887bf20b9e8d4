// stencil_f32.cu -- temporal-blocking kernels for f32 storage.
#define STORAGE_T float
#define STORAGE_HAS_VARCOEF 1
#define STORAGE_HAS_FAST 1
#define LAUNCH_FN launch_stencil_f32
#define OCC_FN occupancy_stencil_f32
#include "stencil_inst.inc"
