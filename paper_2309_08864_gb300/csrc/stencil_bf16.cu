// stencil_bf16.cu -- temporal-blocking kernels for bf16 storage.
#define STORAGE_T __nv_bfloat16
#define STORAGE_HAS_VARCOEF 0
#define STORAGE_HAS_FAST 1
#define LAUNCH_FN launch_stencil_bf16
#define OCC_FN occupancy_stencil_bf16
#include "stencil_inst.inc"
