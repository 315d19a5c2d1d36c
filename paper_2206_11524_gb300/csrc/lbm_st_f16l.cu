// lbm_st_f16l.cu -- kernels and launchers for storage kind kF16L.
#define HMCSC_ST kF16L
#define HMCSC_SUF f16l
#include "lbm_storage_impl.cuh"
