// lbm_st_f16.cu -- kernels and launchers for storage kind kF16.
#define HMCSC_ST kF16
#define HMCSC_SUF f16
#include "lbm_storage_impl.cuh"
