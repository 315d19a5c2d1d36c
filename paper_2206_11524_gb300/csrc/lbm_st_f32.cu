// lbm_st_f32.cu -- kernels and launchers for storage kind kF32.
#define HMCSC_ST kF32
#define HMCSC_SUF f32
#include "lbm_storage_impl.cuh"
