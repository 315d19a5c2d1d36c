// lbm_st_bf16.cu -- kernels and launchers for storage kind kBF16.
#define HMCSC_ST kBF16
#define HMCSC_SUF bf16
#include "lbm_storage_impl.cuh"
