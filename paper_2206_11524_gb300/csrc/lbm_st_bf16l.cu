// lbm_st_bf16l.cu -- kernels and launchers for storage kind kBF16L.
#define HMCSC_ST kBF16L
#define HMCSC_SUF bf16l
#include "lbm_storage_impl.cuh"
