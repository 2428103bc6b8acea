// Sweep kernels, float, threads per walker 256/512/1024.
#define QMC_T float
#define QMC_NAME launch_sweep_f32_big
#define QMC_TPW_A 256
#define QMC_TPW_B 512
#define QMC_TPW_C 1024
#define QMC_OCC_NAME occupancy_sweep_f32_big
#include "qmc_k_sweep.inc"
