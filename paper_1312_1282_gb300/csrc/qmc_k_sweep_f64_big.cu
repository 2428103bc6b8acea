// Sweep kernels, double, threads per walker 256/512/1024.
#define QMC_T double
#define QMC_NAME launch_sweep_f64_big
#define QMC_TPW_A 256
#define QMC_TPW_B 512
#define QMC_TPW_C 1024
#define QMC_OCC_NAME occupancy_sweep_f64_big
#include "qmc_k_sweep.inc"
