// Sweep kernels, double, threads per walker 32/64/128.
#define QMC_T double
#define QMC_NAME launch_sweep_f64_small
#define QMC_TPW_A 32
#define QMC_TPW_B 64
#define QMC_TPW_C 128
#define QMC_OCC_NAME occupancy_sweep_f64_small
#include "qmc_k_sweep.inc"
