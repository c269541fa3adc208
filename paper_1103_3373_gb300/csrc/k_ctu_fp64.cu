// CTU kernels, fp64 form: PLM/PPM on primitive variables x Riemann solvers for N = 16.
#include "kernels.cuh"

void hyd_reg_ctu_fp64(hyd::KernelEntry* tab) { hyd::put_scheme<hyd::CTU, hyd::P_FP64, 16, false>(tab); }
