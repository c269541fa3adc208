// CTU kernels, fp64 form: all reconstructions x Riemann solvers for N = 16.
#include "kernels.cuh"

void hyd_reg_ctu_fp64(hyd::KernelEntry* tab) { hyd::put_scheme<hyd::CTU, hyd::P_FP64, 16>(tab); }
