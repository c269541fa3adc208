// VL kernels, fp64 form: all reconstructions x Riemann solvers for N = 16.
#include "kernels.cuh"

void hyd_reg_vl_fp64(hyd::KernelEntry* tab) { hyd::put_scheme<hyd::VL, hyd::P_FP64, 16>(tab); }
