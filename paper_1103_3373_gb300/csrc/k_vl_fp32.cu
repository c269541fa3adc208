// VL kernels, fp32 form: PLM/PPM on primitive variables x Riemann solvers for N = 16.
#include "kernels.cuh"

void hyd_reg_vl_fp32(hyd::KernelEntry* tab) { hyd::put_scheme<hyd::VL, hyd::P_FP32, 16, false>(tab); }
