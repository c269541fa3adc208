// CTU kernels, fp32 form: PLM/PPM on characteristic variables x Riemann
// solvers for N = 16.
#include "kernels.cuh"

void hyd_reg_ctu_char_fp32(hyd::KernelEntry* tab) { hyd::put_scheme<hyd::CTU, hyd::P_FP32, 16, true>(tab); }
