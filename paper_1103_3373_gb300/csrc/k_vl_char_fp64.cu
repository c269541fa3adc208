// VL kernels, fp64 form: PLM/PPM on characteristic variables x Riemann
// solvers for N = 16.
#include "kernels.cuh"

void hyd_reg_vl_char_fp64(hyd::KernelEntry* tab) { hyd::put_scheme<hyd::VL, hyd::P_FP64, 16, true>(tab); }
