// CTU kernels, mixed form: PLM/PPM on characteristic variables x Riemann
// solvers for N = 16.
#include "kernels.cuh"

void hyd_reg_ctu_char_mixed(hyd::KernelEntry* tab) { hyd::put_scheme<hyd::CTU, hyd::P_MIXED, 16, true>(tab); }
