// MHM kernels, mixed form: PLM/PPM on primitive variables x Riemann solvers for N = 16.
#include "kernels.cuh"

void hyd_reg_mhm_mixed(hyd::KernelEntry* tab) { hyd::put_scheme<hyd::MHM, hyd::P_MIXED, 16, false>(tab); }
