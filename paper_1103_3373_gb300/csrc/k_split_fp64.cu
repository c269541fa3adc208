// Directionally split schemes (RTVD, WAF), fp64 form, for N = 16.
#include "kernels.cuh"

void hyd_reg_split_fp64(hyd::KernelEntry* tab) {
  hyd::put_split<hyd::SCH_RTVD, hyd::P_FP64, 16>(tab);
  hyd::put_split<hyd::SCH_WAF, hyd::P_FP64, 16>(tab);
}
