// Directionally split schemes (RTVD, WAF), fp32 form, for N = 16.
#include "kernels.cuh"

void hyd_reg_split_fp32(hyd::KernelEntry* tab) {
  hyd::put_split<hyd::SCH_RTVD, hyd::P_FP32, 16>(tab);
  hyd::put_split<hyd::SCH_WAF, hyd::P_FP32, 16>(tab);
}
