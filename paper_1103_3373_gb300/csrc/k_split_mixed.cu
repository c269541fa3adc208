// Directionally split schemes (RTVD, WAF), mixed form, for N = 16.
#include "kernels.cuh"

void hyd_reg_split_mixed(hyd::KernelEntry* tab) {
  hyd::put_split<hyd::SCH_RTVD, hyd::P_MIXED, 16>(tab);
  hyd::put_split<hyd::SCH_WAF, hyd::P_MIXED, 16>(tab);
}
