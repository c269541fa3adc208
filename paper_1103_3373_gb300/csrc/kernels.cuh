// Persistent patch-group kernel: each CTA takes a contiguous share of the
// flat list of groups of all work-table entries (levels / boxes / one batch;
// the shares differ by at most one group) and runs the selected scheme on it
// (Sec. 3.1: one thread block per patch group; here the blocks are
// persistent, one per SM).  In a uniform field consecutive work items are
// z-neighbours, and a CTA streams through each run of them as one chain.
#pragma once
#include "ctu.cuh"
#include "mhm.cuh"
#include "split.cuh"
#include "vl.cuh"

namespace hyd {

template <int SCH, int REC, int PR, int N> struct KTraits {
  using P = Prec<PR>;
  using T = typename P::T;
  using S = typename P::S;
  static constexpr int S_ = REC == PPM ? 2 : 1;
  static constexpr int MS = N + 2 * SplitGhost<SCH>::value;  // padded edge of the split schemes
  static constexpr int RING = SCH == CTU   ? CtuLayout<N, S_>::TOTAL
                              : SCH == MHM ? MhmLayout<N, S_>::TOTAL
                              : SCH == VL  ? VlLayout<N, S_>::TOTAL
                                           : 5 * MS * MS * MS;
  static constexpr bool SMEM = PR != P_FP64;  // FP64 rings do not fit in shared memory
};

// Largest CTA: FP64 kernels need up to 255 registers per thread; the FP32
// kernels run 16 warps per SM (128 registers per thread) except the exact
// solver, whose Newton iteration needs more registers, and the split
// schemes, whose threads each carry a row's sliding window.
template <int PR, int RS, int SCH = 0> struct MaxThreads {
  static constexpr int value = PR == P_FP64 ? 256 : ((RS == RS_EXACT || SCH >= SCH_RTVD) ? 384 : 512);
};

// RUNS: the variant that also streams runs of gathered groups as chains
// (hydro_params.zrun; the unsplit schemes).  It is a kernel of its own so that the code
// of the other forms stays as it is; every form of one launch runs the same
// compiled copy, so they give the same bytes.
template <int SCH, int REC, int RS, int PR, int N, bool CH, bool RUNS = false>
__global__ void __launch_bounds__(MaxThreads<PR, RS, SCH>::value, 1)
    advance_kernel(const __grid_constant__ WorkTable wt, const KConst kc, void* ws) {
  using Tr = KTraits<SCH, REC, PR, N>;
  using T = typename Tr::T;
  using S = typename Tr::S;
  constexpr bool MIXED = Tr::P::MIXED;
  constexpr bool GCH = RUNS && SCH <= CTU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned sts[CHAIN_MAX];  // status of the groups of the current chain
  __shared__ double sc[6];
  T* ring;
  if constexpr (Tr::SMEM)
    ring = reinterpret_cast<T*>(smem_raw);
  else
    ring = reinterpret_cast<T*>(ws) + (long long)blockIdx.x * kc.ring_elems;
  Opts<T> o;
  o.gas.gamma = (T)kc.gamma;
  o.gas.gm1 = (T)(kc.gamma - 1.0);
  o.gas.igm1 = (T)(1.0 / (kc.gamma - 1.0));
  o.gas.dens_floor = (T)kc.dens_floor;
  o.gas.pres_floor = (T)kc.pres_floor;
  o.theta = (T)kc.theta;
  o.limiter = kc.limiter;
  o.fallback = kc.fallback;
  o.split_order = kc.split_order;
  if (threadIdx.x < CHAIN_MAX) sts[threadIdx.x] = 0;
  const int b = blockIdx.x;
  const int per = wt.total / gridDim.x, extra = wt.total % gridDim.x;
  int w = b * per + (b < extra ? b : extra);
  const int wend = w + per + (b < extra ? 1 : 0);
  while (w < wend) {
    int s = 0;
    while (s + 1 < wt.nseg && w >= wt.seg[s + 1].first) ++s;
    const SegDesc& sg = wt.seg[s];
    const int gi = w - sg.first;
    int K = 1;
    if (sg.mode == 1 && SCH <= CTU) {
      const int left = seg_pos(sg, gi).left;  // groups left in this z-segment
      K = wend - w < left ? wend - w : left;
      K = K < CHAIN_MAX ? K : CHAIN_MAX;
    } else if (GCH && sg.zrun) {
      // gathered groups: the run of z-continuations starting here, cut at
      // the CTA's share, the entry's end and the chain limit
      int left = sg.zrun[gi];
      left = left < sg.G - gi ? left : sg.G - gi;
      left = left < sg.lc ? left : sg.lc;
      K = wend - w < left ? wend - w : left;
      K = K > 1 ? K : 1;
    }
    if (threadIdx.x == 0) group_consts(sg, sc);
    __syncthreads();
    // one compiled copy of the group pipeline serves every form of an entry,
    // so that all forms give the same bytes
    GroupCtx<T, S, N, GCH> C;
    C.init(sg, gi, kc, sc, K);
    if constexpr (SCH == CTU)
      ctu_group<T, S, MIXED, RS, REC, CH, N>(C, o, ring, K, sts);
    else if constexpr (SCH == MHM)
      mhm_group<T, S, MIXED, RS, REC, CH, N>(C, o, ring, K, sts);
    else if constexpr (SCH == VL)
      vl_group<T, S, MIXED, RS, REC, CH, N>(C, o, ring, K, sts);
    else
      split_group<T, S, MIXED, SCH, N>(C, o, ring, sts);
    __syncthreads();
    if (threadIdx.x < K) {
      if (sg.status) sg.status[C.user_index(threadIdx.x)] = sts[threadIdx.x];
      sts[threadIdx.x] = 0;
    }
    w += K;
  }
}

// Host-side description of one compiled kernel.
struct KernelEntry {
  const void* fn;
  const void* fn_runs;  // the RUNS variant, or null
  long long ring_elems;
  int elem_bytes;
  int max_threads;
  int smem;  // 1: rings in shared memory
};

// (scheme, reconstruction, characteristic, solver, precision)
constexpr int NKEY = 5 * 2 * 2 * 4 * 3;
inline int kernel_key(int sch, int rec, int ch, int rs, int pr) {
  return (((sch * 2 + rec) * 2 + ch) * 4 + rs) * 3 + pr;
}

template <int SCH, int REC, int RS, int PR, int N, bool CH> inline void put_kernel(KernelEntry* tab) {
  using Tr = KTraits<SCH, REC, PR, N>;
  KernelEntry& e = tab[kernel_key(SCH, REC, CH ? 1 : 0, RS, PR)];
  e.fn = (const void*)&advance_kernel<SCH, REC, RS, PR, N, CH>;
  if constexpr (SCH <= CTU) e.fn_runs = (const void*)&advance_kernel<SCH, REC, RS, PR, N, CH, true>;
  e.ring_elems = Tr::RING;
  e.elem_bytes = (int)sizeof(typename Tr::T);
  e.max_threads = MaxThreads<PR, RS, SCH>::value;
  e.smem = Tr::SMEM ? 1 : 0;
}

template <int SCH, int PR, int N, bool CH> inline void put_scheme(KernelEntry* tab) {
  put_kernel<SCH, PLM, RS_EXACT, PR, N, CH>(tab);
  put_kernel<SCH, PLM, RS_HLLE, PR, N, CH>(tab);
  put_kernel<SCH, PLM, RS_HLLC, PR, N, CH>(tab);
  put_kernel<SCH, PLM, RS_ROE, PR, N, CH>(tab);
  put_kernel<SCH, PPM, RS_EXACT, PR, N, CH>(tab);
  put_kernel<SCH, PPM, RS_HLLE, PR, N, CH>(tab);
  put_kernel<SCH, PPM, RS_HLLC, PR, N, CH>(tab);
  put_kernel<SCH, PPM, RS_ROE, PR, N, CH>(tab);
}

// The split schemes ignore reconstruction, characteristic and solver: one
// kernel serves every key of (scheme, precision).
template <int SCH, int PR, int N> inline void put_split(KernelEntry* tab) {
  put_kernel<SCH, PLM, RS_HLLC, PR, N, false>(tab);
  const KernelEntry e = tab[kernel_key(SCH, PLM, 0, RS_HLLC, PR)];
  for (int rec = 0; rec < 2; ++rec)
    for (int ch = 0; ch < 2; ++ch)
      for (int rs = 0; rs < 4; ++rs) tab[kernel_key(SCH, rec, ch, rs, PR)] = e;
}

}  // namespace hyd

// Registration functions, one per (scheme, reconstructed variables,
// precision) translation unit.
#define HYD_DECLARE_REG(name) void name(hyd::KernelEntry* tab)
HYD_DECLARE_REG(hyd_reg_mhm_fp64);
HYD_DECLARE_REG(hyd_reg_mhm_fp32);
HYD_DECLARE_REG(hyd_reg_mhm_mixed);
HYD_DECLARE_REG(hyd_reg_vl_fp64);
HYD_DECLARE_REG(hyd_reg_vl_fp32);
HYD_DECLARE_REG(hyd_reg_vl_mixed);
HYD_DECLARE_REG(hyd_reg_ctu_fp64);
HYD_DECLARE_REG(hyd_reg_ctu_fp32);
HYD_DECLARE_REG(hyd_reg_ctu_mixed);
HYD_DECLARE_REG(hyd_reg_mhm_char_fp64);
HYD_DECLARE_REG(hyd_reg_mhm_char_fp32);
HYD_DECLARE_REG(hyd_reg_mhm_char_mixed);
HYD_DECLARE_REG(hyd_reg_vl_char_fp64);
HYD_DECLARE_REG(hyd_reg_vl_char_fp32);
HYD_DECLARE_REG(hyd_reg_vl_char_mixed);
HYD_DECLARE_REG(hyd_reg_ctu_char_fp64);
HYD_DECLARE_REG(hyd_reg_ctu_char_fp32);
HYD_DECLARE_REG(hyd_reg_ctu_char_mixed);
HYD_DECLARE_REG(hyd_reg_split_fp64);
HYD_DECLARE_REG(hyd_reg_split_fp32);
HYD_DECLARE_REG(hyd_reg_split_mixed);
