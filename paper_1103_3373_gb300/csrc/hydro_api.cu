// C-ABI of libhydro (declared in include/hydro.h): argument checks, kernel
// selection, launch configuration and launches on the caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "../../include/hydro.h"
#include "kernels.cuh"

namespace hyd {
cudaError_t launch_gather(const void* field, int X, int Y, int Z, int bc, const int* origin, int G, int N, int g,
                          int dbl, void* out, cudaStream_t st, int nsm);
cudaError_t launch_cfl(const void* U, int G, long long gs, long long vs, long long cells, int dbl, double gamma,
                       double dfl, double pfl, const double* dx, double cfl, double* dt, double* smax, double* ws,
                       cudaStream_t st, int nsm);
size_t cfl_boxes_workspace_bytes();
cudaError_t launch_cfl_boxes(const hydro_cfl_box* boxes, int n, int dbl, double gamma, double dfl, double pfl,
                             double cfl, double* dt_min, double* ws, cudaStream_t st);
cudaError_t launch_totals(const void* U, int G, long long gs, long long vs, long long cells, int dbl, double* out,
                          double* ws, cudaStream_t st, int nsm);
constexpr int RED_MAX_CTAS = 2048;
}  // namespace hyd

using namespace hyd;

namespace {

constexpr int MAX_DEV = 16;

struct State {
  std::mutex mu;
  bool registered = false;
  KernelEntry tab[NKEY];
  int nsm[MAX_DEV] = {0};
  int smem_optin[MAX_DEV] = {0};
  bool attr_set[MAX_DEV][NKEY][2] = {{{false}}};  // [.][.][RUNS variant]
};

State& state() {
  static State s;
  return s;
}

thread_local std::string g_cuda_err;

int cuda_fail(cudaError_t e) {
  g_cuda_err = cudaGetErrorString(e);
  return HYDRO_ECUDA;
}

}  // namespace

// Shared with the other C-ABI translation units: records the CUDA error for
// hydro_last_cuda_error and returns HYDRO_ECUDA.
namespace hyd {
int record_cuda_error(cudaError_t e) { return cuda_fail(e); }
}  // namespace hyd

namespace {

void ensure_registered(State& s) {
  if (s.registered) return;
  memset(s.tab, 0, sizeof(s.tab));
  hyd_reg_mhm_fp64(s.tab);
  hyd_reg_mhm_fp32(s.tab);
  hyd_reg_mhm_mixed(s.tab);
  hyd_reg_vl_fp64(s.tab);
  hyd_reg_vl_fp32(s.tab);
  hyd_reg_vl_mixed(s.tab);
  hyd_reg_ctu_fp64(s.tab);
  hyd_reg_ctu_fp32(s.tab);
  hyd_reg_ctu_mixed(s.tab);
  hyd_reg_mhm_char_fp64(s.tab);
  hyd_reg_mhm_char_fp32(s.tab);
  hyd_reg_mhm_char_mixed(s.tab);
  hyd_reg_vl_char_fp64(s.tab);
  hyd_reg_vl_char_fp32(s.tab);
  hyd_reg_vl_char_mixed(s.tab);
  hyd_reg_ctu_char_fp64(s.tab);
  hyd_reg_ctu_char_fp32(s.tab);
  hyd_reg_ctu_char_mixed(s.tab);
  hyd_reg_split_fp64(s.tab);
  hyd_reg_split_fp32(s.tab);
  hyd_reg_split_mixed(s.tab);
  s.registered = true;
}

int current_device(int* dev) {
  cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (*dev < 0 || *dev >= MAX_DEV) return HYDRO_EUNSUPPORTED;
  return HYDRO_OK;
}

int device_sms(State& s, int dev) {
  if (s.nsm[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return -1;
    s.nsm[dev] = v;
    int o = 0;
    cudaDeviceGetAttribute(&o, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    s.smem_optin[dev] = o;
  }
  return s.nsm[dev];
}

bool valid_enums(const hydro_params* p) {
  return p->chain >= 0 && p->chain <= HYDRO_CHAIN_MAX && p->scheme >= 0 && p->scheme <= 4 && p->recon >= 0 && p->recon <= 1 && p->limiter >= 0 && p->limiter <= 3 &&
         (p->characteristic == 0 || p->characteristic == 1) && (p->split_order == 0 || p->split_order == 1) &&
         p->riemann >= 0 && p->riemann <= 3 && p->precision >= 0 && p->precision <= 2 &&
         (p->riemann != HYDRO_RS_ROE ||
          (p->roe_fallback == HYDRO_RS_HLLE || p->roe_fallback == HYDRO_RS_HLLC || p->roe_fallback == HYDRO_RS_EXACT));
}

bool valid_physics(const hydro_params* p) {
  return p->gamma > 1.0 && p->theta >= 1.0 && p->theta <= 2.0 && p->dens_floor >= 0.0 && p->pres_floor >= 0.0;
}

// Resolved launch of one configuration on the current device.
struct Launch {
  const KernelEntry* k;
  const void* fn;  // the kernel: k->fn, or k->fn_runs for launches with runs of gathered groups
  int dev, key, threads, grid;
  size_t smem_bytes;
  size_t ws_bytes;
};

int resolve(const hydro_params* p, int N, long long total_groups, Launch& L, bool runs = false) {
  if (!p) return HYDRO_EINVAL;
  if (!valid_enums(p)) return HYDRO_EINVAL;
  if (N != 16) return HYDRO_EUNSUPPORTED;
  State& s = state();
  std::lock_guard<std::mutex> lk(s.mu);
  ensure_registered(s);
  int rc = current_device(&L.dev);
  if (rc) return rc;
  int nsm = device_sms(s, L.dev);
  if (nsm <= 0) return cuda_fail(cudaErrorInvalidDevice);
  L.key = kernel_key(p->scheme, p->recon, p->characteristic, p->riemann, p->precision);
  L.k = &s.tab[L.key];
  if (!L.k->fn) return HYDRO_EUNSUPPORTED;
  const bool rv = runs && L.k->fn_runs;
  L.fn = rv ? L.k->fn_runs : L.k->fn;
  int maxt = L.k->max_threads;
  L.threads = p->block_threads ? p->block_threads : maxt;
  if (L.threads < 32 || L.threads > maxt || (L.threads & 31)) return HYDRO_EINVAL;
  L.smem_bytes = L.k->smem ? (size_t)L.k->ring_elems * L.k->elem_bytes : 0;
  if (L.k->smem && (int)L.smem_bytes > s.smem_optin[L.dev]) return HYDRO_EUNSUPPORTED;
  if (!s.attr_set[L.dev][L.key][rv]) {
    if (L.k->smem) {
      cudaError_t e = cudaFuncSetAttribute(L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    s.attr_set[L.dev][L.key][rv] = true;
  }
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, L.fn, L.threads, L.smem_bytes);
  if (e != cudaSuccess) return cuda_fail(e);
  if (occ < 1) return HYDRO_EUNSUPPORTED;
  long long g = p->grid_ctas > 0 ? p->grid_ctas : (long long)nsm * occ;
  if (p->grid_ctas < 0) return HYDRO_EINVAL;
  if (total_groups >= 0 && g > total_groups) g = total_groups > 0 ? total_groups : 1;
  L.grid = (int)g;
  // FP64 scratch: one ring per CTA of the largest grid this config may use
  long long gmax = p->grid_ctas > 0 ? p->grid_ctas : (long long)nsm * occ;
  L.ws_bytes = L.k->smem ? 0 : (size_t)gmax * L.k->ring_elems * L.k->elem_bytes;
  return HYDRO_OK;
}

int launch_table(const hydro_params* p, const WorkTable& wt, int N, int ghost, void* stream) {
  Launch L;
  bool runs = false;  // an entry of gathered groups with runs of z-continuations
  for (int s = 0; s < wt.nseg; ++s) runs = runs || (wt.seg[s].mode == 0 && wt.seg[s].zrun);
  int rc = resolve(p, N, wt.total, L, runs);
  if (rc) return rc;
  if (wt.total == 0) return HYDRO_OK;
  if (!L.k->smem) {
    if (!p->workspace || p->workspace_bytes < L.ws_bytes) return HYDRO_EWORKSPACE;
  }
  KConst kc;
  kc.gamma = p->gamma;
  kc.dens_floor = p->dens_floor;
  kc.pres_floor = p->pres_floor;
  kc.theta = p->theta;
  kc.limiter = p->limiter;
  kc.fallback = p->roe_fallback;
  kc.split_order = p->split_order;
  kc.ghost = ghost;
  kc.ring_elems = L.k->ring_elems;
  void* ws = p->workspace;
  void* args[] = {(void*)&wt, (void*)&kc, (void*)&ws};
  cudaError_t e = cudaLaunchKernel(L.fn, dim3(L.grid), dim3(L.threads), args, L.smem_bytes, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e);
  return HYDRO_OK;
}

bool finite_pos(double a) { return a > 0.0 && a < 1e300; }

// z-segment length of a mode-1 entry of GZ group layers
int segment_layers(const hydro_params* p, int GZ) {
  int lc = p->chain > 0 ? p->chain : CHAIN_MAX;
  if (lc > GZ) lc = GZ;
  return lc < 1 ? 1 : lc;
}

// [a, a + na) and [b, b + nb) share a byte
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return na > 0 && nb > 0 && x < y + nb && y < x + na;
}

size_t elem_size(const hydro_params* p) { return p->precision == HYDRO_FP64 ? 8 : 4; }

}  // namespace

extern "C" {

int hydro_required_ghost(int scheme, int recon) {
  if (scheme < 0 || scheme > 4 || recon < 0 || recon > 1) return HYDRO_EINVAL;
  if (scheme == HYDRO_RTVD) return 3;
  if (scheme == HYDRO_WAF) return 2;
  int s = recon == HYDRO_PPM ? 2 : 1;
  return scheme == HYDRO_VL ? s + 2 : s + 1;
}

size_t hydro_workspace_bytes(const hydro_params* p, int N) {
  Launch L;
  if (resolve(p, N, -1, L) != HYDRO_OK) return 0;
  return L.ws_bytes;
}

int hydro_max_block_threads(const hydro_params* p, int N) {
  if (!p || !valid_enums(p)) return HYDRO_EINVAL;
  if (N != 16) return HYDRO_EUNSUPPORTED;
  State& s = state();
  std::lock_guard<std::mutex> lk(s.mu);
  ensure_registered(s);
  const KernelEntry& k = s.tab[kernel_key(p->scheme, p->recon, p->characteristic, p->riemann, p->precision)];
  return k.fn ? k.max_threads : HYDRO_EUNSUPPORTED;
}

int hydro_advance(const hydro_params* p, const void* U_in, void* U_out, void* flux, int G, int N, int ghost,
                  unsigned* dev_status, void* stream) {
  if (!p || G < 0) return HYDRO_EINVAL;
  if (!valid_enums(p) || !valid_physics(p)) return HYDRO_EINVAL;
  int req = hydro_required_ghost(p->scheme, p->recon);
  if (ghost < req) return HYDRO_EGHOST;
  if (G > 0 && (!U_in || !U_out)) return HYDRO_EINVAL;
  {
    const size_t M = (size_t)N + 2 * (size_t)ghost;
    if (overlap(U_in, (size_t)G * 5 * M * M * M * elem_size(p), U_out, (size_t)G * 5 * N * N * N * elem_size(p)))
      return HYDRO_EINVAL;
  }
  if (!p->dt_dev && !(p->dt >= 0.0)) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!finite_pos(p->dx[d])) return HYDRO_EINVAL;
  WorkTable wt;
  memset(&wt, 0, sizeof(wt));
  wt.nseg = 1;
  wt.total = G;
  SegDesc& s = wt.seg[0];
  s.in = U_in;
  s.out = U_out;
  s.flux = flux;
  s.status = dev_status;
  s.dt_dev = p->dt_dev;
  s.dt = p->dt;
  for (int d = 0; d < 3; ++d) s.dx[d] = p->dx[d];
  s.G = G;
  s.mode = 0;
  s.zrun = p->zrun;
  s.lc = p->chain > 0 ? p->chain : CHAIN_MAX;
  s.first = 0;
  return launch_table(p, wt, N, ghost, stream);
}

int hydro_advance_uniform(const hydro_params* p, const void* field_in, void* field_out, int X, int Y, int Z, int N,
                          int bc, void* flux, unsigned* dev_status, void* stream) {
  if (!p || !valid_enums(p) || !valid_physics(p)) return HYDRO_EINVAL;
  if (N != 16) return HYDRO_EUNSUPPORTED;
  if (X <= 0 || Y <= 0 || Z <= 0 || X % N || Y % N || Z % N) return HYDRO_EINVAL;
  if (bc != HYDRO_BC_PERIODIC && bc != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
  if (!field_in || !field_out) return HYDRO_EINVAL;
  if (overlap(field_in, (size_t)5 * X * Y * Z * elem_size(p), field_out, (size_t)5 * X * Y * Z * elem_size(p)))
    return HYDRO_EINVAL;
  if (!p->dt_dev && !(p->dt >= 0.0)) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!finite_pos(p->dx[d])) return HYDRO_EINVAL;
  long long G = (long long)(X / N) * (Y / N) * (Z / N);
  if (G > 0x7fffffffLL) return HYDRO_EINVAL;
  WorkTable wt;
  memset(&wt, 0, sizeof(wt));
  wt.nseg = 1;
  wt.total = (int)G;
  SegDesc& s = wt.seg[0];
  s.in = field_in;
  s.out = field_out;
  s.flux = flux;
  s.status = dev_status;
  s.dt_dev = p->dt_dev;
  s.dt = p->dt;
  for (int d = 0; d < 3; ++d) s.dx[d] = p->dx[d];
  s.G = (int)G;
  s.mode = 1;
  s.bc = bc;
  s.X = X;
  s.Y = Y;
  s.Z = Z;
  s.GX = X / N;
  s.GY = Y / N;
  s.GZ = Z / N;
  s.lc = segment_layers(p, s.GZ);
  s.first = 0;
  return launch_table(p, wt, N, hydro_required_ghost(p->scheme, p->recon), stream);
}

int hydro_advance_uniform_zrange(const hydro_params* p, const void* field_in, void* field_out, int X, int Y, int Z,
                                 int N, int bc, int z_begin, int z_end, void* flux, unsigned* dev_status,
                                 void* stream) {
  if (!p || !valid_enums(p) || !valid_physics(p)) return HYDRO_EINVAL;
  if (N != 16) return HYDRO_EUNSUPPORTED;
  if (X <= 0 || Y <= 0 || Z <= 0 || X % N || Y % N || Z % N) return HYDRO_EINVAL;
  if (z_begin < 0 || z_end > Z || z_begin > z_end || z_begin % N || z_end % N) return HYDRO_EINVAL;
  if (bc != HYDRO_BC_PERIODIC && bc != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
  if (!field_in || !field_out) return HYDRO_EINVAL;
  if (overlap(field_in, (size_t)5 * X * Y * Z * elem_size(p), field_out, (size_t)5 * X * Y * Z * elem_size(p)))
    return HYDRO_EINVAL;
  if (!p->dt_dev && !(p->dt >= 0.0)) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!finite_pos(p->dx[d])) return HYDRO_EINVAL;
  long long G = (long long)(X / N) * (Y / N) * ((z_end - z_begin) / N);
  if (G > 0x7fffffffLL) return HYDRO_EINVAL;
  WorkTable wt;
  memset(&wt, 0, sizeof(wt));
  wt.nseg = 1;
  wt.total = (int)G;
  SegDesc& s = wt.seg[0];
  s.in = field_in;
  s.out = field_out;
  s.flux = flux;
  s.status = dev_status;
  s.dt_dev = p->dt_dev;
  s.dt = p->dt;
  for (int d = 0; d < 3; ++d) s.dx[d] = p->dx[d];
  s.G = (int)G;
  s.mode = 1;
  s.bc = bc;
  s.X = X;
  s.Y = Y;
  s.Z = Z;
  s.GX = X / N;
  s.GY = Y / N;
  s.GZ = (z_end - z_begin) / N;
  s.lc = segment_layers(p, s.GZ);
  s.gz0 = z_begin / N;
  s.first = 0;
  return launch_table(p, wt, N, hydro_required_ghost(p->scheme, p->recon), stream);
}

int hydro_advance_levels(const hydro_params* p, const hydro_level* levels, int nlev, int N, int ghost, void* stream) {
  if (!p || !valid_enums(p) || !valid_physics(p)) return HYDRO_EINVAL;
  if (nlev < 0 || nlev > HYDRO_MAX_LEVELS || (nlev > 0 && !levels)) return HYDRO_EINVAL;
  if (N != 16) return HYDRO_EUNSUPPORTED;
  int req = hydro_required_ghost(p->scheme, p->recon);
  bool any_groups_mode = false;
  for (int l = 0; l < nlev; ++l) any_groups_mode = any_groups_mode || levels[l].mode == 0;
  if (any_groups_mode && ghost < req) return HYDRO_EGHOST;
  WorkTable wt;
  memset(&wt, 0, sizeof(wt));
  long long total = 0;
  for (int l = 0; l < nlev; ++l) {
    const hydro_level& lv = levels[l];
    SegDesc& s = wt.seg[l];
    if (lv.mode != 0 && lv.mode != 1) return HYDRO_EINVAL;
    if (!lv.dt_dev && !(lv.dt >= 0.0)) return HYDRO_EINVAL;
    for (int d = 0; d < 3; ++d) {
      if (!finite_pos(lv.dx[d])) return HYDRO_EINVAL;
      s.dx[d] = lv.dx[d];
    }
    long long G;
    if (lv.mode == 0) {
      if (lv.G < 0) return HYDRO_EINVAL;
      G = lv.G;
      s.zrun = lv.zrun;
      s.lc = p->chain > 0 ? p->chain : CHAIN_MAX;
    } else {
      if (lv.X <= 0 || lv.Y <= 0 || lv.Z <= 0 || lv.X % N || lv.Y % N || lv.Z % N) return HYDRO_EINVAL;
      if (lv.bc != HYDRO_BC_PERIODIC && lv.bc != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
      G = (long long)(lv.X / N) * (lv.Y / N) * (lv.Z / N);
      s.bc = lv.bc;
      s.X = lv.X;
      s.Y = lv.Y;
      s.Z = lv.Z;
      s.GX = lv.X / N;
      s.GY = lv.Y / N;
      s.GZ = lv.Z / N;
      s.lc = segment_layers(p, s.GZ);
    }
    if (G > 0 && (!lv.U_in || !lv.U_out)) return HYDRO_EINVAL;
    {
      const size_t M = (size_t)N + 2 * (size_t)ghost;
      const size_t nin = lv.mode == 0 ? (size_t)G * 5 * M * M * M : (size_t)5 * lv.X * lv.Y * lv.Z;
      const size_t nout = lv.mode == 0 ? (size_t)G * 5 * N * N * N : nin;
      if (overlap(lv.U_in, nin * elem_size(p), lv.U_out, nout * elem_size(p))) return HYDRO_EINVAL;
    }
    s.in = lv.U_in;
    s.out = lv.U_out;
    s.flux = lv.flux;
    s.status = lv.status;
    s.dt_dev = lv.dt_dev;
    s.dt = lv.dt;
    s.G = (int)G;
    s.mode = lv.mode;
    s.first = (int)total;
    total += G;
    if (total > 0x7fffffffLL) return HYDRO_EINVAL;
  }
  wt.nseg = nlev;
  wt.total = (int)total;
  // mode-1 entries read their halo with the minimal ghost width
  return launch_table(p, wt, N, any_groups_mode ? ghost : req, stream);
}

int hydro_gather_uniform(const void* field, int X, int Y, int Z, int bc, const int* origin, int G, int N, int ghost,
                         int precision, void* U_out, void* stream) {
  if (G < 0 || N <= 0 || ghost < 0 || X <= 0 || Y <= 0 || Z <= 0) return HYDRO_EINVAL;
  if (bc != HYDRO_BC_PERIODIC && bc != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
  if (precision < 0 || precision > 2) return HYDRO_EINVAL;
  if (G == 0) return HYDRO_OK;
  if (!field || !origin || !U_out) return HYDRO_EINVAL;
  int dev;
  int rc = current_device(&dev);
  if (rc) return rc;
  int nsm;
  {
    State& s = state();
    std::lock_guard<std::mutex> lk(s.mu);
    nsm = device_sms(s, dev);
  }
  cudaError_t e = launch_gather(field, X, Y, Z, bc, origin, G, N, ghost, precision == HYDRO_FP64, U_out,
                                (cudaStream_t)stream, nsm);
  return e == cudaSuccess ? HYDRO_OK : cuda_fail(e);
}

size_t hydro_cfl_workspace_bytes(void) { return (size_t)5 * RED_MAX_CTAS * sizeof(double); }

int hydro_cfl_dt(const void* U, int G, long long group_stride, long long var_stride, long long cells, int precision,
                 double gamma, double dens_floor, double pres_floor, const double* dx, double cfl, double* dt_dev,
                 double* smax_dev, void* workspace, size_t workspace_bytes, void* stream) {
  if (!U || G < 0 || cells < 0 || !dx || !dt_dev || !(gamma > 1.0) || !(cfl > 0.0)) return HYDRO_EINVAL;
  if (precision < 0 || precision > 2) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!finite_pos(dx[d])) return HYDRO_EINVAL;
  if (!workspace || workspace_bytes < (size_t)3 * RED_MAX_CTAS * sizeof(double)) return HYDRO_EWORKSPACE;
  int dev;
  int rc = current_device(&dev);
  if (rc) return rc;
  int nsm;
  {
    State& s = state();
    std::lock_guard<std::mutex> lk(s.mu);
    nsm = device_sms(s, dev);
  }
  cudaError_t e = launch_cfl(U, G, group_stride, var_stride, cells, precision == HYDRO_FP64, gamma, dens_floor,
                             pres_floor, dx, cfl, dt_dev, smax_dev, (double*)workspace, (cudaStream_t)stream, nsm);
  return e == cudaSuccess ? HYDRO_OK : cuda_fail(e);
}

size_t hydro_cfl_boxes_workspace_bytes(void) { return cfl_boxes_workspace_bytes(); }

int hydro_cfl_dt_boxes(const hydro_cfl_box* boxes, int nbox, int precision, double gamma, double dens_floor,
                       double pres_floor, double cfl, double* dt_min_dev, void* workspace, size_t workspace_bytes,
                       void* stream) {
  if (!boxes || nbox < 1 || nbox > HYDRO_CFL_MAX_BOXES || !(gamma > 1.0) || !(cfl > 0.0)) return HYDRO_EINVAL;
  if (precision < 0 || precision > 2) return HYDRO_EINVAL;
  for (int b = 0; b < nbox; ++b) {
    const hydro_cfl_box& x = boxes[b];
    if (!x.U || !x.dt_dev || x.G < 0 || x.cells < 0 || !finite_pos(x.dt_scale)) return HYDRO_EINVAL;
    for (int d = 0; d < 3; ++d)
      if (!finite_pos(x.dx[d])) return HYDRO_EINVAL;
    if (x.ghost < 0) return HYDRO_EINVAL;
    if (x.ghost > 0) {
      const long long n = x.interior_n, M = n + 2LL * x.ghost;
      if (n < 1 || n > 1024 || x.ghost > 1024 || x.cells != n * n * n || x.var_stride < M * M * M)
        return HYDRO_EINVAL;
    }
  }
  if (!workspace || workspace_bytes < cfl_boxes_workspace_bytes()) return HYDRO_EWORKSPACE;
  int dev;
  int rc = current_device(&dev);
  if (rc) return rc;
  cudaError_t e = launch_cfl_boxes(boxes, nbox, precision == HYDRO_FP64, gamma, dens_floor, pres_floor, cfl,
                                   dt_min_dev, (double*)workspace, (cudaStream_t)stream);
  return e == cudaSuccess ? HYDRO_OK : cuda_fail(e);
}

int hydro_conserved_totals(const void* U, int G, long long group_stride, long long var_stride, long long cells,
                           int precision, double* totals_dev, void* workspace, size_t workspace_bytes, void* stream) {
  if (!U || G < 0 || cells < 0 || !totals_dev) return HYDRO_EINVAL;
  if (precision < 0 || precision > 2) return HYDRO_EINVAL;
  if (!workspace || workspace_bytes < hydro_cfl_workspace_bytes()) return HYDRO_EWORKSPACE;
  int dev;
  int rc = current_device(&dev);
  if (rc) return rc;
  int nsm;
  {
    State& s = state();
    std::lock_guard<std::mutex> lk(s.mu);
    nsm = device_sms(s, dev);
  }
  cudaError_t e = launch_totals(U, G, group_stride, var_stride, cells, precision == HYDRO_FP64, totals_dev,
                                (double*)workspace, (cudaStream_t)stream, nsm);
  return e == cudaSuccess ? HYDRO_OK : cuda_fail(e);
}

const char* hydro_strerror(int code) {
  switch (code) {
    case HYDRO_OK: return "ok";
    case HYDRO_EINVAL: return "invalid argument";
    case HYDRO_EGHOST: return "ghost width below what the scheme needs";
    case HYDRO_EUNSUPPORTED: return "configuration not built or not supported on this device";
    case HYDRO_ECUDA: return "CUDA call failed";
    case HYDRO_EWORKSPACE: return "workspace missing or too small";
    case HYDRO_ETOOBIG: return "input larger than this fixed-size entry point takes";
    default: return "unknown error";
  }
}

const char* hydro_last_cuda_error(void) { return g_cuda_err.c_str(); }

}  // extern "C"
