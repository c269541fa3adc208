// End-to-end step of a uniform box with the host<->device copies overlapped
// with the solver on z-slabs (Sec. 4.1, asynchronous memory copy over chunks
// of patch groups).  Host-side runtime only: every arithmetic step runs in the
// group kernels (hydro_advance_uniform_zrange) and the CFL reduction
// (hydro_cfl_dt).
#include <cuda_runtime.h>

#include <new>
#include <utility>
#include <vector>

#include "../../include/hydro.h"
#include "../../include/hydro_pipeline.h"

namespace hyd {
int record_cuda_error(cudaError_t e);
}

struct hydro_pipeline {
  int X, Y, Z, N, ghost, bc, nslab;
  std::vector<int> zb;                                  // slab s = planes [zb[s], zb[s+1])
  std::vector<std::vector<std::pair<int, int>>> chunk;  // input plane ranges completing slab s
  cudaStream_t s_in = nullptr, s_out = nullptr, s_comp[2] = {nullptr, nullptr};
  cudaEvent_t ev_start = nullptr, ev_c1 = nullptr, ev_cfl = nullptr, ev_done = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_comp;
  std::vector<cudaEvent_t> ev_out;  // copy-out of slab s done (last step)
  // buffers of the last step (chained steps: see hydro_pipeline_step)
  bool has_prev = false;
  const void* prev_host_out = nullptr;
  const void* prev_dev_in = nullptr;
  const void* prev_dev_out = nullptr;
};

namespace {

void release(hydro_pipeline* h) {
  cudaStream_t ss[4] = {h->s_in, h->s_out, h->s_comp[0], h->s_comp[1]};
  for (cudaStream_t s : ss)
    if (s) cudaStreamSynchronize(s);
  for (cudaEvent_t e : h->ev_in)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_comp)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_out)
    if (e) cudaEventDestroy(e);
  cudaEvent_t es[4] = {h->ev_start, h->ev_c1, h->ev_cfl, h->ev_done};
  for (cudaEvent_t e : es)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : ss)
    if (s) cudaStreamDestroy(s);
  delete h;
}

// Input plane ranges per slab, in copy order: the ranges whose arrival
// completes slab s's input and halo.  Periodic boxes send the last `ghost`
// planes first (slab 0's lower halo); slab s < S-1 then needs the planes up
// to zb[s+1] + ghost; the last slab needs the rest.  chunk[s] = {lo0, hi0,
// lo1, hi1}: up to two ranges (the second empty: lo1 = hi1 = 0).
void plan_ranges(int Z, int ghost, int bc, int S, const int* zb, int (*chunk)[4]) {
  const bool periodic = bc == HYDRO_BC_PERIODIC;
  int lo = 0;
  for (int s = 0; s < S; ++s) {
    int k = 0;
    chunk[s][0] = chunk[s][1] = chunk[s][2] = chunk[s][3] = 0;
    if (s == 0 && periodic && ghost > 0) {
      chunk[s][0] = Z - ghost;
      chunk[s][1] = Z;
      k = 2;
    }
    const int hi = s < S - 1 ? zb[s + 1] + ghost : (periodic ? Z - ghost : Z);
    chunk[s][k] = lo;
    chunk[s][k + 1] = hi;
    lo = hi;
  }
}

// Slab boundaries from the layer counts (NULL: an even split).
int slab_bounds(int Z, int N, int nslab, const int* layers, int* zb) {
  const int GZ = Z / N;
  if (nslab < 1 || nslab > GZ) return HYDRO_EINVAL;
  zb[0] = 0;
  for (int s = 0; s < nslab; ++s) {
    const int l = layers ? layers[s] : (s + 1) * GZ / nslab - s * GZ / nslab;
    if (l < 1) return HYDRO_EINVAL;
    zb[s + 1] = zb[s] + l * N;
  }
  return zb[nslab] == Z ? HYDRO_OK : HYDRO_EINVAL;
}

void plan(hydro_pipeline* h) {
  std::vector<int> c(4 * h->nslab);
  plan_ranges(h->Z, h->ghost, h->bc, h->nslab, h->zb.data(), reinterpret_cast<int(*)[4]>(c.data()));
  h->chunk.assign(h->nslab, {});
  for (int s = 0; s < h->nslab; ++s)
    for (int k = 0; k < 4; k += 2)
      if (c[4 * s + k + 1] > c[4 * s + k]) h->chunk[s].push_back({c[4 * s + k], c[4 * s + k + 1]});
}

// The five variables of planes [z0, z1) of a [5][Z][Y][X] field, as one 2-D copy.
cudaError_t copy_planes(void* dst, const void* src, const hydro_pipeline* h, int z0, int z1, size_t es,
                        cudaMemcpyKind kind, cudaStream_t st) {
  if (z1 <= z0) return cudaSuccess;
  const size_t plane = (size_t)h->X * h->Y * es;
  const size_t pitch = plane * h->Z;
  const size_t off = plane * z0;
  return cudaMemcpy2DAsync((char*)dst + off, pitch, (const char*)src + off, pitch, plane * (z1 - z0), 5, kind, st);
}

// An error after some work was enqueued: the caller's stream waits for the
// pipeline's streams (what was enqueued completes before later work there),
// and the next step starts unchained.
int fail(hydro_pipeline* h, cudaStream_t user, int rc) {
  h->has_prev = false;
  cudaStream_t ss[4] = {h->s_in, h->s_comp[0], h->s_comp[1], h->s_out};
  for (cudaStream_t s : ss)
    if (cudaEventRecord(h->ev_done, s) == cudaSuccess) cudaStreamWaitEvent(user, h->ev_done, 0);
  return rc;
}

}  // namespace

extern "C" {

int hydro_pipeline_create(int X, int Y, int Z, int N, int ghost, int bc, int nslab, const int* layers,
                          hydro_pipeline** out) {
  if (!out) return HYDRO_EINVAL;
  if (N != 16) return HYDRO_EUNSUPPORTED;
  if (X <= 0 || Y <= 0 || Z <= 0 || X % N || Y % N || Z % N) return HYDRO_EINVAL;
  if (ghost < 0 || ghost >= N) return HYDRO_EINVAL;
  if (bc != HYDRO_BC_PERIODIC && bc != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
  std::vector<int> zb(nslab > 0 ? nslab + 1 : 1);
  if (nslab < 1 || slab_bounds(Z, N, nslab, layers, zb.data()) != HYDRO_OK) return HYDRO_EINVAL;
  hydro_pipeline* h = new (std::nothrow) hydro_pipeline;
  if (!h) return HYDRO_EINVAL;
  h->X = X;
  h->Y = Y;
  h->Z = Z;
  h->N = N;
  h->ghost = ghost;
  h->bc = bc;
  h->nslab = nslab;
  h->zb = zb;
  plan(h);
  h->ev_in.assign(nslab, nullptr);
  h->ev_comp.assign(nslab, nullptr);
  h->ev_out.assign(nslab, nullptr);
  cudaError_t e = cudaSuccess;
  cudaStream_t* ss[4] = {&h->s_in, &h->s_out, &h->s_comp[0], &h->s_comp[1]};
  for (cudaStream_t* s : ss)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
  cudaEvent_t* es[4] = {&h->ev_start, &h->ev_c1, &h->ev_cfl, &h->ev_done};
  for (cudaEvent_t* ev : es)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  for (int s = 0; s < nslab && e == cudaSuccess; ++s) {
    e = cudaEventCreateWithFlags(&h->ev_in[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_comp[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out[s], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    release(h);
    return hyd::record_cuda_error(e);
  }
  *out = h;
  return HYDRO_OK;
}

int hydro_pipeline_step(hydro_pipeline* h, const hydro_params* p, const void* host_in, void* host_out,
                        double* host_dt, void* dev_in, void* dev_out, void* flux, unsigned* dev_status, double cfl,
                        void* red_ws, size_t red_ws_bytes, void* ws2, size_t ws2_bytes, void* stream) {
  if (!h || !p || !host_in || !host_out || !dev_in || !dev_out || !p->dt_dev) return HYDRO_EINVAL;
  if (host_in == host_out || dev_in == dev_out || !(cfl > 0.0)) return HYDRO_EINVAL;
  const int need = hydro_required_ghost(p->scheme, p->recon);
  if (need < 0 || need > h->ghost) return HYDRO_EINVAL;
  if (p->precision < HYDRO_FP64 || p->precision > HYDRO_FP32_MIXED) return HYDRO_EINVAL;
  // scratch of both compute streams and of the reduction, before any work
  const size_t need_ws = hydro_workspace_bytes(p, h->N);
  if (need_ws && (!p->workspace || p->workspace_bytes < need_ws || !ws2 || ws2_bytes < need_ws))
    return HYDRO_EWORKSPACE;
  if (!red_ws || red_ws_bytes < hydro_pipeline_workspace_bytes(h)) return HYDRO_EWORKSPACE;
  const size_t es = p->precision == HYDRO_FP64 ? sizeof(double) : sizeof(float);
  const long long XYZ = (long long)h->X * h->Y * h->Z;
  cudaStream_t user = (cudaStream_t)stream;
  cudaStream_t* c = h->s_comp;
  // Chained step: the input is the last step's output on the host and the
  // device input buffer is neither of the last step's.  Then each input
  // chunk only waits for the last step's copies out of the slabs it covers,
  // and the slab advances wait for the last step's dt (which follows all of
  // its advances): the copy-in overlaps the end of the last step.
  const bool chained = h->has_prev && host_in == h->prev_host_out && dev_in != h->prev_dev_in &&
                       dev_in != h->prev_dev_out && dev_out != h->prev_dev_out;
  cudaError_t e = cudaSuccess;
  if (chained) {
    e = cudaStreamWaitEvent(c[0], h->ev_cfl, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c[1], h->ev_cfl, 0);
  } else {
    e = cudaEventRecord(h->ev_start, user);
    cudaStream_t ss[4] = {h->s_in, c[0], c[1], h->s_out};
    for (cudaStream_t s : ss)
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_start, 0);
  }
  // input, slab by slab
  for (int s = 0; s < h->nslab && e == cudaSuccess; ++s) {
    for (const auto& r : h->chunk[s]) {
      if (chained)
        for (int t = 0; t < h->nslab && e == cudaSuccess; ++t)
          if (h->zb[t] < r.second && r.first < h->zb[t + 1]) e = cudaStreamWaitEvent(h->s_in, h->ev_out[t], 0);
      if (e == cudaSuccess)
        e = copy_planes(dev_in, host_in, h, r.first, r.second, es, cudaMemcpyHostToDevice, h->s_in);
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[s], h->s_in);
  }
  if (e != cudaSuccess) return fail(h, user, hyd::record_cuda_error(e));
  // advance each slab when its input is in; return it at once
  hydro_params p2 = *p;
  p2.workspace = ws2;
  p2.workspace_bytes = ws2_bytes;
  const hydro_params* pc[2] = {p, &p2};
  for (int s = 0; s < h->nslab; ++s) {
    const int k = s & 1;
    e = cudaStreamWaitEvent(c[k], h->ev_in[s], 0);
    if (e != cudaSuccess) return fail(h, user, hyd::record_cuda_error(e));
    int rc = hydro_advance_uniform_zrange(pc[k], dev_in, dev_out, h->X, h->Y, h->Z, h->N, h->bc, h->zb[s],
                                          h->zb[s + 1], flux, dev_status, c[k]);
    if (rc != HYDRO_OK) return fail(h, user, rc);
    e = cudaEventRecord(h->ev_comp[s], c[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, h->ev_comp[s], 0);
    if (e == cudaSuccess)
      e = copy_planes(host_out, dev_out, h, h->zb[s], h->zb[s + 1], es, cudaMemcpyDeviceToHost, h->s_out);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_out[s], h->s_out);
    if (e != cudaSuccess) return fail(h, user, hyd::record_cuda_error(e));
  }
  // next dt from the whole new state, after both compute streams
  e = cudaEventRecord(h->ev_c1, c[1]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c[0], h->ev_c1, 0);
  if (e != cudaSuccess) return fail(h, user, hyd::record_cuda_error(e));
  // (one reduction over the whole box: per-slab reductions interleaved with
  // the slab kernels measured slower, their CTAs competing for the SMs)
  int rc = hydro_cfl_dt(dev_out, 1, 5 * XYZ, XYZ, XYZ, p->precision, p->gamma, p->dens_floor, p->pres_floor, p->dx,
                        cfl, const_cast<double*>(p->dt_dev), nullptr, red_ws, red_ws_bytes, c[0]);
  if (rc != HYDRO_OK) return fail(h, user, rc);
  // dt to the host on the same stream, before the next step's reduction can
  // overwrite it (the next step's advances wait for ev_cfl)
  if (host_dt) e = cudaMemcpyAsync(host_dt, p->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, c[0]);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_cfl, c[0]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, h->ev_cfl, 0);
  // the caller's stream resumes after the copies out (which follow everything)
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_done, h->s_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, h->ev_done, 0);
  if (e != cudaSuccess) return fail(h, user, hyd::record_cuda_error(e));
  h->has_prev = true;
  h->prev_host_out = host_out;
  h->prev_dev_in = dev_in;
  h->prev_dev_out = dev_out;
  return HYDRO_OK;
}

size_t hydro_pipeline_workspace_bytes(const hydro_pipeline* h) { return h ? hydro_cfl_workspace_bytes() : 0; }

int hydro_pipeline_plan(int Z, int N, int ghost, int bc, int nslab, const int* layers, int* zb, int* chunks) {
  if (!zb || !chunks || N <= 0 || Z <= 0 || Z % N || ghost < 0 || ghost >= N) return HYDRO_EINVAL;
  if (bc != HYDRO_BC_PERIODIC && bc != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
  int rc = slab_bounds(Z, N, nslab, layers, zb);
  if (rc != HYDRO_OK) return rc;
  plan_ranges(Z, ghost, bc, nslab, zb, reinterpret_cast<int(*)[4]>(chunks));
  return HYDRO_OK;
}

int hydro_pipeline_destroy(hydro_pipeline* h) {
  if (h) release(h);
  return HYDRO_OK;
}

}  // extern "C"
