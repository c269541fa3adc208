/*
 * libhydro — end-to-end step of a uniform box whose state lives in host
 * memory, with the host<->device copies overlapped with the solver.
 *
 * Sec. 4.1 (asynchronous memory copy): the patch groups of one call are split
 * into chunks and CUDA streams let the copies of one chunk run while the
 * solver works on another.  Here the chunks are z-slabs of whole group layers
 * of a uniform field [5][Z][Y][X]:
 *   - a copy-in stream sends the slabs in an order that completes each slab's
 *     halo (ghost planes of its neighbours, periodic wrap first);
 *   - slab s is advanced (hydro_advance_uniform_zrange) as soon as its input
 *     and halo have arrived, alternately on two compute streams so that the
 *     last CTAs of one slab overlap the first of the next;
 *   - a copy-out stream returns slab s while later slabs are advanced;
 *   - after the last slab, the CFL reduction of the whole new state
 *     (hydro_cfl_dt) writes the next dt to p->dt_dev, and dt is copied out;
 *   - consecutive steps on rotating buffers overlap: the next step's
 *     copy-in of a slab starts once this step has returned the slabs it
 *     covers (see hydro_pipeline_step).
 * Each copy is one cudaMemcpy2DAsync over the five variables of a z-range.
 * The result equals hydro_advance_uniform + hydro_cfl_dt on the whole box bit
 * for bit.
 *
 * The pipeline object owns host memory, four CUDA streams and its events (on
 * the device current at creation); it never allocates device memory.  Between
 * calls it keeps the last step's buffer addresses, only to recognise a
 * chained step; it never reads through them.
 */
#ifndef HYDRO_PIPELINE_H
#define HYDRO_PIPELINE_H

#include <stddef.h>

#include "hydro.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hydro_pipeline hydro_pipeline;

/*
 * hydro_pipeline_create — the asynchronous-copy scheme of Sec. 4.1: plan the
 * slabs of an X x Y x Z box (multiples of N)
 * for schemes needing at most `ghost` halo cells (hydro_required_ghost).
 *   nslab >= 1 slabs; layers = NULL splits the Z/N group layers evenly, else
 *   layers[s] >= 1 group layers of slab s (sum Z/N).
 *   bc: HYDRO_BC_PERIODIC or HYDRO_BC_OUTFLOW (fixes the halo order).
 * Returns HYDRO_EINVAL for bad sizes / layers / ghost >= N,
 * HYDRO_EUNSUPPORTED for N != 16, HYDRO_ECUDA if streams or events cannot be
 * created.  *out is set only on HYDRO_OK.
 */
int hydro_pipeline_create(int X, int Y, int Z, int N, int ghost, int bc, int nslab, const int* layers,
                          hydro_pipeline** out);

/*
 * hydro_pipeline_step — one step with its copies overlapped (Sec. 4.1); its
 * completion (state and dt on the host)
 * is ordered before later work on `stream`.  No host synchronisation.
 *   Chained steps: when host_in is the last step's host_out, dev_in is
 *   neither of the last step's device buffers and dev_out is not the last
 *   step's dev_out (three device buffers in rotation: in = D[2n % 3],
 *   out = D[(2n+1) % 3]), the step is ordered after the last step only:
 *   each input chunk waits for the last step's copy-out of the slabs it
 *   covers, and the advances wait for the last step's dt.  Its copy-in thus
 *   overlaps the end of the last step.  Work the caller put on `stream`
 *   after the last step is then not waited for.  Any other step (the first
 *   one, or other buffers) starts after the work already on `stream`.
 *   p        scheme parameters; p->dt_dev is required (read as this step's dt,
 *            then overwritten with the next dt); p->workspace serves the
 *            first compute stream;
 *   host_in  [5][Z][Y][X] state U^n, page-locked host memory (pageable
 *            memory works but is not overlapped);
 *   host_out [5][Z][Y][X] new state, page-locked; may not alias host_in;
 *   host_dt  optional (NULL): the next dt, page-locked;
 *   dev_in, dev_out  device fields of the same shape (distinct);
 *   flux, dev_status optional, as hydro_advance_uniform (whole-box order);
 *   cfl      Courant number of the next dt;
 *   red_ws   hydro_pipeline_workspace_bytes(h) of device scratch;
 *   ws2      the second compute stream's scratch (hydro_workspace_bytes(p);
 *            may be NULL when that is 0).
 * Returns HYDRO_EINVAL for bad arguments (also a scheme needing more halo
 * than the plan's ghost), the codes of hydro_advance_uniform_zrange and
 * hydro_cfl_dt, or HYDRO_ECUDA.
 */
int hydro_pipeline_step(hydro_pipeline* h, const hydro_params* p, const void* host_in, void* host_out,
                        double* host_dt, void* dev_in, void* dev_out, void* flux, unsigned* dev_status, double cfl,
                        void* red_ws, size_t red_ws_bytes, void* ws2, size_t ws2_bytes, void* stream);

/* hydro_pipeline_workspace_bytes — device scratch hydro_pipeline_step needs
 * as red_ws (the CFL reduction's, Sec. 4.3); 0 for NULL. */
size_t hydro_pipeline_workspace_bytes(const hydro_pipeline* h);

/*
 * hydro_pipeline_plan — the copy plan (Sec. 4.1) hydro_pipeline_create makes, on the
 * host only (no device call): zb[nslab+1] slab boundaries (planes) and, per
 * slab, up to two input plane ranges chunks[s] = {lo0, hi0, lo1, hi1} (an
 * empty range has lo = hi) whose copy completes slab s's input and halo, in
 * copy order.  Same argument rules as hydro_pipeline_create (N need not be
 * 16 here); HYDRO_EINVAL otherwise.
 */
int hydro_pipeline_plan(int Z, int N, int ghost, int bc, int nslab, const int* layers, int* zb, int* chunks);

/* hydro_pipeline_destroy — release the streams and events of the Sec. 4.1 scheme
 * and the object (NULL: no-op).  Synchronises the pipeline's own streams first. */
int hydro_pipeline_destroy(hydro_pipeline* h);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_PIPELINE_H */
