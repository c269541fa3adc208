/*
 * hydro_amr.h — device-side AMR level operations around the patch-group
 * solver of libhydro (arXiv:1103.3373).
 *
 * Sec. 4.2 names the preparation step's spatial and temporal interpolation
 * of the ghost zones of patch groups next to coarse-fine boundaries (the
 * bottleneck of the paper's CPU preparation step); Sec. 2 step (5) stores
 * the fluxes across patch-group boundaries for the coarse-grid correction
 * that Sec. 4.3 lists among the CPU tasks.  Here all of it runs on the GPU:
 *
 *   hydro_amr_map       group map of a level (slot -> group index)
 *   hydro_amr_prepare   halo-padded input of every group of a level
 *                       (copy from same-level groups, else interpolation
 *                       from the parent level in space and time)
 *   hydro_amr_reflux    coarse cells next to coarse-fine faces take the
 *                       fine fluxes of the two substeps instead of their own
 *   hydro_amr_restrict  coarse cells covered by a fine group take the mean
 *                       of their 8 fine cells
 *
 * Conventions (the paper gives none of these formulas; the library and its
 * tests take one reading, stated here):
 *   - refinement ratio 2 in space and time; the finer level takes two
 *     substeps of dt/2 per step of its parent;
 *   - a level covers whole patch groups of N^3 cells (N = 16); a refined
 *     coarse group is covered by the 8 fine groups of twice the resolution
 *     over it (an octet), so every coarse-fine face lies on a coarse group
 *     face, where step (5) stored the coarse flux;
 *   - proper nesting: the cells a fine ghost zone and its interpolation
 *     stencil need exist at the fine level or at the parent level;
 *   - prolongation, per conserved component: u = ((Uc + qx) + qy) + qz,
 *     q_d = (s_d / 4) minmod(Uc[+e_d] - Uc, Uc - Uc[-e_d]), s_d = -1 for the
 *     lower child along d and +1 for the upper one; the 8 children average
 *     to the parent;
 *   - time interpolation: Uc(theta) = U^n + theta (U^{n+1} - U^n);
 *   - refluxing: Fbar = 0.125 (S0 + S1), S_k = ((F_k[a0][b0] + F_k[a0][b1])
 *     + F_k[a1][b0]) + F_k[a1][b1] over the 2 x 2 fine faces of the coarse
 *     face; U += -h (Fbar - Fc) on the cell's +d face, +h (Fbar - Fc) on its
 *     -d face, h = dt / dx_d, faces in the order -x, +x, -y, +y, -z, +z;
 *   - restriction: 0.125 x the sum of the 8 fine cells in the order
 *     (dz, dy, dx) = 000, 001, 010, 011, 100, 101, 110, 111.
 *
 * Arrays (device memory, caller-owned, storage type per precision: double for
 * HYDRO_FP64, float for HYDRO_FP32 and HYDRO_FP32_MIXED; the arithmetic is
 * done in the storage type):
 *   group data   [G][5][N][N][N], x fastest;
 *   padded input [G][5][M][M][M], M = N + 2*ghost (hydro_advance's U_in);
 *   face fluxes  [G][6][5][N][N] as hydro_advance writes them: faces -x, +x,
 *                -y, +y, -z, +z; [a][b] = [z][y] on x faces, [z][x] on y
 *                faces, [y][x] on z faces;
 *   group map    int [Z/N][Y/N][X/N].
 *
 * Errors: the return value reports argument errors (HYDRO_EINVAL,
 * HYDRO_EUNSUPPORTED for N != 16) and launch failures (HYDRO_ECUDA);
 * inconsistencies only the data can show (a cell missing at both levels, two
 * groups on one slot) set bits in the optional device word dev_error
 * (HYDRO_AMR_E*) and the affected outputs are written as NaN (prepare) or
 * left unchanged (reflux, restrict).  No kernel traps or waits.
 */
#ifndef HYDRO_AMR_H
#define HYDRO_AMR_H

#include <stddef.h>

#include "hydro.h"

#ifdef __cplusplus
extern "C" {
#endif

#define HYDRO_AMR_ENESTING 1u  /* a needed cell exists at neither level     */
#define HYDRO_AMR_EDUPLICATE 2u /* two groups on one slot of a group map    */
#define HYDRO_AMR_EOCTET 4u    /* a refined group without its full octet    */

/* One level of the hierarchy. */
typedef struct hydro_amr_level {
  void* U;              /* [G][5][N][N][N]: read, or corrected in place (reflux, restrict target) */
  const int* origin;    /* int[G][3]: (x, y, z) interior corner in this level's cells, multiples of N */
  const int* map;       /* int[Z/N][Y/N][X/N]: group index on each slot, -1 where none             */
  int G;                /* groups of the level                                                    */
  int X, Y, Z;          /* extent of the level in its own cells (2^l x the base box)              */
} hydro_amr_level;

/*
 * hydro_amr_map — the level lookup that the preparation step (Sec. 4.2) and
 * the corrections (Sec. 4.3) use: fill map (int[Z/N][Y/N][X/N]) with -1,
 * then store each group's index at its slot origin/N.  Origins must be multiples of N inside
 * the box (else HYDRO_EINVAL is not detectable on the host: such groups set
 * HYDRO_AMR_ENESTING and are skipped); a slot claimed twice sets
 * HYDRO_AMR_EDUPLICATE.
 */
int hydro_amr_map(const int* origin, int G, int X, int Y, int Z, int N, int* map, unsigned* dev_error,
                  void* stream);

/*
 * hydro_amr_prepare — the preparation step (Sec. 4.2) on the device: the
 * halo-padded input [G][5][M][M][M] of every group of `fine`.  A cell (in
 * fine coordinates, mapped into the box by bc) inside a group of `fine` is
 * copied from fine->U; any other cell is interpolated from `coarse` (the
 * parent level, NULL for the base level) at time theta of the parent's
 * step: coarse->U holds its state before the step, coarse_new after it
 * (NULL when theta == 0).
 *   bc      HYDRO_BC_PERIODIC or HYDRO_BC_OUTFLOW at every level.
 *   ghost   >= hydro_required_ghost of the scheme that reads U_out.
 */
int hydro_amr_prepare(const hydro_amr_level* fine, const hydro_amr_level* coarse, const void* coarse_new,
                      double theta, int bc, int N, int ghost, int precision, void* U_out, unsigned* dev_error,
                      void* stream);

/*
 * hydro_amr_reflux — the coarse-grid correction by the stored fluxes
 * (Sec. 2 step (5), Sec. 4.3): every cell of coarse->U (the parent's data
 * after its step, corrected in place) that is not covered by `fine` and
 * shares a face with a refined coarse group replaces that face's coarse flux
 * (coarse_flux, the parent step's output) by the mean of the fine fluxes of
 * the two substeps (fine_flux0, fine_flux1, outputs of the fine level's
 * steps).  dt and dx are the parent's.
 */
int hydro_amr_reflux(const hydro_amr_level* coarse, const void* coarse_flux, const hydro_amr_level* fine,
                     const void* fine_flux0, const void* fine_flux1, double dt, const double* dx, int bc, int N,
                     int precision, unsigned* dev_error, void* stream);

/*
 * hydro_amr_restrict — the correction of the coarse-grid data (Sec. 4.3): every
 * coarse cell of coarse->U covered by a group of
 * `fine` (fine->U after its last substep) takes the mean of its 8 fine
 * cells (in place).
 */
int hydro_amr_restrict(const hydro_amr_level* fine, const hydro_amr_level* coarse, int N, int precision,
                       unsigned* dev_error, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_AMR_H */
