/*
 * libhydro — GB300 (sm_103a) directionally unsplit Riemann-solver fluid update
 * of a batch of AMR patch groups (3D Euler equations of an ideal gas).
 *
 * Method: Schive, Zhang & Chiueh, "Directionally Unsplit Hydrodynamic Schemes
 * with Hybrid MPI/OpenMP/GPU Parallelization in AMR" (arXiv:1103.3373).
 *   Sec. 2      the MHM, VL and 6-solve CTU schemes; PLM/PPM reconstruction
 *               with the generalized minmod, van Leer, van Albada and hybrid
 *               limiters; exact, HLLE, HLLC and Roe solvers with the Roe
 *               failure fallback; the five CTU steps (reconstruct + trace,
 *               Riemann, transverse correction + Riemann, conservative
 *               update, store the patch-boundary fluxes).
 *   Sec. 3.1    one patch group = 2x2x2 patches of 8^3 cells (16^3 cells)
 *               plus ghost zones, computed by one thread block; arrays
 *               flattened as [z][y][x] with x fastest.
 *   Sec. 4.1    solver input / output arrays are group-major, contiguous per
 *               group ([groups][size per group]).
 *   Sec. 4.2    the preparation step (ghost-zone gather) and Sec. 4.3 the
 *               evolution time step, here device kernels.
 *
 * Conventions shared by every entry point
 *   - Conserved variables, in this order: rho, rho*u, rho*v, rho*w, E.
 *   - A "group" holds N^3 interior cells (N = 16, or 8 for single patches).
 *     Group input  U_in : [G][5][M][M][M], M = N + 2*ghost, x fastest.
 *     Group output U_out: [G][5][N][N][N].
 *     Boundary flux     : [G][6][5][N][N]; faces -x,+x,-y,+y,-z,+z; the two
 *                         transverse indices in [z][y][x] order with the
 *                         normal one removed; time-centred flux F (not dt*F),
 *                         positive along +axis.
 *     Uniform field     : [5][Z][Y][X].
 *   - Storage precision: FP64 -> double; FP32 and FP32_MIXED -> float.
 *   - All pointers named *_dev or documented as "device" are device memory
 *     owned by the caller; the library never allocates, frees or keeps them.
 *   - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *     void*; NULL = legacy default stream).  No call synchronises the device,
 *     except where stated.
 *   - Return value: HYDRO_OK or a negative HYDRO_E* code for argument,
 *     configuration or launch errors, detected synchronously.  Numerical
 *     failures are reported asynchronously through the per-group status word.
 *     The library never traps.
 */
#ifndef HYDRO_H
#define HYDRO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- enumerations (Sec. 2) ---------------------------------------------- */
enum { HYDRO_MHM = 0, HYDRO_VL = 1, HYDRO_CTU = 2,                  /* scheme: unsplit */
       HYDRO_RTVD = 3, HYDRO_WAF = 4 };                                /* split (Sec. 3.2) */
enum { HYDRO_PLM = 0, HYDRO_PPM = 1 };                               /* recon    */
enum { HYDRO_LIM_MINMOD = 0, HYDRO_LIM_VANLEER = 1,                  /* limiter  */
       HYDRO_LIM_VANALBADA = 2, HYDRO_LIM_HYBRID = 3 };
enum { HYDRO_RS_EXACT = 0, HYDRO_RS_HLLE = 1, HYDRO_RS_HLLC = 2,     /* Riemann  */
       HYDRO_RS_ROE = 3 };
enum { HYDRO_FP64 = 0, HYDRO_FP32 = 1, HYDRO_FP32_MIXED = 2 };       /* precision */
enum { HYDRO_BC_PERIODIC = 0, HYDRO_BC_OUTFLOW = 1 };                /* box edge  */

/* ---- return codes ----------------------------------------------------------- */
#define HYDRO_OK 0
#define HYDRO_EINVAL (-1)       /* bad argument (null pointer, size, enum)        */
#define HYDRO_EGHOST (-2)       /* ghost width below what the scheme needs        */
#define HYDRO_EUNSUPPORTED (-3) /* valid but not built (e.g. N other than 16)     */
#define HYDRO_ECUDA (-4)        /* a CUDA call failed (see hydro_last_cuda_error) */
#define HYDRO_EWORKSPACE (-5)   /* workspace missing or smaller than required     */
#define HYDRO_ETOOBIG (-6)      /* input larger than a fixed-size entry point takes */

/* ---- per-group status bits (written, not OR-ed, once per group and call) --- */
#define HYDRO_ST_ROE_FALLBACK 1u /* informational: Roe failed at >= 1 face and the
                                    fallback solver was used there (Sec. 2)       */
#define HYDRO_ST_NEG_DENS 2u     /* an updated density <= 0                      */
#define HYDRO_ST_NEG_PRES 4u     /* an updated pressure <= 0                     */
#define HYDRO_ST_NAN 8u          /* NaN in the updated state                     */
#define HYDRO_ST_EXACT_FAIL 16u  /* exact solver: vacuum or no convergence       */
#define HYDRO_ST_ERROR_MASK (HYDRO_ST_NEG_DENS | HYDRO_ST_NEG_PRES | HYDRO_ST_NAN | HYDRO_ST_EXACT_FAIL)

/*
 * Parameters of one step (Sec. 2).
 *   theta        generalized-minmod parameter, 1 <= theta <= 2 (also bounds
 *                the hybrid limiter).
 *   roe_fallback solver used where Roe's linearisation fails: HLLE, HLLC or
 *                EXACT (Sec. 2).  Ignored for other solvers.
 *   dt, dx[3]    time step and cell widths.  If dt_dev is non-NULL the step
 *                reads dt from that device double instead (so a device-side
 *                CFL reduction can feed it without a host round trip).
 *   dens_floor, pres_floor  floors applied as max(q, floor) whenever
 *                primitive variables are recovered (0 disables).
 *   block_threads  threads per CTA; 0 = the library default (the autotuner
 *                  sets it).  Must be a multiple of 32 and <= the kernel's
 *                  maximum (hydro_max_block_threads).
 *   grid_ctas    CTAs of the persistent launch; 0 = one per SM (x the
 *                resident count).
 *   workspace    device scratch for the FP64 kernels (their stage buffers do
 *                not fit in shared memory); size from hydro_workspace_bytes.
 *                May be NULL when that size is 0.
 *   characteristic  0: PLM / PPM act on the primitive variables; 1: on the
 *                characteristic variables (Sec. 2: the reconstruction "can
 *                be applied to either"): the stencil is projected on the left
 *                eigenvectors of the primitive Jacobian at the cell along the
 *                sweep, each wave is reconstructed with the same scalar PLM /
 *                PPM and limiter, and the faces are projected back with the
 *                right eigenvectors.  Same ghost widths.
 *   split_order  HYDRO_RTVD / HYDRO_WAF only: the sweeps of a step run
 *                x, y, z (0) or z, y, x (1); alternate them between steps
 *                (Strang).  The other schemes ignore it.
 *   chain        uniform fields (hydro_advance_uniform*, mode-1 levels) of
 *                the unsplit schemes: a CTA streams through runs of up to
 *                `chain` z-consecutive groups without restarting (the ghost
 *                planes between them are traced and solved once), 1 <= chain
 *                <= HYDRO_CHAIN_MAX; 0 = min(group layers, HYDRO_CHAIN_MAX).
 *                The work list takes the box in z-segments of `chain`
 *                layers, every column's first segment before any second
 *                one, so CTAs on neighbouring columns pass the same layers
 *                at about the same time and share their halo planes in L2.
 *                Results do not depend on it (the autotuner picks it).
 *                For prepared groups with zrun it caps the runs a CTA
 *                streams through (0 = HYDRO_CHAIN_MAX).
 *   zrun         prepared groups (hydro_advance; hydro_level.zrun for
 *                hydro_advance_levels): device int[G] or NULL.  zrun[g] >= 1
 *                is the number of groups g, g+1, ... each of which continues
 *                the one before it along +z: its interior lies directly
 *                above, and the ghost zones of the two hold each other's
 *                interior values (as a gather or the AMR ghost preparation
 *                from one level makes them).  A CTA then streams through up
 *                to `chain` such groups without restarting, reading the
 *                planes between them from the interiors.  Values are
 *                clamped to [1, groups left in the entry]; NULL = every
 *                group alone.  Used by the unsplit schemes (the split ones
 *                advance every group alone): a launch with runs runs a
 *                variant of the kernel, whose results equal byte for byte
 *                those of the same launch with runs of one (every group
 *                alone), and those of a launch without runs to rounding
 *                (FP64 byte for byte).
 *
 * The split schemes (the directionally split comparison schemes of Sec.
 * 3.2): RTVD = relaxing TVD in the flux-split form of Trac & Pen (2003),
 * freezing speed |u_n| + c_s, first-order half step, limited full step;
 * WAF = Toro's TVD weighted average flux on the HLLC fan, the limiter
 * applied to the upwind/local ratio of each wave's density jump.  Both use
 * `limiter` / `theta`; recon, characteristic and riemann are ignored.
 */
typedef struct hydro_params {
  int scheme, recon, limiter, riemann, roe_fallback, precision;
  double theta, gamma, dt;
  double dx[3];
  double dens_floor, pres_floor;
  const double* dt_dev;
  int block_threads, grid_ctas;
  void* workspace;
  size_t workspace_bytes;
  int characteristic;
  int split_order;
  int chain;
  const int* zrun;
} hydro_params;

/* Ghost layers the scheme needs (Sec. 2): MHM and CTU 2 (PLM) / 3 (PPM);
 * VL 3 (PLM) / 4 (PPM); RTVD 3 and WAF 2 (any recon).  Returns HYDRO_EINVAL
 * for unknown enums. */
int hydro_required_ghost(int scheme, int recon);

/* Device scratch (bytes) hydro_advance* needs for this configuration and
 * launch shape; 0 for the FP32 forms (their stage buffers live in shared
 * memory). */
size_t hydro_workspace_bytes(const hydro_params* p, int N);

/* Largest block_threads the (scheme, recon, riemann, precision) kernel was
 * built for, or a negative error code. */
int hydro_max_block_threads(const hydro_params* p, int N);

/*
 * hydro_advance — one step of G patch groups (Sec. 2 steps (1)-(5); Sec. 3.1
 * one CTA per group, run as a persistent loop over the groups).
 *   U_in       device [G][5][M][M][M], read only.  Interior + ghost zones.
 *   U_out      device [G][5][N][N][N]; must not alias U_in.
 *   flux       device [G][6][5][N][N] or NULL: fluxes through the six faces
 *              of each group (step (5), for the coarse-fine correction).
 *   dev_status device unsigned[G] or NULL: HYDRO_ST_* bits of each group.
 *   G >= 0 (0 is a no-op), N = 16 (the only group size built; others
 *   return HYDRO_EUNSUPPORTED), ghost >= hydro_required_ghost.
 */
int hydro_advance(const hydro_params* p, const void* U_in, void* U_out, void* flux, int G, int N, int ghost,
                  unsigned* dev_status, void* stream);

/*
 * hydro_gather_uniform — the preparation step (Sec. 4.2) on the device:
 * halo-padded groups from a uniform field.
 *   field   device [5][Z][Y][X] (storage type per precision).
 *   origin  device int[G][3]: interior corner (x0, y0, z0) of each group.
 *   bc      HYDRO_BC_PERIODIC or HYDRO_BC_OUTFLOW (zero gradient).
 *   U_out   device [G][5][M][M][M], M = N + 2*ghost.
 */
int hydro_gather_uniform(const void* field, int X, int Y, int Z, int bc, const int* origin, int G, int N, int ghost,
                         int precision, void* U_out, void* stream);

/*
 * hydro_advance_uniform — the preparation step's gather (Sec. 4.2) fused into
 * the step of Sec. 2 for a uniform box tiled by N^3 groups (group index (gz*GY + gy)*GX + gx): every CTA reads its
 * groups' halos straight from field_in with the boundary condition bc and
 * writes their interiors to field_out (double buffering; no aliasing).  Each
 * CTA takes a contiguous run of groups in column order (z fastest) and
 * streams through the z-consecutive ones without restarting; the bytes of
 * field_out, flux and dev_status are those of the same groups advanced one by
 * one (gather + hydro_advance), whatever the launch shape.
 *   field_in, field_out  device [5][Z][Y][X]; X, Y, Z multiples of N.
 *   flux, dev_status     as hydro_advance, indexed by that group order.
 */
int hydro_advance_uniform(const hydro_params* p, const void* field_in, void* field_out, int X, int Y, int Z, int N,
                          int bc, void* flux, unsigned* dev_status, void* stream);

/*
 * hydro_advance_uniform_zrange — hydro_advance_uniform restricted to the
 * groups whose interior lies in z_begin <= z < z_end (multiples of N): the
 * halos are still read from the whole field_in (periodic / outflow as bc),
 * only those groups' cells of field_out, flux and dev_status (full-box group
 * order) are written.  Lets a caller overlap the host transfers of one z-slab
 * with the computation of another (Sec. 4.1, asynchronous memory copy).
 * z_begin and z_end must be multiples of N with 0 <= z_begin <= z_end <= Z
 * (else HYDRO_EINVAL, checked before any device work); z_begin == z_end is a
 * no-op.  Slabs of one step may run concurrently on several streams provided
 * each launch has its own workspace (FP64 forms); they write disjoint cells.
 */
int hydro_advance_uniform_zrange(const hydro_params* p, const void* field_in, void* field_out, int X, int Y, int Z,
                                 int N, int bc, int z_begin, int z_end, void* flux, unsigned* dev_status,
                                 void* stream);

/* One entry of a multi-level (or multi-box) batch. */
typedef struct hydro_level {
  const void* U_in;     /* groups [G][5][M^3] (mode 0) or field [5][Z][Y][X] (mode 1) */
  void* U_out;          /* groups [G][5][N^3] (mode 0) or field (mode 1)              */
  void* flux;           /* [G][6][5][N][N] or NULL                                    */
  unsigned* status;     /* [G] or NULL                                                */
  const double* dt_dev; /* optional device dt of this entry (overrides dt)            */
  double dt;
  double dx[3];
  int G;                /* groups (mode 0); ignored in mode 1 (derived from X, Y, Z)  */
  int mode;             /* 0 = prepared groups, 1 = uniform field with bc             */
  int bc, X, Y, Z;      /* mode 1 only                                                */
  const int* zrun;      /* mode 0: device int[G] runs of z-continuations, or NULL
                           (as hydro_params.zrun)                                    */
} hydro_level;

/* Most entries one hydro_advance_levels call accepts. */
#define HYDRO_MAX_LEVELS 32
#define HYDRO_CHAIN_MAX 32

/*
 * hydro_advance_levels — one persistent launch (Sec. 3.1: patch groups to
 * thread blocks; Sec. 4.3: every level with its own time step) that advances
 * uneven per-AMR-level group lists (or independent boxes) in one go: the work of all
 * entries is one flat list of groups shared round-robin by the CTAs.  Every
 * entry has its own dx and dt; scheme, reconstruction, limiter, solver,
 * precision and ghost width come from p (p->dt and p->dx are ignored).
 *   nlev in [0, HYDRO_MAX_LEVELS].
 */
int hydro_advance_levels(const hydro_params* p, const hydro_level* levels, int nlev, int N, int ghost, void* stream);

/*
 * hydro_cfl_dt — evolution time step (Sec. 4.3) as a device reduction:
 *   dt = cfl / max over cells of max_d (|v_d| + c) / dx_d,  c = sqrt(gamma p / rho),
 * with primitives recovered with the floors.  The per-cell speeds are
 * evaluated in the storage precision; the maxima, the division by dx and dt
 * in FP64 (for FP64 data the result is exactly the FP64 formula above).
 *   U        device, element (g, v, i) at U[g*group_stride + v*var_stride + i],
 *            i < cells, g < G (a field: G = 1, var_stride = cells = X*Y*Z).
 *   dt_dev   device double[1]: receives dt.  smax_dev (optional) receives the
 *            maximum signal speed / dx.
 *   workspace device scratch of hydro_cfl_workspace_bytes() bytes.
 */
size_t hydro_cfl_workspace_bytes(void);
int hydro_cfl_dt(const void* U, int G, long long group_stride, long long var_stride, long long cells, int precision,
                 double gamma, double dens_floor, double pres_floor, const double* dx, double cfl, double* dt_dev,
                 double* smax_dev, void* workspace, size_t workspace_bytes, void* stream);

/*
 * hydro_conserved_totals — global sums of the five conserved variables (the
 * quantities that the conservative update of Sec. 2 step (4) keeps) over
 * the same addressing as hydro_cfl_dt, accumulated in FP64 (the
 * conservation check of the mixed-precision form).
 *   totals_dev  device double[5].
 */
int hydro_conserved_totals(const void* U, int G, long long group_stride, long long var_stride, long long cells,
                           int precision, double* totals_dev, void* workspace, size_t workspace_bytes, void* stream);

/*
 * hydro_cfl_dt_boxes — the CFL time step (Sec. 4.3) of many independent
 * boxes (or AMR levels) in one pass: three launches whatever the number of
 * boxes, instead of two per box.  Box b is laid out as for hydro_cfl_dt (G
 * groups of 5 variables: U + g*group_stride + v*var_stride + i, i < cells;
 * a uniform field is G = 1, var_stride = cells = X*Y*Z) in `precision`'s
 * storage type, and gets its own dt in dt_dev (device double; max speed /
 * dx in smax_dev if not NULL).  Each box's dt equals hydro_cfl_dt's on the
 * same data bit for bit.
 *   dt_min_dev  (device double, may be NULL) min over boxes of
 *               dt_scale * dt_b, NaN if any dt_b is NaN: with dt_scale = 2^l
 *               for level l of an AMR hierarchy stepped with dt_l = dt_0 /
 *               2^l, the largest dt_0 that satisfies every level.
 *   workspace   device scratch of hydro_cfl_boxes_workspace_bytes() bytes.
 * 1 <= nbox <= HYDRO_CFL_MAX_BOXES (call again for more).  Returns
 * HYDRO_OK, HYDRO_EINVAL (null pointer, nbox out of range, G or cells < 0,
 * dx or dt_scale not positive and finite, gamma <= 1, cfl <= 0, ghost < 0,
 * or ghost > 0 with interior_n < 1, cells != interior_n^3 or var_stride
 * below M^3),
 * HYDRO_EWORKSPACE, or HYDRO_ECUDA.  Allocates nothing.
 */
#define HYDRO_CFL_MAX_BOXES 256
typedef struct hydro_cfl_box {
  const void* U;
  int G;
  long long group_stride, var_stride, cells;
  double dx[3];
  double* dt_dev;
  double* smax_dev;
  double dt_scale;
  /* ghost > 0: each group is a halo-padded cube of M = interior_n + 2 ghost
   * cells per edge (x fastest, at U + g*group_stride + v*var_stride), cells
   * = interior_n^3, and only the interior cells are reduced: the time step
   * of a level of halo-prepared groups, whose ghost cells belong to other
   * groups or are interpolated from the coarser level.  var_stride must be
   * at least M^3.  ghost = 0: the cells of a group are contiguous (above). */
  int interior_n, ghost;
} hydro_cfl_box;
size_t hydro_cfl_boxes_workspace_bytes(void);
int hydro_cfl_dt_boxes(const hydro_cfl_box* boxes, int nbox, int precision, double gamma, double dens_floor,
                       double pres_floor, double cfl, double* dt_min_dev, void* workspace, size_t workspace_bytes,
                       void* stream);

/*
 * hydro_cfl_dt_noalloc — hydro_cfl_dt (the time step of Sec. 4.3) for callers
 * that cannot allocate device memory.  The paper has no counterpart: it serves code that runs where no
 * allocator is reachable, e.g. a plug-in enqueued inside another framework's
 * CUDA graph capture (where cudaMalloc is not allowed) or a host runtime
 * that hands out only the input and output buffers.  It allocates nothing
 * and calls no allocating routine: its scratch (three FP64 partial maxima
 * per CTA, one per direction) is a static device array of
 * HYDRO_NOALLOC_MAX_PARTIALS doubles (64 KiB) that every GPU which loads the
 * library keeps until the process exits.  Each CTA reduces
 * HYDRO_NOALLOC_CELLS_PER_CTA cells, so G * cells may be at most
 * (HYDRO_NOALLOC_MAX_PARTIALS / 3) * HYDRO_NOALLOC_CELLS_PER_CTA (1.79e8; a
 * 512^3 box fits); larger inputs return HYDRO_ETOOBIG before anything is
 * launched.
 *   Arguments, result and numerics are those of hydro_cfl_dt (dt_dev and
 *   smax_dev are device outputs the caller provides), including empty
 *   inputs (G == 0 or cells == 0 give dt = +inf); no workspace argument.
 *   The first call on a device looks up the array's device address (with
 *   that device current) and caches it: make that first call before any
 *   stream capture.  The cached address belongs to the device's primary
 *   context and is assumed to live as long as the process: after a
 *   cudaDeviceReset the cache is stale, so do not reset a device that this
 *   entry point has used.  Every call shares the one array and leaves its partials
 *   in it; nothing in it needs to start at zero (each call writes every
 *   partial it reads).  Calls that overlap on the GPU (different streams or
 *   host threads at once) race on the array: serialise them.
 */
#define HYDRO_NOALLOC_MAX_PARTIALS 8192
#define HYDRO_NOALLOC_CELLS_PER_CTA 65536
int hydro_cfl_dt_noalloc(const void* U, int G, long long group_stride, long long var_stride, long long cells,
                         int precision, double gamma, double dens_floor, double pres_floor, const double* dx,
                         double cfl, double* dt_dev, double* smax_dev, void* stream);

/* Text for a return code. */
const char* hydro_strerror(int code);

/* The last CUDA error string seen by the library on this thread ("" if none). */
const char* hydro_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_H */
