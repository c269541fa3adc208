"""Python binding of libhydro (include/hydro.h): argument marshalling only.

Each function has the name of the C entry point it calls and takes torch CUDA
tensors (device memory and streams come from PyTorch); every step of the
computation runs in the library's kernels.  There is no CPU fallback: if
libhydro.so is missing or no GPU is present the calls raise.
"""
import ctypes
import os
from dataclasses import dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhydro.so")

# enumerations (include/hydro.h; Sec. 2 of the paper)
MHM, VL, CTU, RTVD, WAF = 0, 1, 2, 3, 4
PLM, PPM = 0, 1
LIM_MINMOD, LIM_VANLEER, LIM_VANALBADA, LIM_HYBRID = 0, 1, 2, 3
RS_EXACT, RS_HLLE, RS_HLLC, RS_ROE = 0, 1, 2, 3
FP64, FP32, FP32_MIXED = 0, 1, 2
BC_PERIODIC, BC_OUTFLOW = 0, 1
OK, EINVAL, EGHOST, EUNSUPPORTED, ECUDA, EWORKSPACE, ETOOBIG = 0, -1, -2, -3, -4, -5, -6
NOALLOC_MAX_PARTIALS, NOALLOC_CELLS_PER_CTA = 8192, 65536
NOALLOC_MAX_CELLS = (NOALLOC_MAX_PARTIALS // 3) * NOALLOC_CELLS_PER_CTA
ST_ROE_FALLBACK, ST_NEG_DENS, ST_NEG_PRES, ST_NAN, ST_EXACT_FAIL = 1, 2, 4, 8, 16
ST_ERROR_MASK = ST_NEG_DENS | ST_NEG_PRES | ST_NAN | ST_EXACT_FAIL
MAX_LEVELS = 32
AMR_ENESTING, AMR_EDUPLICATE, AMR_EOCTET = 1, 2, 4  # include/hydro_amr.h dev_error bits

SCHEMES = {"mhm": MHM, "vl": VL, "ctu": CTU, "rtvd": RTVD, "waf": WAF}
RECONS = {"plm": PLM, "ppm": PPM}
SOLVERS = {"exact": RS_EXACT, "hlle": RS_HLLE, "hllc": RS_HLLC, "roe": RS_ROE}
LIMITERS = {"minmod": LIM_MINMOD, "vanleer": LIM_VANLEER, "vanalbada": LIM_VANALBADA, "hybrid": LIM_HYBRID}
PRECISIONS = {"fp64": FP64, "fp32": FP32, "mixed": FP32_MIXED}


class HydroError(RuntimeError):
    def __init__(self, code, where):
        msg = "%s: %s" % (where, _lib().hydro_strerror(code).decode())
        if code == ECUDA:
            msg += " (%s)" % _lib().hydro_last_cuda_error().decode()
        super().__init__(msg)
        self.code = code


class _CParams(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("recon", ctypes.c_int), ("limiter", ctypes.c_int),
                ("riemann", ctypes.c_int), ("roe_fallback", ctypes.c_int), ("precision", ctypes.c_int),
                ("theta", ctypes.c_double), ("gamma", ctypes.c_double), ("dt", ctypes.c_double),
                ("dx", ctypes.c_double * 3), ("dens_floor", ctypes.c_double), ("pres_floor", ctypes.c_double),
                ("dt_dev", ctypes.c_void_p), ("block_threads", ctypes.c_int), ("grid_ctas", ctypes.c_int),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("characteristic", ctypes.c_int), ("split_order", ctypes.c_int), ("chain", ctypes.c_int),
                ("zrun", ctypes.c_void_p)]


class _CLevel(ctypes.Structure):
    _fields_ = [("U_in", ctypes.c_void_p), ("U_out", ctypes.c_void_p), ("flux", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("dt_dev", ctypes.c_void_p), ("dt", ctypes.c_double),
                ("dx", ctypes.c_double * 3), ("G", ctypes.c_int), ("mode", ctypes.c_int), ("bc", ctypes.c_int),
                ("X", ctypes.c_int), ("Y", ctypes.c_int), ("Z", ctypes.c_int), ("zrun", ctypes.c_void_p)]


class _CAmrLevel(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p), ("origin", ctypes.c_void_p), ("map", ctypes.c_void_p),
                ("G", ctypes.c_int), ("X", ctypes.c_int), ("Y", ctypes.c_int), ("Z", ctypes.c_int)]


@dataclass
class Params:
    """hydro_params.  dt_dev / workspace are torch tensors (or None)."""
    scheme: int = CTU
    recon: int = PPM
    limiter: int = LIM_MINMOD
    riemann: int = RS_ROE
    roe_fallback: int = RS_HLLE
    precision: int = FP32
    theta: float = 1.0
    gamma: float = 1.4
    dt: float = 0.0
    dx: tuple = field(default_factory=lambda: (1.0, 1.0, 1.0))
    dens_floor: float = 0.0
    pres_floor: float = 0.0
    dt_dev: object = None
    block_threads: int = 0
    grid_ctas: int = 0
    workspace: object = None
    characteristic: int = 0  # 1: PLM / PPM on characteristic variables (Sec. 2)
    split_order: int = 0     # RTVD / WAF: sweeps x, y, z (0) or z, y, x (1)
    chain: int = 0           # uniform fields: z-segment / chain length (0 = whole columns, <= CHAIN_MAX)
    zrun: object = None      # prepared groups: device int32 [G] runs of z-continuations (zrun_of)

    def c(self):
        p = _CParams()
        for k in ("scheme", "recon", "limiter", "riemann", "roe_fallback", "precision", "block_threads",
                  "grid_ctas", "characteristic", "split_order", "chain"):
            setattr(p, k, int(getattr(self, k)))
        for k in ("theta", "gamma", "dt", "dens_floor", "pres_floor"):
            setattr(p, k, float(getattr(self, k)))
        for d in range(3):
            p.dx[d] = float(self.dx[d])
        p.dt_dev = _ptr(self.dt_dev, "dt_dev", dtype="float64") if self.dt_dev is not None else None
        p.zrun = _ptr(self.zrun, "zrun", dtype="int32") if self.zrun is not None else None
        if self.workspace is not None:
            p.workspace = self.workspace.data_ptr()
            p.workspace_bytes = self.workspace.numel() * self.workspace.element_size()
        return p


class _CCflBox(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p), ("G", ctypes.c_int), ("group_stride", ctypes.c_longlong),
                ("var_stride", ctypes.c_longlong), ("cells", ctypes.c_longlong), ("dx", ctypes.c_double * 3),
                ("dt_dev", ctypes.c_void_p), ("smax_dev", ctypes.c_void_p), ("dt_scale", ctypes.c_double),
                ("interior_n", ctypes.c_int), ("ghost", ctypes.c_int)]


CFL_MAX_BOXES = 256
CHAIN_MAX = 32

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhydro.so is not built (run __graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, ll, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        P = ctypes.POINTER(_CParams)
        L.hydro_required_ghost.argtypes = [i, i]
        L.hydro_workspace_bytes.argtypes = [P, i]
        L.hydro_workspace_bytes.restype = ctypes.c_size_t
        L.hydro_max_block_threads.argtypes = [P, i]
        L.hydro_advance.argtypes = [P, vp, vp, vp, i, i, i, vp, vp]
        L.hydro_advance_uniform.argtypes = [P, vp, vp, i, i, i, i, i, vp, vp, vp]
        L.hydro_advance_levels.argtypes = [P, ctypes.POINTER(_CLevel), i, i, i, vp]
        L.hydro_advance_uniform_zrange.argtypes = [P, vp, vp, i, i, i, i, i, i, i, vp, vp, vp]
        L.hydro_pipeline_create.argtypes = [i, i, i, i, i, i, i, vp, ctypes.POINTER(vp)]
        L.hydro_pipeline_step.argtypes = [vp, P, vp, vp, vp, vp, vp, vp, vp, d, vp, ctypes.c_size_t, vp,
                                          ctypes.c_size_t, vp]
        L.hydro_pipeline_destroy.argtypes = [vp]
        L.hydro_pipeline_workspace_bytes.argtypes = [vp]
        L.hydro_pipeline_workspace_bytes.restype = ctypes.c_size_t
        L.hydro_pipeline_plan.argtypes = [i, i, i, i, i, vp, vp, vp]
        L.hydro_gather_uniform.argtypes = [vp, i, i, i, i, vp, i, i, i, i, vp, vp]
        L.hydro_cfl_workspace_bytes.argtypes = []
        L.hydro_cfl_workspace_bytes.restype = ctypes.c_size_t
        L.hydro_cfl_dt.argtypes = [vp, i, ll, ll, ll, i, d, d, d, ctypes.POINTER(ctypes.c_double), d, vp, vp, vp,
                                   ctypes.c_size_t, vp]
        L.hydro_conserved_totals.argtypes = [vp, i, ll, ll, ll, i, vp, vp, ctypes.c_size_t, vp]
        L.hydro_cfl_dt_noalloc.argtypes = [vp, i, ll, ll, ll, i, d, d, d, ctypes.POINTER(ctypes.c_double), d, vp,
                                           vp, vp]
        A = ctypes.POINTER(_CAmrLevel)
        L.hydro_amr_map.argtypes = [vp, i, i, i, i, i, vp, vp, vp]
        L.hydro_amr_prepare.argtypes = [A, A, vp, d, i, i, i, i, vp, vp, vp]
        L.hydro_amr_reflux.argtypes = [A, vp, A, vp, vp, d, ctypes.POINTER(ctypes.c_double), i, i, i, vp, vp]
        L.hydro_amr_restrict.argtypes = [A, A, i, i, vp, vp]
        L.hydro_cfl_boxes_workspace_bytes.argtypes = []
        L.hydro_cfl_boxes_workspace_bytes.restype = ctypes.c_size_t
        L.hydro_cfl_dt_boxes.argtypes = [ctypes.POINTER(_CCflBox), i, i, d, d, d, d, vp, vp, ctypes.c_size_t, vp]
        L.hydro_fma_peak.argtypes = [i, i, i, i, vp, vp, ctypes.POINTER(ctypes.c_double)]
        L.hydro_strerror.argtypes = [i]
        L.hydro_strerror.restype = ctypes.c_char_p
        L.hydro_last_cuda_error.argtypes = []
        L.hydro_last_cuda_error.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


def library():
    """The loaded ctypes library (loads it on first use)."""
    return _lib()


def _storage_dtype(precision):
    return "float64" if precision == FP64 else "float32"


def _ptr(t, name, dtype=None):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA tensor" % name)
    if dtype is not None and str(t.dtype).split(".")[-1] != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc, where):
    if rc != OK:
        raise HydroError(rc, where)


def hydro_required_ghost(scheme, recon):
    return _lib().hydro_required_ghost(int(scheme), int(recon))


def hydro_workspace_bytes(params: Params, N=16):
    return int(_lib().hydro_workspace_bytes(ctypes.byref(params.c()), N))


def hydro_max_block_threads(params: Params, N=16):
    return int(_lib().hydro_max_block_threads(ctypes.byref(params.c()), N))


def hydro_advance(params: Params, U_in, U_out, flux=None, status=None, N=16, ghost=None, stream=None):
    """One step of the groups in U_in [G,5,M,M,M] -> U_out [G,5,N,N,N]."""
    dt = _storage_dtype(params.precision)
    G = U_in.shape[0]
    M = U_in.shape[-1]
    g = (M - N) // 2 if ghost is None else ghost
    rc = _lib().hydro_advance(ctypes.byref(params.c()), _ptr(U_in, "U_in", dt), _ptr(U_out, "U_out", dt),
                              _ptr(flux, "flux", dt), G, N, g, _ptr(status, "status", "int32"), _stream(stream))
    _check(rc, "hydro_advance")


def hydro_advance_uniform(params: Params, field_in, field_out, bc=BC_PERIODIC, flux=None, status=None, N=16,
                          stream=None):
    """One step of a uniform box [5,Z,Y,X] tiled by N^3 groups, gather fused."""
    dt = _storage_dtype(params.precision)
    _, Z, Y, X = field_in.shape
    rc = _lib().hydro_advance_uniform(ctypes.byref(params.c()), _ptr(field_in, "field_in", dt),
                                      _ptr(field_out, "field_out", dt), X, Y, Z, N, bc, _ptr(flux, "flux", dt),
                                      _ptr(status, "status", "int32"), _stream(stream))
    _check(rc, "hydro_advance_uniform")


def hydro_advance_uniform_zrange(params: Params, field_in, field_out, z_begin, z_end, bc=BC_PERIODIC, flux=None,
                                 status=None, N=16, stream=None):
    """hydro_advance_uniform for the groups of the z-slab [z_begin, z_end)
    only (halos still read from the whole field_in); flux and status keep
    the whole box's group order."""
    dt = _storage_dtype(params.precision)
    _, Z, Y, X = field_in.shape
    rc = _lib().hydro_advance_uniform_zrange(ctypes.byref(params.c()), _ptr(field_in, "field_in", dt),
                                             _ptr(field_out, "field_out", dt), X, Y, Z, N, bc, int(z_begin),
                                             int(z_end), _ptr(flux, "flux", dt), _ptr(status, "status", "int32"),
                                             _stream(stream))
    _check(rc, "hydro_advance_uniform_zrange")


def _host_ptr(t, name, dtype=None):
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous host tensor" % name)
    if dtype is not None and str(t.dtype).split(".")[-1] != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    return t.data_ptr()


def pipeline_plan(Z, ghost, bc=BC_PERIODIC, slabs=8, N=16):
    """The copy plan of a Pipeline (host only): slab boundaries zb (planes)
    and, per slab, the input plane ranges whose copy completes its input and
    halo, in copy order."""
    if isinstance(slabs, (list, tuple)):
        n, lay = len(slabs), (ctypes.c_int * len(slabs))(*[int(a) for a in slabs])
    else:
        n, lay = int(slabs), None
    zb = (ctypes.c_int * (max(n, 0) + 1))()
    ch = (ctypes.c_int * (4 * max(n, 1)))()
    _check(_lib().hydro_pipeline_plan(Z, N, ghost, bc, n, lay, zb, ch), "hydro_pipeline_plan")
    chunks = [[(ch[4 * s + k], ch[4 * s + k + 1]) for k in (0, 2) if ch[4 * s + k + 1] > ch[4 * s + k]]
              for s in range(n)]
    return list(zb), chunks


class Pipeline:
    """hydro_pipeline (include/hydro_pipeline.h): the end-to-end step of a
    uniform box held in page-locked host memory, copies overlapped with the
    solver on z-slabs (Sec. 4.1).  slabs: a count (even split of the group
    layers) or a list of group layers per slab."""

    def __init__(self, X, Y, Z, ghost, bc=BC_PERIODIC, slabs=8, N=16):
        if isinstance(slabs, (list, tuple)):
            n, lay = len(slabs), (ctypes.c_int * len(slabs))(*[int(a) for a in slabs])
        else:
            n, lay = int(slabs), None
        h = ctypes.c_void_p()
        _check(_lib().hydro_pipeline_create(X, Y, Z, N, ghost, bc, n, lay, ctypes.byref(h)), "hydro_pipeline_create")
        self._h = h
        self.shape = (5, Z, Y, X)
        self.nslab = n
        self.workspace_bytes = int(_lib().hydro_pipeline_workspace_bytes(h))

    def step(self, params: Params, host_in, host_out, dev_in, dev_out, cfl, red_ws, host_dt=None, flux=None,
             status=None, ws2=None, stream=None):
        dt = _storage_dtype(params.precision)
        for a in (host_in, host_out, dev_in, dev_out):
            if tuple(a.shape) != self.shape:
                raise ValueError("field shape %s, pipeline planned for %s" % (tuple(a.shape), self.shape))
        rc = _lib().hydro_pipeline_step(self._h, ctypes.byref(params.c()), _host_ptr(host_in, "host_in", dt),
                                        _host_ptr(host_out, "host_out", dt), _host_ptr(host_dt, "host_dt", "float64"),
                                        _ptr(dev_in, "dev_in", dt), _ptr(dev_out, "dev_out", dt),
                                        _ptr(flux, "flux", dt), _ptr(status, "status", "int32"), float(cfl),
                                        red_ws.data_ptr(), red_ws.numel() * red_ws.element_size(),
                                        ws2.data_ptr() if ws2 is not None else None,
                                        ws2.numel() * ws2.element_size() if ws2 is not None else 0, _stream(stream))
        _check(rc, "hydro_pipeline_step")

    def close(self):
        if getattr(self, "_h", None) and _LIB is not None:
            _LIB.hydro_pipeline_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()


@dataclass
class Level:
    """One hydro_level entry: prepared groups (mode 0) or a uniform field (mode 1)."""
    U_in: object
    U_out: object
    dx: tuple
    dt: float = 0.0
    dt_dev: object = None
    flux: object = None
    status: object = None
    mode: int = 0
    bc: int = BC_PERIODIC
    zrun: object = None  # mode 0: device int32 [G] runs of z-continuations (hydro_params.zrun)


def make_levels(levels, precision):
    dt = _storage_dtype(precision)
    arr = (_CLevel * max(1, len(levels)))()
    for k, lv in enumerate(levels):
        c = arr[k]
        c.U_in = _ptr(lv.U_in, "U_in", dt)
        c.U_out = _ptr(lv.U_out, "U_out", dt)
        c.flux = _ptr(lv.flux, "flux", dt)
        c.status = _ptr(lv.status, "status", "int32")
        c.dt_dev = _ptr(lv.dt_dev, "dt_dev", "float64")
        c.dt = float(lv.dt)
        for d in range(3):
            c.dx[d] = float(lv.dx[d])
        c.mode = int(lv.mode)
        if lv.mode == 0:
            c.G = lv.U_in.shape[0]
            c.zrun = _ptr(lv.zrun, "zrun", "int32") if lv.zrun is not None else None
        else:
            c.bc = int(lv.bc)
            _, c.Z, c.Y, c.X = (int(s) for s in lv.U_in.shape)
    return arr


def hydro_advance_levels(params: Params, levels, N=16, ghost=3, stream=None, _carray=None):
    """One persistent launch over all entries of `levels` (list of Level)."""
    if len(levels) > MAX_LEVELS:
        raise ValueError("at most %d entries per call" % MAX_LEVELS)
    arr = _carray if _carray is not None else make_levels(levels, params.precision)
    rc = _lib().hydro_advance_levels(ctypes.byref(params.c()), arr, len(levels), N, ghost, _stream(stream))
    _check(rc, "hydro_advance_levels")


def hydro_gather_uniform(field, origins, U_out, N=16, ghost=3, bc=BC_PERIODIC, precision=FP32, stream=None):
    dt = _storage_dtype(precision)
    _, Z, Y, X = field.shape
    G = origins.shape[0]
    rc = _lib().hydro_gather_uniform(_ptr(field, "field", dt), X, Y, Z, bc, _ptr(origins, "origins", "int32"), G, N,
                                     ghost, precision, _ptr(U_out, "U_out", dt), _stream(stream))
    _check(rc, "hydro_gather_uniform")


def hydro_cfl_workspace_bytes():
    return int(_lib().hydro_cfl_workspace_bytes())


def _red_layout(U):
    """(G, group_stride, var_stride, cells) of a field [5,...] or groups [G,5,...]."""
    if U.shape[0] == 5 and U.dim() in (2, 4):
        cells = U[0].numel()
        return 1, 5 * cells, cells, cells
    G = U.shape[0]
    cells = U[0, 0].numel()
    return G, 5 * cells, cells, cells


def hydro_cfl_dt(U, dx, cfl, dt_out, workspace, gamma=1.4, dens_floor=0.0, pres_floor=0.0, precision=FP32,
                 smax_out=None, stream=None):
    dt = _storage_dtype(precision)
    G, gs, vs, cells = _red_layout(U)
    dxa = (ctypes.c_double * 3)(*[float(a) for a in dx])
    rc = _lib().hydro_cfl_dt(_ptr(U, "U", dt), G, gs, vs, cells, precision, gamma, dens_floor, pres_floor, dxa,
                             float(cfl), _ptr(dt_out, "dt_out", "float64"), _ptr(smax_out, "smax_out", "float64"),
                             workspace.data_ptr(), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "hydro_cfl_dt")


def hydro_conserved_totals(U, totals_out, workspace, precision=FP32, stream=None):
    dt = _storage_dtype(precision)
    G, gs, vs, cells = _red_layout(U)
    rc = _lib().hydro_conserved_totals(_ptr(U, "U", dt), G, gs, vs, cells, precision,
                                       _ptr(totals_out, "totals_out", "float64"), workspace.data_ptr(),
                                       workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "hydro_conserved_totals")


def hydro_cfl_dt_noalloc(U, dx, cfl, dt_out, gamma=1.4, dens_floor=0.0, pres_floor=0.0, precision=FP32,
                         smax_out=None, stream=None):
    """hydro_cfl_dt without a workspace: for callers that cannot allocate
    device memory (its scratch is a fixed static device array; at most
    NOALLOC_MAX_CELLS cells per call)."""
    dt = _storage_dtype(precision)
    G, gs, vs, cells = _red_layout(U)
    dxa = (ctypes.c_double * 3)(*[float(a) for a in dx])
    rc = _lib().hydro_cfl_dt_noalloc(_ptr(U, "U", dt), G, gs, vs, cells, precision, gamma, dens_floor, pres_floor,
                                     dxa, float(cfl), _ptr(dt_out, "dt_out", "float64"),
                                     _ptr(smax_out, "smax_out", "float64"), _stream(stream))
    _check(rc, "hydro_cfl_dt_noalloc")


def hydro_cfl_boxes_workspace_bytes():
    return int(_lib().hydro_cfl_boxes_workspace_bytes())


def make_cfl_boxes(boxes, precision):
    """ctypes table for hydro_cfl_dt_boxes from (U, dx, dt_out[, dt_scale[,
    smax_out[, ghost]]]) tuples: U a contiguous field [5,Z,Y,X] or groups
    [G,5,...]; dt_out / smax_out 1-element float64 device tensors; ghost > 0:
    U holds halo-padded groups [G,5,M,M,M] and only their (M - 2 ghost)^3
    interior cells count."""
    dt = _storage_dtype(precision)
    arr = (_CCflBox * len(boxes))()
    for k, b in enumerate(boxes):
        U, dx, dt_out = b[0], b[1], b[2]
        scale = float(b[3]) if len(b) > 3 else 1.0
        smax = b[4] if len(b) > 4 else None
        ghost = int(b[5]) if len(b) > 5 else 0
        G, gs, vs, cells = _red_layout(U)
        e = arr[k]
        e.U = _ptr(U, "U", dt)
        e.G, e.group_stride, e.var_stride, e.cells = G, gs, vs, cells
        if ghost > 0:
            if U.dim() != 5 or U.shape[1] != 5 or not (U.shape[2] == U.shape[3] == U.shape[4]):
                raise ValueError("ghost > 0 needs halo-padded groups [G,5,M,M,M]")
            n = U.shape[-1] - 2 * ghost
            e.interior_n, e.ghost, e.cells = n, ghost, n ** 3
        for d_ in range(3):
            e.dx[d_] = float(dx[d_])
        e.dt_dev = _ptr(dt_out, "dt_out", "float64")
        e.smax_dev = _ptr(smax, "smax_out", "float64")
        e.dt_scale = scale
    return arr


def hydro_cfl_dt_boxes(boxes, cfl, workspace, dt_min_out=None, gamma=1.4, dens_floor=0.0, pres_floor=0.0,
                       precision=FP32, stream=None, _carray=None):
    """CFL dt of every box in one pass (at most CFL_MAX_BOXES per call); see
    make_cfl_boxes for the tuples.  dt_min_out receives min_b dt_scale_b dt_b."""
    arr = _carray if _carray is not None else make_cfl_boxes(boxes, precision)
    rc = _lib().hydro_cfl_dt_boxes(arr, len(arr), precision, gamma, dens_floor, pres_floor, float(cfl),
                                   _ptr(dt_min_out, "dt_min_out", "float64"), _ptr(workspace, "workspace"),
                                   workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "hydro_cfl_dt_boxes")


# ---------------------------------------------------------------- peaks (include/hydro_peaks.h)
PEAK_FP32, PEAK_FP32X2, PEAK_FP64 = 0, 1, 2


def hydro_fma_peak(kind, ctas, threads, iters, out, stream=None):
    """Enqueue one FMA-loop launch; returns its exact flop count (the caller
    times it).  `out` holds ctas * threads floats (doubles for PEAK_FP64)."""
    fl = ctypes.c_double(0.0)
    n = ctas * threads
    if out.numel() < n:
        raise ValueError("out must hold ctas * threads elements")
    rc = _lib().hydro_fma_peak(int(kind), int(ctas), int(threads), int(iters),
                               _ptr(out, "out", "float64" if kind == PEAK_FP64 else "float32"), _stream(stream),
                               ctypes.byref(fl))
    _check(rc, "hydro_fma_peak")
    return fl.value


# ---------------------------------------------------------------- AMR (include/hydro_amr.h)

@dataclass
class AmrLevel:
    """One level of an AMR hierarchy: U [G][5][N][N][N] (storage dtype),
    origin int32 [G][3] (x, y, z corner in the level's cells), map int32
    [Z/N][Y/N][X/N] (hydro_amr_map), box (X, Y, Z) in the level's cells."""
    U: object
    origin: object
    map: object
    box: tuple

    def c(self, precision):
        X, Y, Z = (int(a) for a in self.box)
        G = int(self.origin.shape[0])
        return _CAmrLevel(_ptr(self.U, "U", _storage_dtype(precision)), _ptr(self.origin, "origin", "int32"),
                          _ptr(self.map, "map", "int32"), G, X, Y, Z)


def hydro_amr_map(origin, box, map_out, N=16, error=None, stream=None):
    """Group map of a level: map_out int32 [Z/N][Y/N][X/N] <- group index or -1."""
    X, Y, Z = (int(a) for a in box)
    G = int(origin.shape[0])
    rc = _lib().hydro_amr_map(_ptr(origin, "origin", "int32") if G else None, G, X, Y, Z, N,
                              _ptr(map_out, "map", "int32"), _ptr(error, "error", "int32"), _stream(stream))
    _check(rc, "hydro_amr_map")


def hydro_amr_prepare(fine: AmrLevel, coarse, coarse_new, theta, U_out, bc=BC_PERIODIC, N=16, ghost=3,
                      precision=FP32, error=None, stream=None):
    """Halo-padded input [G][5][M][M][M] of every group of `fine` (copy from
    the level, else interpolation from `coarse` at time theta)."""
    dt = _storage_dtype(precision)
    cf = fine.c(precision)
    cc = coarse.c(precision) if coarse is not None else None
    rc = _lib().hydro_amr_prepare(ctypes.byref(cf), ctypes.byref(cc) if cc is not None else None,
                                  _ptr(coarse_new, "coarse_new", dt), float(theta), bc, N, ghost, precision,
                                  _ptr(U_out, "U_out", dt), _ptr(error, "error", "int32"), _stream(stream))
    _check(rc, "hydro_amr_prepare")


def hydro_amr_reflux(coarse: AmrLevel, coarse_flux, fine: AmrLevel, fine_flux0, fine_flux1, dt, dx,
                     bc=BC_PERIODIC, N=16, precision=FP32, error=None, stream=None):
    """Coarse-grid correction of coarse.U (in place) by the fine fluxes of the
    two substeps."""
    st = _storage_dtype(precision)
    cc, cf = coarse.c(precision), fine.c(precision)
    dxa = (ctypes.c_double * 3)(*[float(a) for a in dx])
    rc = _lib().hydro_amr_reflux(ctypes.byref(cc), _ptr(coarse_flux, "coarse_flux", st), ctypes.byref(cf),
                                 _ptr(fine_flux0, "fine_flux0", st), _ptr(fine_flux1, "fine_flux1", st), float(dt),
                                 dxa, bc, N, precision, _ptr(error, "error", "int32"), _stream(stream))
    _check(rc, "hydro_amr_reflux")


def hydro_amr_restrict(fine: AmrLevel, coarse: AmrLevel, N=16, precision=FP32, error=None, stream=None):
    """Coarse cells covered by fine groups take the mean of their 8 fine cells
    (coarse.U in place)."""
    cf, cc = fine.c(precision), coarse.c(precision)
    rc = _lib().hydro_amr_restrict(ctypes.byref(cf), ctypes.byref(cc), N, precision, _ptr(error, "error", "int32"),
                                   _stream(stream))
    _check(rc, "hydro_amr_restrict")
