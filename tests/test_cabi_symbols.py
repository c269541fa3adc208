"""The C-ABI library builds here (nvcc cross-compiles sm_103a without a GPU),
loads, and exports every entry point the headers in include/ declare.  No compute
call is made (there is no GPU in the CPU suite)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(hydro_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared()
    for n in ("hydro_advance", "hydro_advance_uniform", "hydro_advance_uniform_zrange", "hydro_advance_levels", "hydro_gather_uniform",
              "hydro_cfl_dt", "hydro_required_ghost", "hydro_strerror", "hydro_amr_map", "hydro_amr_prepare",
              "hydro_amr_reflux", "hydro_amr_restrict"):
        assert n in names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no nvcc")
def test_library_exports_every_declared_symbol():
    from paper_1103_3373_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in declared():
        assert hasattr(lib, n), n
    # host-only calls (no device needed)
    assert lib.hydro_required_ghost(0, 0) == 2 and lib.hydro_required_ghost(2, 1) == 3
    assert lib.hydro_required_ghost(1, 1) == 4 and lib.hydro_required_ghost(5, 0) < 0
    lib.hydro_strerror.restype = ctypes.c_char_p
    assert lib.hydro_strerror(-2).decode().startswith("ghost")


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no nvcc")
def test_zrange_arguments_are_checked_on_the_host():
    """hydro_advance_uniform_zrange rejects a slab that is not a range of
    whole group layers inside the box before any device work (the pointers
    are never dereferenced on these paths)."""
    from paper_1103_3373_gb300 import hydro as H
    lib = H._lib()
    p = H.Params(scheme=H.CTU, recon=H.PPM, riemann=H.RS_ROE, precision=H.FP32, dt=0.1, dx=(0.5, 0.5, 0.5)).c()
    f = lib.hydro_advance_uniform_zrange
    a, b = ctypes.c_void_p(16), ctypes.c_void_p(32)
    for z0, z1 in ((8, 32), (0, 40), (32, 16), (-16, 16), (0, 80)):
        assert f(ctypes.byref(p), a, b, 32, 32, 64, 16, 0, z0, z1, None, None, None) == H.EINVAL, (z0, z1)
    assert f(ctypes.byref(p), a, b, 32, 32, 64, 8, 0, 0, 16, None, None, None) == H.EUNSUPPORTED
    assert f(ctypes.byref(p), a, a, 32, 32, 64, 16, 0, 0, 16, None, None, None) == H.EINVAL


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1103_3373_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_binding_marshals_its_structs():
    """Host-side marshalling of the binding (no device call): parameter and
    level structs build from Python values with the header's field order."""
    from paper_1103_3373_gb300 import hydro as H
    p = H.Params(scheme=H.CTU, recon=H.PPM, riemann=H.RS_ROE, precision=H.FP32, dt=0.1, dx=(0.5, 0.25, 0.125))
    c = p.c()
    assert (c.scheme, c.recon, c.riemann, c.precision) == (H.CTU, H.PPM, H.RS_ROE, H.FP32)
    assert tuple(c.dx) == (0.5, 0.25, 0.125) and c.dt == 0.1
    names = [f[0] for f in H._CParams._fields_]
    assert names[:6] == ["scheme", "recon", "limiter", "riemann", "roe_fallback", "precision"]
    a = H._CAmrLevel(1, 2, 3, 4, 5, 6, 7)
    assert (a.G, a.X, a.Y, a.Z) == (4, 5, 6, 7)
    assert [f[0] for f in H._CAmrLevel._fields_] == ["U", "origin", "map", "G", "X", "Y", "Z"]


def _header_struct_fields(src, name):
    """Field names of `typedef struct name { ... } name;` in declaration order."""
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            names.append(re.sub(r"\[.*\]", "", part).replace("*", " ").split()[-1])
    return names


def test_binding_structs_follow_the_header():
    """The ctypes mirrors of hydro_params and hydro_level list the header's
    fields in the header's order."""
    from paper_1103_3373_gb300 import hydro as H
    src = open(os.path.join(ROOT, "include", "hydro.h")).read()
    assert _header_struct_fields(src, "hydro_params") == [f[0] for f in H._CParams._fields_]
    assert _header_struct_fields(src, "hydro_level") == [f[0] for f in H._CLevel._fields_]


def test_python_constants_match_the_header():
    """Sizes the binding copies from include/hydro.h (the no-allocation
    entry point's scratch limit, the level-table size) are the header's."""
    from paper_1103_3373_gb300 import hydro as H
    src = open(os.path.join(ROOT, "include", "hydro.h")).read()
    macro = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(HYDRO_\w+)\s+\(?(-?\d+)u?\)?", src)}
    assert macro["HYDRO_NOALLOC_MAX_PARTIALS"] == H.NOALLOC_MAX_PARTIALS
    assert macro["HYDRO_NOALLOC_CELLS_PER_CTA"] == H.NOALLOC_CELLS_PER_CTA
    assert H.NOALLOC_MAX_CELLS == (macro["HYDRO_NOALLOC_MAX_PARTIALS"] // 3) * macro["HYDRO_NOALLOC_CELLS_PER_CTA"]
    assert macro["HYDRO_MAX_LEVELS"] == H.MAX_LEVELS
    for name in ("ETOOBIG", "EINVAL", "EGHOST", "EUNSUPPORTED", "ECUDA", "EWORKSPACE"):
        assert macro["HYDRO_" + name] == getattr(H, name), name
    for name in ("ST_ROE_FALLBACK", "ST_NEG_DENS", "ST_NEG_PRES", "ST_NAN", "ST_EXACT_FAIL"):
        assert macro["HYDRO_" + name] == getattr(H, name), name


# query and error calls, and the measurement kernel: no passage of the paper
# defines them
NO_PASSAGE = {"hydro_required_ghost", "hydro_workspace_bytes", "hydro_max_block_threads", "hydro_strerror",
              "hydro_last_cuda_error", "hydro_cfl_workspace_bytes", "hydro_cfl_boxes_workspace_bytes",
              "hydro_fma_peak"}


def test_every_call_cites_its_passage():
    """Each declaration of the C ABI has one comment block headed by its name
    that cites the section of the paper defining the operation (query, error
    and measurement calls excepted)."""
    missing = []
    for path in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        src = open(path).read()
        blocks = re.findall(r"/\*.*?\*/", src, re.S)
        for name in re.findall(r"^(?:int|size_t|const char\*|double|void)\s+(hydro_\w+)\s*\(", src, re.M):
            if name in NO_PASSAGE:
                continue
            # the block whose heading is "name — ..."
            heads = [b for b in blocks if re.search(r"(?:^/\*|\n \*)\s*%s\b[^\n]*\u2014" % name, b)]
            if len(heads) != 1 or "Sec." not in heads[0]:
                missing.append(name)
    assert not missing, missing


def test_readme_c_example_compiles_against_the_header(tmp_path):
    """The C example in README.md is valid C99 against include/hydro.h."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    import subprocess
    src = open(os.path.join(ROOT, "README.md")).read()
    code = re.search(r"```c\n(.*?)```", src, re.S).group(1)
    f = tmp_path / "example.c"
    f.write_text(code)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I" + os.path.join(ROOT, "include"),
                        str(f)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_cfl_box_interior_description_is_checked_on_the_host():
    """hydro_cfl_dt_boxes refuses a malformed description of halo-padded
    groups (ghost > 0) before any device work, and lets a well-formed one
    through to its workspace check (the pointers are never dereferenced on
    these paths)."""
    from paper_1103_3373_gb300 import hydro as H
    lib = H._lib()
    lib.hydro_cfl_dt_boxes.restype = ctypes.c_int
    n, g = 16, 3
    M = n + 2 * g

    def box(**kw):
        arr = (H._CCflBox * 1)()
        e = arr[0]
        e.U, e.dt_dev = 16, 32
        e.G, e.group_stride, e.var_stride, e.cells = 4, 5 * M ** 3, M ** 3, n ** 3
        for d in range(3):
            e.dx[d] = 0.1
        e.dt_scale, e.interior_n, e.ghost = 1.0, n, g
        for k, v in kw.items():
            setattr(e, k, v)
        return arr

    def call(arr, ws=None, nbytes=0):
        return lib.hydro_cfl_dt_boxes(arr, 1, H.FP32, ctypes.c_double(1.4), ctypes.c_double(0.0),
                                      ctypes.c_double(0.0), ctypes.c_double(0.4), None, ws, ctypes.c_size_t(nbytes),
                                      None)

    for kw in (dict(ghost=-1), dict(interior_n=0), dict(cells=n ** 3 - 1), dict(var_stride=M ** 3 - 1),
               dict(cells=M ** 3)):
        assert call(box(**kw)) == H.EINVAL, kw
    assert call(box()) == H.EWORKSPACE
    assert call(box(ghost=0, cells=M ** 3, interior_n=0)) == H.EWORKSPACE  # contiguous cells
