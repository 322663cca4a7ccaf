"""The C-ABI library builds for sm_103a and exports every entry point include/mpm.h declares
(CPU only: loading the library makes no CUDA call)."""
import ctypes
import os

from paper_1810_01054_gb300 import build as B
from paper_1810_01054_gb300 import mpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpm.h")


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    so = ctypes.CDLL(path)
    names = mpm.header_symbols(HEADER)
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_signatures_cover_the_header():
    names = set(mpm.header_symbols(HEADER))
    assert names == set(mpm._SIGS), names ^ set(mpm._SIGS)


def _header_fields(start_marker, end_marker):
    import re
    text = open(HEADER).read()
    body = text[text.index("typedef struct {", text.index(start_marker)):]
    body = body[: body.index(end_marker)]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip().replace("typedef struct {", "").strip()
        if not decl:
            continue
        for part in decl.split(","):
            fields.append(re.findall(r"[A-Za-z_][A-Za-z0-9_]*", part.split("[")[0])[-1])
    return fields


def test_scene_descriptor_layout_matches_header():
    """The ctypes mirror of mpm_scene_desc lists the header's fields in the header's order."""
    assert _header_fields("MPM_IMPL_PLAIN", "} mpm_scene_desc;") == [f[0] for f in mpm.SceneDesc._fields_]


def test_fp64_descriptor_layout_matches_header():
    """The same for mpm_scene64_desc, and the field types are the header's double/int ones."""
    import ctypes as C
    assert _header_fields("typedef struct mpm_scene64 mpm_scene64;", "} mpm_scene64_desc;") == \
        [f[0] for f in mpm.SceneDesc64._fields_]
    types = dict(mpm.SceneDesc64._fields_)
    for name in ("dx", "dt", "E", "nu", "p_mass", "p_vol"):
        assert types[name] is C.c_double
    assert types["wall_c"]._type_ is C.c_double and types["gravity"]._type_ is C.c_double
