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


def test_scene_descriptor_layout_matches_header():
    """The ctypes mirror of mpm_scene_desc lists the header's fields in the header's order."""
    import re
    text = open(HEADER).read()
    body = text[text.index("typedef struct {", text.index("MPM_IMPL_PLAIN")):]
    body = body[: body.index("} mpm_scene_desc;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip().replace("typedef struct {", "").strip()
        if not decl:
            continue
        for part in decl.split(","):
            name = re.findall(r"[A-Za-z_][A-Za-z0-9_]*", part.split("[")[0])[-1]
            fields.append(name)
    assert fields == [f[0] for f in mpm.SceneDesc._fields_]
