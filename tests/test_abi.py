"""The C-ABI library builds, loads and exports every entry point include/pic.h declares
(no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(pic_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("pic_init", "pic_step", "pic_field_solve", "pic_moments", "pic_destroy"):
        assert name in d


def test_library_exports_every_declared_symbol():
    from paper_1001_2969_gb300 import build

    path = build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1001_2969_gb300 import pic

    for n in _declared():
        assert hasattr(pic, n) or n in ("pic_status_string",), n


def test_status_strings_without_gpu():
    from paper_1001_2969_gb300 import pic

    L = pic.lib()
    assert L.pic_status_string(0) == b"ok"
    assert L.pic_status_string(2) == b"capacity exceeded"


def test_init_rejects_bad_config_without_touching_the_gpu():
    """Validation happens before any CUDA call: a bad mesh is PIC_ERR_ARG."""
    import workloads as W
    from paper_1001_2969_gb300 import pic

    cfg = W.config("c1", nz=34)  # nz - 1 not a power of two
    with pytest.raises(pic.PicError) as e:
        pic.pic_init(cfg, torch_memory=False, stream=0)
    assert e.value.status == pic.PIC_ERR_ARG
