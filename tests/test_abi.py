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


def _c_layout(tmp_path, include_dir, header, structs):
    """sizeof and every field's offsetof of the named C structs, as gcc lays
    them out from the header."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{header}"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for field in cls._fields_:
            lines.append(f'printf("{cname}.{field[0]} %zu\\n", offsetof({cname}, {field[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", include_dir, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def _c_fields(header_path, cname):
    """Member names of `typedef struct ... { ... } cname;` in declaration order."""
    src = re.sub(r"/\*.*?\*/", "", open(header_path).read(), flags=re.S)
    m = re.search(r"typedef\s+struct\s*\w*\s*\{([^{}]*)\}\s*" + cname + r"\s*;", src)
    assert m, cname
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            names.append(re.search(r"(\w+)\s*(?:\[[^\]]*\])?\s*$", part.strip()).group(1))
    return names


def _ctypes_layout(structs):
    out = {}
    for cname, cls in structs.items():
        out[cname] = ctypes.sizeof(cls)
        for field in cls._fields_:
            out[f"{cname}.{field[0]}"] = getattr(cls, field[0]).offset
    return out


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of include/pic.h's structs (pic.py) have the C
    compiler's sizes and field offsets: a field added on one side only (as the
    multigrid starting value was to both) would shift every later field."""
    from paper_1001_2969_gb300 import pic

    structs = {n: getattr(pic, n) for n in ("pic_mesh", "pic_species", "pic_xsec", "pic_rf", "pic_gas",
                                            "pic_config", "pic_particles_view", "pic_solve_info",
                                            "pic_moments_out")}
    for cname, cls in structs.items():
        assert _c_fields(os.path.join(ROOT, "include", "pic.h"), cname) == [f[0] for f in cls._fields_], cname
    assert _c_layout(tmp_path, os.path.join(ROOT, "include"), "pic.h", structs) == _ctypes_layout(structs)


def test_oracle_config_matches_its_header_layout(tmp_path):
    """The same check for the oracle's configuration (oracle/oracle.h)."""
    import oracle

    structs = {"orc_config": oracle.OrcConfig}
    assert _c_fields(os.path.join(ROOT, "oracle", "oracle.h"), "orc_config") == [f[0] for f in oracle.OrcConfig._fields_]
    assert _c_layout(tmp_path, os.path.join(ROOT, "oracle"), "oracle.h", structs) == _ctypes_layout(structs)
