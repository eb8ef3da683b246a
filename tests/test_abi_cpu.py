"""The C-ABI library builds, loads and exports every declared symbol (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ldpcgb.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^LDPC_API\s+(?:int|const char \*)\s*(\w+)\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_00167_gb300 import build
    build.build()
    from paper_2506_00167_gb300 import abi
    return abi.load()


def test_header_declares_the_path_entry_points():
    names = _declared()
    for n in ["ldpc_session_create", "puncture_demap", "decode_batch", "tb_crc_goodput"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n
    from paper_2506_00167_gb300 import abi
    assert sorted(abi.EXPORTED) == _declared()
    assert b"sm_103a" in lib.ldpc_version()


def test_descriptor_layouts_agree():
    from paper_2506_00167_gb300 import abi
    from workload.configs import CB_DTYPE, TB_DTYPE
    assert ctypes.sizeof(abi.CbDescC) == CB_DTYPE.itemsize == 56
    assert ctypes.sizeof(abi.TbDescC) == TB_DTYPE.itemsize == 20
    for name, (_, off) in abi.CB_NP.fields.items():
        assert CB_DTYPE.fields[name][1] == off, name
    for name, (_, off) in abi.TB_NP.fields.items():
        assert TB_DTYPE.fields[name][1] == off


def test_host_validation_without_gpu(lib):
    # argument checks run before any device work: a null descriptor is rejected
    from paper_2506_00167_gb300 import abi
    h = ctypes.c_void_p()
    rc = lib.ldpc_session_create(None, ctypes.byref(h))
    assert rc == -1 and b"null" in lib.ldpc_last_error()
    assert lib.decode_batch(None, None, None, None, None) == -1
    assert lib.ldpc_batch_destroy(None) == 0


def test_product_path_has_no_cpu_fallback():
    # the binding refuses to run without CUDA rather than computing on the CPU
    import torch
    from paper_2506_00167_gb300 import Session
    from workload import default_bgs
    if torch.cuda.is_available():
        pytest.skip("CUDA present")
    with pytest.raises(RuntimeError, match="CUDA"):
        Session(default_bgs(), [16])
    src = open(os.path.join(ROOT, "paper_2506_00167_gb300", "session.py")).read()
    src += open(os.path.join(ROOT, "paper_2506_00167_gb300", "abi.py")).read()
    assert "oracle" not in src and "workload" not in src


# every public struct of the header and its ctypes mirror in the binding
_STRUCTS = [("ldpc_base_graph", "BaseGraphC"), ("ldpc_session_desc", "SessionDescC"), ("ldpc_cb_desc", "CbDescC"),
            ("ldpc_tb_desc", "TbDescC"), ("ldpc_batch_info", "BatchInfoC"), ("ldpc_tile", "TileC"),
            ("ldpc_launch_info", "LaunchInfoC"), ("ldpc_serve_desc", "ServeDescC"), ("ldpc_serve_tb", "ServeTbC"),
            ("ldpc_serve_done", "ServeDoneC")]


def _header_fields(struct_text):
    """Member names of a typedef'd struct body, in order (comments stripped)."""
    body = re.sub(r"/\*.*?\*/", "", struct_text, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            m = re.search(r"(\w+)\s*(\[\s*\w+\s*\])?\s*$", part.strip())
            names.append(m.group(1))
    return names


def test_binding_structs_match_the_header_layout(tmp_path):
    """sizeof / offsetof of every member as the C compiler lays the header out, against ctypes."""
    import shutil
    import subprocess
    from paper_2506_00167_gb300 import abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    txt = open(HEADER).read()
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ldpcgb.h"', "int main(void) {"]
    members = {}
    for cname, _ in _STRUCTS:
        m = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + r";", txt)
        assert m, cname
        members[cname] = _header_fields(m.group(1))
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in members[cname]:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n"):
        if ln:
            s, f, v = ln.split()
            got[(s, f)] = int(v)
    for cname, pyname in _STRUCTS:
        cls = getattr(abi, pyname)
        assert [f for f, _ in cls._fields_] == members[cname], cname
        assert ctypes.sizeof(cls) == got[(cname, "size")], cname
        for f in members[cname]:
            assert getattr(cls, f).offset == got[(cname, f)], (cname, f)
