"""The ctypes mirrors of the C ABI's structures (CPU only): a small C program
built with gcc against include/crac.h prints the size of every structure and
the offset of every field; the Python binding's ctypes structures must agree
byte for byte, so that no field is read from the wrong place."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# ctypes class name -> C typedef
PAIRS = {
    "CracConfig": "crac_config_t",
    "CracImageInfo": "crac_image_info_t",
    "CracPassInfo": "crac_pass_info_t",
    "CracRestartInfo": "crac_restart_info_t",
    "CracTuneResult": "crac_tune_result_t",
    "CracServerConfig": "crac_server_config_t",
    "CracRequestResult": "crac_request_result_t",
    "CracServerStats": "crac_server_stats_t",
    "CracMemoryStats": "crac_memory_stats_t",
}


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    import paper_2008_10596_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def c_layout(binding, tmp_path_factory):
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "crac.h"', "int main(void) {"]
    for cls, ctype in PAIRS.items():
        lines.append(f'printf("{cls} . %zu\\n", sizeof({ctype}));')
        for f, _ in getattr(binding, cls)._fields_:
            lines.append(f'printf("{cls} {f} %zu\\n", offsetof({ctype}, {f}));')
    lines += ["return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for ln in out.splitlines():
        cls, f, v = ln.split()
        table[(cls, f)] = int(v)
    return table


@pytest.mark.parametrize("cls", sorted(PAIRS))
def test_struct_layout_matches_header(binding, c_layout, cls):
    ct = getattr(binding, cls)
    assert c_layout[(cls, ".")] == ctypes.sizeof(ct), cls
    for f, _ in ct._fields_:
        assert c_layout[(cls, f)] == getattr(ct, f).offset, (cls, f)


def test_header_compiles_as_c_and_cxx(tmp_path):
    for compiler, ext in (("gcc", "c"), ("g++", "cpp")):
        src = tmp_path / f"inc.{ext}"
        src.write_text('#include "crac.h"\nint crac_header_probe;\n')
        subprocess.run([compiler, "-Wall", "-Wextra", "-Werror", "-c", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(tmp_path / f"inc_{ext}.o")], check=True)
