"""Host-only checks of the C-ABI boundary (no GPU needed).

* the library builds for sm_103a and loads;
* it exports every entry point declared in include/bem.h, and the Python
  binding declares each of them;
* the ctypes structures have the C layout (sizes and field offsets taken from
  a tiny C program compiled against the header);
* the oracle and the CUDA path share no code: neither imports or includes
  the other.
"""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bem.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(bem_\w+)\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_1007_4591_gb300 as pkg
    return pkg.load_library()


def test_python_constants_match_the_header():
    """Every integer constant the header defines (status codes, precisions,
    BIBEE lambdas, flags, option values) has a Python constant of the same
    name and value in the binding."""
    import paper_1007_4591_gb300 as pkg
    txt = open(HEADER).read()
    defs = []
    for name, body in re.findall(r"^#define\s+(BEM_\w+)\s+([^/\n]+)", txt, re.M):
        expr = re.sub(r"(\d)u\b", r"\1", body.strip())
        if re.fullmatch(r"[\d\s()<>+\-]+", expr):  # integer literals and shifts only
            defs.append((name, eval(expr)))
    assert len(defs) >= 20
    for name, val in defs:
        assert hasattr(pkg, name), name
        assert getattr(pkg, name) == val, (name, getattr(pkg, name), val)


def test_header_declares_the_call_list():
    names = _declared()
    for want in ("bem_mesh_create", "bem_mesh_destroy", "bem_matvec", "bem_solve", "bem_bibee",
                 "bem_energy", "bem_energy_backward", "bem_rhs", "bem_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    import paper_1007_4591_gb300 as pkg
    for name in _declared():
        assert name in pkg._SIGS, name
        assert hasattr(pkg, name), name


def test_struct_layout_matches_c(tmp_path):
    import paper_1007_4591_gb300 as pkg
    src = tmp_path / "layout.c"
    structs = {"bem_options": pkg.bem_options, "bem_solve_stats": pkg.bem_solve_stats,
               "bem_mesh_info": pkg.bem_mesh_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', 'int main(void){']
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} %zu\\n", sizeof({sname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{sname}.{f} %zu\\n", offsetof({sname}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in out if l.strip())
    for sname, cls in structs.items():
        assert int(got[sname]) == ctypes.sizeof(cls), sname
        for f, _ in cls._fields_:
            assert int(got[f"{sname}.{f}"]) == getattr(cls, f).offset, (sname, f)


def test_oracle_and_cuda_path_share_nothing():
    pkg_dir = os.path.join(ROOT, "paper_1007_4591_gb300")
    for dp, _, files in os.walk(pkg_dir):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dp, fn), errors="ignore").read()
                assert not re.search(r"\bimport\s+oracle\b|\bfrom\s+oracle\b|bem_oracle", txt), fn
    for fn in os.listdir(os.path.join(ROOT, "oracle")):
        if fn.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", fn), errors="ignore").read()
            assert "paper_1007_4591_gb300" not in txt and "bem.h" not in txt, fn
            assert "#include \"" not in txt, fn


def test_binding_refuses_when_library_missing(tmp_path):
    code = ("import paper_1007_4591_gb300 as p\n"
            "try:\n    p.load_library('%s')\nexcept ImportError:\n    print('raised')\n"
            % str(tmp_path / "nope.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT)
    assert "raised" in r.stdout
