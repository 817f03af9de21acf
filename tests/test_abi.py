"""The C ABI library loads and exports every function the headers in include/
declare (no compute calls: runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fusedpr.h")
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(pr_[a-z_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2203_09284_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pr_graph_create", "pr_solve", "pr_solve_batched", "pr_backward",
                     "pr_solve_multi", "pr_graph_destroy", "pr_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (pr_[a-z_]+)\b", out))
    assert set(declared_functions()) <= exported


def test_status_strings_without_gpu(libpath):
    import paper_2203_09284_gb300 as fp
    assert fp.pr_status_string(fp.PR_OK) == "ok"
    assert "converged" in fp.pr_status_string(fp.PR_NOT_CONVERGED)
    o = fp.pr_options_default()
    assert o.d == 0.85 and o.threshold == 1e-10 and o.use_graph == 1


def test_header_compiles_as_c():
    for h in HEADERS:
        r = subprocess.run(["gcc", "-std=c99", "-fsyntax-only", "-x", "c", h],
                           capture_output=True, text=True)
        assert r.returncode == 0, (h, r.stderr)


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2203_09284_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "oracle." not in text, f


def test_python_structs_match_the_header(tmp_path):
    """The ctypes mirrors of pr_tune / pr_options / pr_result have the C
    layout (sizes and the offset of every field)."""
    import paper_2203_09284_gb300 as fp
    structs = {"pr_tune": fp.PrTune, "pr_options": fp.PrOptions, "pr_result": fp.PrResult}
    lines = ['#include <stddef.h>', '#include <stdio.h>', f'#include "{HEADER}"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{cname}.{field} %zu\\n", offsetof({cname}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-o", str(exe), str(src)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert int(got[f"{cname}.{field}"]) == getattr(py, field).offset, (cname, field)
