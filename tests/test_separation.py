"""The oracle and the CUDA path share no code: the package that ships
libmlmc.so and its C sources never import or include anything of oracle/,
the oracle imports nothing of the package, and the one module both sides
read (workloads.py) imports neither."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1506_04694_gb300")


def _py_imports(path):
    tree = ast.parse(open(path).read(), path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            names.add(node.module.split(".")[0])
    return names


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_does_not_import_the_oracle():
    pys = list(_files(PKG, (".py",)))
    assert pys
    for p in pys:
        assert "oracle" not in _py_imports(p), p


def test_cuda_sources_include_only_their_own_headers():
    srcs = list(_files(PKG, (".cu", ".cuh", ".h"))) + list(_files(os.path.join(ROOT, "include"), (".h",)))
    assert len(srcs) >= 5
    own = {os.path.basename(p) for p in srcs}
    for p in srcs:
        for inc in re.findall(r'#include\s+"([^"]+)"', open(p).read()):
            assert os.path.basename(inc) in own and "oracle" not in inc, (p, inc)


def test_oracle_imports_nothing_of_the_package():
    pys = list(_files(os.path.join(ROOT, "oracle"), (".py",)))
    assert pys
    for p in pys:
        names = _py_imports(p)
        assert "paper_1506_04694_gb300" not in names and "workloads" not in names, p
    assert not list(_files(os.path.join(ROOT, "oracle"), (".cu", ".cuh")))


def test_shared_input_module_imports_neither_side():
    names = _py_imports(os.path.join(ROOT, "workloads.py"))
    assert "oracle" not in names and "paper_1506_04694_gb300" not in names
