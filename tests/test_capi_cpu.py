"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function that include/mlmc.h declares, and its structs have the layout
the Python binding marshals; without a GPU, context creation fails cleanly."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mlmc.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"MLMC_API\s+[\w\s\*]*?\b(mlmc_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def pk():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_1506_04694_gb300 as pk
    pk.build.build()
    return pk


def test_exports_every_declared_function(pk):
    names = declared_functions()
    assert len(names) >= 10
    lib = pk.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pk.EXPORTS), "binding and header disagree"


def test_struct_layout_matches_c(pk, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "mlmc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(mlmc_model), offsetof(mlmc_model, tol),
         offsetof(mlmc_model, max_it), sizeof(mlmc_level_sums), sizeof(mlmc_estimate_out),
         offsetof(mlmc_estimate_out, rounds));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(pk.Model), pk.Model.tol.offset, pk.Model.max_it.offset,
            ctypes.sizeof(pk.LevelSums), ctypes.sizeof(pk.EstimateOut), pk.EstimateOut.rounds.offset]
    assert got == want


def test_error_strings(pk):
    lib = pk.lib()
    assert lib.mlmc_error_string(0) == b"success"
    assert b"invalid" in lib.mlmc_error_string(-1)


def test_create_without_gpu_fails_cleanly(pk):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = pk.make_model({"n_layers": 2, "k_kind": 0, "m0": 8, "L": 1, "tol": 1e-10, "max_it": 10,
                       "norm_r": 2, "if_lo": 0.3, "if_hi": 0.7, "mu": [0.0], "sigma2": [1.0],
                       "lam": [0.3]})
    h = ctypes.c_void_p()
    rc = pk.lib().mlmc_create(0, ctypes.byref(m), None, ctypes.byref(h))
    assert rc == -5 and not h.value  # MLMC_ERR_NODEV
    with pytest.raises(pk.MLMCError):
        pk.Context({"n_layers": 2})


def test_bad_model_rejected_before_device(pk):
    m = pk.make_model({"n_layers": 9, "k_kind": 0, "m0": 8, "L": 1, "tol": 1e-10, "max_it": 10,
                       "norm_r": 2})
    h = ctypes.c_void_p()
    assert pk.lib().mlmc_create(0, ctypes.byref(m), None, ctypes.byref(h)) == -1
