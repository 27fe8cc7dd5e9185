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


def _checkpoint_text(d, levels):
    """A checkpoint file in the documented version-2 text format (model block,
    estimator header, one line per level), written without a GPU."""
    pad = lambda v, n: list(v) + [v[-1]] * (n - len(v))
    g = lambda x: "%.17g" % x
    lines = ["mlmc_checkpoint 2",
             "model %d %d %d %d %d %d %d %d %d %d %d %d" % (
                 d["n_layers"], d["k_kind"], d["norm_r"], d["m0"], d["L"], d["cgv"], d["prec"], d["max_it"],
                 d.get("problem", 0), d.get("geometry", 0), d.get("dim", 2), d.get("embed", 0)),
             "model_if %s %s" % (g(d["if_lo"]), g(d["if_hi"])), "model_tol %s" % g(d["tol"])]
    for key in ("mu", "sigma2", "lam"):
        lines.append("model_%s %s" % (key, " ".join(g(x) for x in pad(d[key], 8))))
    for key in ("qoi_box", "line_lo", "line_hi"):
        lines.append("model_%s %s" % (key, " ".join(g(x) for x in d.get(key, [0.0] * 4))))
    lines += ["seed 0", "eps 0.001", "cost_model 0", "rounds 1", "levels %d" % levels]
    for l in range(levels):
        lines.append("level %d 64 0 640 %s" % (l, " ".join(["1"] * 12)))
    return "\n".join(lines) + "\n"


def test_checkpoint_check_rejects_other_models(pk, tmp_path):
    # merging the level sums of another model would bias the telescoping sum of
    # Eq. 3.6 silently, so a checkpoint must match every field that changes Q
    import workloads
    d = workloads.workload("lognormal_2layer_16to256")
    path = tmp_path / "ck.txt"
    path.write_text(_checkpoint_text(d, d["L"] + 1))
    pk.checkpoint_check(d, str(path))  # the same model is accepted
    for key, val in (("sigma2", [1.5, 1.5]), ("lam", [0.2, 0.2]), ("mu", [0.0, 0.1]), ("tol", 1e-12),
                     ("if_lo", 0.25), ("if_hi", 0.75), ("norm_r", 1), ("prec", 1), ("cgv", 1), ("m0", 8),
                     ("max_it", 100), ("embed", 1)):
        with pytest.raises(pk.MLMCError, match="differs"):
            pk.checkpoint_check(dict(d, **{key: val}), str(path))
    # fields that do not change Q for this model are not compared: the box of
    # Model Problem 1 and the line ranges of the sloped geometry
    pk.checkpoint_check(dict(d, qoi_box=[0.1, 0.2, 0.3, 0.4]), str(path))
    pk.checkpoint_check(dict(d, line_lo=[0.1] * 4, line_hi=[0.2] * 4), str(path))
    # a version-1 file (model line without the per-layer parameters) is refused
    old = tmp_path / "v1.txt"
    old.write_text("mlmc_checkpoint 1\nmodel 2 1 16 4 0 0 2 2\n")
    with pytest.raises(pk.MLMCError, match="version-2"):
        pk.checkpoint_check(d, str(old))


def test_solve_wrappers_check_shapes_on_host(pk):
    # the binding rejects tensors of the wrong shape or device before any C
    # call, so no wrong-sized pointer reaches a kernel
    import torch
    q = torch.empty(2, dtype=torch.float64)
    with pytest.raises(pk.MLMCError, match="equal sides"):
        pk.solve_k_static(torch.ones((2, 8, 4), dtype=torch.float64), q)
    with pytest.raises(pk.MLMCError, match="equal sides"):
        pk.solve_k_static(torch.ones((8, 8), dtype=torch.float64), q)
    with pytest.raises(pk.MLMCError, match="CUDA"):
        pk.solve_k_static(torch.ones((2, 8, 8), dtype=torch.float64), q)


def test_null_context_is_an_argument_error(pk):
    # the scheduling, tuning and cost entry points check their context and
    # host arguments before any CUDA call: MLMC_ERR_ARG with a message
    import ctypes
    L = pk.lib()
    ERR_ARG = -1
    nul = ctypes.c_void_p(None)
    C = (ctypes.c_double * 4)(1.0, 2.0, 3.0, 4.0)
    i64 = (ctypes.c_int64 * 2)(0, 0)
    assert L.mlmc_set_schedule(nul, 1) == ERR_ARG
    assert L.mlmc_calibrate_costs(nul, 0, C) == ERR_ARG
    assert L.mlmc_set_costs(nul, C) == ERR_ARG
    assert L.mlmc_set_launch_ex(nul, 0, 0, 0, 256, 0, 1, 1, 0, 0, 0, 1e-5) == ERR_ARG
    assert L.mlmc_autotune_schedule(nul, 1e-3, 0, 64, 0, 1, None, None) == ERR_ARG
    assert L.mlmc_multilevel_batch_host(nul, 2, i64, i64, 0, 0, None, None, None, None, None) == ERR_ARG
    assert b"null" in L.mlmc_last_error()


def test_every_struct_field_matches_c(pk, tmp_path):
    """Each ctypes structure of the binding against its C struct in the
    header: the size and the offset of every member, by name."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    pairs = [(pk.Model, "mlmc_model"), (pk.LevelSums, "mlmc_level_sums"), (pk.EstimateOut, "mlmc_estimate_out"),
             (pk.ProfileStats, "mlmc_profile_stats"), (pk.TuneReport, "mlmc_tune_report")]
    lines, want = [], []
    for cls, cname in pairs:
        lines.append('  printf("%%zu\\n", sizeof(%s));' % cname)
        want.append(ctypes.sizeof(cls))
        for name, _ in cls._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (cname, name))
            want.append(getattr(cls, name).offset)
    prog = tmp_path / "fields.c"
    prog.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"mlmc.h\"\nint main(void) {\n"
                    + "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "fields"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == want


def _prototypes():
    """name -> (return type, [parameter types]) of every MLMC_API declaration
    in the header, comments removed, whitespace normalised ("double* const*")."""
    src = re.sub(r"/\*.*?\*/", " ", open(HEADER).read(), flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    norm = lambda t: re.sub(r"\s*\*", "*", " ".join(t.split())).strip()
    out = {}
    for ret, name, params in re.findall(r"MLMC_API\s+([^;(]*?)\b(mlmc_\w+)\s*\(([^;]*?)\)\s*;", src, flags=re.S):
        ps = [] if params.strip() in ("", "void") else [norm(re.sub(r"\w+\s*$", "", p)) for p in params.split(",")]
        out[name] = (norm(ret), ps)
    return out


_SCALARS = {"int": (4, "i"), "int32_t": (4, "i"), "int64_t": (8, "i"), "uint64_t": (8, "u"), "double": (8, "f")}


def _ctypes_scalar(t):
    code = getattr(t, "_type_", None)
    if not isinstance(code, str) or code not in "bBhHiIlLqQfd":
        return None
    return ctypes.sizeof(t), "f" if code in "fd" else ("u" if code.isupper() else "i")


def _matches(pk, ctype, t):
    structs = {pk.Model: "mlmc_model", pk.LevelSums: "mlmc_level_sums", pk.EstimateOut: "mlmc_estimate_out",
               pk.ProfileStats: "mlmc_profile_stats", pk.TuneReport: "mlmc_tune_report"}
    if t == "void":
        return ctype is None
    if not t.endswith("*"):
        return t in _SCALARS and _ctypes_scalar(ctype) == _SCALARS[t]
    pointee = re.sub(r"^const ", "", t[:-1].strip())
    pointee = re.sub(r" const$", "", pointee)
    if ctype is ctypes.c_void_p:  # an untyped address: any data pointer
        return True
    if ctype is ctypes.c_char_p:
        return pointee == "char"
    target = getattr(ctype, "_type_", None)
    if not isinstance(target, type):
        return False
    if target in structs:
        return pointee == structs[target]
    if target is ctypes.c_void_p:
        return pointee.endswith("*")
    return pointee in _SCALARS and _ctypes_scalar(target) == _SCALARS[pointee]


def test_binding_signatures_match_prototypes(pk):
    """The argument and return types the binding declares to ctypes agree
    with the header's prototypes: same count, scalars of the same size and
    kind, pointers where the header has pointers (typed ones to the same
    struct or scalar)."""
    protos = _prototypes()
    assert set(protos) == set(pk.EXPORTS)
    for name, (ret, params) in protos.items():
        cret, cargs = pk.EXPORTS[name]
        assert _matches(pk, cret, ret), (name, "return", ret, cret)
        assert len(cargs) == len(params), (name, params, cargs)
        for i, (ca, p) in enumerate(zip(cargs, params)):
            assert _matches(pk, ca, p), (name, i, p, ca)


def test_signature_check_catches_a_wrong_type(pk):
    # the check above is not vacuous: a 32-bit integer where the header has
    # int64_t, a scalar where it has a pointer, or the wrong struct all fail
    assert not _matches(pk, ctypes.c_int32, "int64_t")
    assert not _matches(pk, ctypes.c_uint64, "int64_t")
    assert not _matches(pk, ctypes.c_double, "double*")
    assert not _matches(pk, ctypes.POINTER(pk.LevelSums), "mlmc_estimate_out*")
    assert not _matches(pk, ctypes.POINTER(ctypes.c_int32), "int64_t*")
    assert _matches(pk, ctypes.POINTER(ctypes.c_void_p), "mlmc_ctx**")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no fallback: without libmlmc.so every entry of the binding raises
    import paper_1506_04694_gb300 as pk
    import workloads
    monkeypatch.setattr(pk, "_lib", None)
    monkeypatch.setattr(pk, "LIB_PATH", str(tmp_path / "libmlmc.so"))
    with pytest.raises(pk.MLMCError, match="not built"):
        pk.lib()
    # (without a GPU the context refuses first, with its own message)
    with pytest.raises(pk.MLMCError, match="not built|no CUDA device"):
        pk.Context(workloads.workload("lognormal_2layer_16to256"))
