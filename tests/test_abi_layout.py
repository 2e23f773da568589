"""The ctypes structures of the Python binding have the C header's layout:
a host program compiled against include/seemps_gb300.h prints every struct's
size and field offsets, and the binding's ctypes mirrors must agree (a field
appended to the header but not to the binding, or the reverse, shows here)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C struct name -> (binding class name, fields in declaration order)
STRUCTS = {
    "seemps_strategy": ("Strategy", ["chi_max", "tol", "rule"]),
    "seemps_pair_dims": ("PairDims", ["chi_l", "chi_r", "d", "D_l", "D_m", "D_r"]),
    "seemps_chain": ("ChainC", ["n_sites", "d", "D", "W", "A", "chi", "Lenv", "Renv", "B", "chib", "Fenv",
                                "Genv"]),
    "seemps_sweep_params": ("SweepParams", ["mode", "n_sweeps", "refine_sweeps", "precision", "krylov_dim",
                                            "breakdown_tol", "strategy", "canonicalize", "pcg_rtol", "pcg_maxiter",
                                            "precond", "mlp", "tdvp_dt"]),
    "seemps_sweep_report": ("SweepReport", ["energy", "max_discarded", "error_bound", "local_iters", "seconds",
                                            "half_sweeps", "half_sweep_energy", "half_sweep_max_rank"]),
    "seemps_cgs_problem": ("CgsProblem", ["n_sites", "d", "D", "W", "chib", "B", "chix", "X", "work",
                                          "work_bytes"]),
    "seemps_cgs_params": ("CgsParams", ["strategy", "n_sweeps", "precision", "maxiter", "rtol"]),
    "seemps_cgs_report": ("CgsReport", ["iterations", "residual", "norm_b", "seconds", "residual_history"]),
    "seemps_mlp_dataset": ("MlpDataset", ["n_systems", "dims", "L", "W1", "W2", "R", "b", "xstar", "site",
                                          "n_sites"]),
    "seemps_mlp_train_params": ("MlpTrainParams", ["steps", "batch", "lr", "beta1", "beta2", "eps"]),
}


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "seemps_gb300.h"', "int main(void) {"]
    for cname, (_, fields) in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as tmp:
        src, exe = os.path.join(tmp, "layout.c"), os.path.join(tmp, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, val = line.split()
        layout[(name, field)] = int(val)
    return layout


def test_binding_structs_match_the_header():
    from paper_2601_16734_gb300 import abi
    layout = _c_layout()
    for cname, (pyname, fields) in STRUCTS.items():
        cls = getattr(abi, pyname)
        assert ctypes.sizeof(cls) == layout[(cname, "size")], (cname, ctypes.sizeof(cls))
        py_fields = [f[0] for f in cls._fields_]
        assert py_fields == fields, (pyname, py_fields)
        for f in fields:
            assert getattr(cls, f).offset == layout[(cname, f)], (cname, f)


def _prototypes():
    """name -> list of C parameter declarations, from the header's prototypes."""
    import re
    text = open(os.path.join(ROOT, "include", "seemps_gb300.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b[a-z_]+\s*\*?\s*(seemps_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        args = [a.strip() for a in m.group(2).replace("\n", " ").split(",")]
        protos[m.group(1)] = [] if args == ["void"] else args
    return protos


def _c_kind(decl: str) -> str:
    if "*" in decl:
        return "ptr"
    words = decl.split()[:-1]
    t = " ".join(w for w in words if w != "const")
    return {"int": "int", "double": "double", "float": "float", "size_t": "size_t", "long long": "int64",
            "seemps_status": "int"}.get(t, t)


def _py_kind(ct) -> str:
    if ct in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(ct, type) and issubclass(ct, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_int: "int", ctypes.c_double: "double", ctypes.c_float: "float", ctypes.c_size_t: "size_t",
            ctypes.c_longlong: "int64"}[ct]


def test_binding_signatures_match_the_prototypes():
    from paper_2601_16734_gb300 import abi
    protos = _prototypes()
    assert len(protos) >= 30
    for name, argtypes in abi._SIGS.items():
        assert name in protos, name
        c_kinds = [_c_kind(a) for a in protos[name]]
        py_kinds = [_py_kind(t) for t in argtypes]
        assert c_kinds == py_kinds, (name, c_kinds, py_kinds)
