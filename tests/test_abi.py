"""The C ABI library loads and exports every entry point declared in
include/flexiwalk.h; host-side argument and CSR validation (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2512_00705_gb300 import _build
from paper_2512_00705_gb300 import flexiwalk as fw
from paper_2512_00705_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    yield


def declared_functions():
    src = open(os.path.join(ROOT, "include", "flexiwalk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fw_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["fw_graph_create", "fw_graph_destroy", "fw_walk", "fw_walk_host", "fw_sample_hist",
                 "fw_step_plan", "fw_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fw_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(_build.LIB)
    for n in declared_functions():
        assert hasattr(L, n)


STRUCTS = [("fw_params", fw.fw_params), ("fw_graph_info_t", fw.fw_graph_info_t), ("fw_counters", fw.fw_counters),
           ("fw_job", fw.fw_job), ("fw_server_config", fw.fw_server_config),
           ("fw_server_stats_t", fw.fw_server_stats_t)]


def test_binding_structs_match_the_header(tmp_path):
    """Size, alignment and every field offset of the binding's ctypes
    structures equal those the C compiler gives the header's structs."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "flexiwalk.h"', "int main(void) {"]
    for cname, py in STRUCTS:
        lines.append(f'  printf("{cname} size %zu align %zu\\n", sizeof({cname}), _Alignof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    got = dict(line.rsplit(" ", 1) for line in out if " size " not in line)
    sizes = {w[0]: (int(w[2]), int(w[4])) for w in (line.split() for line in out if " size " in line)}
    assert len(sizes) == len(STRUCTS) and len(got) == sum(len(py._fields_) for _, py in STRUCTS)
    for cname, py in STRUCTS:
        assert sizes[cname] == (ctypes.sizeof(py), ctypes.alignment(py)), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_binding_constants_match_the_header(tmp_path):
    """Status codes, algorithms, modes, pointer kinds and flags of the
    binding equal the header's enumerators (values printed by a C program
    compiled against the header)."""
    want = {f"FW_ALGO_{k.upper()}": v for k, v in fw.ALGO.items()}
    want.update({f"FW_MODE_{k.upper()}": v for k, v in fw.MODE.items()})
    want.update({name: code for code, name in fw.STATUS.items()})
    want.update({"FW_PTR_HOST": fw.PTR_HOST, "FW_PTR_DEVICE": fw.PTR_DEVICE})
    want.update({f"FW_{k}": getattr(fw, k) for k in dir(fw) if k.startswith("FLAG_")})
    lines = ["#include <stdio.h>", '#include "flexiwalk.h"', "int main(void) {"]
    lines += [f'  printf("{k} %d\\n", (int){k});' for k in sorted(want)]
    lines += ["  return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = {out[i]: int(out[i + 1]) for i in range(0, len(out), 2)}
    assert got == want
    header = open(os.path.join(ROOT, "include", "flexiwalk.h")).read()
    assert set(re.findall(r"\b(FW_FLAG_\w+)\s*=", header)) == {k for k in want if k.startswith("FW_FLAG_")}


def test_params_default():
    p = fw.make_params()
    assert (p.p, p.q, p.mode, p.flags, p.schema_len, p.rjs_cap, p.walker_base) == (1.0, 1.0, 0, 0, 0, 0, 0)


def _create_status(offsets, cols, h=None, labels=None):
    L = fw.lib()
    out = ctypes.c_void_p()
    offsets = np.ascontiguousarray(offsets, np.int32)
    cols = np.ascontiguousarray(cols, np.int32)
    hp = None if h is None else np.ascontiguousarray(h, np.float32)
    return L.fw_graph_create(offsets.ctypes.data, cols.ctypes.data, None if hp is None else hp.ctypes.data, None,
                             offsets.shape[0] - 1, cols.shape[0], fw.PTR_HOST, None, ctypes.byref(out)), out


@pytest.mark.parametrize("offsets,cols,h,why", [
    ([1, 2, 3], [1, 0], None, "offsets[0]"),
    ([0, 2, 1, 3], [1, 2, 0], None, "monotone"),
    ([0, 1, 2], [1, 0, 0], None, "offsets[n]"),
    ([0, 2, 3, 4], [2, 1, 0, 0], None, "increasing"),
    ([0, 2, 3, 4], [1, 1, 0, 0], None, "increasing"),
    ([0, 1, 2], [1, 5], None, "range"),
    ([0, 1, 2], [1, -1], None, "range"),
    ([0, 1, 2], [1, 0], [1.0, 0.0], "weight"),
    ([0, 1, 2], [1, 0], [1.0, float("nan")], "weight"),
    ([0, 1, 2], [1, 0], [float("inf"), 1.0], "weight"),
    ([0, 1, 2], [1, 0], [-2.0, 1.0], "weight"),
])
def test_host_csr_validation(offsets, cols, h, why):
    st, out = _create_status(offsets, cols, h)
    assert st == -2, (st, fw.lib().fw_last_error())
    assert out.value is None
    assert why in fw.lib().fw_last_error().decode()


def test_argument_errors_without_device():
    L = fw.lib()
    out = ctypes.c_void_p()
    assert L.fw_graph_create(None, None, None, None, 3, 0, fw.PTR_HOST, None, ctypes.byref(out)) == -1
    assert L.fw_graph_create(None, None, None, None, -1, 0, fw.PTR_HOST, None, ctypes.byref(out)) == -1
    o = np.array([0, 0], np.int32)
    assert L.fw_graph_create(o.ctypes.data, o.ctypes.data, None, None, 1, 0, 7, None, ctypes.byref(out)) == -1
    prm = fw.make_params()
    assert L.fw_walk(None, None, 0, 1, 0, ctypes.byref(prm), 1, None, None) == -1
    assert L.fw_graph_destroy(None) == -1
    assert L.fw_status_string(-2) == b"FW_ERR_CSR"
    rate = ctypes.c_double()
    assert L.fw_gather_ceiling(None, 1 << 30, ctypes.byref(rate), None) == -1
    assert L.fw_gather_ceiling(ctypes.c_void_p(1 << 20), (1 << 30) + 32, ctypes.byref(rate), None) == -1
    assert L.fw_gather_ceiling(ctypes.c_void_p(1 << 20), 1 << 20, ctypes.byref(rate), None) == -1


def test_valid_host_graph_passes_validation():
    """A valid CSR gets past host validation; without a GPU the next step
    (device selection) fails with FW_ERR_CUDA, never FW_ERR_CSR."""
    g = synth.workload_graph("small")
    st, _ = _create_status(g.offsets, g.cols, g.h)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        assert st == 0
    else:
        assert st == -4
