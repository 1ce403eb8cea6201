"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point include/phd.h declares, and the binding's struct matches."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "phd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(phd_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1503_03769_gb300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(L, n), n
    from paper_1503_03769_gb300 import phd
    assert sorted(phd.ABI) == names


@pytest.mark.parametrize("name", ["phd_config", "phd_stats", "phd_tuning"])
def test_struct_layout_matches_header(tmp_path, name):
    """The binding's structs have the C compiler's size and field offsets."""
    import subprocess
    from paper_1503_03769_gb300 import phd
    st = getattr(phd, name)
    fields = [f[0] for f in st._fields_]
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "phd.h"', "int main(void){",
            f'printf("%zu\\n", sizeof({name}));']
    prog += [f'printf("%zu\\n", offsetof({name}, {n}));' for n in fields]
    prog += ["return 0;}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert out[0] == ctypes.sizeof(st)
    assert out[1:] == [getattr(st, n).offset for n in fields]


def test_workspace_size_and_config_validation_without_gpu():
    import scenario
    from paper_1503_03769_gb300 import phd
    L = phd.lib()
    w = scenario.workload("dist16_10t")
    c = phd.make_config(w)
    n = ctypes.c_size_t(0)
    assert L.phd_workspace_size(ctypes.byref(c), ctypes.byref(n)) == phd.PHD_OK
    assert n.value > 0 and n.value % 256 == 0
    for field, bad in [("num_pe", 0), ("num_pe", 300), ("m_max", 5000), ("pe_cap", 0),
                       ("p_d", 1.5), ("exchange_frac", 0.6), ("precision", 7), ("birth_model", 2),
                       ("sigma_a_y", -1.0), ("theta_span", 7.0), ("exchange_mode", 2), ("reserved1", 1),
                       ("exchange_threshold", -0.5), ("gate_sigma", -1.0)]:
        c2 = phd.make_config(w)
        setattr(c2, field, bad)
        assert L.phd_workspace_size(ctypes.byref(c2), ctypes.byref(n)) == phd.PHD_ERR_INVALID_ARG, field
    c2 = phd.make_config(w)
    c2.birth_model = phd.PHD_BIRTH_GAUSSIAN
    c2.birth_std[1] = -1.0
    assert L.phd_workspace_size(ctypes.byref(c2), ctypes.byref(n)) == phd.PHD_ERR_INVALID_ARG
    c2.birth_std[1] = 1.0
    assert L.phd_workspace_size(ctypes.byref(c2), ctypes.byref(n)) == phd.PHD_OK
    assert L.phd_init(None, ctypes.byref(c), None, 0, None) == phd.PHD_ERR_INVALID_ARG
    assert L.phd_status_string(phd.PHD_ERR_CAPACITY) == b"capacity exceeded"


def test_bench_ospa_metric_matches_permutation_brute_force():
    """bench.py scores the GPU arms with its own OSPA; check it against the
    definition by brute force over assignments on small sets."""
    import itertools
    import math
    import sys
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(0)
    for m, n in [(0, 0), (0, 3), (2, 0), (3, 3), (2, 5), (5, 4)]:
        X = rng.uniform(0, 150, (m, 2))
        Y = rng.uniform(0, 150, (n, 2))
        c, p = 100.0, 2.0
        if m == 0 and n == 0:
            want = 0.0
        elif m == 0 or n == 0:
            want = c
        else:
            A, B = (X, Y) if m <= n else (Y, X)
            a, b = len(A), len(B)
            best = min(sum(min(c, float(np.linalg.norm(A[i] - B[perm[i]]))) ** p for i in range(a))
                       for perm in itertools.permutations(range(b), a))
            want = ((best + c ** p * (b - a)) / b) ** (1 / p)
        assert math.isclose(bench.ospa_metric(X, Y, c, p), want, rel_tol=1e-12, abs_tol=1e-12)


def test_c_program_builds_against_the_header(tmp_path):
    """tests/c_abi_track.c (the C-ABI example the GPU tests run) compiles as
    C99 with -Wall -Werror and links against libphd.so here, without a GPU."""
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import test_gpu_c_abi
    test_gpu_c_abi.build_c_program(str(tmp_path / "track"))
    assert os.path.exists(tmp_path / "track")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libphd.so the binding raises before it computes
    anything, for the library loader and for a filter handle alike."""
    import scenario
    from paper_1503_03769_gb300 import phd
    monkeypatch.setattr(phd, "LIB_PATH", str(tmp_path / "libphd.so"))
    monkeypatch.setattr(phd, "_lib", None)
    with pytest.raises(ImportError):
        phd.lib()
    with pytest.raises(ImportError):
        phd.ParticlePHD(scenario.workload("linear4_fp64"), device="cpu")


def test_colsum_static_binding_refuses_wrong_buffers_before_any_launch():
    """The binding checks dtype, shape and device of phd_colsum_static's
    buffers against the config before the library is called: a float32
    state array under a PHD_FP64 config (the kernel would read twice its
    bytes), a float32 or short C (the kernel would write past it), a wrong
    row width, or host tensors are refused with ValueError."""
    import torch
    import scenario
    from paper_1503_03769_gb300 import phd
    w64 = scenario.workload("linear4_fp64")
    w32 = scenario.workload("dist16_10t")
    c64, c32 = phd.make_config(w64), phd.make_config(w32)
    n, M = 10, 4
    f32 = lambda *s: torch.zeros(*s, dtype=torch.float32)
    f64 = lambda *s: torch.zeros(*s, dtype=torch.float64)
    cases = [
        (c64, f32(n, 4), f64(n), f64(M, 2), f64(M), "x is"),
        (c64, f64(n, 4), f64(n), f32(M, 2), f64(M), "Z is"),
        (c32, f32(n, 4), f32(n), f32(M, 2), f32(M), "C is"),
        (c32, f32(n, 4), f32(n), f32(M, 2), f64(M - 1), "fewer than M"),
        (c32, f32(n, 3), f32(n), f32(M, 2), f64(M), "x must be"),
        (c32, f32(n, 4), f32(n + 1), f32(M, 2), f64(M), "w must be"),
        (c32, f32(n, 4), f32(n), f32(M, 3), f64(M), "Z must be"),
        (c32, f32(n, 4), f32(n), f32(M, 2), f64(M), "one CUDA device"),
    ]
    for cfg, x, wt, Z, C, msg in cases:
        with pytest.raises(ValueError, match=msg):
            phd.colsum_static(cfg, x, wt, Z, C)
