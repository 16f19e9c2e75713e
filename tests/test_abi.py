"""CPU checks of the C-ABI boundary: the library builds, loads and exports every
symbol include/bpm.h declares.  No compute call is made (no GPU here)."""
import os
import re

import pytest

from paper_2201_08500_gb300 import bpm
from paper_2201_08500_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "bpm.h")).read()
    return sorted(set(re.findall(r"BPM_API\s+[\w\s\*]+?\b(bpm_\w+)\s*\(", txt)))


def test_header_declares_the_binding_exports():
    assert sorted(bpm.EXPORTS) == declared_symbols()


def test_library_builds_loads_and_exports_every_symbol():
    try:
        libbuild.nvcc()
    except RuntimeError:
        pytest.skip("no nvcc")
    path = libbuild.build()
    L = bpm.load(path)
    for name in declared_symbols():
        assert hasattr(L, name), name
    assert "sm_103a" in bpm.version()


def test_error_path_without_plan_is_reported():
    try:
        L = bpm.load(libbuild.build())
    except RuntimeError:
        pytest.skip("no nvcc")
    grid = bpm.Grid(2, 300, 1, 10, 1e-6, 0.0, 1e-6, 1, 1)
    h = bpm._P()
    st = L.bpm_plan_create(bpm.ctypes.byref(grid), 0, None, bpm.ctypes.byref(h))
    assert st == 1  # INVALID_ARG: n_channels < 1 is rejected before any device call
    assert b"n_channels" in L.bpm_last_error(None)


def test_tune_file_parsing_without_a_gpu(tmp_path):
    """Tune files: comment lines are skipped, lines of another device are
    ignored, malformed lines are an error (host logic only, no device call)."""
    from paper_2201_08500_gb300 import bpm
    bpm.load()
    good = tmp_path / "tune.txt"
    good.write_text("# header\nSomeOtherGPU/132 2 1024 1 1 611 0 4 256 1.5\n")
    assert bpm.tune_load(str(good)) == 0
    bad = tmp_path / "bad.txt"
    bad.write_text("SomeOtherGPU/132 2 1024 one\n")
    with pytest.raises(bpm.BpmError):
        bpm.tune_load(str(bad))
    with pytest.raises(bpm.BpmError):
        bpm.tune_load(str(tmp_path / "missing.txt"))


def test_noalloc_binding_refuses_bad_buffers_before_any_library_call(monkeypatch):
    """bpm_run_noalloc takes no buffer sizes, so the binding checks every tensor
    (CUDA, dtype, contiguity, element count) and raises before it loads or calls
    the library.  Without a GPU every tensor here is refused; the GPU suite
    (tests/test_zz_no_alloc.py) refuses mis-sized CUDA tensors the same way."""
    import torch
    from paper_2201_08500_gb300 import workloads

    def no_library(*a, **k):
        raise AssertionError("the library was reached")

    monkeypatch.setattr(bpm, "load", no_library)
    w = workloads.tiny(n_ch=4)
    good = torch.zeros((w.n_ch, w.nx), dtype=torch.complex64)
    R = torch.zeros(w.n_ch, dtype=torch.float64)
    for e0, eh, r in [(good, good, R),                                  # host tensors
                      (good[:, :-1], good, R),                          # too few elements
                      (good.to(torch.complex128), good, R),             # wrong dtype
                      (good, good.t(), R),                              # not contiguous
                      (good, good, R[:-1]),
                      (good.numpy(), good, R)]:                         # not a tensor
        with pytest.raises(bpm.BpmError) as ei:
            bpm.run_noalloc(w, e0, eh, r)
        assert ei.value.status == 1 and "run_noalloc" in str(ei.value)


def test_w32_twiddle_constants_are_the_correctly_rounded_values():
    """The 8192-point kernels take the W_32 powers of their third stage as
    immediates (w32_re / w32_im in csrc/bpm_internal.h), and the host twiddle
    table uses the same values: they must be the FP32 roundings of cos and
    -sin of 2 pi m / 32 (m = 8: of the double cos(pi/2))."""
    import numpy as np
    txt = open(os.path.join(ROOT, "paper_2201_08500_gb300", "csrc", "bpm_internal.h")).read()

    def values(name):
        body = txt[txt.index(f"constexpr float {name}(int m)"):]
        body = body[:body.index("}")]
        lits = re.findall(r"(-?0x[0-9a-f.]+p[-+]?\d+)f", body)
        assert len(lits) == 15, (name, lits)
        return [float.fromhex(x) for x in lits]

    re_, im_ = values("w32_re"), values("w32_im")
    for m in range(1, 16):
        a = 2.0 * np.pi * float(256 * m) / 8192.0        # the host's angle for k = 256 m, n = 8192
        assert re_[m - 1] == float(np.float32(np.cos(a))), m
        assert im_[m - 1] == float(np.float32(-np.sin(a))), m
