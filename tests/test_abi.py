"""The C-ABI library builds, loads and exports every symbol include/pic.h declares.

No compute call is made here (no GPU on the CPU runners); only host-side
entry points that touch no device run.
"""
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "pic.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1404_1160_gb300 import build

    build.build()
    from paper_1404_1160_gb300 import pic

    return pic.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pic_init", "pic_step", "pic_moments", "pic_deposit", "pic_poisson", "pic_gather"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1404_1160_gb300 import pic

    out = subprocess.run(["nm", "-D", "--defined-only", pic.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pic_[a-z_0-9]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in declared_functions():
        assert hasattr(lib, n)


def test_build_targets_sm_103a_only():
    from paper_1404_1160_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_entry_points(lib):
    from paper_1404_1160_gb300 import pic

    p = pic.pic_default_params()
    assert (p.eps, p.dt, p.n_cells, p.steps_per_turn, p.r_max) == (0.01, 0.1, 256, 100, 4.0)
    assert p.weight_fixed == 1 << 32 and p.max_window_steps == 300
    assert p.field_parity == pic.PIC_PARITY_EVEN
    assert pic.pic_strerror(pic.PIC_ERR_TIMEOUT).startswith("device-side wait")


def test_struct_layout_matches_header(lib):
    import ctypes

    from paper_1404_1160_gb300 import pic

    # pic_params: 2 doubles, 4 int32, 3 doubles, uint64, 6 int32, int64, 2 int32
    assert ctypes.sizeof(pic.pic_params) == 2 * 8 + 4 * 4 + 3 * 8 + 8 + 6 * 4 + 8 + 2 * 4
    assert ctypes.sizeof(pic.pic_moments_t) == 22 * 8


def test_bad_arguments_rejected_without_device(lib):
    import numpy as np

    from paper_1404_1160_gb300 import pic

    p = pic.pic_default_params(n_cells=255)  # odd mesh: r = 0 is not a node
    with pytest.raises(pic.PicError) as ei:
        pic.pic_init(p, np.zeros(4), np.zeros(4))
    assert ei.value.status == pic.PIC_ERR_INVALID_ARG
    # the FP32 form needs the exact-rotation solver and W <= 2^32; other
    # precision values do not exist
    for kw, rc in (({"precision": 1, "fine_solver": pic.PIC_FINE_RK4}, pic.PIC_ERR_UNSUPPORTED),
                   ({"precision": 1, "weight_fixed": 1 << 33}, pic.PIC_ERR_UNSUPPORTED),
                   ({"precision": 1, "dt": 1e5}, pic.PIC_ERR_UNSUPPORTED),
                   ({"precision": 2}, pic.PIC_ERR_INVALID_ARG),
                   ({"field_parity": 2}, pic.PIC_ERR_INVALID_ARG)):
        with pytest.raises(pic.PicError) as ei:
            pic.pic_init(pic.pic_default_params(**kw), np.zeros(4), np.zeros(4))
        assert ei.value.status == rc


def test_no_cpu_fallback_without_device(lib):
    import numpy as np
    import torch

    from paper_1404_1160_gb300 import pic

    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(pic.PicError) as ei:
        pic.pic_init(pic.pic_default_params(), np.zeros(8), np.zeros(8))
    assert ei.value.status == pic.PIC_ERR_CUDA
