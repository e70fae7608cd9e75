"""The C-ABI library builds, loads, exports every function qt.h declares, and
rejects bad arguments without touching a GPU."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qt_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def qt():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1110_0573_gb300 import build
    build.build()
    from paper_1110_0573_gb300 import qt as q
    return q


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qt_mesolve", "qt_mcsolve", "qt_expect", "qt_mesolve_dev", "qt_mcsolve_dev",
                     "qt_expect_dev", "qt_system_create", "qt_last_error"):
        assert required in names


def test_header_is_plain_c():
    # the boundary header compiles as C99 and as C++ (no torch or CUDA types)
    import subprocess
    cc = shutil.which("gcc")
    if not cc:
        pytest.skip("gcc not available")
    for lang, std in (("c", "-std=c99"), ("c++", "-std=c++17")):
        r = subprocess.run([cc, std, "-fsyntax-only", "-Wall", "-Wextra", "-x", lang, HEADER],
                           capture_output=True, text=True)
        assert r.returncode == 0 and not r.stderr, r.stderr
    text = open(HEADER).read()
    assert "torch" not in text and "cuda_runtime" not in text


def test_library_exports_every_declared_symbol(qt):
    lib = ctypes.CDLL(qt.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the binding wraps every declared function
    assert sorted(n for n, _, _ in qt.SIGNATURES) == declared_functions()


def test_struct_layouts(qt):
    assert ctypes.sizeof(qt.qt_op) == 40
    assert ctypes.sizeof(qt.qt_opts) == 56
    assert ctypes.sizeof(qt.qt_stats) == 56 == qt.STATS_DTYPE.itemsize
    assert qt.JUMP_DTYPE.itemsize == 40


def test_defaults_and_version(qt):
    o = qt.qt_opts_default()
    assert o.rtol == 1e-8 and o.atol == 1e-10 and o.max_steps == 10**6
    assert o.precision == qt.QT_FP64
    assert "sm_103a" in qt.qt_version()


def test_validation_happens_before_any_device_work(qt):
    from paper_1110_0573_gb300 import systems as S
    s = S.jaynes_cummings(N=3, n0=1)
    bad = qt.qt_opts_default(rtol=-1.0)
    with pytest.raises(qt.QtError) as e:
        qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 4, opts=bad)
    assert e.value.code == qt.QT_EINVAL
    with pytest.raises(qt.QtError) as e:
        qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"][::-1])
    assert e.value.code == qt.QT_EINVAL
    # a wrong-sized collapse operator is caught while packing
    with pytest.raises(qt.QtError) as e:
        qt.qt_mesolve(s["H"], [np.eye(3)], s["e_ops"], s["psi0"], s["tlist"])
    assert e.value.code in (qt.QT_EINVAL, qt.QT_ENODEV)


def test_new_entry_points_validate_before_device_work(qt):
    from paper_1110_0573_gb300 import systems as S
    s = S.jaynes_cummings(N=3, n0=1)
    a = S.tensor(S.destroy(3), S.qeye(2))
    # correlation: taulist must start at 0 and increase; tlist must increase
    for tl, tau in (([0.0, 1.0], [0.1, 0.2]), ([0.0, 1.0], [0.0, 0.0]), ([1.0, 0.0], [0.0])):
        with pytest.raises(qt.QtError) as e:
            qt.qt_correlation_2op_2t(s["H"], s["c_ops"], S.dag(a), a, s["psi0"], tl, tau)
        assert e.value.code == qt.QT_EINVAL
    # propagator: increasing times; bad options
    with pytest.raises(qt.QtError) as e:
        qt.qt_propagator(s["H"], s["c_ops"], [0.0, 0.0])
    assert e.value.code == qt.QT_EINVAL
    with pytest.raises(qt.QtError) as e:
        qt.qt_propagator(s["H"], s["c_ops"], [0.0, 1.0], opts=qt.qt_opts_default(rtol=0.0))
    assert e.value.code == qt.QT_EINVAL
    # steady states: tolerances, iteration and period limits
    for call in (lambda: qt.qt_steadystate(s["H"], s["c_ops"], tol=0.0),
                 lambda: qt.qt_steadystate(s["H"], s["c_ops"], max_iter=-1),
                 lambda: qt.qt_propagator_steadystate(s["H"], s["c_ops"], period=0.0),
                 lambda: qt.qt_propagator_steadystate(s["H"], s["c_ops"], period=1.0,
                                                      max_periods=0),
                 lambda: qt.qt_correlation_ss(s["H"], s["c_ops"], S.dag(a), a, [0.0, 1.0],
                                              tol=-1.0),
                 lambda: qt.qt_correlation_ss(s["H"], s["c_ops"], S.dag(a), a, [0.5, 1.0])):
        with pytest.raises(qt.QtError) as e:
            call()
        assert e.value.code == qt.QT_EINVAL


def test_without_a_gpu_the_library_refuses(qt):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    from paper_1110_0573_gb300 import systems as S
    s = S.jaynes_cummings(N=3, n0=1)
    with pytest.raises(qt.QtError) as e:
        qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 4)
    assert e.value.code == qt.QT_ENODEV
