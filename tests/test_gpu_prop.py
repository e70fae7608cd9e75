"""GPU parity of the master-equation propagator U(t) (the paper's
propagator) against the FP64 oracle, through the C ABI: one CTA per matrix
unit, time-independent and time-dependent Hamiltonians, both precisions.

FP64: identical step counts, entries within 1e-8.  Mixed: the solve's own
integration error at rtol 1e-6 over the Jaynes-Cummings phase (|H| t ~ 30
rad) plus the FP32 state's rounding, within 1e-4."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1110_0573_gb300 import systems as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qt():
    from paper_1110_0573_gb300 import build
    build.build()
    from paper_1110_0573_gb300 import qt as q
    return q


@pytest.mark.parametrize("name", ["random4", "jc10", "random20"])
def test_fp64(qt, name):
    s = {"random4": lambda: S.random_system(4, 2, 1, seed=8, density=0.8),
         "jc10": lambda: S.jaynes_cummings(N=5, n0=2, kappa=0.3, gamma=0.2),
         "random20": lambda: S.random_system(20, 2, 1, seed=20, density=0.3)}[name]()
    tlist = np.array([0.0, 0.3, 0.8, 1.5])
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12)
    U, st = qt.qt_propagator(s["H"], s["c_ops"], tlist, opts=o)
    ref, ost = oracle.propagator(s["H"], s["c_ops"], tlist, rtol=1e-10, atol=1e-12)
    assert st["status"] == 0
    assert np.abs(U - ref).max() < 1e-8
    assert np.abs(U[0] - np.eye(U.shape[1])).max() == 0.0
    assert st["accepted"] == ost["accepted"] and st["rejected"] == ost["rejected"]


def test_time_dependent(qt):
    s = S.random_system(5, 1, 1, seed=9, density=0.8)
    X = sp.random(5, 5, density=0.6, random_state=3, dtype=float)
    td = [(sp.csr_matrix(0.5 * (X + X.T), dtype=np.complex128), np.array([-1.0, 0.5, 3.0]),
           np.array([0.0, 2.0, -1.0]))]
    tlist = np.array([0.2, 0.5, 1.0, 2.0])
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12)
    U, _ = qt.qt_propagator(s["H"], s["c_ops"], tlist, opts=o, td=td)
    ref, _ = oracle.propagator(s["H"], s["c_ops"], tlist, rtol=1e-10, atol=1e-12, td=td)
    assert np.abs(U - ref).max() < 1e-8


def test_mixed_and_device_entry(qt):
    s = S.jaynes_cummings(N=5, n0=2, kappa=0.3, gamma=0.2)
    tlist = np.array([0.0, 0.5, 1.0])
    ref, _ = oracle.propagator(s["H"], s["c_ops"], tlist, rtol=1e-10, atol=1e-12)
    o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED)
    U, st = qt.qt_propagator(s["H"], s["c_ops"], tlist, opts=o)
    assert st["status"] == 0 and np.abs(U - ref).max() < 1e-4
    sysm = qt.System(s["H"], s["c_ops"], [])
    tl = torch.tensor(tlist, dtype=torch.float64, device="cuda")
    Ud = torch.zeros((3, 100, 100), dtype=torch.complex128, device="cuda")
    sysm.qt_propagator_dev(tl, qt.qt_opts_default(rtol=1e-10, atol=1e-12), Ud)
    torch.cuda.synchronize()
    assert np.abs(Ud.cpu().numpy() - ref).max() < 1e-8
    sysm.close()


def test_dimension_limit(qt):
    H = sp.diags(np.arange(65, dtype=complex)).tocsr()
    with pytest.raises(qt.QtError) as e:
        qt.qt_propagator(H, [], [0.0, 1.0])
    assert e.value.code == qt.QT_ENOTIMPL
