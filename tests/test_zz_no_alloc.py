"""qt_mesolve_dev_noalloc, the master-equation entry point for callers that
cannot allocate device memory (a process whose free memory belongs to
another allocator, or a solve path that must stay out of cudaMalloc/cudaFree):
it must give the same results as qt_mesolve_dev, on two calls in a row that
reuse its one preallocated workspace, and refuse systems too large for it.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_1110_0573_gb300 import systems as S

pytestmark = pytest.mark.gpu

TOL = 1e-8  # the FP64 tolerance of the master-equation parity tests


@pytest.fixture(scope="module")
def qt():
    from paper_1110_0573_gb300 import build
    build.build()
    from paper_1110_0573_gb300 import qt as q
    return q


def _solve(qt, torch, sysm, s, opts, noalloc):
    dev = torch.device("cuda")
    psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
    tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
    ex = torch.zeros((len(s["tlist"]), len(s["e_ops"])), dtype=torch.complex128, device=dev)
    d = s["H"].shape[0]
    states = torch.zeros((len(s["tlist"]), d, d), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    fn = sysm.qt_mesolve_dev_noalloc if noalloc else sysm.qt_mesolve_dev
    fn(psi0, tl, opts, ex, states=states, stats=stb)
    torch.cuda.synchronize()
    st = qt.stats_from_bytes(stb)
    assert st["status"] == 0
    return ex.cpu().numpy(), states.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice_in_a_row(qt):
    torch = pytest.importorskip("torch")
    cases = [(S.jaynes_cummings(N=6, n0=3, kappa=0.2, gamma=0.3, t_end=6.0, nt=13),
              qt.qt_opts_default(rtol=1e-8, atol=1e-10)),
             (S.kerr_cavity(N=40, t_end=4.0, nt=9),
              qt.qt_opts_default(rtol=1e-8, atol=1e-10))]
    for s, o in cases:  # two consecutive calls share the one workspace
        sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
        ref_ex, ref_states = _solve(qt, torch, sysm, s, o, noalloc=False)
        ex, states = _solve(qt, torch, sysm, s, o, noalloc=True)
        assert np.abs(ex - ref_ex).max() < TOL
        assert np.abs(states - ref_states).max() < TOL
        sysm.close()


def _diagonal_solve(qt, torch, d, precision):
    H = np.diag(np.linspace(0.0, 1.0, d))
    sysm = qt.System(H, [], [np.eye(d)])
    dev = torch.device("cuda")
    psi0 = torch.zeros(d, dtype=torch.complex128, device=dev)
    psi0[0] = 1
    tl = torch.tensor([0.0, 0.5], dtype=torch.float64, device=dev)
    ex = torch.zeros((2, 1), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    try:
        sysm.qt_mesolve_dev_noalloc(psi0, tl, qt.qt_opts_default(precision=precision), ex,
                                    stats=stb)
        torch.cuda.synchronize()
        return ex.cpu().numpy(), qt.stats_from_bytes(stb)
    finally:
        sysm.close()


@pytest.mark.parametrize("d,precision", [(307, "fp64"), (431, "mixed")])
def test_noalloc_accepts_its_largest_dimensions(qt, d, precision):
    torch = pytest.importorskip("torch")
    ex, st = _diagonal_solve(qt, torch, d, qt.QT_FP64 if precision == "fp64" else qt.QT_MIXED)
    assert st["status"] == 0
    assert np.abs(ex - 1.0).max() < 1e-6  # Tr(rho) = 1 under a Hermitian H


@pytest.mark.parametrize("d,precision", [(308, "fp64"), (432, "mixed"), (600, "mixed")])
def test_noalloc_rejects_systems_beyond_its_workspace(qt, d, precision):
    torch = pytest.importorskip("torch")
    with pytest.raises(qt.QtError) as e:
        _diagonal_solve(qt, torch, d, qt.QT_FP64 if precision == "fp64" else qt.QT_MIXED)
    assert e.value.code == qt.QT_EINVAL and "workspace" in str(e.value)
