"""GPU parity of the two-time correlation functions <A(t + tau) B(t)> (the
ODE form of the paper's correlation functions, quantum regression theorem)
against the FP64 oracle, through the C ABI: the batched one-CTA-per-t_k path
(dim <= 64) and the cooperative path (one launch per t_k), time-independent
and time-dependent Hamiltonians.

FP64: identical step counts, values within 1e-8 of the oracle.  Mixed: the
FP32 state's rounding over the run, within 2e-5 of the largest |C|."""
import math

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


def cavity(N=20, n_th=0.2):
    omega, kappa, alpha = 1.1, 0.5, 1.2
    a = S.destroy(N)
    ad = S.create(N)
    c_ops = [np.sqrt(kappa * (1 + n_th)) * a, np.sqrt(kappa * n_th) * ad]
    psi0 = np.array([np.exp(-alpha ** 2 / 2) * alpha ** k / math.sqrt(math.factorial(k))
                     for k in range(N)], dtype=complex)
    return dict(H=omega * (ad @ a), c_ops=c_ops, A=ad, B=a, psi0=psi0, omega=omega,
                kappa=kappa, n_th=n_th, alpha=alpha)


def random_case(d, seed, td=False):
    s = S.random_system(d, 2, 2, seed=seed, density=min(1.0, 6.0 / d))
    rng = np.random.default_rng(seed)
    Bm = sp.random(d, d, density=min(1.0, 4.0 / d), random_state=seed, dtype=float)
    B = sp.csr_matrix(Bm + 1j * sp.random(d, d, density=min(1.0, 4.0 / d),
                                          random_state=seed + 1, dtype=float))
    out = dict(H=s["H"], c_ops=s["c_ops"], A=s["e_ops"][0], B=B, psi0=s["psi0"], td=None)
    if td:
        X = sp.random(d, d, density=min(1.0, 4.0 / d), random_state=seed + 2, dtype=float)
        H1 = sp.csr_matrix(0.5 * (X + X.T), dtype=np.complex128)
        out["td"] = [(H1, np.array([-0.5, 0.25, 0.75, 2.5]), rng.uniform(-1.5, 1.5, 4))]
    return out


TLIST = np.array([0.0, 0.25, 0.75])
TAULIST = np.array([0.0, 0.25, 0.5, 1.0, 1.25])


def run_both(qt, c, o, rtol, atol, tlist=TLIST, taulist=TAULIST):
    corr, st = qt.qt_correlation_2op_2t(c["H"], c["c_ops"], c["A"], c["B"], c["psi0"], tlist,
                                        taulist, opts=o, td=c.get("td"))
    ref, ost = oracle.correlation_2op_2t(c["H"], c["c_ops"], c["A"], c["B"], c["psi0"], tlist,
                                         taulist, rtol=rtol, atol=atol, td=c.get("td"))
    assert st["status"] == 0
    return corr, st, ref, ost


def test_fp64_cavity_batched_path(qt):
    c = cavity()
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12)
    corr, st, ref, ost = run_both(qt, c, o, 1e-10, 1e-12)
    assert np.abs(corr - ref).max() < 1e-8
    assert st["accepted"] == ost["accepted"] and st["rejected"] == ost["rejected"]
    # and the closed form n(t) exp((i omega - kappa/2) tau), to the truncation
    for k, t in enumerate(TLIST):
        n_t = c["n_th"] + (c["alpha"] ** 2 - c["n_th"]) * np.exp(-c["kappa"] * t)
        want = n_t * np.exp((1j * c["omega"] - c["kappa"] / 2) * TAULIST)
        assert np.abs(corr[k] - want).max() < 1e-7


@pytest.mark.parametrize("d,method", [(40, "auto"), (100, "auto"), (100, "sparse")])
def test_fp64_random(qt, d, method):
    c = random_case(d, d)
    m = qt.QT_ME_AUTO if method == "auto" else qt.QT_ME_SPARSE
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12, me_method=m)
    corr, st, ref, ost = run_both(qt, c, o, 1e-10, 1e-12)
    assert np.abs(corr - ref).max() < 1e-8
    assert st["accepted"] == ost["accepted"] and st["rejected"] == ost["rejected"]


@pytest.mark.parametrize("d", [30, 100])
def test_fp64_time_dependent(qt, d):
    c = random_case(d, d + 1, td=True)
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12)
    corr, _, ref, _ = run_both(qt, c, o, 1e-10, 1e-12)
    assert np.abs(corr - ref).max() < 1e-8


@pytest.mark.parametrize("d", [20, 100])
def test_mixed(qt, d):
    c = cavity() if d == 20 else random_case(d, d + 2)
    o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED)
    corr, _, ref, _ = run_both(qt, c, o, 1e-10, 1e-12)
    assert np.abs(corr - ref).max() < 2e-5 * max(1.0, np.abs(ref).max())


def test_mixed_tensor_core_first_solve(qt):
    # rho(t_k) by the tensor-core method; the tau evolutions by the general solver
    c = random_case(160, 7)
    o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED,
                           me_method=qt.QT_ME_DENSE_TC)
    corr, _, ref, _ = run_both(qt, c, o, 1e-10, 1e-12)
    assert np.abs(corr - ref).max() < 1e-4 * max(1.0, np.abs(ref).max())


def test_more_times_than_ctas(qt):
    # n_t above the batched launch's grid: each CTA takes several t_k
    c = cavity(N=8, n_th=0.1)
    tlist = np.linspace(0.0, 4.0, 1201)
    taulist = np.array([0.0, 0.5, 1.0])
    o = qt.qt_opts_default(rtol=1e-9, atol=1e-11)
    corr, st, ref, ost = run_both(qt, c, o, 1e-9, 1e-11, tlist=tlist, taulist=taulist)
    assert np.abs(corr - ref).max() < 1e-8
    assert st["accepted"] == ost["accepted"]


def test_single_tau_and_single_time(qt):
    c = random_case(24, 3)
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12)
    corr, _, ref, _ = run_both(qt, c, o, 1e-10, 1e-12, tlist=np.array([0.3]),
                               taulist=np.array([0.0]))
    assert corr.shape == (1, 1) and abs(corr[0, 0] - ref[0, 0]) < 1e-10
    # tau = 0: Tr(A B rho(t)) with rho(t0) = rho0 exactly
    rho0 = np.outer(c["psi0"], c["psi0"].conj())
    want = np.trace(c["A"].toarray() @ c["B"].toarray() @ rho0)
    assert abs(corr[0, 0] - want) < 1e-12


def test_device_entry_all_observables(qt):
    c = cavity()
    N = 20
    n_op = S.num(N)
    sysm = qt.System(c["H"], c["c_ops"], [c["A"], c["B"], n_op])
    tl = torch.tensor(TLIST, dtype=torch.float64, device="cuda")
    tau = torch.tensor(TAULIST, dtype=torch.float64, device="cuda")
    psi = torch.tensor(c["psi0"], dtype=torch.complex128, device="cuda")
    out = torch.zeros((len(TLIST), len(TAULIST), 3), dtype=torch.complex128, device="cuda")
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12)
    sysm.qt_correlation_2op_2t_dev(psi, tl, tau, 1, o, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for m, A in enumerate([c["A"], c["B"], n_op]):
        ref, _ = oracle.correlation_2op_2t(c["H"], c["c_ops"], A, c["B"], c["psi0"], TLIST,
                                           TAULIST, rtol=1e-10, atol=1e-12)
        assert np.abs(got[:, :, m] - ref).max() < 1e-8
    sysm.close()


def test_invalid_tau(qt):
    c = cavity(N=6)
    with pytest.raises(qt.QtError) as e:
        qt.qt_correlation_2op_2t(c["H"], c["c_ops"], c["A"], c["B"], c["psi0"], TLIST,
                                 TAULIST + 0.1)
    assert e.value.code == qt.QT_EINVAL


def test_steady_state_correlation(qt):
    # <a^dag(tau) a(0)> in the thermal cavity's steady state: n_th exp((i w - k/2) tau)
    N, omega, kappa, n_th = 16, 0.9, 0.6, 0.3
    a = S.destroy(N)
    ad = S.create(N)
    c_ops = [np.sqrt(kappa * (1 + n_th)) * a, np.sqrt(kappa * n_th) * ad]
    H = omega * (ad @ a)
    taulist = np.linspace(0.0, 4.0, 9)
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12)
    corr, st = qt.qt_correlation_ss(H, c_ops, ad, a, taulist, opts=o)
    assert st["status"] == 0
    want = n_th * np.exp((1j * omega - kappa / 2) * taulist)
    assert np.abs(corr - want).max() < 1e-8
    ref, _ = oracle.correlation_ss(H, c_ops, ad, a, taulist, rtol=1e-10, atol=1e-12)
    assert np.abs(corr - ref).max() < 1e-8
