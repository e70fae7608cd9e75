"""GPU parity of qt_mesolve (paper section 3.1) and qt_expect against the
FP64 oracle, through the C ABI.  FP64 mode: expectation values and states
within 1e-8 absolute; mixed mode (complex FP32 state): within the stated
tolerance."""
import numpy as np
import pytest

import oracle
from paper_1110_0573_gb300 import systems as S

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-8
# complex FP32 state at rtol = 1e-6, atol = 1e-8 on both sides: rounding of
# the stored state (~6e-8 relative per step) accumulates over ~1e3 steps
MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def qt():
    from paper_1110_0573_gb300 import build
    build.build()
    from paper_1110_0573_gb300 import qt as q
    return q


def test_fp64_jaynes_cummings_full_config(qt):
    s = S.jaynes_cummings()
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    ex, _, st = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o)
    ref, _, ost = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                 rtol=1e-8, atol=1e-10)
    assert np.abs(ex - ref).max() < FP64_TOL
    assert st["status"] == 0 and abs(st["accepted"] - ost["accepted"]) <= 2


@pytest.mark.parametrize("d,n_c,density,seed", [(1, 1, 1.0, 0), (3, 1, 0.7, 1), (7, 2, 0.5, 2),
                                                (16, 3, 0.3, 3), (41, 2, 0.15, 4)])
def test_fp64_random_systems_with_states(qt, d, n_c, density, seed):
    s = S.random_system(d, n_c, 2, seed=seed, density=density, nt=6, t_end=1.5)
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12)
    ex, states, _ = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o,
                                  store_states=True)
    ref, rstates, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                     rtol=1e-10, atol=1e-12, store_states=True)
    assert np.abs(ex - ref).max() < FP64_TOL
    assert np.abs(states - rstates).max() < FP64_TOL
    # trace and Hermiticity are kept
    for r in states:
        assert abs(np.trace(r) - 1) < 1e-8 and np.abs(r - r.conj().T).max() < 1e-8


def test_density_matrix_input_and_no_observables(qt):
    s = S.cavity_thermal_decay(N=6, kappa=0.8, nth=0.2, n0=2, t_end=3.0, nt=7)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6))
    rho0 = X @ X.conj().T
    rho0 /= np.trace(rho0)
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12)
    ex, states, _ = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], rho0, s["tlist"], opts=o,
                                  store_states=True)
    ref, rst, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], rho0, s["tlist"], rtol=1e-10,
                                 atol=1e-12, store_states=True)
    assert np.abs(ex - ref).max() < FP64_TOL and np.abs(states - rst).max() < FP64_TOL
    _, states2, _ = qt.qt_mesolve(s["H"], s["c_ops"], [], rho0, s["tlist"], opts=o,
                                  store_states=True)
    assert np.abs(states2 - rst).max() < FP64_TOL


def test_fp64_xxz_chain_six_sites(qt):
    s = S.xxz_chain(L=6, t_end=2.0, nt=11)
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    ex, _, _ = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o)
    ref, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-8,
                               atol=1e-10)
    assert np.abs(ex - ref).max() < FP64_TOL


def test_mixed_kerr(qt):
    s = S.kerr_cavity(t_end=20.0, nt=401)
    o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED)
    ex, _, _ = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o)
    ref, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-6,
                               atol=1e-8)
    err = np.abs(ex - ref).max()
    print(f"mixed kerr ME: max |diff| {err:.2e}")
    assert err < MIXED_TOL


def test_step_limit(qt):
    s = S.jaynes_cummings(N=3, n0=1, t_end=10.0, nt=3)
    with pytest.raises(qt.QtError) as e:
        qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                      opts=qt.qt_opts_default(max_steps=3))
    assert e.value.code == qt.QT_ESTEP


def test_expect_kets_and_density_matrices(qt):
    s = S.random_system(9, 1, 1, seed=8, density=0.5)
    O = s["e_ops"][0]
    rng = np.random.default_rng(2)
    kets = rng.standard_normal((5, 9)) + 1j * rng.standard_normal((5, 9))
    assert np.abs(qt.qt_expect(O, kets, True) - oracle.expect(O, kets, True)).max() < 1e-12
    dms = rng.standard_normal((3, 9, 9)) + 1j * rng.standard_normal((3, 9, 9))
    assert np.abs(qt.qt_expect(O, dms, False) - oracle.expect(O, dms, False)).max() < 1e-12


def test_hermitian_solver_matches_general_solver_at_dim_1024(qt):
    # QT_ME_AUTO (Hermitian solver: one product Y = H_eff rho per right-hand
    # side, upper-triangle combine) against QT_ME_SPARSE (general solver, no
    # symmetry assumed) on the dim-1024 XXZ chain in FP64; the mixed Hermitian
    # solver (FP32 state and step control) against that FP64 result
    s = S.xxz_chain(t_end=0.2, nt=5)
    res = {}
    for key, p, m, rtol, atol in [("auto64", qt.QT_FP64, qt.QT_ME_AUTO, 1e-8, 1e-10),
                                  ("gen64", qt.QT_FP64, qt.QT_ME_SPARSE, 1e-8, 1e-10),
                                  ("auto32", qt.QT_MIXED, qt.QT_ME_AUTO, 1e-6, 1e-8)]:
        o = qt.qt_opts_default(rtol=rtol, atol=atol, precision=p, me_method=m)
        res[key] = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o)
        assert res[key][2]["status"] == 0
    assert np.abs(res["auto64"][0] - res["gen64"][0]).max() < 1e-10
    assert np.abs(res["auto32"][0] - res["auto64"][0]).max() < MIXED_TOL


@pytest.fixture(scope="module")
def xxz_oracle():
    # the dissipative XXZ chain at its full size (L = 10, dim 1024) on a short
    # window: the oracle's literal Lindblad form in FP64 (about 20 right-hand
    # sides of ~1.5 s each on one host core)
    s = S.xxz_chain(t_end=0.02, nt=3)
    ex, _, st = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-8,
                               atol=1e-10)
    return s, ex


@pytest.mark.parametrize("method,precision,tol", [("auto", "fp64", FP64_TOL),
                                                  ("sparse", "fp64", FP64_TOL),
                                                  ("auto", "mixed", MIXED_TOL),
                                                  ("dense_tc", "mixed", MIXED_TOL)])
def test_xxz_dim1024_against_the_oracle(qt, xxz_oracle, method, precision, tol):
    s, ref = xxz_oracle
    m = {"auto": qt.QT_ME_AUTO, "sparse": qt.QT_ME_SPARSE, "dense_tc": qt.QT_ME_DENSE_TC}[method]
    fp64 = precision == "fp64"
    o = qt.qt_opts_default(rtol=1e-8 if fp64 else 1e-6, atol=1e-10 if fp64 else 1e-8,
                           precision=qt.QT_FP64 if fp64 else qt.QT_MIXED, me_method=m)
    ex, _, st = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o)
    assert st["status"] == 0
    err = np.abs(ex - ref).max()
    print(f"xxz dim 1024 {method} {precision}: max |diff| {err:.2e}")
    assert err < tol


def test_xxz_dim1024_right_hand_side_against_the_oracle(qt):
    # one right-hand side of the full-size chain at a random density matrix,
    # entry by entry against the largest entry: FP64 paths to 1e-12, the FP32
    # path (rho rounded to FP32, FP32 arithmetic) to 1e-5
    torch = pytest.importorskip("torch")
    s = S.xxz_chain()
    d = 1024
    rng = np.random.default_rng(11)
    X = rng.standard_normal((d, 64)) + 1j * rng.standard_normal((d, 64))
    rho = X @ X.conj().T
    rho /= np.trace(rho).real
    ref = oracle.me_rhs(s["H"], s["c_ops"], rho)
    scale = np.abs(ref).max()
    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
    r = torch.tensor(rho, dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(r)
    for m, p, tol in [(qt.QT_ME_AUTO, qt.QT_FP64, 1e-12), (qt.QT_ME_SPARSE, qt.QT_FP64, 1e-12),
                      (qt.QT_ME_AUTO, qt.QT_MIXED, 1e-5)]:
        sysm.qt_me_rhs_dev(r, out, qt.qt_opts_default(me_method=m, precision=p))
        torch.cuda.synchronize()
        err = np.abs(out.cpu().numpy() - ref).max() / scale
        assert err < tol, (m, p, err)
    sysm.close()


def test_non_hermitian_initial_matrix_takes_the_general_solver(qt):
    # an initial operator that is not Hermitian (e.g. a |0><1| coherence, as
    # in two-time correlation functions) is evolved by the general solver
    s = S.cavity_thermal_decay(N=5, kappa=0.7, nth=0.1, n0=1, t_end=2.0, nt=5)
    X = np.zeros((5, 5), dtype=np.complex128)
    X[0, 1] = 1.0
    X[2, 2] = 0.5
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12)
    ex, states, st = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], X, s["tlist"], opts=o,
                                   store_states=True)
    ref, rstates, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], X, s["tlist"], rtol=1e-10,
                                     atol=1e-12, store_states=True)
    assert st["status"] == 0
    assert np.abs(states - rstates).max() < FP64_TOL
