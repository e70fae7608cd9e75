"""GPU parity of the tensor-core master-equation path (QT_ME_DENSE_TC):
H_eff rho as one dense product on tcgen05 tensor cores with BF16 hi/lo
operands and FP32 accumulation, rho H_eff^dag as its conjugate transpose,
collapse terms in FP32 -- against the FP64 oracle of Eq. (master_equation).

Tolerances follow from the arithmetic.  Splitting x = hi + lo in BF16 leaves
|x - hi - lo| <= 2^-17 |x|, and the dropped lo*lo product is below
2^-16 |a||b|, so each entry of the product is within ~2^-15 of
(|H_eff||rho|)_ij; FP32 accumulation over K = 2 dim terms adds
~K * 2^-24 relative.  The right-hand side is compared entry by entry against
that bound; solutions against the FP64 oracle with a bound stated per test."""
import numpy as np
import pytest

import oracle
from paper_1110_0573_gb300 import systems as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RHS_REL = 2.0 ** -14  # per entry, relative to (|H_eff||rho|)_ij + (|rho||H_eff^dag|)_ij


@pytest.fixture(scope="module")
def qt():
    from paper_1110_0573_gb300 import build
    build.build()
    from paper_1110_0573_gb300 import qt as q
    return q


def dense(m):
    return np.asarray(m.todense()) if hasattr(m, "todense") else np.asarray(m)


def random_dm(d, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    r = X @ X.conj().T
    return r / np.trace(r)


def rhs_on_device(qt, s, rho, precision, method):
    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
    r = torch.tensor(rho, dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(r)
    stb = torch.zeros(56, dtype=torch.uint8, device="cuda")
    o = qt.qt_opts_default(precision=precision, me_method=method)
    sysm.qt_me_rhs_dev(r, out, o, stats=stb)
    torch.cuda.synchronize()
    st = qt.stats_from_bytes(stb)
    sysm.close()
    return out.cpu().numpy(), st


def bounds(s, rho):
    H = dense(s["H"])
    Cs = [dense(c) for c in s["c_ops"]]
    Heff = H - 0.5j * sum((c.conj().T @ c for c in Cs), np.zeros_like(H))
    b = np.abs(Heff) @ np.abs(rho)
    hb = b + b.T
    cb = sum((np.abs(c) @ np.abs(rho) @ np.abs(c).T for c in Cs), np.zeros(rho.shape))
    return hb, cb


@pytest.mark.parametrize("d,density,seed", [(20, 0.5, 0), (100, 0.3, 1), (200, 1.0, 2),
                                            (256, 0.05, 3), (300, 0.1, 4)])
def test_rhs_matches_oracle_entrywise(qt, d, density, seed):
    # one M tile (d <= 128), ragged tails (100, 200, 300), an exact multiple
    # of the tile (256), a dense H (density 1)
    s = S.random_system(d, 2, 1, seed=seed, density=density)
    rho = random_dm(d, seed)
    ref = oracle.me_rhs(s["H"], s["c_ops"], rho)
    got, st = rhs_on_device(qt, s, rho, qt.QT_MIXED, qt.QT_ME_DENSE_TC)
    assert st["status"] == 0
    hb, cb = bounds(s, rho)
    err = np.abs(got - ref)
    lim = RHS_REL * hb + 1e-6 * (cb + np.abs(rho).max()) + 1e-12
    worst = np.unravel_index(np.argmax(err / lim), err.shape)
    assert np.all(err <= lim), (worst, err[worst], lim[worst])
    # the result is Hermitian (the Hamiltonian part exactly by construction)
    assert np.abs(got - got.conj().T).max() <= 1e-5 * np.abs(got).max()


def test_rhs_agrees_with_sparse_mixed_path(qt):
    s = S.xxz_chain(L=8)
    rho = random_dm(256, 7)
    a, sa = rhs_on_device(qt, s, rho, qt.QT_MIXED, qt.QT_ME_DENSE_TC)
    b, sb = rhs_on_device(qt, s, rho, qt.QT_MIXED, qt.QT_ME_SPARSE)
    ref = oracle.me_rhs(s["H"], s["c_ops"], rho)
    assert sa["status"] == 0 and sb["status"] == 0
    hb, cb = bounds(s, rho)
    assert np.all(np.abs(a - ref) <= RHS_REL * hb + 1e-6 * cb + 1e-12)
    assert np.all(np.abs(b - ref) <= 1e-5 * (hb + cb) + 1e-12)


def test_dense_method_needs_mixed_precision(qt):
    s = S.jaynes_cummings()
    o = qt.qt_opts_default(me_method=qt.QT_ME_DENSE_TC)  # FP64 default
    with pytest.raises(qt.QtError) as e:
        qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"][:3], opts=o)
    assert e.value.code == qt.QT_EINVAL


@pytest.mark.parametrize("L,t_end", [(6, 2.0), (8, 1.0)])
def test_xxz_solve_against_fp64_oracle(qt, L, t_end):
    # dim 64 (one tile row, half of it padding) and dim 256 (2 x 4 tiles)
    s = S.xxz_chain(L=L, t_end=t_end, nt=11)
    o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED,
                           me_method=qt.QT_ME_DENSE_TC)
    ex, _, st = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o)
    ref, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                               rtol=1e-9, atol=1e-11)
    assert st["status"] == 0 and st["accepted"] > 0
    err = np.abs(ex - ref).max()
    print(f"L={L} dense tensor-core solve: max |<sz_i> - oracle| = {err:.3e}, "
          f"{st['accepted']} steps")
    assert err < 1e-4
    # the same call again gives the same numbers (fixed reduction orders)
    ex2, _, _ = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o)
    assert np.array_equal(ex, ex2)


def test_jaynes_cummings_solve(qt):
    s = S.jaynes_cummings(t_end=10.0, nt=41)
    o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED,
                           me_method=qt.QT_ME_DENSE_TC)
    ex, _, st = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o)
    ref, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                               rtol=1e-9, atol=1e-11)
    assert st["status"] == 0
    err = np.abs(ex - ref).max()
    print(f"Jaynes-Cummings dense tensor-core solve: max error {err:.3e}")
    assert err < 1e-4
