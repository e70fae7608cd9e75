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


def dense_collapse(s):
    # the library forms all collapse terms on the tensor cores when one
    # collapse operator holds at least 32 entries in some row
    return any(np.diff(c.tocsr().indptr).max(initial=0) >= 32 for c in s["c_ops"])


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
    # collapse terms: FP32 sparse sums, or the BF16 hi/lo bound of the two
    # dense products when the operators are dense (T = C rho then T C^dag)
    crel = 2 * RHS_REL if dense_collapse(s) else 1e-6
    lim = RHS_REL * hb + crel * cb + 1e-6 * np.abs(rho).max() + 1e-12
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


def dense_collapse_system(d, n_c, seed, t_end=0.3, nt=4):
    """A random Hermitian H (Gaussian entries / sqrt(d)) with n_c dense
    random collapse operators (entries / sqrt(d) scaled by 0.3), a random ket,
    the ladder number operator / d and a random dense Hermitian observable."""
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0 * d)
    H = 0.5 * (X + X.conj().T)
    cs = [0.3 * (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0 * d)
          for _ in range(n_c)]
    O = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    O = 0.5 * (O + O.conj().T) / np.sqrt(d)
    psi = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    import scipy.sparse as sp
    return dict(H=sp.csr_matrix(H), c_ops=[sp.csr_matrix(c) for c in cs],
                e_ops=[sp.csr_matrix(np.diag(np.arange(d) / d)), sp.csr_matrix(O)],
                psi0=psi / np.linalg.norm(psi), tlist=np.linspace(0.0, t_end, nt))


@pytest.mark.parametrize("d,n_c,seed", [(96, 1, 5), (200, 2, 6), (256, 3, 7)])
def test_dense_collapse_rhs_matches_oracle_entrywise(qt, d, n_c, seed):
    # every collapse term C_n rho C_n^dag from the two dense tensor-core
    # products; one tile (96), ragged (200), exact tiles with three operators
    s = dense_collapse_system(d, n_c, seed)
    assert dense_collapse(s)
    rho = random_dm(d, seed)
    ref = oracle.me_rhs(s["H"], s["c_ops"], rho)
    got, st = rhs_on_device(qt, s, rho, qt.QT_MIXED, qt.QT_ME_DENSE_TC)
    assert st["status"] == 0
    hb, cb = bounds(s, rho)
    err = np.abs(got - ref)
    lim = RHS_REL * hb + 2 * RHS_REL * cb + 1e-12
    worst = np.unravel_index(np.argmax(err / lim), err.shape)
    assert np.all(err <= lim), (worst, err[worst], lim[worst])
    # the same right-hand side through the sparse FP32 path, as a cross-check
    sp32, _ = rhs_on_device(qt, s, rho, qt.QT_MIXED, qt.QT_ME_SPARSE)
    assert np.all(np.abs(sp32 - ref) <= 1e-5 * (hb + cb) + 1e-12)


def test_dense_collapse_solve_against_fp64_oracle(qt):
    s = dense_collapse_system(160, 2, 8, t_end=0.5, nt=6)
    o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED,
                           me_method=qt.QT_ME_DENSE_TC)
    ex, states, st = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                   opts=o, store_states=True)
    ref, rstates, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                     rtol=1e-9, atol=1e-11, store_states=True)
    assert st["status"] == 0 and st["accepted"] > 0
    err = np.abs(ex - ref).max()
    print(f"dense collapse tensor-core solve: max error {err:.3e}")
    assert err < 1e-4
    for r in states:  # trace kept, Hermitian
        assert abs(np.trace(r) - 1) < 1e-4 and np.abs(r - r.conj().T).max() < 1e-6
