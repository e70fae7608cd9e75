"""Pins of the input builders: hand-checkable matrix entries and algebra."""
import numpy as np
import pytest

from paper_1110_0573_gb300 import systems as S


def dense(m):
    return np.asarray(m.todense())


def test_destroy_entries_and_commutator():
    a = dense(S.destroy(4))
    expect = np.zeros((4, 4))
    expect[0, 1], expect[1, 2], expect[2, 3] = 1.0, np.sqrt(2.0), np.sqrt(3.0)
    assert np.array_equal(a, expect)
    ad = dense(S.create(4))
    comm = a @ ad - ad @ a
    # [a, a^dag] = 1 except in the last row of the truncated space
    assert np.allclose(np.diag(comm)[:-1], 1.0)
    assert np.isclose(comm[-1, -1], -3.0)
    assert np.allclose(dense(S.num(4)), ad @ a)


def test_two_level_conventions():
    sm, sp_, sz = dense(S.sigmam()), dense(S.sigmap()), dense(S.sigmaz())
    sx, sy = dense(S.sigmax()), dense(S.sigmay())
    g, e = S.basis(2, 0), S.basis(2, 1)
    assert np.allclose(sm @ e, g) and np.allclose(sm @ g, 0)
    assert np.allclose(sz, sp_ @ sm - sm @ sp_)
    assert np.allclose(np.diag(sz), [-1, 1])
    # Pauli algebra: [sx, sy] = 2 i sz, and each squares to one
    assert np.allclose(sx @ sy - sy @ sx, 2j * sz)
    for s in (sx, sy, sz):
        assert np.allclose(s @ s, np.eye(2))


def test_tensor_order_first_factor_most_significant():
    a = S.tensor(S.destroy(3), S.qeye(2))
    # |n=1, q=0> is index 2; a maps it to |0, 0> (index 0) with amplitude 1
    v = np.zeros(6, complex)
    v[2] = 1
    assert np.allclose(a @ v, np.eye(6)[0])
    ket = S.tensor(S.basis(3, 2), S.basis(2, 1))
    assert np.argmax(np.abs(ket)) == 2 * 2 + 1


@pytest.mark.parametrize("builder", [S.jaynes_cummings, S.kerr_cavity, S.cavity_thermal_decay,
                                     S.driven_tls, S.iswap_pair])
def test_hamiltonians_hermitian(builder):
    s = builder()
    H = dense(s["H"])
    assert np.allclose(H, H.conj().T)
    for e in s["e_ops"]:
        E = dense(e)
        assert np.allclose(E, E.conj().T) or builder is S.kerr_cavity
    assert np.isclose(np.linalg.norm(s["psi0"]), 1.0)


def test_xxz_small_chain_structure():
    s = S.xxz_chain(L=4)
    H = dense(s["H"])
    assert np.allclose(H, H.conj().T)
    # Neel |e,g,e,g> with site 0 most significant: bits 1010 -> index 10
    assert np.argmax(np.abs(s["psi0"])) == 0b1010
    assert len(s["c_ops"]) == 8 and len(s["e_ops"]) == 4
    # <sz_0> on the Neel state is +1 (excited), <sz_1> is -1
    psi = s["psi0"]
    assert np.isclose(np.vdot(psi, s["e_ops"][0] @ psi).real, 1.0)
    assert np.isclose(np.vdot(psi, s["e_ops"][1] @ psi).real, -1.0)


def test_xxz_full_size_nnz():
    s = S.xxz_chain(L=10)
    H = s["H"]
    assert H.shape == (1024, 1024)
    row_nnz = np.diff(H.indptr)
    # diagonal + 10 field flips + up to 9 flip-flops per row
    assert row_nnz.max() <= 20 and row_nnz.min() >= 11


def test_xxz_off_diagonal_columns_are_bit_flips():
    # every off-diagonal entry of H (and of H_eff: the collapse operators add
    # only diagonal terms) joins states that differ by one flipped site or by
    # a flipped neighbouring pair, 10 + 9 masks at L = 10
    s = S.xxz_chain(L=10)
    H = s["H"].tocoo()
    off = H.row != H.col
    masks = set((H.row[off] ^ H.col[off]).tolist())
    want = {1 << k for k in range(10)} | {3 << k for k in range(9)}
    assert masks == want
    for c in s["c_ops"]:
        cc = (c.conj().T @ c).tocoo()
        assert np.all(cc.row == cc.col)


def test_tight_binding_chain_structure():
    s = S.tight_binding_chain(d=10)
    H = dense(s["H"])
    assert np.allclose(H, H.conj().T)
    assert np.count_nonzero(H) == 18 and np.allclose(np.diag(H, 1), -1.0)
    C = dense(s["c_ops"][0])
    assert np.count_nonzero(C) == 9 and C[0, 1] != 0 and C[1, 0] == 0
    assert np.argmax(np.abs(s["psi0"])) == 5


def test_jc_resonant_rabi_structure():
    # |1, g> and |0, e> are degenerate under the uncoupled part (resonance)
    s = S.jaynes_cummings(N=3, g=0.0, kappa=0.0, gamma=0.0, n0=0)
    H = dense(s["H"])
    i1g = 1 * 2 + 0
    i0e = 0 * 2 + 1
    assert np.isclose(H[i1g, i1g], H[i0e, i0e])
