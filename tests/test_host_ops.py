"""Host logic of the operator preparation (paper section 3.2, Eq. (heff);
no GPU): the library's own conversion of CSR input, H_eff = H - (i/2)
sum_n C_n^dag C_n, its ELL packing and the shared-memory dictionary forms,
compiled from csrc/qt_host.cpp into a small checker (tests/host_ops_check.cu)
and compared with scipy entry for entry."""
import json
import os
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1110_0573_gb300 import systems as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    from paper_1110_0573_gb300 import build
    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    build.build()
    out = str(tmp_path_factory.mktemp("hostops") / "host_ops_check")
    lib = os.path.join(ROOT, "paper_1110_0573_gb300", "_build")
    cmd = [nvcc, "-std=c++17", "-O1", f"-I{os.path.join(ROOT, 'include')}",
           os.path.join(ROOT, "tests", "host_ops_check.cu"), "-o", out, f"-L{lib}", "-lqt",
           "-Xlinker", f"-rpath={lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return out


def run(checker, tmp_path, H, c_ops, raw=None):
    """raw: optional (indptr, indices, values) for H, passed as given."""
    d = H.shape[0]
    f = tmp_path / "ops.bin"
    with open(f, "wb") as fp:
        np.array([d, len(c_ops)], dtype=np.int64).tofile(fp)
        mats = [raw] + [None] * len(c_ops) if raw is not None else [None] * (1 + len(c_ops))
        for m, A in zip(mats, [H] + list(c_ops)):
            if m is None:
                A = sp.csr_matrix(A)
                m = (A.indptr, A.indices, A.data)
            ptr, idx, val = m
            np.array([len(idx)], dtype=np.int64).tofile(fp)
            np.asarray(ptr, dtype=np.int64).tofile(fp)
            np.asarray(idx, dtype=np.int32).tofile(fp)
            np.asarray(val, dtype=np.complex128).tofile(fp)
    r = subprocess.run([checker, str(f)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return json.loads(r.stdout)


def csr_of(j, d):
    return sp.csr_matrix((np.array(j["re"]) + 1j * np.array(j["im"]), j["col"], j["ptr"]),
                         shape=(d, d))


def heff_of(H, c_ops):
    return (sp.csr_matrix(H) - 0.5j * sum((sp.csr_matrix(c).conj().T @ sp.csr_matrix(c))
                                         for c in c_ops)).toarray()


def check_dict_exact(j, d, H, c_ops):
    """The dictionary reproduces the library's H_eff exactly, and that H_eff
    is scipy's to rounding."""
    lib = csr_of(j["heff"], d).toarray()
    assert np.array_equal(dict_matrix(j["dict"], d), lib)
    want = heff_of(H, c_ops)
    assert np.abs(lib - want).max() <= 1e-14 * np.abs(want).max()


def dict_matrix(dj, d):
    """H_eff rebuilt from its dictionary: diagonal, then every coded entry."""
    M = np.diag(np.array(dj["diag_re"]) + 1j * np.array(dj["diag_im"]))
    tab = np.array(dj["tab_re"]) + 1j * np.array(dj["tab_im"])
    code = np.array(dj["code"], dtype=np.int64).reshape(dj["w"], d)
    if dj["groups"] == 0:  # column | value index << 16; padding: own column, value 0
        for s in range(dj["w"]):
            for i in range(d):
                c, v = code[s, i] & 0xFFFF, code[s, i] >> 16
                if v:
                    assert M[i, c] == 0  # one code per entry
                    M[i, c] = tab[v]
                else:
                    assert c == i
    else:  # plain columns, the slots of value g + 1 contiguous; padding: column d
        start = 0
        for g, end in enumerate(dj["gend"]):
            for s in range(start, end):
                for i in range(d):
                    c = code[s, i]
                    if c != d:
                        assert M[i, c] == 0
                        M[i, c] = tab[g + 1]
            start = end
    return M


def test_conversion_and_effective_hamiltonian(checker, tmp_path):
    # unsorted and repeated columns and an explicit zero in H's input: the
    # conversion sorts, sums and drops; H_eff against scipy
    rng = np.random.default_rng(5)
    s = S.random_system(12, 2, 1, seed=5, density=0.4)
    H = sp.csr_matrix(s["H"])
    ptr, idx, val = [0], [], []
    for i in range(12):
        row = H.getrow(i)
        cols, vals = list(row.indices), list(row.data)
        if cols:  # split the first entry in two halves, append a zero
            cols += [cols[0], (cols[0] + 1) % 12]
            vals[0] = vals[0] / 2
            vals += [vals[0], 0.0]
        order = rng.permutation(len(cols))
        idx += [cols[k] for k in order]
        val += [vals[k] for k in order]
        ptr.append(len(idx))
    j = run(checker, tmp_path, H, s["c_ops"], raw=(ptr, idx, val))
    Hc = csr_of(j["H"], 12)
    assert np.all(np.diff(Hc.indptr) >= 0)
    for i in range(12):
        cols = Hc.indices[Hc.indptr[i]:Hc.indptr[i + 1]]
        assert np.all(np.diff(cols) > 0)  # sorted, merged
    assert np.all(Hc.data != 0)
    assert np.abs(Hc.toarray() - H.toarray()).max() < 1e-15
    want = heff_of(H, s["c_ops"])
    got = csr_of(j["heff"], 12).toarray()
    assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


def test_ell_packing_has_an_own_column_slot(checker, tmp_path):
    # slot-major ELL (entry s of row i at s d + i), padded with value 0 at
    # column = row, every row holding a slot in its own column
    s = S.kerr_cavity(N=16)
    j = run(checker, tmp_path, s["H"], s["c_ops"])
    d, w = 16, j["ell"]["w"]
    col = np.array(j["ell"]["col"]).reshape(w, d)
    v = (np.array(j["ell"]["re"]) + 1j * np.array(j["ell"]["im"])).reshape(w, d)
    M = np.zeros((d, d), complex)
    for s_ in range(w):
        for i in range(d):
            M[i, col[s_, i]] += v[s_, i]
    assert np.all((col == np.arange(d)).any(axis=0))
    want = heff_of(s["H"], s["c_ops"])
    assert np.abs(M - want).max() <= 1e-14 * np.abs(want).max()
    assert w == 3  # tridiagonal H_eff


@pytest.mark.parametrize("L", [8, 10])
def test_spin_chain_dictionary_one_mask_per_slot(checker, tmp_path, L):
    # the XXZ chain: two off-diagonal values (field, flip-flop), grouped, and
    # every slot of a value holds one bit-flip mask i ^ j for all its rows
    s = S.xxz_chain(L=L)
    d = 2 ** L
    j = run(checker, tmp_path, s["H"], s["c_ops"])
    dj = j["dict"]
    assert dj is not None and dj["groups"] == 2
    assert dj["gend"] == [L, 2 * L - 1] and dj["w"] == 2 * L - 1
    check_dict_exact(j, d, s["H"], s["c_ops"])
    code = np.array(dj["code"], dtype=np.int64).reshape(dj["w"], d)
    rows = np.arange(d)
    for sl in range(dj["w"]):
        present = code[sl] != d
        masks = set((rows[present] ^ code[sl][present]).tolist())
        assert len(masks) == 1
        m = masks.pop()
        assert m in {1 << k for k in range(L)} | {3 << k for k in range(L - 1)}


def test_tight_binding_dictionary_grouped_by_value(checker, tmp_path):
    # one hopping value at columns i +- 1 (masks i ^ (i +- 1) take many
    # values): grouped, two slots, entries in column order
    s = S.tight_binding_chain(d=300)
    j = run(checker, tmp_path, s["H"], s["c_ops"])
    dj = j["dict"]
    assert dj["groups"] == 1 and dj["gend"] == [2] and dj["w"] == 2
    check_dict_exact(j, 300, s["H"], s["c_ops"])


def test_ladder_dictionary_plain_codes_and_too_many_values(checker, tmp_path):
    # Kerr cavity at dim 200: 200 distinct ladder values, plain codes;
    # a dense random Hamiltonian has more distinct values than the table holds
    s = S.kerr_cavity(N=200)
    j = run(checker, tmp_path, s["H"], s["c_ops"])
    dj = j["dict"]
    assert dj["groups"] == 0 and len(dj["tab_re"]) == 200
    check_dict_exact(j, 200, s["H"], s["c_ops"])
    rng = np.random.default_rng(7)
    A = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    j = run(checker, tmp_path, sp.csr_matrix(A + A.conj().T), [])
    assert j["dict"] is None
