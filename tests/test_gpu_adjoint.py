"""GPU master-equation adjoint against the FP64 oracle adjoint and against
central finite differences (h = 1e-6, FP64) on the frozen step grid."""
import numpy as np
import pytest

import oracle
from paper_1110_0573_gb300 import systems as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 1e-6  # gradients vs finite differences


@pytest.fixture(scope="module")
def qt():
    from paper_1110_0573_gb300 import build
    build.build()
    from paper_1110_0573_gb300 import qt as q
    return q


def setup(qt, N, n_seg, batch, amp, gamma_scale, seed=0):
    s = S.transmon_cavity(N=N, n_seg=n_seg)
    adj = qt.Adjoint(s["H0"], s["Hd"], s["A"], s["P1"], s["P2"], s["psi0"], n_seg, s["t_seg"],
                     batch)
    omega = S.drive_vectors(batch, n_seg, amp=amp, seed=seed)
    gamma = np.tile(s["gamma"] * gamma_scale, (batch, 1))
    pr = oracle.AdjointProblem(s["H0"], s["Hd"], s["A"], s["P1"], s["P2"], s["psi0"], n_seg,
                               s["t_seg"], max_per_seg=256)
    return s, adj, omega, gamma, pr


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_forward_and_gradients_match_oracle_and_finite_differences(qt):
    batch, n_seg = 3, 6
    s, adj, omega, gamma, pr = setup(qt, 4, n_seg, batch, 0.3, np.array([3.0, 2.0, 50.0]))
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    om, ga = dev(omega), dev(gamma)
    loss = torch.zeros(batch, dtype=torch.float64, device="cuda")
    stb = torch.zeros(56, dtype=torch.uint8, device="cuda")
    adj.forward(om, ga, o, loss, stats=stb)
    go = torch.zeros((batch, n_seg), dtype=torch.float64, device="cuda")
    gg = torch.zeros((batch, 3), dtype=torch.float64, device="cuda")
    adj.backward(None, go, gg)
    torch.cuda.synchronize()
    assert qt.stats_from_bytes(stb)["status"] == 0
    loss, go, gg = loss.cpu().numpy(), go.cpu().numpy(), gg.cpu().numpy()
    h = 1e-6
    for b in range(batch):
        # forward: same controller as the oracle
        ol, ons, ohg = pr.forward(omega[b], gamma[b], rtol=1e-8, atol=1e-10)
        ns, hg = adj.grid(b)
        assert abs(loss[b] - ol) < 1e-9
        # gradients: the oracle's discrete adjoint on the GPU's grid
        l2, ogo, ogg = pr.grad(omega[b], gamma[b], ns, hg)
        assert abs(l2 - loss[b]) < 1e-12
        assert np.abs(go[b] - ogo).max() <= 1e-9 * max(1.0, np.abs(ogo).max())
        assert np.abs(gg[b] - ogg).max() <= 1e-9 * max(1.0, np.abs(ogg).max())
    # central finite differences of the GPU's own fixed-grid loss
    lp = torch.zeros(batch, dtype=torch.float64, device="cuda")
    lm = torch.zeros(batch, dtype=torch.float64, device="cuda")
    for i in range(n_seg):
        e = np.zeros_like(omega)
        e[:, i] = h
        adj.loss_fixed(dev(omega + e), ga, lp)
        adj.loss_fixed(dev(omega - e), ga, lm)
        fd = ((lp - lm) / (2 * h)).cpu().numpy()
        assert np.all(np.abs(fd - go[:, i]) <= REL * np.maximum(np.abs(go[:, i]), 1e-3)), (i, fd, go[:, i])
    for k in range(3):
        e = np.zeros_like(gamma)
        e[:, k] = h
        adj.loss_fixed(om, dev(gamma + e), lp)
        adj.loss_fixed(om, dev(gamma - e), lm)
        fd = ((lp - lm) / (2 * h)).cpu().numpy()
        assert np.all(np.abs(fd - gg[:, k]) <= REL * np.maximum(np.abs(gg[:, k]), 1e-3)), (k, fd, gg[:, k])
    adj.close()


def test_autograd_function(qt):
    batch, n_seg = 2, 4
    s, adj, omega, gamma, pr = setup(qt, 3, n_seg, batch, 0.2, np.array([2.0, 1.0, 10.0]),
                                     seed=5)
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    om = dev(omega).requires_grad_(True)
    ga = dev(gamma).requires_grad_(True)
    loss = qt.master_equation_loss(adj, om, ga, o)
    w = torch.tensor([0.7, -1.3], dtype=torch.float64, device="cuda")
    (loss * w).sum().backward()
    for b in range(batch):
        ns, hg = adj.grid(b)
        _, ogo, ogg = pr.grad(omega[b], gamma[b], ns, hg)
        assert np.allclose(om.grad[b].cpu().numpy(), w[b].item() * ogo, rtol=1e-9, atol=1e-12)
        assert np.allclose(ga.grad[b].cpu().numpy(), w[b].item() * ogg, rtol=1e-9, atol=1e-12)
    adj.close()


def test_full_size_transmon_cavity_sample(qt):
    # dim 60, 64 segments; a batch of 4 of the 256 drive vectors
    batch, n_seg = 4, 64
    s, adj, omega, gamma, pr = setup(qt, 20, n_seg, batch, 0.05, np.ones(3), seed=2)
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    om, ga = dev(omega), dev(gamma)
    loss = torch.zeros(batch, dtype=torch.float64, device="cuda")
    adj.forward(om, ga, o, loss)
    go = torch.zeros((batch, n_seg), dtype=torch.float64, device="cuda")
    gg = torch.zeros((batch, 3), dtype=torch.float64, device="cuda")
    adj.backward(None, go, gg)
    torch.cuda.synchronize()
    go, gg = go.cpu().numpy(), gg.cpu().numpy()
    # finite differences for a few segments and every rate
    h = 1e-6
    lp = torch.zeros(batch, dtype=torch.float64, device="cuda")
    lm = torch.zeros(batch, dtype=torch.float64, device="cuda")
    for i in (0, 31, 63):
        e = np.zeros_like(omega)
        e[:, i] = h
        adj.loss_fixed(dev(omega + e), ga, lp)
        adj.loss_fixed(dev(omega - e), ga, lm)
        fd = ((lp - lm) / (2 * h)).cpu().numpy()
        assert np.all(np.abs(fd - go[:, i]) <= REL * np.maximum(np.abs(go[:, i]), 1e-4)), (i, fd, go[:, i])
    for k in range(3):
        e = np.zeros_like(gamma)
        e[:, k] = h
        adj.loss_fixed(om, dev(gamma + e), lp)
        adj.loss_fixed(om, dev(gamma - e), lm)
        fd = ((lp - lm) / (2 * h)).cpu().numpy()
        assert np.all(np.abs(fd - gg[:, k]) <= REL * np.maximum(np.abs(gg[:, k]), 1e-4)), (k, fd, gg[:, k])
    # the oracle adjoint on the GPU's grid for one vector
    ns, hg = adj.grid(0)
    _, ogo, ogg = pr.grad(omega[0], gamma[0], ns, hg)
    assert np.abs(go[0] - ogo).max() <= 1e-9 * max(1.0, np.abs(ogo).max())
    assert np.abs(gg[0] - ogg).max() <= 1e-9 * max(1.0, np.abs(ogg).max())
    adj.close()
