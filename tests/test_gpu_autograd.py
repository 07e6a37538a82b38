"""Differentiation stage: dJ/dw and dJ/df0 of the cost (Eq. 2 with Eq. A.1),
through the C ABI and through the torch.autograd wrapper, against the FP64
oracle and central finite differences.

Tolerances: dJ/df0 elementwise max |d| <= 1e-4 * max |oracle| (float32 P^T r,
exact fixed-point scatter); dJ/dw as the parity tests (1e-3 of the norm);
finite differences on the float32 cost as stated per test."""
import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S

from cases import SEQUENCE, make_problem, tiny_problem, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1102_1712_gb300 import build as B
    B.build()
    from paper_1102_1712_gb300 import pcasolve
    pcasolve.lib()
    return pcasolve


def test_grad_f0_matches_oracle_and_is_deterministic(P):
    pb = tiny_problem()
    d = to_dev(pb)
    w = np.array([0.5, -0.2, 0.4])
    J, G, ab, g1 = P.cost_grad_f0(d["f0"], None, d["U"], w, d["y"], pb["vol"], pb["cb"], pb["step"])
    _, _, _, g2 = P.cost_grad_f0(d["f0"], None, d["U"], w, d["y"], pb["vol"], pb["cb"], pb["step"])
    assert torch.equal(g1, g2)                                  # fixed-point scatter: same bits
    Jo, go, abo = O.cost_grad_f0(pb["f0"], None, pb["U"], w, pb["y"], pb["vol"], pb["cb"], pb["step"])
    Jc, Gc, _ = P.cost_grad(d["f0"], None, d["U"], w, d["y"], pb["vol"], pb["cb"], pb["step"])
    assert J == Jc and np.array_equal(G, Gc)
    assert abs(J - Jo) <= 1e-4 * Jo
    got = g1.cpu().numpy().astype(np.float64)
    assert np.abs(got - go).max() <= 1e-4 * np.abs(go).max()
    # J only
    J3, G3, _, g3 = P.cost_grad_f0(d["f0"], None, d["U"], w, d["y"], pb["vol"], pb["cb"], pb["step"],
                                   want_grad=False, want_grad_f0=False)
    assert J3 == J and G3 is None and g3 is None


def test_grad_f0_with_mean_and_k5(P):
    pb = make_problem((61, 53, 29, 4.0, 3.5, 4.5), 5, (101, 77, 3.5, 3.5), 4.0, np.linspace(0.6, -0.4, 5),
                      with_mean=True, seeds=(21, 22, 23))
    d = to_dev(pb)
    w = 0.3 * np.ones(5)
    J, G, ab, g = P.cost_grad_f0(d["f0"], d["mean"], d["U"], w, d["y"], pb["vol"], pb["cb"], pb["step"])
    Jo, go, abo = O.cost_grad_f0(pb["f0"], pb["mean"], pb["U"], w, pb["y"], pb["vol"], pb["cb"], pb["step"])
    assert abs(J - Jo) <= 1e-4 * Jo
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-4 * np.abs(go).max()


def test_autograd_tiny_against_oracle_and_fd(P):
    from paper_1102_1712_gb300.autograd import pca_cost, problem
    pb = tiny_problem()
    d = to_dev(pb)
    prob = problem(d["U"], d["y"], pb["vol"], pb["cb"], pb["step"])
    w = torch.tensor([0.5, -0.2, 0.4], dtype=torch.float64, requires_grad=True)
    f0 = d["f0"].clone().requires_grad_(True)
    J = pca_cost(w, f0, prob)
    J.backward()
    Jo, Go, _ = O.cost_grad(pb["f0"], None, pb["U"], w.detach().numpy(), pb["y"], pb["vol"], pb["cb"], pb["step"])
    _, go, _ = O.cost_grad_f0(pb["f0"], None, pb["U"], w.detach().numpy(), pb["y"], pb["vol"], pb["cb"], pb["step"])
    assert abs(J.item() - Jo) <= 1e-4 * Jo
    assert np.linalg.norm(w.grad.numpy() - Go) <= 1e-3 * np.linalg.norm(Go)
    assert np.abs(f0.grad.cpu().numpy() - go).max() <= 1e-4 * np.abs(go).max()
    # backward of a scaled cost scales the gradients
    w2 = w.detach().clone().requires_grad_(True)
    (3.0 * pca_cost(w2, d["f0"], prob)).backward()
    np.testing.assert_allclose(w2.grad.numpy(), 3.0 * w.grad.numpy(), rtol=1e-12)
    # w on the GPU: its gradient comes back on w's device
    w3 = w.detach().cuda().requires_grad_(True)
    pca_cost(w3, d["f0"], prob).backward()
    assert w3.grad.is_cuda
    np.testing.assert_allclose(w3.grad.cpu().numpy(), w.grad.numpy(), rtol=1e-12)


@pytest.fixture(scope="module")
def diff_problem():
    """Differentiation workload: 256x256x100 CT at 2x2x2.5 mm, 512x384 view."""
    s = SEQUENCE
    w_true = S.breathing_trace(s["n_proj"], s["fps"], s["period"], s["amp"], K=3)[23]
    angle = S.gantry_angles(s["n_proj"])[23]
    return make_problem(s["vol"], 3, s["det"], angle, w_true, noise=0.01, seeds=(20, 21, 22), tumor=s["tumor"])


def test_differentiation_workload(P, diff_problem):
    from paper_1102_1712_gb300.autograd import pca_cost, problem
    pb = diff_problem
    d = to_dev(pb)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    prob = problem(d["U"], d["y"], pb["vol"], pb["cb"], pb["step"])
    w0 = 0.6 * pb["w_true"]
    w = torch.tensor(w0, dtype=torch.float64, requires_grad=True)
    f0 = d["f0"].clone().requires_grad_(True)
    J = pca_cost(w, f0, prob)
    J.backward()
    torch.cuda.synchronize()
    peak = torch.cuda.max_memory_allocated() - base
    N = f0.numel()
    # workspace + gradient buffer + the f0 copy; no warped volume kept between passes
    print(f"differentiation workload: J={J.item():.6g}, peak extra device memory {peak / 2**20:.1f} MiB "
          f"(N={N}, workspace {prob.ws.nbytes / 2**20:.1f} MiB)")
    assert peak < prob.ws.nbytes + 3 * 4 * N + (64 << 20)
    # central differences in w (h = 1e-3) on the float32 cost
    G = w.grad.numpy()
    fd = np.zeros(3)
    for k in range(3):
        e = np.zeros(3); e[k] = 1e-3
        Jp = pca_cost(torch.tensor(w0 + e), d["f0"], prob).item()
        Jm = pca_cost(torch.tensor(w0 - e), d["f0"], prob).item()
        fd[k] = (Jp - Jm) / 2e-3
    assert np.linalg.norm(fd - G) <= 2e-3 * np.linalg.norm(G), (fd, G)
    # 64 random voxels of the CT, where the gradient is non-zero
    gf = f0.grad.detach()
    nz = torch.nonzero(gf.abs() > 0.05 * gf.abs().max()).flatten().cpu().numpy()
    idx = S.rng(24).choice(nz, 64, replace=False)
    h = 1e-2                     # J* is quadratic in f0 up to the (a, b) refit
    errs = []
    for n in idx:
        fp = d["f0"].clone(); fp[n] += h
        fm = d["f0"].clone(); fm[n] -= h
        fdv = (pca_cost(torch.tensor(w0), fp, prob).item() - pca_cost(torch.tensor(w0), fm, prob).item()) / (2 * h)
        errs.append(abs(fdv - gf[n].item()))
    assert max(errs) <= 0.02 * gf.abs().max().item(), (max(errs), gf.abs().max().item())
    # the FP64 oracle gradient at full size
    Jo, Go, _ = O.cost_grad(pb["f0"], None, pb["U"], w0, pb["y"], pb["vol"], pb["cb"], pb["step"])
    _, go, _ = O.cost_grad_f0(pb["f0"], None, pb["U"], w0, pb["y"], pb["vol"], pb["cb"], pb["step"])
    assert abs(J.item() - Jo) <= 1e-4 * Jo
    assert np.linalg.norm(G - Go) <= 1e-3 * np.linalg.norm(Go)
    assert np.abs(gf.cpu().numpy() - go).max() <= 1e-4 * np.abs(go).max()
