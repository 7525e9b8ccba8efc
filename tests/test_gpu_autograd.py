"""The autograd wrapper of the hand-written backward (row a9): log|psi| from
nqs_amplitude, gradients from nqs_grad_log_psi_vjp through torch.autograd,
against the oracle's per-sample gradients and central differences of the
forward itself."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_19276_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_19276_gb300 import nqs  # noqa: E402


@pytest.mark.parametrize("graph", [False, True])
def test_autograd_energy_gradient_matches_oracle(graph):
    sys_ = W.tiny_system(K=6, na=3, nb=3, D=4, n_hidden=5, seed=41, graph=graph)
    P = O.Problem(sys_)
    ctx = nqs.Context(0)
    try:
        ctx.set_system(sys_)
        T = torch.tensor(sys_.tensors, device="cuda", requires_grad=True)
        Wt = torch.tensor(sys_.rbm_W, device="cuda", requires_grad=True)
        bt = torch.tensor(sys_.rbm_b, device="cuda", requires_grad=True)
        s = torch.from_numpy(sys_.samples.view(np.int64)).cuda()
        la, sg = nqs.log_psi(ctx, s, T, Wt, bt, sys_.pred_ptr, sys_.pred_idx)
        e, _ = ctx.local_energy(sys_.samples, sys_.counts, 0.0, 0, 0)
        c = sys_.counts
        u = 2 * c * (e - np.sum(c * e) / np.sum(c)) / np.sum(c)      # Eq. egrad weights
        (torch.from_numpy(u).cuda() * la).sum().backward()
        rT = np.zeros_like(sys_.tensors); rW = np.zeros_like(sys_.rbm_W); rb = np.zeros_like(sys_.rbm_b)
        for ui, d in zip(u, sys_.samples):
            t, w, bb = O.grad_log_psi(P, d)
            rT += ui * t; rW += ui * w; rb += ui * bb
            l_ref, s_ref, _ = O.log_psi(P, d)
        for got, ref in ((T.grad, rT), (Wt.grad, rW), (bt.grad, rb)):
            g = got.cpu().numpy()
            assert np.max(np.abs(g - ref)) < 1e-10 * max(1.0, np.max(np.abs(ref)))
        la_ref = np.array([O.log_psi(P, d)[0] for d in sys_.samples])
        assert np.max(np.abs(la.detach().cpu().numpy() - la_ref)) < 1e-12 * np.max(np.abs(la_ref))
    finally:
        ctx.close()


def test_autograd_central_differences_of_the_forward():
    sys_ = W.tiny_system(K=5, na=2, nb=3, D=3, n_hidden=4, seed=43)
    ctx = nqs.Context(0)
    try:
        ctx.set_system(sys_)
        s = torch.from_numpy(sys_.samples[:7].view(np.int64)).cuda()
        T = torch.tensor(sys_.tensors, device="cuda", requires_grad=True)
        Wt = torch.tensor(sys_.rbm_W, device="cuda", requires_grad=True)
        bt = torch.tensor(sys_.rbm_b, device="cuda", requires_grad=True)
        v = torch.linspace(-1.0, 1.0, 7, dtype=torch.float64, device="cuda")
        la, _ = nqs.log_psi(ctx, s, T, Wt, bt)
        (v * la).sum().backward()
        h = 1e-6
        rng = np.random.default_rng(3)
        for pi, p in enumerate((T, Wt, bt)):
            flat = p.detach().clone().view(-1)
            for i in rng.choice(flat.numel(), size=min(6, flat.numel()), replace=False):
                vals = []
                for sgn in (+1, -1):
                    q = flat.clone(); q[i] += sgn * h
                    args = [x.detach() for x in (T, Wt, bt)]
                    args[pi] = q.view(p.shape)
                    l, _ = nqs.log_psi(ctx, s, *args)
                    vals.append(float((v * l).sum()))
                fd = (vals[0] - vals[1]) / (2 * h)
                g = float(p.grad.view(-1)[i])
                assert abs(fd - g) < 1e-6 * max(1.0, abs(g)), (p.shape, int(i), fd, g)
    finally:
        ctx.close()
