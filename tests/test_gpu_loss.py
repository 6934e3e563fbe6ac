"""The differentiable topological loss (tsf_loss_and_gradient) on the GPU:
against the oracle's fp64 loss and gradient, against central differences of
the GPU loss itself at pairing-stable vertices, and through torch.autograd."""
import numpy as np
import pytest

import oracle
from paper_2407_12399_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2407_12399_gb300 import build as B
    B.build()
    oracle.build()


def _field(f0, tau):
    import torch

    import paper_2407_12399_gb300 as tsf
    fld = tsf.Field(torch.from_numpy(np.ascontiguousarray(f0, np.float32)).cuda())
    fld.set_threshold(tau)
    return fld


def _moved(f0, seed, amp):
    rng = np.random.default_rng(seed)
    return (f0 + rng.uniform(-amp, amp, f0.shape)).astype(np.float32)


@pytest.mark.parametrize("name,shape,tau", [("plain_32", None, 0.1), ("mixture_40", (40, 40, 40), 0.1)])
def test_loss_and_gradient_equal_the_oracle(name, shape, tau):
    f0 = S.plain_32() if shape is None else S.gaussian_mixture(shape, n_bumps=12, seed=5)
    fld = _field(f0, tau)
    ref = oracle.Solver(f0, tau=tau)
    for f in (f0, _moved(f0, 1, 0.01), _moved(f0, 2, 0.03)):
        loss, grad = fld.loss_and_grad(f)
        rl, rg = ref.loss_grad(f)
        assert loss == pytest.approx(rl, rel=1e-12, abs=1e-300)
        # same diagram, same matching, same per-vertex addition order in fp64
        assert np.array_equal(grad, rg)
        assert np.count_nonzero(grad) > 0


def _pairing(fld):
    d = fld.diagram()
    tgt, _ = fld.assignment()
    return np.stack([d["dim"].astype(np.int64), d["v_birth"].astype(np.int64), d["v_death"].astype(np.int64),
                     tgt.astype(np.int64)])


def test_loss_gradient_matches_central_differences_96():
    """Central differences with eps = 1e-3 at 256 random vertices whose
    perturbation changes neither the pairing nor the matching (there L is
    quadratic in f(v), so the quotient is exact up to h (d - d') with d, d'
    the fp32 perturbations actually applied)."""
    import torch
    tau = 0.1
    f0 = S.mixture_96()
    f = _moved(f0, 7, 0.005)
    fld = _field(f0, tau)
    ft = torch.from_numpy(f).cuda()
    gt = torch.empty(f.shape, dtype=torch.float64, device="cuda")
    fld.loss_and_grad(ft, gt)
    g = gt.cpu().numpy().ravel()
    base = _pairing(fld)
    rng = np.random.default_rng(3)
    nz = np.nonzero(g)[0]
    cand = np.concatenate([rng.permutation(nz)[:1500], rng.choice(f.size, 100, replace=False)])
    rng.shuffle(cand)
    flat = ft.view(-1)
    checked = 0
    for v in cand:
        x = flat[v].item()
        xp, xm = np.float32(np.float32(x) + np.float32(1e-3)), np.float32(np.float32(x) - np.float32(1e-3))
        flat[v] = float(xp)
        lp, _ = fld.loss_and_grad(ft, gt)
        stable = np.array_equal(_pairing(fld), base)
        if stable:
            flat[v] = float(xm)
            lm, _ = fld.loss_and_grad(ft, gt)
            stable = np.array_equal(_pairing(fld), base)
        flat[v] = x
        if not stable:
            continue
        fd = (lp - lm) / ((float(xp) - x) + (x - float(xm)))
        assert fd == pytest.approx(g[v], abs=2e-6), int(v)
        checked += 1
        if checked == 256:
            break
    assert checked == 256
    # back at f the gradient is as before
    fld.loss_and_grad(ft, gt)
    assert np.array_equal(gt.cpu().numpy().ravel(), g)


def test_autograd_backward_is_the_library_gradient():
    import torch

    from paper_2407_12399_gb300.autograd import topological_loss
    f0 = S.plain_32()
    fld = _field(f0, 0.1)
    f = torch.from_numpy(_moved(f0, 4, 0.02)).cuda().requires_grad_(True)
    L = topological_loss(f, fld)
    L.backward()
    ref_loss, ref_grad = oracle.Solver(f0, tau=0.1).loss_grad(f.detach().cpu().numpy())
    assert L.item() == pytest.approx(ref_loss, rel=1e-12)
    assert f.grad.dtype == torch.float32
    assert np.array_equal(f.grad.cpu().numpy(), ref_grad.astype(np.float32))
    # a scaled loss scales the gradient
    f.grad = None
    (3.0 * topological_loss(f, fld)).backward()
    assert np.array_equal(f.grad.cpu().numpy(), (3.0 * ref_grad).astype(np.float32))
