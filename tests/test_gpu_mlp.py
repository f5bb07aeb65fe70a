"""GPU: the MLP cost model's own forward, backward, Adam and argmin kernels
against the FP64 oracle (gradients <= 1e-4 relative to the gradient's scale,
one Adam step <= 1e-5)."""
import numpy as np
import pytest

from gpu_util import dev, tri

pytestmark = pytest.mark.gpu


def _setup(F=14, H1=64, H2=64, B=500, seed=0):
    rng = np.random.default_rng(seed)
    import oracle
    theta = (rng.normal(size=oracle.mlp_nparams(F, H1, H2)) * 0.2).astype(np.float32)
    X = rng.normal(size=(B, F)).astype(np.float32)
    y = rng.normal(size=B).astype(np.float32)
    return theta, X, y


def test_mlp_forward_and_grad(orc):
    import torch
    t = tri()
    F, H1, H2, B = 14, 64, 64, 500
    theta, X, y = _setup(F, H1, H2, B)
    D = dev()
    th, Xd, yd = (torch.from_numpy(a).to(D) for a in (theta, X, y))
    ws = torch.empty(t.tri_mlp_workspace_size(B, H1, H2) // 4, dtype=torch.float32, device=D)
    pred = torch.empty(B, device=D)
    t.tri_mlp_forward(th, Xd, pred, H1, H2, ws)
    loss = torch.empty(1, device=D)
    grad = torch.empty_like(th)
    t.tri_mlp_grad(th, Xd, yd, loss, grad, H1, H2, ws)
    torch.cuda.synchronize()
    ref_pred = orc.mlp_forward(theta.astype(np.float64), X, H1, H2)
    np.testing.assert_allclose(pred.cpu().numpy(), ref_pred, rtol=1e-4, atol=1e-5)
    ref_loss, ref_g = orc.mlp_grad(theta.astype(np.float64), X, y, H1, H2)
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-5)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - ref_g)) <= 1e-4 * np.max(np.abs(ref_g))


def test_mlp_adam_step(orc):
    import torch
    t = tri()
    rng = np.random.default_rng(3)
    n = 5185
    th = rng.normal(size=n).astype(np.float32)
    g = rng.normal(size=n).astype(np.float32)
    m = (rng.normal(size=n) * 0.1).astype(np.float32)
    v = np.abs(rng.normal(size=n) * 0.01).astype(np.float32)
    D = dev()
    td, gd, md, vd = (torch.from_numpy(a.copy()).to(D) for a in (th, g, m, v))
    t.tri_mlp_adam(td, gd, md, vd, 7, 1e-3)
    torch.cuda.synchronize()
    # the kernel receives the hyper-parameters as FP32; the oracle gets the same values
    b1, b2, lr = (float(np.float32(v_)) for v_ in (0.9, 0.999, 1e-3))
    rt, rm, rv = orc.adam_step(th, g, m, v, 7, lr, beta1=b1, beta2=b2)
    np.testing.assert_allclose(td.cpu().numpy(), rt, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(md.cpu().numpy(), rm, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(vd.cpu().numpy(), rv, rtol=1e-5, atol=1e-9)


def test_mlp_argmin(orc):
    import torch
    t = tri()
    theta, X, _ = _setup(B=77, seed=4)
    D = dev()
    ws = torch.empty(t.tri_mlp_workspace_size(77, 64, 64) // 4, dtype=torch.float32, device=D)
    best = torch.zeros(1, dtype=torch.int32, device=D)
    t.tri_mlp_argmin(torch.from_numpy(theta).to(D), torch.from_numpy(X).to(D), best, 64, 64, ws)
    torch.cuda.synchronize()
    ref = orc.mlp_forward(theta.astype(np.float64), X)
    k = int(best.item())
    assert ref[k] <= np.min(ref) + 1e-4 * max(1.0, abs(np.min(ref)))
