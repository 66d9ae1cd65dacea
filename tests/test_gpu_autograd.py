"""Differentiable attribute codec: RAHT forward / inverse as autograd
functions (each one's backward is the other kernel, Sec. 3.2: RAHT is
orthonormal) and the codec layer A_hat = T^T(step * q(T A)) with a
straight-through quantiser.

FP64 instantiation of the transform kernels:
  * equals the oracle's recursive FP64 RAHT;
  * torch.autograd.gradcheck against finite differences;
  * the codec layer's output and gradient equal a dense-matrix torch
    reference, T built column by column by the oracle (2,000 points, J = 8).
FP32 at 500,000 points (J = 16): the per-channel reconstruction error obeys
the orthonormal quantisation bound and the gradient is the identity.
"""
import numpy as np
import pytest

from paper_2606_05650_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05650_gb300 import gsnfs
    return gsnfs


def _frame(orc, seed, n, J, C):
    pos, _ = syn.static_gs_frame(seed, n)
    codes, _, _ = orc.voxelize(pos, np.zeros((n, 1), np.float32), J)[:3]
    A = np.random.default_rng(seed).normal(0.0, 1.0, (codes.shape[0], C))
    return codes, A


def _plan(G, codes, J, C):
    return G.RahtPlan(torch.from_numpy(codes.astype(np.int64)).cuda(), J, C)


def test_fp64_kernels_equal_the_oracle(G, orc):
    codes, A = _frame(orc, 1, 2000, 8, 5)
    plan = _plan(G, codes, 8, 5)
    Y = plan.forward(torch.from_numpy(A).cuda()).cpu().numpy()
    Yo = orc.raht_forward(codes, A, 8)
    assert np.abs(Y - Yo).max() <= 1e-13 * (1 + np.abs(Yo).max())
    back = plan.inverse(torch.from_numpy(Yo).cuda()).cpu().numpy()
    assert np.abs(back - orc.raht_inverse(codes, Yo, 8)).max() <= 1e-13 * (1 + np.abs(A).max())
    assert np.abs(back - A).max() <= 1e-12


def test_fp64_kernels_at_depth16_several_passes(G, orc):
    # enough voxels for every grid-wide pass and the one-CTA finisher
    pos, _ = syn.DynamicScene(4).frame(1, n=60_000)
    codes = orc.voxelize(pos, np.zeros((pos.shape[0], 1), np.float32), 16)[0]
    A = np.random.default_rng(4).normal(0.0, 1.0, (codes.shape[0], 6))
    plan = _plan(G, codes, 16, 6)
    Y = plan.forward(torch.from_numpy(A).cuda()).cpu().numpy()
    Yo = orc.raht_forward(codes, A, 16)
    assert np.abs(Y - Yo).max() <= 1e-12 * (1 + np.abs(Yo).max())


@pytest.mark.parametrize("fn", ["forward", "inverse"])
def test_gradcheck_transforms(G, orc, fn):
    codes, A = _frame(orc, 2, 2000, 8, 2)
    plan = _plan(G, codes, 8, 2)
    x = torch.from_numpy(A).cuda().requires_grad_(True)
    f = G.RahtForwardFn if fn == "forward" else G.RahtInverseFn
    assert torch.autograd.gradcheck(lambda t: f.apply(t, plan), (x,), eps=1e-6, atol=1e-9, rtol=1e-7)


def test_gradcheck_fast_mode_56_channels(G, orc):
    codes, A = _frame(orc, 3, 2000, 8, 56)
    plan = _plan(G, codes, 8, 56)
    x = torch.from_numpy(A).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: G.RahtForwardFn.apply(t, plan), (x,), eps=1e-6, atol=1e-9,
                                    rtol=1e-7, fast_mode=True)


def test_codec_layer_equals_dense_matrix_reference(G, orc):
    J, C = 8, 56
    codes, A = _frame(orc, 5, 2000, J, C)
    nv = codes.shape[0]
    T = orc.raht_forward(codes, np.eye(nv), J)  # column k = T e_k
    assert np.abs(T.T @ T - np.eye(nv)).max() < 1e-12
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    step = torch.from_numpy(qp.steps[qp.groups])
    # dense torch reference on the CPU, straight-through quantiser
    Tt = torch.from_numpy(T)
    a_ref = torch.from_numpy(A).requires_grad_(True)
    y = Tt @ a_ref
    t = y.detach().abs() / step + qp.tau
    assert (torch.minimum(t - t.floor(), t.floor() + 1 - t) > 1e-9).all()  # no coefficient at a rounding boundary
    yq = torch.sign(y.detach()) * torch.floor(t) * step
    rec_ref = Tt.T @ (y + (yq - y).detach())
    loss_ref = ((rec_ref - a_ref.detach()) ** 2).mean()
    loss_ref.backward()
    # the kernels
    plan = _plan(G, codes, J, C)
    a = torch.from_numpy(A).cuda().requires_grad_(True)
    rec = G.AttrCodecFn.apply(a, plan, qp)
    loss = ((rec - a.detach()) ** 2).mean()
    loss.backward()
    assert torch.allclose(rec.detach().cpu(), rec_ref.detach(), rtol=0, atol=1e-10)
    assert torch.allclose(a.grad.cpu(), a_ref.grad, rtol=0, atol=1e-14)
    assert abs(loss.item() - loss_ref.item()) <= 1e-12 * loss_ref.item()


def test_fp32_codec_layer_at_500k(G, orc):
    pos, attr = syn.DynamicScene(7).frame(2, n=500_000)
    codes, merged, _ = orc.voxelize(pos, attr, 16)[:3]
    nv, C = merged.shape
    plan = _plan(G, codes, 16, C)
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    a = torch.from_numpy(merged.astype(np.float32)).cuda().requires_grad_(True)
    rec = G.AttrCodecFn.apply(a, plan, qp)
    # orthonormal T: per channel ||A_hat - A||^2 = ||y_hat - y||^2 <= nv (step/2)^2 (tau = 0.5)
    err = ((rec.detach() - a.detach()).double() ** 2).sum(0).cpu().numpy()
    step = qp.steps[qp.groups]
    assert (err <= nv * (step / 2) ** 2 * (1 + 1e-3)).all()
    g = torch.randn_like(a)
    rec.backward(g)
    # gradient = T^T T g = g up to FP32 rounding of 2 x 48 butterfly levels
    rms = g.pow(2).mean().sqrt().item()
    assert (a.grad - g).abs().max().item() <= 1e-4 * rms
