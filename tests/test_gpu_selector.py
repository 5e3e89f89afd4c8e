"""The learned selector's GPU kernels against the oracle: forward logits bit
for bit (fixed-order fmaf chain), loss and gradient against the FP64
backward, the Adam step bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_02494_gb300 as sp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1511_02494_gb300.build import build
    build()
    assert torch.cuda.is_available()


def _params(h1, h2, k, seed):
    g = np.random.default_rng(seed)
    return {"mean": g.standard_normal(16).astype(np.float32),
            "istd": (0.5 + g.random(16)).astype(np.float32),
            "W1": (g.standard_normal((h1, 16)) * 0.3).astype(np.float32),
            "b1": (g.standard_normal(h1) * 0.1).astype(np.float32),
            "W2": (g.standard_normal((h2, h1)) * 0.15).astype(np.float32),
            "b2": (g.standard_normal(h2) * 0.1).astype(np.float32),
            "W3": (g.standard_normal((k, h2)) * 0.15).astype(np.float32),
            "b3": (g.standard_normal(k) * 0.1).astype(np.float32)}


def _packed(P):
    return torch.from_numpy(np.concatenate(
        [P[n].reshape(-1) for n in ("W1", "b1", "W2", "b2", "W3", "b3")])).cuda()


@pytest.mark.parametrize("shape", [(64, 64, 7), (16, 32, 4), (128, 8, 2)])
def test_forward_bit_exact(shape):
    h1, h2, k = shape
    P = _params(h1, h2, k, 0)
    v = np.random.default_rng(1).standard_normal((301, 16)).astype(np.float32) * 2
    out = torch.empty((301, k), dtype=torch.float32, device="cuda")
    sp.spmv_mlp_forward(_packed(P), torch.from_numpy(P["mean"]).cuda(),
                        torch.from_numpy(P["istd"]).cuda(), h1, h2, k,
                        torch.from_numpy(v).cuda(), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.mlp_forward_f32(P, v))


@pytest.mark.parametrize("n", [1, 31, 32, 200, 1600])
def test_loss_and_gradient_against_fp64_oracle(n):
    h1, h2, k = 64, 64, 7
    P = _params(h1, h2, k, n)
    g = np.random.default_rng(n)
    z = g.standard_normal((n, 16)).astype(np.float32)
    lab = g.integers(0, k, n).astype(np.int32)
    grad = torch.empty(_packed(P).numel(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    sp.spmv_mlp_loss_grad(_packed(P), h1, h2, k, torch.from_numpy(z).cuda(),
                          torch.from_numpy(lab).cuda(), grad, loss)
    torch.cuda.synchronize()
    ref_loss, G = oracle.mlp_loss_grad_f64({n_: P[n_].astype(np.float64) for n_ in P}, z, lab)
    ref = np.concatenate([G[n_].reshape(-1) for n_ in ("W1", "b1", "W2", "b2", "W3", "b3")])
    got = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss))
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
    # deterministic: a second evaluation is bit-identical
    grad2 = torch.empty_like(grad)
    sp.spmv_mlp_loss_grad(_packed(P), h1, h2, k, torch.from_numpy(z).cuda(),
                          torch.from_numpy(lab).cuda(), grad2, loss)
    assert torch.equal(grad, grad2)


def test_soft_target_loss_grad_matches_oracle():
    P = _params(64, 64, 7, seed=3)
    g = np.random.default_rng(12)
    n, k = 203, 7
    z = g.standard_normal((n, 16)).astype(np.float32)
    t = np.exp(g.standard_normal((n, k)))
    q = (t.min(1, keepdims=True) / t) ** 8
    q = (q / q.sum(1, keepdims=True)).astype(np.float32)
    grad = torch.empty(_packed(P).numel(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    sp.spmv_mlp_loss_grad_soft(_packed(P), 64, 64, k, torch.from_numpy(z).cuda(),
                               torch.from_numpy(q).cuda(), grad, loss)
    torch.cuda.synchronize()
    ref_loss, G = oracle.mlp_loss_grad_soft_f64({n_: P[n_].astype(np.float64) for n_ in P}, z, q)
    ref = np.concatenate([G[n_].reshape(-1) for n_ in ("W1", "b1", "W2", "b2", "W3", "b3")])
    got = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss))
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_adam_bit_exact():
    g = np.random.default_rng(5)
    n = 5703
    p = g.standard_normal(n).astype(np.float32)
    gr = g.standard_normal(n).astype(np.float32) * 0.01
    m = g.standard_normal(n).astype(np.float32) * 0.001
    v = g.random(n).astype(np.float32) * 1e-4
    dp, dg, dm, dv = (torch.from_numpy(a.copy()).cuda() for a in (p, gr, m, v))
    step, lr, b1, b2, eps, wd = 7, 3e-3, 0.9, 0.999, 1e-8, 1e-4
    sp.spmv_mlp_adam(dp, dg, dm, dv, step, lr, b1, b2, eps, wd)
    torch.cuda.synchronize()
    c1 = np.float32(1) - np.float32(b1) ** np.float32(step)
    c2 = np.float32(1) - np.float32(b2) ** np.float32(step)
    rp, rm, rv = oracle.adam_f32(p, gr, m, v, lr, b1, b2, eps, wd, float(c1), float(c2))
    assert np.array_equal(dm.cpu().numpy(), rm) and np.array_equal(dv.cpu().numpy(), rv)
    assert np.max(np.abs(dp.cpu().numpy() - rp)) <= 1e-7 * np.max(np.abs(rp))
