"""Training the GNN on the GPU (Sec. 3.3 / Sec. 4.1): the AdamW step of the
library against the update rule written out in numpy, and a few steps of
the training loop (forward, SAI loss gradient, reverse pass, AdamW) lowering
the SAI loss."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def adamw_ref(theta, m, v, g, step, lr, b1, b2, eps, wd, clip):
    """Decoupled weight decay Adam (Loshchilov & Hutter), float64."""
    n = np.linalg.norm(g)
    if clip > 0 and n > clip:
        g = g * (clip / n)
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta), m, v, n


@pytest.mark.parametrize("clip", [0.0, 0.5])
def test_adamw_step_matches_update_rule(spai_lib, clip):
    spai = spai_lib
    rng = np.random.default_rng(3)
    count = 1000
    th = rng.standard_normal(count)
    master = torch.tensor(th, device="cuda")
    m = torch.zeros(count, dtype=torch.float64, device="cuda")
    v = torch.zeros_like(m)
    blob = torch.zeros(count, dtype=torch.float32, device="cuda")
    mr, vr = np.zeros(count), np.zeros(count)
    for step in range(1, 4):
        g = rng.standard_normal(count) * (0.1 * step)
        gn = spai.adamw_step(master, m, v, torch.tensor(g, device="cuda"), blob, step, lr=1e-2, weight_decay=0.05,
                             max_grad_norm=clip)
        th, mr, vr, n = adamw_ref(th, mr, vr, g, step, 1e-2, 0.9, 0.999, 1e-8, 0.05, clip)
        assert gn == pytest.approx(n, rel=1e-13)
        assert np.allclose(master.cpu().numpy(), th, rtol=1e-12, atol=1e-14)
        assert np.allclose(m.cpu().numpy(), mr, rtol=1e-12, atol=1e-15)
        assert np.array_equal(blob.cpu().numpy(), master.cpu().numpy().astype(np.float32))


def test_adamw_rejects_bad_parameters(spai_lib):
    spai = spai_lib
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    blob = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(spai.SpaiError):
        spai.adamw_step(t, t.clone(), t.clone(), t.clone(), blob, 1, lr=1e-3, beta1=1.0)
    with pytest.raises(spai.SpaiError):
        spai.adamw_step(t, t.clone(), t.clone(), t.clone(), blob, 0, lr=1e-3)


def test_training_steps_lower_the_sai_loss(spai_lib):
    # the training loop of paper_2510_27517_gb300.train on two small diffusion
    # matrices: 30 AdamW steps on the SAI loss with fresh probes each step
    spai = spai_lib
    from paper_2510_27517_gb300 import train
    items = [train.to_device(it) for it in train.dataset(2, [6, 8], W.BASE_SEED + 900)]
    blob = torch.tensor(W.gnn_random_weights(4, 4, seed=W.BASE_SEED + 100), device="cuda")
    master = blob.to(torch.float64).clone()
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    before = train.mean_loss(items, blob, 1e-4, 8, 11)
    rng = np.random.default_rng(5)
    for step in range(1, 31):
        g = torch.zeros_like(master)
        for it in items:
            _, dW = train.loss_and_grad(it, blob, train.probes(it["A"].n, 4, int(rng.integers(1 << 62))), 1e-4)
            g += dW
        spai.adamw_step(master, m, v, g / len(items), blob, step, lr=3e-3, max_grad_norm=1.0)
    after = train.mean_loss(items, blob, 1e-4, 8, 11)
    assert np.isfinite(after) and after < 0.5 * before, (before, after)
