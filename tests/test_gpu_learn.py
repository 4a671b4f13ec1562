"""The proposal network's GPU kernels against the FP64 oracle: forward, gradients (the
oracle's own gradients are pinned by finite differences), one Adam step, and training
that lowers the loss on data the simulator generated."""

import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _data(nf, hidden, batch, seed):
    from paper_2012_02430_gb300 import learn
    from paper_2012_02430_gb300.inputs import SplitMix64
    p = learn.init_params(nf, hidden, seed)
    rng = SplitMix64(seed + 99)
    x = np.array([[2 * rng.uniform() - 1 for _ in range(nf)] for _ in range(batch)], dtype=np.float32)
    t = np.array([rng.uniform() for _ in range(batch)], dtype=np.float32)
    return p, x, t


@pytest.mark.parametrize("nf,hidden,batch", [(16, 64, 257), (5, 7, 3), (16, 32, 1024)])
def test_gpu_forward_and_gradients(qt, nf, hidden, batch):
    from paper_2012_02430_gb300 import learn
    p, x, t = _data(nf, hidden, batch, 11)
    net = learn.GPUMLP(nf, hidden, batch)
    net.set_params(p)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = net.forward(xd).cpu().numpy()
    g, loss = net.gradients(xd, td)
    g = g.cpu().numpy()
    yr, _ = mlp.forward(p.astype(np.float64), x.astype(np.float64), nf, hidden)
    gr = mlp.gradients(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), nf, hidden)
    lr = mlp.loss(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), nf, hidden)
    assert np.max(np.abs(y - yr)) <= 1e-5 * max(1.0, np.max(np.abs(yr)))
    assert np.max(np.abs(g - gr)) <= 1e-4 * max(1e-3, np.max(np.abs(gr)))
    assert abs(loss.item() - lr) <= 1e-5 * max(1.0, lr)


def test_gpu_adam_step_matches_oracle(qt):
    from paper_2012_02430_gb300 import learn
    nf, hidden, batch = 16, 32, 200
    p, x, t = _data(nf, hidden, batch, 5)
    net = learn.GPUMLP(nf, hidden, batch)
    net.set_params(p)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    pr = p.astype(np.float64)
    m = np.zeros_like(pr)
    v = np.zeros_like(pr)
    for step in range(1, 4):
        net.train_step(xd, td, 1e-3, loss)
        g = mlp.gradients(pr, x.astype(np.float64), t.astype(np.float64), nf, hidden)
        pr, m, v = mlp.adam_step(pr, g, m, v, step, 1e-3)
    got = net.get_params()
    assert np.max(np.abs(got - pr)) <= 2e-5


def test_gpu_training_lowers_loss_on_simulator_data(qt):
    from paper_2012_02430_gb300 import learn
    X, Y = learn.make_dataset([(50, 2, 7001), (70, 1, 7002), (60, 2, 7003)])
    assert X.shape[0] > 300
    params, info = learn.train(X, Y, hidden=32, steps=400, batch=256, lr=3e-3, seed=3)
    first = info["log"][0][1]
    assert info["train_mse"] < 0.5 * first
    assert np.all(np.isfinite(params))
