"""GPU parity of the fused Adam / VectorAdam step (ds_adam_step) against the
FP64 oracle (oracle/optim.py) over 25 steps of seeded gradients: parameters
and moments within 1e-5 (|ref| + lr) (FP32 arithmetic, rounding that
accumulates over the steps)."""
import numpy as np
import pytest

from oracle import optim as OP

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return "cuda"


@pytest.mark.parametrize("n,dim,offset", [(4096, 1, 0), (1001, 1, 0), (4096, 1, 1), (3 * 777, 3, 0), (3 * 64, 3, 1),
                                          (2 * 50, 2, 0)])
def test_adam_step_matches_the_oracle(dev, n, dim, offset):
    import torch
    from paper_2603_27151_gb300 import native as N
    rng = np.random.default_rng(n + dim + offset)
    x0 = rng.normal(size=n)
    # an offset view makes the buffers 4-byte but not 16-byte aligned (the per-vector path)
    buf = torch.zeros(4 * (n + 4), device=dev)
    x, g, m = (buf[k * (n + 4) + offset: k * (n + 4) + offset + n] for k in range(3))
    v = torch.zeros(n // dim + 4, device=dev)[offset: offset + n // dim]
    x.copy_(torch.from_numpy(x0.astype(np.float32)))
    xr, mr, vr = x0.astype(np.float32).astype(np.float64), np.zeros(n), np.zeros(n // dim)
    for t in range(1, 26):
        lr = OP.annealed_lr(0.05, t - 1, 25)
        gr = rng.normal(size=n) * (10.0 ** rng.uniform(-3, 1))
        g.copy_(torch.from_numpy(gr.astype(np.float32)))
        N.adam_step(x, g, m, v, lr, t, dim=dim)
        # the oracle takes the hyperparameters the kernel receives (float32 values)
        xr, mr, vr = OP.adam_step(xr, gr.astype(np.float32).astype(np.float64), mr, vr, float(np.float32(lr)), t,
                                  dim=dim, b1=float(np.float32(0.9)), b2=float(np.float32(0.999)),
                                  eps=float(np.float32(1e-8)))
    torch.cuda.synchronize()
    for got, ref in ((x, xr), (m, mr), (v, vr)):
        err = np.abs(got.cpu().numpy() - ref)
        assert np.all(err <= 1e-5 * (np.abs(ref) + 0.05)), float(err.max())


def test_adam_step_rejects_bad_arguments(dev):
    import torch
    from paper_2603_27151_gb300 import native as N
    x = torch.zeros(10, device=dev)
    # shapes are checked by the binding before the raw pointers go down
    for kw in (dict(dim=3), dict(dim=5)):
        args = dict(lr=0.1, step=1, dim=1)
        args.update(kw)
        with pytest.raises(ValueError):
            N.adam_step(x, x, x, x, **args)
    with pytest.raises(ValueError):
        N.adam_step(x, torch.zeros(9, device=dev), x, x, lr=0.1, step=1)
    # hyperparameters by the library
    for kw in (dict(step=0), dict(beta1=1.0)):
        args = dict(lr=0.1, step=1, dim=1)
        args.update(kw)
        with pytest.raises(N.DsError):
            N.adam_step(x, x, x, x, **args)
