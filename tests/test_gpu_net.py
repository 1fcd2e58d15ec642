"""The learned preconditioner's network on the tensor cores (feast_nh_net_*)
against the oracle's FP64 reference (oracle/net.py) with the same bfloat16
rounding points: forward output and every parameter gradient."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from oracle import net as ON  # noqa: E402
from paper_1506_04463_gb300 import feast_nh as F  # noqa: E402

C = F.NET_CH


def _case(L=4, N=12, nimg=3, seed=0):
    rng = np.random.default_rng(seed)
    Ws = [rng.standard_normal((3, 3, C, C)) * np.sqrt(2.0 / (9 * C)) for _ in range(L)]
    bs = [rng.standard_normal(C) * 0.05 for _ in range(L)]
    x = np.zeros((nimg, N, N, C))
    x[..., :4] = rng.standard_normal((nimg, N, N, 4))
    t = rng.standard_normal((nimg, N, N, 2))
    flat = np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in zip(Ws, bs)])
    return Ws, bs, x, t, flat


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("N,nimg", [(12, 3), (16, 8), (7, 5)])
def test_forward_matches_oracle(N, nimg):
    Ws, bs, x, t, flat = _case(N=N, nimg=nimg)
    net = F.Net(len(Ws), N, nimg)
    net.set_params(flat)
    out = net.forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    ref_q, _ = ON.forward(x, Ws, bs, quant=True)
    ref, _ = ON.forward(x, Ws, bs)
    assert _rel(out, ref_q) < 5e-3
    assert _rel(out, ref) < 3e-2
    net.close()


def test_gradients_match_oracle():
    Ws, bs, x, t, flat = _case()
    net = F.Net(len(Ws), 12, 3)
    net.set_params(flat)
    loss, g = net.train_step(torch.from_numpy(x.astype(np.float32)).cuda(),
                             torch.from_numpy(t.astype(np.float32)).cuda(), 0.0, want_grad=True)
    g = g.cpu().numpy().astype(np.float64)
    out, cache = ON.forward(x, Ws, bs, quant=True)
    dWs, dbs, _ = ON.backward(out, t, cache, Ws, quant=True)
    assert abs(loss - ON.loss(out, t)) < 1e-3 * ON.loss(out, t)
    P = 9 * C * C + C
    for l in range(len(Ws)):
        gl = g[l * P:(l + 1) * P]
        assert _rel(gl[:9 * C * C], dWs[l].reshape(-1)) < 2e-2, l
        assert _rel(gl[9 * C * C:], dbs[l]) < 2e-2, l
    # parameters untouched with lr = 0, and a step with lr > 0 lowers the loss
    assert np.array_equal(net.get_params(), flat.astype(np.float32))
    xs, ts = torch.from_numpy(x.astype(np.float32)).cuda(), torch.from_numpy(t.astype(np.float32)).cuda()
    l0 = net.train_step(xs, ts, 1e-3)[0]
    for _ in range(20):
        l1 = net.train_step(xs, ts, 1e-3)[0]
    assert l1 < l0
    net.close()
