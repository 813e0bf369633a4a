"""The surrogate network's CUDA kernels (forward, backward, ridge fit, Adam, training)
through the C ABI against the FP64 oracle (oracle/surrogate.py)."""
import numpy as np
import pytest

from oracle import surrogate as S
from paper_2011_01400_gb300.synth import surrogate_init

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_01400_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def blocks(dims, v):
    out, o = {}, 0
    for name, shape in S.layout(*dims):
        n = int(np.prod(shape))
        out[name] = v[o:o + n]
        o += n
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("dims,n", [((12, 256, 48), 300), ((5, 40, 7), 33)])
def test_forward_and_gradient_match_oracle(dims, n):
    from paper_2011_01400_gb300 import gw
    rng = np.random.default_rng(1)
    th = (rng.standard_normal(S.n_params(*dims)) * 0.3).astype(np.float32)
    th[-1] = 0.7
    x = rng.standard_normal((n, dims[0])).astype(np.float32)
    y = rng.standard_normal((n, dims[2])).astype(np.float32)
    m = gw.gw_surrogate_create(*dims, dev(th))
    try:
        f = torch.empty((n, dims[2]), device="cuda")
        g = torch.empty((n, dims[2]), device="cuda")
        gw.gw_surrogate_forward(m, dev(x), f, g)
        grad = torch.empty(len(th), device="cuda")
        loss = gw.gw_surrogate_loss_grad(m, dev(x), dev(y), grad)
        f_ref, g_ref, _ = S.forward(th.astype(np.float64), dims, x.astype(np.float64), parts=True)
        l_ref, gr_ref = S.loss_grad(th.astype(np.float64), dims, x.astype(np.float64), y.astype(np.float64))
        assert rel(f.cpu().numpy(), f_ref) < 2e-6
        assert rel(g.cpu().numpy(), g_ref) < 2e-6
        assert abs(loss - l_ref) <= 2e-6 * l_ref
        gb, rb = blocks(dims, grad.cpu().numpy().astype(np.float64)), blocks(dims, gr_ref)
        for name in gb:
            if name == "s":
                assert gb[name][0] == 0.0
                continue
            e = rel(gb[name], rb[name])
            print(f"{dims} grad {name}: rel error {e:.2e}")
            assert e < 2e-5, name
    finally:
        gw.gw_surrogate_destroy(m)


def test_fit_linear_matches_oracle():
    from paper_2011_01400_gb300 import gw
    dims = (12, 32, 48)
    rng = np.random.default_rng(2)
    n = 20000
    x = rng.standard_normal((n, 12)).astype(np.float32)
    L0 = rng.standard_normal((48, 12))
    y = (x @ L0.T + 1e-3 * np.sin(3 * x[:, :1])).astype(np.float32)
    m = gw.gw_surrogate_create(*dims, dev(surrogate_init(*dims, seed=3)))
    try:
        rms = gw.gw_surrogate_fit_linear(m, dev(x), dev(y), 1e-8)
        th = torch.empty(S.n_params(*dims), device="cuda")
        gw.gw_surrogate_get_params(m, th)
        p = blocks(dims, th.cpu().numpy().astype(np.float64))
    finally:
        gw.gw_surrogate_destroy(m)
    L_ref, rms_ref = S.fit_linear(x.astype(np.float64), y.astype(np.float64), 1e-8)
    assert rel(p["L"].reshape(48, 12), L_ref) < 1e-6
    assert abs(rms - rms_ref) <= 1e-4 * rms_ref
    assert abs(p["s"][0] - rms_ref) <= 1e-4 * rms_ref


def test_adam_first_step_matches_oracle():
    """One full-batch step from zero moments: Adam moves every trained weight by lr * sign(g)
    of the residual-form gradient (the f-loss gradient / s^2); L and s do not move."""
    from paper_2011_01400_gb300 import gw
    dims = (6, 32, 10)
    rng = np.random.default_rng(4)
    th = (rng.standard_normal(S.n_params(*dims)) * 0.3).astype(np.float32)
    th[-1] = 0.5
    n = 128
    x = rng.standard_normal((n, 6)).astype(np.float32)
    y = rng.standard_normal((n, 10)).astype(np.float32)
    m = gw.gw_surrogate_create(*dims, dev(th))
    try:
        gw.gw_surrogate_train(m, dev(x), dev(y), 1, n, 1e-3, 7)
        out = torch.empty(len(th), device="cuda")
        gw.gw_surrogate_get_params(m, out)
        got = out.cpu().numpy().astype(np.float64)
    finally:
        gw.gw_surrogate_destroy(m)
    _, g = S.loss_grad(th.astype(np.float64), dims, x.astype(np.float64), y.astype(np.float64))
    g = g / th[-1] ** 2
    want, _, _ = S.adam_step(th.astype(np.float64), g, 0.0, 0.0, 1, 1e-3)
    o_L = S.n_params(*dims) - dims[0] * dims[2] - 1
    assert np.array_equal(got[o_L:], th[o_L:].astype(np.float64))       # L and s unchanged
    d = np.abs(got[:o_L] - want[:o_L])
    tiny = np.abs(g[:o_L]) < 1e-4 * np.abs(g[:o_L]).max()                # sign of a ~0 gradient may differ
    assert (d[~tiny] < 2e-7 + 1e-6 * np.abs(th[:o_L][~tiny])).all()


def test_training_reduces_the_residual():
    from paper_2011_01400_gb300 import gw
    dims = (8, 64, 16)
    rng = np.random.default_rng(5)
    n = 8192
    x = rng.uniform(-1, 1, (n, 8)).astype(np.float32)
    A = rng.standard_normal((16, 8))
    y = (x @ A.T + 0.05 * np.tanh(2 * x[:, :1] * x[:, 1:2]) * np.ones((1, 16))).astype(np.float32)
    m = gw.gw_surrogate_create(*dims, dev(surrogate_init(*dims, seed=6)))
    try:
        rms = gw.gw_surrogate_fit_linear(m, dev(x), dev(y), 1e-10)
        hist = gw.gw_surrogate_train(m, dev(x), dev(y), 40, 256, 2e-3, 11)
        f = torch.empty((n, 16), device="cuda")
        gw.gw_surrogate_forward(m, dev(x), f)
        res = np.sqrt(np.mean((f.cpu().numpy() - y) ** 2))
    finally:
        gw.gw_surrogate_destroy(m)
    print(f"linear rms {rms:.3e} -> trained rms {res:.3e}; loss {hist[0]:.3e} -> {hist[-1]:.3e}")
    assert hist[-1] < hist[0]
    assert res < 0.2 * rms
