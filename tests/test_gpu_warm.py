"""GPU checks of the learned warm start against the FP64 oracle.

* neighbour-shell features: bitwise equal to the oracle on an unsheared cell
  (same FP64 operations in the same order), within 1e-12 on a sheared one;
* network forward pass: BF16 tensor-core kernel vs the oracle's FP64 network
  evaluated on the same BF16-rounded weights and inputs (relative error of
  the outputs below 2e-2, the size of BF16 rounding of the activations);
* gradients of the training loss: cosine similarity above 0.999 per layer
  and loss within 1e-2 relative;
* training on data the method generates lowers the loss;
* the gated warm start leaves the AQS path unchanged (same energies, events
  and final positions as the plain affine start) and reports its FIRE
  iteration gain.
"""
import numpy as np
import pytest

from conftest import load_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return pytest.importorskip("torch")


@pytest.fixture(scope="module")
def A():
    from paper_2507_20802_gb300 import aqs
    aqs.lib()
    return aqs


def bf16_round(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def wrapped_glass():
    g = load_golden("glass_2d_n256_s0.npz")
    x, t, H = g["x"].copy(), g["types"], g["H"]
    L = np.diag(H)
    x = x - np.floor(x / L) * L
    return x, t, H


def features(A, torch, syn, x, t, H):
    s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_MIXED)
    fb = torch.zeros((len(x), A.WARM_IN), dtype=torch.bfloat16, device="cuda")
    f64 = torch.zeros((len(x), 66), dtype=torch.float64, device="cuda")
    s.warm_features(fb, f64)
    torch.cuda.synchronize()
    return s, fb, f64.cpu().numpy()


def test_features_match_oracle(A, torch, orc, syn):
    x, t, H = wrapped_glass()
    _, _, f = features(A, torch, syn, x, t, H)
    fo = orc.knn_features(x, t, H, 2, 32)
    np.testing.assert_array_equal(f, fo)
    # sheared cell: positions wrapped by the library may move by one ulp
    xs, Hs = orc.affine_shear(x, H, 0.03)
    _, _, f2 = features(A, torch, syn, xs, t, Hs)
    fo2 = orc.knn_features(xs, t, Hs, 2, 32)
    np.testing.assert_allclose(f2, fo2, rtol=0, atol=1e-12)


def test_forward_matches_oracle(A, torch, orc, syn):
    x, t, H = wrapped_glass()
    _, fb, _ = features(A, torch, syn, x, t, H)
    w = A.Warm(seed=7)
    y = torch.zeros((len(x), 2), dtype=torch.float32, device="cuda")
    w.predict(fb, y)
    torch.cuda.synchronize()
    Ws, bs = A.unpack_params(w.params())
    Wo = [bf16_round(W) for W in Ws]
    X = fb.float().cpu().numpy().astype(np.float64)
    yo = orc.mlp_forward(Wo, [b.astype(np.float64) for b in bs], X)[:, :2]
    err = np.abs(y.cpu().numpy() - yo).max() / np.abs(yo).max()
    assert err < 2e-2, err


def test_gradients_match_oracle(A, torch, orc, syn):
    x, t, H = wrapped_glass()
    _, fb, _ = features(A, torch, syn, x, t, H)
    w = A.Warm(seed=3)
    rng = np.random.default_rng(0)
    T = rng.standard_normal((len(x), 2)).astype(np.float32)
    Td = torch.tensor(T, device="cuda")
    loss, g = w.loss_grad(fb, Td)
    Ws, bs = A.unpack_params(w.params())
    Wo = [bf16_round(W) for W in Ws]
    X = fb.float().cpu().numpy().astype(np.float64)
    To = np.zeros((len(x), 16))
    To[:, :2] = T
    # the oracle loss counts all 16 padded outputs; their targets equal the
    # (zero) padded outputs, so they add nothing; rescale the 1/m of the mean
    lo, dWo, dbo = orc.mlp_loss_grad(Wo, [b.astype(np.float64) for b in bs], X, To)
    assert loss == pytest.approx(lo, rel=1e-2)
    gW, gb = A.unpack_params(g)
    for l in range(4):
        a, b = gW[l].ravel().astype(np.float64), dWo[l].ravel()
        if l == 3:
            a, b = gW[l][:2].ravel().astype(np.float64), dWo[l][:2].ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert cos > 0.999, (l, cos)
        ab, bb = gb[l][: (2 if l == 3 else None)].astype(np.float64), dbo[l][: (2 if l == 3 else None)]
        cosb = ab @ bb / (np.linalg.norm(ab) * np.linalg.norm(bb))
        assert cosb > 0.999, (l, cosb)
    # padding stays exactly zero
    assert np.all(gW[3][2:] == 0.0) and np.all(gb[3][2:] == 0.0)
    assert np.all(gW[0][:, 66:] == 0.0)


@pytest.fixture(scope="module")
def trained(A, torch, syn):
    """A network trained on 24 AQS steps of the N = 1024 oracle glass (the
    method's own data), and the data."""
    g = load_golden("glass_2d_n1024_s0.npz")
    x, t, H = g["x"], g["types"], g["H"]
    s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_MIXED)
    n_steps = 24
    F = torch.zeros((n_steps * len(x), A.WARM_IN), dtype=torch.bfloat16, device="cuda")
    T = torch.zeros((n_steps * len(x), 2), dtype=torch.float32, device="cuda")
    s.warm_collect(1e-4, n_steps, F, T)
    w = A.Warm(seed=1)
    n_train = 20 * len(x)
    losses = []
    for it in range(300):
        lo = w.train_step(F[:n_train], T[:n_train], lr=2e-3 if it < 200 else 5e-4)
        losses.append(lo)
    held, _ = w.loss_grad(F[n_train:], T[n_train:])
    base = 0.5 * float((T[n_train:] ** 2).sum(dim=1).mean())
    return dict(w=w, losses=losses, held=held, base=base, x=s.positions(), t=t, H=s.box())


def test_training_lowers_the_loss(trained):
    L = trained["losses"]
    assert L[-1] < 0.8 * L[0], (L[0], L[-1])
    # held-out steps: better than predicting zero displacement
    assert trained["held"] < trained["base"], (trained["held"], trained["base"])


def test_gated_warm_start_keeps_the_aqs_path(A, syn, trained):
    x, t, H = trained["x"], trained["t"], trained["H"]
    plain = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_MIXED)
    ref = plain.run_sequential(1e-4, 12)
    warm = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_MIXED)
    out = warm.run_sequential_warm(trained["w"], 1e-4, 12)
    np.testing.assert_allclose(out["E"][:, 0], ref["E"][:, 0], rtol=1e-9)
    assert np.array_equal(out["D"][:, 0] > 1e-2, ref["D"][:, 0] > 1e-2)
    d = warm.positions() - plain.positions()
    L = np.diag(H)
    d -= np.round(d / L) * L
    d -= d.mean(axis=0)
    assert np.sqrt((d * d).sum(1)).max() < 1e-6
    gain = ref["iters"].sum() / max(1, out["iters"].sum())
    print(f"warm start: FIRE iterations {out['iters'].sum()} vs plain {ref['iters'].sum()} "
          f"(x{gain:.3f}), learned start kept on {int(out['used'].sum())}/12 steps; "
          f"training loss {trained['losses'][0]:.4g} -> {trained['losses'][-1]:.4g}, "
          f"held-out {trained['held']:.4g} vs zero-prediction {trained['base']:.4g}")
