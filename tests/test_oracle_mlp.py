"""Pins of the oracle's warm-start pieces (no GPU): the GELU network against
tabulated normal-CDF values and a least-squares closed form, its gradients by
finite differences, and the neighbour-shell features against a numpy
brute-force search."""
import numpy as np
import pytest


def _net(rng, widths, scale=0.5):
    Ws = [rng.standard_normal((widths[i + 1], widths[i])) * scale / np.sqrt(widths[i])
          for i in range(len(widths) - 1)]
    bs = [rng.standard_normal(widths[i + 1]) * 0.1 for i in range(len(widths) - 1)]
    return Ws, bs


def test_gelu_matches_normal_cdf_table(orc):
    """GELU(z) = z Phi(z); Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208."""
    z = np.array([[0.0], [1.0], [-1.0], [2.0]])
    Y = orc.mlp_forward([np.eye(1), np.eye(1)], [np.zeros(1), np.zeros(1)], z)
    want = np.array([0.0, 0.8413447460685429, -(1 - 0.8413447460685429), 2 * 0.9772498680518208])
    np.testing.assert_allclose(Y[:, 0], want, rtol=1e-15, atol=1e-16)


def test_linear_layer_gradient_closed_form(orc):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((50, 7))
    T = rng.standard_normal((50, 3))
    Ws, bs = _net(rng, [7, 3])
    loss, dW, db = orc.mlp_loss_grad(Ws, bs, X, T)
    Y = X @ Ws[0].T + bs[0]
    R = Y - T
    assert loss == pytest.approx(0.5 * np.sum(R * R) / 50, rel=1e-13)
    np.testing.assert_allclose(dW[0], R.T @ X / 50, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(db[0], R.mean(axis=0), rtol=1e-12, atol=1e-14)
    # at the least-squares solution the gradient vanishes
    Xa = np.hstack([X, np.ones((50, 1))])
    sol = np.linalg.lstsq(Xa, T, rcond=None)[0]
    _, dW2, db2 = orc.mlp_loss_grad([sol[:7].T], [sol[7]], X, T)
    assert np.abs(dW2[0]).max() < 1e-12 and np.abs(db2[0]).max() < 1e-12


def test_mlp_gradients_finite_difference(orc):
    rng = np.random.default_rng(2)
    widths = [6, 5, 5, 4, 2]
    Ws, bs = _net(rng, widths, scale=1.2)
    X = rng.standard_normal((9, 6))
    T = rng.standard_normal((9, 2))
    _, dW, db = orc.mlp_loss_grad(Ws, bs, X, T)
    h = 1e-6
    for l in range(len(Ws)):
        for (o, k) in [(0, 0), (1, 2), (widths[l + 1] - 1, widths[l] - 1)]:
            Wp = [w.copy() for w in Ws]; Wp[l][o, k] += h
            Wm = [w.copy() for w in Ws]; Wm[l][o, k] -= h
            g = (orc.mlp_loss_grad(Wp, bs, X, T)[0] - orc.mlp_loss_grad(Wm, bs, X, T)[0]) / (2 * h)
            assert g == pytest.approx(dW[l][o, k], rel=1e-6, abs=1e-9)
        bp = [b.copy() for b in bs]; bp[l][0] += h
        bm = [b.copy() for b in bs]; bm[l][0] -= h
        g = (orc.mlp_loss_grad(Ws, bp, X, T)[0] - orc.mlp_loss_grad(Ws, bm, X, T)[0]) / (2 * h)
        assert g == pytest.approx(db[l][0], rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_knn_features_brute_force(orc, syn, dim):
    n = 120 if dim == 2 else 150
    x, t, H = syn.random_glass_start(n, dim, seed=5, density=0.5 if dim == 3 else 1.2)
    if dim == 2:
        H = H.copy(); H[0, 1] = 0.1 * H[1, 1]
    k = 12
    feat = orc.knn_features(x, t, H, 2, k)
    assert feat.shape == (n, k * dim + 2)
    Hi = np.linalg.inv(H)
    for i in range(0, n, 13):
        d = x - x[i]
        # minimum image by scanning all images with |n| <= 1 (cells are large)
        best = None
        for nv in np.array(np.meshgrid(*([[-1, 0, 1]] * dim))).reshape(dim, -1).T:
            c = d + (H @ nv)[None, :]
            best = c if best is None else np.where((c * c).sum(1)[:, None] < (best * best).sum(1)[:, None], c, best)
        s = (best * best).sum(1)
        order = [j for j in np.lexsort((np.arange(n), s)) if j != i][:k]
        np.testing.assert_allclose(feat[i, :k * dim].reshape(k, dim), best[order], atol=1e-12)
        assert feat[i, k * dim + t[i]] == 1.0 and feat[i, k * dim:].sum() == 1.0
