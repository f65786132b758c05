"""Pins of the MLP oracle: torch's float64 layers for the forward pass,
central finite differences for the gradient, exact BF16 rounding cases."""
import numpy as np
import pytest
import torch

from oracle import mlp


def _data(n=7, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 12))
    T = rng.normal(size=(n, 4))
    M = (rng.random((n, 4)) < 0.7).astype(np.float64)
    return X, T, M


def test_forward_matches_torch_float64_layers():
    theta = mlp.init_params(1) + 0.01 * np.random.default_rng(2).normal(size=mlp.param_count())
    X, _, _ = _data()
    Y, _, _ = mlp.forward(theta, X)
    layers = mlp.unflatten(theta)
    h = torch.tensor(X, dtype=torch.float64)
    for i, (W, b) in enumerate(layers):
        h = torch.nn.functional.linear(h, torch.tensor(W.T), torch.tensor(b))
        if i < 3:
            h = torch.tanh(h)
    assert np.allclose(Y, h.numpy(), rtol=1e-13, atol=1e-13)


def test_gradient_matches_central_differences():
    theta = mlp.init_params(3) + 0.05 * np.random.default_rng(4).normal(size=mlp.param_count())
    X, T, M = _data(5, 1)
    loss, g = mlp.loss_grad(theta, X, T, M)
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.choice(mlp.param_count(), 40, replace=False),
                          [0, mlp.param_count() - 1, 12 * 256, 12 * 256 + 255]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss_grad(theta + e, X, T, M)[0] - mlp.loss_grad(theta - e, X, T, M)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_masked_outputs_do_not_contribute():
    theta = mlp.init_params(6)
    X, T, M = _data(6, 2)
    M[:, 2] = 0.0
    T2 = T.copy()
    T2[:, 2] += 100.0
    l1, g1 = mlp.loss_grad(theta, X, T, M)
    l2, g2 = mlp.loss_grad(theta, X, T2, M)
    assert l1 == l2 and np.array_equal(g1, g2)


def test_loss_is_the_masked_mean_squared_error():
    """The loss is the mean of the squared errors over the unmasked outputs
    (numpy's mean of the selected entries): zero with zero gradient where the
    targets are the network's own outputs, the single squared error where one
    output is unmasked, and zero where none is."""
    rng = np.random.default_rng(7)
    theta = mlp.init_params(3)
    X = rng.normal(size=(9, 12))
    Y = mlp.forward(theta, X)[0]
    T = Y + rng.normal(size=Y.shape)
    M = (rng.uniform(size=Y.shape) < 0.6).astype(np.float64)
    loss, _ = mlp.loss_grad(theta, X, T, M)
    assert abs(loss / np.mean((Y - T)[M > 0] ** 2) - 1.0) < 1e-13
    loss, g = mlp.loss_grad(theta, X, Y, np.ones_like(Y))
    assert loss == 0.0 and not np.any(g)
    one = np.zeros_like(Y)
    one[4, 2] = 1.0
    assert abs(mlp.loss_grad(theta, X, T, one)[0] / (Y[4, 2] - T[4, 2]) ** 2 - 1.0) < 1e-13
    assert mlp.loss_grad(theta, X, T, np.zeros_like(Y))[0] == 0.0


def test_init_is_xavier_uniform():
    """Weights uniform on +-sqrt(6 / (fan_in + fan_out)) (Glorot & Bengio
    2010): inside the bound, reaching near it, with the uniform law's
    variance bound^2 / 3; biases zero."""
    for i, (W, b) in enumerate(mlp.unflatten(mlp.init_params(11))):
        k, n = mlp.SIZES[i], mlp.SIZES[i + 1]
        lim = np.sqrt(6.0 / (k + n))
        assert np.all(np.abs(W) <= lim) and not np.any(b)
        assert np.max(np.abs(W)) > (0.98 if W.size > 1000 else 0.9) * lim
        if W.size > 1000:
            assert abs(W.var() / (lim * lim / 3.0) - 1.0) < 0.03


def test_surrogate_features_floor_the_logs():
    """Absent species and numbers enter the features as the logs of their
    floors: q_min for the water contents, one particle per kg for cloud
    droplets and aerosol, 1e-3 per kg for raindrops, 1e-10 for vapour."""
    from oracle import surrogate as OS
    from paper_2010_14823_gb300 import synth
    F = synth.FIDX
    st = np.zeros(16)
    st[F["T"]], st[F["p"]], st[F["rho"]] = 280.0, 8e4, 1.0
    f = OS.features(st)
    qmin = 1e-14
    assert f[0] == np.log(qmin) and f[1] == np.log(qmin)
    assert f[2] == 0.0 and f[9] == 0.0 and f[3] == np.log(1e-3) and f[7] == np.log(1e-10)
    assert f[4] == 0.0 and f[10] == 0.0 and f[11] == 0.0


def test_bf16_rounding_is_round_to_nearest_even():
    # exactly representable values stay, halfway cases go to the even neighbour
    one = np.float32(1.0)
    ulp = 2.0 ** -7
    assert mlp.bf16(1.0) == 1.0 and mlp.bf16(-2.5) == -2.5
    assert mlp.bf16(1.0 + ulp / 2) == 1.0                 # tie -> even (1.0)
    assert mlp.bf16(1.0 + 3 * ulp / 2) == 1.0 + 2 * ulp   # tie -> even (1 + 2 ulp)
    assert mlp.bf16(1.0 + 0.6 * ulp) == 1.0 + ulp
    x = np.random.default_rng(7).normal(size=1000)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 + 1e-300)   # unit roundoff 2^-8
    assert np.all((r.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)
    del one


def test_param_count_and_layout():
    assert mlp.param_count() == 12 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 4 + 4
    theta = np.arange(mlp.param_count(), dtype=np.float64)
    assert np.array_equal(mlp.flatten(mlp.unflatten(theta)), theta)
    W1, b1 = mlp.unflatten(theta)[0]
    assert W1[0, 1] == 1 and W1[1, 0] == 256 and b1[0] == 12 * 256


def test_surrogate_targets_and_masks_follow_the_scheme():
    """The surrogate's targets are the natural logs of the scheme oracle's four
    warm-rain rates, defined exactly where the scheme computes each (cloud:
    autoconversion and cloud self-collection; cloud and rain: accretion;
    rain: rain self-collection), and its features recover the state they
    came from."""
    import oracle as O
    from oracle import surrogate as OS
    from paper_2010_14823_gb300 import synth
    F = synth.FIDX

    def state(**kw):
        st = np.zeros(16)
        base = dict(T=285.0, qv=8e-3, p=9e4, rho=1.1, na=1e8, w=0.3)
        base.update(kw)
        for k, v in base.items():
            st[F[k]] = v
        return st

    cases = {(1, 0, 1, 0): dict(qc=3e-4, nc=1e8),
             (0, 0, 0, 1): dict(qr=1e-4, nr=1e3),
             (1, 1, 1, 1): dict(qc=3e-4, nc=1e8, qr=1e-4, nr=1e3)}
    for mask, kw in cases.items():
        st = state(**kw)
        y, m = OS.targets(st, 1.0)
        assert tuple(m) == tuple(float(v) for v in mask)          # exactly 0 or 1
        r = O.rates(st, 1.0)
        for j, name in enumerate(("aut", "acc", "scc", "scr")):
            if m[j]:
                assert abs(np.exp(y[j]) / r[name] - 1.0) < 1e-14
            else:
                assert y[j] == 0.0
        f = OS.features(st)
        assert OS.warm(st)
        for j, name in ((0, "qc"), (1, "qr"), (2, "nc"), (3, "nr")):
            if st[F[name]] > 0:
                assert abs(np.exp(f[j]) / st[F[name]] - 1.0) < 1e-14
        assert f[5] == st[F["T"]] - 273.15 and f[8] == st[F["w"]]
        assert (f[10], f[11]) == (float(st[F["qc"]] > 1e-14), float(st[F["qr"]] > 1e-14))
    assert not OS.warm(state())
