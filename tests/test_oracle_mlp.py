"""Pins of the oracle's forcing network (Sec. 2.2) and Algorithm 1 (Sec. 2.1)."""
import numpy as np
import pytest

from oracle import algorithm1, dgsem, mlp, physics
from paper_2207_11571_gb300 import inputs


def small_net(seed=0, dims=(12, 16, 16, 12)):
    return mlp.he_uniform_init(list(dims), inputs.uniform_draws(list(dims), seed))


def test_round_bf16_matches_library_conversion():
    torch = pytest.importorskip("torch")
    x = np.concatenate([inputs.normal(4096, 1, 3.0), inputs.normal(64, 2, 1e-30),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 65504.0, -3.0e38]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.round_bf16(x), ref)


def test_forward_matches_library_linear_relu():
    torch = pytest.importorskip("torch")
    params = small_net(1)
    for W, b in params:
        b += inputs.normal(b.shape, 9, 0.1)
    x = inputs.normal((7, 12), 3)
    y, _ = mlp.forward(params, x)
    h = torch.tensor(x)
    for l, (W, b) in enumerate(params):
        h = torch.nn.functional.linear(h, torch.tensor(W), torch.tensor(b))
        if l < len(params) - 1:
            h = torch.relu(h)
    np.testing.assert_allclose(y, h.numpy(), rtol=1e-14, atol=1e-14)


def test_backward_matches_central_finite_differences():
    params = small_net(2)
    params = [(W, b + inputs.normal(b.shape, 17 + i, 0.05)) for i, (W, b) in enumerate(params)]
    x = inputs.normal((9, 12), 4)
    t = inputs.normal((9, 12), 5)
    y, cache = mlp.forward(params, x)
    _, dy = mlp.mse_loss(y, t)
    grads = mlp.backward(params, cache, dy)
    eps = 1e-6
    for l in range(len(params)):
        for which in (0, 1):
            P = params[l][which]
            flat = P.reshape(-1)
            for idx in np.random.default_rng(l * 2 + which).choice(flat.size, 6, replace=False):
                orig = flat[idx]
                flat[idx] = orig + eps
                lp = mlp.mse_loss(mlp.forward(params, x)[0], t)[0]
                flat[idx] = orig - eps
                lm = mlp.mse_loss(mlp.forward(params, x)[0], t)[0]
                flat[idx] = orig
                fd = (lp - lm) / (2 * eps)
                an = grads[l][which].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-7 * max(1e-3, abs(fd)), (l, which, idx, fd, an)


def test_mse_loss_closed_form_on_a_two_by_three_example():
    """Sec. 2.2 trains on the mean squared error: the mean over the batch and the outputs.
    On y - t = [[1, -2, 0], [3, 0, -1]] the sum of squares is 15 over 6 entries, so
    L = 2.5 and dL/dy = 2 (y - t) / 6."""
    y = np.array([[1.0, -1.0, 2.0], [3.5, 0.25, 0.0]])
    t = np.array([[0.0, 1.0, 2.0], [0.5, 0.25, 1.0]])
    L, dy = mlp.mse_loss(y, t)
    assert L == 2.5
    np.testing.assert_array_equal(dy, np.array([[1.0, -2.0, 0.0], [3.0, 0.0, -1.0]]) / 3.0)


def test_mse_loss_and_gradient_match_torch():
    """The normalisation (batch x outputs) equals torch's mean-reduced MSE, and the
    gradient equals autograd's."""
    torch = pytest.importorskip("torch")
    y = inputs.normal((17, 5), 11)
    t = inputs.normal((17, 5), 12)
    L, dy = mlp.mse_loss(y, t)
    yt = torch.tensor(y, requires_grad=True)
    Lt = torch.nn.functional.mse_loss(yt, torch.tensor(t), reduction="mean")
    Lt.backward()
    assert L == pytest.approx(Lt.item(), rel=1e-15)
    np.testing.assert_allclose(dy, yt.grad.numpy(), rtol=1e-14, atol=0)


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g, bias correction makes m_hat = g and v_hat = g^2 exactly,
    so every step moves each weight by -lr g / (|g| + eps) (Kingma & Ba)."""
    params = [(np.array([[0.5, -1.0], [2.0, 0.0]]), np.array([0.1, -0.2]))]
    g = [(np.array([[0.3, -2.0], [1e-3, -4e-4]]), np.array([5.0, -0.01]))]
    state = {}
    lr, eps = 1e-3, 1e-7
    p = params
    for _ in range(5):
        p = mlp.adam_step(p, g, state, lr=lr, eps=eps)
    for (W0, b0), (W, b), (gW, gb) in zip(params, p, g):
        np.testing.assert_allclose(W, W0 - 5 * lr * gW / (np.abs(gW) + eps), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(b, b0 - 5 * lr * gb / (np.abs(gb) + eps), rtol=1e-12, atol=1e-15)


def test_training_reduces_loss_on_learnable_map():
    dims = [12, 32, 32, 12]
    params = mlp.he_uniform_init(dims, inputs.uniform_draws(dims, 3))
    A = inputs.normal((12, 12), 6, 0.3)
    X = inputs.normal((256, 12), 7)
    T = np.tanh(X @ A)
    scalers = algorithm1.scalers_from_data(X, T)
    state = {}
    losses = []
    for _ in range(300):
        params, loss, _ = mlp.train_step(params, state, scalers, X, T, lr=3e-3)
        losses.append(loss)
    assert losses[-1] < 0.1 * losses[0]


def test_bf16_rounding_points_stay_close_to_fp64():
    params = small_net(4, (64, 64, 64, 64))
    x = inputs.normal((32, 64), 8)
    y64, _ = mlp.forward(params, x)
    y16, _ = mlp.forward(params, x, bf16=True)
    rel = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-5 < rel < 2e-2


# ----------------------------------------------------------------------------- Algorithm 1

def test_pairs_vanish_when_high_and_low_order_coincide():
    """With P_HO = P_LO and one HO step per LO step, G is the identity and the HO and LO
    evolutions coincide, so s_n = 0 (Algorithm 1, first loop)."""
    mesh = dgsem.Mesh(2, 3)
    flow = physics.Flow(Re=200.0)
    q = dgsem.tgv_state(mesh, flow, inputs.perturbation((5, 512)))
    X, T, _ = algorithm1.generate_pairs(q, mesh, mesh, flow, flow, dt_lo=1e-3, ratio=1, n_steps=2)
    assert X.shape == (2 * 8, 320) and T.shape == (2 * 8, 320)
    assert np.abs(T).max() < 1e-8


def test_exact_forcing_reproduces_filtered_high_order_trajectory():
    """Adding dt * s_n after the uncorrected LO step (Algorithm 1, third loop) with the
    generated s_n lands exactly on G q_HO^{n+1}: checks pair bookkeeping and layout."""
    m8, m3 = dgsem.Mesh(2, 5), dgsem.Mesh(2, 3)
    flow = physics.Flow(Re=200.0)
    q8 = dgsem.tgv_state(m8, flow, inputs.perturbation((5, 8 * 216)))
    dt = 2e-3
    X, T, q_end = algorithm1.generate_pairs(q8, m8, m3, flow, flow, dt_lo=dt, ratio=2, n_steps=2)
    K, n = 2, 4
    q_nn1 = dgsem.field_from_features(X[8:16], K, n)       # q_NN^1 = G q_HO^1
    s1 = dgsem.field_from_features(T[8:16], K, n)
    corrected = dgsem.rk3_step(q_nn1, dt, lambda z: dgsem.rhs(z, m3, flow)) + dt * s1
    np.testing.assert_allclose(corrected, dgsem.project(q_end, 5, 3), rtol=1e-12, atol=1e-12)
    # the forcing is nonzero and the momentum-only layout picks rho u, rho v, rho w
    assert np.abs(T).max() > 1e-6
    Xm = dgsem.element_features(q_nn1, (1, 2, 3))
    np.testing.assert_array_equal(Xm, X[8:16][:, 64:256])


@pytest.mark.parametrize("mode", ["stage", "post"])
def test_momentum_only_forcing_conserves_mass_and_energy(mode):
    """Sec. 2.2's network acts on the momenta only (s_rho = s_rhoe = 0): the corrected
    steps keep total mass and energy to round-off, as the operator does, while the
    forcing moves total momentum."""
    mesh = dgsem.Mesh(2, 3)
    flow = physics.Flow(Re=200.0)
    q = dgsem.tgv_state(mesh, flow, inputs.perturbation((5, 512)))
    dims = [192, 32, 192]
    params = mlp.he_uniform_init(dims, inputs.uniform_draws(dims, 9))
    feats = dgsem.element_features(q, (1, 2, 3))
    scalers = (feats.mean(0), feats.std(0) + 1.0, np.zeros(192), np.full(192, 0.5))
    W = mesh.quadrature_weights()
    total = lambda z: (W * z).sum(axis=(-1, -2, -3, -4, -5, -6))
    t0 = total(q)
    z = q
    for _ in range(3):
        z = algorithm1.corrected_step(z, 1e-3, mesh, flow, params, scalers, mode=mode, io_vars=(1, 2, 3))
    t1 = total(z)
    assert abs(t1[0] - t0[0]) < 1e-13 * t0[0] and abs(t1[4] - t0[4]) < 1e-13 * t0[4]
    assert np.abs(t1[1:4] - t0[1:4]).max() > 1e-6


def test_stage_and_post_forcing_modes_agree_to_second_order():
    """Forcing inside every RK stage vs Algorithm 1's post-step correction: the two
    differ by O(dt^2) per step."""
    mesh = dgsem.Mesh(2, 3)
    flow = physics.Flow(Re=200.0)
    q = dgsem.tgv_state(mesh, flow, inputs.perturbation((5, 512)))
    dims = [320, 32, 320]
    params = mlp.he_uniform_init(dims, inputs.uniform_draws(dims, 5))
    params = [(W * 0.1, b) for W, b in params]
    feats = dgsem.element_features(q)
    scalers = (feats.mean(0), feats.std(0) + 1.0, np.zeros(320), np.full(320, 0.5))
    diffs = []
    for dt in (2e-3, 1e-3):
        a = algorithm1.corrected_step(q, dt, mesh, flow, params, scalers, mode='stage')
        b = algorithm1.corrected_step(q, dt, mesh, flow, params, scalers, mode='post')
        diffs.append(np.abs(a - b).max())
    assert diffs[1] < diffs[0] / 3.0 and diffs[1] > 0


def test_he_uniform_initialisation_has_variance_two_over_fan_in():
    """He et al.'s initialisation keeps Var(W) = 2 / fan_in (a uniform law on [-a, a]
    has variance a^2 / 3); biases start at zero."""
    dims = [320, 512, 256]
    params = mlp.he_uniform_init(dims, inputs.uniform_draws(dims, 17))
    for (W, b), fan_in, fan_out in zip(params, dims[:-1], dims[1:]):
        assert W.shape == (fan_out, fan_in) and not b.any()
        # sample variance of fan_in * fan_out >= 131072 draws: within 2 % of 2 / fan_in
        assert abs(W.var() * fan_in / 2.0 - 1.0) < 0.02
        assert np.abs(W).max() <= np.sqrt(6.0 / fan_in)


def test_scalers_are_population_mean_and_std_with_unit_std_for_constant_features():
    X = inputs.normal((500, 6), 3) * np.arange(1, 7) + np.arange(6)
    X[:, 2] = 4.0
    T = inputs.normal((500, 4), 4)
    mi, si, mo, so = algorithm1.scalers_from_data(X, T)
    np.testing.assert_allclose(mi, X.mean(axis=0), rtol=1e-14, atol=1e-14)
    ref = X.std(axis=0, ddof=0)
    ref[2] = 1.0
    np.testing.assert_allclose(si, ref, rtol=1e-13)
    np.testing.assert_allclose(so, T.std(axis=0, ddof=0), rtol=1e-13)
    np.testing.assert_allclose(mo, T.mean(axis=0), atol=1e-15)
