"""GPU parity of the forcing network (tcgen05 BF16 GEMMs, training kernels) against the
FP64 oracle with the same bf16 rounding points, through the C ABI."""
import os

import numpy as np
import pytest

from oracle import algorithm1, dgsem, mlp, physics
from paper_2207_11571_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# BF16 network against the oracle with the same rounding points: FP32 vs FP64
# accumulation (~1e-6) plus rare one-ulp (2^-8) differences in bf16-rounded activations
# near rounding ties.
NN_RTOL = 2e-3


@pytest.fixture(scope="module")
def L():
    from tests.libbuild import ensure_built
    ensure_built()
    from paper_2207_11571_gb300 import dg
    dg.lib()
    return dg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def bf16_dev(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("M,N,K,bias,relu", [
    (128, 64, 64, False, False), (300, 320, 320, True, False), (4096, 512, 320, True, True),
    (1000, 192, 512, False, True), (77, 100, 135, True, False), (4096, 320, 512, True, False),
    (256, 256, 4096, False, False)])
def test_tcgen05_gemm_matches_float64_reference(L, M, N, K, bias, relu):
    from paper_2207_11571_gb300 import nn
    k8 = (K + 7) // 8 * 8
    lda = k8 + 16
    A = torch.randn(M, lda, generator=torch.Generator().manual_seed(M + K)).to(torch.bfloat16)
    B = torch.randn(N, lda, generator=torch.Generator().manual_seed(N + 3 * K)).to(torch.bfloat16)
    # columns K .. k8-1 share a 16-byte chunk with valid data and must be zero (contract of
    # nn_gemm_bf16); columns from k8 on hold garbage that TMA must read as zeros
    A[:, K:k8] = 0
    B[:, K:k8] = 0
    A[:, k8:] = 1e4
    B[:, k8:] = -1e4
    b = torch.randn(N, generator=torch.Generator().manual_seed(7)) if bias else None
    C = nn.nn_gemm_bf16(A.cuda(), B.cuda(), b.cuda() if bias else None, relu, K=K).cpu().double()
    ref = A[:, :K].double() @ B[:, :K].double().T
    if bias:
        ref += b.double()
    if relu:
        ref = ref.clamp_min(0)
    err = (C - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err


def make_net(nn, n_in, width, n_hidden, seed, max_batch=512, first_var=0, n_vars=5):
    dims = [n_in] + [width] * n_hidden + [n_in]
    draws = inputs.uniform_draws(dims, seed)
    h = nn.nn_create(n_in, n_in, width, n_hidden, first_var, n_vars, max_batch, draws)
    params = mlp.he_uniform_init(dims, draws)
    # the library keeps FP32 masters: the oracle starts from the same FP32 values
    params = [(W.astype(np.float32).astype(np.float64), b) for W, b in params]
    return h, params


def set_random_scalers(nn, h, n, seed):
    rng = np.random.default_rng(seed)
    sc = (rng.normal(0, 0.5, n).astype(np.float32), rng.uniform(0.5, 2.0, n).astype(np.float32),
          rng.normal(0, 0.1, n).astype(np.float32), rng.uniform(0.1, 1.0, n).astype(np.float32))
    nn.nn_set_scalers(h, *sc)
    return tuple(s.astype(np.float64) for s in sc)


@pytest.mark.parametrize("n_in,width,n_hidden,rows", [(320, 256, 4, 300), (192, 512, 2, 129), (320, 512, 6, 512)])
def test_forward_matches_oracle(L, n_in, width, n_hidden, rows):
    from paper_2207_11571_gb300 import nn
    h, params = make_net(nn, n_in, width, n_hidden, seed=n_in + width)
    sc = set_random_scalers(nn, h, n_in, 1)
    X = inputs.normal((rows, n_in), 2).astype(np.float32)
    S = torch.empty(rows, n_in, dtype=torch.float32, device="cuda")
    nn.nn_forward(h, torch.from_numpy(X).cuda(), S)
    ref = mlp.infer(params, sc, X.astype(np.float64), bf16=True)
    assert rel(S.cpu().numpy(), ref) < NN_RTOL
    nn.nn_destroy(h)


@pytest.mark.parametrize("n_in,width,n_hidden,rows", [(320, 512, 4, 4096), (320, 256, 4, 300), (192, 512, 2, 129),
                                                     (320, 512, 6, 512), (80, 96, 3, 257), (320, 104, 2, 200)])
def test_fused_inference_equals_per_layer_gemms(L, n_in, width, n_hidden, rows):
    """The fused multi-layer kernel and the one-GEMM-per-layer path compute the same network
    (same bf16 rounding points, same K order); width 96 exercises zero-padded panels,
    width 104 (not a multiple of 16) falls back to the per-layer path."""
    from paper_2207_11571_gb300 import nn
    h, _ = make_net(nn, n_in, width, n_hidden, seed=7 + width, max_batch=max(rows, 512))
    set_random_scalers(nn, h, n_in, 3)
    X = torch.from_numpy(inputs.normal((rows, n_in), 4).astype(np.float32)).cuda()
    S_fused = torch.full((rows, n_in), float("nan"), dtype=torch.float32, device="cuda")
    S_layer = torch.full_like(S_fused, float("nan"))
    nn.nn_set_fused(h, True)
    nn.nn_forward(h, X, S_fused)
    nn.nn_set_fused(h, False)
    nn.nn_forward(h, X, S_layer)
    torch.cuda.synchronize()
    assert torch.isfinite(S_fused).all()
    err = ((S_fused - S_layer).norm() / S_layer.norm()).item()
    assert err < 1e-5, err
    nn.nn_destroy(h)


def test_train_step_gradients_loss_and_adam_match_oracle(L):
    from paper_2207_11571_gb300 import nn
    n, width, nh, B = 320, 256, 3, 384
    h, params = make_net(nn, n, width, nh, seed=11)
    sc = set_random_scalers(nn, h, n, 2)
    X = inputs.normal((1000, n), 3).astype(np.float32)
    Y = (0.3 * inputs.normal((1000, n), 4)).astype(np.float32)
    idx = np.random.default_rng(5).permutation(1000)[:B].astype(np.int64)
    loss = nn.nn_train_step(h, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), torch.from_numpy(idx).cuda(),
                            lr=1e-3)
    state = {}
    new, loss_or, grads = mlp.train_step(params, state, sc, X[idx].astype(np.float64), Y[idx].astype(np.float64),
                                         bf16=True, lr=1e-3, eps=1e-7)
    assert loss == pytest.approx(loss_or, rel=NN_RTOL)
    for l in range(nh + 1):
        dW, db = nn.nn_get_grads(h, l)
        assert rel(dW, grads[l][0]) < NN_RTOL, l
        assert rel(db, grads[l][1]) < NN_RTOL, l
    # Adam on the library's own gradients: isolate the optimiser arithmetic
    params2 = [(W, b) for W, b in params]
    g_lib = [tuple(a.astype(np.float64) for a in nn.nn_get_grads(h, l)) for l in range(nh + 1)]
    new_lib = mlp.adam_step(params2, g_lib, {}, lr=1e-3, eps=1e-7)
    for l in range(nh + 1):
        W, b = nn.nn_get_params(h, l)
        np.testing.assert_allclose(W, new_lib[l][0], rtol=0, atol=2e-6 * max(1.0, np.abs(W).max()))
        np.testing.assert_allclose(b, new_lib[l][1], rtol=0, atol=2e-6)
    nn.nn_destroy(h)


@pytest.mark.parametrize("bad", [dict(lr=-1e-3), dict(lr=float("nan")), dict(beta1=1.0), dict(beta2=-0.1),
                                 dict(eps=0.0), dict(eps=float("inf"))])
def test_train_step_rejects_bad_adam_hyperparameters(L, bad):
    """Adam's update divides by sqrt(v) + eps and by 1 - beta^t: out-of-range values are
    refused before any launch and leave the weights as they were."""
    from paper_2207_11571_gb300 import nn
    h, _ = make_net(nn, 64, 64, 1, seed=3, max_batch=128)
    X = torch.zeros((128, 64), device="cuda")
    W0, b0 = nn.nn_get_params(h, 0)
    with pytest.raises(L.DGError) as e:
        nn.nn_train_step(h, X, X, **bad)
    assert e.value.status == L.DG_ERR_INVALID_ARG
    W1, b1 = nn.nn_get_params(h, 0)
    assert np.array_equal(W0, W1) and np.array_equal(b0, b1)
    nn.nn_destroy(h)


def test_training_follows_oracle_loss_curve(L):
    """Mini-batch Adam training on the GPU (BF16 GEMMs) tracks the FP64 oracle's loss
    curve on the same data, shuffles and initial weights, and cuts the loss > 5x."""
    from paper_2207_11571_gb300 import nn
    n, B, epochs = 192, 256, 30
    h, params = make_net(nn, n, 256, 3, seed=21, max_batch=B, first_var=1, n_vars=3)
    X = inputs.normal((4096, n), 6).astype(np.float32)
    A = inputs.normal((n, n), 7, 1.0 / np.sqrt(n)).astype(np.float32)
    Y = (X @ A).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    nn.nn_compute_scalers(h, Xd, Yd)
    sc = tuple(a.astype(np.float64) for a in nn.nn_get_scalers(h))
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    gpu, ora, state = [], [], {}
    for epoch in range(epochs):
        perm = inputs.epoch_permutation(4096, 9, epoch)
        permd = torch.from_numpy(perm).cuda()
        for b0 in range(0, 4096, B):
            gpu.append(nn.nn_train_step(h, Xd, Yd, permd[b0:b0 + B], lr=2e-3))
            idx = perm[b0:b0 + B]
            params, loss, _ = mlp.train_step(params, state, sc, X64[idx], Y64[idx], lr=2e-3)
            ora.append(loss)
    for k in (10, 20, 30):
        g, o = np.mean(gpu[(k - 1) * 16:k * 16]), np.mean(ora[(k - 1) * 16:k * 16])
        assert abs(g - o) < 0.15 * o, (k, g, o)
    assert gpu[-1] < 0.2 * gpu[0]
    nn.nn_destroy(h)


def test_compute_scalers_matches_numpy(L):
    from paper_2207_11571_gb300 import nn
    h, _ = make_net(nn, 320, 64, 1, seed=3)
    X = (5 + 2 * inputs.normal((3000, 320), 8)).astype(np.float32)
    Y = inputs.normal((3000, 320), 9).astype(np.float32)
    Y[:, 7] = 1.5  # zero spread -> std 1
    nn.nn_compute_scalers(h, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    mi, si, mo, so = nn.nn_get_scalers(h)
    ref = algorithm1.scalers_from_data(X.astype(np.float64), Y.astype(np.float64))
    for a, b in zip((mi, si, mo, so), ref):
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6)
    assert so[7] == 1.0
    nn.nn_destroy(h)


@pytest.mark.parametrize("mode", [0, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_forcing_infer_matches_oracle_on_element_features(L, prec, mode):
    """Network forcing of every element of a solver state (per-layer GEMMs in chunks of
    max_batch, or the one-launch cluster kernel) against the oracle network on the FP64
    element features (bf16 rounding points)."""
    from paper_2207_11571_gb300 import dg, nn
    K, P = 3, 3
    ctx = dg.dg_create(K, P, 1600.0, 0.1, 0.71, 0, precision=prec)
    N = K ** 3 * 64
    q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
    dg.dg_init_tgv(ctx, q, torch.from_numpy(inputs.perturbation((5, N)).ravel()).cuda())
    h, params = make_net(nn, 320, 256, 2, seed=4, max_batch=10)   # 27 elements in chunks of 10
    feats = dgsem.element_features(q.cpu().numpy().reshape(5, K, K, K, 4, 4, 4))
    sc32 = (feats.mean(0).astype(np.float32), (feats.std(0) + 1e-3).astype(np.float32),
            np.zeros(320, np.float32), np.full(320, 0.01, np.float32))
    nn.nn_set_scalers(h, *sc32)
    nn.nn_set_fused(h, mode)
    s = torch.empty(K ** 3 * 320, dtype=torch.float32, device="cuda")
    nn.nn_forcing_infer(h, ctx, q, s)
    ref = mlp.infer(params, tuple(a.astype(np.float64) for a in sc32), feats, bf16=True)
    assert rel(s.cpu().numpy().reshape(27, 320), ref) < NN_RTOL
    nn.nn_destroy(h)
    dg.dg_destroy(ctx)


# (K, P, n_vars, width, hidden, precision): 64 elements (one tile), 125 (a ragged tile),
# 216 (two tiles, ragged), 512 (four tiles); momentum-only I/O (192 features); the
# benchmark network on 16^3 elements (4096, 32 clusters of 4 CTAs)
CLUSTER_CASES = [(4, 3, 5, 256, 2, 1), (5, 3, 5, 512, 4, 0), (6, 3, 3, 256, 3, 1), (8, 3, 5, 512, 4, 1),
                 (8, 3, 3, 512, 6, 0), (16, 3, 5, 512, 4, 1)]


@pytest.mark.parametrize("K,P,nv,width,hidden,prec", CLUSTER_CASES)
def test_cluster_forcing_equals_per_layer_gemms(L, K, P, nv, width, hidden, prec):
    """The one-launch forcing (features, every layer and the unscaling in clusters of CTAs
    that share activations through distributed shared memory) computes what the per-layer
    path computes: the same bf16 features and weights, FP32 accumulation.  A CTA's K loop
    starts on its own slice of the input (then the peers' slices), so the FP32 sums are
    taken in another order, which flips the bf16 rounding of a few hidden activations by
    one bf16 ulp (2^-8 relative); measured 9e-5 relative L2 on the output, bounded here at
    5e-4, where a stale or missing panel gives O(1).  Two launches on the same input are
    bitwise equal (no race between the slice copies and the tensor core)."""
    from paper_2207_11571_gb300 import dg, nn
    ctx = dg.dg_create(K, P, 1600.0, 0.1, 0.71, 0, precision=prec)
    N = dg.dg_sizes(ctx)[0]
    first = 0 if nv == 5 else 1
    feat = nv * (P + 1) ** 3
    q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
    dg.dg_init_tgv(ctx, q, torch.from_numpy(inputs.perturbation((5, N), eps=1e-3).ravel()).cuda())
    h, _ = make_net(nn, feat, width, hidden, seed=40 + K, max_batch=512, first_var=first, n_vars=nv)
    set_random_scalers(nn, h, feat, 6)
    out = {}
    for mode in (0, 2, 3):
        nn.nn_set_fused(h, min(mode, 2))
        s = torch.full((K ** 3 * feat,), float("nan"), dtype=torch.float32, device="cuda")
        nn.nn_forcing_infer(h, ctx, q, s)
        torch.cuda.synchronize()
        out[mode] = s
    assert torch.isfinite(out[2]).all()
    assert torch.equal(out[2], out[3])
    err = ((out[2] - out[0]).norm() / out[0].norm()).item()
    assert err < 5e-4, err
    nn.nn_destroy(h)
    dg.dg_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_corrected_rk3_with_features_from_the_gradient_phase_equals_separate_features(L, prec):
    """With the one-launch network path, the forcing's input features come out of the
    gradient phase of each RK stage (no feature launch); the corrected RK3 steps equal those
    of the per-layer path with its separate feature kernel (same bf16 features; the
    tensor core's accumulation order differs, which flips a few bf16 roundings of hidden
    activations: the two runs may differ by 5e-4 of what the forcing changed)."""
    from paper_2207_11571_gb300 import dg, nn
    K, P = 4, 3
    ctx = dg.dg_create(K, P, 200.0, 0.1, 0.71, 0, precision=prec)
    N = dg.dg_sizes(ctx)[0]
    q0 = torch.empty(5 * N, dtype=torch.float64, device="cuda")
    dg.dg_init_tgv(ctx, q0, torch.from_numpy(inputs.perturbation((5, N), eps=1e-3).ravel()).cuda())
    h, _ = make_net(nn, 192, 256, 3, seed=17, max_batch=128, first_var=1, n_vars=3)
    set_random_scalers(nn, h, 192, 9)
    out = {}
    for mode in (nn.NN_INFER_LAYERS, nn.NN_INFER_CLUSTER):
        nn.nn_set_fused(h, mode)
        q = q0.clone()
        dg.dg_rk3_step(ctx, q, 2e-3, 3, forcing=h)
        torch.cuda.synchronize()
        out[mode] = q
    plain = q0.clone()
    dg.dg_rk3_step(ctx, plain, 2e-3, 3)
    d = (out[nn.NN_INFER_CLUSTER] - out[nn.NN_INFER_LAYERS]).norm().item()
    effect = (out[nn.NN_INFER_LAYERS] - plain).norm().item()   # what the forcing changed
    assert effect > 0 and d < 5e-4 * effect, (d, effect)
    nn.nn_destroy(h)
    dg.dg_destroy(ctx)


@pytest.mark.parametrize("block_shape", [0, 1])
def test_rhs_and_rk3_with_forcing_match_oracle(L, block_shape):
    """dq/dt = p_LO(q) + s(q) (Eq. 4) and RK3 with s in every stage, FP64 operator, with
    rows of elements and with 2 x 2 x 2 cube blocks."""
    from paper_2207_11571_gb300 import dg, nn
    K, P = 2, 3
    flow = physics.Flow(Re=200.0, Mach=0.1)
    mesh = dgsem.Mesh(K, P)
    N = K ** 3 * 64
    pert = inputs.perturbation((5, N))
    q_or = dgsem.tgv_state(mesh, flow, pert)
    ctx = dg.dg_create(K, P, 200.0, 0.1, 0.71, 0, block_shape=block_shape)
    q = torch.from_numpy(q_or.reshape(5, -1).copy()).cuda()
    h, params = make_net(nn, 320, 128, 2, seed=8, max_batch=8)
    feats = dgsem.element_features(q_or)
    sc32 = (feats.mean(0).astype(np.float32), (feats.std(0) + 1e-2).astype(np.float32),
            np.zeros(320, np.float32), np.full(320, 0.05, np.float32))
    nn.nn_set_scalers(h, *sc32)
    sc = tuple(s.astype(np.float64) for s in sc32)
    R = torch.empty_like(q)
    dg.dg_rhs(ctx, q, R, forcing=h)
    s_or = algorithm1.forcing_field(params, sc, q_or, 4, bf16=True)
    R_plain = dgsem.rhs(q_or, mesh, flow)
    got_s = R.cpu().numpy().reshape(q_or.shape) - R_plain
    assert rel(got_s, s_or) < NN_RTOL
    dg.dg_rk3_step(ctx, q, 1e-3, 2, forcing=h)
    ref = q_or
    for _ in range(2):
        ref = algorithm1.corrected_step(ref, 1e-3, mesh, flow, params, sc, mode="stage", bf16=True)
    incr_gpu = q.cpu().numpy().reshape(q_or.shape) - q_or
    assert rel(incr_gpu, ref - q_or) < NN_RTOL
    nn.nn_destroy(h)
    dg.dg_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_momentum_only_forcing_conserves_mass_and_energy(L, prec):
    """Sec. 2.2's momentum-only network (s_rho = s_rhoe = 0) inside every RK stage: total
    mass and energy stay conserved to the operator's own bound (FP64 1e-13, FP32 1e-10,
    as for the plain operator) while the forcing moves total momentum."""
    from paper_2207_11571_gb300 import dg, nn
    K, P = 4, 3
    ctx = dg.dg_create(K, P, 200.0, 0.1, 0.71, 0, precision=prec)
    N = K ** 3 * 64
    q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
    dg.dg_init_tgv(ctx, q, torch.from_numpy(inputs.perturbation((5, N)).ravel()).cuda())
    h, _ = make_net(nn, 192, 128, 2, seed=21, max_batch=64, first_var=1, n_vars=3)
    nn.nn_set_scalers(h, np.zeros(192, np.float32), np.ones(192, np.float32), np.zeros(192, np.float32),
                      np.full(192, 0.05, np.float32))
    d0 = dg.dg_diagnostics(ctx, q)
    dg.dg_rk3_step(ctx, q, 2e-3, 10, h)
    d1 = dg.dg_diagnostics(ctx, q)
    tol = 1e-13 if prec == 0 else 1e-10
    assert abs(d1["mass"] - d0["mass"]) < tol * d0["mass"]
    assert abs(d1["energy"] - d0["energy"]) < tol * d0["energy"]
    assert max(abs(a - b) for a, b in zip(d1["momentum"], d0["momentum"])) > 1e-6
    nn.nn_destroy(h)
    dg.dg_destroy(ctx)


def test_rk3_with_post_step_forcing_matches_oracle(L):
    """Algorithm 1's placement (dg_set_forcing_mode POST), FP64 operator: the uncorrected
    RK3 step, then q += dt s(q^n), against the oracle's corrected_step(mode='post')."""
    from paper_2207_11571_gb300 import dg, nn
    K, P = 2, 3
    flow = physics.Flow(Re=200.0, Mach=0.1)
    mesh = dgsem.Mesh(K, P)
    q_or = dgsem.tgv_state(mesh, flow, inputs.perturbation((5, K ** 3 * 64)))
    ctx = dg.dg_create(K, P, 200.0, 0.1, 0.71, 0)
    dg.dg_set_forcing_mode(ctx, dg.DG_FORCING_POST)
    h, params = make_net(nn, 192, 128, 2, seed=9, max_batch=8, first_var=1, n_vars=3)
    feats = dgsem.element_features(q_or, (1, 2, 3))
    sc32 = (feats.mean(0).astype(np.float32), (feats.std(0) + 1e-2).astype(np.float32),
            np.zeros(192, np.float32), np.full(192, 0.05, np.float32))
    nn.nn_set_scalers(h, *sc32)
    sc = tuple(s.astype(np.float64) for s in sc32)
    q = torch.from_numpy(q_or.reshape(5, -1).copy()).cuda()
    dg.dg_rk3_step(ctx, q, 1e-3, 2, forcing=h)
    ref, plain = q_or, q_or
    for _ in range(2):
        ref = algorithm1.corrected_step(ref, 1e-3, mesh, flow, params, sc, mode="post", io_vars=(1, 2, 3), bf16=True)
        plain = dgsem.rk3_step(plain, 1e-3, lambda z: dgsem.rhs(z, mesh, flow))
    got = q.cpu().numpy().reshape(q_or.shape)
    # the forcing's effect over the two steps (the momenta directly, density and energy
    # through the second step's fluxes) within the network tolerance
    assert rel(got[1:4] - plain[1:4], ref[1:4] - plain[1:4]) < NN_RTOL
    assert rel(got - plain, ref - plain) < NN_RTOL
    # and it differs from the in-stage placement only at second order in dt
    stage = algorithm1.corrected_step(algorithm1.corrected_step(q_or, 1e-3, mesh, flow, params, sc, mode="stage",
                                                                io_vars=(1, 2, 3), bf16=True),
                                      1e-3, mesh, flow, params, sc, mode="stage", io_vars=(1, 2, 3), bf16=True)
    assert np.linalg.norm(got[1:4] - stage[1:4]) < 0.05 * np.linalg.norm(ref[1:4] - plain[1:4])
    nn.nn_destroy(h)
    dg.dg_destroy(ctx)


def test_training_resumes_after_save_and_load_with_the_adam_state(L, tmp_path):
    """Transfer learning warm-starts from a saved network (Sec. 3.6): nn_save keeps the
    weights, scalers, Adam moments m, v and step count t, so the first step after nn_load
    is the step the saved network would have taken.  Checked against the oracle's Adam
    with the restored t = 2, m, v (accumulated from the library's own gradients of the two
    steps before the save); a restart from zero moments would move the weights by lr
    sign(g) instead, which the bound separates."""
    from paper_2207_11571_gb300 import nn
    n, width, nh, B = 192, 128, 2, 256
    h, _ = make_net(nn, n, width, nh, seed=31, max_batch=B, first_var=1, n_vars=3)
    set_random_scalers(nn, h, n, 4)
    X = inputs.normal((600, n), 13).astype(np.float32)
    Y = (0.3 * inputs.normal((600, n), 14)).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    idx = [torch.from_numpy(np.random.default_rng(s).permutation(600)[:B].astype(np.int64)).cuda() for s in (1, 2, 3)]
    layers = range(nh + 1)

    def params_of(net):
        return [tuple(a.astype(np.float64) for a in nn.nn_get_params(net, l)) for l in layers]

    def grads_of(net):
        return [tuple(a.astype(np.float64) for a in nn.nn_get_grads(net, l)) for l in layers]

    state = {}
    for k in range(2):
        before = params_of(h)
        nn.nn_train_step(h, Xd, Yd, idx[k], lr=1e-3)
        mlp.adam_step(before, grads_of(h), state, lr=1e-3, eps=1e-7)
    assert state["t"] == 2
    path = tmp_path / "net.bin"
    nn.nn_save(h, path)
    h2 = nn.nn_load(path, max_batch=B)
    before = params_of(h2)
    nn.nn_train_step(h2, Xd, Yd, idx[2], lr=1e-3)
    g3 = grads_of(h2)
    fresh = mlp.adam_step(before, g3, {}, lr=1e-3, eps=1e-7)
    want = mlp.adam_step(before, g3, state, lr=1e-3, eps=1e-7)
    sep = 0.0
    for l in layers:
        W, b = nn.nn_get_params(h2, l)
        np.testing.assert_allclose(W, want[l][0], rtol=0, atol=2e-6 * max(1.0, np.abs(W).max()))
        np.testing.assert_allclose(b, want[l][1], rtol=0, atol=2e-6)
        sep = max(sep, np.abs(fresh[l][0] - want[l][0]).max())
    assert sep > 1e-4, sep   # the check would see lost moments
    # the saved network itself takes the same step
    nn.nn_train_step(h, Xd, Yd, idx[2], lr=1e-3)
    for l in layers:
        for a, b in zip(nn.nn_get_params(h, l), nn.nn_get_params(h2, l)):
            np.testing.assert_array_equal(a, b)
    nn.nn_destroy(h)
    nn.nn_destroy(h2)


def test_save_load_roundtrip_and_corruption_detection(L, tmp_path):
    from paper_2207_11571_gb300 import dg, nn
    h, _ = make_net(nn, 192, 64, 2, seed=5, first_var=1, n_vars=3)
    set_random_scalers(nn, h, 192, 3)
    path = tmp_path / "net.bin"
    nn.nn_save(h, path)
    h2 = nn.nn_load(path, max_batch=64)
    for l in range(3):
        for a, b in zip(nn.nn_get_params(h, l), nn.nn_get_params(h2, l)):
            np.testing.assert_array_equal(a, b)
    for a, b in zip(nn.nn_get_scalers(h), nn.nn_get_scalers(h2)):
        np.testing.assert_array_equal(a, b)
    raw = bytearray(path.read_bytes())
    raw[100] ^= 0xFF
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(raw))
    with pytest.raises(dg.DGError) as e:
        nn.nn_load(bad)
    assert e.value.status == dg.DG_ERR_IO
    (tmp_path / "short.bin").write_bytes(bytes(raw[:50]))
    with pytest.raises(dg.DGError):
        nn.nn_load(tmp_path / "short.bin")
    with pytest.raises(dg.DGError):
        nn.nn_load(tmp_path / "missing.bin")
    nn.nn_destroy(h)
    nn.nn_destroy(h2)


def test_backward_then_adam_equals_train_step(L):
    """nn_train_step is nn_backward (normalised over its own batch) followed by
    nn_adam_apply: two networks with the same weights end bitwise equal after two steps,
    with the same losses."""
    from paper_2207_11571_gb300 import nn
    n, B = 192, 200
    X = torch.from_numpy(inputs.normal((B, n), 41).astype(np.float32)).cuda()
    Y = torch.from_numpy(inputs.normal((B, n), 42).astype(np.float32)).cuda()
    a, _ = make_net(nn, n, 128, 2, seed=43, max_batch=B, first_var=1, n_vars=3)
    b, _ = make_net(nn, n, 128, 2, seed=43, max_batch=B, first_var=1, n_vars=3)
    for h in (a, b):
        nn.nn_compute_scalers(h, X, Y)
    for _ in range(2):
        la = nn.nn_train_step(a, X, Y, lr=2e-3)
        lb = nn.nn_backward(b, X, Y)
        nn.nn_adam_apply(b, lr=2e-3)
        assert la == lb
    for layer in range(3):
        for x, y in zip(nn.nn_get_params(a, layer), nn.nn_get_params(b, layer)):
            assert np.array_equal(x, y)
    nn.nn_destroy(a)
    nn.nn_destroy(b)


def test_backward_shares_sum_to_the_batch_gradient(L):
    """Data-parallel training on one device: two halves of a batch, each normalised over
    the whole batch (nn_backward's global_batch), give gradients and loss shares that sum
    to the whole batch's (FP32: the weight-gradient GEMMs sum the rows in other groups);
    the gradient buffers seen through nn_grad_buffers are what nn_adam_apply reads (zeroed
    gradients leave the parameters unchanged at Adam's first step)."""
    from paper_2207_11571_gb300 import nn
    n, B = 192, 256
    X = torch.from_numpy(inputs.normal((B, n), 44).astype(np.float32)).cuda()
    Y = torch.from_numpy(inputs.normal((B, n), 45).astype(np.float32)).cuda()
    h, _ = make_net(nn, n, 256, 3, seed=46, max_batch=B, first_var=1, n_vars=3)
    nn.nn_compute_scalers(h, X, Y)
    idx = torch.arange(B, dtype=torch.int64, device="cuda")
    full_loss = nn.nn_backward(h, X, Y, idx)
    full = [g.clone() for layer in range(4) for g in nn.nn_grad_buffers(h, layer)]
    l0 = nn.nn_backward(h, X, Y, idx[:100], global_batch=B)
    part = [g.clone() for layer in range(4) for g in nn.nn_grad_buffers(h, layer)]
    l1 = nn.nn_backward(h, X, Y, idx[100:], global_batch=B)
    for f, p0, layer_g in zip(full, part, [g for layer in range(4) for g in nn.nn_grad_buffers(h, layer)]):
        s = p0 + layer_g
        assert ((s - f).norm() / f.norm()).item() < 1e-5
    assert abs(l0 + l1 - full_loss) < 1e-6 * full_loss
    before = [nn.nn_get_params(h, layer) for layer in range(4)]
    for layer in range(4):
        for g in nn.nn_grad_buffers(h, layer):
            g.zero_()
    nn.nn_adam_apply(h)
    for layer in range(4):
        for x, y in zip(before[layer], nn.nn_get_params(h, layer)):
            assert np.array_equal(x, y)
    nn.nn_destroy(h)


def test_data_parallel_step_on_one_rank_equals_train_step(L):
    """partition.nn_dp_train_step over a one-rank process group (the all-reduce is the
    identity) equals nn_train_step bitwise."""
    import socket

    import torch.distributed as dist
    from paper_2207_11571_gb300 import nn, partition
    n, B = 192, 128
    X = torch.from_numpy(inputs.normal((B, n), 47).astype(np.float32)).cuda()
    Y = torch.from_numpy(inputs.normal((B, n), 48).astype(np.float32)).cuda()
    a, _ = make_net(nn, n, 128, 2, seed=49, max_batch=B, first_var=1, n_vars=3)
    b, _ = make_net(nn, n, 128, 2, seed=49, max_batch=B, first_var=1, n_vars=3)
    for h in (a, b):
        nn.nn_compute_scalers(h, X, Y)
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    group = None
    own = not dist.is_initialized()
    if own:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        la = nn.nn_train_step(a, X, Y)
        lb = partition.nn_dp_train_step(b, X, Y, group=group)
        assert abs(la - lb) <= 1e-7 * abs(la)
        for layer in range(3):
            for x, y in zip(nn.nn_get_params(a, layer), nn.nn_get_params(b, layer)):
                assert np.array_equal(x, y)
    finally:
        if own:
            dist.destroy_process_group()
        nn.nn_destroy(a)
        nn.nn_destroy(b)
