"""dg_rhs_noalloc: the operator for callers that may not allocate device memory (an
in-situ hook with a fixed memory budget, a host thread that must not take the
allocator's locks).  It must give the same result as the context-based dg_rhs, call
after call, while reusing one scratch array inside the library, and match the FP64
oracle on its own.  Collected last so that a stop-at-first-failure run has already run
every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

from oracle import dgsem, physics
from paper_2207_11571_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    from tests.libbuild import ensure_built
    ensure_built()
    from paper_2207_11571_gb300 import dg as _dg
    _dg.lib()
    return _dg


def rel_l2(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# (K, P): rows of elements at P3; the streamed high-order kernel at P6 with N % 4 == 0
# (own tiles by TMA bulk copies out of the scratch array) and at P7 with one element
# (N = 512, also bulk); both operator precisions
SHAPES = [(4, 3), (2, 6), (1, 7)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("K,P", SHAPES)
def test_noalloc_rhs_equals_context_rhs_on_two_calls_in_a_row(dg, K, P, prec):
    Re, Mach, Pr = 1600.0, 0.1, 0.71
    N = K ** 3 * (P + 1) ** 3
    ctx = dg.dg_create(K, P, Re, Mach, Pr, 0, precision=prec)
    try:
        q1 = torch.empty(5 * N, dtype=torch.float64, device="cuda")
        dg.dg_init_tgv(ctx, q1, torch.from_numpy(inputs.perturbation((5, N), seed=1).ravel()).cuda())
        q2 = torch.empty_like(q1)
        dg.dg_init_tgv(ctx, q2, torch.from_numpy(inputs.perturbation((5, N), seed=2, eps=1e-3).ravel()).cuda())
        for q in (q1, q2):   # two calls in a row on different states: the shared scratch is reused
            ref = torch.empty_like(q)
            dg.dg_rhs(ctx, q, ref)
            out = torch.full_like(q, float("nan"))
            dg.dg_rhs_noalloc(K, P, Re, Mach, Pr, 0, prec, q, out)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            # both paths run the same kernels with the same constants on the same inputs:
            # within the FP64 parity bar of the operator tests, and in fact bitwise equal
            assert rel_l2(out, ref) < 1e-12
            assert torch.equal(out, ref)
    finally:
        dg.dg_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("K,P", [(3, 6), (2, 6)])
def test_noalloc_rhs_matches_oracle(dg, K, P, prec):
    """Against the FP64 oracle itself (not only the context path), at P6 through the
    streamed kernel: K = 3 (N odd: own tiles by 4-byte copies) and K = 2 (bulk copies)."""
    from tests import fp32_bounds
    from tests.test_gpu_dg import assert_fp64_parity
    Re, Mach, Pr = 1600.0, 0.1, 0.71
    flow = physics.Flow(Re=Re, Mach=Mach, Pr=Pr)
    mesh = dgsem.Mesh(K, P)
    N = K ** 3 * (P + 1) ** 3
    q_or = dgsem.tgv_state(mesh, flow, inputs.perturbation((5, N), seed=4))
    q = torch.from_numpy(np.ascontiguousarray(q_or.reshape(5, -1))).cuda().reshape(-1)
    out = torch.full_like(q, float("nan"))
    dg.dg_rhs_noalloc(K, P, Re, Mach, Pr, 0, prec, q, out)
    torch.cuda.synchronize()
    R = out.cpu().numpy().reshape(q_or.shape)
    if prec == 0:
        assert_fp64_parity(R, q_or, mesh, flow)
    else:
        fp32_bounds.check(f"noalloc K{K} P{P}", R, dgsem.rhs(q_or, mesh, flow))


def test_noalloc_rhs_at_its_largest_mesh(dg):
    K, P, Re, Mach, Pr = 8, 3, 1600.0, 0.1, 0.71   # 8^3 (3+1)^3 = 32,768 nodes: the limit
    N = K ** 3 * (P + 1) ** 3
    assert N == 32768
    ctx = dg.dg_create(K, P, Re, Mach, Pr, 1, precision=0)
    try:
        q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
        dg.dg_init_tgv(ctx, q, torch.from_numpy(inputs.perturbation((5, N), seed=3, eps=1e-3).ravel()).cuda())
        ref = torch.empty_like(q)
        dg.dg_rhs(ctx, q, ref)
        out = torch.full_like(q, float("nan"))
        dg.dg_rhs_noalloc(K, P, Re, Mach, Pr, 1, 0, q, out)
        torch.cuda.synchronize()
        assert rel_l2(out, ref) < 1e-12
    finally:
        dg.dg_destroy(ctx)


def test_noalloc_rhs_rejects_meshes_beyond_its_scratch(dg):
    K, P = 9, 3                       # 9^3 (3+1)^3 = 46,656 nodes > 32,768
    N = K ** 3 * (P + 1) ** 3
    q = torch.ones(5 * N, dtype=torch.float64, device="cuda")
    out = torch.empty_like(q)
    with pytest.raises(dg.DGError) as e:
        dg.dg_rhs_noalloc(K, P, 1600.0, 0.1, 0.71, 0, 0, q, out)
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    assert "32768" in str(e.value)
