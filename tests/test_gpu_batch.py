"""Batches of independent solvers (dg_create_batch / dg_batch_rk3_step): every member
must come out as if it had been advanced alone by dg_rk3_step (bit-identical in the FP32
operator, to a rounding of the state in FP64), with the graph replay and with direct
launches, across re-recordings (new dt) and autotuning; the FP64 batch also matches the
oracle.  Members mix orders, meshes (ragged element blocks),
Reynolds numbers and the LES closure, the shape of a sweep of small flows."""
import numpy as np
import pytest

from oracle import dgsem, physics
from paper_2207_11571_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (K, P, Re, Mach, Pr, closure): orders 3, 4 and 6 with several meshes, Re in {30, 200, 1600}
MEMBERS = [(3, 3, 30.0, 0.1, 0.71, 0), (2, 6, 200.0, 0.1, 0.71, 0), (4, 3, 1600.0, 0.1, 0.71, 1),
           (2, 3, 200.0, 0.1, 0.71, 0), (3, 6, 1600.0, 0.1, 0.71, 0), (5, 3, 1600.0, 0.1, 0.71, 0),
           (3, 4, 200.0, 0.1, 0.71, 1)]


@pytest.fixture(scope="module")
def dg():
    from tests.libbuild import ensure_built
    ensure_built()
    from paper_2207_11571_gb300 import dg as _dg
    _dg.lib()
    return _dg


def init_states(dg, b, members):
    qs = []
    for i, (K, P, *_rest) in enumerate(members):
        N = K ** 3 * (P + 1) ** 3
        q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
        pert = inputs.perturbation((5, N), seed=inputs.TGV_SEED + i)
        dg.dg_init_tgv(dg.dg_batch_member(b, i), q, torch.from_numpy(pert.ravel()).cuda())
        qs.append(q)
    return qs


def alone(dg, b, qs, dts, nsteps):
    out = [q.clone() for q in qs]
    for i, q in enumerate(out):
        dg.dg_rk3_step(dg.dg_batch_member(b, i), q, dts[i], nsteps)
    return out


def assert_same(got, ref, prec, what):
    """FP32 operator: bit-identical.  FP64 operator: the batched kernels are separate
    compilations of the same source and may contract a multiply-add differently, so the
    results may differ by a rounding of the state (observed: 1 ulp of rho e ~ 179)."""
    if prec == 1:
        assert torch.equal(got, ref), what
    else:
        d = (got - ref).abs().max().item()
        assert d <= 4e-16 * ref.abs().max().item(), (what, d)


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_members_advanced_alone(dg, prec):
    b = dg.dg_create_batch(MEMBERS, precision=prec)
    try:
        qs = init_states(dg, b, MEMBERS)
        dts = [dg.dg_stable_dt(dg.dg_batch_member(b, i), q, 0.7) for i, q in enumerate(qs)]
        ref = alone(dg, b, qs, dts, 3)
        graph = [q.clone() for q in qs]
        dg.dg_batch_rk3_step(b, graph, dts, 3)
        direct = [q.clone() for q in qs]
        dg.dg_batch_rk3_step(b, direct, dts, 3, flags=dg.DG_BATCH_NO_GRAPH)
        torch.cuda.synchronize()
        for i in range(len(MEMBERS)):
            assert torch.equal(graph[i], direct[i]), i      # graph replay = direct launches
            assert_same(graph[i], ref[i], prec, i)
        # new step sizes: the step is recorded again
        dts2 = [0.5 * d for d in dts]
        ref2 = alone(dg, b, graph, dts2, 2)
        dg.dg_batch_rk3_step(b, graph, dts2, 2)
        torch.cuda.synchronize()
        for i in range(len(MEMBERS)):
            assert_same(graph[i], ref2[i], prec, i)
    finally:
        dg.dg_batch_destroy(b)


def test_batch_autotune_changes_no_result(dg):
    b = dg.dg_create_batch(MEMBERS, precision=1)
    try:
        qs = init_states(dg, b, MEMBERS)
        dts = [dg.dg_stable_dt(dg.dg_batch_member(b, i), q, 0.7) for i, q in enumerate(qs)]
        before = [q.clone() for q in qs]
        dg.dg_batch_rk3_step(b, before, dts, 2)
        dg.dg_batch_autotune(b, qs, dts)
        after = [q.clone() for q in qs]
        dg.dg_batch_rk3_step(b, after, dts, 2)
        torch.cuda.synchronize()
        for i in range(len(MEMBERS)):
            assert torch.equal(after[i], before[i]), i   # the block partition changes no arithmetic
    finally:
        dg.dg_batch_destroy(b)


def test_batch_fp64_matches_oracle(dg):
    members = [(2, 3, 200.0, 0.1, 0.71, 0), (2, 4, 1600.0, 0.1, 0.71, 1)]
    b = dg.dg_create_batch(members, precision=0)
    try:
        qs = init_states(dg, b, members)
        dts = [1e-3, 7e-4]
        q0 = [q.cpu().numpy().reshape(5, -1) for q in qs]
        dg.dg_batch_rk3_step(b, qs, dts, 2)
        torch.cuda.synchronize()
        for i, (K, P, Re, Mach, Pr, les) in enumerate(members):
            mesh = dgsem.Mesh(K, P)
            flow = physics.Flow(Re=Re, Mach=Mach, Pr=Pr, les=bool(les))
            n = P + 1
            ref = q0[i].reshape(5, K, K, K, n, n, n)
            for _ in range(2):
                ref = dgsem.rk3_step(ref, dts[i], lambda z: dgsem.rhs(z, mesh, flow))
            got = qs[i].cpu().numpy().reshape(ref.shape)
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err < 1e-13, (i, err)
    finally:
        dg.dg_batch_destroy(b)


def test_borrowed_member_cannot_be_destroyed(dg):
    b = dg.dg_create_batch(MEMBERS[:2])
    try:
        with pytest.raises(dg.DGError) as e:
            dg.dg_destroy(dg.dg_batch_member(b, 0))
        assert e.value.status == dg.DG_ERR_INVALID_ARG
        with pytest.raises(dg.DGError):
            dg.dg_batch_member(b, 2)
    finally:
        dg.dg_batch_destroy(b)


def test_batch_rejects_shared_states(dg):
    members = [(2, 3, 200.0, 0.1, 0.71, 0)] * 2
    b = dg.dg_create_batch(members)
    try:
        qs = init_states(dg, b, members)
        with pytest.raises(dg.DGError) as e:
            dg.dg_batch_rk3_step(b, [qs[0], qs[0]], [1e-3, 1e-3], 1)
        assert e.value.status == dg.DG_ERR_INVALID_ARG
    finally:
        dg.dg_batch_destroy(b)


def test_persistent_stage_launch_equals_members_advanced_alone(dg):
    """DG_BATCH_PERSISTENT: each RK stage of every member (orders 3, 4 and 6 together) is
    one cooperative launch with a grid barrier between the gradient and flux phases.  The
    per-element arithmetic is the single-mesh kernels', so the members come out as if
    advanced alone by dg_rk3_step, within a rounding of the increments (the streamed
    high-order kernel and the row kernel may contract a multiply-add differently); graph
    replay equals direct launches bitwise."""
    b = dg.dg_create_batch(MEMBERS, precision=1)
    try:
        qs = init_states(dg, b, MEMBERS)
        dts = [dg.dg_stable_dt(dg.dg_batch_member(b, i), q, 0.7) for i, q in enumerate(qs)]
        ref = alone(dg, b, qs, dts, 3)
        graph = [q.clone() for q in qs]
        dg.dg_batch_rk3_step(b, graph, dts, 3, flags=dg.DG_BATCH_PERSISTENT)
        direct = [q.clone() for q in qs]
        dg.dg_batch_rk3_step(b, direct, dts, 3, flags=dg.DG_BATCH_PERSISTENT | dg.DG_BATCH_NO_GRAPH)
        torch.cuda.synchronize()
        for i in range(len(MEMBERS)):
            assert torch.isfinite(graph[i]).all(), i
            assert torch.equal(graph[i], direct[i]), i
            incr = (ref[i] - qs[i]).abs().max().item()
            d = (graph[i] - ref[i]).abs().max().item()
            assert d <= 1e-5 * incr, (i, d, incr)
        for i in range(len(MEMBERS)):   # the barrier's error flag stayed clear
            dg.dg_diagnostics(dg.dg_batch_member(b, i), graph[i])
    finally:
        dg.dg_batch_destroy(b)


def test_persistent_stage_launch_refuses_what_it_does_not_run(dg):
    b = dg.dg_create_batch(MEMBERS[:2], precision=0)          # FP64 operator
    try:
        qs = init_states(dg, b, MEMBERS[:2])
        with pytest.raises(dg.DGError) as e:
            dg.dg_batch_rk3_step(b, qs, [1e-3, 1e-3], 1, flags=dg.DG_BATCH_PERSISTENT)
        assert e.value.status == dg.DG_ERR_UNSUPPORTED
    finally:
        dg.dg_batch_destroy(b)
    members = [(2, 8, 200.0, 0.1, 0.71, 0), (2, 3, 200.0, 0.1, 0.71, 0)]
    b = dg.dg_create_batch(members, precision=1)              # order 8
    try:
        qs = init_states(dg, b, members)
        with pytest.raises(dg.DGError) as e:
            dg.dg_batch_rk3_step(b, qs, [1e-3, 1e-3], 1, flags=dg.DG_BATCH_PERSISTENT)
        assert e.value.status == dg.DG_ERR_UNSUPPORTED
    finally:
        dg.dg_batch_destroy(b)
