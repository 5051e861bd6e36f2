"""Element-layer domain decomposition on one GPU: the slabs of a mesh (dg_create_part)
advanced together by dg_group_rk3_step, which moves their face traces between the slabs'
buffers by device copies, against the whole-mesh path (the same arithmetic per node, so
bitwise equal in both precisions) and the FP64 oracle; a slab that spans the mesh with an
exchange function written in Python (the callback path a multi-rank run uses); the
combined diagnostics; argument checks."""
import numpy as np
import pytest

from oracle import dgsem, physics
from paper_2207_11571_gb300 import inputs, partition

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    from tests.libbuild import ensure_built
    ensure_built()
    from paper_2207_11571_gb300 import dg as _dg
    _dg.lib()
    return _dg


class Slabs:
    def __init__(self, dg, K, P, nparts, Re=1600.0, Mach=0.1, les=False, precision=0):
        self.dg, self.K, self.n = dg, K, P + 1
        self.bounds = partition.slab_bounds(K, nparts)
        self.parts = [dg.dg_create_part(K, P, Re, Mach, 0.71, int(les), zb, zc, precision=precision)
                      for zb, zc in self.bounds]

    def scatter(self, q):
        return [partition.local_from_global(q, self.K, self.n, zb, zc) for zb, zc in self.bounds]

    def gather(self, qs):
        return torch.cat([partition.owned_part(q, self.K, self.n, zc) for q, (_, zc) in zip(qs, self.bounds)],
                         dim=1).reshape(-1)

    def close(self):
        for c in self.parts:
            self.dg.dg_destroy(c)


def tgv(dg, ctx, N, seed=inputs.TGV_SEED, eps=1e-6):
    q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
    dg.dg_init_tgv(ctx, q, torch.from_numpy(inputs.perturbation((5, N), seed=seed, eps=eps).ravel()).cuda())
    return q


# (K, P, precision, slabs): rows at P2/P3, the streamed high-order kernel at P6/P8, uneven
# slabs (6 layers in 4), one slab spanning the mesh (its own neighbour)
GROUPS = [(4, 3, 1, 2), (4, 3, 0, 3), (3, 6, 1, 2), (2, 8, 1, 2), (6, 2, 1, 4), (4, 3, 1, 1), (3, 6, 0, 3)]


@pytest.mark.parametrize("K,P,prec,nparts", GROUPS)
def test_group_rk3_steps_equal_the_whole_mesh_bitwise(dg, K, P, prec, nparts):
    whole = dg.dg_create(K, P, 1600.0, 0.1, 0.71, 0, precision=prec)
    s = Slabs(dg, K, P, nparts, precision=prec)
    try:
        N = dg.dg_sizes(whole)[0]
        q = tgv(dg, whole, N, eps=1e-3)
        qs = s.scatter(q)
        dt = dg.dg_stable_dt(whole, q, 0.7)
        dg.dg_rk3_step(whole, q, dt, 3)
        dg.dg_group_rk3_step(s.parts, qs, dt, 3)
        torch.cuda.synchronize()
        got = s.gather(qs)
        assert torch.isfinite(got).all()
        assert torch.equal(got, q), (got - q).abs().max().item()
    finally:
        s.close()
        dg.dg_destroy(whole)


@pytest.mark.parametrize("K,P,nparts,rough", [(4, 3, 3, False), (3, 6, 2, False), (4, 2, 2, True), (3, 3, 3, True)])
def test_group_rhs_fp64_matches_oracle(dg, K, P, nparts, rough):
    """Rough per-node states make every interface jump, the slab boundaries included."""
    from tests.test_gpu_dg import assert_fp64_parity
    Re, Mach, les = (50.0, 0.3, True) if rough else (1600.0, 0.1, False)
    flow = physics.Flow(Re=Re, Mach=Mach, les=les)
    mesh = dgsem.Mesh(K, P)
    n = P + 1
    if rough:
        q_or = inputs.random_conserved((K,) * 3 + (n,) * 3, seed=400 + P, rhoE=(1 / (1.4 * 0.09) / 0.4, 1.0))
    else:
        q_or = dgsem.tgv_state(mesh, flow, inputs.perturbation((5, K ** 3 * n ** 3)))
    s = Slabs(dg, K, P, nparts, Re=Re, Mach=Mach, les=les)
    try:
        q = torch.from_numpy(np.ascontiguousarray(q_or.reshape(5, -1))).cuda().reshape(-1)
        qs = s.scatter(q)
        outs = [torch.full_like(x, float("nan")) for x in qs]
        dg.dg_group_rhs(s.parts, qs, outs)
        torch.cuda.synchronize()
        R = s.gather(outs).cpu().numpy().reshape(q_or.shape)
        assert_fp64_parity(R, q_or, mesh, flow)
    finally:
        s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_group_diagnostics_equal_the_whole_mesh(dg, prec):
    K, P = 4, 3
    whole = dg.dg_create(K, P, 1600.0, 0.1, 0.71, 0, precision=prec)
    s = Slabs(dg, K, P, 3, precision=prec)
    try:
        N = dg.dg_sizes(whole)[0]
        q = tgv(dg, whole, N, eps=1e-3)
        qs = s.scatter(q)
        d = dg.dg_diagnostics(whole, q)
        g = dg.dg_group_diagnostics(s.parts, qs)
        for k in ("mass", "energy", "ke", "dke_dt"):
            assert g[k] == pytest.approx(d[k], rel=1e-13), k
        np.testing.assert_allclose(g["momentum"], d["momentum"], rtol=0, atol=1e-13)
        assert g["max_wave"] == d["max_wave"] and g["nonfinite"] == 0
    finally:
        s.close()
        dg.dg_destroy(whole)


def test_slab_init_and_layout(dg):
    K, P = 4, 3
    whole = dg.dg_create(K, P, 1600.0, 0.1, 0.71, 0)
    s = Slabs(dg, K, P, 3)
    try:
        N = dg.dg_sizes(whole)[0]
        q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
        dg.dg_init_tgv(whole, q)
        for c, (zb, zc) in zip(s.parts, s.bounds):
            nl = dg.dg_sizes(c)[0]
            assert nl == (zc + 2) * K * K * (P + 1) ** 3
            assert dg.dg_part_layout(c) == (zb, zc, K * K * (P + 1) ** 3, zc * K * K * (P + 1) ** 3)
            ql = torch.empty(5 * nl, dtype=torch.float64, device="cuda")
            dg.dg_init_tgv(c, ql)   # every local layer from the global coordinates, ghosts included
            assert torch.equal(ql, partition.local_from_global(q, K, P + 1, zb, zc))
        assert dg.dg_part_layout(whole) == (0, K, 0, N)
        assert dg.dg_part_trace_bytes(s.parts[0], 0) == 5 * 8 * K * K * (P + 1) ** 2
        assert dg.dg_part_trace_bytes(s.parts[0], 2) == 9 * 8 * K * K * (P + 1) ** 2
    finally:
        s.close()
        dg.dg_destroy(whole)


def test_single_slab_with_a_python_exchange_function(dg):
    """The callback path of a multi-rank run, on one rank: a slab spanning the mesh whose
    exchange function (partition.SlabExchange, torch tensors over the library's buffers on
    the library's stream) is its own neighbour; equal to the whole mesh, two exchanges per
    RK stage, diagnostics through the same function."""
    K, P = 4, 3
    whole = dg.dg_create(K, P, 1600.0, 0.1, 0.71, 0, precision=1)
    slab = dg.dg_create_part(K, P, 1600.0, 0.1, 0.71, 0, 0, K, precision=1)
    try:
        calls = []
        ex = partition.SlabExchange(slab, 0, 1)
        inner = ex._call

        def counting(*a):
            calls.append(a[1])
            return inner(*a)

        ex._fn = dg.EXCHANGE_FN(counting)
        dg.dg_part_set_exchange(slab, ex._fn)
        N = dg.dg_sizes(whole)[0]
        q = tgv(dg, whole, N, eps=1e-3)
        ql = partition.local_from_global(q, K, P + 1, 0, K)
        dt = dg.dg_stable_dt(whole, q, 0.7)
        dg.dg_rk3_step(whole, q, dt, 2)
        dg.dg_rk3_step(slab, ql, dt, 2)
        torch.cuda.synchronize()
        assert ex.error is None
        assert calls == [0, 2, 1, 2, 1, 2] * 2     # FP32: state, then increments; phase B data
        assert torch.equal(partition.owned_part(ql, K, P + 1, K).reshape(-1), q)
        d, g = dg.dg_diagnostics(whole, q), dg.dg_diagnostics(slab, ql)
        assert g["ke"] == pytest.approx(d["ke"], rel=1e-14) and g["dke_dt"] == pytest.approx(d["dke_dt"], rel=1e-13)
        # a failing exchange function is reported, and the call returns
        bad = dg.EXCHANGE_FN(lambda *a: 3)
        dg.dg_part_set_exchange(slab, bad)
        with pytest.raises(dg.DGError) as e:
            dg.dg_rk3_step(slab, ql, dt, 1)
        assert e.value.status == dg.DG_ERR_EXCHANGE
    finally:
        dg.dg_destroy(slab)
        dg.dg_destroy(whole)


def test_slab_argument_checks(dg):
    K, P = 4, 3
    with pytest.raises(dg.DGError) as e:
        dg.dg_create_part(K, P, 1600.0, 0.1, 0.71, 0, 3, 2)           # layers beyond K
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    with pytest.raises(dg.DGError) as e:
        dg.dg_create_part(K, P, 1600.0, 0.1, 0.71, 0, 0, 2, block_shape=1)
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    s = Slabs(dg, K, P, 2)
    try:
        qs = [torch.zeros(5 * dg.dg_sizes(c)[0], dtype=torch.float64, device="cuda") for c in s.parts]
        with pytest.raises(dg.DGError) as e:                          # a slab alone, no exchange function
            dg.dg_rk3_step(s.parts[0], qs[0], 1e-3, 1)
        assert e.value.status == dg.DG_ERR_INVALID_ARG
        with pytest.raises(dg.DGError) as e:                          # slabs out of order
            dg.dg_group_rk3_step(s.parts[::-1], qs[::-1], 1e-3, 1)
        assert e.value.status == dg.DG_ERR_INVALID_ARG
        with pytest.raises(dg.DGError) as e:                          # not covering the mesh
            dg.dg_group_rk3_step(s.parts[:1], qs[:1], 1e-3, 1)
        assert e.value.status == dg.DG_ERR_INVALID_ARG
    finally:
        s.close()


def test_autotuned_slabs_still_equal_the_whole_mesh(dg):
    """dg_autotune on a slab times its kernels without exchanging traces (on a scratch
    copy) and only changes the blocking: the group's steps stay equal to the whole mesh's."""
    K, P = 4, 3
    whole = dg.dg_create(K, P, 1600.0, 0.1, 0.71, 0, precision=1)
    s = Slabs(dg, K, P, 2, precision=1)
    try:
        N = dg.dg_sizes(whole)[0]
        q = tgv(dg, whole, N, eps=1e-3)
        qs = s.scatter(q)
        dt = dg.dg_stable_dt(whole, q, 0.7)
        for c, x in zip(s.parts, qs):
            before = x.clone()
            E, ms = dg.dg_autotune(c, x, dt)
            assert E >= 1 and ms > 0 and torch.equal(x, before)
            assert dg.dg_blocking(c)[1] == 0          # rows: slabs take no cube blocks
        dg.dg_rk3_step(whole, q, dt, 2)
        dg.dg_group_rk3_step(s.parts, qs, dt, 2)
        torch.cuda.synchronize()
        assert torch.equal(s.gather(qs), q)
    finally:
        s.close()
        dg.dg_destroy(whole)
