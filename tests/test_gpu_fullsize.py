"""Parity at the benchmark's full sizes, in the benchmark's launch configuration.

Meshes 32^3/P3, 16^3/P6 and 16^3/P8 (Re 1600, Mach 0.1), FP32 operator with the
elements-per-block the autotuner picks (the streamed phase-B kernel at P >= 6), and the
FP64 operator.  The oracle cannot evaluate these meshes whole in test time, so it is
checked on sampled elements: the operator at element e depends only on the states of
elements at most two face steps away (the Roe/BR1 interface flux of e reads its face
neighbours' states and lifted gradients, and a neighbour's gradient reads that
neighbour's face neighbours), so the oracle evaluates a 5 x 5 x 5 block of elements
centred on e, cut from the full state and closed periodically (the wrap only touches
elements three steps away), with the full mesh's element size h.  Inputs come from the
oracle's own Taylor-Green field plus the seeded perturbation.  Properties that hold at
any size (conservation over RK3 steps) are checked on the whole mesh."""
import numpy as np
import pytest

from oracle import dgsem, physics
from paper_2207_11571_gb300 import inputs
from tests import fp32_bounds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MESHES = [(32, 3), (16, 6), (16, 8)]


@pytest.fixture(scope="module")
def dg():
    from tests.libbuild import ensure_built
    ensure_built()
    from paper_2207_11571_gb300 import dg as _dg
    _dg.lib()
    return _dg


def samples(K):
    """(ez, ey, ex) of the sampled elements: corners of the periodic cube, block edges,
    interior, and seeded random picks."""
    fixed = [(0, 0, 0), (K - 1, K - 1, K - 1), (K // 2, 1, K - 2), (3, K - 1, 7 % K), (K // 3, K // 2, 0)]
    rng = np.random.default_rng(K)
    return fixed + [tuple(int(v) for v in rng.integers(0, K, 3)) for _ in range(7)]


def patch_state(q, K, centre):
    """The 5^3 block of elements around one element, cut from the full state."""
    idx = [[(c - 2 + i) % K for i in range(5)] for c in centre]
    return np.take(np.take(np.take(q, idx[0], axis=1), idx[1], axis=2), idx[2], axis=3)


def patch_mesh(mesh, dtype=np.float64):
    mp = dgsem.Mesh(5, mesh.P)
    mp.h = mesh.h
    if dtype != np.float64:   # the same FP64 tables, evaluated in extended precision
        mp.w, mp.xi, mp.D = (np.asarray(a, dtype) for a in (mp.w, mp.xi, mp.D))
        mp.h = dtype(mesh.h)
    return mp


def patch_rhs(q, mesh, flow, centre, dtype=np.float64):
    """Oracle operator at one element from the 5^3 block of elements around it."""
    qp = np.asarray(patch_state(q, mesh.K, centre), dtype)
    return dgsem.rhs(qp, patch_mesh(mesh, dtype), flow)[:, 2, 2, 2]


@pytest.fixture(scope="module")
def cases():
    """Full-size oracle input states and the oracle operator at the sampled elements."""
    out = {}
    flow = physics.Flow(Re=1600.0, Mach=0.1, Pr=0.71)
    for K, P in MESHES:
        mesh = dgsem.Mesh(K, P)
        n = P + 1
        N = K ** 3 * n ** 3
        q = dgsem.tgv_state(mesh, flow, inputs.perturbation((5, N)))
        ref = {s: patch_rhs(q, mesh, flow, s) for s in samples(K)}
        out[(K, P)] = (q, ref)
    return out


def gpu_rhs(dg, K, P, q, precision):
    c = dg.dg_create(K, P, 1600.0, 0.1, 0.71, 0, precision=precision)
    try:
        qd = torch.from_numpy(np.ascontiguousarray(q.reshape(5, -1))).cuda().reshape(-1)
        if precision == dg.DG_PREC_FP32:
            dg.dg_autotune(c, qd, dg.dg_stable_dt(c, qd, 0.7))   # the benchmark's launch configuration
        R = torch.empty_like(qd)
        dg.dg_rhs(c, qd, R)
        torch.cuda.synchronize()
        n = P + 1
        return R.cpu().numpy().reshape(5, K, K, K, n, n, n)
    finally:
        dg.dg_destroy(c)


@pytest.mark.parametrize("K,P", MESHES)
def test_fp32_operator_at_full_size_matches_oracle_on_sampled_elements(dg, cases, K, P):
    q, ref = cases[(K, P)]
    R = gpu_rhs(dg, K, P, q, dg.DG_PREC_FP32)
    got = np.stack([R[:, ez, ey, ex] for ez, ey, ex in ref])
    want = np.stack(list(ref.values()))
    fp32_bounds.check(f"fullsize K{K} P{P}", got, want, axis_vars=1)


def rel_l2(a, b):
    a = np.asarray(a, np.longdouble)
    b = np.asarray(b, np.longdouble)
    return float(np.sqrt(np.sum((a - b) ** 2)) / np.sqrt(np.sum(b ** 2)))


@pytest.mark.parametrize("K,P", MESHES)
def test_fp64_operator_at_full_size_matches_oracle_on_sampled_elements(dg, cases, K, P):
    """FP64 parity bar of the operator tests: 1e-12 relative L2 against the FP64 oracle, or,
    where the FP64 arithmetic floor of the case itself exceeds 1e-12 (Mach 0.1, the
    background pressure and energy cancel in the derivatives), the GPU no farther from the
    extended-precision oracle than the FP64 oracle is (x 1.5), on the same sampled
    elements."""
    q, ref = cases[(K, P)]
    R = gpu_rhs(dg, K, P, q, dg.DG_PREC_FP64)
    got = np.stack([R[:, ez, ey, ex] for ez, ey, ex in ref])
    want = np.stack(list(ref.values()))
    direct = rel_l2(got, want)
    if direct < 1e-12:
        return
    flow = physics.Flow(Re=1600.0, Mach=0.1, Pr=0.71)
    mesh = dgsem.Mesh(K, P)
    ext = np.stack([patch_rhs(q, mesh, flow, s, np.longdouble) for s in ref])
    e_gpu, e_or = rel_l2(got, ext), rel_l2(want, ext)
    assert e_or > 1e-12 and e_gpu <= 1.5 * e_or, (direct, e_gpu, e_or)


@pytest.mark.parametrize("K,P", MESHES)
def test_full_size_rk3_steps_conserve_mass_momentum_energy(dg, cases, K, P):
    """Two RK3 steps of the FP32 operator in the benchmark configuration: the periodic DGSEM
    conserves the integrals of all five variables (to FP32 rounding of the increments)."""
    q, _ = cases[(K, P)]
    c = dg.dg_create(K, P, 1600.0, 0.1, 0.71, 0, precision=dg.DG_PREC_FP32)
    try:
        qd = torch.from_numpy(np.ascontiguousarray(q.reshape(5, -1))).cuda().reshape(-1)
        dt = dg.dg_stable_dt(c, qd, 0.7)
        dg.dg_autotune(c, qd, dt)
        d0 = dg.dg_diagnostics(c, qd)
        dg.dg_rk3_step(c, qd, dt, 2)
        d1 = dg.dg_diagnostics(c, qd)
        vol = 8 * np.pi ** 3
        assert abs(d1["mass"] - d0["mass"]) < 1e-10 * vol
        assert abs(d1["energy"] - d0["energy"]) < 1e-10 * abs(d0["energy"])
        for i in range(3):
            assert abs(d1["momentum"][i] - d0["momentum"][i]) < 1e-9 * vol
        assert d1["ke"] < d0["ke"]   # the decaying flow loses kinetic energy
    finally:
        dg.dg_destroy(c)
