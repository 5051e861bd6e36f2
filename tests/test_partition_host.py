"""Element-layer domain decomposition on CPU: the slab arithmetic, the point-to-point
exchange of the slabs' traces over gloo ranks (world sizes 2 and 3), the locality the
decomposition rests on (the oracle's operator on a slab plus two ghost layers per side
equals the whole mesh's), the oracle advanced by RK3 on gloo ranks that exchange their
ghost layers every stage, and the host-side combination of the slabs' diagnostics."""
import os
import socket
import sys

import numpy as np
import pytest

from oracle import dgsem, physics
from paper_2207_11571_gb300 import inputs, partition

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(target, ws, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=target, args=(r, ws, port, q) + args) for r in range(ws)]
    for p in procs:
        p.start()
    # results first: a rank that put a large item on the queue exits only once it is read
    res = [q.get(timeout=300) for _ in range(ws)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    return sorted(res, key=lambda r: r[0])


def test_slab_bounds_cover_the_mesh_evenly():
    for K in (1, 4, 7, 16, 32):
        for n in range(1, K + 1):
            b = partition.slab_bounds(K, n)
            assert len(b) == n and b[0][0] == 0
            assert all(a + c == b2[0] for (a, c), b2 in zip(b, b[1:]))
            assert sum(c for _, c in b) == K and max(c for _, c in b) - min(c for _, c in b) <= 1
    with pytest.raises(ValueError):
        partition.slab_bounds(4, 5)
    assert partition.local_layers(8, 0, 3) == [7, 0, 1, 2, 3]
    assert partition.local_layers(8, 6, 2) == [5, 6, 7, 0]
    assert partition.neighbours(0, 3) == (2, 1) and partition.neighbours(2, 3) == (1, 0)


def test_local_state_and_owned_part_round_trip():
    K, n = 4, 3
    q = torch.arange(5 * K ** 3 * n ** 3, dtype=torch.float64)
    for zb, zc in partition.slab_bounds(K, 3):
        loc = partition.local_from_global(q, K, n, zb, zc)
        assert loc.numel() == 5 * (zc + 2) * K * K * n ** 3
        own = partition.owned_part(loc, K, n, zc)
        want = q.reshape(5, K, -1)[:, zb:zb + zc].reshape(5, -1)
        assert torch.equal(own, want)
        ghosts = loc.reshape(5, zc + 2, -1)
        assert torch.equal(ghosts[:, 0], q.reshape(5, K, -1)[:, (zb - 1) % K])
        assert torch.equal(ghosts[:, -1], q.reshape(5, K, -1)[:, (zb + zc) % K])


def _exchange_worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2207_11571_gb300 import partition as part
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        n = 37
        send_lo = torch.full((n,), 10.0 * rank + 1)
        send_hi = torch.full((n,), 10.0 * rank + 2)
        recv_lo, recv_hi = torch.zeros(n), torch.zeros(n)
        for _ in range(3):   # repeated exchanges stay matched
            part.exchange_with_peers(send_lo, send_hi, recv_lo, recv_hi, rank, ws)
        out.put((rank, float(recv_lo[0]), float(recv_hi[0]), bool((recv_lo == recv_lo[0]).all()),
                 bool((recv_hi == recv_hi[0]).all())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_exchange_delivers_each_neighbours_traces(ws):
    """recv_lo holds the lower neighbour's send_hi, recv_hi the upper neighbour's send_lo
    (periodic); with two ranks both neighbours are the same rank."""
    for rank, lo, hi, lo_uniform, hi_uniform in run_ranks(_exchange_worker, ws):
        lower, upper = (rank - 1) % ws, (rank + 1) % ws
        assert lo == 10.0 * lower + 2 and hi == 10.0 * upper + 1
        assert lo_uniform and hi_uniform


def test_single_rank_exchange_is_its_own_neighbour():
    a, b = torch.tensor([1.0, 2.0]), torch.tensor([3.0, 4.0])
    rl, rh = torch.zeros(2), torch.zeros(2)
    partition.exchange_with_peers(a, b, rl, rh, 0, 1)
    assert torch.equal(rl, b) and torch.equal(rh, a)


def slab_rhs(q_pad, mesh, flow):
    """The oracle operator on a slab padded with two ghost layers per side, owned part."""
    return dgsem.rhs(q_pad, mesh, flow)[:, 2:-2]


@pytest.mark.parametrize("nslabs", [2, 4])
def test_oracle_on_slabs_with_two_ghost_layers_equals_the_whole_mesh(nslabs):
    """The operator at an element reads elements at most two face steps away (the
    interface flux reads the neighbour's lifted gradient, which reads the neighbour's
    neighbour): the oracle on each slab plus two ghost layers per side gives the whole
    mesh's operator on the slab (rough per-node states, so every interface jumps)."""
    K, P = 4, 2
    flow = physics.Flow(Re=50.0, Mach=0.3, les=True)
    mesh = dgsem.Mesh(K, P)
    q = inputs.random_conserved((K,) * 3 + (P + 1,) * 3, seed=5, rhoE=(1 / (1.4 * 0.09) / 0.4, 1.0))
    R = dgsem.rhs(q, mesh, flow)
    for zb, zc in partition.slab_bounds(K, nslabs):
        layers = [(zb - 2 + i) % K for i in range(zc + 4)]
        Rs = slab_rhs(np.take(q, layers, axis=1), mesh, flow)
        np.testing.assert_allclose(Rs, R[:, zb:zb + zc], rtol=0, atol=1e-14 * np.abs(R).max())


def _oracle_rk3_worker(rank, ws, port, out, K, P, steps):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from oracle import dgsem as dgs
    from oracle import physics as phys
    from paper_2207_11571_gb300 import inputs as inp
    from paper_2207_11571_gb300 import partition as part
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        flow = phys.Flow(Re=1600.0, Mach=0.1)
        mesh = dgs.Mesh(K, P)
        q = dgs.tgv_state(mesh, flow, inp.perturbation((5, K ** 3 * (P + 1) ** 3), eps=1e-3))
        zb, zc = part.slab_bounds(K, ws)[rank]
        own = q[:, zb:zb + zc].copy()

        def rhs(z):
            # every stage: the two boundary layers of each side go to the neighbours
            send_lo = torch.from_numpy(np.ascontiguousarray(z[:, :2])).reshape(-1)
            send_hi = torch.from_numpy(np.ascontiguousarray(z[:, -2:])).reshape(-1)
            recv_lo, recv_hi = torch.empty_like(send_lo), torch.empty_like(send_hi)
            part.exchange_with_peers(send_lo, send_hi, recv_lo, recv_hi, rank, ws)
            shape = (5, 2) + z.shape[2:]
            pad = np.concatenate([recv_lo.numpy().reshape(shape), z, recv_hi.numpy().reshape(shape)], axis=1)
            return dgs.rhs(pad, mesh, flow)[:, 2:-2]

        for _ in range(steps):
            own = dgs.rk3_step(own, 2e-3, rhs)
        out.put((rank, zb, own))
    finally:
        dist.destroy_process_group()


def test_oracle_rk3_on_gloo_ranks_with_ghost_exchange_equals_whole_mesh():
    """Two ranks each advance their slab of the Taylor-Green state by the oracle's RK3,
    exchanging two ghost layers per side through partition.exchange_with_peers before
    every stage: the slabs reassemble the whole-mesh oracle run."""
    K, P, steps = 4, 2, 2
    res = run_ranks(_oracle_rk3_worker, 2, K, P, steps)
    flow = physics.Flow(Re=1600.0, Mach=0.1)
    mesh = dgsem.Mesh(K, P)
    q = dgsem.tgv_state(mesh, flow, inputs.perturbation((5, K ** 3 * (P + 1) ** 3), eps=1e-3))
    for _ in range(steps):
        q = dgsem.rk3_step(q, 2e-3, lambda z: dgsem.rhs(z, mesh, flow))
    whole = np.concatenate([r[2] for r in res], axis=1)
    assert [r[1] for r in res] == [0, 2]
    np.testing.assert_allclose(whole, q, rtol=1e-14, atol=0)


def test_diag_combine_sums_in_order_and_takes_maxima():
    """dg_diag_combine (host code of the library, no GPU): sums of the integrals, maxima
    of e_inf and the wave speed, non-finite counts added and reported."""
    from tests.libbuild import ensure_built
    ensure_built()
    from paper_2207_11571_gb300 import dg
    parts = [{"mass": 1.0 + i, "momentum": [0.1 * i, -0.2, 0.3], "energy": 10.0 * i, "ke": 0.01 * (i + 1),
              "dke_dt": -1e-3 * i, "e_inf": [i, 3 - i, 0.5], "max_wave": 11.0 + (i % 2), "nonfinite": 0}
             for i in range(3)]
    d = dg.dg_diag_combine(parts)
    assert d["mass"] == 6.0 and d["energy"] == 30.0 and d["ke"] == pytest.approx(0.06, rel=1e-15)
    assert d["momentum"] == pytest.approx([0.3, -0.6, 0.9], rel=1e-15)
    assert d["dke_dt"] == pytest.approx(-3e-3, rel=1e-15)
    assert d["e_inf"] == [2.0, 3.0, 0.5] and d["max_wave"] == 12.0 and d["nonfinite"] == 0
    parts[1]["nonfinite"] = 2
    with pytest.raises(dg.DGError) as e:
        dg.dg_diag_combine(parts)
    assert e.value.status == dg.DG_ERR_NONFINITE
    assert dg.dg_diag_combine(parts, raise_nonfinite=False)["nonfinite"] == 2


def _dp_worker(rank, ws, port, q, shards, steps):
    """Rank `rank` holds rows shards[rank] of the batch and runs dp_train_step with the
    oracle MLP: its gradients normalised over the global batch, summed over ranks."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from oracle import mlp
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        X, T, params, scalers = _dp_problem()
        rows = np.asarray(shards[rank])
        mean_in, std_in, mean_out, std_out = scalers
        xs, ts = (X[rows] - mean_in) / std_in, (T[rows] - mean_out) / std_out
        state, cur, losses = {}, [params], []
        holder = {}

        def backward(global_batch):
            y, cache = mlp.forward(cur[0], xs)
            diff = y - ts
            g = mlp.backward(cur[0], cache, 2.0 * diff / (global_batch * diff.shape[1]))
            holder["g"] = [torch.from_numpy(np.ascontiguousarray(a)) for gw, gb in g for a in (gw, gb)]
            return float((diff ** 2).sum() / (global_batch * diff.shape[1]))

        def apply():
            t = [a.numpy() for a in holder["g"]]
            cur[0] = mlp.adam_step(cur[0], [(t[2 * i], t[2 * i + 1]) for i in range(len(cur[0]))], state)

        for _ in range(steps):
            losses.append(partition.dp_train_step(backward, lambda: holder["g"], apply, len(rows)))
        q.put((rank, [(W.copy(), b.copy()) for W, b in cur[0]], losses))
    finally:
        dist.destroy_process_group()


def _dp_problem():
    from oracle import mlp
    dims = mlp.layer_dims(12, 12, 16, 2)
    params = mlp.he_uniform_init(dims, inputs.uniform_draws(dims, 31))
    X = inputs.normal((10, 12), 32)
    T = inputs.normal((10, 12), 33)
    scalers = (X.mean(0), X.std(0), T.mean(0), T.std(0))
    return X, T, params, scalers


@pytest.mark.parametrize("shards", [[range(0, 5), range(5, 10)], [range(0, 2), range(2, 9), range(9, 10)]])
def test_data_parallel_training_equals_the_whole_batch(shards):
    """Ranks holding uneven parts of a batch, each normalising its MSE gradient over the
    global batch and summing the gradients over ranks, take the whole batch's Adam steps:
    the parameters (identical on every rank) and the losses equal the oracle's
    single-process train_step on all rows (FP64, to rounding of the reduction order)."""
    from oracle import mlp
    steps = 3
    res = run_ranks(_dp_worker, len(shards), [list(s) for s in shards], steps)
    X, T, params, scalers = _dp_problem()
    state, ref_losses = {}, []
    for _ in range(steps):
        params, loss, _ = mlp.train_step(params, state, scalers, X, T)
        ref_losses.append(loss)
    for rank, got, losses in res:
        for (W, b), (Wr, br) in zip(got, params):
            np.testing.assert_allclose(W, Wr, rtol=0, atol=1e-12)
            np.testing.assert_allclose(b, br, rtol=0, atol=1e-12)
        np.testing.assert_allclose(losses, ref_losses, rtol=1e-12)
    for (_, a, _), (_, b, _) in zip(res, res[1:]):   # the same bits on every rank
        assert all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) for x, y in zip(a, b))
