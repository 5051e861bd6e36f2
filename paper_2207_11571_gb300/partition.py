"""Element-layer domain decomposition of the periodic K^3 mesh over ranks.

The paper runs its solver in parallel over MPI ranks (Sec. 2.6, implementation details).
Here every rank (one GPU each) owns a slab of whole element layers along z and a
library context made by ``dg_create_part``; each RK stage exchanges the face traces of
the slabs' boundary layers twice (see ``dg_exchange_fn`` in include/dgnn.h).  This
module holds the host side of that arrangement: which layers a rank owns, how a global
state maps to a slab's local arrays, and the point-to-point exchange of one slab's
trace buffers with its two neighbours through ``torch.distributed`` (NCCL on GPUs; the
same function runs on CPU tensors with gloo).  Nothing here computes any part of the
method: the operator, the traces and their packing run in the library's kernels.
"""
import ctypes

from . import dg


def slab_bounds(K, nranks):
    """(z_begin, z_count) of every rank: layers [K r / n, K (r + 1) / n), as even as
    possible; every rank owns at least one layer (nranks <= K)."""
    if not 1 <= nranks <= K:
        raise ValueError(f"{nranks} ranks cannot each own a layer of {K}")
    edges = [K * r // nranks for r in range(nranks + 1)]
    return [(a, b - a) for a, b in zip(edges, edges[1:])]


def neighbours(rank, nranks):
    """Ranks owning the layers below and above (periodic)."""
    return (rank - 1) % nranks, (rank + 1) % nranks


def local_layers(K, z_begin, z_count):
    """Global element layers of a slab's local layers 0 .. z_count + 1 (ghosts first and
    last)."""
    return [(z_begin - 1 + i) % K for i in range(z_count + 2)]


def local_from_global(q, K, n, z_begin, z_count):
    """The local state of a slab (5, (z_count + 2) K^2 n^3) from a global state
    (5 K^3 n^3 values, layout [var][elem][node]), ghost layers included."""
    import torch
    layers = torch.tensor(local_layers(K, z_begin, z_count), device=q.device)
    g = q.reshape(5, K, K * K * n ** 3)
    return g.index_select(1, layers).reshape(-1).contiguous()


def owned_part(q_local, K, n, z_count):
    """The owned layers of a slab's local state, shape (5, z_count K^2 n^3)."""
    per_layer = K * K * n ** 3
    return q_local.reshape(5, z_count + 2, per_layer)[:, 1:z_count + 1].reshape(5, -1)


def exchange_with_peers(send_lo, send_hi, recv_lo, recv_hi, rank, nranks, group=None):
    """One slab's exchange: send_hi goes to the rank above (its recv_lo), send_lo to the
    rank below (its recv_hi).  Tag 0 carries the upward, tag 1 the downward traces, and
    both ranks post their operations in the same order, so that with two ranks (whose
    lower and upper neighbour coincide) each message finds its buffer.  One rank: the
    slab is its own neighbour."""
    if nranks == 1:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return
    import torch.distributed as dist
    lower, upper = neighbours(rank, nranks)
    ops = [dist.P2POp(dist.isend, send_hi, upper, group, tag=0),
           dist.P2POp(dist.isend, send_lo, lower, group, tag=1),
           dist.P2POp(dist.irecv, recv_lo, lower, group, tag=0),
           dist.P2POp(dist.irecv, recv_hi, upper, group, tag=1)]
    for w in dist.batch_isend_irecv(ops):
        w.wait()


class _DeviceBytes:
    """A device buffer of the library seen by torch (CUDA array interface, no copy)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class SlabExchange:
    """Installs the exchange function of a slab context: at every exchange point the
    library's trace buffers are handed to ``exchange_with_peers`` on the library's
    stream (torch.distributed, NCCL for CUDA buffers).  Keep the object alive while the
    context is used."""

    def __init__(self, ctx, rank, nranks, group=None):
        self.ctx, self.rank, self.nranks, self.group = ctx, rank, nranks, group
        self.error = None
        self._fn = dg.EXCHANGE_FN(self._call)
        dg.dg_part_set_exchange(ctx, self._fn)

    def _call(self, user, what, send_lo, send_hi, recv_lo, recv_hi, nbytes, stream):
        import torch
        try:
            st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(st):
                t = [torch.as_tensor(_DeviceBytes(p, nbytes), device="cuda")
                     for p in (send_lo, send_hi, recv_lo, recv_hi)]
                exchange_with_peers(*t, self.rank, self.nranks, self.group)
            return 0
        except Exception as e:   # reported to the library as a failed exchange
            self.error = e
            return 1

    def close(self):
        dg.dg_part_set_exchange(self.ctx, None)
        self._fn = ctypes.cast(None, dg.EXCHANGE_FN)


def gather_diagnostics(ctx, q, group=None, q_ref=None):
    """Diagnostics of the whole mesh on every rank: each rank's slab diagnostics, gathered
    and combined in rank order (a fixed-order FP64 sum: the same bits on every rank)."""
    import torch
    import torch.distributed as dist
    d = dg.dg_diagnostics(ctx, q, q_ref=q_ref, raise_nonfinite=False)
    vec = torch.tensor([d["mass"], *d["momentum"], d["energy"], d["ke"], d["dke_dt"], *d["e_inf"],
                        d["max_wave"], float(d["nonfinite"])], dtype=torch.float64,
                       device="cuda" if dist.get_backend(group) == "nccl" else "cpu")
    out = [torch.empty_like(vec) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, vec, group=group)
    parts = []
    for v in out:
        v = v.cpu().tolist()
        parts.append({"mass": v[0], "momentum": v[1:4], "energy": v[4], "ke": v[5], "dke_dt": v[6],
                      "e_inf": v[7:10], "max_wave": v[10], "nonfinite": int(v[11])})
    return dg.dg_diag_combine(parts, raise_nonfinite=False)


# ----------------------------------------------------------------------------- training

def dp_train_step(backward, grads, apply, local_batch, group=None):
    """One data-parallel optimisation step over the ranks of ``group``, each holding
    ``local_batch`` rows of the batch.  The MSE of Sec. 2.2 is a mean over the batch's
    rows, so its gradient is the sum over ranks of each rank's gradient normalised by the
    global row count:

    * ``backward(global_batch)`` computes this rank's share (gradients into the tensors
      ``grads()`` returns, normalised over ``global_batch`` rows) and returns its share of
      the loss;
    * the gradient tensors are summed over the ranks in place (``all_reduce``; every rank
      receives the same sums, so the parameters stay identical on every rank);
    * ``apply()`` takes the optimiser step.

    Returns the loss of the whole batch (the sum of the shares)."""
    import torch
    import torch.distributed as dist
    cpu = dist.get_backend(group) == "gloo"
    dev = "cpu" if cpu else "cuda"
    n = torch.tensor([int(local_batch)], dtype=torch.int64, device=dev)
    dist.all_reduce(n, group=group)
    loss = backward(int(n.item()))
    for t in grads():
        if cpu and t.is_cuda:   # gloo reduces host tensors
            h = t.cpu()
            dist.all_reduce(h, group=group)
            t.copy_(h)
        else:
            dist.all_reduce(t, group=group)
    apply()
    tot = torch.tensor([float(loss)], dtype=torch.float64, device=dev)
    dist.all_reduce(tot, group=group)
    return float(tot.item())


def nn_dp_train_step(net, X, Y, idx=None, batch=None, group=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-7,
                     stream=None):
    """dp_train_step on the library's network: ``nn_backward`` normalised over the global
    batch, an in-place all-reduce of every layer's gradient buffers, ``nn_adam_apply``."""
    from . import nn
    d = nn.nn_get_desc(net)
    if batch is None:
        batch = int(idx.numel()) if idx is not None else int(X.shape[0])
    layers = d.n_hidden + 1

    def bufs():
        out = []
        for layer in range(layers):
            out.extend(nn.nn_grad_buffers(net, layer))
        return out

    return dp_train_step(lambda gb: nn.nn_backward(net, X, Y, idx, batch, gb, stream=stream), bufs,
                         lambda: nn.nn_adam_apply(net, lr, beta1, beta2, eps, stream=stream), batch, group)
