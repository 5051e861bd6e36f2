"""Thin Python binding of the forcing network in libdgnn.so (C ABI in include/dgnn_nn.h).

Same names as the C entry points; arguments are marshalled (tensors to device
pointers, numpy arrays to host pointers) and statuses raised as ``DGError``.
"""
import ctypes

import numpy as np


class nn_desc(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int), ("n_out", ctypes.c_int), ("width", ctypes.c_int),
                ("n_hidden", ctypes.c_int), ("first_var", ctypes.c_int), ("n_vars", ctypes.c_int),
                ("max_batch", ctypes.c_int)]


class nn_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "nn_create": [ctypes.POINTER(nn_desc), _P, ctypes.POINTER(_P)],
    "nn_destroy": [_P],
    "nn_set_scalers": [_P, _P, _P, _P, _P],
    "nn_get_scalers": [_P, _P, _P, _P, _P],
    "nn_compute_scalers": [_P, _P, _P, ctypes.c_int64, _P],
    "nn_forward": [_P, _P, _P, _I, _P],
    "nn_set_fused": [_P, _I],
    "nn_forcing_infer": [_P, _P, _P, _P, _P],
    "nn_train_step": [_P, _P, _P, _P, _I, ctypes.POINTER(nn_adam), ctypes.POINTER(ctypes.c_float), _P],
    "nn_get_params": [_P, _I, _P, _P],
    "nn_set_params": [_P, _I, _P, _P],
    "nn_get_grads": [_P, _I, _P, _P],
    "nn_backward": [_P, _P, _P, _P, _I, _I, ctypes.POINTER(ctypes.c_float), _P],
    "nn_grad_buffers": [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P)],
    "nn_adam_apply": [_P, ctypes.POINTER(nn_adam), _P],
    "nn_get_desc": [_P, ctypes.POINTER(nn_desc)],
    "nn_save": [_P, ctypes.c_char_p],
    "nn_load": [ctypes.c_char_p, _I, ctypes.POINTER(_P)],
    "nn_gemm_bf16": [_I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P],
}


def _register(L):
    for name, args in _SIGS.items():
        f = getattr(L, name, None)
        if f is None:
            continue
        f.argtypes = args
        f.restype = ctypes.c_int
    return L


def _dg():
    from . import dg
    return dg


def _h(net):
    return ctypes.c_void_p(net)


def layer_dims(desc):
    return [desc.n_in] + [desc.width] * desc.n_hidden + [desc.n_out]


def nn_create(n_in, n_out, width, n_hidden, first_var=0, n_vars=5, max_batch=4096, init_uniform=None):
    """Returns an opaque handle.  init_uniform: list of U(-1,1) arrays (out, in) per layer, or None."""
    dg = _dg()
    d = nn_desc(n_in, n_out, width, n_hidden, first_var, n_vars, max_batch)
    flat = None
    if init_uniform is not None:
        flat = np.ascontiguousarray(np.concatenate([np.asarray(a, np.float32).ravel() for a in init_uniform]))
        if flat.size != sum(a * b for a, b in zip(layer_dims(d)[:-1], layer_dims(d)[1:])):
            raise ValueError("init_uniform does not match the layer shapes")
    h = ctypes.c_void_p()
    dg.check(dg.lib().nn_create(ctypes.byref(d), dg.ptr(flat), ctypes.byref(h)))
    return h.value


def nn_destroy(net):
    dg = _dg()
    dg.check(dg.lib().nn_destroy(_h(net)))


def nn_get_desc(net):
    dg = _dg()
    d = nn_desc()
    dg.check(dg.lib().nn_get_desc(_h(net), ctypes.byref(d)))
    return d


def _check_rows(t, width, name, rows=None, dtype="float32"):
    """A CUDA tensor of ``rows`` rows (its first dimension if None) of ``width`` values
    of ``dtype``; returns the row count.  The kernels index the rows without bounds of
    their own, so a wrong size is refused here."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor")
    if str(t.dtype).split(".")[-1] != dtype:
        raise TypeError(f"{name} must be {dtype}")
    r = int(t.shape[0]) if rows is None else int(rows)
    if t.numel() != r * width:
        raise ValueError(f"{name} must hold {r} rows of {width} values, got {t.numel()} values")
    return r


def nn_set_scalers(net, mean_in, std_in, mean_out, std_out):
    dg = _dg()
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (mean_in, std_in, mean_out, std_out)]
    dg.check(dg.lib().nn_set_scalers(_h(net), *[dg.ptr(a) for a in arrs]))


def nn_get_scalers(net):
    dg = _dg()
    d = nn_get_desc(net)
    out = [np.zeros(n, np.float32) for n in (d.n_in, d.n_in, d.n_out, d.n_out)]
    dg.check(dg.lib().nn_get_scalers(_h(net), *[dg.ptr(a) for a in out]))
    return tuple(out)


def nn_compute_scalers(net, X, Y, stream=None):
    dg = _dg()
    d = nn_get_desc(net)
    rows = _check_rows(X, d.n_in, "X")
    _check_rows(Y, d.n_out, "Y", rows)
    dg.check(dg.lib().nn_compute_scalers(_h(net), dg.ptr(X), dg.ptr(Y), rows, dg.stream_ptr(stream)))


def nn_forward(net, X, S, stream=None):
    dg = _dg()
    d = nn_get_desc(net)
    rows = _check_rows(X, d.n_in, "X")
    _check_rows(S, d.n_out, "S", rows)
    dg.check(dg.lib().nn_forward(_h(net), dg.ptr(X), dg.ptr(S), rows, dg.stream_ptr(stream)))


NN_INFER_LAYERS, NN_INFER_FUSED, NN_INFER_CLUSTER = 0, 1, 2


def nn_set_fused(net, mode=NN_INFER_FUSED):
    """Inference path: NN_INFER_CLUSTER (the default: the forcing of a solver state in one
    cluster launch), NN_INFER_FUSED (one fused kernel of 128 rows per CTA) or
    NN_INFER_LAYERS (one GEMM per layer).  True / False select FUSED / LAYERS."""
    if mode is True or mode is False:
        mode = NN_INFER_FUSED if mode else NN_INFER_LAYERS
    dg = _dg()
    dg.check(dg.lib().nn_set_fused(_h(net), int(mode)))


def nn_forcing_infer(net, ctx, q, s, stream=None):
    dg = _dg()
    dg._check_state(ctx, q, "q")
    _check_rows(s, nn_get_desc(net).n_vars * dg.dg_sizes(ctx)[0], "s", rows=1)
    dg.check(dg.lib().nn_forcing_infer(_h(net), ctypes.c_void_p(ctx), dg.ptr(q), dg.ptr(s), dg.stream_ptr(stream)))


def nn_train_step(net, X, Y, idx=None, batch=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-7, want_loss=True,
                  stream=None):
    """One Adam step on rows idx of (X, Y) (all rows if idx is None).  The values of idx
    must lie in [0, rows of X): they are not read back to the host to check."""
    dg = _dg()
    d = nn_get_desc(net)
    rows = _check_rows(X, d.n_in, "X")
    _check_rows(Y, d.n_out, "Y", rows)
    if idx is not None:
        _check_rows(idx, idx.numel(), "idx", rows=1, dtype="int64")
    if batch is None:
        batch = int(idx.numel()) if idx is not None else rows
    if batch > (idx.numel() if idx is not None else rows):
        raise ValueError(f"batch {batch} exceeds the rows available ({rows} rows of X, idx of "
                         f"{None if idx is None else idx.numel()})")
    hp = nn_adam(lr, beta1, beta2, eps)
    loss = ctypes.c_float()
    dg.check(dg.lib().nn_train_step(_h(net), dg.ptr(X), dg.ptr(Y), dg.ptr(idx), int(batch), ctypes.byref(hp),
                                    ctypes.byref(loss) if want_loss else None, dg.stream_ptr(stream)))
    return loss.value if want_loss else None


def nn_backward(net, X, Y, idx=None, batch=None, global_batch=None, want_loss=True, stream=None):
    """Gradients of the MSE of rows idx of (X, Y) into the network's gradient buffers,
    normalised over global_batch rows (default: this batch); returns this call's share of
    the loss.  No parameter changes (nn_adam_apply does the update)."""
    dg = _dg()
    d = nn_get_desc(net)
    rows = _check_rows(X, d.n_in, "X")
    _check_rows(Y, d.n_out, "Y", rows)
    if idx is not None:
        _check_rows(idx, idx.numel(), "idx", rows=1, dtype="int64")
    if batch is None:
        batch = int(idx.numel()) if idx is not None else rows
    if batch > (idx.numel() if idx is not None else rows):
        raise ValueError(f"batch {batch} exceeds the rows available")
    if global_batch is None:
        global_batch = batch
    loss = ctypes.c_float()
    dg.check(dg.lib().nn_backward(_h(net), dg.ptr(X), dg.ptr(Y), dg.ptr(idx), int(batch), int(global_batch),
                                  ctypes.byref(loss) if want_loss else None, dg.stream_ptr(stream)))
    return loss.value if want_loss else None


class _DeviceFloats:
    """FP32 device memory of the library seen by torch (CUDA array interface, no copy)."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(int(n) for n in shape), "typestr": "<f4",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def nn_grad_buffers(net, layer):
    """(dW [out][in], db [out]): torch views of layer `layer`'s gradient buffers on the
    device (no copy), owned by the network; valid until nn_destroy."""
    import torch
    dg = _dg()
    o, i = _layer_shape(net, layer)
    pw, pb = ctypes.c_void_p(), ctypes.c_void_p()
    dg.check(dg.lib().nn_grad_buffers(_h(net), int(layer), ctypes.byref(pw), ctypes.byref(pb)))
    return (torch.as_tensor(_DeviceFloats(pw.value, (o, i)), device="cuda"),
            torch.as_tensor(_DeviceFloats(pb.value, (o,)), device="cuda"))


def nn_adam_apply(net, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-7, stream=None):
    """One Adam step of every parameter from the gradient buffers."""
    dg = _dg()
    hp = nn_adam(lr, beta1, beta2, eps)
    dg.check(dg.lib().nn_adam_apply(_h(net), ctypes.byref(hp), dg.stream_ptr(stream)))


def _layer_shape(net, layer):
    dims = layer_dims(nn_get_desc(net))
    return dims[layer + 1], dims[layer]


def nn_get_params(net, layer):
    dg = _dg()
    o, i = _layer_shape(net, layer)
    W, b = np.zeros((o, i), np.float32), np.zeros(o, np.float32)
    dg.check(dg.lib().nn_get_params(_h(net), int(layer), dg.ptr(W), dg.ptr(b)))
    return W, b


def nn_set_params(net, layer, W, b):
    dg = _dg()
    W = np.ascontiguousarray(W, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    dg.check(dg.lib().nn_set_params(_h(net), int(layer), dg.ptr(W), dg.ptr(b)))


def nn_get_grads(net, layer):
    dg = _dg()
    o, i = _layer_shape(net, layer)
    dW, db = np.zeros((o, i), np.float32), np.zeros(o, np.float32)
    dg.check(dg.lib().nn_get_grads(_h(net), int(layer), dg.ptr(dW), dg.ptr(db)))
    return dW, db


def nn_save(net, path):
    dg = _dg()
    dg.check(dg.lib().nn_save(_h(net), str(path).encode()))


def nn_load(path, max_batch=4096):
    dg = _dg()
    h = ctypes.c_void_p()
    dg.check(dg.lib().nn_load(str(path).encode(), int(max_batch), ctypes.byref(h)))
    return h.value


def nn_gemm_bf16(A, B, bias=None, relu=False, K=None, stream=None):
    """C = A[:, :K] B[:, :K]^T (+ bias, ReLU) for row-major bf16 CUDA tensors A (M x lda) and
    B (N x ldb); K defaults to A's width.  Returns float32 C (M x N)."""
    import torch
    dg = _dg()
    M = A.shape[0]
    K = A.shape[1] if K is None else int(K)
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    dg.check(dg.lib().nn_gemm_bf16(M, N, K, dg.ptr(A), A.stride(0), dg.ptr(B), B.stride(0), dg.ptr(bias),
                                   int(bool(relu)), dg.ptr(C), N, dg.stream_ptr(stream)))
    return C
