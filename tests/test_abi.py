"""Host-side checks of the C ABI: the library loads, exports every declared symbol,
validates arguments, and its host-built basis matches closed forms and the oracle.
No GPU needed (no device compute is launched)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from tests.libbuild import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    ensure_built()
    from paper_2207_11571_gb300 import dg
    return dg.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*((?:dg|nn)_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("dg_create", "dg_rhs", "dg_rk3_step", "dg_diagnostics", "dg_project", "dg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_opts_defaults(L):
    from paper_2207_11571_gb300 import dg
    o = dg.dg_opts_default()
    assert o.precision == dg.DG_PREC_FP64 and o.gamma == 1.4 and o.Cs == 0.1 and o.Prt == 0.9


@pytest.mark.parametrize("bad", [dict(K=0), dict(K=300), dict(P=0), dict(P=9), dict(Re=-1.0),
                                 dict(Mach=0.0), dict(closure=2), dict(block_shape=2),
                                 dict(block_shape=1, K=5), dict(block_shape=1, P=4), dict(volume_flux=2),
                                 dict(volume_flux=1, block_shape=1), dict(gamma=1.0), dict(gamma=float("inf")),
                                 dict(Cs=-0.1), dict(Cs=float("nan")), dict(Prt=0.0), dict(les_delta=float("nan"))])
def test_create_rejects_bad_arguments_before_touching_cuda(L, bad):
    from paper_2207_11571_gb300 import dg
    args = dict(K=4, P=3, Re=1600.0, Mach=0.1, Pr=0.71, closure=0)
    args.update(bad)
    with pytest.raises(dg.DGError) as e:
        dg.dg_create(**args)
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    assert b"dg_create" in L.dg_last_error()


def test_null_handles_are_rejected(L):
    from paper_2207_11571_gb300 import dg
    assert L.dg_rhs(None, None, None, None, None) == dg.DG_ERR_INVALID_ARG
    assert L.dg_destroy(None) == dg.DG_ERR_INVALID_ARG
    assert L.dg_rk3_step(None, None, 1e-3, 1, None, None) == dg.DG_ERR_INVALID_ARG


@pytest.mark.parametrize("members", [[], [(4, 3, 1600.0, 0.1, 0.71, 0)] * 17, [(4, 9, 1600.0, 0.1, 0.71, 0)],
                                     [(0, 3, 1600.0, 0.1, 0.71, 0), (4, 3, 200.0, 0.1, 0.71, 0)]])
def test_create_batch_rejects_bad_members_before_touching_cuda(L, members):
    from paper_2207_11571_gb300 import dg
    with pytest.raises(dg.DGError) as e:
        dg.dg_create_batch(members)
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    assert b"dg_create" in L.dg_last_error()


def test_batch_rejects_cube_blocks_before_touching_cuda(L):
    from paper_2207_11571_gb300 import dg
    with pytest.raises(dg.DGError) as e:
        dg.dg_create_batch([(4, 3, 1600.0, 0.1, 0.71, 0)], block_shape=1)
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    with pytest.raises(dg.DGError) as e:
        dg.dg_create_batch([(4, 3, 1600.0, 0.1, 0.71, 0)], volume_flux=1)
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    assert L.dg_blocking(None, None, None) == dg.DG_ERR_INVALID_ARG
    assert L.dg_advance_host_async(None, None, 1e-3, 1, None, 0, None) == dg.DG_ERR_INVALID_ARG
    assert L.dg_advance_host_wait(None, None, None) == dg.DG_ERR_INVALID_ARG
    assert L.dg_set_forcing_mode(None, 0) == dg.DG_ERR_INVALID_ARG


def test_batch_calls_reject_null_handles(L):
    from paper_2207_11571_gb300 import dg
    assert L.dg_batch_destroy(None) == dg.DG_ERR_INVALID_ARG
    assert L.dg_batch_rk3_step(None, None, None, 1, 0, None) == dg.DG_ERR_INVALID_ARG
    assert L.dg_batch_member(None, 0, None) == dg.DG_ERR_INVALID_ARG


def test_host_basis_matches_closed_forms_and_oracle(L):
    from oracle import basis
    from paper_2207_11571_gb300 import dg
    xi, w, D = dg.dg_basis_1d(3)
    np.testing.assert_allclose(xi, [-1, -5 ** -0.5, 5 ** -0.5, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-14)
    for P in range(1, 9):
        xi, w, D = dg.dg_basis_1d(P)
        xo, wo = basis.gl_nodes_weights(P)
        np.testing.assert_allclose(xi, xo, atol=2e-15)
        np.testing.assert_allclose(w, wo, rtol=1e-13)
        np.testing.assert_allclose(D, basis.lagrange_derivative_matrix(xo), atol=1e-12 * P * P)


def test_network_bindings_check_rows_dtype_and_device():
    """The nn bindings refuse a tensor of the wrong size, dtype or device before the
    library sees its pointer (the kernels index rows without bounds of their own)."""
    torch = pytest.importorskip("torch")
    from paper_2207_11571_gb300 import nn

    class OnDevice:   # a host tensor standing in for a CUDA one (no GPU here)
        def __init__(self, t):
            self.t, self.is_cuda, self.dtype, self.shape = t, True, t.dtype, t.shape

        def numel(self):
            return self.t.numel()

    assert nn._check_rows(OnDevice(torch.zeros(10, 320)), 320, "X") == 10
    assert nn._check_rows(OnDevice(torch.zeros(7, dtype=torch.int64)), 7, "idx", rows=1, dtype="int64") == 1
    with pytest.raises(ValueError):
        nn._check_rows(OnDevice(torch.zeros(10, 321)), 320, "X")
    with pytest.raises(ValueError):
        nn._check_rows(OnDevice(torch.zeros(9, 320)), 320, "S", rows=10)
    with pytest.raises(TypeError):
        nn._check_rows(OnDevice(torch.zeros(10, 320, dtype=torch.float64)), 320, "X")
    with pytest.raises(ValueError):
        nn._check_rows(torch.zeros(10, 320), 320, "X")          # host tensor


def test_training_calls_reject_bad_arguments_before_touching_cuda(L):
    """The data-parallel training calls check their handles and sizes before any CUDA call."""
    from paper_2207_11571_gb300 import dg, nn
    nn._register(L)
    assert L.nn_backward(None, None, None, None, 1, 1, None, None) == dg.DG_ERR_INVALID_ARG
    dW, db = ctypes.c_void_p(), ctypes.c_void_p()
    assert L.nn_grad_buffers(None, 0, ctypes.byref(dW), ctypes.byref(db)) == dg.DG_ERR_INVALID_ARG
    assert L.nn_adam_apply(None, None, None) == dg.DG_ERR_INVALID_ARG
