"""Thin Python binding of the forcing-network part of libdgnn.so (include/dgnn_nn.h)."""


def _register(L):
    """Declares the C signatures of the network entry points present in the library."""
    return L
