"""Surrogate-network layer calls on torch tensors (argument marshalling
only; the arithmetic runs in the library's BF16 tensor-core kernels, see
include/fdtd_mlp.h).  Tensors must be contiguous CUDA tensors."""
from __future__ import annotations

import ctypes

from . import _lib

ACT_NONE, ACT_GELU = 0, 1


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc, what):
    if rc != 0:
        raise _lib.FdtdError(rc, what)


def forward(x, wt, bias, act, y_bf16=None, y_f32=None, z_f32=None):
    import torch
    lib = _lib.load()
    rows, k = x.shape
    n = wt.shape[0]
    _check(lib.fdtd_mlp_forward(_p(x), int(x.dtype == torch.bfloat16), rows, k, _p(wt), _p(bias), n, act,
                                _p(y_bf16), _p(y_f32), _p(z_f32), _stream()), "mlp_forward")


def backward(x, z, dy, wt, act, dz, dw=None, db=None, dx=None):
    import torch
    lib = _lib.load()
    rows, k = x.shape
    n = dy.shape[1]
    _check(lib.fdtd_mlp_backward(_p(x), int(x.dtype == torch.bfloat16), _p(z), _p(dy), rows, k, n, act, _p(wt),
                                 _p(dz), _p(dw), _p(db), _p(dx), _stream()), "mlp_backward")


def adam(w, m, v, g, w_bf16, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    lib = _lib.load()
    _check(lib.fdtd_mlp_adam(_p(w), _p(m), _p(v), _p(g), _p(w_bf16), w.numel(), lr, beta1, beta2, eps,
                             weight_decay, int(t), _stream()), "mlp_adam")


def mse(y, target, scale, dy, loss, row_weight=None):
    lib = _lib.load()
    rows, cols = y.shape
    _check(lib.fdtd_mlp_mse(_p(y), _p(target), _p(row_weight), rows, cols, scale, _p(dy), _p(loss), _stream()),
           "mlp_mse")


def row_rel_err(y, target, err):
    lib = _lib.load()
    rows, cols = y.shape
    _check(lib.fdtd_mlp_row_rel_err(_p(y), _p(target), rows, cols, _p(err), _stream()), "mlp_row_rel_err")


def gather_rows(src, idx, dst):
    lib = _lib.load()
    _check(lib.fdtd_mlp_gather_rows(_p(src), _p(idx), idx.numel(), src.shape[1], _p(dst), _stream()),
           "mlp_gather_rows")


def scale_rows(y, scale):
    lib = _lib.load()
    rows, cols = y.shape
    _check(lib.fdtd_mlp_scale_rows(_p(y), _p(scale), rows, cols, _stream()), "mlp_scale_rows")


def to_bf16(src, dst):
    lib = _lib.load()
    _check(lib.fdtd_mlp_to_bf16(_p(src), _p(dst), src.numel(), _stream()), "mlp_to_bf16")


def check():
    """synchronise the current stream; raise if a bounded wait inside a
    network kernel ran out since the last check"""
    _check(_lib.load().fdtd_mlp_check(_stream()), "mlp kernels")


def _ints(v):
    return (ctypes.c_int * len(v))(*[int(a) for a in v])


def net_pack_bytes(sizes):
    """bytes of the packed weight image of a network with these layer sizes"""
    lib = _lib.load()
    n = ctypes.c_size_t(0)
    _check(lib.fdtd_mlp_net_pack_bytes(_ints(sizes), len(sizes) - 1, ctypes.byref(n)), "mlp_net_pack_bytes")
    return n.value


def net_pack(sizes, wts, image):
    """pack the BF16 weights wts[l] [sizes[l+1], sizes[l]] into image (a
    uint8 CUDA tensor of net_pack_bytes(sizes) bytes)"""
    lib = _lib.load()
    L = len(sizes) - 1
    ptrs = (ctypes.c_void_p * L)(*[w.data_ptr() for w in wts])
    _check(lib.fdtd_mlp_net_pack(_ints(sizes), L, ptrs, _p(image), _stream()), "mlp_net_pack")


def net_forward(x, sizes, acts, image, biases, y, out_scale=1.0):
    """y = the whole network on x (FP32 [rows, sizes[0]]) in one launch;
    y FP32 [rows, sizes[-1]]"""
    lib = _lib.load()
    L = len(sizes) - 1
    bp = (ctypes.c_void_p * L)(*[(b.data_ptr() if b is not None else None) for b in biases])
    _check(lib.fdtd_mlp_net_forward(_p(x), x.shape[0], _ints(sizes), L, _ints(acts), _p(image), bp,
                                    float(out_scale), _p(y), _stream()), "mlp_net_forward")
