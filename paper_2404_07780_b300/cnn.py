"""The learned initialiser: a small CNN that predicts starting parameters for
the LM fit from a galaxy stamp.

The paper starts every fit from hand-set values and names that as a
limitation, citing convolutional networks that estimate galaxy parameters
(arxiv 2404.07780, Sec. 1 and Sec. 6).  This module builds such a network on
the library's own BF16 tensor-core layers (include/gm_cnn.h), trains it on the
GPU on stamps rendered by gm_model, and turns its predictions into starting
points for gm_fit_batch; the default-start fit stays the fallback.

Architecture (input: the stamp's 2x2 block mean, asinh-scaled by the sky
noise, 64 x 64 x 1):
    conv 3x3/2  1 -> 32, ReLU   (32 x 32)
    conv 3x3/2 32 -> 64, ReLU   (16 x 16)
    conv 3x3/2 64 -> 128, ReLU  ( 8 x  8)
    conv 3x3/2 128 -> 128, ReLU ( 4 x  4)
    dense 2048 -> 256, ReLU
    dense 256 -> 16 (FP32; the first `dv` outputs are the normalised targets)
BF16 weights and activations, FP32 accumulation, FP32 master weights and Adam
moments.  This module only marshals arguments and orders the layer calls:
every step runs in the library's kernels.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from . import gm as _gm


class CNNError(RuntimeError):
    pass


_cnn = None


def lib():
    global _cnn
    if _cnn is None:
        L = _gm.load()
        P, S, I, F = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_float
        L.gm_cnn_last_error.restype = ctypes.c_char_p
        L.gm_cnn_last_error.argtypes = []
        L.gm_cnn_check_error.restype = I
        L.gm_cnn_check_error.argtypes = [P]
        L.gm_cnn_conv_fwd.restype = I
        L.gm_cnn_conv_fwd.argtypes = [P, P, P, P, I, I, I, I, I, I, P]
        L.gm_cnn_conv_bwd_data.restype = I
        L.gm_cnn_conv_bwd_data.argtypes = [P, P, P, P, I, I, I, I, I, P]
        L.gm_cnn_conv_bwd_weight_workspace.restype = S
        L.gm_cnn_conv_bwd_weight_workspace.argtypes = [I, I, I, I, I]
        L.gm_cnn_conv_bwd_weight.restype = I
        L.gm_cnn_conv_bwd_weight.argtypes = [P, P, P, P, I, I, I, I, I, P, S, P]
        L.gm_cnn_dense_fwd.restype = I
        L.gm_cnn_dense_fwd.argtypes = [P, P, P, P, P, I, I, I, I, P]
        L.gm_cnn_dense_bwd_data.restype = I
        L.gm_cnn_dense_bwd_data.argtypes = [P, P, P, P, I, I, I, P]
        L.gm_cnn_dense_bwd_weight_workspace.restype = S
        L.gm_cnn_dense_bwd_weight_workspace.argtypes = [I, I, I]
        L.gm_cnn_dense_bwd_weight.restype = I
        L.gm_cnn_dense_bwd_weight.argtypes = [P, P, P, P, I, I, I, P, S, P]
        L.gm_cnn_prep.restype = I
        L.gm_cnn_prep.argtypes = [P, I, I, I, F, P, P]
        L.gm_cnn_mse.restype = I
        L.gm_cnn_mse.argtypes = [P, P, I, I, I, P, P, P]
        L.gm_cnn_adam.restype = I
        L.gm_cnn_adam.argtypes = [P, P, P, P, P, ctypes.c_longlong, F, F, F, F, I, P]
        _cnn = L
    return _cnn


EXPORTS = ("gm_cnn_last_error", "gm_cnn_check_error", "gm_cnn_conv_fwd", "gm_cnn_conv_bwd_data",
           "gm_cnn_conv_bwd_weight_workspace", "gm_cnn_conv_bwd_weight", "gm_cnn_dense_fwd", "gm_cnn_dense_bwd_data",
           "gm_cnn_dense_bwd_weight_workspace", "gm_cnn_dense_bwd_weight", "gm_cnn_prep", "gm_cnn_mse", "gm_cnn_adam")


def _check(rc, what):
    if rc != 0:
        raise CNNError(f"{what} failed ({rc}): {lib().gm_cnn_last_error().decode()}")


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, dtype, name):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise CNNError(f"{name} must be a contiguous {dtype} CUDA tensor")
    return t


# ---------------------------------------------------------------------------
# layer calls (shapes as in include/gm_cnn.h)
# ---------------------------------------------------------------------------

def conv_fwd(x, w, b, relu=True):
    """x [n,h,w,ci] bf16, w [co,3,3,ci] bf16, b [co] f32 -> y [n,(h+1)/2,(w+1)/2,co] bf16."""
    import torch
    bf, f32 = torch.bfloat16, torch.float32
    n, h, wd, ci = x.shape
    co = w.shape[0]
    y = torch.empty((n, (h + 1) // 2, (wd + 1) // 2, co), dtype=bf, device=x.device)
    _check(lib().gm_cnn_conv_fwd(_p(_need(x, bf, "x")), _p(_need(w, bf, "w")), _p(_need(b, f32, "b")), _p(y), n, h,
                                 wd, ci, co, int(relu), _stream()), "gm_cnn_conv_fwd")
    return y


def conv_bwd_data(dy, w, h, wd, mask=None):
    import torch
    bf = torch.bfloat16
    n, ho, wo, co = dy.shape
    ci = w.shape[3]
    dx = torch.empty((n, h, wd, ci), dtype=bf, device=dy.device)
    _check(lib().gm_cnn_conv_bwd_data(_p(_need(dy, bf, "dy")), _p(_need(w, bf, "w")), _p(_need(mask, bf, "mask")),
                                      _p(dx), n, h, wd, ci, co, _stream()), "gm_cnn_conv_bwd_data")
    return dx


def conv_bwd_weight(x, dy, ws=None):
    """(dw [co,3,3,ci] f32, db [co] f32)."""
    import torch
    bf, f32 = torch.bfloat16, torch.float32
    n, h, wd, ci = x.shape
    co = dy.shape[3]
    dw = torch.empty((co, 3, 3, ci), dtype=f32, device=x.device)
    db = torch.empty(co, dtype=f32, device=x.device)
    nbytes = lib().gm_cnn_conv_bwd_weight_workspace(n, h, wd, ci, co)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=x.device)
    _check(lib().gm_cnn_conv_bwd_weight(_p(_need(x, bf, "x")), _p(_need(dy, bf, "dy")), _p(dw), _p(db), n, h, wd, ci,
                                        co, _p(ws), ws.numel(), _stream()), "gm_cnn_conv_bwd_weight")
    return dw, db


def dense_fwd(x, w, b, relu=True, fp32_out=False):
    import torch
    bf, f32 = torch.bfloat16, torch.float32
    n, fin = x.shape
    fout = w.shape[0]
    y = torch.empty((n, fout), dtype=f32 if fp32_out else bf, device=x.device)
    _check(lib().gm_cnn_dense_fwd(_p(_need(x, bf, "x")), _p(_need(w, bf, "w")), _p(_need(b, f32, "b")),
                                  None if fp32_out else _p(y), _p(y) if fp32_out else None, n, fin, fout, int(relu),
                                  _stream()), "gm_cnn_dense_fwd")
    return y


def dense_bwd_data(dy, w, mask=None):
    import torch
    bf = torch.bfloat16
    n, fout = dy.shape
    fin = w.shape[1]
    dx = torch.empty((n, fin), dtype=bf, device=dy.device)
    _check(lib().gm_cnn_dense_bwd_data(_p(_need(dy, bf, "dy")), _p(_need(w, bf, "w")), _p(_need(mask, bf, "mask")),
                                       _p(dx), n, fin, fout, _stream()), "gm_cnn_dense_bwd_data")
    return dx


def dense_bwd_weight(x, dy, ws=None):
    import torch
    bf, f32 = torch.bfloat16, torch.float32
    n, fin = x.shape
    fout = dy.shape[1]
    dw = torch.empty((fout, fin), dtype=f32, device=x.device)
    db = torch.empty(fout, dtype=f32, device=x.device)
    nbytes = lib().gm_cnn_dense_bwd_weight_workspace(n, fin, fout)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=x.device)
    _check(lib().gm_cnn_dense_bwd_weight(_p(_need(x, bf, "x")), _p(_need(dy, bf, "dy")), _p(dw), _p(db), n, fin,
                                         fout, _p(ws), ws.numel(), _stream()), "gm_cnn_dense_bwd_weight")
    return dw, db


def prep(image, scale):
    """image [G,h,w] f32 -> [G,h/2,w/2,1] bf16 = asinh(scale * 2x2 mean)."""
    import torch
    G, h, wd = image.shape
    out = torch.empty((G, h // 2, wd // 2, 1), dtype=torch.bfloat16, device=image.device)
    _check(lib().gm_cnn_prep(_p(_need(image, torch.float32, "image")), G, h, wd, float(scale), _p(out), _stream()),
           "gm_cnn_prep")
    return out


def mse(pred, target, dv):
    """(loss [1] f32 device tensor, dpred [n,d] bf16)."""
    import torch
    n, d = pred.shape
    loss = torch.empty(1, dtype=torch.float32, device=pred.device)
    dpred = torch.empty((n, d), dtype=torch.bfloat16, device=pred.device)
    _check(lib().gm_cnn_mse(_p(_need(pred, torch.float32, "pred")), _p(_need(target, torch.float32, "target")), n, d,
                            dv, _p(loss), _p(dpred), _stream()), "gm_cnn_mse")
    return loss, dpred


def adam(param, grad, m, v, param_bf16, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(lib().gm_cnn_adam(_p(param), _p(grad), _p(m), _p(v), _p(param_bf16), param.numel(), float(lr),
                             float(beta1), float(beta2), float(eps), int(step), _stream()), "gm_cnn_adam")


def check_device_error():
    flag = ctypes.c_int(0)
    _check(lib().gm_cnn_check_error(ctypes.byref(flag)), "gm_cnn_check_error")
    if flag.value:
        raise CNNError("a CNN kernel gave up waiting for its tensor-core work")
