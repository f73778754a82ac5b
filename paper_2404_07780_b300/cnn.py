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
        L.gm_cnn_fwd_path.restype = I
        L.gm_cnn_fwd_path.argtypes = [I, I, I, I, I, I, I]
        L.gm_cnn_conv12_fwd.restype = I
        L.gm_cnn_conv12_fwd.argtypes = [P, P, P, P, P, P, I, P]
        L.gm_cnn_test_starve_next.restype = I
        L.gm_cnn_test_starve_next.argtypes = [ctypes.c_uint]
        _cnn = L
    return _cnn


EXPORTS = ("gm_cnn_last_error", "gm_cnn_check_error", "gm_cnn_conv_fwd", "gm_cnn_conv_bwd_data",
           "gm_cnn_conv_bwd_weight_workspace", "gm_cnn_conv_bwd_weight", "gm_cnn_dense_fwd", "gm_cnn_dense_bwd_data",
           "gm_cnn_dense_bwd_weight_workspace", "gm_cnn_dense_bwd_weight", "gm_cnn_prep", "gm_cnn_mse", "gm_cnn_adam",
           "gm_cnn_fwd_path", "gm_cnn_conv12_fwd", "gm_cnn_test_starve_next")

PATH_GATHER, PATH_TMA = 0, 1  # kernels of a forward layer (gm_cnn_fwd_path)


def fwd_path(kind: str, n: int, h: int, w: int, ci: int, co: int, fp32_out: bool = False) -> int:
    """The kernel a forward layer of these sizes runs on: PATH_TMA or PATH_GATHER
    (kind "conv": n x h x w x ci input, co outputs; kind "dense": n rows, ci = fin, co = fout)."""
    rc = lib().gm_cnn_fwd_path(0 if kind == "conv" else 1, n, h, w, ci, co, int(fp32_out))
    if rc < 0:
        raise CNNError(f"fwd_path: sizes refused ({kind} n={n} {h}x{w} ci={ci} co={co})")
    return rc


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


def conv12_fwd(x, w1, b1, w2, b2):
    """The first two convolutions fused (both with ReLU): x [n,64,64,1] bf16 -> [n,16,16,64] bf16."""
    import torch
    bf, f32 = torch.bfloat16, torch.float32
    n = x.shape[0]
    if tuple(x.shape[1:]) != (64, 64, 1) or tuple(w1.shape) != (32, 3, 3, 1) or tuple(w2.shape) != (64, 3, 3, 32):
        raise CNNError("conv12_fwd: the network's first two layers on 64x64x1 inputs only")
    y = torch.empty((n, 16, 16, 64), dtype=bf, device=x.device)
    _check(lib().gm_cnn_conv12_fwd(_p(_need(x, bf, "x")), _p(_need(w1, bf, "w1")), _p(_need(b1, f32, "b1")),
                                   _p(_need(w2, bf, "w2")), _p(_need(b2, f32, "b2")), _p(y), n, _stream()),
           "gm_cnn_conv12_fwd")
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


# ---------------------------------------------------------------------------
# the network
# ---------------------------------------------------------------------------
# (kind, input channels or features, output channels or features); the four
# convolutions halve a 64 x 64 input to 4 x 4
LAYERS = (("conv", 1, 32), ("conv", 32, 64), ("conv", 64, 128), ("conv", 128, 128), ("dense", 2048, 256),
          ("dense", 256, 16))
INPUT_SIDE = 64
OUT = 16  # network outputs; the codec uses the first `dv`


class Net:
    """Parameters in flat FP32 buffers (master weights, gradients, Adam moments) with a BF16
    copy the layers read; layer views into them."""

    def __init__(self, seed: int = 0, device="cuda"):
        import torch
        self.device = torch.device(device)
        shapes = []
        for kind, i, o in LAYERS:
            shapes.append((o, 3, 3, i) if kind == "conv" else (o, i))
            shapes.append((o,))
        sizes = [int(np.prod(s)) for s in shapes]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.shapes = shapes
        n = int(self.offsets[-1])
        self.n_params = n
        rng = np.random.default_rng(seed)
        init = np.zeros(n, np.float32)
        for li, (kind, i, o) in enumerate(LAYERS):
            fan_in = 9 * i if kind == "conv" else i
            std = math.sqrt(2.0 / fan_in) if li < len(LAYERS) - 1 else math.sqrt(1.0 / fan_in)
            a, b = self.offsets[2 * li], self.offsets[2 * li + 1]
            init[a:b] = rng.normal(0.0, std, b - a)
        f32 = dict(dtype=torch.float32, device=self.device)
        self.p = torch.from_numpy(init).to(self.device)
        self.p_bf = self.p.to(torch.bfloat16)
        self.grad = torch.zeros(n, **f32)
        self.m = torch.zeros(n, **f32)
        self.v = torch.zeros(n, **f32)
        self.step_count = 0
        self._ws = None

    def save(self, path) -> None:
        """Checkpoint: FP32 master weights, Adam moments and step count in one .npz file
        (the BF16 copy is rebuilt on load; the target codec depends only on the stamp side)."""
        np.savez(path, p=self.p.cpu().numpy(), m=self.m.cpu().numpy(), v=self.v.cpu().numpy(),
                 step=np.int64(self.step_count), offsets=self.offsets)

    @classmethod
    def load(cls, path, device="cuda") -> "Net":
        """A network restored from save(): training resumes where it stopped."""
        import torch
        z = np.load(path)
        net = cls(device=device)
        if not np.array_equal(z["offsets"], net.offsets):
            raise ValueError(f"{path}: the checkpoint's layer layout differs from this network's")
        for name in ("p", "m", "v"):
            getattr(net, name).copy_(torch.from_numpy(z[name]))
        net.p_bf.copy_(net.p.to(torch.bfloat16))
        net.step_count = int(z["step"])
        return net

    def _view(self, buf, j):
        return buf[int(self.offsets[j]):int(self.offsets[j + 1])].view(self.shapes[j])

    def w(self, li):
        return self._view(self.p_bf, 2 * li)

    def b(self, li):
        return self._view(self.p, 2 * li + 1)

    def forward(self, x):
        """x [n,64,64,1] BF16 -> (activations, prediction [n,16] FP32)."""
        acts = [x]
        a = x
        for li, (kind, i, o) in enumerate(LAYERS):
            last = li == len(LAYERS) - 1
            if kind == "conv":
                a = conv_fwd(a, self.w(li), self.b(li), relu=True)
            else:
                a = a.reshape(a.shape[0], -1)
                a = dense_fwd(a, self.w(li), self.b(li), relu=not last, fp32_out=last)
            acts.append(a)
        return acts, acts[-1]

    def backward(self, acts, dpred):
        """Gradients of the loss (dpred = d loss / d prediction, BF16) into self.grad."""
        import torch
        if self._ws is None:
            nb = acts[0].shape[0]
            need = max(lib().gm_cnn_conv_bwd_weight_workspace(nb, 64, 64, 128, 128),
                       lib().gm_cnn_dense_bwd_weight_workspace(nb, 2048, 256))
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        d = dpred
        for li in range(len(LAYERS) - 1, -1, -1):
            kind, i, o = LAYERS[li]
            x = acts[li]
            if kind == "dense":
                xf = x.reshape(x.shape[0], -1)
                dw, db = dense_bwd_weight(xf, d, ws=self._ws)
                if li > 0:
                    d = dense_bwd_data(d, self.w(li), mask=xf)
            else:
                d4 = d.reshape(x.shape[0], (x.shape[1] + 1) // 2, (x.shape[2] + 1) // 2, o)
                dw, db = conv_bwd_weight(x, d4, ws=self._ws)
                if li > 0:
                    d = conv_bwd_data(d4, self.w(li), x.shape[1], x.shape[2], mask=x)
            self._view(self.grad, 2 * li).copy_(dw)
            self._view(self.grad, 2 * li + 1).copy_(db)

    def adam_step(self, lr):
        self.step_count += 1
        adam(self.p, self.grad, self.m, self.v, self.p_bf, lr, self.step_count)

    def train_step(self, x, target, dv, lr):
        """One forward, loss, backward and Adam step; returns the loss (a device scalar)."""
        acts, pred = self.forward(x)
        loss, dpred = mse(pred, target, dv)
        self.backward(acts, dpred)
        self.adam_step(lr)
        return loss

    def infer(self, x):
        """Prediction [n,16] FP32 without keeping activations: the first two convolutions run
        fused (their result equals forward()'s bit for bit), the rest layer by layer."""
        a = conv12_fwd(x, self.w(0), self.b(0), self.w(1), self.b(1))
        for li in range(2, len(LAYERS)):
            kind, i, o = LAYERS[li]
            last = li == len(LAYERS) - 1
            if kind == "conv":
                a = conv_fwd(a, self.w(li), self.b(li), relu=True)
            else:
                a = dense_fwd(a.reshape(a.shape[0], -1), self.w(li), self.b(li), relu=not last, fp32_out=last)
        return a

    def predict(self, x, batch: int = 16384):
        import torch
        out = torch.empty((x.shape[0], OUT), dtype=torch.float32, device=x.device)
        for s in range(0, x.shape[0], batch):
            out[s:s + batch] = self.infer(x[s:s + batch].contiguous())
        return out


# ---------------------------------------------------------------------------
# targets: the bulge + disk + sky parameters as normalised network outputs
# ---------------------------------------------------------------------------

@dataclass
class BulgeDiskCodec:
    """Maps the 13 slots of synth.bulge_disk_sky (bulge x0 y0 q pa Ie Re n, disk q pa I0 rs n,
    sky) to 14 outputs of order one and back: the centre offset from the stamp centre / 2 px,
    q, log10 of the amplitudes, ln of the radii, n and the sky scaled by their prior ranges,
    and each position angle as (cos 2 pa, sin 2 pa) (period pi).  Ranges are those of
    synth.draw_uneven_bulge_disk at stamp side `side`."""
    side: int = 128

    dv = 14

    def _ranges(self):
        f = self.side / 96.0
        reb = (1.5 * f, 8 * f)
        return {"qb": (0.3, 1.0), "lie": (0.5, 3.0), "lreb": (math.log(reb[0]), math.log(reb[1])), "nb": (1.0, 6.0),
                "qd": (0.2, 1.0), "li0": (0.0, 2.0),
                "lred": (math.log(1.5 * reb[0]), math.log(4 * reb[1])), "sky": (0.0, 5.0)}

    @staticmethod
    def _z(v, r):
        lo, hi = r
        return (v - 0.5 * (lo + hi)) / (0.5 * (hi - lo))

    @staticmethod
    def _unz(z, r):
        lo, hi = r
        return 0.5 * (lo + hi) + 0.5 * (hi - lo) * z

    def encode(self, p: np.ndarray) -> np.ndarray:
        r = self._ranges()
        c = self.side / 2.0
        t = np.empty((p.shape[0], self.dv), np.float32)
        t[:, 0] = (p[:, 0] - c) / 2.0
        t[:, 1] = (p[:, 1] - c) / 2.0
        t[:, 2] = self._z(p[:, 2], r["qb"])
        t[:, 3], t[:, 4] = np.cos(2 * p[:, 3]), np.sin(2 * p[:, 3])
        t[:, 5] = self._z(np.log10(p[:, 4]), r["lie"])
        t[:, 6] = self._z(np.log(p[:, 5]), r["lreb"])
        t[:, 7] = self._z(p[:, 6], r["nb"])
        t[:, 8] = self._z(p[:, 7], r["qd"])
        t[:, 9], t[:, 10] = np.cos(2 * p[:, 8]), np.sin(2 * p[:, 8])
        t[:, 11] = self._z(np.log10(p[:, 9]), r["li0"])
        t[:, 12] = self._z(np.log(p[:, 10]), r["lred"])
        t[:, 13] = self._z(p[:, 12], r["sky"])
        return t

    def decode(self, t: np.ndarray, spec) -> np.ndarray:
        """Network outputs -> parameters [G, 13] inside the spec's bounds (disk n = 1)."""
        r = self._ranges()
        c = self.side / 2.0
        t = np.asarray(t, np.float64)
        p = np.empty((t.shape[0], 13))
        p[:, 0] = c + 2.0 * t[:, 0]
        p[:, 1] = c + 2.0 * t[:, 1]
        p[:, 2] = self._unz(t[:, 2], r["qb"])
        p[:, 3] = 0.5 * np.arctan2(t[:, 4], t[:, 3]) % math.pi
        p[:, 4] = 10 ** self._unz(t[:, 5], r["lie"])
        p[:, 5] = np.exp(self._unz(t[:, 6], r["lreb"]))
        p[:, 6] = self._unz(t[:, 7], r["nb"])
        p[:, 7] = self._unz(t[:, 8], r["qd"])
        p[:, 8] = 0.5 * np.arctan2(t[:, 10], t[:, 9]) % math.pi
        p[:, 9] = 10 ** self._unz(t[:, 11], r["li0"])
        p[:, 10] = np.exp(self._unz(t[:, 12], r["lred"]))
        p[:, 11] = 1.0
        p[:, 12] = self._unz(t[:, 13], r["sky"])
        lo, hi = np.asarray(spec.lo), np.asarray(spec.hi)
        # stay strictly inside the bounds the LM clamps to (q below 1 keeps the PA meaningful)
        p[:, [2, 7]] = np.clip(p[:, [2, 7]], 0.06, 0.99)
        return np.clip(p, lo + 1e-9 * np.abs(lo), hi - 1e-9 * np.abs(hi))


# ---------------------------------------------------------------------------
# training data: stamps rendered by gm_model, prepared as network inputs
# ---------------------------------------------------------------------------
SKY_SIGMA = 2.0  # sqrt of the recipe's sky variance: the asinh scale of the inputs


def make_training_set(n: int, seed: int, side: int = 128, ks=tuple(range(25, 52, 2)), chunk: int = 8192,
                      device="cuda"):
    """(inputs [n,64,64,1] BF16, targets [n,dv] FP32, codec) for n bulge + disk galaxies drawn as
    synth.draw_uneven_bulge_disk on side x side stamps; noise from a seeded device generator."""
    import torch
    from . import synth, workloads
    if side != 2 * INPUT_SIDE:
        raise CNNError(f"the network reads {INPUT_SIDE} x {INPUT_SIDE} inputs: stamps must be {2 * INPUT_SIDE} wide")
    dev = torch.device(device)
    codec = BulgeDiskCodec(side)
    X = torch.empty((n, INPUT_SIDE, INPUT_SIDE, 1), dtype=torch.bfloat16, device=dev)
    T = torch.empty((n, codec.dv), dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev)
    for c, s in enumerate(range(0, n, chunk)):
        g = min(chunk, n - s)
        rb = synth.draw_uneven_bulge_disk(seed=seed * 100003 + c, G=g, sides=(side,), ks=ks, noise=False)
        gen.manual_seed(seed * 100003 + c)
        z = torch.randn(g * side * side, generator=gen, device=dev, dtype=torch.float32)
        image, _, _ = workloads.render_uneven(rb, dev, z=z)
        X[s:s + g] = prep(image.view(g, side, side), 1.0 / SKY_SIGMA)
        T[s:s + g] = torch.from_numpy(codec.encode(rb.truth)).to(dev)
    return X, T, codec


def train(net: Net, X, T, dv: int, epochs: int = 1, batch: int = 512, lr: float = 2e-3, seed: int = 0,
          log=None) -> list[float]:
    """Adam on shuffled mini-batches with a cosine learning-rate decay; returns per-epoch mean losses."""
    import torch
    n = X.shape[0]
    steps = epochs * (n // batch)
    gen = torch.Generator(device=X.device)
    gen.manual_seed(seed)
    out = []
    k = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen, device=X.device)
        tot = torch.zeros(1, dtype=torch.float32, device=X.device)
        nb = n // batch
        for bi in range(nb):
            idx = perm[bi * batch:(bi + 1) * batch]
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * k / max(steps, 1)))
            tot += net.train_step(X[idx].contiguous(), T[idx].contiguous(), dv, rate)
            k += 1
        out.append(float(tot.item()) / max(nb, 1))
        if log:
            log(f"epoch {ep}: mean loss {out[-1]:.4f}")
    check_device_error()
    return out


def learned_start(net: Net, image, codec: BulgeDiskCodec, spec):
    """Starting parameters [G,13] (FP64 CUDA) from equal side x side stamps [G,side,side]."""
    import torch
    x = prep(image, 1.0 / SKY_SIGMA)
    pred = net.predict(x)[:, :codec.dv].cpu().numpy()
    return torch.from_numpy(codec.decode(pred, spec)).to(image.device)


def _take(t, offsets, idx):
    """The segments [offsets[g], offsets[g+1]) of a packed tensor for galaxies idx, packed."""
    import torch
    if t is None:
        return None
    return torch.cat([t[int(offsets[g]):int(offsets[g + 1])] for g in idx]).contiguous()


def fit_with_fallback(fitter, spec, p_learned, p_default, image, sigma, mask, psf, opts, geom=None):
    """LM from the learned start for every galaxy; the ones that do not converge from it are
    fitted again from the default start and keep the refit when it converged or reached a
    lower chi^2.  Equal stamps (image [G,H,W]) or an uneven batch (geom [G,3], packed arrays).
    Returns (result dict of CUDA tensors, info) with info = {"refits", "evals" (galaxy
    evaluations of both fits), "fused_ms" (device time of their fused tile kernels)}."""
    import torch
    params = p_learned.clone().contiguous()
    res = {k: v.clone() for k, v in fitter.fit(params, image, sigma, mask, psf, opts).items()}
    st = _gm.gm_fit_last_stats()
    info = {"refits": 0, "evals": st["galaxy_evals"], "fused_ms": st["fused_ms"]}
    bad = torch.nonzero(res["status"] != _gm.ST_CONVERGED).flatten()
    n = int(bad.numel())
    if n == 0:
        return res, info
    p2 = p_default[bad].clone().contiguous()
    if geom is None:
        sub = [None if t is None else t[bad].contiguous() for t in (image, sigma, mask, psf)]
        f2 = _gm.Fitter(spec, n, image.shape[1], image.shape[2], psf.shape[-1], device=image.device)
    else:
        g = _gm.geom_array(geom)
        idx = bad.cpu().numpy()
        po = np.concatenate([[0], np.cumsum(g[:, 0].astype(np.int64) * g[:, 1])])
        ko = np.concatenate([[0], np.cumsum(g[:, 2].astype(np.int64) ** 2)])
        sub = [_take(image, po, idx), _take(sigma, po, idx), _take(mask, po, idx), _take(psf, ko, idx)]
        f2 = _gm.Fitter(spec, n, device=image.device, geom=g[idx])
    r2 = f2.fit(p2, sub[0], sub[1], sub[2], sub[3], opts)
    st = _gm.gm_fit_last_stats()
    info = {"refits": n, "evals": info["evals"] + st["galaxy_evals"], "fused_ms": info["fused_ms"] + st["fused_ms"]}
    take = (r2["status"] == _gm.ST_CONVERGED) | (r2["chi2"] < res["chi2"][bad])
    idx_t = bad[take]
    for k in ("params", "chi2", "dof", "iters", "status", "sigma_p"):
        res[k][idx_t] = r2[k][take]
    return res, info
