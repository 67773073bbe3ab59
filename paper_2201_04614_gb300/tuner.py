"""The learned tuner of block size and padding mode (binding of the
vsz_tuner_* / vsz_mlp_* calls of include/vsz.h).

The paper picks the block size with a sampling autotuner (Sec. III-D,
Sec. V-E) and compares padding values by hand (Sec. IV, Sec. V-H).  Here a
small MLP (12 -> 64 -> 64 -> 12, fp32) maps 12 sampled statistics of a field
to a class (block size x padding mode).  Training, inference, features, the
labelling sweep and the guard all run in the library's CUDA kernels; this
module only sequences the calls, draws minibatch orders and reads and writes
the weights file.

Classes: c = 3 * slot + padslot; padslot 0 zero, 1 global average, 2 block
average; block slots 1D (32, 64, 128, 256), 2D (8, 16, 32, 64), 3D
(8, 16, 32).  The default class (block 256 / 16 / 8, zero padding) is the
fallback whenever the guard finds more outliers in the tuned class.
"""
from __future__ import annotations

import ctypes
import os
import struct

import numpy as np

from . import Params, VszError, _check, _need, _ptr, _stream_handle, lib, PAD_MODES

NFEAT, NCLASS, HIDDEN = 12, 12, 64
NPARAM = HIDDEN * NFEAT + HIDDEN + HIDDEN * HIDDEN + HIDDEN + NCLASS * HIDDEN + NCLASS
BLOCKS = {1: (32, 64, 128, 256), 2: (8, 16, 32, 64), 3: (8, 16, 32)}
PAD_SLOTS = ("zero", "global_avg", "block_avg")
DEFAULT_BLOCK = {1: 256, 2: 16, 3: 8}
WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuner_weights.bin")
_MAGIC = b"VSZMLP01"


def class_params(ndim: int, c: int):
    """(block, pad name) of class c for this rank, or None if not allowed."""
    slot, ps = divmod(int(c), 3)
    if slot >= len(BLOCKS[ndim]):
        return None
    return BLOCKS[ndim][slot], PAD_SLOTS[ps]


def class_mask(ndim: int) -> int:
    """Bit c set for every class c allowed at this rank."""
    return sum(1 << c for c in range(NCLASS) if class_params(ndim, c) is not None)


def default_class(ndim: int) -> int:
    """The class of the default configuration: the rank's default block, zero padding."""
    return 3 * BLOCKS[ndim].index(DEFAULT_BLOCK[ndim])


def params_for(p: Params, c: int) -> Params:
    """`p` with the block size and padding mode of class c."""
    b, pad = class_params(len(p.dims), c)
    return Params(p.dims, b, p.eb, p.eb_mode, p.radius, PAD_MODES[pad])


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the tuner needs a CUDA device (no CPU fallback)")
    return torch


def _bind():
    L = lib()
    if getattr(L, "_tuner_bound", False):
        return L
    P = ctypes.POINTER
    vp, sz, i32, f32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_float
    from . import _CParams
    L.vsz_tuner_features_workspace_size.restype = sz
    L.vsz_tuner_features_workspace_size.argtypes = []
    L.vsz_tuner_features.argtypes = [P(_CParams), vp, vp, vp, vp, sz, vp]
    L.vsz_tuner_sweep_workspace_size.restype = sz
    L.vsz_tuner_sweep_workspace_size.argtypes = [P(_CParams)]
    L.vsz_tuner_sweep.argtypes = [P(_CParams), vp, vp, vp, vp, sz, vp]
    L.vsz_tuner_guard_workspace_size.restype = sz
    L.vsz_tuner_guard_workspace_size.argtypes = [P(_CParams), i32, i32]
    L.vsz_tuner_guard.argtypes = [P(_CParams), vp, i32, i32, vp, vp, vp, sz, vp]
    L.vsz_tuner_guard_sample_dims.argtypes = [P(_CParams), P(ctypes.c_uint64)]
    L.vsz_mlp_forward.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp]
    L.vsz_mlp_grad_workspace_size.restype = sz
    L.vsz_mlp_grad_workspace_size.argtypes = [i32]
    L.vsz_mlp_grad.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp, vp, vp, sz, vp]
    L.vsz_mlp_adam.argtypes = [vp, vp, vp, vp, i32, f32, f32, f32, f32, i32, vp]
    L.vsz_sampling_autotune_workspace_size.restype = sz
    L.vsz_sampling_autotune_workspace_size.argtypes = [P(_CParams), ctypes.c_double]
    L.vsz_sampling_autotune.argtypes = [P(_CParams), vp, ctypes.c_double, i32, P(ctypes.c_uint32),
                                        P(ctypes.c_float), P(ctypes.c_uint64), vp, sz, vp]
    for name in ("vsz_tuner_features", "vsz_tuner_sweep", "vsz_tuner_guard", "vsz_tuner_guard_sample_dims",
                 "vsz_mlp_forward", "vsz_mlp_grad", "vsz_mlp_adam", "vsz_sampling_autotune"):
        getattr(L, name).restype = ctypes.c_int
    L._tuner_bound = True
    return L


def _ws(nbytes: int, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _xcheck(x, p: Params):
    torch = _torch()
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise TypeError("x must be a contiguous float32 CUDA tensor")
    if x.numel() != p.n:
        raise ValueError(f"x has {x.numel()} elements, params describe {p.n}")


def _rows_check(X, *per_row):
    """X must be a matrix of NFEAT features per sample, and every per-sample
    array must cover its rows: the kernels read them by sample index."""
    if X.dim() != 2 or X.shape[1] != NFEAT:
        raise ValueError(f"X must have shape [n, {NFEAT}], not {tuple(X.shape)}")
    for a in per_row:
        if a.numel() < X.shape[0]:
            raise ValueError(f"a per-sample array holds {a.numel()} entries for {X.shape[0]} samples")


# ---------------------------------------------------------------- field-level calls
def features(p: Params, x, out64=None, out32=None, stream=None):
    """The 12 features of a field on the device: (float64[12], float32[12])."""
    torch = _torch()
    L = _bind()
    _xcheck(x, p)
    dev = x.device
    f64 = out64 if out64 is not None else torch.empty(NFEAT, dtype=torch.float64, device=dev)
    f32 = out32 if out32 is not None else torch.empty(NFEAT, dtype=torch.float32, device=dev)
    _need(f64, "out64", 8, NFEAT)
    _need(f32, "out32", 4, NFEAT)
    ws = _ws(L.vsz_tuner_features_workspace_size(), dev)
    _check(L.vsz_tuner_features(ctypes.byref(p.c()), _ptr(x), _ptr(f64), _ptr(f32), _ptr(ws), ws.numel(),
                                _stream_handle(stream)), "vsz_tuner_features")
    return f64, f32


def sweep(p: Params, x, stream=None, with_nout: bool = False):
    """Estimated compressed size (bytes) of every class: float64[12] on the
    device, +inf for classes the rank does not allow; with_nout also returns
    each class's outlier count (int64[12], -1 where not allowed)."""
    torch = _torch()
    L = _bind()
    _xcheck(x, p)
    need = L.vsz_tuner_sweep_workspace_size(ctypes.byref(p.c()))
    if need == 0:
        raise ValueError("invalid parameters for the sweep")
    ws = _ws(need, x.device)
    cost = torch.empty(NCLASS, dtype=torch.float64, device=x.device)
    nout = torch.empty(NCLASS, dtype=torch.int64, device=x.device)
    _check(L.vsz_tuner_sweep(ctypes.byref(p.c()), _ptr(x), _ptr(cost), _ptr(nout), _ptr(ws), ws.numel(),
                             _stream_handle(stream)), "vsz_tuner_sweep")
    return (cost, nout) if with_nout else cost


def guard_counts(p: Params, x, class_a: int, class_b: int, stream=None, with_cost: bool = False):
    """Exact outlier counts of two classes on the guard's fixed sample
    (device uint64[2] viewed as int64); with_cost also returns the two
    classes' estimated sizes on the sample (float64[2], as the sweep's)."""
    torch = _torch()
    L = _bind()
    _xcheck(x, p)
    need = L.vsz_tuner_guard_workspace_size(ctypes.byref(p.c()), int(class_a), int(class_b))
    if need == 0:
        raise ValueError("invalid parameters or classes for the guard")
    ws = _ws(need, x.device)
    out = torch.zeros(2, dtype=torch.int64, device=x.device)
    cost = torch.zeros(2, dtype=torch.float64, device=x.device) if with_cost else None
    _check(L.vsz_tuner_guard(ctypes.byref(p.c()), _ptr(x), int(class_a), int(class_b), _ptr(out),
                             _ptr(cost) if with_cost else None, _ptr(ws), ws.numel(), _stream_handle(stream)),
           "vsz_tuner_guard")
    return (out, cost) if with_cost else out


def guard_sample_dims(p: Params) -> tuple:
    """Extents of the fixed block sample the guard compresses (vsz_tuner_guard_sample_dims)."""
    L = _bind()
    d = (ctypes.c_uint64 * 3)()
    _check(L.vsz_tuner_guard_sample_dims(ctypes.byref(p.c()), d), "vsz_tuner_guard_sample_dims")
    return tuple(int(v) for v in d[: len(p.dims)])


def sampling_autotune(p: Params, x, sample_frac: float = 0.05, iters: int = 3, stream=None) -> dict:
    """The paper's sampling autotuner (vsz_sampling_autotune): times the
    dual-quant of every block size of the rank on a sample of the field and
    returns {"block", "ms" (per block size), "sample_elems"}.  Synchronous."""
    torch = _torch()
    L = _bind()
    _xcheck(x, p)
    wsb = int(L.vsz_sampling_autotune_workspace_size(ctypes.byref(p.c()), float(sample_frac)))
    if wsb == 0:
        raise VszError(1, "vsz_sampling_autotune_workspace_size")
    ws = torch.empty(wsb, dtype=torch.uint8, device=x.device)
    best = ctypes.c_uint32(0)
    ms = (ctypes.c_float * 4)()
    ne = ctypes.c_uint64(0)
    _check(L.vsz_sampling_autotune(ctypes.byref(p.c()), _ptr(x), float(sample_frac), int(iters), ctypes.byref(best),
                                   ms, ctypes.byref(ne), _ptr(ws), wsb, _stream_handle(stream)),
           "vsz_sampling_autotune")
    blocks = {1: (32, 64, 128, 256), 2: (8, 16, 32, 64), 3: (8, 16, 32, 0)}[len(p.dims)]
    return {"block": int(best.value), "ms": {b: float(m) for b, m in zip(blocks, ms) if b},
            "sample_elems": int(ne.value)}


# Estimated sizes within SIZE_TOL of the least count as equal; among them the
# padding that costs least to compute wins (zero, then per block, then
# global: a field-wide statistic and a pass over the block origins).
SIZE_TOL = 0.005
PAD_RANK = (0, 2, 1)  # by padding slot: zero, global average, block average


def label_of(costs) -> int:
    """The label from the classes' estimated sizes (the sweep's costs): among
    the classes within SIZE_TOL of the least size, the cheapest padding, then
    the smaller size, then the lower index."""
    c = np.asarray(costs, np.float64)
    lo = float(np.min(c))
    best = None
    for k in range(c.size):
        if not (c[k] <= lo * (1.0 + SIZE_TOL)):
            continue
        key = (PAD_RANK[k % 3], float(c[k]), k)
        if best is None or key < best[0]:
            best = (key, k)
    return best[1]


# ---------------------------------------------------------------- network
class MLP:
    """Flat fp32 parameters and input normalisation on the device, with the
    library's forward, gradient and Adam kernels."""

    def __init__(self, theta=None, mu=None, sigma=None, device=None, seed: int = 0):
        torch = _torch()
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if theta is None:
            theta = self.init_params(seed)
        self.theta = torch.as_tensor(np.asarray(theta, np.float32)).to(dev).contiguous()
        mu = np.zeros(NFEAT, np.float32) if mu is None else np.asarray(mu, np.float32)
        sigma = np.ones(NFEAT, np.float32) if sigma is None else np.asarray(sigma, np.float32)
        self.norm = torch.as_tensor(np.concatenate([mu, sigma]).astype(np.float32)).to(dev).contiguous()
        self.device = dev

    @staticmethod
    def init_params(seed: int) -> np.ndarray:
        """He-uniform weights, zero biases (numpy PCG64, seeded)."""
        rng = np.random.Generator(np.random.PCG64(seed))
        parts = []
        for fan_in, fan_out in ((NFEAT, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, NCLASS)):
            lim = np.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
            parts.append(np.zeros(fan_out))
        return np.concatenate(parts).astype(np.float32)

    def forward(self, X, masks, stream=None):
        """(logits [n, 12], class [n]) on the device."""
        torch = _torch()
        L = _bind()
        X = torch.as_tensor(X, dtype=torch.float32, device=self.device).contiguous()
        M = torch.as_tensor(np.asarray(masks, np.uint32).view(np.int32) if not isinstance(masks, torch.Tensor)
                            else masks, device=self.device).to(torch.int32).contiguous()
        _rows_check(X, M)
        n = X.shape[0]
        logits = torch.empty((max(n, 1), NCLASS), dtype=torch.float32, device=self.device)
        cls = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        _check(L.vsz_mlp_forward(_ptr(self.theta), _ptr(self.norm), _ptr(X), _ptr(M), n, _ptr(logits), _ptr(cls),
                                 _stream_handle(stream)), "vsz_mlp_forward")
        return logits[:n], cls[:n]

    def grad(self, X, y, masks, idx=None, stream=None):
        """(mean loss, gradient [NPARAM]) over the minibatch idx (all samples if None)."""
        torch = _torch()
        L = _bind()
        X = torch.as_tensor(X, dtype=torch.float32, device=self.device).contiguous()
        Y = torch.as_tensor(y, dtype=torch.int32, device=self.device).contiguous()
        M = torch.as_tensor(np.asarray(masks, np.uint32).view(np.int32) if not isinstance(masks, torch.Tensor)
                            else masks, device=self.device).to(torch.int32).contiguous()
        I = None if idx is None else torch.as_tensor(idx, dtype=torch.int32, device=self.device).contiguous()
        _rows_check(X, M, Y)
        if I is not None and I.numel() and bool(((I < 0) | (I >= X.shape[0])).any()):
            raise ValueError(f"idx holds a sample index outside 0..{X.shape[0] - 1}")
        batch = X.shape[0] if I is None else I.numel()
        g = torch.empty(NPARAM, dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        ws = _ws(L.vsz_mlp_grad_workspace_size(batch), self.device)
        _check(L.vsz_mlp_grad(_ptr(self.theta), _ptr(self.norm), _ptr(X), _ptr(Y), _ptr(M),
                              _ptr(I) if I is not None else ctypes.c_void_p(0), batch, _ptr(g), _ptr(loss),
                              _ptr(ws), ws.numel(), _stream_handle(stream)), "vsz_mlp_grad")
        return loss, g

    def train(self, X, y, masks, epochs: int = 300, batch: int = 256, lr: float = 2e-3, seed: int = 0,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, log_every: int = 0):
        """Minibatch Adam on the device; the host only draws the sample
        order of each epoch (seeded) and sequences the kernels.  Returns the
        per-epoch mean training loss."""
        torch = _torch()
        L = _bind()
        X = torch.as_tensor(X, dtype=torch.float32, device=self.device).contiguous()
        Y = torch.as_tensor(y, dtype=torch.int32, device=self.device).contiguous()
        M = torch.as_tensor(np.asarray(masks, np.uint32).view(np.int32), device=self.device).contiguous()
        n = X.shape[0]
        m = torch.zeros(NPARAM, dtype=torch.float32, device=self.device)
        v = torch.zeros(NPARAM, dtype=torch.float32, device=self.device)
        g = torch.empty(NPARAM, dtype=torch.float32, device=self.device)
        nsteps = (n + batch - 1) // batch
        losses_dev = torch.zeros(epochs * nsteps, dtype=torch.float32, device=self.device)
        ws = _ws(L.vsz_mlp_grad_workspace_size(batch), self.device)
        rng = np.random.Generator(np.random.PCG64(seed))
        s = _stream_handle(None)
        step = 0
        for ep in range(epochs):
            order = torch.as_tensor(rng.permutation(n).astype(np.int32), device=self.device)
            for k in range(nsteps):
                idx = order[k * batch:(k + 1) * batch]
                b = idx.numel()
                _check(L.vsz_mlp_grad(_ptr(self.theta), _ptr(self.norm), _ptr(X), _ptr(Y), _ptr(M), _ptr(idx), b,
                                      _ptr(g), ctypes.c_void_p(losses_dev.data_ptr() + 4 * step), _ptr(ws),
                                      ws.numel(), s), "vsz_mlp_grad")
                step += 1
                _check(L.vsz_mlp_adam(_ptr(self.theta), _ptr(g), _ptr(m), _ptr(v), NPARAM, lr, beta1, beta2, eps,
                                      step, s), "vsz_mlp_adam")
            if log_every and (ep + 1) % log_every == 0:
                print(f"[tuner] epoch {ep + 1}: loss {losses_dev[ep * nsteps:(ep + 1) * nsteps].mean().item():.4f}",
                      flush=True)
        return losses_dev.view(epochs, nsteps).mean(dim=1).cpu().numpy()

    # ---- weights file: magic, nfeat, hidden, nclass, nparam (u32), mu, sigma, theta (f32)
    def save(self, path: str = WEIGHTS_PATH) -> None:
        """Write the weights file (header with the shape, normalisation, parameters)."""
        norm = self.norm.cpu().numpy()
        with open(path, "wb") as f:
            f.write(_MAGIC + struct.pack("<4I", NFEAT, HIDDEN, NCLASS, NPARAM))
            f.write(norm.astype("<f4").tobytes())
            f.write(self.theta.cpu().numpy().astype("<f4").tobytes())

    @classmethod
    def load(cls, path: str = WEIGHTS_PATH, device=None) -> "MLP":
        """Read a weights file written by save(); its shape must match this library's."""
        with open(path, "rb") as f:
            head = f.read(len(_MAGIC) + 16)
            if head[:len(_MAGIC)] != _MAGIC:
                raise ValueError(f"{path}: not a tuner weights file")
            nf, hid, nc, npar = struct.unpack("<4I", head[len(_MAGIC):])
            if (nf, hid, nc, npar) != (NFEAT, HIDDEN, NCLASS, NPARAM):
                raise ValueError(f"{path}: shape {(nf, hid, nc, npar)} does not match this library")
            norm = np.frombuffer(f.read(4 * 2 * NFEAT), "<f4")
            theta = np.frombuffer(f.read(4 * NPARAM), "<f4")
        return cls(theta, norm[:NFEAT], norm[NFEAT:], device=device)


# ---------------------------------------------------------------- choosing
def guard_pick(tuned: int, default: int, nout, cost) -> int:
    """The guard's decision between the network's class and the default
    from their outlier counts and estimated sizes on the guard's sample: the
    default wins when the tuned class has more outliers, and, when the tuned
    class's padding costs more to compute, when the two sizes tie by the
    labels' rule (within SIZE_TOL of the smaller one; among tied classes the
    cheaper padding wins, as in label_of)."""
    if tuned == default:
        return default
    if int(nout[0]) > int(nout[1]):
        return default
    if cost is not None and PAD_RANK[tuned % 3] > PAD_RANK[default % 3]:
        lo = min(float(cost[0]), float(cost[1]))
        if float(cost[1]) <= lo * (1.0 + SIZE_TOL):
            return default
    return tuned


def choose(fields, mlp: MLP | None = None, guard: bool = True, stream=None) -> list:
    """Tuned class for each (Params, x) of `fields`: features of every field,
    one batched MLP inference, then the guard on a fixed sample of the field
    (guard_pick: the default class wins when the tuned one has more outliers,
    or when its dearer padding buys no size outside the labels' tie
    tolerance).  Returns a list of dicts {class, predicted, default,
    guard_nout, guard_cost}."""
    torch = _torch()
    if mlp is None:
        mlp = MLP.load()
    n = len(fields)
    if n == 0:
        return []
    feats = torch.empty((n, NFEAT), dtype=torch.float32, device=mlp.device)
    f64 = torch.empty((n, NFEAT), dtype=torch.float64, device=mlp.device)
    for i, (p, x) in enumerate(fields):
        features(p, x, out64=f64[i], out32=feats[i], stream=stream)
    masks = np.array([class_mask(len(p.dims)) for p, _ in fields], np.uint32)
    _, cls = mlp.forward(feats, masks, stream=stream)
    pred = cls.cpu().numpy()
    out = []
    for i, (p, x) in enumerate(fields):
        nd = len(p.dims)
        d = default_class(nd)
        c = int(pred[i])
        rec = {"predicted": c, "default": d, "class": c, "guard_nout": None, "guard_cost": None}
        if guard and c != d and p.n > 0:
            cnt, cost = guard_counts(p, x, c, d, stream=stream, with_cost=True)
            cnt, cost = cnt.cpu().numpy(), cost.cpu().numpy()
            rec["guard_nout"] = (int(cnt[0]), int(cnt[1]))
            rec["guard_cost"] = (float(cost[0]), float(cost[1]))
            rec["class"] = guard_pick(c, d, cnt, cost)
        out.append(rec)
    return out
