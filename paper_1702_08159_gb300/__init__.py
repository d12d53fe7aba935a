"""GB300-native McKernel / Fastfood feature maps (arXiv 1702.08159).

Python binding of libmck.so: argument marshalling only. Every computation
runs in the library's CUDA kernels; PyTorch provides device memory, streams
and autograd. Calls run on the current CUDA stream of the tensors' device.

    import paper_1702_08159_gb300 as mck
    plan = mck.Plan(d=1024, E=16, kernel="rbf", sigma=1.0, seed=42)
    phi = mck.features(plan, x)            # x: (n, in_dim) float32 CUDA
    logits = mck.fused_logits(plan, x, W, b)

The map is Z-hat = (1/(sigma sqrt d)) C H G Pi H B (Eq. etn:mckernel) and the
features are [cos(Z-hat x-hat), sin(Z-hat x-hat)] per expansion
(Eq. etn:mcfeatures); the classifier is softmax(W phi + b) (Sec. "Empirical
Analysis and Experiments").
"""

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import MckError, check, load

__all__ = [
    "Plan", "MckError", "fwht_", "features", "features_host", "HostPipeline", "features_backward",
    "fused_logits",
    "fused_logits_backward", "softmax_xent", "library_path",
]

_KERNELS = {"rbf": _lib.MCK_RBF, "matern": _lib.MCK_MATERN, "laplace": _lib.MCK_LAPLACE}


def library_path():
    return _lib.LIB_PATH


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _f32_cuda(t, name, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float32 or not t.is_cuda:
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on {t.device}, expected cuda:{device}")
    return t


def _rows(x, name="x"):
    """(n, in_dim) view with unit stride in the last dimension; returns (n, in_dim, ldx)."""
    if x.dim() != 2:
        raise ValueError(f"{name} must be 2-D (n, in_dim)")
    if x.stride(1) != 1 or (x.size(0) > 1 and x.stride(0) < x.size(1)):
        x = x.contiguous()
    ld = x.stride(0) if x.size(0) > 1 else x.size(1)
    return x, x.size(0), x.size(1), ld


class Plan:
    """Tables B, Pi, G and C of E expansions of dimension d, made from a seed.

    Sec. "API Description": a factory instantiates the parameters of a
    pre-specified kernel; they are deterministic functions of a hash, so only
    (d, E, kernel, sigma, t, seed) identify a plan.
    """

    def __init__(self, d, E, kernel="rbf", sigma=1.0, seed=0, matern_t=40, device=None):
        lib = load()
        if isinstance(kernel, str):
            kernel = _KERNELS[kernel.lower()]
        if device is None:
            device = torch.cuda.current_device()
        handle = ctypes.c_void_p()
        check(lib.mck_plan_ex(ctypes.byref(handle), int(d), int(E), int(kernel), float(sigma),
                              int(matern_t), int(seed) & 0xFFFFFFFFFFFFFFFF, int(device)),
              "mck_plan")
        self._h = handle
        self.d, self.E, self.kernel, self.sigma = int(d), int(E), int(kernel), float(sigma)
        self.matern_t = int(matern_t) if kernel == _lib.MCK_MATERN else 0
        self.seed, self.device = int(seed), int(device)
        self.L = self.d.bit_length() - 1

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("plan is closed")
        return self._h

    @property
    def num_features(self):
        return 2 * self.E * self.d

    def tables(self):
        """Host copies: B_bits (E, ceil(d/32)) uint32, perm (E, d) uint32, G and Cs (E, d) float32."""
        words = (self.d + 31) // 32
        B = np.empty((self.E, words), np.uint32)
        P = np.empty((self.E, self.d), np.uint32)
        G = np.empty((self.E, self.d), np.float32)
        C = np.empty((self.E, self.d), np.float32)
        check(load().mck_plan_tables(self.handle, B.ctypes.data, P.ctypes.data, G.ctypes.data,
                                     C.ctypes.data), "mck_plan_tables")
        return {"B_bits": B, "perm": P, "G": G, "Cs": C}

    def signs(self):
        """B as an (E, d) float32 array of +-1."""
        bits = self.tables()["B_bits"]
        k = np.arange(self.d)
        return np.ascontiguousarray(
            np.where((bits[:, k // 32] >> (k % 32)) & 1, -1.0, 1.0), dtype=np.float32)

    def set_signs(self, B):
        """Replace the sign diagonals: B_e[k] = -1 where B[e, k] < 0, else +1.
        B is a contiguous (E, d) float32 tensor on the plan's device; the
        update is ordered on the current stream."""
        _f32_cuda(B, "B", self.device)
        if tuple(B.shape) != (self.E, self.d) or not B.is_contiguous():
            raise ValueError(f"B must be a contiguous ({self.E}, {self.d}) tensor")
        check(load().mck_plan_set_signs(self.handle, _ptr(B), _stream(B.device)),
              "mck_plan_set_signs")

    def set_launch(self, rows_per_item=0, staged=-1):
        """Launch shape of the batched feature kernels (mck_plan_set_launch):
        0 / -1 = automatic; results are identical for every shape."""
        check(load().mck_plan_set_launch(self.handle, int(rows_per_item), int(staged)),
              "mck_plan_set_launch")

    def launch(self):
        """(rows_per_item, staged) as set (0 / -1 = automatic)."""
        r, st = ctypes.c_int32(), ctypes.c_int32()
        check(load().mck_plan_get_launch(self.handle, ctypes.byref(r), ctypes.byref(st)),
              "mck_plan_get_launch")
        return r.value, st.value

    def launch_candidates(self):
        """Every accepted (rows_per_item, staged) shape of this plan's d."""
        L = self.d.bit_length() - 1
        if 5 <= L <= 10:
            vpw = 32 // (1 << (L - 5))
            return sorted({(vpw, -1), (max(4, vpw), -1)})
        if 11 <= L <= 14:
            return [(r, st) for r in (1, 2, 4) for st in (0, 1)]
        return [(0, -1)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().mck_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __repr__(self):
        k = {_lib.MCK_RBF: "rbf", _lib.MCK_LAPLACE: "laplace"}.get(
            self.kernel, f"matern(t={self.matern_t})")
        return f"Plan(d={self.d}, E={self.E}, kernel={k}, sigma={self.sigma}, seed={self.seed})"


def _tables(plan, Cs, G):
    shape = (plan.E, plan.d)
    for t, name in ((Cs, "Cs"), (G, "G")):
        if t is not None:
            _f32_cuda(t, name, plan.device)
            if tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous ({plan.E}, {plan.d}) tensor")
    return Cs, G


def fwht_(x, prec="fp32", regime="auto"):
    """In-place unnormalised Walsh-Hadamard transform of the rows of x (last dim d).

    prec: "fp32" (float32 butterflies, any d <= 2^20) or, for 256 <= d <= 2^20,
    the tensor-core Kronecker-H16 forms "bf16", "fp16", "bf16_split",
    "fp16_split" (16-bit operands, FP32 accumulation; *_split = hi + lo).
    regime (FP32 at d = 2^16, 2^17 only): "auto", "cluster_2_15",
    "cluster_2_14" or "two_pass" (mck_fwht_ex; identical results).
    """
    _f32_cuda(x, "x")
    if not x.is_contiguous():
        raise ValueError("x must be contiguous")
    d = x.size(-1)
    n = x.numel() // d if d else 0
    p = _lib.PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    r = _lib.FWHT_REGIMES[regime] if isinstance(regime, str) else int(regime)
    with torch.cuda.device(x.device):
        check(load().mck_fwht_ex(_ptr(x), n, d, p, r, _stream(x.device)), "mck_fwht_ex")
    return x


def features(plan, x, Cs=None, G=None, out=None, prec="fp32"):
    """phi(x): (n, 2 E d); row = E blocks of [cos | sin] (Eq. etn:mcfeatures).

    prec: "fp32" (float32 butterflies), or at d = 1024 the tensor-core forms
    "fp16_split", "bf16_split", "fp16", "bf16" (mck_features_ex)."""
    _f32_cuda(x, "x", plan.device)
    x, n, in_dim, ld = _rows(x)
    Cs, G = _tables(plan, Cs, G)
    if out is None:
        out = torch.empty((n, plan.num_features), device=x.device, dtype=torch.float32)
    else:
        _f32_cuda(out, "out", plan.device)
        if tuple(out.shape) != (n, plan.num_features) or not out.is_contiguous():
            raise ValueError("out must be a contiguous (n, 2 E d) tensor")
    p = _lib.PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    if p == _lib.MCK_FP32:
        check(load().mck_features(plan.handle, _ptr(x), n, in_dim, ld, _ptr(Cs), _ptr(G),
                                  _ptr(out), _stream(x.device)), "mck_features")
    else:
        check(load().mck_features_ex(plan.handle, _ptr(x), n, in_dim, ld, _ptr(Cs), _ptr(G),
                                     _ptr(out), p, _stream(x.device)), "mck_features_ex")
    return out


class HostPipeline:
    """A host-buffer pipeline of the C ABI (mck_host_pipe_create): `streams`
    CUDA streams, each with device buffers for a chunk of `chunk_rows` input
    rows (in_dim wide) and of their features, made once and reused, so calls
    allocate nothing. Each chunk's host-to-device copy, feature kernel and
    device-to-host copy run on one stream (mck_features_host)."""

    def __init__(self, plan, in_dim, chunk_rows=2048, streams=4):
        self.plan, self.in_dim = plan, int(in_dim)
        self.rows = max(1, int(chunk_rows))
        self.handle = None
        h = ctypes.c_void_p()
        with torch.cuda.device(plan.device):
            check(load().mck_host_pipe_create(ctypes.byref(h), plan.handle, self.in_dim, self.rows,
                                              int(streams)), "mck_host_pipe_create")
        self.handle = h

    def run(self, x, out, Cs=None, G=None):
        """Features of the host batch x into the host array out; stream-ordered
        (the current stream waits for every chunk)."""
        Cs, G = _tables(self.plan, Cs, G)
        n = x.shape[0]
        dev = torch.device("cuda", self.plan.device)
        with torch.cuda.device(dev):
            check(load().mck_features_host(self.handle, _ptr(x), n, self.in_dim, _ptr(Cs), _ptr(G),
                                           _ptr(out), _stream(dev)), "mck_features_host")
        return out

    def close(self):
        if self.handle is not None:
            load().mck_host_pipe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def features_host(plan, x, out=None, Cs=None, G=None, chunk_rows=2048, streams=4,
                  pipeline=None):
    """phi(x) for a batch in host memory: x (n, in_dim) float32 on the host
    (pinned, for copies that overlap), out (n, 2 E d) float32 on the host
    (pinned; allocated pinned when None). The batch moves in chunks of
    `chunk_rows` rows over `streams` CUDA streams: each chunk's host-to-device
    copy, feature kernel and device-to-host copy are queued on one stream, so
    the copies of different chunks overlap one another and the kernels. A
    ``HostPipeline`` made once (same plan and in_dim) avoids allocating the
    streams and device buffers on every call.

    Stream-ordered like a non_blocking copy: the current stream waits for
    every chunk, so `out` is complete once the current stream has reached
    this point (synchronise before reading it on the host)."""
    if x.is_cuda or x.dtype != torch.float32 or x.dim() != 2:
        raise TypeError("x must be a 2-d float32 host tensor")
    x = x.contiguous()
    n, in_dim = x.shape
    F = plan.num_features
    if out is None:
        out = torch.empty((n, F), dtype=torch.float32, pin_memory=True)
    elif out.is_cuda or out.dtype != torch.float32 or tuple(out.shape) != (n, F) \
            or not out.is_contiguous():
        raise ValueError("out must be a contiguous (n, 2 E d) float32 host tensor")
    if n == 0:
        return out
    if pipeline is None:
        pipeline = HostPipeline(plan, in_dim, min(int(chunk_rows), n), streams)
    elif pipeline.plan is not plan or pipeline.in_dim != in_dim:
        raise ValueError("pipeline was made for another plan or input width")
    return pipeline.run(x, out, Cs, G)


def features_backward(plan, x, dphi, Cs=None, G=None, need_dx=True, need_dCs=True, need_dG=True,
                      need_dB=False):
    """(dx, dCs, dG) of sum(phi(x) * dphi), and dB (B read as a real
    diagonal) as a fourth entry when ``need_dB``; entries not requested are
    None."""
    _f32_cuda(x, "x", plan.device)
    x, n, in_dim, ld = _rows(x)
    Cs, G = _tables(plan, Cs, G)
    dphi = _f32_cuda(dphi, "dphi", plan.device).contiguous()
    dev = x.device
    dx = torch.empty((n, in_dim), device=dev, dtype=torch.float32) if need_dx else None
    dCs = torch.empty((plan.E, plan.d), device=dev, dtype=torch.float32) if need_dCs else None
    dG = torch.empty((plan.E, plan.d), device=dev, dtype=torch.float32) if need_dG else None
    dB = torch.empty((plan.E, plan.d), device=dev, dtype=torch.float32) if need_dB else None
    if dx is not None and ld != in_dim:
        x = x.contiguous()
        ld = in_dim
    check(load().mck_features_backward_ex(plan.handle, _ptr(x), n, in_dim, ld, _ptr(Cs), _ptr(G),
                                          _ptr(dphi), _ptr(dx), _ptr(dCs), _ptr(dG), _ptr(dB),
                                          _stream(dev)),
          "mck_features_backward")
    return (dx, dCs, dG, dB) if need_dB else (dx, dCs, dG)


def fused_logits(plan, x, W, b=None, Cs=None, G=None, out=None, prec="fp32"):
    """W phi(x) + b without materialising phi: (n, num_classes). prec "fp32"
    contracts with FP32 FMAs (any d); "fp16_split" on the tensor cores (fp16
    hi/lo split of features and weights, FP32 accumulation; d = 1024)."""
    _f32_cuda(x, "x", plan.device)
    x, n, in_dim, ld = _rows(x)
    Cs, G = _tables(plan, Cs, G)
    W = _f32_cuda(W, "W", plan.device).contiguous()
    C = W.size(0)
    if W.dim() != 2 or W.size(1) != plan.num_features:
        raise ValueError(f"W must be (num_classes, {plan.num_features})")
    if b is not None:
        b = _f32_cuda(b, "b", plan.device).contiguous()
    if out is None:
        out = torch.empty((n, C), device=x.device, dtype=torch.float32)
    if prec == "fp32":
        check(load().mck_fused_logits(plan.handle, _ptr(x), n, in_dim, ld, _ptr(Cs), _ptr(G),
                                      _ptr(W), _ptr(b), C, _ptr(out), _stream(x.device)),
              "mck_fused_logits")
    else:
        check(load().mck_fused_logits_ex(plan.handle, _ptr(x), n, in_dim, ld, _ptr(Cs), _ptr(G),
                                         _ptr(W), _ptr(b), C, _ptr(out),
                                         _lib.PRECISIONS[prec] if isinstance(prec, str) else int(prec),
                                         _stream(x.device)), "mck_fused_logits_ex")
    return out


def fused_logits_backward(plan, x, W, dlogits, Cs=None, G=None, need_dx=False, need_dCs=True,
                          need_dG=True, need_dW=True, need_db=True, need_dB=False):
    """Gradients of sum(logits * dlogits) for fused_logits; dict of dx, dCs,
    dG, dB (B read as a real diagonal), dW and db (None where not requested)."""
    _f32_cuda(x, "x", plan.device)
    x, n, in_dim, ld = _rows(x)
    Cs, G = _tables(plan, Cs, G)
    W = _f32_cuda(W, "W", plan.device).contiguous()
    dlogits = _f32_cuda(dlogits, "dlogits", plan.device).contiguous()
    C = W.size(0)
    dev = x.device
    if need_dx and ld != in_dim:
        x = x.contiguous()
        ld = in_dim
    mk = lambda need, shape: torch.empty(shape, device=dev, dtype=torch.float32) if need else None
    g = {"dx": mk(need_dx, (n, in_dim)), "dCs": mk(need_dCs, (plan.E, plan.d)),
         "dG": mk(need_dG, (plan.E, plan.d)), "dB": mk(need_dB, (plan.E, plan.d)),
         "dW": mk(need_dW, tuple(W.shape)), "db": mk(need_db, (C,))}
    check(load().mck_fused_logits_backward_ex(
        plan.handle, _ptr(x), n, in_dim, ld, _ptr(Cs), _ptr(G), _ptr(W), C, _ptr(dlogits),
        _ptr(g["dx"]), _ptr(g["dCs"]), _ptr(g["dG"]), _ptr(g["dB"]), _ptr(g["dW"]), _ptr(g["db"]),
        _stream(dev)),
        "mck_fused_logits_backward")
    return g


def softmax_xent(logits, labels, need_grad=True):
    """(mean cross-entropy as a 0-d tensor, dlogits or None); labels int32."""
    logits = _f32_cuda(logits, "logits").contiguous()
    if labels.dtype != torch.int32 or labels.device != logits.device:
        raise TypeError("labels must be int32 on the logits' device")
    labels = labels.contiguous()
    n, C = logits.shape
    loss = torch.empty((), device=logits.device, dtype=torch.float32)
    dl = torch.empty_like(logits) if need_grad else None
    with torch.cuda.device(logits.device):
        check(load().mck_softmax_xent(_ptr(logits), _ptr(labels), n, C, _ptr(loss), _ptr(dl),
                                      _stream(logits.device)), "mck_softmax_xent")
    return loss, dl


GROUP_ITEM_DTYPE = np.dtype([("plan", "<i4"), ("E", "<i4"), ("in_dim", "<i8"),
                             ("x_offset", "<i8"), ("phi_offset", "<i8")])


class Group:
    """A prepared uneven batch (mck_group_*): every item's features in one persistent launch.

    plans: list of Plan (32 <= d <= 2^14, one device; kept alive by the group).
    items: structured array of GROUP_ITEM_DTYPE, or a sequence of
           (plan_index, E, in_dim, x_offset, phi_offset) tuples.
    x_len, phi_len: element counts of the x and phi arrays passed to features().
    """

    def __init__(self, plans, items, x_len, phi_len, grain=0):
        lib = load()
        self.plans = list(plans)
        arr = np.asarray(items, dtype=GROUP_ITEM_DTYPE) if not (
            isinstance(items, np.ndarray) and items.dtype == GROUP_ITEM_DTYPE) else items
        arr = np.ascontiguousarray(arr)
        handles = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        check(lib.mck_group_create(ctypes.byref(h), handles, len(self.plans),
                                   arr.ctypes.data if len(arr) else None, len(arr), int(x_len),
                                   int(phi_len), int(grain)), "mck_group_create")
        self._h = h
        self.items = arr
        self.x_len, self.phi_len = int(x_len), int(phi_len)
        self.device = self.plans[0].device

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("group is closed")
        return self._h

    def features(self, x, phi):
        """Write every item's features into phi (in place); returns phi."""
        _f32_cuda(x, "x", self.device)
        _f32_cuda(phi, "phi", self.device)
        if x.numel() < self.x_len or phi.numel() < self.phi_len:
            raise ValueError("x or phi smaller than the group's x_len / phi_len")
        check(load().mck_group_features(self.handle, _ptr(x), _ptr(phi), _stream(x.device)),
              "mck_group_features")
        return phi

    def set_grain(self, grain):
        check(load().mck_group_set_grain(self.handle, int(grain)), "mck_group_set_grain")

    def info(self):
        u, s, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        g = ctypes.c_int32()
        check(load().mck_group_info(self.handle, ctypes.byref(u), ctypes.byref(s), ctypes.byref(b),
                                    ctypes.byref(g)), "mck_group_info")
        return {"units": u.value, "warp_steps": s.value, "block_items": b.value,
                "grain": g.value}

    def set_signs(self, B):
        """Replace the sign diagonals: B_e[k] = -1 where B[e, k] < 0, else +1.
        B is a contiguous (E, d) float32 tensor on the plan's device; the
        update is ordered on the current stream."""
        _f32_cuda(B, "B", self.device)
        if tuple(B.shape) != (self.E, self.d) or not B.is_contiguous():
            raise ValueError(f"B must be a contiguous ({self.E}, {self.d}) tensor")
        check(load().mck_plan_set_signs(self.handle, _ptr(B), _stream(B.device)),
              "mck_plan_set_signs")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().mck_group_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CapturedGroup:
    """A Group's launch (counter reset + persistent kernel) captured in a CUDA graph
    for fixed x and phi; replay() re-runs it with one graph launch."""

    def __init__(self, group, x, phi):
        self.group, self.x, self.phi = group, x, phi
        side = torch.cuda.Stream(device=x.device)
        side.wait_stream(torch.cuda.current_stream(x.device))
        with torch.cuda.stream(side):
            group.features(x, phi)  # first call outside capture
        torch.cuda.current_stream(x.device).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            group.features(x, phi)

    def replay(self):
        self.graph.replay()
        return self.phi


def group_layout(plans, plan_index, E, in_dim, order=None):
    """Items for a Group with packed x and phi: item i's input occupies
    x[x_offset : x_offset + in_dim] (slots rounded up to 4 floats) and its
    features phi[phi_offset : phi_offset + 2 E d]. `order` (default: as given)
    sets the packing order. Returns (items, x_len, phi_len)."""
    plan_index = np.asarray(plan_index, dtype=np.int64)
    E = np.asarray(E, dtype=np.int64)
    in_dim = np.asarray(in_dim, dtype=np.int64)
    n = len(plan_index)
    order = np.arange(n) if order is None else np.asarray(order)
    d = np.array([plans[p].d for p in plan_index], dtype=np.int64)
    xs = (in_dim[order] + 3) // 4 * 4
    fs = 2 * E[order] * d[order]
    items = np.zeros(n, dtype=GROUP_ITEM_DTYPE)
    items["plan"][order] = plan_index[order]
    items["E"][order] = E[order]
    items["in_dim"][order] = in_dim[order]
    items["x_offset"][order] = np.concatenate([[0], np.cumsum(xs)[:-1]]) if n else []
    items["phi_offset"][order] = np.concatenate([[0], np.cumsum(fs)[:-1]]) if n else []
    return items, int(xs.sum()), int(fs.sum())
