"""Torch-facing binding of libdegraf.so: argument marshalling only.

Every step of detection, pyramid construction and tracking runs in the library's
CUDA kernels; torch supplies device memory and the current stream. Functions
raise DegrafError with the library's status text on any failure.
"""
from __future__ import annotations

import ctypes
import dataclasses
import threading

import torch

from . import _abi, tune
from ._abi import F16, F32, check, load


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _frame(frame: torch.Tensor):
    if frame.dtype != torch.uint8 or frame.dim() != 2 or not frame.is_cuda:
        raise ValueError("frame must be a 2-D uint8 CUDA tensor")
    if frame.stride(1) != 1:
        raise ValueError("frame rows must be contiguous")
    H, W = frame.shape
    return W, H, frame.stride(0)


def _nbytes(t: torch.Tensor) -> int:
    return t.numel() * t.element_size()


def _points(pts: torch.Tensor, name: str = "pts") -> int:
    """Number of points of a contiguous float32 CUDA tensor [n, 2]."""
    if pts.dtype != torch.float32 or pts.dim() != 2 or pts.shape[1] != 2 or not pts.is_contiguous() or not pts.is_cuda:
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor [n, 2]")
    return pts.shape[0]


def _buffer(t, name: str, dtype, shape, device):
    """Checks a caller's buffer (the kernels write or read every element of it); None passes."""
    if t is not None and (t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous()
                          or t.device != device):
        raise ValueError(f"{name} must be a contiguous {dtype} tensor {list(shape)} on {device}")
    return t


def _bytes_buffer(t: torch.Tensor, name: str, device) -> torch.Tensor:
    """A byte buffer (pyramid or workspace): contiguous uint8 on the device."""
    if t.dtype != torch.uint8 or not t.is_contiguous() or t.device != device:
        raise ValueError(f"{name} must be a contiguous uint8 tensor on {device}")
    return t


def _grad_plane(g: torch.Tensor, name: str, W: int, H: int, device) -> None:
    """A float32 [H, W] gradient image with unit column stride (rows may be padded)."""
    if (g.dtype != torch.float32 or tuple(g.shape) != (H, W) or g.stride(1) != 1 or g.stride(0) < W
            or g.device != device):
        raise ValueError(f"{name} must be a float32 tensor [{H}, {W}] with contiguous rows on {device}")


def _pyramids(pyr1, pyr2, W: int, H: int, levels: int, storage: int, device, grad2: bool = False):
    """The tracker reads frame 1's pyramid at the offsets of a `levels`-level pyramid with
    gradients, and frame 2's intensity planes (a prefix of any pyramid with at least
    `levels` levels; with grad2, frame 2's gradients too, at the offsets of exactly
    `levels` levels): check both buffers against those layouts."""
    _bytes_buffer(pyr1, "pyr1", device)
    _bytes_buffer(pyr2, "pyr2", device)
    need1 = pyramid_bytes(W, H, levels, storage, True)
    need2 = pyramid_bytes(W, H, levels, storage, grad2)
    if need1 and pyr1.numel() != need1:  # 0: invalid sizes, which the library reports itself
        raise ValueError(f"pyr1 must be a {levels}-level pyramid with gradients ({need1} bytes)")
    if need2 and (pyr2.numel() != need2 if grad2 else pyr2.numel() < need2):
        raise ValueError(f"pyr2 must hold a {levels}-level pyramid{' with gradients' if grad2 else ''} "
                         f"({need2} bytes)")


@dataclasses.dataclass
class RlofParams:
    """Tracking parameters (mirror of dgf_rlof_params)."""

    levels: int = 3
    radius: int = 4
    max_iter: int = 30
    model: int = 4
    storage: int = F32
    eps: float = 1e-3
    hampel_a: float = 8.0
    hampel_b: float = 16.0
    hampel_c: float = 32.0
    min_eig: float = 1e-3
    cross_tau: float = 0.0  # adaptive cross-based support threshold; 0 keeps the square support

    def c(self) -> _abi.RlofParamsC:
        return _abi.RlofParamsC(_abi.RLOF_PARAMS_VERSION, self.levels, self.radius, self.max_iter,
                                self.model, self.storage, self.eps, self.hampel_a, self.hampel_b,
                                self.hampel_c, self.min_eig, self.cross_tau)


@dataclasses.dataclass
class GmParams:
    """Global-motion prior parameters (mirror of dgf_gm_params)."""

    stride: int = 4
    extra_levels: int = 2
    iters: int = 8
    c0: float = 32.0
    c_min: float = 2.0

    def c(self) -> _abi.GmParamsC:
        return _abi.GmParamsC(_abi.GM_PARAMS_VERSION, self.stride, self.extra_levels, self.iters, self.c0,
                              self.c_min)


@dataclasses.dataclass
class EpicParams:
    """EPIC interpolation parameters (mirror of dgf_epic_params; k = 128 as in the paper)."""

    k: int = 128
    model: int = 1  # 1: locally affine, 0: weighted mean
    cost_base: int = 4
    cost_gain: int = 1
    a: float = 0.1
    min_spread: float = 1.0

    def c(self) -> _abi.EpicParamsC:
        return _abi.EpicParamsC(_abi.EPIC_PARAMS_VERSION, self.k, self.model, self.cost_base, self.cost_gain, self.a,
                                self.min_spread)


def device_status(reset: bool = False) -> int:
    """Thread blocks of detection or the pyramid that gave up waiting for their
    staging copies on the current device since the last reset (0: every launch ran
    to the end). Synchronises the device."""
    v = ctypes.c_uint(0)
    check("dgf_device_status", load().dgf_device_status(ctypes.byref(v), int(reset)))
    return int(v.value)


def version() -> int:
    return int(load().dgf_version())


def degraf_count(W: int, H: int, win: int, step: int, win_h: int | None = None) -> int:
    n = int(load().dgf_degraf_count(W, H, win, win if win_h is None else win_h, step))
    if n < 0:
        raise _abi.DegrafError("dgf_degraf_count", _abi.DGF_ERR_ARG, "invalid argument")
    return n


def detect(frame: torch.Tensor, win: int, step: int, win_h: int | None = None,
           with_sums: bool = False, out: torch.Tensor | None = None):
    """DeGraF key-points of a uint8 frame: float32 [N, 2] (and int32 [N, 4] sums)."""
    W, H, pitch = _frame(frame)
    wh = win if win_h is None else win_h
    n = degraf_count(W, H, win, step, wh)
    pts = (_buffer(out, "out", torch.float32, (n, 2), frame.device) if out is not None
           else torch.empty((n, 2), dtype=torch.float32, device=frame.device))
    sums = torch.empty((n, 4), dtype=torch.int32, device=frame.device) if with_sums else None
    check("degraf_detect", load().degraf_detect(_ptr(frame), W, H, pitch, win, wh, step, _ptr(pts),
                                                _ptr(sums), _stream()))
    return (pts, sums) if with_sums else pts


def pyramid_layout(W: int, H: int, levels: int, storage: int = F32, with_grad: bool = True) -> dict:
    L = _abi.PyramidLayout()
    check("dgf_pyramid_layout_get",
          load().dgf_pyramid_layout_get(W, H, levels, storage, int(with_grad), ctypes.byref(L)))
    n = L.levels
    return dict(levels=n, storage=L.storage, with_grad=bool(L.with_grad), W=list(L.W[:n]),
                H=list(L.H[:n]), pitch=list(L.pitch[:n]), off_I=list(L.off_I[:n]),
                off_Ix=list(L.off_Ix[:n]), off_Iy=list(L.off_Iy[:n]), bytes=int(L.bytes))


def pyramid_bytes(W: int, H: int, levels: int, storage: int = F32, with_grad: bool = True) -> int:
    return int(load().dgf_pyramid_bytes(W, H, levels, storage, int(with_grad)))


def build_pyramid(frame: torch.Tensor, levels: int, storage: int = F32, with_grad: bool = True,
                  out: torch.Tensor | None = None) -> torch.Tensor:
    """Pyramid buffer (uint8 tensor laid out as pyramid_layout describes)."""
    W, H, pitch = _frame(frame)
    nbytes = pyramid_bytes(W, H, levels, storage, with_grad)
    buf = _bytes_buffer(out, "out", frame.device) if out is not None else torch.empty(
        nbytes, dtype=torch.uint8, device=frame.device)
    check("pyramid_build", load().pyramid_build(_ptr(frame), W, H, pitch, levels, storage,
                                                int(with_grad), _ptr(buf), buf.numel(), _stream()))
    return buf


def pyramid_planes(buf: torch.Tensor, layout: dict):
    """[(I, Ix, Iy)] per level as float32/float16 views [H_l, W_l] into buf."""
    dt = torch.float32 if layout["storage"] == F32 else torch.float16
    es = 4 if dt == torch.float32 else 2
    out = []
    for l in range(layout["levels"]):
        Wl, Hl, p = layout["W"][l], layout["H"][l], layout["pitch"][l]

        def plane(off):
            return buf[off: off + p * Hl * es].view(dt).view(Hl, p)[:, :Wl]

        grads = (plane(layout["off_Ix"][l]), plane(layout["off_Iy"][l])) if layout["with_grad"] else (None, None)
        out.append((plane(layout["off_I"][l]), *grads))
    return out


# The lanes setting is process-wide; a BatchTracker holds this lock from setting its
# own value to restoring the previous one, so concurrent trackers never see each
# other's value.
_lanes_lock = threading.Lock()


def set_lanes(lanes: int) -> int:
    prev = int(load().dgf_rlof_set_lanes(lanes))
    if prev < 0:
        raise _abi.DegrafError("dgf_rlof_set_lanes", prev, "lanes must be 0, 8, 16 or 32")
    return prev


def track(pyr1: torch.Tensor, pyr2: torch.Tensor, W: int, H: int, pts: torch.Tensor, params: RlofParams,
          with_iters: bool = False, with_illum: bool = False, out=None):
    """RLOF tracking of pts [n, 2] (float32, CUDA): returns flow, status[, iters][, illum].
    pyr1 is frame 1's pyramid with gradients and params.levels levels; out = (flow,
    status, iters or None, illum or None) are caller buffers."""
    n = _points(pts)
    dev = pts.device
    _pyramids(pyr1, pyr2, W, H, params.levels, params.storage, dev)
    if out is None:
        flow = torch.empty((n, 2), dtype=torch.float32, device=dev)
        status = torch.empty(n, dtype=torch.uint8, device=dev)
        iters = torch.empty(n, dtype=torch.uint8, device=dev) if with_iters else None
        illum = torch.empty((n, 2), dtype=torch.float32, device=dev) if with_illum else None
    else:
        flow, status, iters, illum = out
        _buffer(flow, "flow", torch.float32, (n, 2), dev)
        _buffer(status, "status", torch.uint8, (n,), dev)
        _buffer(iters, "iters", torch.uint8, (n,), dev)
        _buffer(illum, "illum", torch.float32, (n, 2), dev)
    prm = params.c()
    check("rlof_track", load().rlof_track(_ptr(pyr1), _ptr(pyr2), W, H, _ptr(pts), n, ctypes.byref(prm),
                                          _ptr(flow), _ptr(status), _ptr(iters), _ptr(illum), _stream()))
    res = [flow, status]
    if with_iters:
        res.append(iters)
    if with_illum:
        res.append(illum)
    return tuple(res)


def gm_workspace_bytes(n: int, gm: GmParams) -> int:
    return int(load().dgf_gm_workspace(n, ctypes.byref(gm.c())))


def track_gm(pyr1: torch.Tensor, pyr2: torch.Tensor, W: int, H: int, pyr_levels: int, pts: torch.Tensor,
             params: RlofParams, gm: GmParams | None = None, with_iters: bool = False, with_illum: bool = False,
             workspace: torch.Tensor | None = None):
    """Tracking with the global-motion prior (rlof_track_gm): the pyramids were built
    with pyr_levels >= params.levels + gm.extra_levels levels. Returns flow, status
    [, iters][, illum], then the fitted affine (float64 [6], device) and its flag
    (int32 [1], device; 1 = fitted)."""
    gm = gm or GmParams()
    n = _points(pts)
    dev = pts.device
    _pyramids(pyr1, pyr2, W, H, pyr_levels, params.storage, dev)
    flow = torch.empty((n, 2), dtype=torch.float32, device=dev)
    status = torch.empty(n, dtype=torch.uint8, device=dev)
    iters = torch.empty(n, dtype=torch.uint8, device=dev) if with_iters else None
    illum = torch.empty((n, 2), dtype=torch.float32, device=dev) if with_illum else None
    need = gm_workspace_bytes(n, gm)
    if workspace is None:
        workspace = torch.zeros(max(need, 256), dtype=torch.uint8, device=dev)
    _bytes_buffer(workspace, "workspace", dev)
    prm, g = params.c(), gm.c()
    check("rlof_track_gm", load().rlof_track_gm(_ptr(pyr1), _ptr(pyr2), W, H, pyr_levels, _ptr(pts), n,
                                                ctypes.byref(prm), ctypes.byref(g), _ptr(flow), _ptr(status),
                                                _ptr(iters), _ptr(illum), _ptr(workspace), workspace.numel(),
                                                _stream()))
    res = [flow, status]
    if with_iters:
        res.append(iters)
    if with_illum:
        res.append(illum)
    res.append(workspace[:48].view(torch.float64))
    res.append(workspace[48:52].view(torch.int32))
    return tuple(res)


def track_fb(pyr1: torch.Tensor, pyr2: torch.Tensor, W: int, H: int, pts: torch.Tensor, params: RlofParams,
             fb_max: float = 0.0, workspace: torch.Tensor | None = None):
    """Forward-backward consistency filter (rlof_track_fb): both pyramids built with
    gradients. Returns flow, status (FB_REJECTED where the round-trip error exceeds
    fb_max > 0) and the round-trip error (float32 [n], +inf where a pass lost the point)."""
    n = _points(pts)
    dev = pts.device
    _pyramids(pyr1, pyr2, W, H, params.levels, params.storage, dev, grad2=True)
    flow = torch.empty((n, 2), dtype=torch.float32, device=dev)
    status = torch.empty(n, dtype=torch.uint8, device=dev)
    err = torch.empty(n, dtype=torch.float32, device=dev)
    if workspace is None:
        workspace = torch.empty(max(int(load().dgf_fb_workspace(n)), 256), dtype=torch.uint8, device=dev)
    _bytes_buffer(workspace, "workspace", dev)
    nbytes = min(pyr1.numel(), pyr2.numel())
    prm = params.c()
    check("rlof_track_fb", load().rlof_track_fb(_ptr(pyr1), _ptr(pyr2), nbytes, W, H, _ptr(pts), n, ctypes.byref(prm),
                                                float(fb_max), _ptr(flow), _ptr(status), _ptr(err), _ptr(workspace),
                                                workspace.numel(), _stream()))
    return flow, status, err


def epic_workspace_bytes(W: int, H: int, n: int) -> int:
    return int(load().dgf_epic_workspace(W, H, n))


def epic_interpolate(frame: torch.Tensor, pts: torch.Tensor, flow: torch.Tensor, status: torch.Tensor,
                     params: EpicParams = EpicParams(), debug: bool = False, workspace: torch.Tensor | None = None,
                     out: torch.Tensor | None = None):
    """Dense flow (float32 [H, W, 2]) from sparse matches by EPIC interpolation
    (epic_interpolate). With debug=True also returns a dict of the labels, geodesic
    distances, neighbourhoods, per-seed models and fit kinds."""
    W, H, pitch = _frame(frame)
    dev = frame.device
    n = _points(pts)
    _buffer(pts, "pts", torch.float32, (n, 2), dev)
    _buffer(flow, "flow", torch.float32, (n, 2), dev)
    _buffer(status, "status", torch.uint8, (n,), dev)
    dense = (_buffer(out, "out", torch.float32, (H, W, 2), dev) if out is not None
             else torch.empty((H, W, 2), dtype=torch.float32, device=dev))
    if workspace is None:
        workspace = torch.empty(max(epic_workspace_bytes(W, H, n), 256), dtype=torch.uint8, device=dev)
    _bytes_buffer(workspace, "workspace", dev)
    out = None
    dbg = None
    if debug:
        k = params.k
        out = {"labels": torch.empty((H, W), dtype=torch.int32, device=dev),
               "dist": torch.empty((H, W), dtype=torch.int64, device=dev),
               "knn_idx": torch.full((n, k), -1, dtype=torch.int32, device=dev),
               "knn_dist": torch.full((n, k), -1, dtype=torch.int64, device=dev),
               "knn_count": torch.empty(n, dtype=torch.int32, device=dev),
               "models": torch.empty((n, 6), dtype=torch.float64, device=dev),
               "fit_kind": torch.empty(n, dtype=torch.uint8, device=dev),
               "retried": torch.zeros(1, dtype=torch.int32, device=dev)}
        dbg = _abi.EpicDebugC(*(_ptr(out[f]) for f, _ in _abi.EpicDebugC._fields_))
    prm = params.c()
    check("epic_interpolate", load().epic_interpolate(
        _ptr(frame), W, H, pitch, _ptr(pts), _ptr(flow), _ptr(status), n, ctypes.byref(prm), _ptr(dense),
        ctypes.byref(dbg) if dbg is not None else None, _ptr(workspace), workspace.numel(), _stream()))
    return (dense, out) if debug else dense


def detect_backward(frame: torch.Tensor, win: int, step: int, grad_pts: torch.Tensor, win_h: int | None = None,
                    grad_img: torch.Tensor | None = None) -> torch.Tensor:
    """Adds sum_k grad_pts[k] . d(point_k)/d(frame) into grad_img (float32 [H, W])."""
    W, H, pitch = _frame(frame)
    wh = win if win_h is None else win_h
    n = degraf_count(W, H, win, step, wh)
    if grad_img is None:
        grad_img = torch.zeros((H, W), dtype=torch.float32, device=frame.device)
    _grad_plane(grad_img, "grad_img", W, H, frame.device)
    grad_pts = grad_pts.contiguous().float()
    _buffer(grad_pts, "grad_pts", torch.float32, (n, 2), frame.device)
    ws = torch.empty(int(load().dgf_degraf_backward_workspace(W, H, win, wh, step)), dtype=torch.uint8,
                     device=frame.device)
    check("degraf_detect_backward", load().degraf_detect_backward(
        _ptr(frame), W, H, pitch, win, wh, step, _ptr(grad_pts), _ptr(ws), ws.numel(), _ptr(grad_img),
        grad_img.stride(0), _stream()))
    return grad_img


def track_backward(pyr1, pyr2, W: int, H: int, pts, params: RlofParams, flow, illum, status, grad_flow,
                   grad_illum=None, grad_I1=None, grad_I2=None):
    """Adds the implicit-function VJP of tracking into (grad_I1, grad_I2) float32 [H, W]
    (rows of both planes equally far apart)."""
    n = _points(pts)
    dev = pts.device
    _pyramids(pyr1, pyr2, W, H, params.levels, params.storage, dev)
    if grad_I1 is None:
        grad_I1 = torch.zeros((H, W), dtype=torch.float32, device=dev)
    if grad_I2 is None:
        grad_I2 = torch.zeros((H, W), dtype=torch.float32, device=dev)
    _grad_plane(grad_I1, "grad_I1", W, H, dev)
    _grad_plane(grad_I2, "grad_I2", W, H, dev)
    if grad_I1.stride(0) != grad_I2.stride(0):
        raise ValueError("grad_I1 and grad_I2 rows must be equally far apart")
    _buffer(flow, "flow", torch.float32, (n, 2), dev)
    _buffer(illum, "illum", torch.float32, (n, 2), dev)
    _buffer(status, "status", torch.uint8, (n,), dev)
    ws = torch.empty(int(load().dgf_rlof_backward_workspace(W, H)), dtype=torch.uint8, device=dev)
    grad_flow = _buffer(grad_flow.contiguous().float(), "grad_flow", torch.float32, (n, 2), dev)
    gi = (_buffer(grad_illum.contiguous().float(), "grad_illum", torch.float32, (n, 2), dev)
          if grad_illum is not None else None)
    prm = params.c()
    check("rlof_track_backward", load().rlof_track_backward(
        _ptr(pyr1), _ptr(pyr2), W, H, _ptr(pts), pts.shape[0], ctypes.byref(prm), _ptr(flow), _ptr(illum),
        _ptr(status), _ptr(grad_flow), _ptr(gi), _ptr(ws), ws.numel(), _ptr(grad_I1), _ptr(grad_I2),
        grad_I1.stride(0), _stream()))
    return grad_I1, grad_I2


def _as_u8(frame: torch.Tensor) -> torch.Tensor:
    return frame.detach().round().clamp(0, 255).to(torch.uint8).contiguous()


class DeGraFDetect(torch.autograd.Function):
    """Key-points of a frame given as float intensities (rounded to uint8 for the
    forward); backward is degraf_detect_backward."""

    @staticmethod
    def forward(ctx, frame: torch.Tensor, win: int, step: int):
        u8 = _as_u8(frame)
        ctx.save_for_backward(u8)
        ctx.win, ctx.step = win, step
        return detect(u8, win, step)

    @staticmethod
    def backward(ctx, grad_pts):
        (u8,) = ctx.saved_tensors
        return detect_backward(u8, ctx.win, ctx.step, grad_pts), None, None


class RLOFTrack(torch.autograd.Function):
    """Flow of fixed key-points from frame 1 to frame 2 (float intensities, rounded
    to uint8 for the forward); backward is rlof_track_backward (gradients for both
    frames, none for the key-points or the parameters). Returns flow and status.

    The key-points must not require grad: the flow's derivative with respect to
    them is not computed, so a chain such as DeGraFDetect -> RLOFTrack would silently
    lose the path flow -> key-points -> frame 1. forward raises instead; detach the
    key-points to differentiate through the frames only."""

    @staticmethod
    def forward(ctx, frame1: torch.Tensor, frame2: torch.Tensor, pts: torch.Tensor, params: RlofParams):
        if pts.requires_grad:
            raise ValueError("RLOFTrack: the key-points require grad, but the flow's derivative with respect to "
                             "them is not computed; pass pts.detach() to differentiate through the frames only")
        f1, f2 = _as_u8(frame1), _as_u8(frame2)
        H, W = f1.shape
        pyr1 = build_pyramid(f1, params.levels, params.storage, True)
        pyr2 = build_pyramid(f2, params.levels, params.storage, False)
        pts = pts.detach().contiguous().float()
        flow, status, illum = track(pyr1, pyr2, W, H, pts, params, with_illum=True)
        ctx.save_for_backward(pyr1, pyr2, pts, flow, illum, status)
        ctx.params, ctx.W, ctx.H = params, W, H
        ctx.mark_non_differentiable(status)
        return flow, status

    @staticmethod
    def backward(ctx, grad_flow, grad_status):
        pyr1, pyr2, pts, flow, illum, status = ctx.saved_tensors
        g1, g2 = track_backward(pyr1, pyr2, ctx.W, ctx.H, pts, ctx.params, flow, illum, status, grad_flow)
        return g1, g2, None, None


class PairTracker:
    """Device-resident DeGraF + RLOF for frame pairs of one size and parameter set.

    Buffers (pyramids, points, outputs) are allocated once; ``run`` enqueues
    detection, both pyramid builds and tracking on the current stream.
    """

    def __init__(self, W: int, H: int, win: int, step: int, params: RlofParams,
                 device: torch.device | str = "cuda"):
        self.W, self.H, self.win, self.step, self.params = W, H, win, step, params
        self.device = torch.device(device)
        self.n = degraf_count(W, H, win, step)
        st = params.storage
        self.pyr1 = torch.empty(pyramid_bytes(W, H, params.levels, st, True), dtype=torch.uint8,
                                device=self.device)
        self.pyr2 = torch.empty(pyramid_bytes(W, H, params.levels, st, False), dtype=torch.uint8,
                                device=self.device)
        self.pts = torch.empty((self.n, 2), dtype=torch.float32, device=self.device)
        self.flow = torch.empty((self.n, 2), dtype=torch.float32, device=self.device)
        self.status = torch.empty(self.n, dtype=torch.uint8, device=self.device)
        self.iters = torch.empty(self.n, dtype=torch.uint8, device=self.device)

    def run(self, frame1: torch.Tensor, frame2: torch.Tensor):
        p = self.params
        detect(frame1, self.win, self.step, out=self.pts)
        build_pyramid(frame1, p.levels, p.storage, True, out=self.pyr1)
        build_pyramid(frame2, p.levels, p.storage, False, out=self.pyr2)
        track(self.pyr1, self.pyr2, self.W, self.H, self.pts, p,
              out=(self.flow, self.status, self.iters, None))
        return self.pts, self.flow, self.status, self.iters


class BatchTracker:
    """Batched DeGraF + pyramids + RLOF over frame pairs of mixed sizes and steps.

    ``specs`` is a list of (W, H, win, step). Outputs (points, flow, status,
    iterations) and the workspace are allocated once; ``run`` takes lists of
    uint8 frames (device tensors of the spec sizes) and enqueues one
    rlof_track_many call (optionally replayed from a captured CUDA graph);
    ``bind`` + ``run()`` reuse validated descriptors of fixed frame buffers.
    """

    def __init__(self, specs, params: RlofParams, device: torch.device | str = "cuda", lanes=0):
        self.specs = [tuple(int(v) for v in sp) for sp in specs]
        self.params = params
        self.device = torch.device(device)
        self.n = [degraf_count(W, H, win, step) for (W, H, win, step) in self.specs]
        # lanes per tracked point: 0 = the library's choice, 8 / 16 / 32, or "auto" =
        # the autotuner's cached choice for this GPU, parameters and batch size
        self.lanes = (tune.lookup(self.tune_key()) or 0) if lanes == "auto" else int(lanes)
        dev = self.device
        self.pts = [torch.empty((n, 2), dtype=torch.float32, device=dev) for n in self.n]
        self.flow = [torch.empty((n, 2), dtype=torch.float32, device=dev) for n in self.n]
        self.status = [torch.empty(n, dtype=torch.uint8, device=dev) for n in self.n]
        self.iters = [torch.empty(n, dtype=torch.uint8, device=dev) for n in self.n]
        self._prm = params.c()
        probe = self._descriptors([None] * len(self.specs), [None] * len(self.specs), probe=True)
        nbytes = int(load().dgf_track_many_workspace(probe, len(self.specs), ctypes.byref(self._prm)))
        if nbytes == 0:
            raise _abi.DegrafError("dgf_track_many_workspace", _abi.DGF_ERR_ARG, "invalid batch")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self._arr = None

    def _descriptors(self, frames1, frames2, probe=False):
        arr = (_abi.PairC * len(self.specs))()
        for i, (W, H, win, step) in enumerate(self.specs):
            f1, f2 = frames1[i], frames2[i]
            if probe:
                p1 = p2 = 1 << 20  # placeholders: the size query dereferences nothing
                pitch = W
            else:
                if f1.shape != (H, W) or f2.shape != (H, W) or f1.stride(0) != f2.stride(0):
                    raise ValueError(f"pair {i}: frames must be {H}x{W} with equal pitch")
                _frame(f1)
                _frame(f2)
                p1, p2, pitch = f1.data_ptr(), f2.data_ptr(), f1.stride(0)
            arr[i] = _abi.PairC(p1, p2, W, H, pitch, win, step, self.pts[i].data_ptr(), self.flow[i].data_ptr(),
                                self.status[i].data_ptr(), self.iters[i].data_ptr())
        return arr

    def bind(self, frames1, frames2):
        """Validates the frames and builds the pair descriptors once. The tracker
        keeps references to the frames, so their memory stays valid; later
        ``run()`` calls without frames track whatever the frames then hold."""
        self._bound = (list(frames1), list(frames2))
        self._arr = self._descriptors(*self._bound)

    def run(self, frames1=None, frames2=None, use_graph: bool = True, stages: int = _abi.STAGE_ALL):
        if frames1 is not None or frames2 is not None:
            self.bind(frames1, frames2)
        elif getattr(self, "_arr", None) is None:
            raise ValueError("run() without frames needs frames bound first")
        def call():
            check("rlof_track_many", load().rlof_track_many(self._arr, len(self.specs), ctypes.byref(self._prm),
                                                            _ptr(self.workspace), self.workspace.numel(), int(stages),
                                                            int(use_graph), _stream()))

        with _lanes_lock:  # this tracker's setting (0 = the library's choice) for exactly this call
            prev = set_lanes(self.lanes)
            try:
                call()
            finally:
                set_lanes(prev)
        return self.pts, self.flow, self.status, self.iters

    def tune_key(self) -> str:
        return tune.key(torch.cuda.get_device_name(self.device), self.params, sum(self.n))

    def autotune(self, frames1=None, frames2=None, reps: int = 5, path: str | None = None) -> dict:
        """Times the whole batch (detection, pyramids, tracking; graph replay) for
        every lane count the library honours at this radius, keeps the fastest for
        this tracker and records it in the autotuner's cache. Returns the record."""
        if frames1 is not None or frames2 is not None:
            self.bind(frames1, frames2)
        stream = torch.cuda.current_stream(self.device)

        def measure(lanes: int) -> float:
            self.lanes = lanes
            for _ in range(2):
                self.run()
            torch.cuda.synchronize(self.device)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                self.run()
            b.record(stream)
            b.synchronize()
            return a.elapsed_time(b) / reps

        rec = tune.tune(measure, self.params.radius, self.tune_key(), path)
        self.lanes = rec["lanes"]
        return rec


class DenseFlow:
    """The DeGraF-Flow pipeline for one frame size (Section 2): DeGraF key-points on
    frame 1, RLOF tracking into frame 2 (with the global-motion prior, the paper's
    RLOF(IM-GM), unless gm is None), optionally the forward-backward filter
    (fb_max > 0; both pyramids then carry gradients), and EPIC interpolation of the
    tracked points into a dense flow field. Pyramids, key-points, workspaces and the
    dense field are allocated once; ``run`` returns the dense field [H, W, 2] and the
    sparse (points, flow, status). A run only enqueues work on the current stream (no
    host round trip; device-side failures go to ``device_status``), so it may be
    captured into a CUDA graph once it has run eagerly on the device."""

    def __init__(self, W: int, H: int, win: int, step: int, params: RlofParams, gm: GmParams | None = None,
                 epic: EpicParams | None = None, fb_max: float = 0.0, device: torch.device | str = "cuda"):
        if gm is not None and fb_max > 0:
            raise ValueError("choose the global-motion prior or the forward-backward filter")
        self.W, self.H, self.win, self.step = W, H, win, step
        self.params, self.gm, self.fb_max = params, gm, float(fb_max)
        self.epic = epic or EpicParams()
        self.device = dev = torch.device(device)
        self.levels = params.levels + (gm.extra_levels if gm is not None else 0)
        grad2 = self.fb_max > 0
        self.pyr1 = torch.empty(pyramid_bytes(W, H, self.levels, params.storage, True), dtype=torch.uint8, device=dev)
        self.pyr2 = torch.empty(pyramid_bytes(W, H, self.levels, params.storage, grad2), dtype=torch.uint8,
                                device=dev)
        self.n = degraf_count(W, H, win, step)
        self.pts = torch.empty((self.n, 2), dtype=torch.float32, device=dev)
        self.dense = torch.empty((H, W, 2), dtype=torch.float32, device=dev)
        self.ws_epic = torch.empty(max(epic_workspace_bytes(W, H, self.n), 256), dtype=torch.uint8, device=dev)
        self.ws_gm = (torch.zeros(max(gm_workspace_bytes(self.n, gm), 256), dtype=torch.uint8, device=dev)
                      if gm is not None else None)
        self.ws_fb = (torch.empty(max(int(load().dgf_fb_workspace(self.n)), 256), dtype=torch.uint8, device=dev)
                      if grad2 else None)

    def run(self, frame1: torch.Tensor, frame2: torch.Tensor):
        prm = self.params
        detect(frame1, self.win, self.step, out=self.pts)
        build_pyramid(frame1, self.levels, prm.storage, True, out=self.pyr1)
        build_pyramid(frame2, self.levels, prm.storage, self.fb_max > 0, out=self.pyr2)
        if self.gm is not None:
            flow, status = track_gm(self.pyr1, self.pyr2, self.W, self.H, self.levels, self.pts, prm, self.gm,
                                    workspace=self.ws_gm)[:2]
        elif self.fb_max > 0:
            flow, status, _ = track_fb(self.pyr1, self.pyr2, self.W, self.H, self.pts, prm, self.fb_max,
                                       workspace=self.ws_fb)
        else:
            flow, status = track(self.pyr1, self.pyr2, self.W, self.H, self.pts, prm)
        epic_interpolate(frame1, self.pts, flow, status, self.epic, workspace=self.ws_epic, out=self.dense)
        return self.dense, (self.pts, flow, status)


class HostPairTracker:
    """Host frames in, host results out, for frame pairs of one size and parameter set.

    The device copies of the two frames, the batched tracker (detection, both
    pyramids and tracking replayed from one captured CUDA graph) and pinned host
    outputs are allocated once. ``run`` copies the two host frames to the device,
    enqueues the pair, copies points, flow and status back to host memory and waits
    for them, so a call allocates nothing on the device after the first.
    """

    def __init__(self, W: int, H: int, win: int, step: int, params: RlofParams,
                 device: torch.device | str = "cuda", lanes=0):
        self.W, self.H = int(W), int(H)
        self.device = dev = torch.device(device)
        if dev.type != "cuda":
            raise ValueError("HostPairTracker runs on a CUDA device")
        with torch.cuda.device(dev):
            self.d1 = torch.empty((self.H, self.W), dtype=torch.uint8, device=dev)
            self.d2 = torch.empty((self.H, self.W), dtype=torch.uint8, device=dev)
            self.tracker = BatchTracker([(self.W, self.H, win, step)], params, dev, lanes=lanes)
            self.tracker.bind([self.d1], [self.d2])
        self.n = self.tracker.n[0]
        self.pts = torch.empty((self.n, 2), dtype=torch.float32).pin_memory()
        self.flow = torch.empty((self.n, 2), dtype=torch.float32).pin_memory()
        self.status = torch.empty(self.n, dtype=torch.uint8).pin_memory()

    def _host_frame(self, frame, name: str) -> torch.Tensor:
        f = torch.as_tensor(frame)
        if f.dtype != torch.uint8 or tuple(f.shape) != (self.H, self.W) or f.is_cuda:
            raise ValueError(f"{name} must be a host uint8 array of shape ({self.H}, {self.W})")
        return f

    def run(self, frame1, frame2, out=None):
        """Tracks one pair of host frames (numpy arrays or CPU tensors; pinned memory
        makes the copies asynchronous). Returns host (pts, flow, status): the given
        ``out`` tensors (contiguous, on the host, of the output shapes and dtypes), else
        this tracker's own pinned buffers, which the next call overwrites."""
        h1 = self._host_frame(frame1, "frame1")
        h2 = self._host_frame(frame2, "frame2")
        if out is None:
            out = (self.pts, self.flow, self.status)
        cpu = torch.device("cpu")
        o_pts = _buffer(out[0], "pts", torch.float32, (self.n, 2), cpu)
        o_flow = _buffer(out[1], "flow", torch.float32, (self.n, 2), cpu)
        o_status = _buffer(out[2], "status", torch.uint8, (self.n,), cpu)
        tr = self.tracker
        with torch.cuda.device(self.device):
            self.d1.copy_(h1, non_blocking=True)
            self.d2.copy_(h2, non_blocking=True)
            tr.run(use_graph=True)
            o_pts.copy_(tr.pts[0], non_blocking=True)
            o_flow.copy_(tr.flow[0], non_blocking=True)
            o_status.copy_(tr.status[0], non_blocking=True)
            torch.cuda.current_stream(self.device).synchronize()
        return o_pts, o_flow, o_status


_host_trackers: dict = {}
_host_trackers_lock = threading.Lock()
_HOST_TRACKERS_KEPT = 4


def track_pair(frame1, frame2, win: int, step: int, params: RlofParams, device="cuda"):
    """End-to-end call on host frames: returns host (pts, flow, status).

    The frames (uint8 numpy arrays or CPU tensors of equal shape) are copied to the
    device, detected, pyramided and tracked there, and the results copied back. The
    device buffers of a frame size and parameter set are made on its first call and
    kept (the last few sizes), so later calls of that size allocate nothing on the
    device; the returned tensors are the caller's own.
    """
    f1 = torch.as_tensor(frame1)
    f2 = torch.as_tensor(frame2)
    if f1.dim() != 2 or f1.shape != f2.shape:
        raise ValueError("frames must be 2-D arrays of equal shape")
    H, W = f1.shape
    dev = torch.device(device)
    if dev.type == "cuda" and dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    key = (W, H, win, step, dataclasses.astuple(params), str(dev))
    with _host_trackers_lock:
        ht = _host_trackers.pop(key, None)
        if ht is None:
            ht = HostPairTracker(W, H, win, step, params, dev)
        _host_trackers[key] = ht  # most recently used last
        while len(_host_trackers) > _HOST_TRACKERS_KEPT:
            _host_trackers.pop(next(iter(_host_trackers)))
        pts, flow, status = ht.run(f1, f2)
        return pts.clone(), flow.clone(), status.clone()
