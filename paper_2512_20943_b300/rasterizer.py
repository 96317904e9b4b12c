"""Python binding of libairgs: argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module checks
tensor devices/dtypes/shapes, passes raw device pointers through the C ABI and
wraps render / render_backward in a torch.autograd.Function.  PyTorch provides
device memory and streams.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _abi
from ._abi import (AIRGS_DELTA_ANCHOR, AIRGS_DELTA_PREV, AIRGS_QUAT_ADD, airgs_backward_args, airgs_camera,
                   airgs_config, airgs_densify_out, airgs_gaussians, airgs_stats, load_library)


class AirGSError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"{_abi.ERROR_NAMES.get(code, code)}: {message}")
        self.code = code


@dataclass
class RasterConfig:
    """Rasterizer settings (3DGS values)."""
    dilation: float = 0.3
    alpha_max: float = 0.99
    alpha_min: float = 1.0 / 255.0
    T_min: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)
    kernel_shape: int = -1   # -1: the autotuned choice for the workload (shape 0 until tuned), else a fixed shape
    sort_mode: int = -1      # 0: global radix ordering; 1: per-tile ordering when lists fit a CTA; -1: per-tile for
                             # batches of at most 65536 (view, Gaussian) pairs, radix above
    autotune_cache: str | None = None
    cull_lists: bool = True  # unobservable lists (no saved state, no n_contrib) hold only live tiles

    def to_c(self):
        c = airgs_config()
        c.dilation, c.alpha_max, c.alpha_min, c.T_min = self.dilation, self.alpha_max, self.alpha_min, self.T_min
        for k in range(3):
            c.bg[k] = float(self.bg[k])
        c.kernel_shape = int(self.kernel_shape)
        c.sort_mode = int(self.sort_mode)
        c.autotune_cache = self.autotune_cache.encode() if self.autotune_cache else None
        c.cull_lists = 1 if self.cull_lists else 0
        return c


def camera_struct(cam: dict) -> airgs_camera:
    """A camera dict (width, height, fx, fy, cx, cy, near, viewmat 4x4
    world->camera, row-major) as the C struct."""
    c = airgs_camera()
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    vm = np.asarray(cam["viewmat"], dtype=np.float64).reshape(16)
    for k in range(16):
        c.viewmat[k] = float(vm[k])
    c.near_plane = float(cam.get("near", 0.2))
    return c


def camera_array(cams):
    arr = (airgs_camera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


def image_sizes(cams):
    return [(int(c["height"]), int(c["width"])) for c in cams]


def split_views(flat: torch.Tensor, cams, channels: int = 3):
    """Views [channels, H, W] of a concatenated per-view planar buffer."""
    out, off = [], 0
    for h, w in image_sizes(cams):
        n = channels * h * w
        out.append(flat[off:off + n].view(channels, h, w) if channels > 1 else flat[off:off + n].view(h, w))
        off += n
    return out


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_cuda(t, name, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


@dataclass
class RenderResult:
    rgb: torch.Tensor                  # flat [sum 3 H W], planar per view
    cams: list
    T: torch.Tensor | None = None      # flat [sum H W]
    n_contrib: torch.Tensor | None = None
    importance_w: torch.Tensor | None = None
    importance_cnt: torch.Tensor | None = None
    state: "RenderState | None" = None

    def views(self):
        return split_views(self.rgb, self.cams)


@dataclass
class RenderState:
    handle: ctypes.c_void_p
    owner: "Rasterizer"
    n: int
    sh_degree: int
    keep: list = field(default_factory=list)  # tensors the state reads
    released: bool = False

    def release(self):
        if not self.released:
            self.owner._release(self)

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Rasterizer:
    """One library context: device state (anchor + current frame), a memory
    pool and a CUDA stream (torch's current stream at creation by default)."""

    def __init__(self, config: RasterConfig | None = None, stream: torch.cuda.Stream | None = None):
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.config = config or RasterConfig()
        self._cfg_c = self.config.to_c()
        self.stream = stream or torch.cuda.current_stream()
        self.ctx = ctypes.c_void_p()
        rc = self.lib.airgs_create(ctypes.byref(self.ctx), ctypes.byref(self._cfg_c),
                                   ctypes.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise AirGSError(rc, "airgs_create failed")
        self.n = 0
        self.sh_degree = -1

    # ------------------------------------------------------------ plumbing
    def _check(self, rc):
        if rc != 0:
            msg = self.lib.airgs_last_error(self.ctx)
            raise AirGSError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.airgs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._check(self.lib.airgs_set_stream(self.ctx, ctypes.c_void_p(stream.cuda_stream)))

    def sync(self):
        self._check(self.lib.airgs_sync(self.ctx))

    def _new(self, shape, dtype):
        with torch.cuda.stream(self.stream):
            return torch.empty(shape, dtype=dtype, device="cuda")

    def _zeros(self, shape, dtype):
        with torch.cuda.stream(self.stream):
            return torch.zeros(shape, dtype=dtype, device="cuda")

    @staticmethod
    def _check_params(means, log_scales, quats, opacity_logit, sh):
        n = means.shape[0]
        _check_cuda(means, "means", torch.float32, (n, 3))
        _check_cuda(log_scales, "log_scales", torch.float32, (n, 3))
        _check_cuda(quats, "quats", torch.float32, (n, 4))
        _check_cuda(opacity_logit, "opacity_logit", torch.float32, (n,))
        _check_cuda(sh, "sh", torch.float32)
        if sh.dim() != 3 or sh.shape[0] != n or sh.shape[2] != 3:
            raise ValueError("sh must be [n, K, 3]")
        K = sh.shape[1]
        deg = int(round(K ** 0.5)) - 1
        if (deg + 1) ** 2 != K or deg > 3:
            raise ValueError("sh must have K = (degree + 1)^2 coefficients, degree <= 3")
        return n, deg

    # ------------------------------------------------------------ anchor / frames
    def set_anchor(self, means, log_scales, quats, opacity_logit, sh):
        """Copy the anchor Gaussian set into the context (resets the frame state)."""
        n, deg = self._check_params(means, log_scales, quats, opacity_logit, sh)
        self._check(self.lib.airgs_set_anchor(self.ctx, n, deg, _ptr(means), _ptr(log_scales), _ptr(quats),
                                              _ptr(opacity_logit), _ptr(sh)))
        self.n, self.sh_degree = n, deg
        self._anchor_sh_shape = tuple(sh.shape)

    def apply_frame_update(self, update_map, lo, hi, mode=AIRGS_DELTA_PREV, quat_add=False, frame_id=0):
        """Decode a [7, H, W] uint16 device map with per-channel ranges lo/hi and
        apply it to the previous frame (mode PREV) or the anchor (mode ANCHOR)."""
        _check_cuda(update_map, "update_map", torch.uint16)
        if update_map.dim() != 3 or update_map.shape[0] != 7:
            raise ValueError("update_map must be [7, H, W]")
        lo_c = (ctypes.c_float * 7)(*[float(x) for x in np.asarray(lo).reshape(7)])
        hi_c = (ctypes.c_float * 7)(*[float(x) for x in np.asarray(hi).reshape(7)])
        m = int(mode) | (AIRGS_QUAT_ADD if quat_add else 0)
        self._check(self.lib.airgs_apply_frame_update(self.ctx, _ptr(update_map), update_map.shape[2],
                                                      update_map.shape[1], lo_c, hi_c, m, int(frame_id)))

    def frame_state(self):
        means = self._new((self.n, 3), torch.float32)
        quats = self._new((self.n, 4), torch.float32)
        self._check(self.lib.airgs_get_frame_state(self.ctx, _ptr(means), _ptr(quats)))
        return means, quats

    # ------------------------------------------------------------ render
    def _outputs(self, cams, T, n_contrib, importance, n):
        P = sum(h * w for h, w in image_sizes(cams))
        rgb = self._new((3 * P,), torch.float32)
        Tt = self._new((P,), torch.float32) if T else None
        nc = self._new((P,), torch.int32) if n_contrib else None
        iw = self._zeros((n,), torch.float32) if importance else None
        ic = self._zeros((n,), torch.int32) if importance else None
        return rgb, Tt, nc, iw, ic

    def render(self, cams, T=False, n_contrib=False, importance=False, save=False) -> RenderResult:
        """Render the current frame state for a list of camera dicts."""
        if self.sh_degree < 0:
            raise AirGSError(_abi.AIRGS_E_STATE, "set_anchor first")
        rgb, Tt, nc, iw, ic = self._outputs(cams, T, n_contrib, importance, self.n)
        st = ctypes.c_void_p()
        arr = camera_array(cams)
        self._check(self.lib.airgs_render(self.ctx, arr, len(cams), _ptr(rgb), _ptr(Tt), _ptr(nc), _ptr(iw), _ptr(ic),
                                          ctypes.byref(st) if save else None))
        res = RenderResult(rgb=rgb, cams=cams, T=Tt, n_contrib=nc, importance_w=iw, importance_cnt=ic)
        if save:
            res.state = RenderState(st, self, self.n, self.sh_degree, keep=[rgb])
        return res

    def render_gaussians(self, means, log_scales, quats, opacity_logit, sh, cams, T=False, n_contrib=False,
                         importance=False, save=False, rgb_out=None) -> RenderResult:
        """Render a caller-owned Gaussian set (the training path)."""
        n, deg = self._check_params(means, log_scales, quats, opacity_logit, sh)
        rgb, Tt, nc, iw, ic = self._outputs(cams, T, n_contrib, importance, n)
        if rgb_out is not None:
            _check_cuda(rgb_out, "rgb_out", torch.float32, rgb.shape)
            rgb = rgb_out
        g = airgs_gaussians(n, deg, means.data_ptr(), log_scales.data_ptr(), quats.data_ptr(),
                            opacity_logit.data_ptr(), sh.data_ptr())
        st = ctypes.c_void_p()
        arr = camera_array(cams)
        self._check(self.lib.airgs_render_gaussians(self.ctx, ctypes.byref(g), arr, len(cams), _ptr(rgb), _ptr(Tt),
                                                    _ptr(nc), _ptr(iw), _ptr(ic),
                                                    ctypes.byref(st) if save else None))
        res = RenderResult(rgb=rgb, cams=cams, T=Tt, n_contrib=nc, importance_w=iw, importance_cnt=ic)
        if save:
            res.state = RenderState(st, self, n, deg, keep=[rgb, means, log_scales, quats, opacity_logit, sh])
        return res

    def _grad_buffers(self, state):
        n, K = state.n, (state.sh_degree + 1) ** 2
        return dict(means=self._new((n, 3), torch.float32), log_scales=self._new((n, 3), torch.float32),
                    quats=self._new((n, 4), torch.float32), opacity_logit=self._new((n,), torch.float32),
                    sh=self._new((n, K, 3), torch.float32))

    def render_backward(self, state: RenderState, dL_drgb: torch.Tensor, importance=None):
        """Gradients w.r.t. the raw parameters given dL/d(rgb) (flat, like rgb).
        importance: optional (w, cnt) tensors that accumulate during the replay."""
        _check_cuda(dL_drgb, "dL_drgb", torch.float32, state.keep[0].shape)
        gr = self._grad_buffers(state)
        iw, ic = importance if importance is not None else (None, None)
        self._check(self.lib.airgs_render_backward(self.ctx, state.handle, _ptr(dL_drgb), _ptr(gr["means"]),
                                                   _ptr(gr["log_scales"]), _ptr(gr["quats"]),
                                                   _ptr(gr["opacity_logit"]), _ptr(gr["sh"]), _ptr(iw), _ptr(ic)))
        return gr

    def render_backward_l1(self, state: RenderState, target: torch.Tensor, importance=None):
        """L1 loss (mean |rgb - target|) and its gradients, fused into the backward."""
        _check_cuda(target, "target", torch.float32, state.keep[0].shape)
        gr = self._grad_buffers(state)
        loss = self._new((1,), torch.float32)
        iw, ic = importance if importance is not None else (None, None)
        self._check(self.lib.airgs_render_backward_l1(self.ctx, state.handle, _ptr(target), _ptr(loss),
                                                      _ptr(gr["means"]), _ptr(gr["log_scales"]), _ptr(gr["quats"]),
                                                      _ptr(gr["opacity_logit"]), _ptr(gr["sh"]), _ptr(iw), _ptr(ic)))
        return loss, gr

    def render_backward_ex(self, state: RenderState, dL_drgb=None, target=None, importance=None, densify=None):
        """The adjoint with every optional output: dL_drgb or an L1 target,
        importance (w, cnt) and densification statistics (grad_norm_sum,
        views) accumulators.  Returns (gradients, loss or None)."""
        a = airgs_backward_args()
        ref = state.keep[0]
        if target is not None:
            _check_cuda(target, "target", torch.float32, ref.shape)
            a.target = target.data_ptr()
            loss = self._new((1,), torch.float32)
            a.loss_out = loss.data_ptr()
        else:
            _check_cuda(dL_drgb, "dL_drgb", torch.float32, ref.shape)
            a.dL_drgb = dL_drgb.data_ptr()
            loss = None
        gr = self._grad_buffers(state)
        a.g_means, a.g_log_scales, a.g_quats = gr["means"].data_ptr(), gr["log_scales"].data_ptr(), gr["quats"].data_ptr()
        a.g_opacity_logit, a.g_sh = gr["opacity_logit"].data_ptr(), gr["sh"].data_ptr()
        if importance is not None:
            a.importance_w, a.importance_cnt = importance[0].data_ptr(), importance[1].data_ptr()
        if densify is not None:
            a.densify_grad, a.densify_views = densify[0].data_ptr(), densify[1].data_ptr()
        self._check(self.lib.airgs_render_backward_ex(self.ctx, state.handle, ctypes.byref(a)))
        return gr, loss

    def densify_select(self, grad_sum: torch.Tensor, views: torch.Tensor, threshold: float) -> torch.Tensor:
        """uint8 mask of Gaussians whose mean screen-space gradient exceeds threshold."""
        _check_cuda(grad_sum, "grad_sum", torch.float32)
        mask = self._new((grad_sum.numel(),), torch.uint8)
        self._check(self.lib.airgs_densify_select(self.ctx, _ptr(grad_sum), _ptr(views), grad_sum.numel(),
                                                  float(threshold), _ptr(mask)))
        return mask

    def densify_apply(self, means, log_scales, quats, opacity_logit, sh, select, z, size_threshold: float,
                      split_factor: float = 1.6, min_opacity: float = 0.0, read_count: bool = True):
        """Clone / split / discard step of keyframe densification (Sec. III-B),
        airgs_densify_apply: selected Gaussians whose largest scale is at most
        size_threshold gain an identical copy, larger selected ones become two
        children sampled with the caller's standard normal z [n, 2, 3], and
        Gaussians of opacity below min_opacity are discarded.  Returns a dict of
        the output Gaussian set (means, log_scales, quats, opacity_logit, sh) and
        `parent` (int32: input index of each output), sliced to the output
        count, which is read back (one wait on the context's stream); with
        read_count=False the buffers keep their capacity 2 n and `n_out` holds
        the device count, with no wait."""
        n, deg = self._check_params(means, log_scales, quats, opacity_logit, sh)
        _check_cuda(select, "select", torch.uint8, (n,))
        _check_cuda(z, "z", torch.float32, (n, 2, 3))
        cap, K = 2 * n, (deg + 1) ** 2
        out = dict(means=self._new((cap, 3), torch.float32), log_scales=self._new((cap, 3), torch.float32),
                   quats=self._new((cap, 4), torch.float32), opacity_logit=self._new((cap,), torch.float32),
                   sh=self._new((cap, K, 3), torch.float32), parent=self._new((cap,), torch.int32))
        n_out = self._new((1,), torch.int64)
        g = airgs_gaussians(n, deg, means.data_ptr(), log_scales.data_ptr(), quats.data_ptr(),
                            opacity_logit.data_ptr(), sh.data_ptr())
        d = airgs_densify_out(cap, out["means"].data_ptr(), out["log_scales"].data_ptr(), out["quats"].data_ptr(),
                              out["opacity_logit"].data_ptr(), out["sh"].data_ptr(), out["parent"].data_ptr(),
                              n_out.data_ptr())
        self._check(self.lib.airgs_densify_apply(self.ctx, ctypes.byref(g), _ptr(select), _ptr(z),
                                                 float(size_threshold), float(split_factor), float(min_opacity),
                                                 ctypes.byref(d)))
        if not read_count:
            out["n_out"] = n_out
            return out
        self.stream.synchronize()
        m = int(n_out.item())
        return {k: v[:m] for k, v in out.items()}

    def gaussian_importance(self, cams):
        w = self._new((self.n,), torch.float32)
        c = self._new((self.n,), torch.int32)
        self._check(self.lib.airgs_gaussian_importance(self.ctx, camera_array(cams), len(cams), _ptr(w), _ptr(c)))
        return w, c

    # ------------------------------------------------------------ pruning (Sec. III-C)
    def prune_mask(self, importance: torch.Tensor, n_prune: int) -> torch.Tensor:
        """uint8 keep mask: 0 for the n_prune Gaussians of lowest usage frequency."""
        _check_cuda(importance, "importance", torch.float32)
        keep = self._new((importance.numel(),), torch.uint8)
        self._check(self.lib.airgs_prune_mask(self.ctx, _ptr(importance), importance.numel(), int(n_prune),
                                              _ptr(keep)))
        return keep

    def prune_delta(self, D_t: torch.Tensor, D_sent: torch.Tensor, keep: torch.Tensor):
        """d'_t = p(D_t - D'_{t-1}) for channel-major [C, n] deltas; updates D_sent
        in place.  Returns (d'_t, number of Gaussians with a non-zero delta)."""
        _check_cuda(D_t, "D_t", torch.float32)
        _check_cuda(D_sent, "D_sent", torch.float32, D_t.shape)
        _check_cuda(keep, "keep", torch.uint8, (D_t.shape[1],))
        d = self._new(tuple(D_t.shape), torch.float32)
        nz = self._new((1,), torch.int64)
        self._check(self.lib.airgs_prune_delta(self.ctx, D_t.shape[1], D_t.shape[0], _ptr(D_t), _ptr(D_sent),
                                               _ptr(keep), _ptr(d), _ptr(nz)))
        return d, nz

    def apply_frame_delta(self, delta: torch.Tensor, mode=AIRGS_DELTA_PREV, quat_add=False, frame_id=0):
        """Apply a decoded float delta [7, n] to the previous frame or the anchor."""
        _check_cuda(delta, "delta", torch.float32, (7, self.n))
        m = int(mode) | (AIRGS_QUAT_ADD if quat_add else 0)
        self._check(self.lib.airgs_apply_frame_delta(self.ctx, _ptr(delta), m, int(frame_id)))

    def image_sse(self, cams, a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        """Per-view sum of squared differences (device float64 [n_views])."""
        _check_cuda(a, "a", torch.float32)
        _check_cuda(b, "b", torch.float32, a.shape)
        out = self._new((len(cams),), torch.float64)
        self._check(self.lib.airgs_image_sse(self.ctx, camera_array(cams), len(cams), _ptr(a), _ptr(b), _ptr(out)))
        return out

    def l3dgs_loss(self, cams, rgb: torch.Tensor, target: torch.Tensor, lam: float = 0.2):
        """L = (1 - lam) L1 + lam (1 - SSIM) of Eq. 1 and dL/d(rgb).  Returns
        (float64 tensor [L, L1, SSIM], gradient laid out like rgb)."""
        _check_cuda(rgb, "rgb", torch.float32)
        _check_cuda(target, "target", torch.float32, rgb.shape)
        loss = self._new((3,), torch.float64)
        grad = self._new(tuple(rgb.shape), torch.float32)
        self._check(self.lib.airgs_l3dgs_loss(self.ctx, camera_array(cams), len(cams), _ptr(rgb), _ptr(target),
                                              float(lam), _ptr(loss), _ptr(grad)))
        return loss, grad

    def _release(self, state: RenderState):
        if not state.released and self.ctx is not None:
            self._check(self.lib.airgs_release_state(self.ctx, state.handle))
        state.released = True
        state.keep = []

    def stats(self, state: RenderState) -> dict:
        s = airgs_stats()
        self._check(self.lib.airgs_state_stats(self.ctx, state.handle, ctypes.byref(s)))
        return dict(n_instances=s.n_instances, n_tiles=s.n_tiles, n_pixels=s.n_pixels,
                    pairs_forward=s.pairs_forward, pairs_backward=s.pairs_backward, kernel_shape=s.kernel_shape)

    def state_projection(self, state: RenderState, view: int):
        n = state.n
        m2 = self._new((n, 2), torch.float32)
        d = self._new((n,), torch.float32)
        r = self._new((n,), torch.int32)
        self._check(self.lib.airgs_state_projection(self.ctx, state.handle, view, _ptr(m2), _ptr(d), _ptr(r)))
        return m2, d, r

    def state_tile_lists(self, state: RenderState, view: int):
        nt, ne = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.airgs_state_view_info(self.ctx, state.handle, view, ctypes.byref(nt), ctypes.byref(ne)))
        ranges = self._new((nt.value, 2), torch.int64)
        ids = self._new((max(ne.value, 1),), torch.int32)
        self._check(self.lib.airgs_state_tile_lists(self.ctx, state.handle, view, _ptr(ranges), _ptr(ids)))
        return ranges, ids[:ne.value]

    def sort_pairs(self, keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 32):
        """Stable radix sort of uint32 (key, value) pairs by the low key_bits bits
        (int32 tensors are read as uint32)."""
        for t, nm in ((keys, "keys"), (vals, "vals")):
            if t.dtype not in (torch.int32, torch.uint32):
                raise ValueError(f"{nm} must be 32-bit")
            _check_cuda(t, nm, t.dtype)
        ko, vo = torch.empty_like(keys), torch.empty_like(vals)
        self._check(self.lib.airgs_sort_pairs(self.ctx, _ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), keys.numel(),
                                              key_bits))
        return ko, vo

    def autotune(self, cams, report: bool = False):
        """Search the compiled kernel shapes for this workload (the current
        frame's Gaussians, these cameras) by timing training steps; later
        renders of the workload use the choice.  Returns the shape index, or
        with report=True (shape, ms of shape 0, ms of the choice)."""
        v, t0, t1 = ctypes.c_int(), ctypes.c_float(), ctypes.c_float()
        self._check(self.lib.airgs_autotune(self.ctx, camera_array(cams), len(cams), ctypes.byref(v),
                                            ctypes.byref(t0), ctypes.byref(t1)))
        return (v.value, t0.value, t1.value) if report else v.value

    def set_profiling(self, enabled: bool = True, blend_only: bool = False):
        """Time each pipeline stage with CUDA events on the context's stream
        (blend_only: only the blend forward and backward stages)."""
        level = (_abi.AIRGS_PROFILE_BLEND if blend_only else _abi.AIRGS_PROFILE_ALL) if enabled else \
            _abi.AIRGS_PROFILE_OFF
        self._check(self.lib.airgs_set_profiling(self.ctx, level))

    def stage_times(self) -> dict:
        """Per-stage device milliseconds and launch counts since the previous
        readout, and the forward/backward evaluated-pair totals (synchronises)."""
        n = _abi.AIRGS_NUM_STAGES
        ms = (ctypes.c_double * n)()
        launches = (ctypes.c_int64 * n)()
        pairs = (ctypes.c_int64 * 4)()
        self._check(self.lib.airgs_stage_times(self.ctx, ms, launches, pairs))
        names = [self.lib.airgs_stage_name(i).decode() for i in range(n)]
        return dict(ms={names[i]: ms[i] for i in range(n)}, launches={names[i]: launches[i] for i in range(n)},
                    pairs_forward=pairs[0], pairs_backward=pairs[1], issued_forward=pairs[2],
                    issued_backward=pairs[3])

    @staticmethod
    def kernel_launch_count() -> int:
        return int(load_library().airgs_kernel_launch_count())

    def measure_fp32_peak(self) -> float:
        """Measured FP32 throughput of this context's GPU, TFLOP/s."""
        v = ctypes.c_double(0.0)
        self._check(self.lib.airgs_measure_fp32_peak(self.ctx, ctypes.byref(v)))
        return v.value

    def measure_smem_peak(self) -> float:
        """Measured shared-memory load throughput of this context's GPU, TB/s."""
        v = ctypes.c_double(0.0)
        self._check(self.lib.airgs_measure_smem_peak(self.ctx, ctypes.byref(v)))
        return v.value

    @staticmethod
    def shape_names():
        """Names of the compiled kernel shapes (index 0 is the default)."""
        lib = load_library()
        return [lib.airgs_shape_name(i).decode() for i in range(lib.airgs_shape_count())]


# ---------------------------------------------------------------- autograd
class RasterizeGaussians(torch.autograd.Function):
    """rgb = render(means, log_scales, quats, opacity_logit, sh; cams), with the
    library's hand-written adjoint as the backward."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logit, sh, rast: Rasterizer, cams):
        res = rast.render_gaussians(means.detach(), log_scales.detach(), quats.detach(), opacity_logit.detach(),
                                    sh.detach(), cams, save=True)
        ctx.rast = rast
        ctx.state = res.state
        return res.rgb

    @staticmethod
    def backward(ctx, grad_rgb):
        gr = ctx.rast.render_backward(ctx.state, grad_rgb.contiguous())
        ctx.state.release()
        return gr["means"], gr["log_scales"], gr["quats"], gr["opacity_logit"], gr["sh"], None, None


def rasterize(rast: Rasterizer, means, log_scales, quats, opacity_logit, sh, cams):
    return RasterizeGaussians.apply(means, log_scales, quats, opacity_logit, sh, rast, cams)
