"""PyTorch-facing layer over the C ABI: tensors are used only as device memory and streams.

* ``SplatContext`` -- owns a libsplatloam context (workspace sized at creation) and the views.
* ``SplatRender`` -- ``torch.autograd.Function``: forward = splat_render_views, backward =
  splat_render_views_backward.
* ``loss`` / ``adam_step`` -- the loss and optimiser entry points.
* ``Refiner`` -- one refinement iteration (render, loss, backward, Adam) over a set of keyframes,
  either as plain per-keyframe launch sequences or as one fused pass over all keyframes captured
  in a CUDA graph.

Every tensor handed to the library must be a contiguous float32 CUDA tensor on the current
device; the helpers check that and raise otherwise.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib

_P = ctypes.c_void_p


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f32(t, shape_tail):
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected contiguous float32 CUDA tensors")
    if tuple(t.shape[1:]) != shape_tail:
        raise ValueError(f"expected shape (n, {shape_tail})")
    return t


@dataclass
class ViewSpec:
    T_ws: np.ndarray
    rows: int
    cols: int
    elev_min: float
    elev_max: float


@dataclass
class RenderConfig:
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    sigma_cut: float = 3.0
    tile_h: int = 16
    tile_w: int = 16
    flip_normals: int = 1

    def c(self):
        return _lib.splat_render_config(self.alpha_min, self.alpha_max, self.t_min,
                                        self.sigma_cut, self.tile_h, self.tile_w, 0,
                                        self.flip_normals)


@dataclass
class LossConfig:
    lambda_n: float = 1.0
    lambda_o: float = 0.0
    o_eps: float = 1e-6
    lambda_s: float = 0.0   # scale term (splat_refine_step only)
    tau_s: float = 0.5
    normal_mode: int = 0    # 0: against target normals; 1: normals of the rendered range map
    rho_exp: float = 0.0    # range weight rho_d = Dt^rho_exp of the L1 term

    def c(self):
        return _lib.splat_loss_config(self.lambda_n, self.lambda_o, self.o_eps, self.lambda_s,
                                      self.tau_s, self.normal_mode, self.rho_exp)


@dataclass
class DensifyConfig:
    """Map growth settings (splat_densify_config): refine = False uses the valid mask only
    (local model initialisation); True adds M_n (O <= lambda_do) or M_e (|D - Dt| >= lambda_de)."""
    refine: bool = False
    lambda_do: float = 0.5
    lambda_de: float = 0.1
    w0: float = 0.05
    w_cap: float = 2.0
    scale_k: float = 2.0
    opacity: float = 0.5
    seed: int = 0

    def c(self):
        return _lib.splat_densify_config(int(self.refine), self.lambda_do, self.lambda_de,
                                         self.w0, self.w_cap, self.scale_k, self.opacity,
                                         self.seed)


@dataclass
class AdamConfig:
    lr_pos: float = 1e-3
    lr_opacity: float = 2e-2
    lr_rot: float = 2e-3
    lr_scale: float = 5e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15

    def c(self):
        return _lib.splat_adam_config(self.lr_pos, self.lr_opacity, self.lr_rot, self.lr_scale,
                                      self.beta1, self.beta2, self.eps)


class SplatContext:
    """A libsplatloam context: workspace for up to max_gaussians primitives, max_views views,
    max_pixels packed pixels and max_pairs (tile, primitive) pairs per render call."""

    def __init__(self, max_gaussians, max_views=1, max_pixels=1 << 20, max_pairs=None,
                 cfg: RenderConfig | None = None, max_tiles=0):
        self.lib = _lib.load()
        self.cfg = cfg or RenderConfig()
        if max_pairs is None:
            max_pairs = min(max(16 * max_gaussians * max_views, 1 << 20), (1 << 32) - 1)
        cap = _lib.splat_capacity(int(max_gaussians), int(max_views), int(max_pixels),
                                  int(max_pairs), int(max_tiles))
        h = ctypes.c_void_p()
        torch.cuda.init()
        _lib.check(self.lib.splat_ctx_create(ctypes.byref(self.cfg.c()), ctypes.byref(cap),
                                             ctypes.byref(h)), "splat_ctx_create")
        self.h = h
        self.cap = cap
        self.views: list[ViewSpec] = []
        self.n_pixels = 0
        self.offsets: list[int] = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.splat_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- views --------------------------------------------------------------------------
    def set_views(self, views):
        views = [v if isinstance(v, ViewSpec) else ViewSpec(np.asarray(v.T_ws), v.rows, v.cols,
                                                             v.elev_min, v.elev_max)
                 for v in views]
        T = np.ascontiguousarray(np.stack([np.asarray(v.T_ws, np.float64) for v in views]))
        intr = (_lib.splat_lidar_intrinsics * len(views))(
            *[_lib.splat_lidar_intrinsics(v.rows, v.cols, v.elev_min, v.elev_max)
              for v in views])
        _lib.check(self.lib.splat_set_views(self.h, len(views), T.ctypes.data_as(_P), intr),
                   "splat_set_views")
        self.views = views
        self.offsets = [int(self.lib.splat_view_pixel_offset(self.h, i))
                        for i in range(len(views))]
        self.n_pixels = sum(v.rows * v.cols for v in views)

    def view_image(self, flat, v):
        """(H, W) or (3, H, W) view of view v inside a packed (P,) or (3, P) tensor."""
        vs = self.views[v]
        o = self.offsets[v]
        if flat.dim() == 1:
            return flat[o:o + vs.rows * vs.cols].view(vs.rows, vs.cols)
        return flat[:, o:o + vs.rows * vs.cols].reshape(3, vs.rows, vs.cols)

    # ---- render / backward --------------------------------------------------------------
    @staticmethod
    def _g(pos_logit, quat, log_scale):
        n = pos_logit.shape[0]
        _f32(pos_logit, (4,))
        _f32(quat, (4,))
        _f32(log_scale, (2,))
        if quat.shape[0] != n or log_scale.shape[0] != n:
            raise ValueError("parameter tensors disagree on n")
        return _lib.splat_gaussians(pos_logit.data_ptr(), quat.data_ptr(), log_scale.data_ptr(), n)

    def alloc_images(self, device=None):
        P = self.n_pixels
        dev = device or torch.device("cuda")
        return (torch.empty(P, device=dev), torch.empty(3, P, device=dev),
                torch.empty(P, device=dev))

    def render(self, pos_logit, quat, log_scale, out=None, stream=None):
        depth, normal, alpha = out if out is not None else self.alloc_images(pos_logit.device)
        g = self._g(pos_logit, quat, log_scale)
        _lib.check(self.lib.splat_render_views(self.h, ctypes.byref(g), _ptr(depth), _ptr(normal),
                                               _ptr(alpha), _stream(stream)),
                   "splat_render_views")
        return depth, normal, alpha

    def backward(self, pos_logit, quat, log_scale, gD, gN, gO, out=None, accumulate=False,
                 stream=None):
        n = pos_logit.shape[0]
        if out is None:
            out = (torch.zeros(n, 4, device=pos_logit.device),
                   torch.zeros(n, 4, device=pos_logit.device),
                   torch.zeros(n, 2, device=pos_logit.device))
        g = self._g(pos_logit, quat, log_scale)
        _lib.check(self.lib.splat_render_views_backward(
            self.h, ctypes.byref(g), _ptr(gD), _ptr(gN), _ptr(gO), _ptr(out[0]), _ptr(out[1]),
            _ptr(out[2]), 1 if accumulate else 0, _stream(stream)), "splat_render_views_backward")
        return out

    def refine_step(self, params, state, target_depth, target_normal, loss_cfg: LossConfig,
                    adam_cfg: AdamConfig, loss_out, stream=None):
        pl, q, ls = params
        m_pl, m_q, m_ls, v_pl, v_q, v_ls, step = state
        _lib.check(self.lib.splat_refine_step(
            self.h, _ptr(pl), _ptr(q), _ptr(ls), pl.shape[0], _ptr(target_depth),
            _ptr(target_normal), ctypes.byref(loss_cfg.c()), ctypes.byref(adam_cfg.c()),
            _ptr(m_pl), _ptr(m_q), _ptr(m_ls), _ptr(v_pl), _ptr(v_q), _ptr(v_ls), _ptr(step),
            _ptr(loss_out), _stream(stream)), "splat_refine_step")

    def view_loss(self, depth, normal, alpha, target_depth, target_normal=None,
                  cfg: LossConfig | None = None, stream=None):
        """The loss over the packed images of the registered views (splat_view_loss), either
        normal mode; returns (L (device double tensor), dL/dD, dL/dN, dL/dO)."""
        cfg = cfg or LossConfig()
        gD = torch.empty_like(depth)
        gN = torch.empty_like(normal)
        gO = torch.empty_like(alpha)
        L = torch.zeros(1, dtype=torch.float64, device=depth.device)
        _lib.check(self.lib.splat_view_loss(
            self.h, _ptr(depth), _ptr(normal), _ptr(alpha), _ptr(target_depth),
            _ptr(target_normal), ctypes.byref(cfg.c()),
            _ptr(gD), _ptr(gN), _ptr(gO), _ptr(L), _stream(stream)), "splat_view_loss")
        return L, gD, gN, gO

    def densify(self, params, n_old: int, n_new: int, target_depth, depth=None, alpha=None,
                cfg: DensifyConfig | None = None, stream=None):
        """Write n_new primitives drawn from the packed target range image into rows
        [n_old, n_old + n_new) of params (pos_logit, quat, log_scale, each with room for them):
        splat_densify.  Empty slots carry opacity logit -30."""
        cfg = cfg or DensifyConfig()
        pl, q, ls = params
        for t, w in ((pl, 4), (q, 4), (ls, 2)):
            _f32(t, (w,))
        cap = min(pl.shape[0], q.shape[0], ls.shape[0])
        _lib.check(self.lib.splat_densify(
            self.h, _ptr(target_depth), _ptr(depth), _ptr(alpha), ctypes.byref(cfg.c()),
            int(n_new), _ptr(pl), _ptr(q), _ptr(ls), int(n_old), int(cap), _stream(stream)),
            "splat_densify")

    def photometric(self, view: int, depth, alpha, query_depth, T_qm, o_min=0.5, huber_delta=0.2,
                    per_pixel=False, out=None, stream=None):
        """Photometric residual of registered view `view` (its own rows x cols pixels) against a
        query range image, reduced to Gauss-Newton normal equations (splat_photometric).
        T_qm: device float32 (3, 4) [R | t], render frame -> query frame.  Returns the device
        double[29] (see unpack_normal_eqs) and, when per_pixel, the (8, P) float32 r, w, J."""
        out = out if out is not None else torch.empty(29, dtype=torch.float64,
                                                      device=depth.device)
        px = None
        if per_pixel and 0 <= view < len(self.views):
            P = self.views[view].rows * self.views[view].cols
            px = torch.empty(8, P, dtype=torch.float32, device=depth.device)
        if T_qm.dtype != torch.float32 or tuple(T_qm.shape) != (3, 4) or not T_qm.is_cuda:
            raise ValueError("T_qm: float32 CUDA tensor of shape (3, 4)")
        _lib.check(self.lib.splat_photometric(
            self.h, int(view), _ptr(depth), _ptr(alpha), _ptr(query_depth),
            _ptr(T_qm.contiguous()), float(o_min), float(huber_delta), _ptr(out), _ptr(px),
            _stream(stream)), "splat_photometric")
        return (out, px) if per_pixel else out

    # ---- inspection ---------------------------------------------------------------------
    def set_view_sampling(self, draws: int, p_newest: float = 0.4, seed: int = 0):
        """Draw `draws` keyframes per render from the truncated geometric law over keyframe age
        (splat_set_view_sampling); draws = 0 renders every view."""
        _lib.check(self.lib.splat_set_view_sampling(self.h, int(draws), float(p_newest),
                                                    int(seed)), "splat_set_view_sampling")

    def active_views(self) -> np.ndarray:
        flags = np.zeros(len(self.views), np.uint8)
        _lib.check(self.lib.splat_get_active_views(self.h, flags.ctypes.data_as(_P)),
                   "splat_get_active_views")
        return flags.astype(bool)

    def backproject(self, depth, alpha, o_min=0.5, stream=None) -> torch.Tensor:
        """World-frame points (3, P) of the packed range images (splat_backproject); NaN where
        alpha < o_min."""
        _f32(depth, ())
        _f32(alpha, ())
        out = torch.empty(3, self.n_pixels, dtype=torch.float32, device=depth.device)
        _lib.check(self.lib.splat_backproject(self.h, _ptr(depth), _ptr(alpha), float(o_min),
                                              _ptr(out), _stream(stream)), "splat_backproject")
        return out

    def set_pose_gradient(self, on: bool):
        """Make the following backward calls also form the per-view pose gradient."""
        _lib.check(self.lib.splat_set_pose_gradient(self.h, 1 if on else 0),
                   "splat_set_pose_gradient")

    def pose_gradients(self, stream=None) -> torch.Tensor:
        """(n_views, 6) float32 on the device: (dL/drho, dL/domega) of each view's pose for the
        left perturbation T^c_w <- exp(xi^) T^c_w of the last backward (splat_pose_gradient)."""
        out = torch.zeros(len(self.views), 6, dtype=torch.float32, device="cuda")
        _lib.check(self.lib.splat_pose_gradient(self.h, _ptr(out), _stream(stream)),
                   "splat_pose_gradient")
        return out

    def status(self) -> int:
        f = ctypes.c_uint32(0)
        _lib.check(self.lib.splat_get_status(self.h, ctypes.byref(f)), "splat_get_status")
        return int(f.value)

    def stats(self) -> dict:
        s = _lib.splat_stats()
        _lib.check(self.lib.splat_get_stats(self.h, ctypes.byref(s)), "splat_get_stats")
        return dict(n_pairs=s.n_pairs, fwd_evals=s.fwd_evals, bwd_evals=s.bwd_evals,
                    n_pixels=s.n_pixels, n_tiles=s.n_tiles, kernel_launches=s.kernel_launches,
                    n_touching=s.n_touching)

    STAGES = ("projection", "range sort", "emission", "tile sort", "tile ranges", "loss",
              "fused Adam")

    def stage_times(self) -> dict:
        """Durations (ms) of the stages of the last profiled render / refinement step
        (splat_stage_times); None for a stage not recorded."""
        ms = (ctypes.c_float * 7)()
        _lib.check(self.lib.splat_stage_times(self.h, ms), "splat_stage_times")
        return {k: (float(v) if v >= 0 else None) for k, v in zip(self.STAGES, ms)}

    def set_profiling(self, on: bool):
        _lib.check(self.lib.splat_set_profiling(self.h, 1 if on else 0), "splat_set_profiling")

    def kernel_times(self):
        """(forward compositing ms, backward adjoint ms) of the last profiled calls."""
        f, b = ctypes.c_float(-1), ctypes.c_float(-1)
        _lib.check(self.lib.splat_kernel_times(self.h, ctypes.byref(f), ctypes.byref(b)),
                   "splat_kernel_times")
        return float(f.value), float(b.value)

    def debug_copy(self, which: int, n_items: int, dtype) -> np.ndarray:
        arr = np.zeros(n_items, dtype=dtype)
        got = self.lib.splat_debug_copy(self.h, which, arr.ctypes.data_as(_P), arr.nbytes)
        if got < 0:
            raise _lib.SplatError("splat_debug_copy failed")
        return arr[: got // arr.itemsize]

    def sorted_lists(self):
        """(sorted global tile ids, sorted pair ids, per-tile [start, end)) of the last render."""
        st = self.stats()
        m, nt = st["n_pairs"], st["n_tiles"]
        keys = self.debug_copy(0, m, np.uint32)
        vals = self.debug_copy(1, m, np.uint32)
        ranges = self.debug_copy(2, 2 * nt, np.uint32).reshape(nt, 2)
        return keys, vals, ranges

    def pair_records(self, n):
        """Per (view, primitive) records of the last render: r0, r1, c0, nc, kappa, count, flags."""
        raw = self.debug_copy(3, 4 * n * len(self.views), np.uint32).reshape(-1, 4)
        rc = raw[:, :2].copy().view(np.int16).reshape(-1, 4)
        kappa = raw[:, 2].copy().view(np.float32)
        cf = raw[:, 3]
        return dict(r0=rc[:, 0], r1=rc[:, 1], c0=rc[:, 2], nc=rc[:, 3], kappa=kappa,
                    count=(cf & 0x3FFFFFFF).astype(np.int64), flip=((cf >> 30) & 1).astype(bool),
                    invalid=((cf >> 31) & 1).astype(bool))


def loss(depth, normal, alpha, target_depth, target_normal, cfg: LossConfig | None = None,
         stream=None):
    """Per-pixel loss and its gradients over packed pixels; returns (L (device double tensor),
    dL/dD, dL/dN, dL/dO)."""
    cfg = cfg or LossConfig()
    lib = _lib.load()
    P = depth.shape[0]
    gD = torch.empty_like(depth)
    gN = torch.empty_like(normal)
    gO = torch.empty_like(alpha)
    L = torch.zeros(1, dtype=torch.float64, device=depth.device)
    _lib.check(lib.splat_loss(_ptr(depth), _ptr(normal), _ptr(alpha), _ptr(target_depth),
                              _ptr(target_normal), P, ctypes.byref(cfg.c()), _ptr(gD), _ptr(gN),
                              _ptr(gO), _ptr(L), _stream(stream)), "splat_loss")
    return L, gD, gN, gO


def unpack_normal_eqs(v):
    """(H (6, 6), g (6,), cost, count) from the 29 values of splat_photometric."""
    v = np.asarray(v.cpu() if hasattr(v, "cpu") else v, np.float64)
    H = np.zeros((6, 6))
    k = 0
    for a in range(6):
        for b in range(a, 6):
            H[a, b] = H[b, a] = v[k]
            k += 1
    return H, v[21:27].copy(), float(v[27]), int(round(v[28]))


def adam_state(n, device="cuda"):
    z = lambda *s: torch.zeros(*s, device=device)  # noqa: E731
    return (z(n, 4), z(n, 4), z(n, 2), z(n, 4), z(n, 4), z(n, 2),
            torch.zeros(1, dtype=torch.int32, device=device))


def adam_step(params, grads, state, cfg: AdamConfig | None = None, stream=None):
    cfg = cfg or AdamConfig()
    lib = _lib.load()
    pl, q, ls = params
    g_pl, g_q, g_ls = grads
    m_pl, m_q, m_ls, v_pl, v_q, v_ls, step = state
    _lib.check(lib.splat_adam_step(_ptr(pl), _ptr(q), _ptr(ls), _ptr(g_pl), _ptr(g_q), _ptr(g_ls),
                                   _ptr(m_pl), _ptr(m_q), _ptr(m_ls), _ptr(v_pl), _ptr(v_q),
                                   _ptr(v_ls), _ptr(step), pl.shape[0], ctypes.byref(cfg.c()),
                                   _stream(stream)), "splat_adam_step")


def save_checkpoint(path, params, state, extra=None):
    """Write the map parameters (pos_logit, quat, log_scale), the Adam moments and step count of
    `state` (as from adam_state) and an optional dict of plain values to `path` (torch.save)."""
    torch.save({"params": [t.detach().cpu() for t in params],
                "state": [t.detach().cpu() for t in state],
                "extra": dict(extra or {})}, path)


def load_checkpoint(path, params=None, state=None, device="cuda"):
    """Read a checkpoint written by save_checkpoint.  With `params` / `state` given (tensors of
    the same shapes), the values are copied into them in place -- a CUDA graph captured on those
    tensors keeps working -- otherwise new tensors are made on `device`.  Returns
    (params, state, extra)."""
    ck = torch.load(path, map_location="cpu")

    def fill(saved, dst):
        if dst is None:
            return tuple(t.to(device) for t in saved)
        if len(dst) != len(saved):
            raise ValueError("checkpoint holds %d tensors, %d given" % (len(saved), len(dst)))
        for t, v in zip(dst, saved):
            if t.shape != v.shape or t.dtype != v.dtype:
                raise ValueError(f"checkpoint tensor {tuple(v.shape)} {v.dtype} does not fit "
                                 f"{tuple(t.shape)} {t.dtype}")
            t.copy_(v)
        return tuple(dst)

    return fill(ck["params"], params), fill(ck["state"], state), ck["extra"]


class SplatRender(torch.autograd.Function):
    """(pos_logit, quat, log_scale) -> (depth (P,), normal (3,P), alpha (P,)) for the views
    registered in the context; gradients through splat_render_views_backward."""

    @staticmethod
    def forward(ctx, pos_logit, quat, log_scale, sctx: SplatContext):
        depth, normal, alpha = sctx.render(pos_logit, quat, log_scale)
        ctx.sctx = sctx
        ctx.save_for_backward(pos_logit, quat, log_scale)
        return depth, normal, alpha

    @staticmethod
    def backward(ctx, gD, gN, gO):
        pl, q, ls = ctx.saved_tensors
        c = lambda t: None if t is None else t.contiguous()  # noqa: E731
        g = ctx.sctx.backward(pl, q, ls, c(gD), c(gN), c(gO))
        return g[0], g[1], g[2], None


def render(pos_logit, quat, log_scale, sctx: SplatContext):
    return SplatRender.apply(pos_logit, quat, log_scale, sctx)


class Refiner:
    """One map-refinement iteration over a set of keyframes sharing one map.

    mode="batched": all keyframes in one fused pass (projection of every (keyframe, primitive),
    one sort, persistent compositing over the tiles of all keyframes, loss, backward, fused
    Adam), captured once in a CUDA graph and replayed.
    mode="plain": one launch sequence per keyframe (render, loss, backward with accumulation),
    then one Adam step -- no graph; every keyframe has its own context, registered once, so a
    step is launches only.
    mode="plain_reregister": the same launch sequences on one shared context that registers each
    keyframe before rendering it (what a caller of the one-view splat_render does: the view
    tables are rebuilt on the host and uploaded synchronously for every keyframe of every step).
    max_pairs is the pair capacity of the batched context, or of each plain context (default:
    generous for the views it renders).
    """

    def __init__(self, params, views, targets, mode="batched", cfg: RenderConfig | None = None,
                 loss_cfg: LossConfig | None = None, adam_cfg: AdamConfig | None = None,
                 max_pairs=None):
        self.params = params
        self.n = params[0].shape[0]
        self.views = list(views)
        self.mode = mode
        self.loss_cfg = loss_cfg or LossConfig()
        self.adam_cfg = adam_cfg or AdamConfig()
        dev = params[0].device
        self.state = adam_state(self.n, dev)
        P = sum(v.rows * v.cols for v in self.views)
        if mode == "batched":
            self.ctx = SplatContext(self.n, len(self.views), P, max_pairs, cfg)
            self.ctx.set_views(self.views)
            self.t_depth = torch.cat([t[0].reshape(-1) for t in targets]).contiguous()
            self.t_normal = torch.cat([t[1].reshape(3, -1) for t in targets], 1).contiguous()
            self.loss_out = torch.zeros(1, dtype=torch.float64, device=dev)
        elif mode == "plain":
            self.ctxs = []
            for v in self.views:
                c = SplatContext(self.n, 1, v.rows * v.cols,
                                 max_pairs or default_capacity_pairs(self.n, [v]), cfg)
                c.set_views([v])
                self.ctxs.append(c)
            self.ctx = self.ctxs[0]
        elif mode == "plain_reregister":
            maxp = max(v.rows * v.cols for v in self.views)
            big = max(self.views, key=lambda v: v.rows * v.cols)
            self.ctx = SplatContext(self.n, 1, maxp,
                                    max_pairs or default_capacity_pairs(self.n, [big]), cfg)
        else:
            raise ValueError(f"unknown mode {mode!r}")
        if mode != "batched":
            self.targets = [(t[0].reshape(-1).contiguous(), t[1].reshape(3, -1).contiguous())
                            for t in targets]
            self.grads = tuple(torch.zeros_like(p) for p in params)
            self.loss_out = torch.zeros(1, dtype=torch.float64, device=dev)
        self.graph = None

    def _batched_step(self):
        self.ctx.refine_step(self.params, self.state, self.t_depth, self.t_normal, self.loss_cfg,
                             self.adam_cfg, self.loss_out)

    def _plain_step(self):
        self.loss_out.zero_()
        for k, v in enumerate(self.views):
            if self.mode == "plain":
                ctx = self.ctxs[k]
            else:
                ctx = self.ctx
                ctx.set_views([v])
            d, nrm, a = ctx.render(*self.params)
            L, gD, gN, gO = loss(d, nrm, a, self.targets[k][0], self.targets[k][1], self.loss_cfg)
            self.loss_out += L
            ctx.backward(*self.params, gD, gN, gO, out=self.grads, accumulate=k > 0)
        adam_step(self.params, self.grads, self.state, self.adam_cfg)

    def capture(self, warmup=2):
        """Capture the batched iteration in a CUDA graph (after warm-up steps on a side stream)."""
        assert self.mode == "batched"
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self._batched_step()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._batched_step()
        return self.graph

    def step(self):
        if self.mode == "batched":
            if self.graph is not None:
                self.graph.replay()
            else:
                self._batched_step()
        else:
            self._plain_step()
        return self.loss_out

    def close(self):
        """Free the contexts' device workspace."""
        for c in getattr(self, "ctxs", None) or [self.ctx]:
            c.close()

    def save(self, path):
        """Checkpoint the map and the optimiser state (save_checkpoint)."""
        torch.cuda.synchronize()
        save_checkpoint(path, self.params, self.state, {"n": self.n, "keyframes": len(self.views)})

    def load(self, path):
        """Resume from a checkpoint of a refiner of the same map size, in place (a captured
        graph stays valid)."""
        torch.cuda.synchronize()
        load_checkpoint(path, self.params, self.state)


def default_capacity_pairs(n, views, per_prim=24):
    """A generous (tile, primitive) pair capacity for n primitives over the given views."""
    return int(min(max(per_prim * n * len(views), 1 << 20), (1 << 32) - 1))


def n_tiles_of(views, th=16, tw=16):
    return sum(math.ceil(v.rows / th) * math.ceil(v.cols / tw) for v in views)


TILE_SHAPES = ((16, 16), (8, 32), (32, 8), (4, 64))


def autotune_tile(params, views, targets, shapes=TILE_SHAPES, steps=3, max_pairs=None,
                  loss_cfg: LossConfig | None = None, adam_cfg: AdamConfig | None = None):
    """Pick the tile shape with the fastest batched refinement step on this workload.

    Each candidate runs on a copy of the parameters: one warm-up step, then `steps` timed
    steps (CUDA events).  Returns ((tile_h, tile_w), {shape: ms per step})."""
    times = {}
    for th, tw in shapes:
        p = [t.clone() for t in params]
        r = Refiner(p, views, targets, mode="batched", cfg=RenderConfig(tile_h=th, tile_w=tw),
                    loss_cfg=loss_cfg, adam_cfg=adam_cfg, max_pairs=max_pairs)
        r.step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            r.step()
        b.record()
        torch.cuda.synchronize()
        times[f"{th}x{tw}"] = a.elapsed_time(b) / steps
        r.ctx.close()
        del r, p
    best = min(times, key=times.get)
    th, tw = (int(x) for x in best.split("x"))
    return (th, tw), times


class Mapper:
    """The local-model loop of Sec. 3.3 on one shared map, built from the library's calls:
    each new keyframe is registered, the map grows from it (splat_densify: the valid mask for the
    first keyframe, the densification masks M_n / M_e against a render of the current map for
    later ones), then refinement iterations (splat_refine_step) run over the registered keyframes
    with keyframe sampling (splat_set_view_sampling).  The parameters and Adam moments live in
    tensors of a fixed capacity; the first `n` rows are the map.  With max_keyframes set, only
    the most recent keyframes stay registered (a sliding window, as in a long run that refines
    over the last few keyframes of each scan); max_views and max_pixels then need to hold the
    window only."""

    def __init__(self, capacity: int, max_views: int, max_pixels: int, n_new: int,
                 cfg: RenderConfig | None = None, loss_cfg: LossConfig | None = None,
                 adam_cfg: AdamConfig | None = None, densify_cfg: DensifyConfig | None = None,
                 draws: int = 2, p_newest: float = 0.4, seed: int = 0, device="cuda",
                 max_keyframes: int | None = None):
        if max_keyframes is not None and not 1 <= int(max_keyframes) <= int(max_views):
            raise ValueError("max_keyframes must lie in [1, max_views]")
        self.max_keyframes = None if max_keyframes is None else int(max_keyframes)
        self.capacity, self.n_new = int(capacity), int(n_new)
        self.draws, self.p_newest, self.seed = int(draws), float(p_newest), int(seed)
        self.loss_cfg = loss_cfg or LossConfig(lambda_n=0.1, normal_mode=1)
        self.adam_cfg = adam_cfg or AdamConfig()
        self.densify_cfg = densify_cfg or DensifyConfig()
        dev = torch.device(device)
        self.ctx = SplatContext(self.capacity, max_views, max_pixels, None, cfg)
        self.params = [torch.zeros(self.capacity, w, device=dev) for w in (4, 4, 2)]
        self.state = adam_state(self.capacity, dev)
        self.n = 0
        self.views: list = []
        self.targets: list = []   # (depth (P,), normal (3, P)) of each registered keyframe
        self.t_depth = torch.zeros(0, device=dev)
        self.t_normal = torch.zeros(3, 0, device=dev)
        self.loss_out = torch.zeros(1, dtype=torch.float64, device=dev)

    def _rows(self, ts):
        return [t[:self.n] for t in ts]

    def add_keyframe(self, view, target_depth, target_normal) -> int:
        """Register a keyframe with its target range (H, W) and normals (3, H, W), grow the map
        from it by n_new slots and return the map size."""
        if self.n + self.n_new > self.capacity:
            raise ValueError("map capacity exhausted")
        td = target_depth.reshape(-1).to(self.t_depth.device, torch.float32)
        tn = target_normal.reshape(3, -1).to(self.t_depth.device, torch.float32)
        self.views.append(view)
        self.targets.append((td, tn))
        if self.max_keyframes is not None and len(self.views) > self.max_keyframes:
            del self.views[0]
            del self.targets[0]
        self.ctx.set_views(self.views)
        self.t_depth = torch.cat([t[0] for t in self.targets]).contiguous()
        self.t_normal = torch.cat([t[1] for t in self.targets], 1).contiguous()
        # only the new keyframe's pixels are drawn from
        only_new = torch.zeros_like(self.t_depth)
        o = self.ctx.offsets[-1]
        only_new[o:o + td.numel()] = td
        cfg = DensifyConfig(**{**self.densify_cfg.__dict__, "refine": self.n > 0})
        depth = alpha = None
        if self.n > 0:
            depth, _, alpha = self.ctx.render(*self._rows(self.params))
        self.ctx.densify(self.params, self.n, self.n_new, only_new, depth, alpha, cfg)
        self.n += self.n_new
        return self.n

    def refine(self, iters: int, read_losses: bool = True) -> list[float]:
        """Refinement iterations over the registered keyframes, each on the keyframes drawn for
        it (a fresh random stream per call); returns each iteration's loss (read_losses=False:
        nothing is read back and the list is empty -- no host synchronisation; the last loss
        stays in loss_out).  Sampling is off outside this call, so renders cover every
        keyframe."""
        m_pl, m_q, m_ls, v_pl, v_q, v_ls, step = self.state
        self._refines = getattr(self, "_refines", 0) + 1
        if self.draws > 0 and len(self.views) > 1:
            self.ctx.set_view_sampling(self.draws, self.p_newest,
                                       self.seed + 1000003 * self._refines)
        losses = []
        try:
            for _ in range(int(iters)):
                self.ctx.refine_step(self._rows(self.params),
                                     (*self._rows((m_pl, m_q, m_ls, v_pl, v_q, v_ls)), step),
                                     self.t_depth, self.t_normal, self.loss_cfg, self.adam_cfg,
                                     self.loss_out)
                if read_losses:
                    losses.append(float(self.loss_out.item()))
        finally:
            self.ctx.set_view_sampling(0)
        return losses

    def render(self):
        """Packed (depth, normal, alpha) of the registered keyframes for the current map."""
        return self.ctx.render(*self._rows(self.params))
