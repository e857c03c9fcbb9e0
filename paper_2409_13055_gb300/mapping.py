"""Mapping-step driver over the C-ABI: map storage, rasteriser, autograd, graphs.

PyTorch provides device memory, streams and CUDA-graph capture here; every
arithmetic step of the mapping iteration (paper Sec. III-B: render with the
3DGS tile rasteriser, Eq. 2 loss, gradient descent with the default 3DGS
Adam of Sec. IV-A) runs in libgs_gb300.so.

* ``GaussianMap`` keeps every parameter group in ONE contiguous float32
  buffer (means | log_scales | quats | opacity_logits | sh[K][N][3]), each
  group starting on a 256-byte boundary, with gradients and Adam moments in
  buffers of the same layout -- so the fused Adam kernel is one pass and a
  later cross-GPU all-reduce of the gradient would be one call.
* ``Rasterizer`` owns a plan and its workspace for one batch of views; a
  recompute rasteriser (checkpointing) keeps the projection and binning of
  a few views in its workspace, runs the views through it a pass at a time
  and repeats a pass's projection and binning in the backward.
* ``GSRender`` is the torch.autograd.Function over the rasteriser; with a
  recompute rasteriser only (final_T, last_idx) survive from the forward to
  the backward, and several of them may share one workspace.
* ``MappingStep`` is one whole iteration, optionally captured as a CUDA graph.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

ALIGN_FLOATS = 64  # 256-byte group alignment
GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh_dc", "sh_rest")
GROUP_STRIDES = (3, 3, 4, 1, 3, 3)  # floats per Gaussian per plane of each group

# Default learning rates of 3DGS (the paper keeps the default optimiser
# configuration, Sec. IV-A); the position rate is scaled by the scene extent.
DEFAULT_LR = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, opacity_logits=0.05,
                  sh_dc=2.5e-3, sh_rest=2.5e-3 / 20.0)


def _align(x):
    return (x + ALIGN_FLOATS - 1) // ALIGN_FLOATS * ALIGN_FLOATS


def param_layout(n: int, degree: int):
    """Offsets (floats) of each group in the packed buffer, and the total."""
    K = (degree + 1) ** 2
    off = {}
    o = 0
    off["means"] = o
    o = _align(o + 3 * n)
    off["log_scales"] = o
    o = _align(o + 3 * n)
    off["quats"] = o
    o = _align(o + 4 * n)
    off["opacity_logits"] = o
    o = _align(o + n)
    off["sh"] = o
    off["sh_dc"] = o
    off["sh_rest"] = o + 3 * n
    o = _align(o + 3 * K * n)
    return off, o


class GaussianMap:
    """Gaussian parameters, gradients and Adam state on one GPU."""

    def __init__(self, params, device="cuda", capacity=None):
        self.n = int(params["means"].shape[0])
        self.degree = int(params["sh_degree"])
        self.K = (self.degree + 1) ** 2
        self.capacity = int(capacity or self.n)
        self.device = torch.device(device)
        self.off, self.total = param_layout(self.capacity, self.degree)
        self.data = torch.zeros(self.total, dtype=torch.float32, device=self.device)
        self.grad = torch.zeros_like(self.data)
        self.m = torch.zeros_like(self.data)
        self.v = torch.zeros_like(self.data)
        self.step = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.load(params)

    # views into the packed buffers ------------------------------------------
    def _views(self, buf, layout=None):
        n, c, K = self.n, self.capacity, self.K
        o = self.off
        if layout is not None:  # (n, offsets) of a buffer laid out for another size
            n, o = layout
            c = n
        return dict(
            means=buf[o["means"]:o["means"] + 3 * n].view(n, 3),
            log_scales=buf[o["log_scales"]:o["log_scales"] + 3 * n].view(n, 3),
            quats=buf[o["quats"]:o["quats"] + 4 * n].view(n, 4),
            opacity_logits=buf[o["opacity_logits"]:o["opacity_logits"] + n],
            sh=buf[o["sh"]:o["sh"] + 3 * K * c].view(K, c, 3)[:, :n],
        )

    def params(self):
        return self._views(self.data)

    def grads(self):
        return self._views(self.grad)

    def load(self, params):
        assert params["means"].shape[0] == self.n
        P = self.params()
        for k in ("means", "log_scales", "quats", "opacity_logits"):
            P[k].copy_(torch.as_tensor(np.asarray(params[k], np.float32)))
        sh = torch.as_tensor(np.asarray(params["sh"], np.float32))
        self.data[self.off["sh"]:self.off["sh"] + 3 * self.K * self.capacity].view(
            self.K, self.capacity, 3)[:, :self.n].copy_(sh)

    def append(self, params):
        """Insert Gaussians after the current ones (streaming insertion): the
        packed buffers are laid out again for the new size and the old values
        copied over, the new Gaussians' Adam moments start at zero and the
        step counter is kept, as when new entries join a running Adam.  Every
        device pointer of the map changes, so rasterisers may be reused but
        captured graphs must be captured again."""
        k = int(params["means"].shape[0])
        if int(params["sh_degree"]) != self.degree:
            raise ValueError("SH degree differs from the map's")
        n0, cap0, off0 = self.n, self.capacity, self.off
        n1 = n0 + k
        off1, total1 = param_layout(n1, self.degree)
        widths = dict(means=3, log_scales=3, quats=4, opacity_logits=1)

        def relayout(old, copy):
            new = torch.zeros(total1, dtype=torch.float32, device=self.device)
            if copy:
                for g, w in widths.items():
                    new[off1[g]:off1[g] + w * n0].copy_(old[off0[g]:off0[g] + w * n0])
                new[off1["sh"]:off1["sh"] + 3 * self.K * n1].view(self.K, n1, 3)[:, :n0].copy_(
                    old[off0["sh"]:off0["sh"] + 3 * self.K * cap0].view(self.K, cap0, 3)[:, :n0])
            return new

        self.data = relayout(self.data, True)
        self.m = relayout(self.m, True)
        self.v = relayout(self.v, True)
        self.grad = relayout(self.grad, False)
        self.n = self.capacity = n1
        self.off, self.total = off1, total1
        P = self.params()
        for g in widths:
            P[g][n0:].copy_(torch.as_tensor(np.asarray(params[g], np.float32)).reshape(P[g][n0:].shape))
        P["sh"][:, n0:].copy_(torch.as_tensor(np.asarray(params["sh"], np.float32)))

    def densify(self, accum, denom, samples, extent=1.0, grad_threshold=0.0004,
                percent_dense=0.01, min_opacity=0.005, split_shrink=1.6, stream=None):
        """Adaptive density control (paper Sec. III-B; rules in gs.h): prune
        low-opacity Gaussians, clone small and split large ones whose mean
        statistic accum/denom reaches grad_threshold.  samples: device float
        tensor [n][2][3] of standard normal draws for the split offsets.  One
        host synchronisation reads the new size; the buffers are laid out
        again for it (pointers change), moments of new Gaussians are zero and
        the step counter is kept.  Returns (kept, cloned, split)."""
        cfg = B.gs_densify_config(float(grad_threshold), float(percent_dense), float(min_opacity),
                                  float(split_shrink), float(extent))
        scratch = torch.empty(max(1, B.gs_densify_scratch_bytes(self.n)), dtype=torch.uint8,
                              device=self.device)
        counts = torch.zeros(4, dtype=torch.int32, device=self.device)
        src = self.gs_map()
        B.gs_densify_count(src, accum, denom, cfg, scratch, counts, stream)
        kept, cloned, split, _ = (int(x) for x in counts.cpu().tolist())
        n_out = kept + cloned + 2 * split
        if n_out == 0:
            raise ValueError("density control would remove every Gaussian")
        off1, total1 = param_layout(n_out, self.degree)
        lay = (n_out, off1)
        bufs = [torch.zeros(total1, dtype=torch.float32, device=self.device) for _ in range(4)]
        data1, m1, v1, grad1 = bufs
        sm, sv = self.gs_map_moments()
        B.gs_densify_apply(src, sm, sv, accum, denom, samples, cfg, scratch, n_out,
                           self._struct(data1, lay), self._struct(m1, lay), self._struct(v1, lay),
                           counts, stream)
        if int(counts[3].item()) != 0:
            raise RuntimeError("gs_densify_apply: output size mismatch")
        self.data, self.m, self.v, self.grad = data1, m1, v1, grad1
        self.n = self.capacity = n_out
        self.off, self.total = off1, total1
        return kept, cloned, split

    def permute(self, perm: torch.Tensor):
        """Reorders the Gaussians (parameters, gradients and moments) so that
        new index i holds old Gaussian perm[i]; renders are unchanged except
        for the order of exactly tied depths."""
        perm = perm.to(self.device, torch.int64)
        for buf in (self.data, self.grad, self.m, self.v):
            V = self._views(buf)
            for k, t in V.items():
                if k == "sh":
                    t.copy_(t[:, perm].clone())
                else:
                    t.copy_(t[perm].clone())

    def to_numpy(self):
        P = self.params()
        out = {k: P[k].detach().cpu().numpy().copy() for k in P}
        out["sh_degree"] = self.degree
        return out

    def gs_map(self) -> B.gs_map:
        P = self.params()
        if self.capacity != self.n:
            raise ValueError("SH planes are strided by capacity; use capacity == n for the C-ABI")
        return B.gs_map(P["means"].data_ptr(), P["log_scales"].data_ptr(), P["quats"].data_ptr(),
                        P["opacity_logits"].data_ptr(), P["sh"].data_ptr(), self.n, self.degree)

    def gs_map_grad(self) -> B.gs_map_grad:
        G = self.grads()
        return B.gs_map_grad(G["means"].data_ptr(), G["log_scales"].data_ptr(),
                             G["quats"].data_ptr(), G["opacity_logits"].data_ptr(),
                             G["sh"].data_ptr())

    def _struct(self, buf, layout=None) -> B.gs_map_grad:
        V = self._views(buf, layout)
        return B.gs_map_grad(V["means"].data_ptr(), V["log_scales"].data_ptr(),
                             V["quats"].data_ptr(), V["opacity_logits"].data_ptr(),
                             V["sh"].data_ptr())

    def gs_map_params(self) -> B.gs_map_grad:
        """The parameter arrays as writable pointers (in-place Adam target)."""
        return self._struct(self.data)

    def gs_map_moments(self):
        return self._struct(self.m), self._struct(self.v)

    def group_lr(self, lr=None, extent=1.0):
        """Learning rates of means, log-scales, quats, opacity, SH DC, SH rest."""
        lr = dict(DEFAULT_LR, **(lr or {}))
        return [lr["means"] * extent] + [lr[g] for g in GROUPS[1:]]

    def adam_groups(self, lr=None, extent=1.0):
        """(offsets, rates) of the six Adam groups over the packed buffer."""
        lr = dict(DEFAULT_LR, **(lr or {}))
        lr = dict(lr, means=lr["means"] * extent)
        starts = [self.off[g] for g in GROUPS]
        offsets = starts + [self.total]
        offsets[0] = 0
        return offsets, [lr[g] for g in GROUPS]

    def adam_step(self, lr=None, extent=1.0, beta1=0.9, beta2=0.999, eps=1e-15, stream=None,
                  visible=None, group_vis=None):
        """One Adam step; with visible (device uint8 [n], e.g. from
        Rasterizer.visibility) the visibility-masked variant; with group_vis
        (from Rasterizer.project_bwd_groups) the same dense step, the
        gradient of the zero groups not read."""
        offs, rates = self.adam_groups(lr, extent)
        if (visible is not None or group_vis is not None) and self.capacity != self.n:
            raise ValueError("the masked and grouped steps need a map without spare capacity")
        if group_vis is not None:
            B.gs_adam_step_groups(self.data, self.grad, self.m, self.v, offs, rates,
                                  GROUP_STRIDES, self.n, group_vis, beta1, beta2, eps, self.step,
                                  stream)
        elif visible is None:
            B.gs_adam_step(self.data, self.grad, self.m, self.v, offs, rates, beta1, beta2, eps,
                           self.step, stream)
        else:
            B.gs_adam_step_sparse(self.data, self.grad, self.m, self.v, offs, rates,
                                  GROUP_STRIDES, self.n, visible, beta1, beta2, eps, self.step,
                                  stream)


def morton_order(means: torch.Tensor, bits: int = 10) -> torch.Tensor:
    """Permutation sorting 3D points along a Z-order curve over their
    bounding box (bits per axis): neighbours in space become neighbours in
    index, so a view's visible Gaussians form long runs in memory."""
    lo = means.min(0).values
    span = (means.max(0).values - lo).clamp_min(1e-12)
    q = ((means - lo) / span * ((1 << bits) - 1)).round().to(torch.int64)
    code = torch.zeros(means.shape[0], dtype=torch.int64, device=means.device)
    for b in range(bits):
        for a in range(3):
            code |= ((q[:, a] >> b) & 1) << (3 * b + a)
    return torch.argsort(code, stable=True)


def make_view(v) -> B.gs_view:
    R = np.asarray(v["R"], np.float32).reshape(9)
    t = np.asarray(v["t"], np.float32).reshape(3)
    return B.gs_view((B.c_float * 9)(*R.tolist()), (B.c_float * 3)(*t.tolist()), float(v["fx"]),
                     float(v["fy"]), float(v["cx"]), float(v["cy"]), int(v["width"]),
                     int(v["height"]), int(v.get("channels", 3)), 0)


def views_to_device(views, device="cuda"):
    arr = (B.gs_view * len(views))(*[make_view(v) for v in views])
    raw = np.frombuffer(bytes(arr), dtype=np.uint8).copy()
    return arr, torch.from_numpy(raw).to(device)


def make_config(tile=(16, 16), smem_batch=128, near_z=0.2, bg=(0.0, 0.0, 0.0),
                pixels_per_thread=0, smem_batch_bwd=0, pixels_per_thread_bwd=0,
                density_stats=False, deterministic=False, tight_rect=True,
                recompute=False) -> B.gs_config:
    """The gs_config of a rasteriser (the defaults of Rasterizer)."""
    return B.gs_config(int(tile[0]), int(tile[1]), int(smem_batch), int(pixels_per_thread),
                       int(smem_batch_bwd), int(pixels_per_thread_bwd), float(near_z),
                       (B.c_float * 3)(*[float(x) for x in bg]), int(bool(density_stats)),
                       int(bool(deterministic)), int(bool(tight_rect)), int(recompute))


def plan_workspace_bytes(views, n_capacity, instance_capacity, **cfg) -> int:
    """Workspace bytes a rasteriser with these views, capacities and
    configuration (make_config's keywords) would need; allocates nothing."""
    plan = B.gs_plan_init(make_config(**cfg), [make_view(v) for v in views], int(n_capacity),
                          int(instance_capacity))
    return B.gs_plan_workspace_bytes(plan)


class Rasterizer:
    """Plan + workspace + output buffers for one batch of views.

    recompute: a checkpointing plan (gs_config.recompute): the workspace
    holds the projection and binning of `recompute` views (True: one);
    forward() and render_bwd() run the views in passes of that many, and
    the backward repeats each pass's projection and binning (bit-identical)
    before its adjoint.  instance capacity is then per pass.  workspace: a uint8 CUDA tensor to use
    instead of allocating one (at least workspace_bytes long); recompute
    rasterisers used one after the other may share one, since nothing in
    it outlives a call sequence."""

    def __init__(self, views, n_capacity, instance_capacity=None, tile=(16, 16), smem_batch=128,
                 near_z=0.2, bg=(0.0, 0.0, 0.0), pixels_per_thread=0, smem_batch_bwd=0,
                 pixels_per_thread_bwd=0, density_stats=False, deterministic=False,
                 tight_rect=True, recompute=False, workspace=None, device="cuda"):
        self.views = list(views)
        self.device = torch.device(device)
        self.views_per_pass = (int(recompute) if recompute else len(self.views))
        self.recompute = bool(recompute)
        self.cfg = make_config(tile, smem_batch, near_z, bg, pixels_per_thread, smem_batch_bwd,
                               pixels_per_thread_bwd, density_stats, deterministic, tight_rect,
                               self.views_per_pass if self.recompute else 0)
        self.n_capacity = int(n_capacity)
        if instance_capacity is None:
            k = self.views_per_pass
            sizes = [v["width"] * v["height"] for v in self.views]
            px = max(sum(sizes[i:i + k]) for i in range(0, len(sizes), k))  # per binning call
            instance_capacity = max(1 << 20, 4 * px, 8 * n_capacity)
        self.instance_capacity = int(instance_capacity)
        self.host_views, self.views_dev = views_to_device(self.views, self.device)
        self.plan = B.gs_plan_init(self.cfg, list(self.host_views), self.n_capacity,
                                   self.instance_capacity)
        # the plans the per-view calls take: the plan itself, or the passes of
        # a recompute plan whose views do not fit one pass
        n_passes = B.gs_plan_passes(self.plan)
        if self.recompute and n_passes > 1:
            self.passes = [B.gs_plan_view_pass(self.plan, k) for k in range(n_passes)]
        else:
            self.passes = [self.plan]
        self.workspace_bytes = B.gs_plan_workspace_bytes(self.plan)
        if workspace is not None:
            dev = workspace.device
            if (workspace.dtype != torch.uint8 or dev.type != self.device.type
                    or (self.device.index is not None and dev.index != self.device.index)
                    or workspace.numel() < self.workspace_bytes
                    or workspace.data_ptr() % 256 != 0):
                raise ValueError("workspace: a 256-byte aligned uint8 tensor of at least "
                                 f"{self.workspace_bytes} bytes on {self.device}")
            self.ws = workspace
        else:
            self.ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            self.ws.zero_()
        # forwards run so far (GSRender checks that its backward follows its
        # own forward in a plan that keeps the projection)
        self.generation = 0
        tot = B.gs_plan_totals(self.plan)
        self.total_values, self.total_pixels = tot["total_values"], tot["total_pixels"]
        self.total_tiles = tot["total_tiles"]
        self.view_info = [B.gs_plan_view(self.plan, v) for v in range(len(self.views))]
        self.images = torch.zeros(self.total_values, dtype=torch.float32, device=self.device)
        self.final_T = torch.zeros(self.total_pixels, dtype=torch.float32, device=self.device)
        self.last_idx = torch.zeros(self.total_pixels, dtype=torch.int32, device=self.device)
        self.dL = torch.zeros(self.total_values, dtype=torch.float32, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)

    # per-view slices --------------------------------------------------------
    def view_slice(self, buf, v, per_pixel=False):
        vw, info = self.views[v], self.view_info[v]
        H, W, C = vw["height"], vw["width"], vw.get("channels", 3)
        if per_pixel:
            return buf[info["pixel_offset"]:info["pixel_offset"] + H * W].view(H, W)
        return buf[info["value_offset"]:info["value_offset"] + C * H * W].view(C, H, W)

    def pack(self, per_view_images):
        """Concatenate [C][H][W] arrays of every view into one packed tensor."""
        flat = [torch.as_tensor(np.asarray(x, np.float32)).reshape(-1) for x in per_view_images]
        return torch.cat(flat).to(self.device)

    def buffer(self, buf_id, dtype=torch.uint8, view=None):
        """A workspace buffer (of pass `view` in a recompute plan)."""
        off, nbytes = B.gs_plan_buffer(self._pass(view), buf_id)
        return self.ws[off:off + nbytes].view(dtype)

    def _pass(self, view):
        if view is None:
            if len(self.passes) > 1:
                raise ValueError("a recompute plan of several passes runs one pass at a time: "
                                 "pass view= (the pass index)")
            return self.passes[0]
        return self.passes[view]

    def set_poses(self, views):
        """Copy new poses (same sizes) to the device copy read by the kernels."""
        arr, dev = views_to_device(views, self.device)
        self.views_dev.copy_(dev)

    # the C-ABI steps (view: the pass index of a recompute plan) ----------------
    def project(self, gmap: B.gs_map, stream=None, view=None):
        B.gs_project(self._pass(view), gmap, self.views_dev, self.ws, stream)

    def bin_sort(self, n, stream=None, view=None):
        B.gs_bin_sort(self._pass(view), n, self.ws, stream)

    def render_fwd(self, images=None, final_T=None, last_idx=None, stream=None, view=None):
        B.gs_render_fwd(self._pass(view), self.ws, self.images if images is None else images,
                        self.final_T if final_T is None else final_T,
                        self.last_idx if last_idx is None else last_idx, stream)

    def forward(self, gmap: B.gs_map, stream=None, images=None, final_T=None, last_idx=None):
        """Projection, binning and compositing of every view (pass by pass in
        a recompute plan)."""
        for v in range(len(self.passes)):
            self.project(gmap, stream, view=v)
            self.bin_sort(gmap.n, stream, view=v)
            self.render_fwd(images, final_T, last_idx, stream=stream, view=v)
        self.generation += 1

    def max_instances(self, gmap: B.gs_map):
        """Largest (Gaussian, tile) instance count any binning call of this
        plan needs for gmap (one synchronising read per pass)."""
        raw = 0
        for v in range(len(self.passes)):
            self.project(gmap, view=v)
            self.bin_sort(gmap.n, view=v)
            raw = max(raw, int(self.counters().n_instances_raw))
        return raw

    def loss_l1_ssim(self, targets, lam, view_weight=None, images=None, stream=None):
        w = 1.0 / len(self.views) if view_weight is None else view_weight
        B.gs_loss_l1_ssim(self.plan, self.images if images is None else images, targets, lam, w,
                          self.loss, self.dL, self.ws, stream)

    def render_bwd(self, gmap: B.gs_map, grads: B.gs_map_grad, dL=None, final_T=None,
                   last_idx=None, accumulate=False, stream=None):
        """Pixel and projection adjoints of every view; in a recompute plan
        each pass's projection and binning are run again first."""
        args = (self.final_T if final_T is None else final_T,
                self.last_idx if last_idx is None else last_idx, self.dL if dL is None else dL)
        for v, pl in enumerate(self.passes):
            if self.recompute:
                self.project(gmap, stream, view=v)
                self.bin_sort(gmap.n, stream, view=v)
            B.gs_render_bwd(pl, gmap, self.views_dev, self.ws, *args, grads,
                            accumulate or v > 0, stream)

    def render_bwd_pixels(self, dL=None, final_T=None, last_idx=None, stream=None, view=None):
        B.gs_render_bwd_pixels(self._pass(view), self.ws,
                               self.final_T if final_T is None else final_T,
                               self.last_idx if last_idx is None else last_idx,
                               self.dL if dL is None else dL, stream)

    def project_bwd(self, gmap: B.gs_map, grads: B.gs_map_grad, accumulate=False, stream=None,
                    view=None):
        B.gs_project_bwd(self._pass(view), gmap, self.views_dev, self.ws, grads, accumulate,
                         stream)

    def project_bwd_groups(self, gmap: B.gs_map, grads: B.gs_map_grad, group_vis, stream=None):
        """The projection adjoint writing only groups of GS_GRAD_GROUP
        Gaussians that touch a tile (group_vis records which)."""
        B.gs_project_bwd_groups(self.plan, gmap, self.views_dev, self.ws, grads, group_vis,
                                stream)

    def project_bwd_adam(self, gmap: GaussianMap, lr=None, extent=1.0, grads_acc=None,
                         grads_out=None, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
        """Projection adjoint fused with one Adam step on gmap (in place)."""
        mm, vv = gmap.gs_map_moments()
        B.gs_project_bwd_adam(self.plan, gmap.gs_map(), self.views_dev, self.ws,
                              gmap.gs_map_params(), mm, vv, gmap.group_lr(lr, extent), beta1,
                              beta2, eps, gmap.step, grads_acc=grads_acc, grads_out=grads_out,
                              stream=stream)

    def visibility(self, n, vis, stream=None):
        """vis[i] = 1 where Gaussian i touched a tile in the last projection."""
        B.gs_visibility(self.plan, n, self.ws, vis, stream)

    def densify_stats(self, n, accum, denom, stream=None, view=None):
        """Adds the last backward's density-control statistic (plan built
        with density_stats) to accum / denom."""
        B.gs_densify_stats(self._pass(view), n, self.ws, accum, denom, stream)

    def counters(self, stream=None) -> B.gs_counters:
        return B.gs_read_counters(self.plan, self.ws, stream)


def fit_instance_capacity(views, gmap: GaussianMap, headroom=1.25, **kw):
    """A rasteriser whose instance capacity fits this map with headroom (one
    synchronising probe at set-up, none afterwards)."""
    probe = Rasterizer(views, gmap.capacity, **kw)
    raw = probe.max_instances(gmap.gs_map())
    if raw > probe.instance_capacity:
        kw = dict(kw)
        probe = Rasterizer(views, gmap.capacity, instance_capacity=int(raw * headroom) + 1024, **kw)
        return probe
    cap = int(raw * headroom) + 1024
    if cap < probe.instance_capacity:
        return Rasterizer(views, gmap.capacity, instance_capacity=cap, **kw)
    return probe


def _map_from_tensors(means, log_scales, quats, opacity_logits, sh, degree):
    for t in (means, log_scales, quats, opacity_logits, sh):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("GSRender inputs must be contiguous float32 CUDA tensors")
    return B.gs_map(means.data_ptr(), log_scales.data_ptr(), quats.data_ptr(),
                    opacity_logits.data_ptr(), sh.data_ptr(), means.shape[0], degree)


class GSRender(torch.autograd.Function):
    """images = GSRender.apply(means, log_scales, quats, opacity_logits, sh, rast, recompute)

    sh is [K][N][3]; the result is the rasteriser's packed image buffer.  The
    backward calls gs_render_bwd.  With a recompute rasteriser
    (Rasterizer(recompute=True)) only final_T and last_idx survive from the
    forward, and every view's projection and binning run again in the
    backward: any number of renders may wait for their backward in one
    autograd graph, and their rasterisers may share one workspace.
    Otherwise the backward reads the projection and binning that the
    forward left in the rasteriser's workspace, so it must come before the
    next forward on that rasteriser (it raises if not), unless recompute=True
    asks for them to be run again into the same workspace.
    """

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, rast: Rasterizer,
                recompute=False):
        degree = int(round(sh.shape[0] ** 0.5)) - 1
        gmap = _map_from_tensors(means, log_scales, quats, opacity_logits, sh, degree)
        rast.forward(gmap)
        images = rast.images.clone()
        final_T = rast.final_T.clone()
        last_idx = rast.last_idx.clone()
        ctx.rast, ctx.degree = rast, degree
        ctx.recompute = bool(recompute) or rast.recompute
        ctx.generation = rast.generation
        ctx.save_for_backward(means, log_scales, quats, opacity_logits, sh, final_T, last_idx)
        return images

    @staticmethod
    def backward(ctx, dimages):
        means, log_scales, quats, opacity_logits, sh, final_T, last_idx = ctx.saved_tensors
        rast = ctx.rast
        gmap = _map_from_tensors(means, log_scales, quats, opacity_logits, sh, ctx.degree)
        if ctx.recompute and not rast.recompute:
            rast.project(gmap)
            rast.bin_sort(gmap.n)
        elif not ctx.recompute and rast.generation != ctx.generation:
            raise RuntimeError("GSRender: the rasteriser ran another forward after this one; its "
                               "workspace no longer holds this render's projection (use a "
                               "recompute rasteriser, recompute=True, or one rasteriser per "
                               "pending render)")
        g = [torch.zeros_like(t) for t in (means, log_scales, quats, opacity_logits, sh)]
        grads = B.gs_map_grad(*[t.data_ptr() for t in g])
        rast.render_bwd(gmap, grads, dL=dimages.contiguous(), final_T=final_T, last_idx=last_idx)
        return (*g, None, None)


class L1SSIMLoss(torch.autograd.Function):
    """loss = L1SSIMLoss.apply(images, targets, rast, lam): Eq. 2 (read as
    (1 - lam) mean|I - I_gt| + lam (1 - mean SSIM), the mean over the
    rasteriser's views) on packed images, with its analytic gradient from
    the same gs_loss_l1_ssim call."""

    @staticmethod
    def forward(ctx, images, targets, rast: Rasterizer, lam):
        images = images.contiguous()
        loss = torch.zeros(1, dtype=torch.float32, device=images.device)
        dL = torch.empty_like(images)
        B.gs_loss_l1_ssim(rast.plan, images, targets, lam, 1.0 / len(rast.views), loss, dL,
                          rast.ws)
        ctx.save_for_backward(dL)
        return loss[0]

    @staticmethod
    def backward(ctx, gout):
        (dL,) = ctx.saved_tensors
        return dL * gout, None, None, None


class MappingStep:
    """One mapping iteration (project, bin, render, loss, backward, Adam) on a
    batch of views, optionally captured as one CUDA graph."""

    def __init__(self, gmap: GaussianMap, rast: Rasterizer, targets: torch.Tensor, lam: float,
                 lr=None, extent=1.0, fused=False, keep_grads=False, recompute=None,
                 stats=None, sparse_adam=False):
        self.gmap, self.rast, self.targets, self.lam = gmap, rast, targets, float(lam)
        self.lr, self.extent, self.fused, self.keep_grads = lr, extent, fused, keep_grads
        # sparse_adam: the visibility-masked Adam variant (Gaussians that touch
        # no tile of any view in this iteration keep parameters and moments)
        self.visible = (torch.zeros(gmap.n, dtype=torch.uint8, device=gmap.device)
                        if sparse_adam else None)
        # stats = (accum, denom): the density-control statistic of every
        # iteration is added to them (the rasteriser needs density_stats)
        self.stats = stats
        # recompute: the checkpointed backward -- projection and binning are
        # run again (bit-identically) between the loss and the adjoint.  With
        # a recompute rasteriser (the default then) the views go through its
        # workspace a pass at a time; recompute=True with another rasteriser
        # re-runs them into the same workspace
        self.recompute = rast.recompute if recompute is None else bool(recompute)
        self.passes = len(rast.passes) if rast.recompute else 1
        if self.passes > 1 and (fused or sparse_adam):
            raise ValueError("the fused and visibility-masked steps need every view at once; "
                             "a recompute rasteriser of several passes runs them a pass at a time")
        # without keep_grads the gradient of groups of GS_GRAD_GROUP Gaussians
        # that touch no tile (all zero) is neither written nor read
        self.groups = (not keep_grads and not fused and self.visible is None
                       and gmap.capacity == gmap.n and self.passes == 1)
        if self.groups:
            ng = (gmap.n + B.GS_GRAD_GROUP - 1) // B.GS_GRAD_GROUP
            self.group_vis = torch.zeros(ng, dtype=torch.uint8, device=gmap.device)
        self.graph = None
        self._m = gmap.gs_map()
        self._g = gmap.gs_map_grad()

    def run(self, stream=None):
        self.run_front(stream)
        self.run_back(stream)

    def run_front(self, stream=None):
        """Projection, binning and forward render (reads the views, not the
        targets)."""
        self.rast.forward(self._m, stream)

    def run_back(self, stream=None):
        """Loss, backward and optimiser step (reads the targets)."""
        r = self.rast
        r.loss_l1_ssim(self.targets, self.lam, stream=stream)
        if r.recompute and self.passes > 1:
            # a pass at a time through the workspace: its projection and
            # binning again, its pixel and projection adjoints (gradients
            # summed over the passes), its statistic
            for v in range(self.passes):
                r.project(self._m, stream, view=v)
                r.bin_sort(self.gmap.n, stream, view=v)
                r.render_bwd_pixels(stream=stream, view=v)
                r.project_bwd(self._m, self._g, accumulate=v > 0, stream=stream, view=v)
                if self.stats is not None:
                    r.densify_stats(self.gmap.n, self.stats[0], self.stats[1], stream, view=v)
            self.gmap.adam_step(self.lr, self.extent, stream=stream)
            return
        if self.recompute:
            r.project(self._m, stream)
            r.bin_sort(self.gmap.n, stream)
        if self.fused:
            # Adam applied inside the projection adjoint (fewer bytes moved,
            # but slower than the two passes on this workload); the gradients
            # are written to gmap.grad only when asked for
            r.render_bwd_pixels(stream=stream)
            r.project_bwd_adam(self.gmap, self.lr, self.extent,
                               grads_out=self._g if self.keep_grads else None, stream=stream)
        else:
            if self.groups:
                r.render_bwd_pixels(stream=stream)
                r.project_bwd_groups(self._m, self._g, self.group_vis, stream)
                self.gmap.adam_step(self.lr, self.extent, stream=stream,
                                    group_vis=self.group_vis)
            else:
                r.render_bwd(self._m, self._g, accumulate=False, stream=stream)
                if self.visible is not None:
                    r.visibility(self.gmap.n, self.visible, stream)
                self.gmap.adam_step(self.lr, self.extent, stream=stream, visible=self.visible)
        if self.stats is not None:
            r.densify_stats(self.gmap.n, self.stats[0], self.stats[1], stream)

    def capture(self, warmup=2):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.run()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def __call__(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.run()


class HostPipeline:
    """Mapping iterations fed from pinned host memory: each call to `submit`
    copies one iteration's targets and camera poses host -> device, runs the
    iteration (one CUDA graph) and copies its loss device -> host.

    No copy sits on the compute stream: inputs and the loss alternate
    between two sets of device buffers, each set with its own captured graph.
    The uploads of iteration i (on an upload stream) run while iteration i-1
    computes from the other set; the loss of iteration i is read back on a
    download stream once its graph ends, while iteration i+1 runs; a set is
    refilled only after the loss read of its previous iteration.  `submit`
    returns the previous iteration's loss (None for the first); `drain` waits
    for and returns the last one."""

    def __init__(self, step: MappingStep, warmup=2):
        self.step = step
        self.rast = step.rast
        self.up = torch.cuda.Stream()
        self.down = torch.cuda.Stream()
        self.targets = [step.targets, torch.empty_like(step.targets)]
        self.views = [self.rast.views_dev, self.rast.views_dev.clone()]
        self.loss = [self.rast.loss, torch.zeros_like(self.rast.loss)]
        self.host_loss = [torch.empty(1, dtype=torch.float32).pin_memory() for _ in range(2)]
        self.ev_in = [torch.cuda.Event(), torch.cuda.Event()]
        self.ev_done = [torch.cuda.Event(), torch.cuda.Event()]
        self.ev_loss = [torch.cuda.Event(), torch.cuda.Event()]
        self.i = 0
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                step.run()
        torch.cuda.current_stream().wait_stream(s)
        # one graph per buffer set: the buffers' addresses are baked in
        self.graphs = []
        for b in range(2):
            self._use(b)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step.run()
            self.graphs.append(g)
        self._use(0)
        main = torch.cuda.current_stream()
        for e in self.ev_loss:
            e.record(main)

    def _use(self, b):
        self.step.targets = self.targets[b]
        self.rast.views_dev = self.views[b]
        self.rast.loss = self.loss[b]

    def submit(self, host_targets: torch.Tensor, host_views: torch.Tensor):
        main = torch.cuda.current_stream()
        b = self.i & 1
        with torch.cuda.stream(self.up):
            self.up.wait_event(self.ev_loss[b])  # set b's last iteration is read out
            self.views[b].copy_(host_views, non_blocking=True)
            self.targets[b].copy_(host_targets, non_blocking=True)
            self.ev_in[b].record(self.up)
        main.wait_event(self.ev_in[b])
        self.graphs[b].replay()
        self.ev_done[b].record(main)
        with torch.cuda.stream(self.down):
            self.down.wait_event(self.ev_done[b])
            self.host_loss[b].copy_(self.loss[b], non_blocking=True)
            self.ev_loss[b].record(self.down)
        self.i += 1
        if self.i < 2:
            return None
        prev = (self.i - 2) & 1
        self.ev_loss[prev].synchronize()
        return float(self.host_loss[prev].item())

    def drain(self):
        if self.i == 0:
            return None
        last = (self.i - 1) & 1
        self.ev_loss[last].synchronize()
        torch.cuda.current_stream().wait_stream(self.down)
        return float(self.host_loss[last].item())


class PerViewLoop:
    """The same iteration as MappingStep over V views, but one plan per view:
    V x (project, bin, render, loss, backward), gradients accumulated, one
    Adam step -- the baseline the batched form is compared with."""

    def __init__(self, gmap: GaussianMap, views, targets_per_view, lam, lr=None, extent=1.0,
                 keep_grads=True, **rast_kw):
        self.gmap, self.lam, self.lr, self.extent = gmap, float(lam), lr, extent
        self.rasts = [fit_instance_capacity([v], gmap, **rast_kw) for v in views]
        self.targets = [r.pack([t]) for r, t in zip(self.rasts, targets_per_view)]
        self._m = gmap.gs_map()
        self._g = gmap.gs_map_grad()
        self.graph = None

    def run(self, stream=None):
        V = len(self.rasts)
        for i, (r, t) in enumerate(zip(self.rasts, self.targets)):
            r.project(self._m, stream)
            r.bin_sort(self.gmap.n, stream)
            r.render_fwd(stream=stream)
            r.loss_l1_ssim(t, self.lam, view_weight=1.0 / V, stream=stream)
            r.render_bwd(self._m, self._g, accumulate=i > 0, stream=stream)
        self.gmap.adam_step(self.lr, self.extent, stream=stream)

    def capture(self, warmup=2):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.run()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def __call__(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.run()
