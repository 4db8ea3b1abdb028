"""torch.autograd wrappers of the differentiable form (marshalling only; the forward and the
backward run in libdis.so's kernels).

DifferentiableDIS(I0, I1, init_flow) returns the flow of the frozen-search DIS map: the
forward records every patch's search increment (FP32 search) and evaluates the map with those
increments frozen in FP64; the backward repeats that replay and runs the FP64 adjoint of the
pyramid, initial displacements, densification and unrolled SOR sweeps.
BatchedDifferentiableDIS runs several pairs of that map side by side on streams of their own.
photometric_loss is the mean Charbonnier penalty sqrt((I1(x + U(x)) - I0(x))^2 + eps^2) with its gradients.
"""
import torch

from . import dis


def _level_dims(w, h, s):
    for _ in range(s):
        w, h = (w + 1) // 2, (h + 1) // 2
    return w, h


class DifferentiableDIS:
    """Grayscale DIS with gradients w.r.t. I0, I1 (H, W float32 CUDA, [0, 1]) and the initial
    flow (level theta_ss resolution, (h_ss, w_ss, 2)).  With finest_scale > 0 the final bilinear
    up-scaling is part of the map.

    The patch searches are replayed from their recorded increments (recorded by the FP32 search
    of each call, or given as `frozen`, dis_levels' total_patches x 2).  search_grad=0 (default)
    treats the increments as constants; search_grad=1 differentiates the converged search by the
    implicit-function theorem (pass increments of converged searches).

    An instance keeps the buffers of its library calls (frames, increments, workspace, results)
    and issues its work on the stream current at each call: use one instance per stream."""

    def __init__(self, max_w, max_h, preset="default", **overrides):
        self.params = dis.dis_default_params(preset, channels=1, **overrides)
        self.handle = dis.dis_create(max_w, max_h, 1, 1)
        self._stage = None
        self._token = None

    def close(self):
        if self.handle:
            if self._stage is not None:
                torch.cuda.synchronize(self._stage["ws"].device)  # graphs may still read the staging
                self._stage = None
            dis.dis_destroy(self.handle)
            self.handle = None

    def _staging(self, I0, n, init):
        """Buffers the library calls read and write.  Their addresses stay the same from call to
        call, so the library replays each call's chain of launches as one CUDA graph (it keys
        its graphs on the call's pointers); inputs are copied in and results copied out."""
        H, W = I0.shape
        key = (I0.device, H, W, n, None if init is None else tuple(init.shape))
        st = self._stage
        if st is None or st["key"] != key:
            dev = I0.device
            nbytes = dis.dis_backward_workspace_bytes(W, H, self.params)
            st = dict(key=key, ws=torch.empty(nbytes, device=dev, dtype=torch.uint8), nbytes=nbytes,
                      I0=torch.empty((H, W), device=dev), I1=torch.empty((H, W), device=dev),
                      rec=torch.empty((n, 2), device=dev), flow=torch.empty((H, W, 2), device=dev),
                      gflow=torch.empty((H, W, 2), device=dev), gI0=torch.empty((H, W), device=dev),
                      gI1=torch.empty((H, W), device=dev),
                      init=None if init is None else torch.empty_like(init),
                      gInit=None if init is None else torch.empty_like(init))
            self._stage, self._token = st, None
        return st

    def _stage_inputs(self, st, token, I0, I1, init, rec):
        if self._token is not token:  # the staging holds another call's inputs
            st["I0"].copy_(I0)
            st["I1"].copy_(I1)
            if init is not None:
                st["init"].copy_(init)
            st["rec"].copy_(rec)
            self._token = token

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coarsest_shape(self, w, h):
        ss, _, _ = dis.dis_levels(w, h, self.params)
        ws, hs = _level_dims(w, h, ss)
        return hs, ws

    def __call__(self, I0, I1, init_flow=None, frozen=None):
        return _DISFlow.apply(I0, I1, init_flow, self, frozen)


class BatchedDifferentiableDIS:
    """The differentiable map on a batch of pairs that run side by side: one handle and one CUDA
    stream per pair slot.  Each pair's forward (FP32 search, FP64 replay) is issued on its slot's
    stream, and autograd runs its backward on that stream too, so the pairs' chains of small
    launches overlap on the GPU.  The flows are those of DifferentiableDIS on each pair alone, bit
    for bit.  Calls order themselves after the caller's current stream, and the caller's stream
    waits for every pair's flow."""

    def __init__(self, max_w, max_h, slots, preset="default", **overrides):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.pairs = [DifferentiableDIS(max_w, max_h, preset, **overrides) for _ in range(slots)]
        self.params = self.pairs[0].params
        self.streams = [torch.cuda.Stream() for _ in range(slots)]

    def close(self):
        for d in self.pairs:
            d.close()

    def coarsest_shape(self, w, h):
        return self.pairs[0].coarsest_shape(w, h)

    def __call__(self, I0s, I1s, init_flows=None):
        n = len(I0s)
        if n > len(self.pairs) or len(I1s) != n or (init_flows is not None and len(init_flows) != n):
            raise ValueError("at most %d pairs, with as many second frames and initial flows" % len(self.pairs))
        caller = torch.cuda.current_stream()
        flows = []
        for k in range(n):
            s = self.streams[k]
            s.wait_stream(caller)
            for t in (I0s[k], I1s[k], None if init_flows is None else init_flows[k]):
                if t is not None:
                    t.record_stream(s)  # the caller's tensors stay allocated until s is done
            with torch.cuda.stream(s):
                init = None if init_flows is None else init_flows[k]
                flows.append(self.pairs[k](I0s[k], I1s[k], init))
        for k in range(n):
            caller.wait_stream(self.streams[k])
            flows[k].record_stream(caller)
        return flows


class _DISFlow(torch.autograd.Function):
    @staticmethod
    def forward(ctx, I0, I1, init_flow, owner, frozen=None):
        I0c, I1c = I0.detach().contiguous(), I1.detach().contiguous()
        H, W = I0c.shape
        p = owner.params
        n = dis.dis_levels(W, H, p)[2]
        init = None if init_flow is None else init_flow.detach().contiguous()
        if frozen is None:
            # the FP32 search records every patch's increment ...
            rec = torch.empty((n, 2), device=I0c.device, dtype=torch.float32)
            tmp = torch.empty((H, W, 2), device=I0c.device, dtype=torch.float32)
            dis.dis_compute_flow_ex(owner.handle, I0c, I1c, W, H, W, p, init, None, rec, None, tmp)
        else:
            rec = frozen.detach().to(device=I0c.device, dtype=torch.float32).contiguous()
            if tuple(rec.shape) != (n, 2):
                raise ValueError("frozen increments must be (%d, 2)" % n)
        # ... and the map with those increments frozen is evaluated in FP64
        st = owner._staging(I0c, n, init)
        token = object()
        owner._stage_inputs(st, token, I0c, I1c, init, rec)
        dis.dis_replay_flow(owner.handle, st["I0"], st["I1"], W, H, W, p, st["init"], st["rec"], st["flow"], st["ws"],
                            st["nbytes"])
        flow = st["flow"].clone()
        ctx.owner, ctx.token = owner, token
        ctx.has_init = init is not None
        ctx.save_for_backward(I0c, I1c, init if init is not None else torch.empty(0, device=I0c.device), rec)
        return flow

    @staticmethod
    def backward(ctx, grad_flow):
        I0, I1, init, rec = ctx.saved_tensors
        owner, p = ctx.owner, ctx.owner.params
        H, W = I0.shape
        it = init if ctx.has_init else None
        st = owner._staging(I0, rec.shape[0], it)
        owner._stage_inputs(st, ctx.token, I0, I1, it, rec)
        st["gflow"].copy_(grad_flow)
        dis.dis_backward(owner.handle, st["I0"], st["I1"], W, H, W, p, st["init"], st["rec"], st["gflow"], st["gI0"],
                         st["gI1"], W, st["gInit"], st["ws"], st["nbytes"])
        gInit = st["gInit"].clone() if ctx.has_init else None
        return st["gI0"].clone(), st["gI1"].clone(), gInit, None, None


class _PhotometricLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, I0, I1, flow, eps):
        I0c, I1c, fc = I0.detach().contiguous(), I1.detach().contiguous(), flow.detach().contiguous()
        C = 1 if I0c.dim() == 2 else I0c.shape[0]
        H, W = I0c.shape[-2:]
        loss = torch.empty(1, device=I0c.device, dtype=torch.float64)
        gf, g0, g1 = torch.empty_like(fc), torch.empty_like(I0c), torch.empty_like(I1c)
        nb = dis.dis_photometric_loss_scratch_bytes(W, H, W, C)
        scratch = torch.empty(nb, device=I0c.device, dtype=torch.uint8)
        dis.dis_photometric_loss(I0c, I1c, W, H, W, C, fc, float(eps), loss, gf, g0, g1, scratch, nb)
        ctx.save_for_backward(g0, g1, gf)
        return loss[0].to(torch.float32)

    @staticmethod
    def backward(ctx, g):
        g0, g1, gf = ctx.saved_tensors
        return g * g0, g * g1, g * gf, None


def photometric_loss(I0, I1, flow, eps=1e-3):
    """Mean Charbonnier photometric error of flow (H, W, 2) between I0 and I1."""
    return _PhotometricLoss.apply(I0, I1, flow, eps)
