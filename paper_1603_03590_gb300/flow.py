"""Convenience wrapper over the C ABI: a handle owner taking torch CUDA tensors.

Marshalling only (allocation of outputs with torch, pointers and the current stream passed to
libdis.so); every step of the method runs in the library's kernels.
"""
import torch

from . import dis


class DenseInverseSearch:
    """DIS optical flow on the current CUDA device.

    >>> d = DenseInverseSearch(1024, 436, preset="dense")
    >>> flow = d(I0, I1)          # I0, I1: (H, W) or (C, H, W) float32 CUDA tensors in [0, 1]
    """

    def __init__(self, max_w, max_h, max_batch=1, channels=1, preset="default", **overrides):
        self.params = dis.dis_default_params(preset, channels=channels, **overrides)
        self.channels = channels
        self.handle = dis.dis_create(max_w, max_h, max_batch, channels)

    def close(self):
        if self.handle:
            dis.dis_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _check_img(t, channels):
        if not (t.is_cuda and t.dtype == torch.float32):
            raise TypeError("images must be float32 CUDA tensors")
        if t.dim() != (2 if channels == 1 else 3) or t.stride(-1) != 1:
            raise ValueError("images must be (H, W) or (C, H, W) with unit column stride")
        if channels > 1 and t.stride(0) != t.stride(-2) * t.shape[-2]:
            raise ValueError("colour planes must be pitch * H elements apart")

    def __call__(self, I0, I1, flow_out=None, stream=None):
        self._check_img(I0, self.channels)
        if I1.shape != I0.shape or I1.stride() != I0.stride():
            raise ValueError("I0 and I1 must have the same shape and strides")
        H, W = I0.shape[-2:]
        if flow_out is None:
            flow_out = torch.empty((H, W, 2), device=I0.device, dtype=torch.float32)
        dis.dis_compute_flow(self.handle, I0, I1, W, H, I0.stride(-2), self.params, flow_out, stream)
        return flow_out

    def batched(self, pairs, flows=None, stream=None):
        """pairs: list of (I0, I1) tensors of any sizes; returns the list of flows."""
        if flows is None:
            flows = [torch.empty((a.shape[-2], a.shape[-1], 2), device=a.device, dtype=torch.float32) for a, _ in pairs]
        items = []
        for (a, b), f in zip(pairs, flows):
            self._check_img(a, self.channels)
            self._check_img(b, self.channels)
            items.append((a, b, a.shape[-1], a.shape[-2], a.stride(-2), f))
        arr = dis.make_pairs(items)
        self._keep = (pairs, flows, arr)
        dis.dis_compute_flow_batched(self.handle, arr, len(items), self.params, stream)
        return flows
