"""Helpers for the GPU parity tests: guarded device buffers (canary bytes on
both sides of the region a call may write) and host copies."""
from __future__ import annotations

import numpy as np

CANARY = 0xA5
GUARD = 256  # bytes on each side


class Guarded:
    """A device byte buffer with `nbytes` of payload starting `offset_bytes`
    after a guard region, followed by another guard region."""

    def __init__(self, nbytes: int, offset_bytes: int = 0, device="cuda"):
        import torch

        self.nbytes = nbytes
        self.start = GUARD + offset_bytes
        self.buf = torch.full((self.start + nbytes + GUARD,), CANARY, dtype=torch.uint8,
                              device=device)

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr() + self.start

    def payload(self, dtype) -> np.ndarray:
        import torch

        torch.cuda.synchronize()
        host = self.buf.cpu().numpy()
        return host[self.start:self.start + self.nbytes].view(dtype).copy()

    def guards_intact(self) -> bool:
        import torch

        torch.cuda.synchronize()
        host = self.buf.cpu().numpy()
        return bool(np.all(host[:self.start] == CANARY) and
                    np.all(host[self.start + self.nbytes:] == CANARY))


def stream_handle() -> int:
    import torch

    return int(torch.cuda.current_stream().cuda_stream)


_SIGNED = {np.dtype(np.uint64): np.int64, np.dtype(np.uint32): np.int32,
           np.dtype(np.uint16): np.int16}


def to_dev(arr: np.ndarray):
    """A CUDA tensor holding the bits of a numpy array (unsigned arrays are
    carried as the signed type of the same width)."""
    import torch

    a = np.ascontiguousarray(arr)
    if a.dtype in _SIGNED:
        a = a.view(_SIGNED[a.dtype])
    return torch.from_numpy(a).cuda()


def filled_u32(n: int, value: int):
    """A CUDA int32 tensor of n words, each holding the 32-bit pattern value."""
    import torch

    v = value - (1 << 32) if value >= (1 << 31) else value
    return torch.full((n,), v, dtype=torch.int32, device="cuda")


def host_u32(t) -> np.ndarray:
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32)
