"""Helpers for the GPU parity tests (placing seeded bytes on the device)."""
import numpy as np
import torch


def to_device(data: np.ndarray, offset: int = 0) -> torch.Tensor:
    """uint8 CUDA tensor holding `data`, starting `offset` bytes past a 256-byte boundary."""
    buf = torch.empty(data.size + offset + 16, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + data.size]
    if data.size:
        view.copy_(torch.from_numpy(np.ascontiguousarray(data)))
    return view


def bitmap_to_cuts(words: torch.Tensor, n: int) -> np.ndarray:
    """Set bits p of a bitmap -> cut positions p + 1."""
    w = words.cpu().numpy().view(np.uint32)
    bits = np.unpackbits(w.view(np.uint8), bitorder="little")[:n]
    return (np.flatnonzero(bits) + 1).astype(np.uint64)
