"""Canary words around caller-owned device buffers (a stand-in for a memory
checker, which is not available on this machine): a buffer is allocated with
GUARD extra elements on each side filled with a fixed pattern; after the call
the pattern must be intact, so a kernel that writes past either end of an
output fails the test."""
import torch

GUARD = 64
PATTERN = {torch.int64: -0x3A5A5A5A5A5A5A5B, torch.int32: -0x3A5A5A5B, torch.int16: -0x3A5B, torch.uint8: 0xA5}


def guarded(n, dtype, device="cuda"):
    """(view of n elements, the whole guarded buffer)."""
    full = torch.full((n + 2 * GUARD,), PATTERN[dtype], dtype=dtype, device=device)
    return full[GUARD:GUARD + n], full


def intact(full, n):
    """True if both guard regions still hold the pattern."""
    torch.cuda.synchronize()
    p = PATTERN[full.dtype]
    return bool((full[:GUARD] == p).all()) and bool((full[GUARD + n:] == p).all())
