"""Shared helpers for the GPU parity tests (conversions between the oracle's
float64 arrays and the library's u_s storage formats)."""
import numpy as np

FP64, FP32, BF16 = 0, 1, 2
PRECS = [FP64, FP32, BF16]
PNAME = {FP64: "fp64", FP32: "fp32", BF16: "bf16"}


def bf16_bits(a):
    """float64 array of BF16-representable values -> uint16 bit patterns."""
    a = np.asarray(a, np.float64).astype(np.float32)
    return (a.view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def bf16_from_bits(b):
    return (np.asarray(b, np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def us_to_device(a, prec):
    """float64 host values (already representable in u_s) -> device tensor in u_s."""
    import torch
    if prec == FP64:
        return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()
    if prec == FP32:
        return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    return torch.from_numpy(bf16_bits(a).view(np.int16)).cuda()


def us_empty(m, prec):
    import torch
    dt = {FP64: torch.float64, FP32: torch.float32, BF16: torch.int16}[prec]
    return torch.zeros(m, dtype=dt, device="cuda")


def us_to_host(t, prec):
    a = t.cpu().numpy()
    if prec == BF16:
        return bf16_from_bits(a.view(np.uint16))
    return a.astype(np.float64)


def dev64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()
