"""Shared helpers of the GPU parity tests: the same complex64-rounded
measurement goes to the oracle (as complex128) and to the CUDA path."""
import numpy as np

from oracle import model


def measurement64(scene):
    """Oracle measurement rounded to complex64, and that value as complex128."""
    Y32 = model.measurement(scene).astype(np.complex64)
    return Y32, Y32.astype(np.complex128)


def to_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def rel_err(gpu, ref):
    """max |gpu - ref| / max |ref| (the frame-normalised error)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.abs(gpu - ref).max() / np.abs(ref).max())


def top2_margin(scores):
    s = np.sort(np.asarray(scores, dtype=np.float64).reshape(-1))
    return float((s[-1] - s[-2]) / s[-1])
