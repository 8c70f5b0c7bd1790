"""Helpers for the GPU parity tests: move seeded inputs to the device, run
the library through its binding, bring results back."""
import numpy as np
import torch

import synth

DEV = torch.device("cuda:0")


def dev(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def modp_inputs(m, k, n, p, tag=0):
    A = synth.modp_matrix(synth.SEED_A, m, k, p, tag)
    B = synth.modp_matrix(synth.SEED_B, k, n, p, tag)
    C = synth.modp_matrix(synth.SEED_C, m, n, p, tag)
    return A, B, C


def fp_inputs(m, k, n, tag=0):
    A = synth.normal_matrix(synth.SEED_A, m, k, tag)
    B = synth.normal_matrix(synth.SEED_B, k, n, tag)
    C = synth.normal_matrix(synth.SEED_C, m, n, tag)
    return A, B, C


def padded(x: np.ndarray, ld: int) -> torch.Tensor:
    """Device copy of x inside a wider buffer (leading dimension ld)."""
    buf = torch.zeros((x.shape[0], ld), dtype=torch.from_numpy(x[:0]).dtype, device=DEV)
    buf[:, : x.shape[1]] = torch.from_numpy(np.ascontiguousarray(x)).to(DEV)
    return buf[:, : x.shape[1]]
