"""Helpers of the GPU tests: host <-> device copies of column-major matrices."""
import numpy as np


def to_dev(a: np.ndarray):
    import torch

    return torch.from_numpy(np.asfortranarray(a)).cuda()


def to_host(t) -> np.ndarray:
    a = t.cpu().numpy()
    return np.asfortranarray(a)


def lower_band_and_v(Aout: np.ndarray, w: int):
    """(band entries 0 <= i-j <= w, reflector entries i-j > w) of the lower triangle."""
    n = Aout.shape[0]
    i, j = np.indices((n, n))
    band = (i - j >= 0) & (i - j <= w)
    refl = i - j > w
    return Aout[band], Aout[refl]
