"""Layout helpers shared by the GPU tests (library layout = column-major)."""
import numpy as np


def t_lib(x, device="cuda", dtype=None):
    """numpy (n1, n2, n3) or (n, n) array -> torch buffer in library (column-major) layout."""
    import torch
    a = np.ascontiguousarray(np.asarray(x).transpose(*reversed(range(np.asarray(x).ndim))))
    t = torch.from_numpy(a)
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device)


def np_lib(t):
    """library-layout torch buffer -> numpy array with reversed axes (float64)."""
    a = t.detach().cpu().double().numpy()
    return a.transpose(*reversed(range(a.ndim)))


def proj_diff(U1, U2):
    return float(np.linalg.norm(U1 @ U1.T - U2 @ U2.T))
