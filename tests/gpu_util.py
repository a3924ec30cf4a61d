"""Helpers shared by the GPU tests: run the GPU path and the oracle on the same inputs."""
import numpy as np


def rel_rms(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    den = (b ** 2).sum()
    return float(np.sqrt(((a - b) ** 2).sum() / den)) if den > 0 else float(np.abs(a).max())


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def gpu_fmm(pos, S, s, p, theta, ncrit, want_phi=True, want_field=True):
    from paper_2005_12351_gb300 import fmm
    tree = fmm.create_tree(max_leaf=ncrit)
    tree.set_sources(to_dev(pos), to_dev(S), s)
    phi, E = tree.evaluate(p, theta, want_phi, want_field)
    import torch
    torch.cuda.synchronize()
    out = (phi.cpu().numpy() if phi is not None else None, E.cpu().numpy() if E is not None else None)
    return out, tree


def close(a, b, tol):
    """Parity of FP64 results: relative RMS below tol and, element by element,
    no error above 100 tol of the largest reference magnitude -- so that a few
    wrong particles cannot hide inside an aggregate over many."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    if b.size == 0:
        return a.size == 0
    worst = float(np.abs(a - b).max())
    return rel_rms(a, b) < tol and worst <= 100.0 * tol * float(np.abs(b).max())
