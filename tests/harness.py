"""Test helpers: run the CUDA path and the oracle on the same seeded inputs.

Both sides number nodes their own way; vectors are moved between them by
matching integer node coordinates (workloads.match_nodes).
"""
import numpy as np

from paper_1912_12453_gb300 import workloads as W


class Pair:
    def __init__(self, leaves, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
        import torch
        from oracle import oracle as O
        from paper_1912_12453_gb300 import chns
        self.torch = torch
        self.chns = chns
        self.leaves = leaves
        self.gm = chns.Mesh(leaves, lo, hi)
        self.om = O.OracleMesh(leaves, lo, hi)
        self.nf = self.om.nf
        # gpu node i  <->  oracle node perm[i]
        self.g_of_o = W.match_nodes(self.gm.coords_int, self.om.coords_int)

    def to_gpu(self, x_or, dtype=None):
        """oracle-ordered (n_nodes, nf) or flat -> flat CUDA tensor in GPU order"""
        torch = self.torch
        x = np.asarray(x_or).reshape(self.om.n_nodes, -1)
        y = np.empty_like(x)
        y[self.g_of_o] = x
        t = torch.from_numpy(np.ascontiguousarray(y.reshape(-1))).to("cuda")
        return t if dtype is None else t.to(dtype)

    def to_oracle(self, t):
        y = t.detach().double().cpu().numpy().reshape(self.gm.n_nodes, -1)
        return y[self.g_of_o].reshape(-1)


def rel(a, b):
    d = np.linalg.norm(np.asarray(a) - np.asarray(b))
    n = np.linalg.norm(np.asarray(b))
    return d / n if n > 0 else d


def random_state(n_nodes, nf, seed, lo=-1.2, hi=1.2):
    return np.random.default_rng(seed).uniform(lo, hi, (n_nodes, nf))


def physical_state(om, wl, eps=1e-2, seed=W.PERTURB_SEED):
    """Workload initial state (mu projected by the oracle is NOT used: mu from
    a smooth field) plus a small seeded perturbation, oracle order."""
    U0 = W.initial_state(om.coords, wl)
    U0[:, om.dim + 2] = (U0[:, om.dim + 1] ** 3 - U0[:, om.dim + 1]) * 0.5
    w = W.perturbation(om.n_nodes, om.nf, 1, seed)[0]
    return U0, U0 + eps * w
