"""Shared helpers of the GPU parity tests: a GPU solver beside the oracle hierarchy of the same
problem, with the map from the library's compact colour-major layout to the oracle's natural
ordering on every level."""
import numpy as np
import torch

from oracle import multigrid as MG


def _dof_map(solver, lev, level):
    coords = solver.layout(level)
    g = lev.geom
    lin = coords[:, 0].astype(np.int64) + g.n * coords[:, 1].astype(np.int64)
    if g.dim == 3:
        lin += g.n * g.n * coords[:, 2].astype(np.int64)
    perm = g.bg2act[lin]
    assert (perm >= 0).all() and len(perm) == g.n_active
    return (perm[:, None] * lev.nb + np.arange(lev.nb)[None, :]).reshape(-1)


class Pair:
    """A GPU solver and the oracle hierarchy of the same problem, with dof maps per level."""

    def __init__(self, prob, precision="f64", tail_max_cells=0, cell_kernel_min_cells=0, **solver_kwargs):
        import paper_2506_12899_gb300 as S
        self.prob = prob
        self.gpu = S.Solver(prob, precision, tail_max_cells=tail_max_cells,
                            cell_kernel_min_cells=cell_kernel_min_cells, **solver_kwargs)
        self.H = MG.Hierarchy(prob)
        assert self.gpu.num_levels == len(self.H.levels)
        self.maps = [_dof_map(self.gpu, lev, l) for l, lev in enumerate(self.H.levels)]

    def to_gpu(self, x_oracle, level, dtype=torch.float64):
        return torch.tensor(x_oracle[self.maps[level]], dtype=dtype, device="cuda")

    def to_oracle(self, t, level):
        out = np.zeros(len(self.maps[level]))
        out[self.maps[level]] = t.double().cpu().numpy()
        return out
