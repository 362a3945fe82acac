"""Seeded synthetic inputs shared by the tests, the bench and the smoke run.

This module holds no arithmetic of the method: it only draws the random
vectors and random problem descriptions that both the CUDA path and the CPU
oracle receive as inputs.
"""
import numpy as np


def uniform_vector(ndofs, seed=0):
    """x ~ U[-1, 1] in FP64, canonical cell-major order (one draw per DoF)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, ndofs)


def normal_vector(ndofs, seed=0):
    """x ~ N(0, 1) in FP64 (the distribution of the precision-loss experiment)."""
    return np.random.default_rng(seed).standard_normal(ndofs)


def sample_cells(ncells, count, seed=0, nx=None, ny=None, nz=None):
    """Random distinct cell indices plus the eight corner cells of the box."""
    rng = np.random.default_rng(seed)
    cells = set(rng.choice(ncells, size=min(count, ncells), replace=False).tolist())
    if nx is not None:
        for cz in (0, nz - 1):
            for cy in (0, ny - 1):
                for cx in (0, nx - 1):
                    cells.add((cz * ny + cy) * nx + cx)
    return np.array(sorted(cells), dtype=np.int64)


def batch_problems(count=32, seed_base=1000, max_total_dofs=3e8,
                   cells_choices=(16, 32, 48, 64, 80, 96), degrees=(1, 2, 3, 4, 5, 6, 7)):
    """Random uneven batch of Poisson problems: list of dicts with cells, k, dofs and four random
    modes (a, p, q, r), a ~ U[-1, 1], p, q, r in {1, 2, 3}. Problem i draws from default_rng(seed_base + i)
    a (cells, k) pair uniformly among the pairs whose size fits its fair share of the remaining budget
    (what is left of max_total_dofs divided by the problems still to draw); if none fits, the smallest
    pair is taken. Always terminates; the total stays within the budget unless even the smallest pairs
    exceed the shares."""
    combos = sorted(((c, k) for c in cells_choices for k in degrees), key=lambda ck: ck[0] ** 3 * (ck[1] + 1) ** 3)
    size = lambda ck: ck[0] ** 3 * (ck[1] + 1) ** 3
    probs = []
    total = 0
    for i in range(count):
        rng = np.random.default_rng(seed_base + i)
        share = (max_total_dofs - total) / (count - i)
        fitting = [ck for ck in combos if size(ck) <= share] or combos[:1]
        c, k = fitting[int(rng.integers(len(fitting)))]
        modes = [(float(rng.uniform(-1, 1)), int(rng.integers(1, 4)), int(rng.integers(1, 4)),
                  int(rng.integers(1, 4))) for _ in range(4)]
        total += size((c, k))
        probs.append({"cells": c, "k": k, "modes": modes, "dofs": size((c, k))})
    return probs
