"""Host checks of the seeded input generators (no arithmetic of the method)."""
from tp_synth import batch_problems, sample_cells, uniform_vector


def test_batch_generator_terminates_within_budget():
    p = batch_problems(count=32)
    assert len(p) == 32
    assert sum(q["dofs"] for q in p) <= 3e8
    assert len({q["k"] for q in p}) >= 3 and len({q["cells"] for q in p}) >= 3
    assert batch_problems(count=32) == p  # seeded


def test_small_batch_generator_and_samples():
    p = batch_problems(count=6, seed_base=2000, cells_choices=(4, 6, 8))
    assert all(q["cells"] in (4, 6, 8) for q in p)
    cells = sample_cells(1000, 50, seed=1, nx=10, ny=10, nz=10)
    assert len(set(cells.tolist())) == len(cells) and {0, 9, 990, 999} <= set(cells.tolist())
    x = uniform_vector(100, seed=3)
    assert x.min() >= -1 and x.max() <= 1
