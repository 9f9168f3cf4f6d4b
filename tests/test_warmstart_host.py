"""Host logic of the learned warm start (no GPU): the collapse filter and the
grouping of samples into same-shape mini-batches."""
import numpy as np

from paper_2503_06610_gb300 import inputs as I
from paper_2503_06610_gb300 import warmstart as W


def test_collapsed_counts_reversed_sites_per_layer():
    nx, ny, nz = 16, 16, 4
    tube = I.skyrmion_tubes(nx, ny, nz, [(8.0, 8.0)], 5.0)     # a disc of reversed sites in every layer
    per_layer = (tube[2] < 0).sum() / nz
    assert per_layer >= 5 and not W.collapsed(tube, nz)
    lone = I.uniform_director(nx, ny, nz)
    lone[:, [8 + nx * (8 + ny * z) for z in range(nz)]] = [[0.0], [0.0], [-1.0]]  # one reversed column
    assert W.collapsed(lone, nz)
    assert W.collapsed(I.uniform_director(nx, ny, nz), nz)
    assert not W.collapsed(lone, nz, min_columns=1)


def test_group_by_shape_and_scalars():
    samples = I.warmstart_samples(6, seed=0, nx=32, ny=32, lz_choices=(16, 24))
    groups = W.group_by_shape(range(6), samples)
    assert sorted(i for g in groups.values() for i in g) == list(range(6))
    for (nx, ny, nz), idx in groups.items():
        assert all((samples[i][0]["nx"], samples[i][0]["ny"], samples[i][0]["nz"]) == (nx, ny, nz) for i in idx)
    p = samples[0][0]
    assert W.scalars_of(p) == [p["q0"], float(p["nz"]), p["W0"]]
