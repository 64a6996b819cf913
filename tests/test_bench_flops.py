"""CPU checks of the roofline accounting in bench.py: the cone (changed
sites) of a connected configuration at each layer equals a brute-force
dilation of the two swapped sites on the periodic lattice, and the FLOP
totals follow from it."""

import numpy as np
import pytest
import torch

import bench
import nqs_synth


def _brute_cone(L, i, j, l):
    """Sites within Chebyshev distance l (periodic) of site i or site j."""
    yi, xi = divmod(i, L)
    yj, xj = divmod(j, L)
    y, x = np.divmod(np.arange(L * L), L)

    def near(y0, x0):
        dy = np.minimum(np.abs(y - y0), L - np.abs(y - y0))
        dx = np.minimum(np.abs(x - x0), L - np.abs(x - x0))
        return np.maximum(dy, dx) <= l

    return int((near(yi, xi) | near(yj, xj)).sum())


@pytest.mark.parametrize('L', [4, 5, 6, 7, 10, 12, 16])
def test_cone_sizes_match_brute_force(L):
    i = (L // 2) * L + L // 2
    nn = ((L // 2) * L + (L // 2 + 1) % L)                      # x + 1
    nny = (((L // 2) + 1) % L) * L + L // 2                      # y + 1
    nnn = (((L // 2) + 1) % L) * L + (L // 2 + 1) % L            # x + 1, y + 1
    for l in range(1, L + 1):
        assert bench.cone_sites(L, l, False) == _brute_cone(L, i, nn, l)
        assert bench.cone_sites(L, l, False) == _brute_cone(L, i, nny, l)
        assert bench.cone_sites(L, l, True) == _brute_cone(L, i, nnn, l)


def test_flop_totals():
    w = nqs_synth.WORKLOADS['j1j2_10x10']
    dense = bench.dense_forward_flops(w)
    assert dense == sum(2 * 9 * (1 if l == 0 else 16) * 16 * 100 for l in range(6))
    pairs = torch.zeros((2, 400, 2), dtype=torch.int32)
    pairs[0, 0] = torch.tensor([0, 1])       # NN along x
    pairs[0, 1] = torch.tensor([0, 11])      # NNN
    pairs[1, 0] = torch.tensor([9, 0])       # NN across the periodic edge
    n_conn = torch.tensor([2, 1], dtype=torch.int32)
    cone, dense_total = bench.eloc_algorithmic_flops(w, 2, pairs, n_conn)
    assert dense_total == 5 * dense
    assert cone == 2 * dense + 2 * bench.cone_forward_flops(w, False) + bench.cone_forward_flops(w, True)
    assert bench.cone_forward_flops(w, False) < dense
