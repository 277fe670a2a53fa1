"""Host logic of the variant sweep (no GPU): the subdomain splits of the paper's Figs. 5-8 (K
boxes along x) and Fig. 9 (K boxes in x and y, the longer side in x)."""
import pytest

from paper_1401_7227_gb300 import sweep


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 6, 10, 12, 16])
def test_x_split(K):
    assert sweep.split(K, "x", 20, 20) == (K, 1, 1)


@pytest.mark.parametrize("K,want", [(4, (2, 2, 1)), (6, (3, 2, 1)), (9, (3, 3, 1)), (10, (5, 2, 1)),
                                    (12, (4, 3, 1)), (16, (4, 4, 1)), (7, (7, 1, 1))])
def test_xy_split_is_the_most_square_factorisation(K, want):
    px, py, pz = sweep.split(K, "xy", 20, 20)
    assert (px, py, pz) == want
    assert px * py == K and px >= py


def test_methods_are_the_papers_five():
    assert sweep.METHODS == ("near", "far", "near+far", "two-level", "two-stage")
