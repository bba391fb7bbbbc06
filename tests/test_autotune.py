"""Host logic of the cycle-settings autotuner (no GPU): the search space and
the choice of the fastest converged candidate."""

import pytest

from paper_1611_06288_gb300.autotune import DEFAULT_SPACE, candidates, select


def test_candidates_cover_the_space():
    c = candidates()
    n = (len(DEFAULT_SPACE["nu"]) * len(DEFAULT_SPACE["inner_cycles"])
         * len(DEFAULT_SPACE["jacobi_factor"]) * len(DEFAULT_SPACE["coarse_sweeps"]))
    assert len(c) == n and len({tuple(sorted(x.items())) for x in c}) == n
    assert {(x["nu1"], x["nu2"]) for x in c} == set(DEFAULT_SPACE["nu"])


def test_select_fastest_converged():
    a, b, c = {"nu1": 0}, {"nu1": 1}, {"nu1": 2}
    assert select([(a, 2.0), (b, None), (c, 1.5)]) is c
    assert select([(a, None), (b, 3.0)]) is b
    with pytest.raises(RuntimeError):
        select([(a, None)])
