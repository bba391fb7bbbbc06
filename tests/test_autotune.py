"""Host logic of the cycle-settings autotuner (no GPU): the search space and
the choice of the fastest converged candidate."""

import pytest

from paper_1611_06288_gb300.autotune import DEFAULT_SPACE, candidates, select, tile_candidates


def test_candidates_cover_the_space():
    c = candidates()
    n = (len(DEFAULT_SPACE["nu"]) * len(DEFAULT_SPACE["inner_cycles"])
         * len(DEFAULT_SPACE["jacobi_factor"]) * len(DEFAULT_SPACE["coarse_sweeps"]))
    assert len(c) == n and len({tuple(sorted(x.items())) for x in c}) == n
    assert {(x["nu1"], x["nu2"]) for x in c} == set(DEFAULT_SPACE["nu"])
    assert all("defect_planes" not in x for x in c)


def test_tile_stage_keeps_the_cycle_settings():
    best = {"nu1": 0, "nu2": 1, "inner_cycles": 2, "jacobi_factor": 4, "coarse_sweeps": 2}
    t = tile_candidates(best)
    assert [x["defect_planes"] for x in t] == DEFAULT_SPACE["defect_planes"]
    assert all({k: v for k, v in x.items() if k != "defect_planes"} == best for x in t)
    assert 0 in DEFAULT_SPACE["defect_planes"]        # the heuristic stays a candidate
    assert tile_candidates(best, {"nu": [(0, 1)]}) == []


def test_select_fastest_converged():
    a, b, c = {"nu1": 0}, {"nu1": 1}, {"nu1": 2}
    assert select([(a, 2.0), (b, None), (c, 1.5)]) is c
    assert select([(a, None), (b, 3.0)]) is b
    with pytest.raises(RuntimeError):
        select([(a, None)])
