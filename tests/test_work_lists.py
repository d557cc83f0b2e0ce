"""The batched launches' work-list planner (host logic, no GPU): teams of
CTAs of one size, the solves dealt largest first to the least-loaded team
(LPT, Graham 1969)."""
import numpy as np
import pytest

from paper_2106_07616_gb300 import _build, rbffd

MAXB = 160  # CTAs a system's partial sums allow at most


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def mix(m=256, seed=3):
    rng = np.random.default_rng(seed)
    rows = np.exp(rng.uniform(np.log(1000), np.log(64000), m)).astype(np.int32)
    iters = rng.integers(20, 400, m)
    return rows * iters.astype(np.float64), np.full(m, MAXB, np.int32), rows


def test_every_solve_once_and_loads_balanced():
    work, cap, rows = mix()
    cmax = 304
    team, nctas, size, nteams = rbffd.plan_work_lists(work, cap, rows, cmax)
    assert nctas == nteams * size and 1 <= nctas <= cmax
    assert 1 <= size <= min(cap.min(), MAXB)
    assert team.min() >= 0 and team.max() < nteams
    load = np.bincount(team, weights=work, minlength=nteams)
    assert np.isclose(load.sum(), work.sum())
    # LPT: the teams' loads differ by at most the largest solve, and the
    # longest is within 4/3 of the lower bound max(mean load, largest solve)
    assert load.max() - load.min() <= work.max() * (1 + 1e-12)
    assert load.max() <= 4.0 / 3.0 * max(work.sum() / nteams, work.max()) * (1 + 1e-12)
    # the largest solve's team holds about its share of the grid
    assert size >= int(np.floor(cmax * work.max() / work.sum()))
    # the same plan every time
    again = rbffd.plan_work_lists(work, cap, rows, cmax)
    assert np.array_equal(again[0], team) and again[1:] == (nctas, size, nteams)


def test_one_large_solve_takes_the_grid_up_to_its_cap():
    team, nctas, size, nteams = rbffd.plan_work_lists([1e9], [MAXB], [500000], 152)
    assert nteams == 1 and size == 152 and nctas == 152 and team[0] == 0
    team, nctas, size, nteams = rbffd.plan_work_lists([1e9], [64], [500000], 152)
    assert nteams == 1 and size == 64


def test_autotuner_scale_and_caps():
    work, cap, rows = mix(64, seed=9)
    base = rbffd.plan_work_lists(work, cap, rows, 304)
    big = rbffd.plan_work_lists(work, cap, rows, 304, scale=4.0)
    small = rbffd.plan_work_lists(work, cap, rows, 304, scale=0.5)
    assert big[2] >= base[2] >= small[2]
    for plan in (base, big, small):
        team, nctas, size, nteams = plan
        assert nctas <= 304 and size <= MAXB and team.max() < nteams
    # a solve whose partial sums allow few CTAs caps every team
    cap2 = cap.copy()
    cap2[5] = 3
    assert rbffd.plan_work_lists(work, cap2, rows, 304)[2] <= 3


def test_bad_plans_rejected():
    for args in (([], [], [], 10), ([1.0], [4], [100], 0), ([-1.0], [4], [100], 10),
                 ([1.0], [0], [100], 10)):
        with pytest.raises(rbffd.RbffdError) as e:
            rbffd.plan_work_lists(*args)
        assert e.value.code == rbffd.EINVAL
