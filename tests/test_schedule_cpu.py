"""The adaptive check schedule (spk_next_check, host only: no GPU needed).

Expected values are worked out by hand from the rule: doubling until the
last three estimates decrease; then d + ceil(0.7 * 1.05 * need) rounded up
to a multiple of p (at least d + p), with need the iterations the line
through the last two (d, log rho) points takes to reach log tol; then
min(., dmax), and at least d + 1."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def spk():
    from paper_2311_16019_gb300 import build, spk as S
    build.build()
    S.load()
    return S


def test_doubling_warm_up(spk):
    assert spk.next_check([20], [1e-3], 1e-8, 20, 1500) == 40
    assert spk.next_check([20, 40], [1e-3, 5e-4], 1e-8, 20, 1500) == 80
    # not strictly decreasing over the last three checks: keep doubling
    assert spk.next_check([20, 40, 80], [1e-3, 1e-3, 5e-4], 1e-8, 20, 1500) == 160
    assert spk.next_check([20, 40, 80], [1e-3, 2e-3, 5e-4], 1e-8, 20, 1500) == 160


def test_extrapolated_step_geometric_decay(spk):
    # rho = 10^(-3 - 0.01 d): from d = 80 (rho = 10^-3.8) the line reaches
    # 1e-8 after 420 iterations; 0.7 * 1.05 * 420 = 308.7 -> 309;
    # 80 + 309 = 389, rounded up to a multiple of 20: 400.
    d = np.array([20, 40, 80])
    rho = 10.0 ** (-3 - 0.01 * d)
    assert spk.next_check(d, rho, 1e-8, 20, 1500) == 400
    # same history, p = 1: 389 exactly
    assert spk.next_check(d, rho, 1e-8, 1, 1500) == 389
    # the slope comes from the last two checks only: a different first
    # value (still decreasing) does not change the step
    rho2 = rho.copy()
    rho2[0] = 0.5
    assert spk.next_check(d, rho2, 1e-8, 20, 1500) == 400


def test_step_is_at_least_p_and_clamped(spk):
    # rho just above tol with a steep slope: need < 1 iteration -> d + p
    d = [20, 40, 80]
    rho = [1e-2, 1e-5, 1.0001e-8]
    assert spk.next_check(d, rho, 1e-8, 20, 1500) == 100
    # dmax caps the prediction, and the next check is always after d
    g = 10.0 ** (-3 - 0.01 * np.array(d))
    assert spk.next_check(d, g, 1e-8, 20, 300) == 300
    assert spk.next_check(d, g, 1e-8, 20, 80) == 81
    assert spk.next_check([20], [1e-3], 1e-8, 20, 30) == 30


def test_invalid_arguments(spk):
    with pytest.raises(spk.SpkError):
        spk.next_check([], [], 1e-8, 20, 100)
    with pytest.raises(spk.SpkError):
        spk.next_check([20], [1e-3], 0.0, 20, 100)
    with pytest.raises(spk.SpkError):
        spk.next_check([20], [1e-3], 1e-8, 0, 100)
