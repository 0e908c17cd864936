"""Host logic of the steady-state driver (tests/table1.py converge()) on a linear model
whose answer is known: a state S that relaxes to S* through one slow mode (ratio r per
step) and carries an undamped period-2 mode, the two features of the two-phase runs.
Checks: the two-state average removes the period-2 mode; the Aitken extrapolation hits the
fixed point of the slow mode, and is refused for a slow spin-up; the stop criterion is the
relative velocity change."""
import numpy as np

from tests.table1 import converge


class LinearSim:
    """S_{t+1} = S* + r P1 (S_t - S*) - P2 (S_t - S*), with P1, P2 complementary
    projections (slow mode and period-2 mode).  The 'velocity' is the state itself."""

    def __init__(self, s_star, r, s0, p2_mask):
        self.s_star, self.r, self.S = s_star, r, s0.copy()
        self.p2 = p2_mask
        self.steps = 0

    def step(self, n):
        d = self.S - self.s_star
        slow = np.where(self.p2, 0.0, d) * self.r**n
        alt = np.where(self.p2, d, 0.0) * (-1.0) ** n
        self.S = self.s_star + slow + alt
        self.steps += n

    def get_state(self):
        return self.S.copy()

    def set_state(self, S):
        self.S = np.asarray(S, dtype=float).copy()

    def moments(self):
        return None, self.S.copy(), np.zeros_like(self.S)


def make(r=0.999):
    rng = np.random.default_rng(3)
    s_star = 1.0 + rng.random(64)
    s0 = s_star + 0.5 * rng.standard_normal(64)
    mask = np.zeros(64, bool)
    mask[::4] = True  # a quarter of the state oscillates with period 2
    return LinearSim(s_star, r, s0, mask), s_star


def test_converges_to_the_fixed_point_and_removes_the_period_two_mode():
    sim, s_star = make()
    change, steps = converge(sim, chunk=100, tol=1e-10, max_chunks=200)
    assert change < 1e-10
    assert np.abs(sim.S - s_star).max() < 1e-8 * np.abs(s_star).max()


def test_extrapolation_saves_most_of_the_chunks():
    """Per chunk the slow mode shrinks by r^100 = 0.905: without the extrapolation the
    relative change would need about 250 chunks to reach 1e-10 (ln(1e-10)/ln(0.905) + the
    start); the extrapolation gets there in a handful."""
    sim, _ = make()
    change, steps = converge(sim, chunk=100, tol=1e-10, max_chunks=400)
    assert steps < 30 * 101, steps  # measured: 21 chunks (it extrapolates once the change is < 1e-2)


def test_stops_when_the_velocity_change_is_below_tol():
    sim, _ = make(r=0.5)  # fast: converges without extrapolating
    change, steps = converge(sim, chunk=10, tol=1e-6, max_chunks=50)
    assert change < 1e-6
    assert steps <= 5 * 11


def test_no_extrapolation_of_a_slow_spin_up():
    """r = 0.985 per chunk (a factor r / (1 - r) = 66): the extrapolation is refused, as it
    is while the state still changes by more than 1e-2 per chunk."""
    sim, _ = make(r=0.99985)
    events = []
    converge(sim, chunk=100, tol=1e-12, max_chunks=60, log=lambda st, c: events.append(c))
    assert not any(isinstance(c, str) and c.startswith("extrapolate") for c in events)
    sim, _ = make()
    events = []
    converge(sim, chunk=100, tol=1e-10, max_chunks=400, log=lambda st, c: events.append(c))
    extrap = [i for i, c in enumerate(events) if isinstance(c, str)]
    assert extrap and all(events[i - 1] < 1e-2 for i in extrap)
