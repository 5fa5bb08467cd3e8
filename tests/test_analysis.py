"""Autocorrelation-time estimator (Sec. 3.3 tunes d and n_M by it) against
processes whose integrated autocorrelation time is known in closed form."""
import numpy as np
import pytest

from paper_1211_1646_gb300.analysis import autocorrelation, integrated_autocorrelation_time


def ar1(a, n, seed, complex_=False):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal(n) + (1j * rng.standard_normal(n) if complex_ else 0)
    x = np.empty(n, dtype=e.dtype)
    x[0] = e[0] / np.sqrt(1 - a * a)
    for t in range(1, n):
        x[t] = a * x[t - 1] + e[t]
    return x


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9, 0.97])
def test_ar1_closed_form(a):
    n = 1 << 18
    tau = integrated_autocorrelation_time(ar1(a, n, 1))
    exact = (1 + a) / (1 - a)
    # three times the estimator's statistical error, window W = 5 tau
    assert abs(tau - exact) < 3 * exact * np.sqrt(2 * (2 * 5 * exact + 1) / n) + 0.02


def test_complex_series_and_autocorrelation_shape():
    x = ar1(0.8, 1 << 17, 2, complex_=True)
    rho = autocorrelation(x)
    assert rho[0] == 1.0
    assert abs(rho[1] - 0.8) < 0.02 and abs(rho[3] - 0.8 ** 3) < 0.02
    assert abs(integrated_autocorrelation_time(x) - 9.0) < 0.5


def test_short_or_constant_series_is_refused():
    with pytest.raises(ValueError):
        integrated_autocorrelation_time(ar1(0.999, 200, 3))
    with pytest.raises(ValueError):
        autocorrelation(np.ones(10))


class _FakeSystem:
    """A stand-in with an AR(1) observable whose coefficient depends on the
    move size: larger moves decorrelate faster (and cost the same time)."""

    def __init__(self, d, nselect):
        self.a = {0.05: 0.95, 0.25: 0.6}[d]
        self.rng = np.random.default_rng(int(d * 100) + nselect)
        self.x = 0.0
        self.closed = False

    def sweep(self, n):
        for _ in range(n):
            self.x = self.a * self.x + self.rng.standard_normal()

    def close(self):
        self.closed = True


def test_tune_sampling_ranks_by_autocorrelation_time_with_any_observable():
    from paper_1211_1646_gb300.analysis import tune_sampling
    made = []

    def make(d, nm):
        s = _FakeSystem(d, nm)
        made.append(s)
        return s

    res = tune_sampling(make, [(0.05, 4), (0.25, 4)], sweeps=40000, every=1, equilibrate=100,
                        observable=lambda s: s.x, sync=lambda: None)
    assert [r["d"] for r in res] == [0.25, 0.05]
    taus = {r["d"]: r["tau_sweeps"] for r in res}
    assert abs(taus[0.25] - 4.0) < 0.6 and abs(taus[0.05] - 39.0) < 8.0   # (1 + a)/(1 - a)
    assert all(s.closed for s in made)
    assert all(r["seconds_per_sweep"] > 0 and r["tau_seconds"] == r["tau_sweeps"] * r["seconds_per_sweep"]
               for r in res)
