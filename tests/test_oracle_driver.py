"""Pins of the oracle's Alg. 4 loop (oracle/driver.py): the epoch bookkeeping
against what the algorithm fixes, independent of the arithmetic inside the
iterations.

- A failed epoch (F-hat above the epoch-start value) restores the factors of
  the epoch start exactly: a run stopped right after the failure ends where a
  run stopped before that epoch ends.
- After a failure alpha shrinks by nu, t is wound back by tau, the failure
  count grows by one and the recorded estimate is the epoch-start one; after
  a success t has advanced by tau and alpha is unchanged.
- The run stops once more than kappa epochs have failed.
"""
import numpy as np

import oracle
from oracle.driver import gcp_adam

DIMS, RANK, TAU = (6, 5, 4), 2, 10


def problem():
    rng = np.random.default_rng(4)
    true = [rng.standard_normal((n, RANK)) for n in DIMS]
    X = np.einsum("ir,jr,kr->ijk", *true) + 0.1 * rng.standard_normal(DIMS)
    A0 = [0.5 * rng.standard_normal((n, RANK)) for n in DIMS]
    return oracle.Tensor(DIMS, dense=X), A0


def run(XO, A0, alpha, kappa=3, nu=0.5, max_epochs=30, first_iter=0):
    logs = []
    A, hist = gcp_adam(XO, A0, oracle.GAUSSIAN, oracle.UNIFORM, 0, 20, 0, 30, 5, 6, alpha=alpha, tau=TAU,
                       kappa=kappa, nu=nu, max_epochs=max_epochs, log=logs.append, first_iter=first_iter)
    return A, hist, logs


def test_epoch_bookkeeping():
    XO, A0 = problem()
    alpha0, nu, kappa = 0.3, 0.5, 3
    _, hist, logs = run(XO, A0, alpha0, kappa, nu)
    F_prev, alpha, t, bad = hist[0], alpha0, 0, 0
    failures = 0
    for e, rec in enumerate(logs, start=1):
        assert rec["epoch"] == e
        if rec["bad"] > bad:  # a failed epoch
            failures += 1
            assert rec["bad"] == bad + 1
            assert rec["alpha"] == alpha * nu
            assert rec["t"] == t  # wound back by tau
            assert rec["F"] == F_prev  # the epoch-start estimate is kept
            assert hist[e] == F_prev
        else:
            assert rec["F"] <= F_prev
            assert rec["alpha"] == alpha
            assert rec["t"] == t + TAU
        F_prev, alpha, t, bad = rec["F"], rec["alpha"], rec["t"], rec["bad"]
    assert failures >= 2  # the scenario exercises both branches
    # stop rule: more than kappa failures end the run, and nothing else does before max_epochs
    assert bad == kappa + 1 or len(logs) == 30
    assert all(r["bad"] <= kappa for r in logs[:-1])


def test_failed_epoch_restores_the_epoch_start():
    XO, A0 = problem()
    _, _, logs = run(XO, A0, 0.3)
    first_fail = next(r["epoch"] for r in logs if r["bad"] == 1)
    assert first_fail >= 2  # at least one accepted epoch before it
    before, _, _ = run(XO, A0, 0.3, max_epochs=first_fail - 1)
    after, _, logs_after = run(XO, A0, 0.3, max_epochs=first_fail)
    assert logs_after[-1]["bad"] == 1
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)


def test_every_epoch_failing_returns_the_initial_factors():
    """A learning rate so large that every step overshoots: kappa + 1 failed
    epochs, alpha shrunk kappa + 1 times, t back at 0, the initial factors."""
    XO, A0 = problem()
    A, hist, logs = run(XO, A0, 1e3, kappa=2, nu=0.1)
    assert [r["bad"] for r in logs] == [1, 2, 3]
    assert [r["t"] for r in logs] == [0, 0, 0]
    np.testing.assert_allclose([r["alpha"] for r in logs], [1e2, 1e1, 1e0], rtol=1e-12)
    assert all(F == hist[0] for F in hist)
    for a, a0 in zip(A, A0):
        np.testing.assert_array_equal(a, a0)


def test_retried_epoch_draws_new_samples():
    """With nu = 1 a retried epoch starts from exactly the state of the failed
    one (factors, moments, t, alpha); only the draws can differ.  The stream
    word counts every iteration ever run, so a retry eventually succeeds where
    a wound-back stream would repeat the same failure forever."""
    XO, A0 = problem()
    _, _, logs = run(XO, A0, 0.3, kappa=5, nu=1.0, max_epochs=12)
    failed = next(r for r in logs if r["bad"] == 1)  # holds the epoch-start t and F
    retries = logs[failed["epoch"]:]
    accepted = next((r for r in retries if r["t"] > failed["t"]), None)
    assert accepted is not None, "no retry of the failed epoch was accepted"
    assert accepted["t"] == failed["t"] + TAU and accepted["F"] < failed["F"]
    assert all(r["t"] == failed["t"] for r in retries[:retries.index(accepted)])  # the retries in between failed


def test_failed_epochs_leave_no_trace_but_alpha_and_the_stream():
    """Failed epochs from the very start: once one succeeds, the run must be
    exactly a fresh run from the initial factors (moments zero, t = 0) at the
    reduced alpha whose draws start where the failed epochs' draws ended.  A
    moment, step count or factor left over from a failed epoch changes it."""
    XO, A0 = problem()
    _, _, logs = run(XO, A0, 1e3, kappa=10, nu=0.1)
    accepted = next(r for r in logs if r["t"] > 0)
    fails = accepted["epoch"] - 1
    assert fails >= 2 and accepted["bad"] == fails
    A_run, _, _ = run(XO, A0, 1e3, kappa=10, nu=0.1, max_epochs=accepted["epoch"])
    A_fresh, _, logs_fresh = run(XO, A0, accepted["alpha"], kappa=10, nu=0.1, max_epochs=1, first_iter=fails * TAU)
    assert logs_fresh[0]["bad"] == 0 and logs_fresh[0]["F"] == accepted["F"]
    for a, b in zip(A_run, A_fresh):
        np.testing.assert_array_equal(a, b)


def test_an_equal_estimate_is_accepted():
    """alpha = 0 leaves every factor where it is, so each epoch's estimate
    equals the previous one: equal is no increase, every epoch is accepted."""
    XO, A0 = problem()
    A, hist, logs = run(XO, A0, 0.0, kappa=0, max_epochs=3)
    assert [r["bad"] for r in logs] == [0, 0, 0]
    assert [r["t"] for r in logs] == [TAU, 2 * TAU, 3 * TAU]
    assert len(set(hist)) == 1
    for a, a0 in zip(A, A0):
        np.testing.assert_array_equal(a, a0)
