"""Measured parity errors beside their bounds.

GPU parity tests call check(quantity, measured, bound) instead of a bare assert; every
check is recorded with the test that made it, and the session's terminal summary (see
conftest.py) prints, per test, the worst measured error against its bound, so the margin
of each bound is visible in a run that passes.
"""
import os

LOG = []


def _test_name() -> str:
    cur = os.environ.get("PYTEST_CURRENT_TEST", "?")
    return cur.split(" ")[0].split("::", 1)[-1]


def check(quantity: str, measured, bound, detail=None) -> None:
    measured, bound = float(measured), float(bound)
    LOG.append((_test_name(), quantity, measured, bound))
    assert measured <= bound, "%s: measured %.3e > bound %.1e%s" % (
        quantity, measured, bound, "" if detail is None else " (%s)" % (detail,))


def summary_lines():
    """One line per test: the check with the largest measured / bound."""
    worst = {}
    for test, q, m, b in LOG:
        ratio = m / b if b > 0 else (0.0 if m == 0 else float("inf"))
        if test not in worst or ratio > worst[test][0]:
            worst[test] = (ratio, q, m, b)
    lines = []
    for test, (ratio, q, m, b) in worst.items():
        lines.append("%-72s %-14s %.2e / %.0e = %5.1f%%" % (test[:72], q[:14], m, b, 100.0 * ratio))
    return lines
