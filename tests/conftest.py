import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    # A planted oracle mistake (tests/oracle_mutants.py), set only by the child processes of
    # tests/test_oracle_mutants.py: the oracle's pins must then fail.
    mutant = os.environ.get("MFWH_ORACLE_MUTANT")
    if mutant:
        sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
        import oracle_mutants
        oracle_mutants.apply(mutant)


def printed_tolerance(text):
    """Half a unit in the last printed digit of a decimal string, plus 1% slack for
    values that sit on a rounding boundary (e.g. 0.683850 printed as 0.6839)."""
    s = text.strip().lstrip("-")
    if "." in s:
        decimals = len(s.split(".")[1])
    else:
        decimals = 0
    return 0.5 * 10.0 ** (-decimals) * 1.01 + 1e-15


@pytest.fixture
def printed_close():
    def check(value, text, what=""):
        tol = printed_tolerance(text)
        assert abs(value - float(text)) <= tol, f"{what}: {value!r} vs printed {text} (tol {tol:g})"
    return check
