"""The oracle's pins catch plausible mistakes in the oracle (CPU only).

Each mutant of tests/oracle_mutants.py plants one slip in one oracle function: a dropped
factor, a wrong sign, a shifted index, a transposed operand, an unadjusted frequency, in the
wave solve and filter sums, the operators, the residual, GMRES, the set-up and Algorithm 2,
and the warm-start network.  For every mutant the oracle's pin files run in a fresh process
with that mutant applied (conftest.py reads MFWH_ORACLE_MUTANT), and at least one pin must
fail on an assertion.  Only the pins run: the planted-mistake tests, which plant mistakes of
their own, are left out, and nothing compares the oracle with the library here.
"""

import concurrent.futures as cf
import inspect
import os
import subprocess
import sys
import textwrap

import pytest

import oracle_mutants as OM

TESTS = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(TESTS)
PINS = ["test_oracle_wave.py", "test_oracle_filters.py", "test_oracle_order4.py",
        "test_oracle_explicit_filter.py", "test_oracle_implicit.py", "test_oracle_cnn.py"]
NOT_PLANTED = "not planted and not catches and not fails_with"


def _run_pins(mutant):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               COLUMNS="250")
    env.pop("MFWH_ORACLE_MUTANT", None)
    if mutant:
        env["MFWH_ORACLE_MUTANT"] = mutant
    p = subprocess.run([sys.executable, "-m", "pytest", *[os.path.join(TESTS, f) for f in PINS],
                        "-q", "-rf", "--tb=no", "-p", "no:cacheprovider", "-k", NOT_PLANTED],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    failed = [line for line in p.stdout.splitlines() if line.startswith("FAILED")]
    return p.returncode, failed, p.stdout[-2000:] + p.stderr[-2000:]


@pytest.fixture(scope="module")
def outcomes():
    names = [None] + list(OM.MUTANTS)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(zip(names, ex.map(_run_pins, names)))


@pytest.mark.parametrize("name", sorted(OM.MUTANTS))
def test_mutant_text_occurs_once(name):
    """Each mutant edits exactly one place (a mutant whose text went missing would test
    nothing)."""
    import importlib

    mod_name, target, old, new, _ = OM.MUTANTS[name]
    owner = importlib.import_module(mod_name)
    for part in target.split("."):
        owner = getattr(owner, part)
    src = textwrap.dedent(inspect.getsource(owner))
    assert src.count(old) == 1 and old != new, name


def test_unmutated_pins_pass(outcomes):
    rc, failed, tail = outcomes[None]
    assert rc == 0 and not failed, tail


@pytest.mark.parametrize("name", sorted(OM.MUTANTS))
def test_pins_catch_mutant(outcomes, name):
    rc, failed, tail = outcomes[name]
    # exit code 1: tests ran and some failed (not a collection or internal error)
    assert rc == 1, (name, rc, tail)
    assert any(" - AssertionError" in f or " - assert" in f for f in failed), (name, failed)
