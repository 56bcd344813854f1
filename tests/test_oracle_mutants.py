"""The oracle's pins catch planted mistakes.

For every mutant in oracle_mutants.MUTANTS the pin suite (test_oracle_pins.py) runs in a
child process with that one mistake planted in the oracle; the child must report a failed
pin.  A mutant that every pin accepts would mean a part of the oracle that no fact from the
paper or from mathematics holds in place.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from oracle import bicadmm_ref as ref

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, HERE)
import oracle_mutants  # noqa: E402


@pytest.mark.parametrize("name", sorted(oracle_mutants.MUTANTS))
def test_mutant_snippet_applies(name):
    """Each planted change still matches the oracle's source exactly once."""
    src = oracle_mutants.mutated_source(ref, name)
    compile(src, name, "exec")


def _run_pins(name):
    env = dict(os.environ, BICADMM_ORACLE_MUTANT=name)
    res = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"),
                          "-x", "-q", "-p", "no:cacheprovider"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, res.returncode, res.stdout[-2000:] + res.stderr[-2000:]


def test_every_mutant_is_caught():
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as pool:
        results = list(pool.map(_run_pins, sorted(oracle_mutants.MUTANTS)))
    survived = [(n, out) for n, rc, out in results if rc != 1]
    # exit code 1 = some pin failed; 0 = every pin passed (mutant survived); others = errors
    assert not survived, "\n\n".join("%s (%s):\n%s" % (n, oracle_mutants.MUTANTS[n][3], out)
                                     for n, out in survived)
