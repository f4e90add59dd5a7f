"""The oracle's short chains equal the recorded ones digit for digit
(tests/golden/oracle_chains.txt, written by tests/golden/make_golden.py from
oracle/ only)."""
import importlib.util
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_chains_match_the_record():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    want = open(os.path.join(HERE, "golden", "oracle_chains.txt")).read()
    assert mod.render(mod.records()) == want
