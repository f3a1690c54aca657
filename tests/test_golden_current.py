"""The stored oracle results under tests/golden/ were written by the current oracle."""
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def test_stored_cycle_energies_match_current_oracle_sources():
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(HERE, "golden", "make_oracle_cycles.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    for path in (mk.OUT, mk.OUT_REFRESH):
        with open(path) as f:
            rec = json.load(f)
        assert rec["converged"]
        assert rec["oracle_sha256"] == mk.oracle_digest(), \
            "oracle or workload sources changed: run tests/golden/make_oracle_cycles.py again"
        assert set(rec["energies"]) == set(mk.KEYS)
