import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: larger CPU cases")


def pytest_terminal_summary(terminalreporter):
    """The LM-step comparisons of the run (condition number, worst ratio to
    the per-component bound, envelope where used), one line each; also written
    as JSON lines to $AP_STEP_REPORT when that is set."""
    mod = sys.modules.get("_helpers")
    rep = getattr(mod, "STEP_REPORT", None) if mod else None
    if not rep:
        return
    terminalreporter.write_sep("-", f"LM step comparisons ({len(rep)})")
    for r in rep:
        env = "-" if r["envelope_ratio"] is None else f"{r['envelope_ratio']:.3f}"
        terminalreporter.write_line(f"{r['case']:<40s} n={r['n']:<5d} kappa={r['kappa']:.3e} "
                                    f"energy={r['energy_ratio']:.3f} strict={r['strict_ratio']:.3f} "
                                    f"past_strict={r['components_past_strict']} envelope={env}")
    path = os.environ.get("AP_STEP_REPORT")
    if path:
        import json
        with open(path, "a") as f:
            for r in rep:
                f.write(json.dumps(r) + "\n")
