import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_sessionfinish(session, exitstatus):
    """With GS_PARITY_REPORT set, write the element-wise error percentiles the
    GPU parity tests recorded (gpu_util.REPORT) to that file as JSON."""
    path = os.environ.get("GS_PARITY_REPORT")
    mod = sys.modules.get("gpu_util")
    if not path or mod is None or not getattr(mod, "REPORT", None):
        return
    with open(path, "w") as f:
        json.dump(mod.REPORT, f, indent=1, sort_keys=True)
