import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libsft.so")


@pytest.fixture(scope="session")
def paper_values():
    import json
    with open(os.path.join(ROOT, "tests", "golden", "paper_values.json")) as f:
        return json.load(f)


# Measured errors against the FP64 oracle, one record per check: printed,
# and written as a JSON list to $SFT_PRECISION_LOG at the end of the session
# when that variable is set.
_PRECISION = []


@pytest.fixture
def record_precision(request):
    def rec(config, rel_linf=None, bar=None, flux_drift=None, **extra):
        d = {"test": request.node.name, "config": config, "rel_linf": rel_linf, "bar": bar,
             "flux_drift": flux_drift}
        d.update(extra)
        _PRECISION.append(d)
        print("PRECISION " + json.dumps(d))
    return rec


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("SFT_PRECISION_LOG")
    if path and _PRECISION:
        with open(path, "w") as f:
            json.dump(_PRECISION, f, indent=1)
