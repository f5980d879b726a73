import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: oracle work of more than a few seconds")


def pytest_collection_modifyitems(config, items):
    # Run the no-allocation entry-point test file last so a first failure there
    # never hides another test's result.
    items.sort(key=lambda it: 1 if os.path.basename(str(it.fspath)).startswith("test_zz") else 0)


_ORACLE_WORKLOADS = {}


@pytest.fixture(scope="session")
def oracle_workload():
    """Oracle plan and inputs of a named workload, built once per session
    (the 256^2 radial plan takes the oracle about half a minute)."""
    def get(name):
        if name not in _ORACLE_WORKLOADS:
            import oracle
            import workloads as W
            spec, om, x, noise = W.make_workload(name)
            _ORACLE_WORKLOADS[name] = (spec, om, x, noise, oracle.make_plan(om, spec["Nd"], spec["Kd"], spec["Jd"]))
        return _ORACLE_WORKLOADS[name]
    return get
