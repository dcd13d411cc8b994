import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu():
    if not has_gpu():
        pytest.skip("no CUDA device")
    import paper_1210_5128_gb300 as bn
    return bn


def _oracle_workload_table(name):
    import oracle
    import synth
    data, arity, k, R, net = synth.workload(name)
    return data, arity, k, R, oracle.build_table(data, arity, k, R=R, threads=None)


@pytest.fixture(scope="session")
def oracle_n40_m1000(gpu):
    """The 40-node shape with 1,000 samples (3 states, k = 4), every entry built by the
    oracle on all host cores."""
    return _oracle_workload_table("n40_k4_m1000")


@pytest.fixture(scope="session")
def oracle_n40(gpu):
    """The 40-node workload (3 states, m = 2000, k = 4) and its every entry built by the
    oracle on all host cores (3.69 M entries: tens of seconds of CPU time)."""
    return _oracle_workload_table("n40_k4_m2000")


@pytest.fixture(scope="session")
def oracle_n60(gpu):
    """The 60-node workload the bench runs (3 states, m = 1000, k = 4) and its every
    entry built by the oracle on all host cores (29.4 M entries: about a minute on
    16 cores)."""
    return _oracle_workload_table("n60_k4_m1000")
