"""Shared pytest configuration.

``-m gpu`` tests need a GB300 and the compiled library; everything else runs on
the CPU (oracle pins, host logic, library loading and exported symbols).
"""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled tfmm library")
    config.addinivalue_line("markers", "slow: oracle pins that take more than a few seconds")


@pytest.fixture(scope="session")
def sphere2_mesh():
    from paper_2103_05822_gb300.inputs import icosphere, WORKLOADS
    w = WORKLOADS["sphere2"]
    return icosphere(w.diameter, w.nu)


@pytest.fixture(scope="session")
def sphere2_oracle(sphere2_mesh):
    """Oracle problem of the 2-lambda sphere (0.5 lambda boxes, 3 digits, gamma 1e-4)."""
    import oracle
    from paper_2103_05822_gb300.inputs import WORKLOADS
    w = WORKLOADS["sphere2"]
    v, f = sphere2_mesh
    return oracle.problem.build(v, f, k=2 * math.pi, box=w.box, digits=w.digits, tol=w.tol)
