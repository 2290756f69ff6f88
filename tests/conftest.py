import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


_CACHE = {}


@pytest.fixture(scope="session")
def bem_cache():
    """Dense oracle BEM matrices keyed by (surface, case id, kappa), shared across tests."""
    return _CACHE


@pytest.fixture(scope="session")
def tiny_case():
    from paper_2511_21713_gb300 import inputs
    return inputs.single_charge_sphere(nu=3, layers=5)


@pytest.fixture(scope="session")
def small_case():
    from paper_2511_21713_gb300 import inputs
    return inputs.single_charge_sphere(nu=5, layers=13)


@pytest.fixture(scope="session")
def tiny_solute_case():
    from paper_2511_21713_gb300 import inputs
    return inputs.single_charge_solute_sphere(nu=3, layers=5, core_layers=6)


@pytest.fixture(scope="session")
def small_solute_case():
    from paper_2511_21713_gb300 import inputs
    return inputs.single_charge_solute_sphere(nu=5, layers=13, core_layers=12)
