import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


_KEYS = {}


@pytest.fixture(scope="session")
def oracle_keys():
    """Session cache of oracle key material: oracle_keys(preset_name, seed)."""
    from oracle import oracle as O
    from paper_2309_09025_gb300 import synth

    def get(name, seed, **override):
        key = (name, seed, tuple(sorted(override.items())))
        if key not in _KEYS:
            P = dict(synth.PRESETS[name])
            P.update(override)
            _KEYS[key] = (P, O.keygen(P, seed))
        return _KEYS[key]

    return get
