import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")
    # Child processes of tests/test_oracle_mutants.py plant one mistake in the oracle.
    mutant = os.environ.get("BICADMM_ORACLE_MUTANT")
    if mutant:
        sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
        import oracle_mutants
        from oracle import bicadmm_ref
        oracle_mutants.apply(bicadmm_ref, mutant)


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
