import os
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the autotuner's cache of this test session: a fresh file, not the user's,
# removed when the session ends
if "RSA_TUNE_CACHE" not in os.environ:
    import atexit
    import shutil
    _tune_dir = tempfile.mkdtemp(prefix="rsa_tune_")
    atexit.register(shutil.rmtree, _tune_dir, True)
    os.environ["RSA_TUNE_CACHE"] = os.path.join(_tune_dir, "tune.jsonl")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU statistics")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
