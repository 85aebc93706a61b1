import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long statistical CPU test")


# GPU modules: the hot path's core parity first, then its extensions, so that
# under -x a failure in an extension still leaves the core record complete.
_GPU_ORDER = ["test_gpu_parity", "test_gpu_h128_mixed", "test_gpu_shard", "test_gpu_pressure", "test_gpu_toy",
              "test_gpu_jastrow34", "test_gpu_serve", "test_gpu_twist", "test_gpu_empirical", "test_zz_no_alloc"]


def pytest_collection_modifyitems(config, items):
    def rank(item):
        mod = item.module.__name__.rsplit(".", 1)[-1] if item.module else ""
        return _GPU_ORDER.index(mod) if mod in _GPU_ORDER else -1
    items.sort(key=rank)   # stable: the order inside a module is kept
