import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    # temporary files of the tests stay inside the repository tree (_build/)
    os.makedirs(os.path.join(ROOT, "_build"), exist_ok=True)
