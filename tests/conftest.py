import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")
    config.addinivalue_line("markers", "holstein_full_oracle: compares with the oracle's full "
                            "Holstein evolution, started in the background at session start")


_BG = {}


def _start_holstein_oracle():
    """Start the oracle's full Holstein evolution as a child process (a fresh interpreter, so
    no CUDA state is inherited); returns (process, output path)."""
    if "holstein" not in _BG:
        d = tempfile.mkdtemp(prefix="cheb_oracle_")
        out = os.path.join(d, "holstein_full.npz")
        log = open(os.path.join(d, "log.txt"), "w")
        proc = subprocess.Popen([sys.executable, os.path.join(ROOT, "tests", "holstein_oracle_run.py"),
                                 out], stdout=log, stderr=subprocess.STDOUT)
        _BG["holstein"] = (proc, out, d)
    return _BG["holstein"]


@pytest.fixture(scope="session")
def holstein_full_reference():
    """The oracle's state after the full Holstein configuration (dict of arrays); waits for the
    background run (started at collection when such a test is selected)."""
    import numpy as np

    proc, out, d = _start_holstein_oracle()
    rc = proc.wait(timeout=1800)
    if rc != 0:
        raise RuntimeError(f"oracle run failed ({rc}): " + open(os.path.join(d, "log.txt")).read())
    with np.load(out) as z:
        return {k: z[k] for k in z.files}


def pytest_sessionfinish(session, exitstatus):
    """A background oracle run still going when the session ends (its test was not reached)
    is stopped."""
    if "holstein" in _BG:
        proc = _BG["holstein"][0]
        if proc.poll() is None:
            proc.terminate()
            try:
                proc.wait(timeout=10)
            except subprocess.TimeoutExpired:
                proc.kill()


@pytest.hookimpl(trylast=True)
def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        if any("holstein_full_oracle" in item.keywords for item in items):
            _start_holstein_oracle()
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
