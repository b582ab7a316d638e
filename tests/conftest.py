import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def species():
    from paper_2312_04830_gb300 import workloads
    return workloads.species_table()


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def prlib():
    """The CUDA library, built in-tree if needed (nvcc cross-compiles without a GPU)."""
    from paper_2312_04830_gb300 import binding, build
    build.build()
    return binding.lib()


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for tests marked gpu")
    return torch.device("cuda:0")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """One line per kind of cell the FP64 parity rule treats apart (tests/parity.py),
    summed over the parity checks of the run, just above pytest's last line."""
    parity = sys.modules.get("tests.parity")
    if parity is None or not parity.REPORTS:
        return
    tot = {k: sum(r[k] for _, r in parity.REPORTS) for k in parity.COUNT_KEYS}
    terminalreporter.write_line(
        "FP64 parity: %d checks, %d cells: %d within 1e-10, %d ill-conditioned roots, %d ambiguous, "
        "%d within the cancellation bound" %
        (len(parity.REPORTS), tot["n_cells"], tot["n_ok"], tot["n_ill"], tot["n_ambiguous"], tot["n_cancel"]))
